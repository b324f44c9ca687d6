"""Pins of the oracle's block-Jacobi pieces (flux Jacobian, per-node blocks,
block inversion, preconditioned stage) against facts that do not come from
those functions: finite differences of the oracle's Euler flux, Euler's
theorem for a flux homogeneous of degree one, the closed form of the blocks
on cells whose normals cancel, M P = I, and the reduction of the
preconditioned stage to local time stepping.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

G14 = 1.4


def cons(rho, u, p, c=0.0, gamma=G14):
    u = np.asarray(u, dtype=np.float64)
    return np.array([rho, rho * u[0], rho * u[1], rho * u[2],
                     p / (gamma - 1) + 0.5 * rho * u @ u, c])


def random_states(rng, k):
    out = []
    for _ in range(k):
        out.append(cons(rng.uniform(0.5, 2.0), rng.uniform(-1.0, 1.0, 3),
                        rng.uniform(0.5, 2.0), rng.uniform(0.0, 1.0)))
    return out


def test_flux_jacobian_matches_finite_differences():
    rng = np.random.default_rng(0)
    for q in random_states(rng, 20):
        n = rng.normal(size=3)
        A = oracle.flux_jacobian(q, n)
        Afd = np.empty((6, 6))
        for c in range(6):
            h = 1e-6 * max(1.0, abs(q[c]))
            e = np.zeros(6)
            e[c] = h
            Afd[:, c] = (oracle.euler_flux(q + e, n) - oracle.euler_flux(q - e, n)) / (2 * h)
        assert np.max(np.abs(A - Afd)) <= 1e-7 * np.max(np.abs(A))


def test_flux_jacobian_euler_theorem():
    # f(lambda q) = lambda f(q) for the ideal-gas flux (the passive scalar
    # too), so A(q) q = f(q).n
    rng = np.random.default_rng(1)
    for q in random_states(rng, 20):
        n = rng.normal(size=3)
        f = oracle.euler_flux(q, n)
        assert np.max(np.abs(oracle.flux_jacobian(q, n) @ q - f)) <= 1e-14 * np.max(np.abs(f)) * 10


def test_flux_jacobian_of_a_state_at_rest_along_x():
    # u = 0, n = e_x: only mass and the x-momentum row survive:
    # d(rho u_x)/dm_x = 1, d p/d rho = 0 (k = 0), d p/d E = gamma - 1
    q = cons(1.3, [0.0, 0.0, 0.0], 0.9, 0.2)
    A = oracle.flux_jacobian(q, [1.0, 0.0, 0.0])
    ref = np.zeros((6, 6))
    ref[0, 1] = 1.0
    ref[1, 4] = G14 - 1.0
    H = (q[4] + 0.9) / 1.3
    ref[4, 1] = H
    ref[5, 1] = 0.2 / 1.3
    assert np.allclose(A, ref, rtol=0, atol=1e-15)


def frozen_residual(m, q, i, s):
    """R_i of the first-order Rusanov residual with the wave speeds s (per
    edge) held fixed, from the oracle's Euler flux."""
    R = np.zeros(6)
    for e in np.nonzero((m.edge[:, 0] == i) | (m.edge[:, 1] == i))[0]:
        a, b = m.edge[e]
        n = m.normal[e]
        F = 0.5 * (oracle.euler_flux(q[a], n) + oracle.euler_flux(q[b], n)) - 0.5 * s[e] * (q[b] - q[a])
        if a == i:
            R += F
        if b == i:
            R -= F
    return R


def test_jacobi_blocks_are_the_frozen_speed_jacobian_diagonal():
    m = meshgen.lattice(4)
    q = meshgen.flow_state(m)
    s = np.array([max(oracle.wave_speed(q[a], m.normal[e]), oracle.wave_speed(q[b], m.normal[e]))
                  for e, (a, b) in enumerate(m.edge)])
    M = oracle.jacobi_blocks(m.edge, q, m.normal)
    for i in (0, 17, 63):
        Mfd = np.empty((6, 6))
        for c in range(6):
            h = 1e-6 * max(1.0, abs(q[i, c]))
            qp, qm = q.copy(), q.copy()
            qp[i, c] += h
            qm[i, c] -= h
            Mfd[:, c] = (frozen_residual(m, qp, i, s) - frozen_residual(m, qm, i, s)) / (2 * h)
        assert np.max(np.abs(M[i] - Mfd)) <= 1e-7 * np.max(np.abs(M[i]))


def test_jacobi_blocks_of_closed_cells_are_half_the_spectral_radius():
    # unperturbed lattice: every node's signed normals cancel exactly, so the
    # flux Jacobians cancel and M_i = Lambda_i / 2 I
    m = meshgen.lattice(5, perturbed=False)
    q = meshgen.flow_state(m)
    M = oracle.jacobi_blocks(m.edge, q, m.normal)
    lam = oracle.spectral_radius(m.edge, q, m.normal)
    ref = 0.5 * lam[:, None, None] * np.eye(6)[None]
    assert np.max(np.abs(M - ref) / lam[:, None, None]) <= 1e-13
    # on the perturbed lattice the blocks are not diagonal
    mp = meshgen.lattice(5)
    Mp = oracle.jacobi_blocks(mp.edge, q, mp.normal)
    off = Mp - Mp * np.eye(6)[None]
    assert np.max(np.abs(off)) > 1e-3


def test_block_invert_inverts_and_pivots():
    rng = np.random.default_rng(2)
    M = rng.normal(size=(50, 6, 6))
    M[:10] += 6 * np.eye(6)  # diagonally dominant
    M[10] = np.eye(6)[[1, 0, 3, 2, 5, 4]] * 3.0  # zero diagonal: needs pivoting
    P, bad = oracle.block_invert(M)
    assert bad == 0
    for i in range(50):
        assert np.max(np.abs(M[i] @ P[i] - np.eye(6))) <= 1e-11 * np.linalg.cond(M[i])
    Ms = M[:3].copy()
    Ms[1] = 0.0
    _, bad = oracle.block_invert(Ms)
    assert bad == 1


def test_precond_update_is_local_time_stepping_on_closed_cells():
    # M = Lambda/2 I, so sigma = CFL/2 gives q0 - alpha CFL R / Lambda,
    # the local-time-step stage with dt = CFL V / Lambda
    m = meshgen.lattice(5, perturbed=False)
    q = meshgen.flow_state(m)
    R, _ = oracle.residual(1, m.edge, q, m.normal, m.dx, m.volume)
    M = oracle.jacobi_blocks(m.edge, q, m.normal)
    P, bad = oracle.block_invert(M)
    assert bad == 0
    lam = oracle.spectral_radius(m.edge, q, m.normal)
    dt = oracle.time_step(m.volume, lam, 0.5)
    a = 0.375
    qp = oracle.precond_update(q, R, P, a * 0.25)
    qr = oracle.rk_update(q, R, m.volume, dt, a)
    assert np.max(np.abs(qp - qr) / np.max(np.abs(q), axis=0)) <= 1e-14


@pytest.mark.parametrize("alpha_sigma", [0.0, 0.7])
def test_precond_update_definition(alpha_sigma):
    rng = np.random.default_rng(3)
    q0, R = rng.normal(size=(7, 6)), rng.normal(size=(7, 6))
    P = rng.normal(size=(7, 6, 6))
    q = oracle.precond_update(q0, R, P, alpha_sigma)
    assert np.allclose(q, q0 - alpha_sigma * np.einsum("irc,ic->ir", P, R), rtol=0, atol=1e-14)
