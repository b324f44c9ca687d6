"""Pins of the oracle's viscous edge flux against closed forms and invariants.

The paper names the viscous edge loop (Table "loopperfmpi") without giving
its formula; the oracle states a textbook Navier-Stokes reading (face
gradient = average of the two nodal gradients with the edge-direction
correction, Newtonian stress with Stokes' hypothesis, Fourier heat flux,
Fickian diffusion of the passive scalar).  These tests pin that reading
against facts derived independently of oracle.c: exact results for linear
primitive fields (written in primitive variables, so the conversion of the
conserved gradients is checked too), the two-point thin-layer form, rotation
and orientation invariance, and conservation over a mesh.  CPU only.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

G14 = 1.4
MU, PR, DIFF = 2.3e-3, 0.72, 1.7e-3
KAPPA = MU * G14 / ((G14 - 1.0) * PR)


def linear_node(x, rho0, r, u0, A, T0, t, c0, b, gamma=G14):
    """Conserved state and exact conserved gradients (18, component 3k+d) at
    the point x of the linear primitive fields rho = rho0 + r.x,
    u = u0 + A x, T = p/rho = T0 + t.x, q5 = c0 + b.x (product rule)."""
    x = np.asarray(x, float)
    rho, u, T, c = rho0 + r @ x, u0 + A @ x, T0 + t @ x, c0 + b @ x
    q = np.concatenate([[rho], rho * u, [rho * (T / (gamma - 1) + 0.5 * u @ u)], [c]])
    G = np.zeros((6, 3))
    G[0] = r
    for a in range(3):
        G[1 + a] = u[a] * r + rho * A[a]          # grad(rho u_a)
    e = T / (gamma - 1) + 0.5 * u @ u           # energy per unit mass
    G[4] = e * r + rho * (t / (gamma - 1) + A.T @ u)
    G[5] = b
    return q, G.reshape(18)


def linear_case(rng):
    return dict(rho0=rng.uniform(0.8, 1.5), r=rng.uniform(-0.1, 0.1, 3),
                u0=rng.uniform(-0.5, 0.5, 3), A=rng.uniform(-0.3, 0.3, (3, 3)),
                T0=rng.uniform(0.8, 1.2), t=rng.uniform(-0.1, 0.1, 3),
                c0=rng.uniform(0, 1), b=rng.uniform(-0.2, 0.2, 3))


def closed_form(A, t, b, u_mid, n):
    """Viscous flux of linear primitive fields: stress of the constant
    velocity gradient A, the velocity at the face midpoint, grad T = t."""
    tau = MU * (A + A.T - 2.0 / 3.0 * np.trace(A) * np.eye(3))
    tn = tau @ n
    return np.concatenate([[0.0], tn, [tn @ u_mid + KAPPA * t @ n], [DIFF * b @ n]])


def vf(qi, qj, Gi, Gj, n, dx, mu=MU, diff=DIFF):
    return oracle.viscous_flux(qi, qj, Gi, Gj, n, dx, G14, mu, PR, diff)


def test_uniform_flow_has_no_viscous_flux():
    rng = np.random.default_rng(3)
    for _ in range(10):
        q = np.array([1.2, 0.3, -0.2, 0.1, 2.9, 0.4])
        F = vf(q, q, np.zeros(18), np.zeros(18), rng.normal(size=3), rng.normal(size=3))
        assert np.all(F == 0.0)


@pytest.mark.parametrize("seed", range(8))
def test_linear_fields_give_the_closed_form(seed):
    # nodal gradients of linear fields are exact and the jumps consistent, so
    # the face gradient is the field's gradient and the flux has a closed form
    rng = np.random.default_rng(seed)
    k = linear_case(rng)
    xi, xj = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
    qi, Gi = linear_node(xi, **k)
    qj, Gj = linear_node(xj, **k)
    n = rng.normal(size=3)
    F = vf(qi, qj, Gi, Gj, n, xj - xi)
    u_mid = k["u0"] + k["A"] @ (0.5 * (xi + xj))
    ref = closed_form(k["A"], k["t"], k["b"], u_mid, n)
    np.testing.assert_allclose(F, ref, rtol=1e-12, atol=1e-15)


def test_couette_shear_and_dilatation():
    # plane Couette u = (a y, 0, 0): tau_xy = mu a, no normal stress
    a = 0.25
    k = dict(rho0=1.0, r=np.zeros(3), u0=np.zeros(3), A=np.zeros((3, 3)), T0=1.0,
             t=np.zeros(3), c0=0.0, b=np.zeros(3))
    k["A"][0, 1] = a
    qi, Gi = linear_node([0, 0, 0], **k)
    qj, Gj = linear_node([0, 1, 0], **k)
    F = vf(qi, qj, Gi, Gj, [0, 1, 0], [0, 1, 0])
    np.testing.assert_allclose(F, [0, MU * a, 0, 0, MU * a * a / 2, 0], rtol=1e-14, atol=1e-18)
    # pure dilatation u = (a x, 0, 0): normal stresses 4/3 and -2/3 mu a
    k["A"] = np.zeros((3, 3))
    k["A"][0, 0] = a
    qi, Gi = linear_node([0, 0, 0], **k)
    qj, Gj = linear_node([1, 0, 0], **k)
    n = np.array([0.3, 0.5, -0.7])
    F = vf(qi, qj, Gi, Gj, n, [1, 0, 0])
    np.testing.assert_allclose(F[1:4], MU * a * np.array([4 / 3, -2 / 3, -2 / 3]) * n,
                               rtol=1e-14)


def test_heat_conduction_with_varying_density():
    # fluid at rest, rho and T linear: only the Fourier term kappa grad T . n
    rng = np.random.default_rng(11)
    k = linear_case(rng)
    k["u0"], k["A"] = np.zeros(3), np.zeros((3, 3))
    k["b"] = np.zeros(3)
    qi, Gi = linear_node([0.1, 0.2, -0.3], **k)
    qj, Gj = linear_node([0.4, -0.1, 0.2], **k)
    n = np.array([0.2, -0.9, 0.4])
    F = vf(qi, qj, Gi, Gj, n, np.array([0.3, -0.3, 0.5]))
    assert np.all(F[:4] == 0.0) and F[5] == 0.0
    assert F[4] == pytest.approx(KAPPA * k["t"] @ n, rel=1e-12)


def test_two_point_thin_layer_form():
    # zero nodal gradients: the face gradient is the jump along the edge,
    # g = (phi_j - phi_i) dx / |dx|^2 (the thin-layer two-point form)
    rho, p, a, h = 1.1, 0.8, 0.3, 0.5
    qi = np.array([rho, 0, 0, 0, p / (G14 - 1), 0.2])
    qj = np.array([rho, rho * a, 0, 0, p / (G14 - 1) + 0.5 * rho * a * a, 0.5])
    F = vf(qi, qj, np.zeros(18), np.zeros(18), [0, 2.0, 0], [0, h, 0])
    assert F[0] == 0.0 and F[2] == 0.0 and F[3] == 0.0
    assert F[1] == pytest.approx(MU * a / h * 2.0, rel=1e-14)
    assert F[4] == pytest.approx(MU * a / h * 2.0 * a / 2, rel=1e-14)
    assert F[5] == pytest.approx(DIFF * 0.3 / h * 2.0, rel=1e-14)


def test_correction_keeps_the_tangential_gradient():
    # scalar with nodal gradient perpendicular to dx and no jump: the face
    # gradient is the nodal gradient itself
    q = np.array([1.0, 0, 0, 0, 2.0, 0.3])
    G = np.zeros(18)
    G[15:18] = [0.0, 0.7, 0.0]
    F = vf(q, q, G, G, [0.2, 1.0, 0.0], [1.0, 0.0, 0.0])
    assert F[5] == pytest.approx(DIFF * 0.7, rel=1e-15)
    # gradient along dx is replaced by the jump (here none): no flux along x
    G[15:18] = [0.7, 0.0, 0.0]
    F = vf(q, q, G, G, [1.0, 0.0, 0.0], [1.0, 0.0, 0.0])
    assert F[5] == 0.0


def _random_pair(rng):
    q = np.array([rng.uniform(0.8, 1.3), *rng.uniform(-0.4, 0.4, 3), 0, rng.uniform(0, 1)])
    q[4] = rng.uniform(1.8, 2.6) + 0.5 * q[1:4] @ q[1:4] / q[0]
    return q, rng.normal(scale=0.3, size=18)


@pytest.mark.parametrize("seed", range(5))
def test_rotation_invariance(seed):
    # rotating the frame rotates the momentum flux and leaves the rest:
    # momentum m -> Q m, gradients of scalars g -> Q g, momentum gradient
    # rows -> Q M Q^T, n and dx -> Q n, Q dx
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    (qi, Gi), (qj, Gj) = _random_pair(rng), _random_pair(rng)
    n, dx = rng.normal(size=3), rng.normal(size=3)

    def rot(q, G):
        G = G.reshape(6, 3)
        qr, Gr = q.copy(), np.empty((6, 3))
        qr[1:4] = Q @ q[1:4]
        Gr[0], Gr[4], Gr[5] = Q @ G[0], Q @ G[4], Q @ G[5]
        Gr[1:4] = Q @ G[1:4] @ Q.T
        return qr, Gr.reshape(18)

    F = vf(qi, qj, Gi, Gj, n, dx)
    (qri, Gri), (qrj, Grj) = rot(qi, Gi), rot(qj, Gj)
    Fr = vf(qri, qrj, Gri, Grj, Q @ n, Q @ dx)
    np.testing.assert_allclose(Fr[[0, 4, 5]], F[[0, 4, 5]], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Fr[1:4], Q @ F[1:4], rtol=1e-12, atol=1e-15)


def test_orientation_and_linearity_in_the_coefficients():
    rng = np.random.default_rng(7)
    (qi, Gi), (qj, Gj) = _random_pair(rng), _random_pair(rng)
    n, dx = rng.normal(size=3), rng.normal(size=3)
    F = vf(qi, qj, Gi, Gj, n, dx)
    # reversing the edge (i <-> j, n -> -n, dx -> -dx) reverses the flux
    np.testing.assert_allclose(vf(qj, qi, Gj, Gi, -n, -dx), -F, rtol=1e-13, atol=1e-17)
    # doubling mu (Pr fixed) doubles the momentum and energy terms; D the scalar
    F2 = vf(qi, qj, Gi, Gj, n, dx, mu=2 * MU, diff=2 * DIFF)
    np.testing.assert_allclose(F2, 2 * F, rtol=1e-14, atol=1e-18)


def test_loop_conserves_and_vanishes_for_uniform_state():
    m = meshgen.lattice(6)
    q = meshgen.flow_state(m)
    rng = np.random.default_rng(0)
    G = rng.normal(scale=0.2, size=(m.num_nodes, 18))
    edge, n, dx = m.edge, m.normal, m.dx
    R, Ra = oracle.viscous(edge, q, G, n, dx, G14, MU, PR, DIFF, with_abs=True)
    # every edge adds +Fv and -Fv: the node sum is zero up to rounding
    assert np.all(np.abs(R.sum(axis=0)) <= 1e-13 * Ra.sum(axis=0) + 1e-300)
    assert np.all(R[:, 0] == 0.0)
    # a single edge: -Fv at i, +Fv at j
    one = oracle.viscous(edge[:1], q, G, n[:1], dx[:1], G14, MU, PR, DIFF)
    i, j = edge[0]
    F = vf(q[i], q[j], G[i], G[j], n[0], dx[0])
    np.testing.assert_array_equal(one[i], -F)
    np.testing.assert_array_equal(one[j], F)
    # a uniform state with zero gradients gives zero residual
    qu = np.tile(q[0], (m.num_nodes, 1))
    assert np.all(oracle.viscous(edge, qu, np.zeros_like(G), n, dx, G14, MU, PR, DIFF) == 0.0)
