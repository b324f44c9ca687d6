"""Pins of the CPU oracle against facts that do not come from the oracle.

Closed forms, invariants and special cases, chosen so that a dropped term, a
wrong sign or index or a transposed operand in oracle.c fails at least one.
CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

EPS = np.finfo(np.float64).eps
G14 = 1.4


def cons(rho, u, p, c=0.0, gamma=G14):
    u = np.asarray(u, dtype=np.float64)
    return np.array([rho, rho * u[0], rho * u[1], rho * u[2],
                     p / (gamma - 1) + 0.5 * rho * u @ u, c])


# ------------------------------------------------------------ Euler flux
def test_euler_flux_one_dimensional_closed_form():
    # rho = 2, u = (3, 0, 0), p = 5, c = 0.1 through n = e_x:
    # (rho u, rho u^2 + p, 0, 0, (rho E + p) u, c u) with rho E = 12.5 + 9
    q = cons(2.0, [3.0, 0.0, 0.0], 5.0, 0.1)
    f = oracle.euler_flux(q, [1.0, 0.0, 0.0])
    assert f[0] == 6.0 and f[1] == 23.0 and f[2] == 0.0 and f[3] == 0.0
    assert f[4] == pytest.approx(79.5, rel=1e-15)
    assert f[5] == pytest.approx(0.3, rel=1e-15)


def test_euler_flux_at_rest_is_pressure_only():
    q = cons(1.3, [0.0, 0.0, 0.0], 0.7, 0.2)
    n = np.array([0.3, -0.4, 1.2])
    f = oracle.euler_flux(q, n)
    assert f[0] == 0.0 and f[4] == 0.0 and f[5] == 0.0
    np.testing.assert_allclose(f[1:4], 0.7 * n, rtol=1e-15)


def test_euler_flux_tangential_velocity_carries_momentum_only():
    # u perpendicular to n: no mass, energy or scalar flux, momentum = p n
    q = cons(1.1, [0.0, 0.4, -0.2], 0.9, 0.3)
    n = np.array([0.7, 0.0, 0.0])
    f = oracle.euler_flux(q, n)
    assert f[0] == 0.0 and f[4] == 0.0 and f[5] == 0.0
    np.testing.assert_allclose(f[1:4], [0.9 * 0.7, 0.0, 0.0], rtol=1e-15)


def test_euler_flux_rotation_invariance():
    # an axis permutation with signs is an exact rotation: f(Rq).(Rn) = R f
    rng = np.random.default_rng(1)
    perm, sign = [2, 0, 1], np.array([1.0, -1.0, 1.0])
    for _ in range(20):
        q = cons(rng.uniform(0.5, 2), rng.uniform(-1, 1, 3), rng.uniform(0.5, 2),
                 rng.uniform(0, 1))
        n = rng.uniform(-1, 1, 3)
        qr = q.copy()
        qr[1:4] = sign * q[1:4][perm]
        f = oracle.euler_flux(q, n)
        fr = oracle.euler_flux(qr, sign * n[perm])
        np.testing.assert_allclose(fr[1:4], sign * f[1:4][perm], rtol=1e-14,
                                   atol=1e-14)
        np.testing.assert_allclose(fr[[0, 4, 5]], f[[0, 4, 5]], rtol=1e-14,
                                   atol=1e-15)


def test_wave_speed_closed_form():
    # rho = gamma, p = 1 gives sound speed exactly 1
    q = cons(G14, [0.5, -0.25, 0.0], 1.0)
    n = np.array([0.0, 2.0, 0.0])
    assert oracle.wave_speed(q, n) == pytest.approx(0.5 + 2.0, rel=1e-15)
    n = np.array([3.0, 4.0, 0.0])  # |n| = 5, u.n = 1.5 - 1.0
    assert oracle.wave_speed(q, n) == pytest.approx(0.5 + 5.0, rel=1e-15)


# --------------------------------------------------------------- Rusanov
def _random_pair(rng):
    qL = cons(rng.uniform(0.8, 1.2), rng.uniform(-0.5, 0.8, 3),
              rng.uniform(0.8, 1.2), rng.uniform(0, 1e-3))
    qR = cons(rng.uniform(0.8, 1.2), rng.uniform(-0.5, 0.8, 3),
              rng.uniform(0.8, 1.2), rng.uniform(0, 1e-3))
    return qL, qR, rng.uniform(-1, 1, 3)


def test_rusanov_consistency_bitwise():
    rng = np.random.default_rng(2)
    for _ in range(50):
        q, _, n = _random_pair(rng)
        assert np.array_equal(oracle.rusanov(q, q, n), oracle.euler_flux(q, n))


def test_rusanov_antisymmetry_and_homogeneity_bitwise():
    rng = np.random.default_rng(3)
    for _ in range(50):
        qL, qR, n = _random_pair(rng)
        F = oracle.rusanov(qL, qR, n)
        assert np.array_equal(oracle.rusanov(qR, qL, -n), -F)
        assert np.array_equal(oracle.rusanov(qL, qR, 2.0 * n), 2.0 * F)


def test_rusanov_dissipation_closed_form():
    # both sound speeds are 1 (rho = gamma, p = 1); |n| = 1 so
    # s = max(|uL.n|, |uR.n|) + 1 and F - (fL + fR)/2 = -s (qR - qL)/2
    n = np.array([0.6, 0.8, 0.0])
    qL = cons(G14, [1.0, 0.5, 0.0], 1.0)        # uL.n = 1.0
    qR = cons(G14, [-0.5, -1.0, 0.3], 1.0)      # uR.n = -1.1
    s = 1.1 + 1.0
    F = oracle.rusanov(qL, qR, n)
    fbar = 0.5 * (oracle.euler_flux(qL, n) + oracle.euler_flux(qR, n))
    np.testing.assert_allclose(F - fbar, -0.5 * s * (qR - qL), rtol=1e-13,
                               atol=1e-14)


def test_rusanov_supersonic_side_dominates_speed():
    # a fast left state: s is taken from the left state
    n = np.array([1.0, 0.0, 0.0])
    qL = cons(G14, [3.0, 0.0, 0.0], 1.0)   # s_L = 3 + 1
    qR = cons(G14, [0.0, 0.0, 0.0], 1.0)   # s_R = 1
    F = oracle.rusanov(qL, qR, n)
    fbar = 0.5 * (oracle.euler_flux(qL, n) + oracle.euler_flux(qR, n))
    np.testing.assert_allclose(F - fbar, -2.0 * (qR - qL), rtol=1e-14)


# ------------------------------------------------------------ van Albada
def test_van_albada_properties():
    rng = np.random.default_rng(4)
    for _ in range(200):
        a, b = rng.uniform(-2, 2, 2)
        phi = oracle.van_albada(a, b)
        assert oracle.van_albada(a, a) == pytest.approx(a, rel=1e-15, abs=0)
        assert oracle.van_albada(a, -a) == 0.0
        assert oracle.van_albada(b, a) == phi
        assert oracle.van_albada(-a, -b) == -phi
        if a * b > 0:      # between the two slopes
            assert min(a, b) - 1e-15 <= phi <= max(a, b) + 1e-15
        if a * b < -1e-6:  # opposite slopes: clipped towards zero
            assert abs(phi) < 0.5 * max(abs(a), abs(b))
    # one-sided zero slope kills the correction (to within eps/|a|)
    assert abs(oracle.van_albada(0.3, 0.0)) < 1e-11
    assert oracle.van_albada(0.0, 0.0) == 0.0


def test_reconstruction_linear_exactness_and_first_order_limit():
    rng = np.random.default_rng(5)
    qi = cons(1.0, [0.5, 0.1, 0.0], 1.0, 1e-4)
    qj = cons(1.1, [0.4, 0.2, -0.1], 0.9, 3e-4)
    dx = np.array([0.9, 0.2, -0.1])
    # gradients that reproduce the jump exactly: G.dx = qj - qi at both ends
    Gi = np.zeros((6, 3))
    Gi[:, 0] = (qj - qi) / dx[0]
    qL, qR = oracle.reconstruct(qi, qj, Gi.ravel(), Gi.ravel(), dx)
    mid = 0.5 * (qi + qj)
    np.testing.assert_allclose(qL, mid, rtol=1e-14, atol=1e-17)
    np.testing.assert_allclose(qR, mid, rtol=1e-14, atol=1e-17)
    # zero gradients: |phi(0, b)| = |b| eps / (b^2 + 2 eps) <= eps / |b|,
    # so the scheme falls back to first order up to that correction
    qL, qR = oracle.reconstruct(qi, qj, np.zeros(18), np.zeros(18), dx)
    bound = 0.5 * 1e-12 / np.abs(qj - qi) + 4 * EPS * np.maximum(
        np.abs(qi), np.abs(qj))
    assert np.all(np.abs(qL - qi) <= bound)
    assert np.all(np.abs(qR - qj) <= bound)
    # the left state uses G_i only, the right state G_j only
    Gj = rng.uniform(-1, 1, 18)
    qL2, _ = oracle.reconstruct(qi, qj, np.zeros(18), Gj, dx)
    np.testing.assert_array_equal(qL2, qL)


# --------------------------------------------------------- 8-node cube
def _read_hand_cube():
    path = os.path.join(os.path.dirname(__file__), "golden", "hand_cube.txt")
    R, G = np.zeros((8, 6)), np.zeros((8, 18))
    with open(path) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            tag, i, *vals = line.split()
            (R if tag == "R" else G)[int(i)] = [float(v) for v in vals]
    return R, G


def test_hand_cube_first_order_residual_and_gradient():
    _, edge, nrm, dx = meshgen.hand_cube_mesh()
    p = 1.0 + np.arange(8) / 8.0
    q = np.stack([cons(1.0, [0, 0, 0], pi) for pi in p])
    Rexp, Gexp = _read_hand_cube()
    R = oracle.flux1(edge, q, nrm)
    np.testing.assert_allclose(R, Rexp, rtol=1e-14, atol=1e-14)
    G = oracle.green_gauss(edge, q, nrm)
    np.testing.assert_allclose(G, Gexp, rtol=1e-14, atol=1e-14)


# ------------------------------------------------- lattice invariants
@pytest.fixture(scope="module")
def lat8():
    m = meshgen.lattice(8)
    return m, meshgen.flow_state(m)


@pytest.mark.parametrize("order", [1, 2])
def test_global_conservation(lat8, order):
    m, q = lat8
    R, _, Ra = oracle.residual(order, m.edge, q, m.normal, m.dx, m.volume,
                               with_abs=True)
    assert np.all(np.abs(R.sum(axis=0)) <= 64 * EPS * Ra.sum(axis=0))


def test_green_gauss_sums_telescope(lat8):
    m, q = lat8
    G, Ga = oracle.green_gauss(m.edge, q, m.normal, with_abs=True)
    assert np.all(np.abs(G.sum(axis=0)) <= 64 * EPS * Ga.sum(axis=0))


def test_green_gauss_linear_field_closed_form():
    # unperturbed, unpermuted lattice; q_k = c_k + g_k . (a, b, c) is linear
    # away from the periodic seam.  For an interior node each offset class o
    # gives (q_{i+o} - q_{i-o})/2 n_o = (g.o) n_o, and sum_o n_o o^T =
    # (1 + 2 sqrt(2)/... ) -> with |n_axis| = 1 and |n_diag| = 1/2 the sum is
    # I + (1/(2 sqrt 2)) * 4 I = (1 + sqrt 2) I: Graw = (1 + sqrt 2) g.
    n = 7
    m = meshgen.lattice(n, perturbed=False, permute=False)
    lid = np.arange(n ** 3)
    pos = np.stack([lid % n, (lid // n) % n, lid // (n * n)], axis=1)
    rng = np.random.default_rng(6)
    g = rng.uniform(-1, 1, (6, 3))
    c0 = rng.uniform(1, 2, 6)
    q = c0[None, :] + pos @ g.T
    Graw = oracle.green_gauss(m.edge, q, m.normal).reshape(-1, 6, 3)
    inner = np.all((pos >= 1) & (pos <= n - 2), axis=1)
    expect = (1.0 + math.sqrt(2.0)) * g
    np.testing.assert_allclose(Graw[inner], np.broadcast_to(
        expect, Graw[inner].shape), rtol=1e-12, atol=1e-12)


def test_flux2_linear_field_has_no_dissipation():
    # with exact gradients the reconstructed face states coincide at the
    # midpoint (linear exactness), so F = f(q_mid).n for interior edges
    n = 7
    m = meshgen.lattice(n, perturbed=False, permute=False, jitter=0.0)
    lid = np.arange(n ** 3)
    pos = np.stack([lid % n, (lid // n) % n, lid // (n * n)], axis=1)
    base = cons(1.0, [0.5, 0.1, -0.1], 1.0, 5e-4)
    g = np.array([[0.01, 0.0, 0.0], [0.0, 0.01, 0.0], [0.0, 0.0, 0.01],
                  [0.01, 0.01, 0.0], [0.0, 0.02, 0.01], [1e-5, 0.0, 0.0]])
    q = base[None, :] + pos @ g.T
    G = np.tile(g.ravel(), (n ** 3, 1))
    e = m.edge
    inner = np.all((pos[e[:, 0]] >= 1) & (pos[e[:, 0]] <= n - 2), axis=1)
    inner &= np.all((pos[e[:, 1]] >= 1) & (pos[e[:, 1]] <= n - 2), axis=1)
    for k in np.nonzero(inner)[0][:40]:
        i, j = e[k]
        qL, qR = oracle.reconstruct(q[i], q[j], G[i], G[j], m.dx[k])
        mid = 0.5 * (q[i] + q[j])
        np.testing.assert_allclose(qL, mid, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(qR, mid, rtol=1e-13, atol=1e-16)
        F = oracle.rusanov(qL, qR, m.normal[k])
        np.testing.assert_allclose(F, oracle.euler_flux(mid, m.normal[k]),
                                   rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("order", [1, 2])
def test_freestream_preservation(order):
    m = meshgen.lattice(8, perturbed=False)
    q = meshgen.flow_state(m, uniform_state=True)
    R, G, Ra = oracle.residual(order, m.edge, q, m.normal, m.dx, m.volume,
                               with_abs=True)
    assert np.all(np.abs(R) <= 32 * EPS * Ra)
    if order == 2:
        assert np.max(np.abs(G)) < 1e-14


@pytest.mark.parametrize("order", [1, 2])
def test_edge_orientation_flip_is_bitwise_invisible(lat8, order):
    m, q = lat8
    rng = np.random.default_rng(7)
    flip = rng.random(m.num_edges) < 0.5
    e2 = m.edge.copy()
    e2[flip] = e2[flip][:, ::-1]
    n2, d2 = m.normal.copy(), m.dx.copy()
    n2[flip] *= -1.0
    d2[flip] *= -1.0
    R1, G1 = oracle.residual(order, m.edge, q, m.normal, m.dx, m.volume)
    R2, G2 = oracle.residual(order, e2, q, n2, d2, m.volume)
    assert np.array_equal(R1, R2)
    if order == 2:
        assert np.array_equal(G1, G2)


def test_spectral_radius_uniform_state_closed_form():
    # rho = gamma, p = 1: a = 1.  Every node meets each offset class twice.
    m = meshgen.lattice(5, perturbed=False)
    u = np.array([0.5, 0.1, -0.2])
    q = np.tile(cons(G14, u, 1.0), (m.num_nodes, 1))
    lam = oracle.spectral_radius(m.edge, q, m.normal)
    cls = meshgen.OFFSETS / np.linalg.norm(meshgen.OFFSETS, axis=1)[:, None]
    nrm = cls * meshgen.AREAS[:, None]
    expect = 2.0 * np.sum(np.abs(nrm @ u) + meshgen.AREAS)
    np.testing.assert_allclose(lam, expect, rtol=1e-14)
    dt = oracle.time_step(m.volume, lam, 0.5)
    np.testing.assert_allclose(dt, 0.5 * m.volume / expect, rtol=1e-14)


def test_rk_update_by_hand():
    q0 = np.array([[1.0, 2.0, 3.0, 4.0, 5.0, 6.0]])
    R = np.array([[8.0, -8.0, 0.0, 16.0, 1.0, -2.0]])
    q = oracle.rk_update(q0, R, np.array([2.0]), np.array([0.5]), 0.25)
    # alpha dt / V = 0.25 * 0.5 / 2 = 1/16
    np.testing.assert_array_equal(q, [[0.5, 2.5, 3.0, 3.0, 4.9375, 6.125]])


def test_march_single_stage_and_freestream():
    m = meshgen.lattice(5)
    q = meshgen.flow_state(m)
    q1, st = oracle.march(2, 1, m.edge, q, m.normal, m.dx, m.volume, stages=1)
    assert st == 0
    lam = oracle.spectral_radius(m.edge, q, m.normal)
    dt = oracle.time_step(m.volume, lam, 0.5)
    R, _ = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume)
    # one stage with alpha = 1: q1 = q - (dt/V) R, written out by hand
    np.testing.assert_allclose(q1, q - (dt / m.volume)[:, None] * R,
                               rtol=1e-15, atol=1e-16)
    mu = meshgen.lattice(5, perturbed=False)
    qu = meshgen.flow_state(mu, uniform_state=True)
    qm, st = oracle.march(2, 3, mu.edge, qu, mu.normal, mu.dx, mu.volume)
    assert st == 0
    np.testing.assert_allclose(qm, qu, rtol=1e-13, atol=1e-16)


def test_march_positivity_detected():
    m = meshgen.lattice(4)
    q = meshgen.flow_state(m)
    _, st = oracle.march(1, 5, m.edge, q, m.normal, m.dx, m.volume, cfl=50.0)
    assert st < 0


# --------------------------------------------------------------- adjoint
def _kink_safe(m, order, q, h):
    """Nodes and edges whose perturbation leaves every kink untouched.

    A kink edge has a face state with |u.n| or |sL - sR| below 50 h.  q_m
    reaches the edges at m (order 1), and through the gradients of m and
    its neighbours the edges at those nodes too (order 2); n_e reaches edge
    e (order 1) and, through the two end gradients, the edges at its ends.
    """
    margin = oracle.kink_margin(order, m.edge, q, m.normal, m.dx, m.volume)
    kink_e = margin < 50 * h
    kink_nodes = np.zeros(m.num_nodes, dtype=bool)
    kink_nodes[m.edge[kink_e].ravel()] = True
    if order == 1:
        return ~kink_nodes, ~kink_e
    bad_nodes = kink_nodes.copy()
    bad_nodes[m.edge[kink_nodes[m.edge].any(axis=1)].ravel()] = True
    bad_edges = kink_nodes[m.edge].any(axis=1)
    return ~bad_nodes, ~bad_edges


def _central(Rfun, lam, x, p, h):
    """d(lam . R)/dx_p by central differences at h and h/2 combined by
    Richardson extrapolation; R is differenced per node first, so nodes the
    perturbation does not reach contribute exact zeros."""
    def d(hh):
        xp, xm = x.copy(), x.copy()
        xp.flat[p] += hh
        xm.flat[p] -= hh
        return float(np.sum(lam * (Rfun(xp) - Rfun(xm)))) / (2 * hh)
    return (4.0 * d(h / 2) - d(h)) / 3.0


@pytest.mark.parametrize("order", [1, 2])
def test_reverse_sweep_against_central_differences(order):
    # h = 1e-6 absolute; the passive scalar (values ~1e-3, jumps ~1e-4,
    # which is also the smoothness scale of its limiter) takes 1e-8
    m = meshgen.lattice(6)
    q = meshgen.flow_state(m)
    lam = meshgen.adjoint_seed(m.num_nodes)
    h = 1e-6
    qb, nb = oracle.residual_reverse(order, m.edge, q, m.normal, m.dx,
                                     m.volume, lam)
    ok_n, ok_e = _kink_safe(m, order, q, h)

    def Rq(x):
        return oracle.residual(order, m.edge, x, m.normal, m.dx, m.volume)[0]

    def Rn(x):
        return oracle.residual(order, m.edge, q, x, m.dx, m.volume)[0]

    picks = meshgen.fd_picks(400, 6 * m.num_nodes)
    picks = [p for p in picks if ok_n[p // 6]][:32]
    assert len(picks) >= 16
    for p in picks:
        fd = _central(Rq, lam, q, p, h if p % 6 < 5 else 1e-8)
        assert fd == pytest.approx(qb.flat[p], rel=1e-6, abs=1e-9)
    picks = meshgen.fd_picks(400, 3 * m.num_edges, seed=1)
    picks = [p for p in picks if ok_e[p // 3]][:32]
    assert len(picks) >= 16
    for p in picks:
        fd = _central(Rn, lam, m.normal, p, h)
        assert fd == pytest.approx(nb.flat[p], rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("order", [1, 2])
def test_dot_product_tangent_vs_reverse(order):
    m = meshgen.lattice(6)
    q = meshgen.flow_state(m)
    lam = meshgen.adjoint_seed(m.num_nodes)
    qd = meshgen.adjoint_seed(m.num_nodes, stream=meshgen.STREAM_V)
    nd = meshgen.normal(0, meshgen.STREAM_V, np.arange(
        6 * m.num_nodes, 6 * m.num_nodes + 3 * m.num_edges,
        dtype=np.uint64)).reshape(-1, 3)
    Rd = oracle.residual_tangent(order, m.edge, q, m.normal, m.dx, m.volume,
                                 qd, nd)
    qb, nb = oracle.residual_reverse(order, m.edge, q, m.normal, m.dx,
                                     m.volume, lam)
    lhs = np.sum(lam * Rd)
    rhs = np.sum(qb * qd) + np.sum(nb * nd)
    scale = np.sum(np.abs(lam * Rd)) + np.sum(np.abs(qb * qd)) + np.sum(
        np.abs(nb * nd))
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_tangent_against_central_differences():
    m = meshgen.lattice(5)
    q = meshgen.flow_state(m)
    qd = meshgen.adjoint_seed(m.num_nodes, stream=meshgen.STREAM_V)
    qd[:, 5] *= 1e-2   # the scalar is ~1e-3: keep its step at 1e-8
    nd = np.zeros_like(m.normal)
    h = 1e-6
    Rd = oracle.residual_tangent(2, m.edge, q, m.normal, m.dx, m.volume, qd,
                                 nd)

    def d(hh):
        Rp, _ = oracle.residual(2, m.edge, q + hh * qd, m.normal, m.dx,
                                m.volume)
        Rm, _ = oracle.residual(2, m.edge, q - hh * qd, m.normal, m.dx,
                                m.volume)
        return (Rp - Rm) / (2 * hh)
    fd = (4.0 * d(h / 2) - d(h)) / 3.0
    ok_n, _ = _kink_safe(m, 2, q, 10 * h)
    np.testing.assert_allclose(fd[ok_n], Rd[ok_n], rtol=1e-6, atol=1e-8)


# ----------------------------------------------------------- renumbering
def test_rcm_on_shuffled_path_recovers_a_path():
    rng = np.random.default_rng(8)
    N = 40
    lab = rng.permutation(N)
    edge = np.array([[lab[k], lab[k + 1]] for k in range(N - 1)])
    new = oracle.rcm_order(N, edge)
    assert sorted(new.tolist()) == list(range(N))
    assert oracle.bandwidth(new[edge]) == 1


def test_rcm_textbook_small_graph():
    # star-plus-tail: 0 is the centre of {1,2,3}, 3-4-5 a tail.  Degrees:
    # 0:3, 1:1, 2:1, 3:2, 4:2, 5:1.  Start = node 1 (degree 1, lowest id);
    # BFS 1 -> 0 -> (2, 3) by (degree, id) -> 4 -> 5; reversed: 5 4 3 2 0 1.
    edge = np.array([[0, 1], [0, 2], [0, 3], [3, 4], [4, 5]])
    new = oracle.rcm_order(6, edge)
    order = np.argsort(new)
    assert order.tolist() == [5, 4, 3, 2, 0, 1]


def test_rcm_reduces_lattice_bandwidth():
    m = meshgen.lattice(10)
    new = oracle.rcm_order(m.num_nodes, m.edge)
    assert sorted(new.tolist()) == list(range(m.num_nodes))
    b_rand = oracle.bandwidth(m.edge)
    b_rcm = oracle.bandwidth(new[m.edge])
    assert b_rcm < b_rand / 2
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    e = m.edge
    A = sp.coo_matrix((np.ones(len(e)), (e[:, 0], e[:, 1])),
                      shape=(m.num_nodes,) * 2).tocsr()
    A = A + A.T
    p = csg.reverse_cuthill_mckee(A.tocsr(), symmetric_mode=True)
    inv = np.empty_like(p)
    inv[p] = np.arange(len(p))
    assert b_rcm <= 2 * oracle.bandwidth(inv[e])


def test_reductions_closed_forms_and_library_norms():
    ones = np.ones((1000, 2))
    ones[:, 1] = -2.0
    np.testing.assert_array_equal(oracle.reduce(ones, 0), [1000.0, -2000.0])
    np.testing.assert_allclose(oracle.reduce(ones, 1), [math.sqrt(1000.0), 2 * math.sqrt(1000.0)],
                               rtol=1e-15)
    np.testing.assert_array_equal(oracle.reduce(ones, 2), [1.0, 2.0])
    np.testing.assert_array_equal(oracle.reduce(ones, 3), [1.0, -2.0])
    rng = np.random.default_rng(9)
    x = rng.normal(size=(5000, 6))
    np.testing.assert_allclose(oracle.reduce(x, 1), np.linalg.norm(x, axis=0), rtol=1e-13)
    np.testing.assert_array_equal(oracle.reduce(x, 2), np.max(np.abs(x), axis=0))
    np.testing.assert_array_equal(oracle.reduce(x, 3), np.min(x, axis=0))
