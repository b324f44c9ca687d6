"""Pins of the oracle's node limiters (Barth-Jespersen, Venkatakrishnan) and
of the node-limited flux, against facts derived outside oracle.c: brute-force
neighbour min/max, closed forms of the limiter functions, a two-node mesh by
hand, linear fields (no limiting), the face-value bound that defines the
Barth-Jespersen limiter, extrema, the first-order special case (phi = 0),
conservation and edge-orientation invariance.  CPU only.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

BJ, VK = oracle.LIM_BJ, oracle.LIM_VENKAT
EPS = np.finfo(np.float64).eps


def neighbours_minmax(edge, q):
    lo, hi = q.copy(), q.copy()
    for a, b in edge:
        lo[a] = np.minimum(lo[a], q[b])
        hi[a] = np.maximum(hi[a], q[b])
        lo[b] = np.minimum(lo[b], q[a])
        hi[b] = np.maximum(hi[b], q[a])
    return lo, hi


def test_minmax_is_the_neighbourhood_extremum():
    m = meshgen.random_graph_mesh(400, seed=3)  # uneven degrees, isolated nodes
    q = np.random.default_rng(0).normal(size=(m.num_nodes, 6))
    lo, hi = oracle.minmax(m.edge, q)
    rlo, rhi = neighbours_minmax(m.edge, q)
    np.testing.assert_array_equal(lo, rlo)
    np.testing.assert_array_equal(hi, rhi)


def test_edge_limiter_closed_forms():
    assert oracle.limiter_edge(BJ, 1.0, 2.0) == 0.5
    assert oracle.limiter_edge(BJ, 3.0, 2.0) == 1.0
    assert oracle.limiter_edge(BJ, -1.0, -4.0) == 0.25
    assert oracle.limiter_edge(BJ, 0.0, 2.0) == 0.0        # extremum: flat
    assert oracle.limiter_edge(BJ, 5.0, 0.0) == 1.0        # nothing to limit
    # Venkatakrishnan (D1^2 + 2 D1 D2) / (D1^2 + 2 D2^2 + D1 D2) at eps2 = 0
    assert oracle.limiter_edge(VK, 1.0, 1.0) == 0.75
    assert oracle.limiter_edge(VK, 1.0, 2.0) == pytest.approx(5.0 / 11.0, rel=EPS)
    assert oracle.limiter_edge(VK, 1.0, 0.25) == pytest.approx(12.0 / 11.0, rel=EPS)  # > 1
    assert oracle.limiter_edge(VK, 1.0, 0.5) == 1.0
    assert oracle.limiter_edge(VK, 0.0, 3.0) == 0.0
    assert oracle.limiter_edge(VK, -2.0, -4.0) == pytest.approx(20.0 / 44.0, rel=EPS)
    # a large eps2 switches the limiter off
    assert oracle.limiter_edge(VK, 0.0, 1e-3, eps2=1e6) == pytest.approx(1.0, rel=1e-8)


def test_two_node_mesh_by_hand():
    # q0 = 0, q1 = 1 for every variable; dx = (1, 0, 0); G = (4, 0, 0) at both
    # nodes, so D2 = +2 at node 0 and -2 at node 1 with D1 = +1 and -1
    edge = np.array([[0, 1]], np.int32)
    q = np.array([[0.0] * 6, [1.0] * 6])
    G = np.zeros((2, 18))
    G[:, 0::3] = 4.0
    dx = np.array([[1.0, 0.0, 0.0]])
    lo, hi = oracle.minmax(edge, q)
    assert np.all(lo == 0.0) and np.all(hi == 1.0)
    np.testing.assert_array_equal(oracle.limiter(BJ, edge, q, G, dx, lo, hi), 0.5)
    np.testing.assert_allclose(oracle.limiter(VK, edge, q, G, dx, lo, hi), 5.0 / 11.0, rtol=EPS)


def linear_graph_case(seed):
    m = meshgen.random_graph_mesh(500, seed=seed)
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(6, 3))
    q = rng.normal(size=6) + m.coords @ B.T
    G = np.repeat(B[None], m.num_nodes, axis=0).reshape(m.num_nodes, 18)
    return m, q, G


@pytest.mark.parametrize("seed", [1, 2])
def test_linear_fields_are_not_limited(seed):
    # exact gradients of a linear field: the midpoint extrapolation is half
    # the jump to the neighbour, so D1 >= 2 D2 at every edge end
    m, q, G = linear_graph_case(seed)
    lo, hi = oracle.minmax(m.edge, q)
    assert np.all(oracle.limiter(BJ, m.edge, q, G, m.dx, lo, hi) == 1.0)
    # Venkatakrishnan is >= 1 for D2/D1 in [0, 1/2] (= 1 at both ends); D1 is
    # a difference of rounded values (relative error eps |q| / |D1|, up to
    # ~1e-13 for the closest neighbours here) and the slope at 1/2 is -1/2
    assert np.all(oracle.limiter(VK, m.edge, q, G, m.dx, lo, hi) >= 1.0 - 1e-11)


def face_values(m, q, G, phi):
    """q_i + phi_i G_i.d/2 at both ends of every edge (numpy)."""
    Gr = G.reshape(-1, 6, 3)
    i, j = m.edge[:, 0], m.edge[:, 1]
    d2i = 0.5 * np.einsum("ekd,ed->ek", Gr[i], m.dx)
    d2j = 0.5 * np.einsum("ekd,ed->ek", Gr[j], -m.dx)
    return (i, q[i] + phi[i] * d2i), (j, q[j] + phi[j] * d2j)


@pytest.mark.parametrize("kind", [BJ, VK])
def test_limited_face_values_stay_within_the_neighbourhood_bounds(kind):
    # the defining property of Barth-Jespersen, and of Venkatakrishnan at
    # eps2 = 0 (D2 phi_e <= D1 there): no new extrema at the faces
    m = meshgen.random_graph_mesh(600, seed=5)
    rng = np.random.default_rng(5)
    q = rng.normal(size=(m.num_nodes, 6))
    G = rng.normal(scale=3.0, size=(m.num_nodes, 18))
    lo, hi = oracle.minmax(m.edge, q)
    phi = oracle.limiter(kind, m.edge, q, G, m.dx, lo, hi)
    assert np.all(phi >= 0.0)
    if kind == BJ:
        assert np.all(phi <= 1.0)
    tol = 1e-14 * (np.abs(q).max() + 1)
    for nodes, f in face_values(m, q, G, phi):
        assert np.all(f <= hi[nodes] + tol) and np.all(f >= lo[nodes] - tol)
    # and the limiting is active: some phi well below 1
    assert np.min(phi) < 0.5


def test_local_extremum_is_flattened():
    m = meshgen.random_graph_mesh(300, seed=7)
    rng = np.random.default_rng(7)
    q = rng.normal(size=(m.num_nodes, 6))
    G = rng.normal(size=(m.num_nodes, 18))
    deg = np.bincount(m.edge.ravel(), minlength=m.num_nodes)
    node = int(np.argmax(deg))
    q[node, 2] = 100.0  # strict maximum of variable 2 in its neighbourhood
    lo, hi = oracle.minmax(m.edge, q)
    for kind in (BJ, VK):
        phi = oracle.limiter(kind, m.edge, q, G, m.dx, lo, hi)
        assert phi[node, 2] == 0.0  # some edge end extrapolates upwards


def test_zero_phi_gives_the_first_order_flux():
    m = meshgen.lattice(4, seed=2)
    q = meshgen.flow_state(m, seed=2)
    G = np.random.default_rng(1).normal(size=(m.num_nodes, 18))
    R0 = oracle.flux2_phi(m.edge, q, G, np.zeros((m.num_nodes, 6)), m.normal, m.dx)
    np.testing.assert_array_equal(R0, oracle.flux1(m.edge, q, m.normal))


@pytest.mark.parametrize("kind", [BJ, VK])
def test_limited_residual_conservation_and_orientation(kind):
    m = meshgen.lattice(5, seed=3)
    q = meshgen.flow_state(m, seed=3)
    out = oracle.residual_limited(kind, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    Rs = np.abs(out["R"].sum(axis=0))
    assert np.all(Rs <= 64 * EPS * out["Rabs"].sum(axis=0))
    # reverse every other edge (i <-> j, n -> -n, dx -> -dx): identical
    flip = np.arange(m.num_edges) % 2 == 1
    edge, n, dx = m.edge.copy(), m.normal.copy(), m.dx.copy()
    edge[flip] = edge[flip][:, ::-1]
    n[flip] *= -1
    dx[flip] *= -1
    out2 = oracle.residual_limited(kind, edge, q, n, dx, m.volume)
    np.testing.assert_array_equal(out2["phi"], out["phi"])
    np.testing.assert_array_equal(out2["R"], out["R"])
