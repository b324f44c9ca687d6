"""Derivatives of the explicit march on the GPU (tangent and stored-state
reverse sweep, fixed local time step) against the oracle, through the C ABI.

Bar: normwise per component, max|gpu - oracle| / max|oracle| <= 1e-11.  Each
stage's adjoint or tangent agrees with the oracle's to ~1e-15 per entry
relative to its contributions (the single-residual bar is 1e-12); through
15 stages of the march those differences are carried and combined, and
1e-11 leaves an order of magnitude over what that compounding can reach on
these meshes (measured errors are printed by the assertion messages).
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-11


def normwise(gpu, ref):
    return np.max(np.abs(gpu - ref), axis=0) / np.max(np.abs(ref), axis=0)


def setup(n=8, seed=0, **kw):
    from paper_1403_7209_gb300.solver import EdgeSolver
    m = meshgen.lattice(n, seed=seed)
    q = meshgen.flow_state(m, seed=seed)
    s = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, adjoint=True, renumber="rcm", **kw)
    s.time_step(0.5)
    dt = s.fetch_nodes("dt")[:, 0]
    return m, q, s, dt


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("keep", [True, False])
def test_march_adjoint_matches_oracle(gpu_lib, order, keep):
    m, q, s, dt = setup()
    g = np.random.default_rng(order).normal(size=q.shape)
    s.load_nodes("sbar", g)
    s.march_adjoint(3, order=order, keep_gradients=keep)
    qb, nb = oracle.march_reverse(order, 3, m.edge, q, m.normal, m.dx, m.volume, dt, g)
    e_q = normwise(s.fetch_nodes("sbar"), qb)
    e_n = normwise(s.fetch_edges("nbar_acc"), nb)
    assert np.all(e_q <= TOL) and np.all(e_n <= TOL), (e_q, e_n)
    # q holds the final state of the march
    qN, st = oracle.march_dt(order, 3, m.edge, q, m.normal, m.dx, m.volume, dt)
    assert st == 0
    assert np.all(normwise(s.fetch_nodes("q"), qN) <= 1e-12)
    s.close()


@pytest.mark.parametrize("order", [1, 2])
def test_march_tangent_matches_oracle(gpu_lib, order):
    m, q, s, dt = setup(seed=1)
    rng = np.random.default_rng(10 + order)
    qd, nd = rng.normal(size=q.shape), rng.normal(size=m.normal.shape)
    s.load_nodes("qd", qd)
    s.load_edges("nd", nd)
    s.march_tangent(3, order=order)
    _, qdN = oracle.march_tangent(order, 3, m.edge, q, m.normal, m.dx, m.volume, dt, qd, nd)
    e = normwise(s.fetch_nodes("qd"), qdN)
    assert np.all(e <= TOL), e
    s.close()


@pytest.mark.parametrize("order", [1, 2])
def test_march_dot_product_on_the_gpu(gpu_lib, order):
    # <g, dq_N> from the GPU tangent march = <qbar_0, dq_0> + <nbar, dn>
    # from the GPU reverse sweep, with the deterministic strategies
    m, q, s, dt = setup(seed=2)
    for loop in range(gpu_lib.NUM_LOOPS):
        s.set_strategy(loop, 0, gpu_lib.STRAT_AUTO_DET)
    rng = np.random.default_rng(20 + order)
    g, qd, nd = rng.normal(size=q.shape), rng.normal(size=q.shape), rng.normal(size=m.normal.shape)
    s.load_nodes("qd", qd)
    s.load_edges("nd", nd)
    s.march_tangent(4, order=order)
    qdN = s.fetch_nodes("qd")
    s.load_nodes("q", q)
    s.load_nodes("sbar", g)
    s.march_adjoint(4, order=order)
    qb, nb = s.fetch_nodes("sbar"), s.fetch_edges("nbar_acc")
    lhs = float(np.sum(g * qdN))
    rhs = float(np.sum(qb * qd) + np.sum(nb * nd))
    assert abs(lhs - rhs) <= 1e-12 * (np.sum(np.abs(g * qdN)) + np.sum(np.abs(qb * qd))), (lhs, rhs)
    s.close()


def test_kept_and_recomputed_gradients_agree_bitwise(gpu_lib):
    # with deterministic strategies the gradient recomputed in the reverse
    # sweep is the one the forward march kept, bit for bit
    m, q, s, dt = setup(seed=3)
    for loop in range(gpu_lib.NUM_LOOPS):
        s.set_strategy(loop, 0, gpu_lib.STRAT_AUTO_DET)
    g = np.random.default_rng(5).normal(size=q.shape)
    out = []
    for keep in (True, False):
        s.load_nodes("q", q)
        s.load_nodes("sbar", g)
        s.march_adjoint(2, keep_gradients=keep)
        out.append((s.t["sbar"].clone(), s.t["nbar_acc"].clone(), s.t["q"].clone()))
    for a, b in zip(*out):
        assert s.torch.equal(a, b)
    s.close()


def test_march_adjoint_matches_plain_march_state(gpu_lib):
    # the forward part of the adjoint is the ordinary march (same loops)
    m, q, s, dt = setup(seed=4)
    for loop in range(gpu_lib.NUM_LOOPS):
        s.set_strategy(loop, 0, gpu_lib.STRAT_AUTO_DET)
    for _ in range(2):
        s.step(order=2)
    qa = s.t["q"].clone()
    s.load_nodes("q", q)
    s.load_nodes("sbar", np.zeros_like(q))
    s.march_adjoint(2)
    assert s.torch.equal(qa, s.t["q"])
    assert np.all(s.fetch_nodes("sbar") == 0.0)  # zero seed, zero adjoint
    s.close()


def test_node_update_adjoint_and_axpy(gpu_lib):
    L = gpu_lib
    m, q, s, dt = setup(n=4, seed=5)
    rng = np.random.default_rng(6)
    sb, acc, y = rng.normal(size=q.shape), rng.normal(size=q.shape), rng.normal(size=m.normal.shape)
    s.load_nodes("sbar", sb)
    s.load_nodes("qacc", acc)
    L.op2b_node_update_adjoint(s.ctx, s.d["sbar"], s.d["qacc"], s.d["lam"], s.d["V"], s.d["dt"],
                               0.375)
    np.testing.assert_array_equal(s.fetch_nodes("qacc"), acc + sb)
    np.testing.assert_allclose(s.fetch_nodes("lam"), -0.375 * (dt / m.volume)[:, None] * sb,
                               rtol=1e-15)
    s.load_edges("nbar", y)
    s.load_edges("nbar_acc", 2 * y)
    L.op2b_dat_axpy(s.ctx, s.d["nbar_acc"], -0.5, s.d["nbar"])
    np.testing.assert_allclose(s.fetch_edges("nbar_acc"), 1.5 * y, rtol=1e-15)
    with pytest.raises(L.Op2bError) as e:
        L.op2b_node_update_adjoint(s.ctx, s.d["sbar"], s.d["sbar"], s.d["lam"], s.d["V"],
                                   s.d["dt"], 1.0)
    assert e.value.code == L.EINVAL
    with pytest.raises(L.Op2bError) as e:
        L.op2b_dat_axpy(s.ctx, s.d["nbar_acc"], 1.0, s.d["q"])
    assert e.value.code == L.ESET
    s.close()
