"""Node limiters (min/max, Barth-Jespersen / Venkatakrishnan) and the
node-limited flux on the GPU against the oracle, through the C ABI.

* min/max selects values: bit-exact.
* phi: the GPU forms G.d/2 with fused multiply-adds and takes the minimum
  over the ends without dividing per end, so it differs from the oracle by
  rounding only: |phi_gpu - phi_ora| <= 1e-12 (phi is O(1)).
* residuals: per node and component |difference| / sum of |edge
  contributions| <= 1e-12 (the inviscid loops' bar), FP32-mixed normwise
  <= 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12
KINDS = [("barth_jespersen", oracle.LIM_BJ, 0.0), ("venkatakrishnan", oracle.LIM_VENKAT, 0.0),
         ("venkatakrishnan", oracle.LIM_VENKAT, 1e-3)]
STRATS = [(1, 256, 0, 0), (1, 128, 0, 0), (2, 256, 512, 0), (2, 128, 256, 1),
          (2, 256, 1024, 1), (3, 256, 0, 0), (5, 256, 1024, 0), (5, 128, 512, 1),
          (6, 128, 0, 0), (7, 128, 0, 0)]


def rel_err(gpu, ref, scale):
    return float(np.max(np.abs(gpu - ref) / (scale + 1e-300)))


def make(m, q, limiter, eps2=0.0, **kw):
    from paper_1403_7209_gb300.solver import EdgeSolver
    return EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, limiter=limiter, limiter_eps2=eps2,
                      **kw)


@pytest.fixture(scope="module")
def lat16():
    m = meshgen.lattice(16)
    q = meshgen.flow_state(m)
    _, G, _ = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    return m, q, G


@pytest.mark.parametrize("renumber", ["none", "rcm", "random"])
def test_minmax_is_bit_exact(gpu_lib, lat16, renumber):
    m, q, _ = lat16
    s = make(m, q, "barth_jespersen", renumber=renumber, mixed=True)
    lo, hi = oracle.minmax(m.edge, q)
    gpu_lib.op2b_node_minmax(s.ctx, s.map, s.d["q"], s.d["qmin"], s.d["qmax"])
    np.testing.assert_array_equal(s.fetch_nodes("qmin"), lo)
    np.testing.assert_array_equal(s.fetch_nodes("qmax"), hi)
    # FP32: the extremum of the FP32 values
    q32 = q.astype(np.float32).astype(np.float64)
    lo32, hi32 = oracle.minmax(m.edge, q32)
    gpu_lib.op2b_node_minmax(s.ctx, s.map, s.d["q32"], s.d["qmin32"], s.d["qmax32"])
    np.testing.assert_array_equal(s.fetch_nodes("qmin32"), lo32)
    np.testing.assert_array_equal(s.fetch_nodes("qmax32"), hi32)
    s.close()


@pytest.mark.parametrize("name,kind,eps2", KINDS)
def test_limiter_matches_oracle(gpu_lib, lat16, name, kind, eps2):
    m, q, G = lat16
    rng = np.random.default_rng(kind)
    for Gin in (G, rng.normal(scale=0.5, size=G.shape)):  # mild and strong limiting
        s = make(m, q, name, eps2, renumber="rcm")
        s.load_nodes("G", Gin)
        s.node_limiter()
        lo, hi = oracle.minmax(m.edge, q)
        phi = oracle.limiter(kind, m.edge, q, Gin, m.dx, lo, hi, eps2)
        err = np.max(np.abs(s.fetch_nodes("phi") - phi))
        assert err <= 1e-12, err
        assert np.min(phi) < 0.9  # the limiter is active on this data
        s.close()


@pytest.mark.parametrize("strat,block,part,staged", STRATS)
def test_limited_flux_loop_all_strategies(gpu_lib, lat16, strat, block, part, staged):
    # the flux loop alone, from the oracle's phi
    m, q, G = lat16
    lo, hi = oracle.minmax(m.edge, q)
    phi = oracle.limiter(oracle.LIM_BJ, m.edge, q, G, m.dx, lo, hi)
    R, Ra = oracle.flux2_phi(m.edge, q, G, phi, m.normal, m.dx, with_abs=True)
    s = make(m, q, "barth_jespersen", renumber="rcm")
    s.load_nodes("G", G)
    s.load_nodes("phi", phi)
    s.set_strategy(gpu_lib.LOOP_FLUX2_PHI, 0, strat, block, part, staged)
    gpu_lib.op2b_edge_flux_limited(s.ctx, s.a_f2phi, s.gamma, gpu_lib.ZERO_INC)
    assert rel_err(s.fetch_nodes("R"), R, Ra) <= TOL
    s.close()


@pytest.mark.parametrize("name,kind,eps2", KINDS)
@pytest.mark.parametrize("renumber", ["rcm", "random"])
def test_limited_residual_matches_oracle(gpu_lib, lat16, name, kind, eps2, renumber):
    m, q, _ = lat16
    ref = oracle.residual_limited(kind, m.edge, q, m.normal, m.dx, m.volume, eps2,
                                  with_abs=True)
    s = make(m, q, name, eps2, renumber=renumber, seed=4)
    s.residual(2)
    assert rel_err(s.fetch_nodes("R"), ref["R"], ref["Rabs"]) <= TOL
    assert np.max(np.abs(s.fetch_nodes("phi") - ref["phi"])) <= 1e-12
    s.close()


@pytest.mark.parametrize("name,kind,eps2", KINDS[:2])
def test_limited_residual_mixed_precision(gpu_lib, lat16, name, kind, eps2):
    m, q, _ = lat16
    ref = oracle.residual_limited(kind, m.edge, q, m.normal, m.dx, m.volume, eps2)
    s = make(m, q, name, eps2, renumber="rcm", mixed=True)
    for strat in (1, 2, 3, 5, 6):
        s.set_strategy(gpu_lib.LOOP_FLUX2_PHI, 1, strat, 256, 512, 1)
        s.residual(2, mixed=True)
        R = s.fetch_nodes("R")
        err = np.max(np.abs(R - ref["R"]), axis=0) / np.max(np.abs(ref["R"]), axis=0)
        assert np.all(err <= 1e-5), (strat, err)
        assert np.max(err) > 0.0
    s.close()


def test_limited_residual_irregular_and_ragged(gpu_lib):
    for m in (meshgen.random_graph_mesh(3000, seed=8), meshgen.lattice(3, seed=1),
              meshgen.lattice(5, seed=2)):
        q = meshgen.flow_state(m, seed=3)
        ref = oracle.residual_limited(oracle.LIM_BJ, m.edge, q, m.normal, m.dx, m.volume,
                                      with_abs=True)
        s = make(m, q, "barth_jespersen", renumber="rcm")
        for strat, block, part, staged in ((1, 64, 0, 0), (2, 64, 64, 1), (3, 64, 0, 0),
                                           (5, 64, 256, 0), (6, 64, 0, 0)):
            for loop in (gpu_lib.LOOP_GREEN_GAUSS, gpu_lib.LOOP_FLUX2_PHI):
                s.set_strategy(loop, 0, strat, block, part, staged)
            s.residual(2)
            assert rel_err(s.fetch_nodes("R"), ref["R"], ref["Rabs"]) <= TOL, (m.num_edges, strat)
        s.close()


def test_limited_march_stays_physical(gpu_lib):
    # 50 steps with the Barth-Jespersen limiter: the state stays positive and
    # finite, and the march changes it
    m = meshgen.lattice(12)
    q = meshgen.flow_state(m)
    s = make(m, q, "barth_jespersen", renumber="rcm")
    s.time_step(0.5)
    for _ in range(50):
        s.step(order=2)
    qn = s.fetch_nodes("q")
    assert np.all(np.isfinite(qn)) and np.all(qn[:, 0] > 0)
    assert np.max(np.abs(qn - q)) > 1e-6
    # the same march through the oracle's residual, stage by stage
    qo = q.copy()
    lam = oracle.spectral_radius(m.edge, q, m.normal)
    dt = oracle.time_step(m.volume, lam, 0.5)
    for _ in range(50):
        q0 = qo.copy()
        for a in oracle.RK_ALPHA:
            R = oracle.residual_limited(oracle.LIM_BJ, m.edge, qo, m.normal, m.dx, m.volume)["R"]
            qo = oracle.rk_update(q0, R, m.volume, dt, a)
    err = np.max(np.abs(qn - qo), axis=0) / np.max(np.abs(qo), axis=0)
    assert np.all(err <= 1e-10), err
    s.close()


def test_limiter_argument_checks(gpu_lib, lat16):
    L = gpu_lib
    m, q, _ = lat16
    s = make(m, q, "venkatakrishnan")
    c, d, mp = s.ctx, s.d, s.map
    with pytest.raises(L.Op2bError) as e:
        L.op2b_node_limiter(c, mp, 7, 0.0, d["q"], d["G"], d["dx"], d["qmin"], d["qmax"], d["phi"])
    assert e.value.code == L.EINVAL
    with pytest.raises(L.Op2bError) as e:
        L.op2b_node_limiter(c, mp, 2, -1.0, d["q"], d["G"], d["dx"], d["qmin"], d["qmax"], d["phi"])
    assert e.value.code == L.EINVAL
    with pytest.raises(L.Op2bError) as e:
        L.op2b_node_limiter(c, mp, 2, 0.0, d["q"], d["G"], d["dx"], d["qmin"], d["qmax"], d["q"])
    assert e.value.code == L.EINVAL
    with pytest.raises(L.Op2bError) as e:  # dx must be an edge dat
        L.op2b_node_limiter(c, mp, 2, 0.0, d["q"], d["G"], d["V"], d["qmin"], d["qmax"], d["phi"])
    assert e.value.code in (L.ESET, L.EDIM)
    with pytest.raises(L.Op2bError) as e:
        L.op2b_node_minmax(c, mp, d["q"], d["q"], d["qmax"])
    assert e.value.code == L.EINVAL
    with pytest.raises(NotImplementedError):
        s.adjoint(2)
    s.close()
