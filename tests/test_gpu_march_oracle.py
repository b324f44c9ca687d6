"""50-step explicit marches on the GPU against the oracle's march.

The oracle marches the 40^3 periodic lattice (64,000 nodes, 576,000 edges)
50 steps of the five-stage scheme (250 stages, local time step frozen from
the initial state, CFL 0.5); its final state is cached on disk by
``oracle.march_cache`` (the cache key includes the oracle's source).

Bars, normwise per component (max |q_gpu - q_ora| / max |q_ora|):
- FP64 march: 1e-12, the relative bar of the FP64 loops against the oracle
  applied to the state.  Each stage's residual matches the oracle's to
  1e-12 of the sum of its absolute contributions (only the summation order
  differs), and a stage moves the state by alpha (dt/V) R, a small fraction
  of |q|, so the 250 stages' differences stay far inside it (measured
  ~2e-15); a loose worst case, 250 x 1e-12, would allow 2.5e-10.
- FP32-mixed march (FP32 node data, gradients, normals and flux arithmetic,
  FP64 residual and update), by the separate loops and by the fused stage:
  1e-5, the mixed path's residual bar, applied to the state after the march.
"""
import numpy as np
import pytest

from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu

N_SIDE, STEPS = 40, 50
BAR_FP64 = 1e-12
BAR_MIXED = 1e-5


@pytest.fixture(scope="module")
def oracle_state():
    from oracle import march_cache
    q, status, _ = march_cache.oracle_march(N_SIDE, STEPS)
    assert status == 0
    return q


def _march(gpu_lib, mixed, strategy=None, fused=False, renumber="rcm"):
    from paper_1403_7209_gb300.solver import EdgeSolver
    m = meshgen.lattice(N_SIDE)
    q = meshgen.flow_state(m)
    s = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, renumber=renumber, mixed=mixed,
                   coords=m.coords)
    prec = gpu_lib.PREC_F32 if mixed else gpu_lib.PREC_F64
    if strategy is not None:
        for loop in (gpu_lib.LOOP_GREEN_GAUSS, gpu_lib.LOOP_FLUX2):
            s.set_strategy(loop, prec, *strategy)
    s.time_step(0.5)
    for _ in range(STEPS):
        s.step(order=2, mixed=mixed, fused=fused)
    qg = s.fetch_nodes("q")
    s.close()
    return qg


def _normwise(qg, qo):
    return np.max(np.abs(qg - qo), axis=0) / np.max(np.abs(qo), axis=0)


@pytest.mark.parametrize("strategy", [None, (3, 256, 0, 0), (6, 128, 0, 0)],
                         ids=["default", "segmented", "owner"])
def test_fp64_march_50_steps_matches_oracle(gpu_lib, oracle_state, strategy):
    err = _normwise(_march(gpu_lib, False, strategy), oracle_state)
    assert np.all(err <= BAR_FP64), err
    assert np.all(np.isfinite(err))


@pytest.mark.parametrize("strategy", [None, (7, 128, 0, 0), (6, 128, 0, 0)],
                         ids=["default", "gather", "owner"])
def test_mixed_march_50_steps_within_bar_of_oracle(gpu_lib, oracle_state, strategy):
    err = _normwise(_march(gpu_lib, True, strategy), oracle_state)
    assert np.all(err <= BAR_MIXED), err
    assert np.max(err) > 0.0  # the FP32 arithmetic really ran


@pytest.mark.parametrize("renumber", ["rcm", "rcb"])
def test_fused_mixed_march_50_steps_within_bar_of_oracle(gpu_lib, oracle_state, renumber):
    """The fused FP32-mixed stage (op2b_stage_mixed) marched 50 steps."""
    err = _normwise(_march(gpu_lib, True, fused=True, renumber=renumber), oracle_state)
    assert np.all(err <= BAR_MIXED), err
    assert np.max(err) > 0.0
