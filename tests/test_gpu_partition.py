"""Owner-compute partitions on one GPU against the whole-mesh oracle.

Every part runs the loops over its own edges (cut edges in both parts) and
refreshes its halo with the library's exchange kernel, so on its owned
nodes it must hold the whole-mesh result: residuals to the oracle within
the same 1e-12 (sum of absolute contributions) bound as the unpartitioned
loops, marches within the same bounds as the unpartitioned march tests.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12


def rel_err(gpu, ref, scale):
    return float(np.max(np.abs(gpu - ref) / (scale + 1e-300)))


def make(m, q, nparts, **kw):
    from paper_1403_7209_gb300.partition import PartitionedSolver
    return PartitionedSolver(m.edge, m.normal, m.dx, m.volume, q, coords=m.coords,
                             nparts=nparts, **kw)


@pytest.fixture(scope="module")
def mesh12():
    m = meshgen.lattice(12)
    q = meshgen.flow_state(m)
    R1, _, R1a = oracle.residual(1, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    R2, G, R2a = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    return m, q, dict(R1=R1, R1a=R1a, R2=R2, R2a=R2a, G=G)


@pytest.mark.parametrize("concurrent", [False, True])
@pytest.mark.parametrize("nparts", [1, 2, 3, 8, 27])
@pytest.mark.parametrize("strat", [1, 3, 6])
def test_partitioned_residual_matches_oracle(gpu_lib, mesh12, nparts, strat, concurrent):
    m, q, ref = mesh12
    s = make(m, q, nparts, concurrent=concurrent)
    for loop in (gpu_lib.LOOP_GREEN_GAUSS, gpu_lib.LOOP_FLUX1, gpu_lib.LOOP_FLUX2):
        s.set_strategy(loop, 0, strat, 128)
    s.residual(1)
    assert rel_err(s.fetch_nodes("R"), ref["R1"], ref["R1a"]) <= TOL
    s.residual(2)
    assert rel_err(s.fetch_nodes("R"), ref["R2"], ref["R2a"]) <= TOL
    G = s.fetch_nodes("G")
    assert np.max(np.abs(G - ref["G"]) / np.max(np.abs(ref["G"]), axis=0)) <= 1e-12
    s.close()


def test_halo_rows_come_from_the_exchange(gpu_lib, mesh12):
    # poison every part's halo rows of q; the residual must not change,
    # because the exchange refreshes them before any loop reads them
    import torch
    m, q, ref = mesh12
    s = make(m, q, 4)
    for P, sv in zip(s.parts, s.solvers):
        n_own = P["sizes"]["owned"]
        rows = torch.as_tensor(sv.perm[np.arange(n_own, P["nodes"].size)], device=sv.t["q"].device)
        sv.t["q"][:, rows] = float("nan")
    s.residual(2)
    assert rel_err(s.fetch_nodes("R"), ref["R2"], ref["R2a"]) <= TOL
    s.close()


@pytest.mark.parametrize("concurrent", [False, True])
def test_partitioned_march_matches_oracle(gpu_lib, concurrent):
    m = meshgen.lattice(8)
    q = meshgen.flow_state(m)
    s = make(m, q, 5, concurrent=concurrent)
    s.time_step(0.5)
    for _ in range(10):
        s.step(order=2)
    qo, st = oracle.march(2, 10, m.edge, q, m.normal, m.dx, m.volume)
    assert st == 0
    qg = s.fetch_nodes("q")
    assert np.max(np.abs(qg - qo) / np.max(np.abs(qo), axis=0)) <= 1e-11
    s.close()


def test_partitioned_mixed_precision(gpu_lib, mesh12):
    m, q, ref = mesh12
    s = make(m, q, 6, mixed=True)
    s.sync_shadow()
    s.residual(2, mixed=True)
    R = s.fetch_nodes("R")
    err = np.max(np.abs(R - ref["R2"]), axis=0) / np.max(np.abs(ref["R2"]), axis=0)
    assert np.all(err <= 1e-5) and np.max(err) > 0.0, err
    s.close()
    m8 = meshgen.lattice(8)
    q8 = meshgen.flow_state(m8)
    s = make(m8, q8, 3, mixed=True)
    s.time_step(0.5)
    s.sync_shadow()
    for _ in range(10):
        s.step(order=2, mixed=True)
    qo, st = oracle.march(2, 10, m8.edge, q8, m8.normal, m8.dx, m8.volume)
    err = np.max(np.abs(s.fetch_nodes("q") - qo), axis=0) / np.max(np.abs(qo), axis=0)
    assert np.all(err <= 1e-5), err
    s.close()


def test_exchange_rejects_rows_outside_a_dat(gpu_lib):
    import torch
    ctx = gpu_lib.op2b_init(0, torch.cuda.current_stream().cuda_stream)
    a = torch.zeros((6, 10), dtype=torch.float64, device="cuda")
    b = torch.zeros((6, 10), dtype=torch.float64, device="cuda")
    for si, di in (([10], [0]), ([0], [-1])):
        with pytest.raises(gpu_lib.Op2bError) as e:
            gpu_lib.op2b_exchange_create(ctx, gpu_lib.F64, 6, [a.data_ptr()], [10],
                                         [b.data_ptr()], [10], [1], si, di)
        assert e.value.code == gpu_lib.EINVAL
    with pytest.raises(gpu_lib.Op2bError) as e:
        gpu_lib.op2b_exchange_create(ctx, gpu_lib.I32, 6, [a.data_ptr()], [10],
                                     [b.data_ptr()], [10], [1], [0], [0])
    assert e.value.code == gpu_lib.ETYPE
    # a valid exchange copies the rows
    a.copy_(torch.arange(60, dtype=torch.float64, device="cuda").reshape(6, 10))
    x = gpu_lib.op2b_exchange_create(ctx, gpu_lib.F64, 6, [a.data_ptr(), a.data_ptr()], [10, 10],
                                     [b.data_ptr(), b.data_ptr()], [10, 10], [2, 1],
                                     [3, 7, 0], [9, 0, 5])
    gpu_lib.op2b_exchange_run(ctx, x)
    torch.cuda.synchronize()
    ref = torch.zeros_like(b)
    ref[:, 9], ref[:, 0], ref[:, 5] = a[:, 3], a[:, 7], a[:, 0]
    assert torch.equal(b, ref)
    gpu_lib.op2b_exchange_destroy(ctx, x)
    gpu_lib.op2b_finalize(ctx)
