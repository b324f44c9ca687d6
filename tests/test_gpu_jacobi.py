"""Block-Jacobi preconditioning on the GPU against the oracle: the per-node
blocks under every strategy, their inverses, the preconditioned stage and a
preconditioned march (FP64)."""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen
from paper_1403_7209_gb300.solver import RK5_ALPHA

pytestmark = pytest.mark.gpu


def make(m, q, **kw):
    from paper_1403_7209_gb300.solver import EdgeSolver
    return EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, precond=True, **kw)


def blockwise(a, b):
    """max over nodes of max |a_i - b_i| / max |b_i| (blocks of 36)."""
    a, b = a.reshape(a.shape[0], -1), b.reshape(b.shape[0], -1)
    return float(np.max(np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)))


@pytest.fixture(scope="module")
def mesh():
    m = meshgen.lattice(9)  # 729 nodes, 6,561 edges: several blocks and a ragged tail
    return m, meshgen.flow_state(m)


@pytest.mark.parametrize("strat,block,part", [(1, 256, 0), (1, 128, 0), (2, 128, 256),
                                              (3, 256, 0), (5, 128, 256), (6, 128, 0),
                                              (7, 128, 0)])
@pytest.mark.parametrize("renumber", ["none", "rcm"])
def test_blocks_and_inverses_match_oracle(gpu_lib, mesh, strat, block, part, renumber):
    m, q = mesh
    M = oracle.jacobi_blocks(m.edge, q, m.normal)
    P, bad = oracle.block_invert(M)
    assert bad == 0
    s = make(m, q, renumber=renumber)
    for loop in (gpu_lib.LOOP_JACOBI, gpu_lib.LOOP_JACOBI_SUMS):
        s.set_strategy(loop, 0, strat, block, part, 0)
    # the 36-value edge loop, then the inversion loop
    s.precondition(factored=False)
    assert s.plan_stats(gpu_lib.LOOP_JACOBI, 0)["strategy"] == strat
    assert blockwise(s.fetch_nodes("M"), M) <= 1e-13
    assert blockwise(s.fetch_nodes("P"), P) <= 1e-12
    # without ZERO_INC the blocks are added
    gpu_lib.op2b_jacobi_blocks(s.ctx, s.a_jac, s.gamma, 0)
    assert blockwise(s.fetch_nodes("M"), 2 * M) <= 1e-13
    # factored: four sums per node, one pass forming and inverting the blocks
    s.t["M"].zero_()
    s.t["P"].zero_()
    s.precondition()
    assert s.plan_stats(gpu_lib.LOOP_JACOBI_SUMS, 0)["strategy"] == strat
    assert blockwise(s.fetch_nodes("M"), M) <= 1e-13
    assert blockwise(s.fetch_nodes("P"), P) <= 1e-12
    lam = oracle.spectral_radius(m.edge, q, m.normal)
    JS = s.fetch_nodes("JS")
    assert np.max(np.abs(JS[:, 0] - lam) / lam) <= 1e-14
    # P alone (M skipped)
    s.t["P"].zero_()
    gpu_lib.op2b_jacobi_from_sums(s.ctx, s.d["q"], s.d["JS"], -1, s.d["P"], s.gamma)
    assert blockwise(s.fetch_nodes("P"), P) <= 1e-12
    s.close()


def test_block_inverse_pivots_and_flags_nothing(gpu_lib):
    # blocks needing row exchanges (zero diagonal) and random ones, loaded
    # directly into M; a zero block gives a non-finite P
    m = meshgen.lattice(4)
    q = meshgen.flow_state(m)
    s = make(m, q)
    rng = np.random.default_rng(0)
    M = rng.normal(size=(m.num_nodes, 6, 6))
    M[0] = np.eye(6)[[1, 0, 3, 2, 5, 4]] * 2.0
    M[1] = np.eye(6)[[5, 4, 3, 2, 1, 0]]
    M[2] = 0.0
    s.load_nodes("M", M.reshape(-1, 36))
    gpu_lib.op2b_block_invert(s.ctx, s.d["M"], s.d["P"])
    P = s.fetch_nodes("P").reshape(-1, 6, 6)
    Po, bad = oracle.block_invert(M)
    assert bad == 1
    assert not np.all(np.isfinite(P[2]))
    keep = np.arange(m.num_nodes) != 2
    for i in np.nonzero(keep)[0]:
        assert np.max(np.abs(M[i] @ P[i] - np.eye(6))) <= 1e-11 * np.linalg.cond(M[i])
    assert blockwise(P[keep], Po[keep]) <= 1e-10
    s.close()


def test_precond_update_matches_oracle(gpu_lib, mesh):
    m, q = mesh
    s = make(m, q, renumber="rcm")
    s.precondition()
    L = gpu_lib
    L.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.residual(2)
    R = s.fetch_nodes("R")
    P = s.fetch_nodes("P").reshape(-1, 6, 6)
    s.update(0.375, sigma=0.25)
    ref = oracle.precond_update(q, R, P, 0.375 * 0.25)
    assert np.max(np.abs(s.fetch_nodes("q") - ref) / np.max(np.abs(ref), axis=0)) <= 1e-14
    s.close()


def test_preconditioned_march_matches_oracle(gpu_lib):
    m = meshgen.lattice(6)
    q = meshgen.flow_state(m)
    sigma, steps = 0.25, 4
    qo = q.copy()
    for _ in range(steps):
        q0 = qo.copy()
        P, bad = oracle.block_invert(oracle.jacobi_blocks(m.edge, q0, m.normal))
        assert bad == 0
        for a in RK5_ALPHA:
            R, _ = oracle.residual(2, m.edge, qo, m.normal, m.dx, m.volume)
            qo = oracle.precond_update(q0, R, P, a * sigma)
    assert oracle.check_state(qo) == 0
    s = make(m, q, renumber="rcm")
    for _ in range(steps):
        s.step(order=2, sigma=sigma)
    qg = s.fetch_nodes("q")
    assert np.max(np.abs(qg - qo) / np.max(np.abs(qo), axis=0)) <= 1e-11
    with pytest.raises(NotImplementedError):
        s.update(0.25, mixed=True, sigma=sigma)
    s.close()


def test_jacobi_argument_checks(gpu_lib, mesh):
    m, q = mesh
    s = make(m, q, mixed=True)
    L = gpu_lib
    a = list(s.a_jac)
    a[0] = (s.d["q32"],) + tuple(a[0][1:])
    a[1] = (s.d["q32"],) + tuple(a[1][1:])
    with pytest.raises(L.Op2bError) as e:
        L.op2b_jacobi_blocks(s.ctx, a, s.gamma, L.ZERO_INC)
    assert e.value.code == L.ETYPE
    for args, code in (((s.d["M"], s.d["M"]), L.EINVAL), ((s.d["q"], s.d["P"]), L.EDIM)):
        with pytest.raises(L.Op2bError) as e:
            L.op2b_block_invert(s.ctx, *args)
        assert e.value.code == code
    with pytest.raises(L.Op2bError) as e:
        L.op2b_node_update_precond(s.ctx, s.d["q0"], s.d["R"], s.d["R"], s.d["P"], 0.1)
    assert e.value.code == L.EINVAL
    for args, code in (((s.d["q"], s.d["M"], s.d["M"], s.d["P"]), L.EDIM),
                       ((s.d["q"], s.d["JS"], s.d["P"], s.d["P"]), L.EINVAL),
                       ((s.d["q32"], s.d["JS"], s.d["M"], -1), L.ETYPE)):
        with pytest.raises(L.Op2bError) as e:
            L.op2b_jacobi_from_sums(s.ctx, *args, s.gamma)
        assert e.value.code == code
    s.close()
