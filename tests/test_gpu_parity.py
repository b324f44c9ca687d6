"""CUDA edge loops against the CPU oracle, through the C ABI.

Error measure for residuals and gradients (per node and component): the
absolute difference divided by the sum of the absolute values of the edge
contributions to that entry (the oracle's Rabs / Gabs).  Only the order of
the scatter and of a few operations differs from the oracle, so the bound
is 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12
STRATS = [("atomic", 1, 256, 0, 0), ("atomic128", 1, 128, 0, 0), ("gather", 7, 128, 0, 0),
          ("colour", 2, 256, 512, 0), ("colour_staged", 2, 128, 256, 1),
          ("colour_staged_big", 2, 256, 1024, 1), ("segmented", 3, 256, 0, 0),
          ("block_atomic", 5, 256, 1024, 0), ("block_atomic_staged", 5, 128, 512, 1),
          ("owner", 6, 128, 0, 0)]


def rel_err(gpu, ref, scale):
    return float(np.max(np.abs(gpu - ref) / (scale + 1e-300)))


def make_solver(op2b, m, q, renumber="none", **kw):
    from paper_1403_7209_gb300.solver import EdgeSolver
    return EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, renumber=renumber, **kw)


@pytest.fixture(scope="module")
def mesh16():
    m = meshgen.lattice(16)
    q = meshgen.flow_state(m)
    return m, q


@pytest.fixture(scope="module")
def ref16(mesh16):
    m, q = mesh16
    R1, _, R1a = oracle.residual(1, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    R2, G, R2a = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    Graw, Ga = oracle.green_gauss(m.edge, q, m.normal, with_abs=True)
    return dict(R1=R1, R1a=R1a, R2=R2, R2a=R2a, G=G, Gabs=Ga / m.volume[:, None])


@pytest.mark.parametrize("name,strat,block,part,staged", STRATS)
def test_flux1_matches_oracle(gpu_lib, mesh16, ref16, name, strat, block, part, staged):
    m, q = mesh16
    s = make_solver(gpu_lib, m, q)
    s.set_strategy(gpu_lib.LOOP_FLUX1, 0, strat, block, part, staged)
    s.flux(1)
    assert rel_err(s.fetch_nodes("R"), ref16["R1"], ref16["R1a"]) <= TOL
    s.close()


@pytest.mark.parametrize("name,strat,block,part,staged", STRATS)
def test_green_gauss_matches_oracle(gpu_lib, mesh16, ref16, name, strat, block, part, staged):
    m, q = mesh16
    s = make_solver(gpu_lib, m, q)
    s.set_strategy(gpu_lib.LOOP_GREEN_GAUSS, 0, strat, block, part, staged)
    s.green_gauss()
    assert rel_err(s.fetch_nodes("G"), ref16["G"], ref16["Gabs"]) <= TOL
    s.close()


@pytest.mark.parametrize("block", [128, 256])
@pytest.mark.parametrize("renumber", ["none", "rcm"])
def test_green_gauss_gather_matches_oracle(gpu_lib, mesh16, ref16, block, renumber):
    # the node-gather strategy (Green-Gauss only) in FP64 and FP32, with
    # and without zeroing, and bitwise reproducible
    m, q = mesh16
    s = make_solver(gpu_lib, m, q, renumber=renumber, mixed=True)
    for prec in (0, 1):
        s.set_strategy(gpu_lib.LOOP_GREEN_GAUSS, prec, gpu_lib.STRAT_GATHER, block)
    s.green_gauss()
    G = s.fetch_nodes("G")
    assert rel_err(G, ref16["G"], ref16["Gabs"]) <= TOL
    s.green_gauss()
    assert np.array_equal(s.fetch_nodes("G"), G)
    gpu_lib.op2b_green_gauss(s.ctx, s.a_gg, 0)  # no ZERO_INC: the sums are added
    Graw, Gabs = oracle.green_gauss(m.edge, q, m.normal, with_abs=True)
    assert rel_err(s.fetch_nodes("G"), ref16["G"] + Graw, ref16["Gabs"] + Gabs) <= TOL
    s.sync_shadow()
    s.green_gauss(mixed=True)
    err = np.max(np.abs(s.fetch_nodes("G32") - ref16["G"]), axis=0) / np.max(np.abs(ref16["G"]), axis=0)
    assert np.all(err <= 1e-5), err
    with pytest.raises(gpu_lib.Op2bError) as e:  # per-edge outputs: no gather
        s.set_strategy(gpu_lib.LOOP_FLUX2_ADJ, 0, gpu_lib.STRAT_GATHER, block)
    assert e.value.code == gpu_lib.EINVAL
    s.close()


@pytest.mark.parametrize("prec,strat", [(0, 7), (0, 3), (0, 2), (1, 7), (1, 3), (2, 0)])
def test_green_gauss_scaled_is_the_loop_then_the_scaling(gpu_lib, mesh16, ref16, prec, strat):
    """op2b_green_gauss_scaled gives the bits of op2b_green_gauss followed by
    op2b_grad_scale: fused into the node gather (7; the float-float loop,
    prec 2) and into the segmented strategy's node phase (3), the scaling
    loop after the colour strategy (2) (all in a fixed order, so bitwise
    comparable); with and without ZERO_INC."""
    import torch
    m, q = mesh16
    s = make_solver(gpu_lib, m, q, renumber="rcm", mixed=True, ff=True)
    s.sync_shadow()
    s.sync_shadow(ff=True)
    if prec < 2:
        s.set_strategy(gpu_lib.LOOP_GREEN_GAUSS, prec, strat, 128, 256, 0)
    a = (s.a_gg, s.a_gg32, s.a_gg_ff)[prec]
    G = ("G", "G32", "G_ff")[prec]
    c, V = s.ctx, s.d["V"]
    gpu_lib.op2b_green_gauss(c, a, gpu_lib.ZERO_INC)
    gpu_lib.op2b_grad_scale(c, s.d[G], V)
    two = s.t[G].clone()
    s.t[G].fill_(float("nan"))
    gpu_lib.op2b_green_gauss_scaled(c, a, V, gpu_lib.ZERO_INC)
    assert torch.equal(s.t[G], two)
    # without ZERO_INC: G = (G_in + sums) / V
    gpu_lib.op2b_green_gauss(c, a, 0)
    gpu_lib.op2b_grad_scale(c, s.d[G], V)
    two_add = s.t[G].clone()
    s.t[G].copy_(two)
    gpu_lib.op2b_green_gauss_scaled(c, a, V, 0)
    assert torch.equal(s.t[G], two_add)
    if prec == 0:
        s.green_gauss()
        assert rel_err(s.fetch_nodes("G"), ref16["G"], ref16["Gabs"]) <= TOL
    # V must be a node dat of dim 1 in FP64
    for bad, code in ((s.d["q"], gpu_lib.EDIM), (s.d["n"], gpu_lib.ESET)):
        with pytest.raises(gpu_lib.Op2bError) as e:
            gpu_lib.op2b_green_gauss_scaled(c, a, bad, gpu_lib.ZERO_INC)
        assert e.value.code == code
    s.close()


@pytest.mark.parametrize("block", [128, 256])
def test_green_gauss_hybrid_matches_oracle(gpu_lib, mesh16, ref16, block):
    # FP64 only: gathered components 0-2, atomically scattered 3-5, one launch
    m, q = mesh16
    s = make_solver(gpu_lib, m, q, renumber="rcm")
    s.set_strategy(gpu_lib.LOOP_GREEN_GAUSS, 0, gpu_lib.STRAT_HYBRID, block)
    s.green_gauss()
    assert rel_err(s.fetch_nodes("G"), ref16["G"], ref16["Gabs"]) <= TOL
    gpu_lib.op2b_green_gauss(s.ctx, s.a_gg, 0)  # no ZERO_INC: the sums are added
    Graw, Gabs = oracle.green_gauss(m.edge, q, m.normal, with_abs=True)
    assert rel_err(s.fetch_nodes("G"), ref16["G"] + Graw, ref16["Gabs"] + Gabs) <= TOL
    for loop, prec in ((gpu_lib.LOOP_GREEN_GAUSS, 1), (gpu_lib.LOOP_FLUX2, 0)):
        with pytest.raises(gpu_lib.Op2bError) as e:
            s.set_strategy(loop, prec, gpu_lib.STRAT_HYBRID, block)
        assert e.value.code == gpu_lib.EINVAL
    s.close()


@pytest.mark.parametrize("name,strat,block,part,staged", STRATS)
def test_flux2_matches_oracle(gpu_lib, mesh16, ref16, name, strat, block, part, staged):
    m, q = mesh16
    s = make_solver(gpu_lib, m, q)
    s.set_strategy(gpu_lib.LOOP_FLUX2, 0, strat, block, part, staged)
    s.set_strategy(gpu_lib.LOOP_GREEN_GAUSS, 0, strat, block, part, staged)
    s.residual(2)
    assert rel_err(s.fetch_nodes("R"), ref16["R2"], ref16["R2a"]) <= TOL
    s.close()


@pytest.mark.parametrize("renumber", ["random", "rcm"])
def test_renumbered_residual_in_user_order(gpu_lib, mesh16, ref16, renumber):
    m, q = mesh16
    s = make_solver(gpu_lib, m, q, renumber=renumber, seed=3)
    # the library's edge order is sorted by (min end, max end)
    lo = np.minimum(s.edge[:, 0], s.edge[:, 1]).astype(np.int64)
    hi = np.maximum(s.edge[:, 0], s.edge[:, 1]).astype(np.int64)
    key = lo * m.num_nodes + hi
    assert np.all(np.diff(key) > 0)
    # and is the user's mesh relabelled
    assert np.array_equal(s.edge, s.perm[m.edge[s.order]])
    for strat in (1, 2, 3, 5, 6):
        s.set_strategy(gpu_lib.LOOP_FLUX2, 0, strat, 256, 512, 1)
        s.set_strategy(gpu_lib.LOOP_GREEN_GAUSS, 0, strat, 256, 512, 1)
        s.residual(2)
        assert rel_err(s.fetch_nodes("R"), ref16["R2"], ref16["R2a"]) <= TOL
        assert rel_err(s.fetch_nodes("G"), ref16["G"], ref16["Gabs"]) <= TOL
    s.close()


def test_ragged_and_tiny_meshes(gpu_lib):
    # E = 243 and 1125: tails shorter than a block and a partition
    for n in (3, 5):
        m = meshgen.lattice(n, seed=1)
        q = meshgen.flow_state(m, seed=1)
        R, _, Ra = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
        for strat, part, staged in ((1, 0, 0), (2, 64, 0), (2, 64, 1), (2, 4096, 1), (3, 0, 0),
                                    (5, 64, 1), (5, 4096, 0), (6, 0, 0)):
            s = make_solver(gpu_lib, m, q)
            s.set_strategy(gpu_lib.LOOP_FLUX2, 0, strat, 64, part, staged)
            s.set_strategy(gpu_lib.LOOP_GREEN_GAUSS, 0, strat, 64, part, staged)
            s.residual(2)
            assert rel_err(s.fetch_nodes("R"), R, Ra) <= TOL
            s.close()


def test_empty_edge_set_gives_zero_residual(gpu_lib):
    N = 10
    q = np.tile([1.0, 0.5, 0.0, 0.0, 2.5, 0.0], (N, 1))
    from paper_1403_7209_gb300.solver import EdgeSolver
    for strat in (1, 2, 3, 5, 6):
        s = EdgeSolver(np.zeros((0, 2), np.int32), np.zeros((0, 3)), np.zeros((0, 3)),
                       np.ones(N), q)
        s.set_strategy(gpu_lib.LOOP_FLUX2, 0, strat)
        s.t["R"].fill_(7.0)
        s.residual(2)
        assert np.all(s.fetch_nodes("R") == 0.0)
        s.close()


def test_spectral_radius_time_step_and_rk_step(gpu_lib, mesh16):
    m, q = mesh16
    s = make_solver(gpu_lib, m, q, renumber="rcm")
    s.time_step(0.5)
    lam = oracle.spectral_radius(m.edge, q, m.normal)
    np.testing.assert_allclose(s.fetch_nodes("lam_s")[:, 0], lam, rtol=1e-13)
    np.testing.assert_allclose(s.fetch_nodes("dt")[:, 0],
                               oracle.time_step(m.volume, lam, 0.5), rtol=1e-13)
    s.step(order=2)
    qo, st = oracle.march(2, 1, m.edge, q, m.normal, m.dx, m.volume)
    assert st == 0
    qg = s.fetch_nodes("q")
    assert np.max(np.abs(qg - qo) / np.max(np.abs(qo), axis=0)) <= 1e-12
    s.close()


def test_march_ten_steps(gpu_lib):
    m = meshgen.lattice(8)
    q = meshgen.flow_state(m)
    s = make_solver(gpu_lib, m, q, renumber="rcm")
    s.set_strategy(gpu_lib.LOOP_FLUX2, 0, 2, 128, 256, 1)
    s.time_step(0.5)
    for _ in range(10):
        s.step(order=2)
    qo, st = oracle.march(2, 10, m.edge, q, m.normal, m.dx, m.volume)
    assert st == 0
    qg = s.fetch_nodes("q")
    assert np.max(np.abs(qg - qo) / np.max(np.abs(qo), axis=0)) <= 1e-11
    s.close()


@pytest.mark.parametrize("strat", [1, 2, 3, 5, 6, 7])
def test_mixed_precision_residual_error(gpu_lib, mesh16, ref16, strat):
    m, q = mesh16
    s = make_solver(gpu_lib, m, q, mixed=True, renumber="rcm")
    for loop in (gpu_lib.LOOP_GREEN_GAUSS, gpu_lib.LOOP_FLUX2, gpu_lib.LOOP_FLUX1):
        s.set_strategy(loop, 1, strat, 256, 512, 1)
    s.residual(2, mixed=True)
    R = s.fetch_nodes("R")
    err = np.max(np.abs(R - ref16["R2"]), axis=0) / np.max(np.abs(ref16["R2"]), axis=0)
    assert np.all(err <= 1e-5), err
    assert np.max(err) > 0.0  # really computed in FP32
    s.flux(1, mixed=True)
    R = s.fetch_nodes("R")
    err = np.max(np.abs(R - ref16["R1"]), axis=0) / np.max(np.abs(ref16["R1"]), axis=0)
    assert np.all(err <= 1e-5), err
    s.close()


def test_mixed_precision_march(gpu_lib):
    m = meshgen.lattice(8)
    q = meshgen.flow_state(m)
    s = make_solver(gpu_lib, m, q, mixed=True, renumber="rcm")
    s.time_step(0.5)
    for _ in range(10):
        s.step(order=2, mixed=True)
    qo, st = oracle.march(2, 10, m.edge, q, m.normal, m.dx, m.volume)
    qg = s.fetch_nodes("q")
    err = np.max(np.abs(qg - qo), axis=0) / np.max(np.abs(qo), axis=0)
    assert np.all(err <= 1e-5), err
    s.close()


def _adj_ok(gpu, ref):
    """Adjoint bar: normwise per component (max |diff| / max |ref|) <= 1e-12,
    and per entry relative to its own size plus the component's median
    <= 1e-11 (the oracle's own result moves by ~2e-12 in that measure when
    only its summation order changes)."""
    nw = np.max(np.abs(gpu - ref), axis=0) / np.max(np.abs(ref), axis=0)
    med = np.median(np.abs(ref), axis=0)
    ew = np.max(np.abs(gpu - ref) / (np.abs(ref) + med))
    return bool(np.all(nw <= TOL) and ew <= 10 * TOL)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("strat", [1, 2, 3, 5, 6])
def test_adjoint_matches_oracle_reverse(gpu_lib, mesh16, order, strat):
    m, q = mesh16
    lam = meshgen.adjoint_seed(m.num_nodes)
    s = make_solver(gpu_lib, m, q, adjoint=True, renumber="rcm")
    for loop in (gpu_lib.LOOP_FLUX1_ADJ, gpu_lib.LOOP_FLUX2_ADJ, gpu_lib.LOOP_GG_ADJ):
        s.set_strategy(loop, 0, strat, 128, 256, 1)
    s.load_nodes("lam", lam)
    s.adjoint(order)
    qb, nb = oracle.residual_reverse(order, m.edge, q, m.normal, m.dx, m.volume, lam)
    assert _adj_ok(s.fetch_nodes("qbar"), qb)
    assert _adj_ok(s.fetch_edges("nbar"), nb)
    s.close()


def test_autograd_backward_and_dot_product(gpu_lib):
    import torch
    from paper_1403_7209_gb300.autograd import residual
    m = meshgen.lattice(8)
    q = meshgen.flow_state(m)
    lam = meshgen.adjoint_seed(m.num_nodes)
    s = make_solver(gpu_lib, m, q, adjoint=True)
    qt = s.t["q"].clone().requires_grad_(True)
    nt = s.t["n"].clone().requires_grad_(True)
    R = residual(s, qt, nt, 2)
    Ro, _ = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume)
    np.testing.assert_allclose(R.detach().cpu().numpy().T, Ro, rtol=1e-11, atol=1e-12)
    lt = torch.from_numpy(np.ascontiguousarray(lam.T)).cuda()
    (R * lt).sum().backward()
    qb, nb = oracle.residual_reverse(2, m.edge, q, m.normal, m.dx, m.volume, lam)
    assert _adj_ok(qt.grad.cpu().numpy().T, qb)
    assert _adj_ok(nt.grad.cpu().numpy().T, nb)
    # dot-product test: <lam, J v> from the oracle's tangent sweep against
    # <J^T lam, v> from the GPU reverse sweep
    qd = meshgen.adjoint_seed(m.num_nodes, stream=meshgen.STREAM_V)
    nd = meshgen.normal(0, meshgen.STREAM_V, np.arange(3 * m.num_edges, dtype=np.uint64)).reshape(-1, 3)
    Rd = oracle.residual_tangent(2, m.edge, q, m.normal, m.dx, m.volume, qd, nd)
    lhs = np.sum(lam * Rd)
    rhs = np.sum(qt.grad.cpu().numpy().T * qd) + np.sum(nt.grad.cpu().numpy().T * nd)
    assert abs(lhs - rhs) <= 1e-12 * (np.sum(np.abs(lam * Rd)))
    s.close()


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("strat", [1, 2, 3, 5, 6])
def test_tangent_matches_oracle_and_reverse(gpu_lib, mesh16, order, strat):
    m, q = mesh16
    qd = meshgen.adjoint_seed(m.num_nodes, stream=meshgen.STREAM_V)
    nd = meshgen.normal(0, meshgen.STREAM_V, np.arange(3 * m.num_edges, dtype=np.uint64)).reshape(-1, 3)
    lam = meshgen.adjoint_seed(m.num_nodes)
    s = make_solver(gpu_lib, m, q, adjoint=True, renumber="rcm")
    for loop in range(gpu_lib.NUM_LOOPS):
        s.set_strategy(loop, 0, strat, 128, 256, 1)
    s.load_nodes("qd", qd)
    s.load_edges("nd", nd)
    s.tangent(order)
    Rd = s.fetch_nodes("Rd")
    ref = oracle.residual_tangent(order, m.edge, q, m.normal, m.dx, m.volume, qd, nd)
    assert _adj_ok(Rd, ref)
    # dot-product test on the GPU: <lam, J v> = <J^T lam, v>
    s.load_nodes("lam", lam)
    s.adjoint(order)
    qb, nb = s.fetch_nodes("qbar"), s.fetch_edges("nbar")
    lhs, rhs = np.sum(lam * Rd), np.sum(qb * qd) + np.sum(nb * nd)
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(lam * Rd))
    s.close()


def test_forward_mode_autograd_runs_the_tangent_loops(gpu_lib):
    import torch
    import torch.autograd.forward_ad as fwAD
    from paper_1403_7209_gb300.autograd import residual
    m = meshgen.lattice(8)
    q = meshgen.flow_state(m)
    s = make_solver(gpu_lib, m, q, adjoint=True)
    qd = meshgen.adjoint_seed(m.num_nodes, stream=meshgen.STREAM_V)
    nd = meshgen.normal(0, meshgen.STREAM_V, np.arange(3 * m.num_edges, dtype=np.uint64)).reshape(-1, 3)
    qt, nt = s.t["q"].clone(), s.t["n"].clone()
    qdt = torch.from_numpy(np.ascontiguousarray(qd.T)).cuda()
    ndt = torch.from_numpy(np.ascontiguousarray(nd.T)).cuda()
    with fwAD.dual_level():
        R = residual(s, fwAD.make_dual(qt, qdt), fwAD.make_dual(nt, ndt), 2)
        Rd = fwAD.unpack_dual(R).tangent
    ref = oracle.residual_tangent(2, m.edge, q, m.normal, m.dx, m.volume, qd, nd)
    assert _adj_ok(Rd.cpu().numpy().T, ref)
    s.close()


def test_autotuner_picks_and_persists(gpu_lib, mesh16, ref16, tmp_path):
    m, q = mesh16
    s = make_solver(gpu_lib, m, q, renumber="rcm")
    for loop in (gpu_lib.LOOP_GREEN_GAUSS, gpu_lib.LOOP_FLUX2):
        s.set_strategy(loop, 0, gpu_lib.STRAT_AUTO)
    s.residual(2)
    assert rel_err(s.fetch_nodes("R"), ref16["R2"], ref16["R2a"]) <= TOL
    st = s.plan_stats(gpu_lib.LOOP_FLUX2)
    assert st["strategy"] in (1, 2, 3) and st["tuned_ms"] > 0
    assert st["ncolours"] >= 2 and st["nblocks"] >= 1
    path = str(tmp_path / "tune.json")
    gpu_lib.op2b_save_tuning(s.ctx, path)
    s2 = make_solver(gpu_lib, m, q, renumber="rcm")
    gpu_lib.op2b_load_tuning(s2.ctx, path)
    s2.set_strategy(gpu_lib.LOOP_FLUX2, 0, gpu_lib.STRAT_AUTO)
    s2.set_strategy(gpu_lib.LOOP_GREEN_GAUSS, 0, gpu_lib.STRAT_AUTO)
    n0 = s2.launch_count()
    s2.residual(2)
    assert s2.plan_stats(gpu_lib.LOOP_FLUX2)["strategy"] == st["strategy"]
    assert s2.launch_count() - n0 <= 64  # table hit: no candidate timing
    s.close()
    s2.close()


@pytest.mark.parametrize("strat", [2, 3])
def test_deterministic_strategies_are_bitwise_reproducible(gpu_lib, mesh16, strat):
    import torch
    m, q = mesh16
    s = make_solver(gpu_lib, m, q, renumber="rcm", adjoint=True)
    for loop in range(gpu_lib.NUM_LOOPS):
        s.set_strategy(loop, 0, strat, 128, 256, 1)
    s.load_nodes("lam", meshgen.adjoint_seed(m.num_nodes))
    outs = []
    for _ in range(3):
        s.residual(2)
        s.adjoint(2)
        torch.cuda.synchronize()
        outs.append((s.t["R"].clone(), s.t["qbar"].clone(), s.t["nbar"].clone()))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)
    s.set_strategy(gpu_lib.LOOP_FLUX2, 0, gpu_lib.STRAT_AUTO_DET)
    s.residual(2)
    assert s.plan_stats(gpu_lib.LOOP_FLUX2)["strategy"] in (2, 3)
    s.close()


def test_global_reductions_match_oracle_and_repeat_bitwise(gpu_lib, mesh16, ref16):
    import torch
    m, q = mesh16
    s = make_solver(gpu_lib, m, q, renumber="rcm")
    s.residual(2)
    s.time_step(0.5)
    R = s.fetch_nodes("R")
    dt = s.fetch_nodes("dt")
    for op in (gpu_lib.RED_SUM, gpu_lib.RED_L2, gpu_lib.RED_MAXABS, gpu_lib.RED_MIN):
        got = s.reduce("R", op)
        again = s.reduce("R", op)
        torch.cuda.synchronize()
        assert torch.equal(got, again)
        ref = oracle.reduce(R, op)
        if op == gpu_lib.RED_SUM:  # cancellation: scale by the absolute sum
            assert np.all(np.abs(got.cpu().numpy() - ref) <= 1e-13 * np.sum(np.abs(R), axis=0))
        else:
            np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=1e-14)
    np.testing.assert_array_equal(s.reduce("dt", gpu_lib.RED_MIN).cpu().numpy(),
                                  oracle.reduce(dt, 3))
    s.close()


def test_autotuner_deadline_reports_timeout(gpu_lib, mesh16):
    m, q = mesh16
    s = make_solver(gpu_lib, m, q)
    gpu_lib.op2b_set_tune_deadline(s.ctx, 1e-6)
    s.set_strategy(gpu_lib.LOOP_FLUX2, 0, gpu_lib.STRAT_AUTO)
    with pytest.raises(gpu_lib.Op2bError) as ei:
        s.residual(2)
    assert ei.value.code in (gpu_lib.ETIMEOUT,)
    s.close()


def test_argument_validation(gpu_lib, mesh16):
    m, q = mesh16
    s = make_solver(gpu_lib, m, q, mixed=True)
    L, d, mp = gpu_lib, s.d, s.map
    c = s.ctx
    bad_dim = [(d["q"], 0, mp, L.READ), (d["q"], 1, mp, L.READ), (d["n"], -1, L.ID, L.READ),
               (d["R"], 0, mp, L.INC), (d["R"], 1, mp, L.INC)]
    with pytest.raises(L.Op2bError) as e:
        L.op2b_green_gauss(c, bad_dim)
    assert e.value.code == L.EDIM
    bad_acc = list(s.a_f1)
    bad_acc[2] = (d["n"], -1, L.ID, L.INC)
    with pytest.raises(L.Op2bError) as e:
        L.op2b_edge_flux(c, bad_acc, 1)
    assert e.value.code == L.EACCESS
    bad_set = list(s.a_f1)
    bad_set[2] = (d["q"], -1, L.ID, L.READ)
    with pytest.raises(L.Op2bError) as e:
        L.op2b_edge_flux(c, bad_set, 1)
    assert e.value.code in (L.ESET, L.EDIM)
    bad_type = list(s.a_f1)
    bad_type[2] = (d["n32"], -1, L.ID, L.READ)
    with pytest.raises(L.Op2bError) as e:
        L.op2b_edge_flux(c, bad_type, 1)
    assert e.value.code == L.ETYPE
    with pytest.raises(L.Op2bError) as e:
        L.op2b_edge_flux(c, s.a_f1, 3)
    assert e.value.code == L.EINVAL
    s.close()


@pytest.mark.parametrize("renumber", ["none", "rcm"])
def test_irregular_graph_all_strategies(gpu_lib, renumber):
    """Uneven degrees (0 to ~30), isolated nodes, repeated pairs, both
    orientations: every strategy against the oracle, forward and adjoint."""
    m = meshgen.random_graph_mesh(3000, seed=4)
    q = meshgen.flow_state(m, seed=4)
    lam = meshgen.adjoint_seed(m.num_nodes, seed=4)
    R, G, Ra = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    R1, _, R1a = oracle.residual(1, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    qb, nb = oracle.residual_reverse(2, m.edge, q, m.normal, m.dx, m.volume, lam)
    s = make_solver(gpu_lib, m, q, renumber=renumber, adjoint=True, mixed=True)
    s.load_nodes("lam", lam)
    for strat, block, part, staged in ((1, 128, 0, 0), (2, 128, 256, 1), (2, 256, 1024, 0),
                                       (3, 128, 0, 0), (5, 128, 512, 1), (6, 128, 0, 0)):
        for loop in range(gpu_lib.NUM_LOOPS):
            # the adjoint keeps 48 values per edge: at most 256-edge blocks
            # fit in shared memory (larger ones give ERANGE)
            lp = min(part, 256) if loop in (gpu_lib.LOOP_FLUX1_ADJ, gpu_lib.LOOP_FLUX2_ADJ) else part
            for prec in (0, 1):
                s.set_strategy(loop, prec, strat, block, lp, staged)
        s.residual(2)
        assert rel_err(s.fetch_nodes("R"), R, Ra) <= TOL, strat
        s.flux(1)
        assert rel_err(s.fetch_nodes("R"), R1, R1a) <= TOL, strat
        s.adjoint(2)
        assert _adj_ok(s.fetch_nodes("qbar"), qb), strat
        assert _adj_ok(s.fetch_edges("nbar"), nb), strat
        s.sync_shadow()
        s.residual(2, mixed=True)
        err = np.max(np.abs(s.fetch_nodes("R") - R), axis=0) / np.max(np.abs(R), axis=0)
        assert np.all(err <= 1e-5), (strat, err)
    s.close()


def test_stream_switch_orders_work_after_the_old_stream(gpu_lib, mesh16, ref16):
    """op2b_set_stream between loops that share the context's scratch: the
    first-order flux runs on stream a, the second-order residual on stream
    b, whose segmented Green-Gauss loop grows the scratch buffer (10 instead
    of 6 values per edge) while a's result is still being copied out."""
    import torch
    m, q = mesh16
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    s = make_solver(gpu_lib, m, q, stream=a)
    for loop in (gpu_lib.LOOP_FLUX1, gpu_lib.LOOP_GREEN_GAUSS, gpu_lib.LOOP_FLUX2):
        s.set_strategy(loop, 0, gpu_lib.STRAT_SEGMENTED, 256)
    torch.cuda.synchronize()
    with torch.cuda.stream(a):
        s.flux(1)
        R1 = s.t["R"].clone()
    gpu_lib.op2b_set_stream(s.ctx, b.cuda_stream)
    with torch.cuda.stream(b):
        s.residual(2)
    torch.cuda.synchronize()
    R1 = R1[:, :s.N].cpu().numpy().T
    assert rel_err(R1, ref16["R1"], ref16["R1a"]) <= TOL
    assert rel_err(s.fetch_nodes("R"), ref16["R2"], ref16["R2a"]) <= TOL
    assert rel_err(s.fetch_nodes("G"), ref16["G"], ref16["Gabs"]) <= TOL
    s.close()
