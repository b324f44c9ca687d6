"""The fused FP32-mixed stage (op2b_stage_mixed) against the oracle and
against the separate FP32-mixed loops, through the C ABI.

Bars: the mixed path's residual and state bar, 1e-5 normwise per component
(max |x - x_ref| / max |x_ref|) against the FP64 oracle.  Against the
separate FP32 loops the gradients are bitwise equal (same operations in the
same order) and the residuals differ only by the summation of the FP32
fluxes (two-sum pairs here, FP64 additions there) and the atomics' order:
a few FP32 roundings of the largest flux, 1e-6 normwise.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu

BAR = 1e-5


def _normwise(x, ref):
    return np.max(np.abs(x - ref), axis=0) / np.max(np.abs(ref), axis=0)


def _solver(m, q, renumber="rcm", **kw):
    from paper_1403_7209_gb300.solver import EdgeSolver
    return EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, renumber=renumber, mixed=True,
                      coords=m.coords, **kw)


@pytest.fixture(scope="module")
def mesh16():
    m = meshgen.lattice(16)
    return m, meshgen.flow_state(m)


@pytest.fixture(scope="module")
def ref16(mesh16):
    m, q = mesh16
    R, G, Ra = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    return R, G, Ra


@pytest.mark.parametrize("staged", [False, True], ids=["direct", "staged"])
@pytest.mark.parametrize("renumber", ["none", "rcm", "rcb"])
def test_fused_residual_and_gradient_match_oracle(gpu_lib, mesh16, ref16, renumber, staged):
    m, q = mesh16
    R_ora, G_ora, Ra = ref16
    s = _solver(m, q, renumber=renumber)
    gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.time_step(0.5)
    s.stage_fused(0.0, gradient=True, staged=staged)  # alpha = 0: q = q0, R and G of q
    R, G = s.fetch_nodes("R"), s.fetch_nodes("G32")
    assert np.all(_normwise(R, R_ora) <= BAR), _normwise(R, R_ora)
    assert np.max(_normwise(R, R_ora)) > 0.0  # computed in FP32
    assert np.all(_normwise(G, G_ora) <= BAR)
    assert np.array_equal(s.fetch_nodes("q"), q)
    # conservation: the two ends of an edge add bitwise opposite fluxes and
    # each node's pair holds its sum to ~2^-48, so sum_i R_i ~ 0
    assert np.all(np.abs(R.sum(axis=0)) <= 1e-12 * Ra.sum(axis=0))
    s.close()


def test_fused_matches_separate_fp32_loops(gpu_lib, mesh16):
    import torch
    m, q = mesh16
    s = _solver(m, q)
    s.set_strategy(gpu_lib.LOOP_GREEN_GAUSS, gpu_lib.PREC_F32, gpu_lib.STRAT_GATHER, 128)
    s.set_strategy(gpu_lib.LOOP_FLUX2, gpu_lib.PREC_F32, gpu_lib.STRAT_OWNER, 128)
    s.time_step(0.5)
    gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.sync_shadow()
    s.residual(2, mixed=True)
    G_sep, R_sep = s.t["G32"].clone(), s.t["R"].clone()
    Rf = {}
    for staged in (True, False):
        s.t["G32"].fill_(float("nan"))
        s.stage_fused(0.0, sync=True, gradient=True, staged=staged)
        torch.cuda.synchronize()
        assert torch.equal(s.t["G32"], G_sep)  # the same FP32 gather, bit for bit
        R = s.t["R"][:, :s.N].cpu().numpy().T
        Rs = R_sep[:, :s.N].cpu().numpy().T
        assert np.all(_normwise(R, Rs) <= 1e-6), _normwise(R, Rs)
        Rf[staged] = R
    # the staged form sums a node's ends in two interleaved halves: the
    # pairs hold each sum to ~2^-48, so the forms agree far below FP32
    assert np.all(_normwise(Rf[False], Rf[True]) <= 1e-12)
    s.close()


def test_fused_stage_update_and_store_q0(gpu_lib, mesh16):
    """q = q0 - alpha (dt/V) R in FP64 from the returned R, and with
    OP2B_STAGE_STORE_Q0 the new state lands in q0 too."""
    m, q = mesh16
    s = _solver(m, q, renumber="none")
    s.time_step(0.5)
    gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.stage_fused(0.375)
    qn, R = s.fetch_nodes("q"), s.fetch_nodes("R")
    dt, V = s.fetch_nodes("dt")[:, 0], m.volume
    expect = q - (0.375 * (dt / V))[:, None] * R
    assert np.max(np.abs(qn - expect) / np.max(np.abs(q), axis=0)) <= 1e-15
    assert np.array_equal(s.fetch_nodes("q0"), q)
    s.stage_fused(0.5, store_q0=True)
    assert np.array_equal(s.fetch_nodes("q0"), s.fetch_nodes("q"))
    s.close()


def test_fused_stage_is_bitwise_reproducible_and_sync_repacks(gpu_lib, mesh16):
    m, q = mesh16
    s = _solver(m, q)
    s.time_step(0.5)
    out = []
    for _ in range(2):
        s.load_nodes("q", q)
        s.step(fused=True)  # the first stage re-packs the records from q
        s.step(fused=True)
        out.append(s.fetch_nodes("q"))
    assert np.array_equal(out[0], out[1])
    # without the re-pack the records still hold the previous state: a
    # stage then starts from it, not from the reloaded q
    s.load_nodes("q", q)
    gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.stage_fused(0.25)
    stale = s.fetch_nodes("R")
    s.load_nodes("q", q)
    gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.stage_fused(0.25, sync=True)
    fresh = s.fetch_nodes("R")
    assert not np.array_equal(stale, fresh)
    s.close()


@pytest.mark.parametrize("staged", [False, True], ids=["direct", "staged"])
def test_fused_march_within_bar_of_oracle(gpu_lib, staged):
    m = meshgen.lattice(8)
    q = meshgen.flow_state(m)
    s = _solver(m, q)
    s.time_step(0.5)
    for _ in range(10):
        s.step(fused=True, staged=staged)
    qo, st = oracle.march(2, 10, m.edge, q, m.normal, m.dx, m.volume)
    assert st == 0
    assert np.all(_normwise(s.fetch_nodes("q"), qo) <= BAR)
    s.close()


@pytest.mark.parametrize("staged", [False, True], ids=["direct", "staged"])
@pytest.mark.parametrize("n", [3, 5, 7, 11])
def test_fused_ragged_lattices(gpu_lib, n, staged):
    """Node counts that fill no block (27, 125, 343, 1331 nodes: the last
    node block is partial), against the oracle."""
    m = meshgen.lattice(n, seed=n)
    q = meshgen.flow_state(m, seed=n)
    R_ora, G_ora, _ = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    s = _solver(m, q, renumber="none")
    gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.time_step(0.5)
    s.stage_fused(0.0, gradient=True, staged=staged)
    assert np.all(_normwise(s.fetch_nodes("R"), R_ora) <= BAR)
    assert np.all(_normwise(s.fetch_nodes("G32"), G_ora) <= BAR)
    s.close()


def test_fused_irregular_graph(gpu_lib):
    """A random graph (node degrees from 0 to ~20, repeated pairs allowed)
    with lattice-like geometry, against the oracle."""
    rng = np.random.default_rng(3)
    N, E = 600, 3000
    edge = rng.integers(0, N, size=(E, 2)).astype(np.int32)
    edge = edge[edge[:, 0] != edge[:, 1]]
    E = edge.shape[0]
    nrm = rng.uniform(-1.0, 1.0, size=(E, 3))
    dx = rng.uniform(-1.0, 1.0, size=(E, 3))
    V = rng.uniform(0.9, 1.1, size=N)
    rho = rng.uniform(0.9, 1.1, size=N)
    u = np.array([0.5, 0.0, 0.0]) + rng.uniform(-0.3, 0.3, size=(N, 3))
    p = rng.uniform(0.9, 1.1, size=N)
    q = np.column_stack([rho, rho[:, None] * u, p / 0.4 + 0.5 * rho * (u * u).sum(1),
                         rng.uniform(0.0, 1e-3, size=N)])
    R_ora, G_ora, _ = oracle.residual(2, edge, q, nrm, dx, V, with_abs=True)
    from paper_1403_7209_gb300.solver import EdgeSolver
    s = EdgeSolver(edge, nrm, dx, V, q, renumber="rcm", mixed=True)
    gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.time_step(0.5)
    for staged in (False, True):
        s.stage_fused(0.0, gradient=True, staged=staged)
        assert np.all(_normwise(s.fetch_nodes("R"), R_ora) <= BAR)
        assert np.all(_normwise(s.fetch_nodes("G32"), G_ora) <= BAR)
    s.close()


@pytest.mark.parametrize("kinds", [("n32", "dx32"), ("n32", "dx"), ("n", "dx32")],
                         ids=["f32_f32", "f32_f64", "f64_f32"])
def test_fused_stage_takes_fp32_geometry(gpu_lib, mesh16, kinds):
    """n and dx given as F32 dats (each the FP32 rounding of the F64 values)
    give bitwise the stage of the F64 dats: the library converts them to
    FP32 either way; switching the geometry dats re-packs the adjacency."""
    m, q = mesh16
    s = _solver(m, q)
    d = s.d
    gpu_lib.op2b_dat_copy(s.ctx, d["q0"], d["q"])
    s.time_step(0.5)

    def stage(n, dx):
        s.load_nodes("q", q)
        gpu_lib.op2b_dat_copy(s.ctx, d["q0"], d["q"])
        gpu_lib.op2b_stage_mixed(s.ctx, s.map, d["q0"], d["q"], d["V"], d["dt"], d[n], d[dx],
                                 d["R"], d["G32"], 0.25, s.gamma, s.eps_lim,
                                 gpu_lib.STAGE_SYNC)
        return s.fetch_nodes("q"), s.fetch_nodes("R"), s.fetch_nodes("G32")

    ref = stage("n", "dx")
    got = stage(*kinds)
    back = stage("n", "dx")
    for a, b, c in zip(ref, got, back):
        assert np.array_equal(a, b)
        assert np.array_equal(a, c)
    s.close()


def test_fused_stage_after_renumbering(gpu_lib, mesh16, ref16):
    """The library renumbers the map (and permutes the declared dats in
    place) after a fused stage has built its records and adjacency: the next
    stage rebuilds them for the new numbering and matches the oracle."""
    from paper_1403_7209_gb300.solver import RENUMBER
    m, q = mesh16
    R_ora, G_ora, _ = ref16
    s = _solver(m, q, renumber="none")
    gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.time_step(0.5)
    s.stage_fused(0.0, sync=True, gradient=True)
    R1 = s.fetch_nodes("R")
    assert np.all(_normwise(R1, R_ora) <= BAR)
    perm, order = gpu_lib.op2b_renumber(s.ctx, s.map, RENUMBER["rcm"], 0, s.N, s.E)
    assert not np.array_equal(perm, np.arange(s.N))
    s.perm, s.order = perm.astype(np.int64), order
    s.stage_fused(0.0, sync=True, gradient=True)
    R2, G2 = s.fetch_nodes("R"), s.fetch_nodes("G32")
    assert np.all(_normwise(R2, R_ora) <= BAR), _normwise(R2, R_ora)
    assert np.all(_normwise(G2, G_ora) <= BAR)
    assert np.array_equal(s.fetch_nodes("q"), q)
    s.close()


def test_fused_march_replayed_from_cuda_graph(gpu_lib, mesh16):
    """A fused step (q0 <- q, five op2b_stage_mixed calls, the first
    re-packing the records) captured once in a CUDA graph and replayed three
    times gives bitwise the state of three eager steps."""
    import torch
    m, q = mesh16
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = _solver(m, q, stream=st)
        s.time_step(0.5)
        s.step(fused=True)  # plans and records built outside the capture
        st.synchronize()
        s.load_nodes("q", q)
        for _ in range(3):
            s.step(fused=True)
        st.synchronize()
        q_eager = s.fetch_nodes("q")
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            s.step(fused=True)
        s.load_nodes("q", q)
        for _ in range(3):
            g.replay()
        st.synchronize()
        q_graph = s.fetch_nodes("q")
    assert not np.array_equal(q_eager, q)
    assert np.array_equal(q_graph, q_eager)
    s.close()


def test_fused_hub_node(gpu_lib):
    """One node joined to every other node plus a ring through the rest
    (degrees N-1+... and 3): the adjacency's 32-node slices differ in width
    by a factor of ~30; against the oracle, in both numberings and both forms."""
    rng = np.random.default_rng(5)
    N = 203
    ring = np.column_stack([np.arange(1, N), np.r_[np.arange(2, N), 1]])
    hub = np.column_stack([np.zeros(N - 1, dtype=np.int64), np.arange(1, N)])
    edge = np.vstack([ring, hub]).astype(np.int32)
    E = edge.shape[0]
    nrm = rng.uniform(-1.0, 1.0, size=(E, 3))
    dx = rng.uniform(-1.0, 1.0, size=(E, 3))
    V = rng.uniform(0.9, 1.1, size=N)
    rho = rng.uniform(0.9, 1.1, size=N)
    u = np.array([0.5, 0.0, 0.0]) + rng.uniform(-0.3, 0.3, size=(N, 3))
    p = rng.uniform(0.9, 1.1, size=N)
    q = np.column_stack([rho, rho[:, None] * u, p / 0.4 + 0.5 * rho * (u * u).sum(1),
                         rng.uniform(0.0, 1e-3, size=N)])
    R_ora, G_ora, _ = oracle.residual(2, edge, q, nrm, dx, V, with_abs=True)
    from paper_1403_7209_gb300.solver import EdgeSolver
    for renumber in ("none", "rcm"):
        s = EdgeSolver(edge, nrm, dx, V, q, renumber=renumber, mixed=True)
        gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
        s.time_step(0.5)
        for staged in (False, True):
            s.stage_fused(0.0, gradient=True, staged=staged)
            assert np.all(_normwise(s.fetch_nodes("R"), R_ora) <= BAR)
            assert np.all(_normwise(s.fetch_nodes("G32"), G_ora) <= BAR)
        s.close()


def test_fused_empty_edge_set(gpu_lib):
    N = 10
    q = np.tile([1.0, 0.5, 0.0, 0.0, 2.5, 0.0], (N, 1))
    from paper_1403_7209_gb300.solver import EdgeSolver
    s = EdgeSolver(np.zeros((0, 2), np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.ones(N), q,
                   mixed=True)
    s.t["dt"].fill_(0.1)
    s.t["R"].fill_(7.0)
    gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.stage_fused(0.5, gradient=True)
    assert np.all(s.fetch_nodes("R") == 0.0)
    assert np.all(s.fetch_nodes("G32") == 0.0)
    assert np.array_equal(s.fetch_nodes("q"), q)
    s.close()


def test_fused_argument_errors(gpu_lib, mesh16):
    m, q = mesh16
    s = _solver(m, q, renumber="none")
    c, d = s.ctx, s.d
    bad = [((s.map, d["q"], d["q"], d["V"], d["dt"], d["n"], d["dx"], -1, -1), gpu_lib.EINVAL),
           ((s.map, d["q0"], d["q"], d["V"], d["dt"], d["n"], d["dx"], d["G"], -1), gpu_lib.EDIM),
           ((s.map, d["q0"], d["q"], d["V"], d["dt"], d["n"], d["dx"], -1, d["G"]), gpu_lib.ETYPE),
           ((s.map, d["q0"], d["q32"], d["V"], d["dt"], d["n"], d["dx"], -1, -1), gpu_lib.ETYPE),
           ((s.map, d["q0"], d["q"], d["V"], d["dt"], d["q"], d["dx"], -1, -1), gpu_lib.ESET)]
    for a, code in bad:
        with pytest.raises(gpu_lib.Op2bError) as e:
            gpu_lib.op2b_stage_mixed(c, *a, 0.25)
        assert e.value.code == code, (a, e.value)
    with pytest.raises(gpu_lib.Op2bError) as e:
        gpu_lib.op2b_stage_mixed(c, s.map, d["q0"], d["q"], d["V"], d["dt"], d["n"], d["dx"], -1,
                                 -1, 0.25, flags=16)
    assert e.value.code == gpu_lib.EINVAL
    s.close()
