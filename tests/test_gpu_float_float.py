"""Float-float path against the FP64 oracle, through the C ABI.

The float-float flux does its arithmetic on the FP32 units with about 47
significant bits; the bar is the FP64 one: 1e-12 relative to the sum of the
absolute edge contributions per node and component (the oracle's Rabs),
1e-11 normwise after a 10-step march, on the same inputs as the FP64
parity tests.  The double -> float-float conversion is checked against its
definition (hi = the top 24 significant bits, lo = the rest rounded to a
float) computed with numpy bit operations.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12
STRATS = [("atomic", 1, 256, 0, 0), ("colour", 2, 256, 512, 0),
          ("colour_staged", 2, 128, 256, 1), ("segmented", 3, 256, 0, 0),
          ("block_atomic", 5, 256, 1024, 0), ("owner", 6, 128, 0, 0), ("gather", 7, 128, 0, 0)]


def rel_err(gpu, ref, scale):
    return float(np.max(np.abs(gpu - ref) / (scale + 1e-300)))


def make_solver(m, q, renumber="none", **kw):
    from paper_1403_7209_gb300.solver import EdgeSolver
    return EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, renumber=renumber, ff=True, **kw)


@pytest.fixture(scope="module")
def mesh16():
    m = meshgen.lattice(16)
    q = meshgen.flow_state(m)
    R2, G, R2a = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    return m, q, dict(R2=R2, R2a=R2a, G=G)


def ff_split_reference(x):
    """hi = x truncated to 24 significant bits, lo = the rest of x rounded
    to the nearest float, for normal x with 2^-75 <= |x| < 2^128."""
    b = x.view(np.uint64)
    hi = (b & ~np.uint64((1 << 29) - 1)).view(np.float64)
    rest = x - hi  # exact: the low 29 fraction bits
    return hi.astype(np.float32), rest.astype(np.float32)


def test_conversion_to_float_float(gpu_lib):
    import torch
    rng = np.random.default_rng(7)
    n = 4096
    x = rng.uniform(1, 2, n) * np.exp2(rng.integers(-75, 127, n)) * rng.choice([-1, 1], n)
    x[:6] = [1.0, -0.1, 1.0 / 3.0, 2.0 ** -75 * 1.5, -(2.0 ** 127) * 1.75, np.nextafter(2.0, 0)]
    ctx = gpu_lib.op2b_init(0, torch.cuda.current_stream().cuda_stream)
    st = gpu_lib.op2b_decl_set(ctx, n, "s")
    a = torch.tensor(x, dtype=torch.float64, device="cuda").reshape(1, n)
    f = torch.zeros((1, n, 2), dtype=torch.float32, device="cuda")
    b = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    da = gpu_lib.op2b_decl_dat(ctx, st, 1, gpu_lib.F64, a.data_ptr(), n, "a")
    df = gpu_lib.op2b_decl_dat(ctx, st, 1, gpu_lib.FF, f.data_ptr(), n, "f")
    db = gpu_lib.op2b_decl_dat(ctx, st, 1, gpu_lib.F64, b.data_ptr(), n, "b")
    gpu_lib.op2b_dat_copy(ctx, df, da)
    gpu_lib.op2b_dat_copy(ctx, db, df)
    torch.cuda.synchronize()
    hi, lo = f[0, :, 0].cpu().numpy(), f[0, :, 1].cpu().numpy()
    rh, rl = ff_split_reference(x)
    assert np.array_equal(hi, rh) and np.array_equal(lo, rl)
    back = b[0].cpu().numpy()
    assert np.all(np.abs(back - x) <= np.exp2(-48) * np.abs(x))
    assert back[0] == 1.0 and hi[0] == 1.0 and lo[0] == 0.0
    # zero, values below the float range, and infinities
    a.copy_(torch.tensor([0.0, -0.0, 1e-40, -1e-35, 1e300, -1e300] + [0.0] * (n - 6),
                         dtype=torch.float64, device="cuda").reshape(1, n))
    gpu_lib.op2b_dat_copy(ctx, df, da)
    torch.cuda.synchronize()
    h6 = f[0, :6, 0].cpu().numpy()
    l6 = f[0, :6, 1].cpu().numpy()
    assert np.all(l6[[0, 1, 2, 4, 5]] == 0.0)
    assert h6[0] == 0.0 and h6[1] == 0.0 and np.signbit(h6[1]) and h6[2] == 0.0
    # -1e-35: hi keeps 24 bits, lo the rest down to the float subnormal step
    assert abs(float(h6[3]) + float(l6[3]) + 1e-35) <= 2.0 ** -149
    assert np.isinf(h6[4]) and h6[4] > 0 and np.isinf(h6[5]) and h6[5] < 0
    gpu_lib.op2b_finalize(ctx)


@pytest.mark.parametrize("name,strat,block,part,staged", STRATS)
def test_float_float_flux2_matches_oracle(gpu_lib, mesh16, name, strat, block, part, staged):
    m, q, ref = mesh16
    s = make_solver(m, q)
    s.set_strategy(gpu_lib.LOOP_FLUX2, gpu_lib.PREC_FF, strat, block, part, staged)
    s.load_nodes("G", ref["G"])
    s.sync_shadow(ff=True)
    import paper_1403_7209_gb300.op2b as L
    L.op2b_dat_copy(s.ctx, s.d["G_ff"], s.d["G"])
    s.flux(2, ff=True)
    assert rel_err(s.fetch_nodes("R"), ref["R2"], ref["R2a"]) <= TOL
    s.close()


@pytest.mark.parametrize("renumber", ["none", "rcm"])
def test_float_float_green_gauss_matches_oracle(gpu_lib, mesh16, renumber):
    import paper_1403_7209_gb300.op2b as L
    m, q, ref = mesh16
    Graw, Gabs = oracle.green_gauss(m.edge, q, m.normal, with_abs=True)
    s = make_solver(m, q, renumber=renumber)
    L.op2b_green_gauss(s.ctx, s.a_gg_ff, L.ZERO_INC)
    g1 = s.fetch_nodes("G_ff")
    assert rel_err(g1, Graw, Gabs) <= TOL
    L.op2b_green_gauss(s.ctx, s.a_gg_ff, L.ZERO_INC)
    assert np.array_equal(s.fetch_nodes("G_ff"), g1)  # a gather: fixed order, same bits
    L.op2b_green_gauss(s.ctx, s.a_gg_ff, 0)  # without ZERO_INC the sums are added
    assert rel_err(s.fetch_nodes("G_ff"), 2 * Graw, 2 * Gabs) <= TOL
    s.green_gauss(ff=True)  # sums, then the float-float scaling by 1/V
    assert rel_err(s.fetch_nodes("G_ff"), ref["G"], Gabs / m.volume[:, None]) <= TOL
    s.close()


def test_float_float_residual_differs_from_fp64_only_at_rounding_level(gpu_lib, mesh16):
    m, q, ref = mesh16
    s = make_solver(m, q, renumber="rcm")
    s.set_strategy(gpu_lib.LOOP_FLUX2, gpu_lib.PREC_FF, 3, 256)  # segmented: fixed order
    s.set_strategy(gpu_lib.LOOP_FLUX2, gpu_lib.PREC_F64, 3, 256)
    s.residual(2, ff=True)
    Rff = s.fetch_nodes("R")
    s.residual(2)
    R64 = s.fetch_nodes("R")
    assert rel_err(Rff, ref["R2"], ref["R2a"]) <= TOL
    d = rel_err(Rff, R64, ref["R2a"])
    assert 0.0 < d <= TOL  # computed differently, FP64-class agreement
    s.close()


def test_float_float_march(gpu_lib):
    m = meshgen.lattice(8)
    q = meshgen.flow_state(m)
    s = make_solver(m, q, renumber="rcm")
    s.time_step(0.5)
    s.sync_shadow(ff=True)
    for _ in range(10):
        s.step(order=2, ff=True)
    qo, st = oracle.march(2, 10, m.edge, q, m.normal, m.dx, m.volume)
    assert st == 0
    qg = s.fetch_nodes("q")
    assert np.max(np.abs(qg - qo) / np.max(np.abs(qo), axis=0)) <= 1e-11
    s.close()


def test_float_float_full_size(gpu_lib):
    # the benchmark's mesh (100^3 lattice, 9M edges), RCM numbering, the
    # autotuned strategy of the float-float flux, every node against the oracle
    m = meshgen.lattice(100)
    q = meshgen.flow_state(m)
    s = make_solver(m, q, renumber="rcm")
    s.set_strategy(gpu_lib.LOOP_GREEN_GAUSS, 0, gpu_lib.STRAT_AUTO)
    s.set_strategy(gpu_lib.LOOP_FLUX2, gpu_lib.PREC_FF, gpu_lib.STRAT_AUTO)
    s.residual(2, ff=True)
    R = s.fetch_nodes("R")
    Ro, _, Ra = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    assert rel_err(R, Ro, Ra) <= TOL
    s.close()


def test_other_loops_reject_float_float_dats(gpu_lib, mesh16):
    m, q, ref = mesh16
    s = make_solver(m, q)
    import paper_1403_7209_gb300.op2b as L
    d = s.d
    args = [(d["q_ff"], 0, s.map, L.READ), (d["q_ff"], 1, s.map, L.READ), (d["n_ff"], -1, L.ID, L.READ),
            (d["R"], 0, s.map, L.INC), (d["R"], 1, s.map, L.INC)]
    with pytest.raises(L.Op2bError) as e:
        L.op2b_edge_flux(s.ctx, args, 1)
    assert e.value.code == L.ETYPE
    with pytest.raises(L.Op2bError) as e:
        L.op2b_grad_scale_adjoint(s.ctx, d["G_ff"], d["V"])
    assert e.value.code == L.ETYPE
    s.close()


# ------------------------------------------------------- viscous flux
VISC = (2.0e-3, 0.72, 1.5e-3)


@pytest.fixture(scope="module")
def visc16(mesh16):
    m, q, ref = mesh16
    mu, pr, diff = VISC
    Rv, Rva = oracle.viscous(m.edge, q, ref["G"], m.normal, m.dx, 1.4, mu, pr, diff, with_abs=True)
    Gr = np.random.default_rng(5).normal(scale=0.3, size=ref["G"].shape)
    Rr, Rra = oracle.viscous(m.edge, q, Gr, m.normal, m.dx, 1.4, mu, pr, diff, with_abs=True)
    return dict(Rv=Rv, Rva=Rva, Gr=Gr, Rr=Rr, Rra=Rra)


@pytest.mark.parametrize("strat,block,part,staged", [(1, 256, 0, 0), (2, 128, 256, 1),
                                                      (3, 256, 0, 0), (6, 128, 0, 0)])
def test_float_float_viscous_matches_oracle(gpu_lib, mesh16, visc16, strat, block, part, staged):
    import paper_1403_7209_gb300.op2b as L
    m, q, ref = mesh16
    s = make_solver(m, q, renumber="rcm", viscous=VISC)
    s.set_strategy(gpu_lib.LOOP_VISCOUS, gpu_lib.PREC_FF, strat, block, part, staged)
    for G, R, Ra in ((ref["G"], visc16["Rv"], visc16["Rva"]),
                     (visc16["Gr"], visc16["Rr"], visc16["Rra"])):
        s.load_nodes("G", G)
        L.op2b_dat_copy(s.ctx, s.d["G_ff"], s.d["G"])
        s.viscous_flux(zero=True, ff=True)
        Rg = s.fetch_nodes("R")
        assert np.all(Rg[:, 0] == 0.0)
        assert rel_err(Rg, R, Ra) <= TOL
    s.close()


def test_float_float_navier_stokes_residual(gpu_lib, mesh16, visc16):
    m, q, ref = mesh16
    s = make_solver(m, q, renumber="rcm", viscous=VISC)
    s.residual(2, ff=True)
    assert rel_err(s.fetch_nodes("R"), ref["R2"] + visc16["Rv"], ref["R2a"] + visc16["Rva"]) <= TOL
    s.close()


# ------------------------------------------------------------ adjoint
def _adj_ok(gpu, ref):
    """Float-float adjoint bar: normwise per component (max |diff| / max
    |ref|) <= 5e-12 and per entry relative to its own size plus the
    component's median <= 2e-11.  Five and two times the FP64 adjoint's bar:
    float-float rounds each operation at ~2^-47 of its operands (FP64:
    2^-53), and the reverse sweep's per-edge terms cancel by about two
    orders of magnitude in qbar and nbar (measured: 1.1e-12 normwise, 4e-12
    per entry on this mesh)."""
    nw = np.max(np.abs(gpu - ref), axis=0) / np.max(np.abs(ref), axis=0)
    med = np.median(np.abs(ref), axis=0)
    ew = np.max(np.abs(gpu - ref) / (np.abs(ref) + med))
    return bool(np.all(nw <= 5 * TOL) and ew <= 20 * TOL)


@pytest.mark.parametrize("strat", [1, 2, 3, 5, 6])
def test_float_float_adjoint_matches_oracle_reverse(gpu_lib, mesh16, strat):
    m, q, ref = mesh16
    lam = meshgen.adjoint_seed(m.num_nodes)
    s = make_solver(m, q, renumber="rcm", adjoint=True)
    s.set_strategy(gpu_lib.LOOP_FLUX2_ADJ, gpu_lib.PREC_FF, strat, 128, 256, 1)
    s.set_strategy(gpu_lib.LOOP_GG_ADJ, gpu_lib.PREC_F64, strat, 128, 256, 1)
    s.load_nodes("lam", lam)
    s.adjoint(2, ff=True)
    qb, nb = oracle.residual_reverse(2, m.edge, q, m.normal, m.dx, m.volume, lam)
    assert _adj_ok(s.fetch_nodes("qbar"), qb)
    assert _adj_ok(s.fetch_edges("nbar"), nb)
    s.close()


# ------------------------------------------------------- node limiters
LIMS = [("barth_jespersen", oracle.LIM_BJ, 0.0), ("venkatakrishnan", oracle.LIM_VENKAT, 0.0),
        ("venkatakrishnan", oracle.LIM_VENKAT, 1e-3)]


@pytest.mark.parametrize("name,kind,eps2", LIMS)
def test_float_float_limiter_matches_oracle(gpu_lib, mesh16, name, kind, eps2):
    import paper_1403_7209_gb300.op2b as L
    m, q, ref = mesh16
    lo, hi = oracle.minmax(m.edge, q)
    rng = np.random.default_rng(kind)
    for Gin in (ref["G"], rng.normal(scale=0.5, size=ref["G"].shape)):  # mild, strong limiting
        s = make_solver(m, q, renumber="rcm", limiter=name, limiter_eps2=eps2)
        s.load_nodes("G", Gin)
        L.op2b_dat_copy(s.ctx, s.d["G_ff"], s.d["G"])
        s.node_limiter(ff=True)
        # the extrema of the float-float shadows of q (within 2^-48 of q)
        assert np.all(np.abs(s.fetch_nodes("qmin_ff") - lo) <= 2.0 ** -47 * np.abs(lo))
        assert np.all(np.abs(s.fetch_nodes("qmax_ff") - hi) <= 2.0 ** -47 * np.abs(hi))
        phi = oracle.limiter(kind, m.edge, q, Gin, m.dx, lo, hi, eps2)
        assert np.max(np.abs(s.fetch_nodes("phi_ff") - phi)) <= TOL
        assert np.min(phi) < 0.9  # the limiter is active on this data
        s.close()


@pytest.mark.parametrize("strat", [1, 3, 6, 7])
@pytest.mark.parametrize("name,kind,eps2", LIMS[:2])
def test_float_float_limited_residual_matches_oracle(gpu_lib, mesh16, name, kind, eps2, strat):
    m, q, ref = mesh16
    s = make_solver(m, q, renumber="rcm", limiter=name, limiter_eps2=eps2)
    s.set_strategy(gpu_lib.LOOP_FLUX2_PHI, gpu_lib.PREC_FF, strat, 128)
    s.residual(2, ff=True)
    o = oracle.residual_limited(kind, m.edge, q, m.normal, m.dx, m.volume, eps2, with_abs=True)
    assert rel_err(s.fetch_nodes("R"), o["R"], o["Rabs"]) <= TOL
    s.close()


# ------------------------------------------------------------ tangent
@pytest.mark.parametrize("strat", [1, 3, 6, 7])
def test_float_float_tangent_matches_oracle(gpu_lib, mesh16, strat):
    m, q, ref = mesh16
    qd = meshgen.adjoint_seed(m.num_nodes, stream=meshgen.STREAM_V)
    nd = meshgen.normal(0, meshgen.STREAM_V, np.arange(3 * m.num_edges, dtype=np.uint64)).reshape(-1, 3)
    s = make_solver(m, q, renumber="rcm", adjoint=True)
    s.set_strategy(gpu_lib.LOOP_FLUX2_TAN, gpu_lib.PREC_FF, strat, 128)
    s.load_nodes("qd", qd)
    s.load_edges("nd", nd)
    s.tangent(2, ff=True)
    ref_t = oracle.residual_tangent(2, m.edge, q, m.normal, m.dx, m.volume, qd, nd)
    assert _adj_ok(s.fetch_nodes("Rd"), ref_t)
    # dot-product test against the float-float adjoint: <lam, J v> = <J^T lam, v>
    lam = meshgen.adjoint_seed(m.num_nodes)
    s.load_nodes("lam", lam)
    s.adjoint(2, ff=True)
    Rd = s.fetch_nodes("Rd")
    lhs = np.sum(lam * Rd)
    rhs = np.sum(s.fetch_nodes("qbar") * qd) + np.sum(s.fetch_edges("nbar") * nd)
    assert abs(lhs - rhs) <= 1e-11 * np.sum(np.abs(lam * Rd))
    s.close()


# ------------------------------------------------ irregular and ragged meshes
@pytest.mark.parametrize("limiter", ["van_albada", "barth_jespersen"])
def test_float_float_irregular_and_ragged(gpu_lib, limiter):
    # a random graph (ragged degrees, unsorted ends) and two small lattices
    # (3^3: every node touches itself through the periodic wrap's
    # neighbours twice) under every strategy of the float-float flux
    kind = {"van_albada": None, "barth_jespersen": oracle.LIM_BJ}[limiter]
    for m in (meshgen.random_graph_mesh(3000, seed=8), meshgen.lattice(3, seed=1),
              meshgen.lattice(5, seed=2)):
        q = meshgen.flow_state(m, seed=3)
        if kind is None:
            R, _, Ra = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
        else:
            o = oracle.residual_limited(kind, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
            R, Ra = o["R"], o["Rabs"]
        s = make_solver(m, q, renumber="rcm", limiter=limiter)
        loop = gpu_lib.LOOP_FLUX2 if kind is None else gpu_lib.LOOP_FLUX2_PHI
        for strat, block, part, staged in ((1, 64, 0, 0), (2, 64, 64, 1), (3, 64, 0, 0),
                                           (5, 64, 256, 0), (6, 64, 0, 0), (7, 64, 0, 0)):
            s.set_strategy(loop, gpu_lib.PREC_FF, strat, block, part, staged)
            s.residual(2, ff=True)
            assert rel_err(s.fetch_nodes("R"), R, Ra) <= TOL, (m.num_edges, strat)
        s.close()


def test_float_float_empty_edge_set(gpu_lib):
    # nodes without edges: every float-float loop runs and leaves R zero
    from paper_1403_7209_gb300.solver import EdgeSolver
    q = np.tile([1.0, 0.5, 0.0, 0.0, 2.5, 0.1], (5, 1))
    s = EdgeSolver(np.zeros((0, 2), np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.ones(5), q,
                   ff=True)
    s.load_nodes("R", np.ones((5, 6)))
    s.residual(2, ff=True)
    assert np.all(s.fetch_nodes("R") == 0.0) and np.all(s.fetch_nodes("G_ff") == 0.0)
    s.close()
