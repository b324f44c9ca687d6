"""Float-float path against the FP64 oracle, through the C ABI.

The float-float flux does its arithmetic on the FP32 units with about 47
significant bits; the bar is the FP64 one: 1e-12 relative to the sum of the
absolute edge contributions per node and component (the oracle's Rabs),
1e-11 normwise after a 10-step march, on the same inputs as the FP64
parity tests.  The double -> float-float conversion is checked against its
definition (truncation to 24 + 23 significant bits) computed with numpy
integer operations.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12
STRATS = [("atomic", 1, 256, 0, 0), ("colour", 2, 256, 512, 0),
          ("colour_staged", 2, 128, 256, 1), ("segmented", 3, 256, 0, 0),
          ("block_atomic", 5, 256, 1024, 0), ("owner", 6, 128, 0, 0)]


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
    """hi = x truncated to 24 significant bits, lo = the next 23 bits of x
    (truncated), for normal x with 2^-103 <= |x| < 2^128."""
    b = x.view(np.uint64)
    hi = (b & ~np.uint64((1 << 29) - 1)).view(np.float64)
    rest = x - hi  # exact: the low 29 fraction bits
    _, e = np.frexp(x)  # x = f 2^e, 1/2 <= |f| < 1: unbiased exponent e - 1
    step = np.ldexp(1.0, e - 1 - 46)  # weight of fraction bit 6
    lo = np.trunc(rest / step) * step
    return hi.astype(np.float32), lo.astype(np.float32)


def test_conversion_to_float_float(gpu_lib):
    import torch
    rng = np.random.default_rng(7)
    n = 4096
    x = rng.uniform(1, 2, n) * np.exp2(rng.integers(-100, 120, n)) * rng.choice([-1, 1], n)
    x[:4] = [1.0, -0.1, 1.0 / 3.0, 2.0 ** -100 * 1.5]
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
    assert np.all(np.abs(back - x) <= np.exp2(-46) * np.abs(x))
    assert back[0] == 1.0 and hi[0] == 1.0 and lo[0] == 0.0
    # zero, values below the float range, and infinities
    a.copy_(torch.tensor([0.0, -0.0, 1e-40, -1e-35, 1e300, -1e300] + [0.0] * (n - 6),
                         dtype=torch.float64, device="cuda").reshape(1, n))
    gpu_lib.op2b_dat_copy(ctx, df, da)
    torch.cuda.synchronize()
    h6 = f[0, :6, 0].cpu().numpy()
    l6 = f[0, :6, 1].cpu().numpy()
    assert np.all(l6 == 0.0)
    assert h6[0] == 0.0 and h6[1] == 0.0 and np.signbit(h6[1]) and h6[2] == 0.0
    assert h6[3] == np.float32(-1e-35) or abs(h6[3] + 1e-35) < 1e-41
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
