"""Viscous flux loop (CUDA, through the C ABI) against the CPU oracle.

The node pass (primitives and half gradients) and the viscous edge loop run
on the GPU from q and G; the oracle evaluates the viscous flux edge by edge
from the same q and G.  Error bar as for the inviscid loops: per node and
component, |difference| / (sum of |edge contributions|) <= 1e-12; the
mixed (FP32-arithmetic) variant, normwise per component, <= 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12
MU, PR, DIFF = 2.0e-3, 0.72, 1.5e-3
VISC = (MU, PR, DIFF)
STRATS = [("atomic", 1, 256, 0, 0), ("atomic128", 1, 128, 0, 0), ("gather", 7, 128, 0, 0),
          ("colour", 2, 256, 512, 0), ("colour_staged", 2, 128, 256, 1),
          ("colour_staged_big", 2, 256, 1024, 1), ("segmented", 3, 256, 0, 0),
          ("block_atomic", 5, 256, 1024, 0), ("block_atomic_staged", 5, 128, 512, 1),
          ("owner", 6, 128, 0, 0)]


def rel_err(gpu, ref, scale):
    return float(np.max(np.abs(gpu - ref) / (scale + 1e-300)))


def make_solver(m, q, **kw):
    from paper_1403_7209_gb300.solver import EdgeSolver
    return EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, viscous=VISC, **kw)


def oracle_visc(m, q, G):
    return oracle.viscous(m.edge, q, G, m.normal, m.dx, 1.4, MU, PR, DIFF, with_abs=True)


@pytest.fixture(scope="module")
def case16():
    m = meshgen.lattice(16)
    q = meshgen.flow_state(m)
    _, G, _ = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    Rv, Rva = oracle_visc(m, q, G)
    # a second, rougher gradient field that exercises every term strongly
    rng = np.random.default_rng(5)
    Gr = rng.normal(scale=0.3, size=G.shape)
    Rr, Rra = oracle_visc(m, q, Gr)
    return m, q, dict(G=G, Rv=Rv, Rva=Rva, Gr=Gr, Rr=Rr, Rra=Rra)


@pytest.mark.parametrize("name,strat,block,part,staged", STRATS)
def test_viscous_loop_matches_oracle(gpu_lib, case16, name, strat, block, part, staged):
    m, q, ref = case16
    s = make_solver(m, q, renumber="rcm")
    s.set_strategy(gpu_lib.LOOP_VISCOUS, 0, strat, block, part, staged)
    for G, R, Ra in ((ref["G"], ref["Rv"], ref["Rva"]), (ref["Gr"], ref["Rr"], ref["Rra"])):
        s.load_nodes("G", G)
        s.viscous_flux(zero=True)
        Rg = s.fetch_nodes("R")
        assert np.all(Rg[:, 0] == 0.0)
        assert rel_err(Rg, R, Ra) <= TOL, name
    s.close()


def test_viscous_adds_onto_the_residual(gpu_lib, case16):
    # without OP2B_ZERO_INC the viscous flux is added to what R holds
    m, q, ref = case16
    s = make_solver(m, q)
    s.load_nodes("G", ref["G"])
    base = np.random.default_rng(1).normal(size=(m.num_nodes, 6))
    s.load_nodes("R", base)
    s.viscous_flux(zero=False)
    # each of a node's 18 additions rounds at the size of the running sum
    # (|base| + the contributions so far): half an ulp of it per addition
    eps = np.finfo(np.float64).eps
    bound = TOL * ref["Rva"] + 9 * eps * (np.abs(base) + ref["Rva"])
    assert np.all(np.abs(s.fetch_nodes("R") - (base + ref["Rv"])) <= bound)
    s.close()


@pytest.mark.parametrize("renumber", ["none", "random", "rcm"])
def test_navier_stokes_residual(gpu_lib, case16, renumber):
    # the whole residual (gradients from the GPU Green-Gauss loop, limited
    # inviscid flux, viscous flux) against the oracle's inviscid residual
    # plus its viscous loop on the oracle's gradients
    m, q, ref = case16
    R2, G, R2a = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    s = make_solver(m, q, renumber=renumber, seed=2)
    s.residual(2)
    assert rel_err(s.fetch_nodes("R"), R2 + ref["Rv"], R2a + ref["Rva"]) <= TOL
    s.close()


@pytest.mark.parametrize("strat", [1, 2, 3, 5, 6])
def test_viscous_mixed_precision(gpu_lib, case16, strat):
    m, q, ref = case16
    s = make_solver(m, q, renumber="rcm", mixed=True)
    s.set_strategy(gpu_lib.LOOP_VISCOUS, 1, strat, 256, 512, 1)
    for G, R in ((ref["G"], ref["Rv"]), (ref["Gr"], ref["Rr"])):
        s.load_nodes("G32", G)
        s.viscous_flux(mixed=True, zero=True)
        Rg = s.fetch_nodes("R")
        assert np.all(Rg[:, 0] == 0.0)
        err = np.max(np.abs(Rg - R)[:, 1:], axis=0) / np.max(np.abs(R)[:, 1:], axis=0)
        assert np.all(err <= 1e-5), err
        assert np.max(err) > 0.0  # really FP32 arithmetic
    s.close()


def test_viscous_deterministic_strategies_reproduce_bitwise(gpu_lib, case16):
    m, q, ref = case16
    s = make_solver(m, q, renumber="rcm")
    s.load_nodes("G", ref["Gr"])
    for strat in (2, 3):
        s.set_strategy(gpu_lib.LOOP_VISCOUS, 0, strat, 256, 512, 1)
        s.viscous_flux(zero=True)
        a = s.t["R"].clone()
        s.viscous_flux(zero=True)
        assert s.torch.equal(a, s.t["R"])
    s.close()


def test_viscous_irregular_graph_and_ragged_meshes(gpu_lib):
    # uneven degrees, isolated nodes, repeated pairs; then E = 243 and 1125
    cases = [meshgen.random_graph_mesh(3000, seed=6), meshgen.lattice(3, seed=1),
             meshgen.lattice(5, seed=1)]
    for m in cases:
        q = meshgen.flow_state(m, seed=1)
        G = np.random.default_rng(2).normal(scale=0.2, size=(m.num_nodes, 18))
        R, Ra = oracle_visc(m, q, G)
        s = make_solver(m, q, renumber="rcm")
        s.load_nodes("G", G)
        for strat, block, part, staged in ((1, 64, 0, 0), (2, 64, 64, 0), (2, 128, 1024, 1),
                                           (2, 256, 4096, 0), (3, 64, 0, 0), (5, 64, 64, 1),
                                           (6, 64, 0, 0)):
            s.set_strategy(gpu_lib.LOOP_VISCOUS, 0, strat, block, part, staged)
            s.viscous_flux(zero=True)
            assert rel_err(s.fetch_nodes("R"), R, Ra) <= TOL, (m.num_edges, strat)
        # 4096-edge blocks with their node data staged need more shared
        # memory than a block has: refused with ERANGE, nothing launched
        s.set_strategy(gpu_lib.LOOP_VISCOUS, 0, 2, 128, 4096, 1)
        if m.num_edges >= 4096:
            with pytest.raises(gpu_lib.Op2bError) as e:
                s.viscous_flux(zero=True)
            assert e.value.code == gpu_lib.ERANGE
        s.close()


def test_viscous_empty_edge_set(gpu_lib):
    from paper_1403_7209_gb300.solver import EdgeSolver
    N = 7
    q = np.tile([1.0, 0.5, 0.0, 0.0, 2.5, 0.1], (N, 1))
    s = EdgeSolver(np.zeros((0, 2), np.int32), np.zeros((0, 3)), np.zeros((0, 3)),
                   np.ones(N), q, viscous=VISC)
    s.load_nodes("R", np.ones((N, 6)))
    s.viscous_flux(zero=True)
    assert np.all(s.fetch_nodes("R") == 0.0)
    s.close()


def test_viscous_argument_checks(gpu_lib, case16):
    L = gpu_lib
    m, q, _ = case16
    s = make_solver(m, q)
    c, d, mp = s.ctx, s.d, s.map
    good = [(d["W"], 0, mp, L.READ), (d["W"], 1, mp, L.READ), (d["n"], -1, L.ID, L.READ),
            (d["dx"], -1, L.ID, L.READ), (d["R"], 0, mp, L.INC), (d["R"], 1, mp, L.INC)]
    L.op2b_viscous_flux(c, good, 1.4, MU, PR, DIFF, L.ZERO_INC)
    bad_dim = [(d["G"], 0, mp, L.READ), (d["G"], 1, mp, L.READ)] + good[2:]
    with pytest.raises(L.Op2bError) as e:
        L.op2b_viscous_flux(c, bad_dim, 1.4, MU, PR, DIFF)
    assert e.value.code == L.EDIM
    with pytest.raises(L.Op2bError) as e:
        L.op2b_viscous_flux(c, good, 1.4, MU, 0.0, DIFF)
    assert e.value.code == L.EINVAL
    with pytest.raises(L.Op2bError) as e:
        L.op2b_viscous_flux(c, good[:5], 1.4, MU, PR, DIFF)
    assert e.value.code == L.EINVAL
    with pytest.raises(L.Op2bError) as e:
        L.op2b_viscous_prims(c, d["q"], d["G"], d["R"], 1.4)
    assert e.value.code == L.EDIM
    s.close()
