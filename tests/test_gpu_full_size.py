"""Parity at the benchmark's sizes, with the autotuned strategies.

100^3 lattice (1M nodes, 9M edges): every node of the FP64 residual and of
the adjoint against the oracle; FP32-mixed residual error, by the separate
loops and by the fused stage (both forms).
200^3 lattice (8M nodes, 72M edges): sampled nodes and edges (FP64 residual
and adjoint, fused FP32-mixed residual).  For a sample
S the oracle runs on a local sub-mesh that holds every edge touching the
nodes within two rings of S, which is exactly what R at S and the adjoint
at S (and at edges meeting S) depend on.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel_err(gpu, ref, scale):
    return float(np.max(np.abs(gpu - ref) / (scale + 1e-300)))


def adj_ok(gpu, ref, scale, med):
    """Adjoint bar: max |diff| / max |ref| per component <= 1e-12 (scale =
    the component's max |ref| over the whole field), and per entry
    |diff| / (|ref| + median) <= 1e-11."""
    nw = np.max(np.abs(gpu - ref), axis=0) / scale
    ew = np.max(np.abs(gpu - ref) / (np.abs(ref) + med))
    return bool(np.all(nw <= TOL) and ew <= 10 * TOL)


def tuned_solver(op2b, m, q, **kw):
    from paper_1403_7209_gb300.solver import EdgeSolver
    s = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, renumber="rcm", **kw)
    for loop in range(op2b.NUM_LOOPS):
        for prec in (0, 1):
            s.set_strategy(loop, prec, op2b.STRAT_AUTO)
    return s


def test_lattice100_full_parity(gpu_lib):
    m = meshgen.lattice(100)
    q = meshgen.flow_state(m)
    lam = meshgen.adjoint_seed(m.num_nodes)
    s = tuned_solver(gpu_lib, m, q, mixed=True, adjoint=True)
    s.residual(2)
    R = s.fetch_nodes("R")
    Ro, _, Ra = oracle.residual(2, m.edge, q, m.normal, m.dx, m.volume, with_abs=True)
    assert rel_err(R, Ro, Ra) <= TOL
    s.residual(2, mixed=True)
    R32 = s.fetch_nodes("R")
    err = np.max(np.abs(R32 - Ro), axis=0) / np.max(np.abs(Ro), axis=0)
    assert np.all(err <= 1e-5), err
    # the fused FP32-mixed stage at alpha = 0 (q unchanged): its residual
    import paper_1403_7209_gb300.op2b as L
    L.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.time_step(0.5)
    for staged in (False, True):
        s.stage_fused(0.0, sync=True, staged=staged)
        Rf = s.fetch_nodes("R")
        err = np.max(np.abs(Rf - Ro), axis=0) / np.max(np.abs(Ro), axis=0)
        assert np.all(err <= 1e-5), err
        assert np.array_equal(s.fetch_nodes("q"), q)
    s.load_nodes("lam", lam)
    s.adjoint(2)
    qb, nb = oracle.residual_reverse(2, m.edge, q, m.normal, m.dx, m.volume, lam)
    assert adj_ok(s.fetch_nodes("qbar"), qb, np.max(np.abs(qb), axis=0),
                  np.median(np.abs(qb), axis=0))
    assert adj_ok(s.fetch_edges("nbar"), nb, np.max(np.abs(nb), axis=0),
                  np.median(np.abs(nb), axis=0))
    s.close()


def _submesh(m, sample):
    """Edges touching the two rings around `sample`, relabelled compactly."""
    e = m.edge
    ring = np.zeros(m.num_nodes, dtype=bool)
    ring[sample] = True
    for _ in range(2):
        touch = ring[e[:, 0]] | ring[e[:, 1]]
        ring[e[touch].ravel()] = True
    keep = np.nonzero(ring[e[:, 0]] | ring[e[:, 1]])[0]
    nodes = np.unique(e[keep].ravel())
    local = np.full(m.num_nodes, -1, dtype=np.int64)
    local[nodes] = np.arange(nodes.size)
    return keep, nodes, local


def test_lattice200_sampled_parity(gpu_lib):
    m = meshgen.lattice(200)
    q = meshgen.flow_state(m)
    lam = meshgen.adjoint_seed(m.num_nodes)
    s = tuned_solver(gpu_lib, m, q, adjoint=True, mixed=True)
    s.residual(2)
    R = s.fetch_nodes("R")
    s.load_nodes("lam", lam)
    s.adjoint(2)
    qbar = s.fetch_nodes("qbar")
    nbar = s.fetch_edges("nbar")
    # the fused FP32-mixed stage at alpha = 0 (q unchanged): its residual,
    # as the bench times it (direct form, RCM numbering)
    gpu_lib.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    s.time_step(0.5)
    s.stage_fused(0.0, sync=True)
    Rf = s.fetch_nodes("R")
    assert np.array_equal(s.fetch_nodes("q"), q)
    s.close()
    sample = np.unique(meshgen.fd_picks(200, m.num_nodes, seed=11))
    keep, nodes, local = _submesh(m, sample)
    se = local[m.edge[keep]].astype(np.int32)
    sn, sd, sv, sq = m.normal[keep], m.dx[keep], m.volume[nodes], q[nodes]
    Rs, _, Ras = oracle.residual(2, se, sq, sn, sd, sv, with_abs=True)
    ls = local[sample]
    assert rel_err(R[sample], Rs[ls], Ras[ls]) <= TOL
    # FP32-mixed bar, per component against the field's largest |R|
    err = np.max(np.abs(Rf[sample] - Rs[ls]), axis=0) / np.max(np.abs(R), axis=0)
    assert np.all(err <= 1e-5), err
    qb, nb = oracle.residual_reverse(2, se, sq, sn, sd, sv, lam[nodes])
    assert adj_ok(qbar[sample], qb[ls], np.max(np.abs(qbar), axis=0),
                  np.median(np.abs(qbar), axis=0))
    # edges meeting the sample (their whole dependence lies in the sub-mesh)
    inS = np.zeros(m.num_nodes, dtype=bool)
    inS[sample] = True
    ek = np.nonzero(inS[m.edge[keep, 0]] | inS[m.edge[keep, 1]])[0]
    assert adj_ok(nbar[keep[ek]], nb[ek], np.max(np.abs(nbar), axis=0),
                  np.median(np.abs(nbar), axis=0))


def test_adjoint_fd_and_dot_product_1M(gpu_lib):
    """The adjoint on the 1M-node mesh: central differences of the GPU forward
    residual on 64 entries (h = 1e-6, 1e-8 for the passive scalar,
    Richardson-combined) against the GPU adjoint, and the dot-product test
    <lam, J v> (oracle tangent sweep) = <J^T lam, v> (GPU reverse sweep)."""
    import torch
    m = meshgen.lattice(100)
    q = meshgen.flow_state(m)
    lam = meshgen.adjoint_seed(m.num_nodes)
    s = tuned_solver(gpu_lib, m, q, adjoint=True)
    s.load_nodes("lam", lam)
    s.adjoint(2)
    qbar = s.fetch_nodes("qbar")
    nbar = s.fetch_edges("nbar")
    lam_t = s.t["lam"].clone()
    # the differenced evaluations must sum in a fixed order: with atomics
    # every node's rounding changes between the two evaluations (~1e-15
    # each, ~1e-12 in J), which 1/(2h) would turn into ~1e-6 noise
    for loop in (gpu_lib.LOOP_GREEN_GAUSS, gpu_lib.LOOP_FLUX2):
        s.set_strategy(loop, 0, gpu_lib.STRAT_AUTO_DET)
    h = 1e-6
    # picks whose dependence stays clear of the |u.n| and max() kinks
    margin = oracle.kink_margin(2, m.edge, q, m.normal, m.dx, m.volume)
    kink_nodes = np.zeros(m.num_nodes, dtype=bool)
    kink_nodes[m.edge[margin < 50 * h].ravel()] = True
    bad = kink_nodes.copy()
    bad[m.edge[kink_nodes[m.edge].any(axis=1)].ravel()] = True
    bad_e = kink_nodes[m.edge].any(axis=1)

    def dJ(tensor, row, col, hh):
        base = tensor[row, col].item()
        out = []
        for sgn in (1.0, -1.0):
            tensor[row, col] = base + sgn * hh
            s.residual(2)
            out.append(s.t["R"].clone())
        tensor[row, col] = base
        return float(torch.sum(lam_t * (out[0] - out[1])).item()) / (2 * hh)

    def central(tensor, row, col, hh):
        return (4.0 * dJ(tensor, row, col, hh / 2) - dJ(tensor, row, col, hh)) / 3.0

    picks = [p for p in meshgen.fd_picks(400, 6 * m.num_nodes, seed=4) if not bad[p // 6]][:32]
    assert len(picks) == 32
    for p in picks:
        i, k = p // 6, p % 6
        fd = central(s.t["q"], k, int(s.perm[i]), h if k < 5 else 1e-8)
        assert fd == pytest.approx(qbar[i, k], rel=1e-6, abs=1e-9)
    inv_order = np.empty(m.num_edges, dtype=np.int64)
    inv_order[s.order] = np.arange(m.num_edges)
    picks = [p for p in meshgen.fd_picks(400, 3 * m.num_edges, seed=5) if not bad_e[p // 3]][:32]
    assert len(picks) == 32
    for p in picks:
        e, d = p // 3, p % 3
        fd = central(s.t["n"], d, int(inv_order[e]), h)
        assert fd == pytest.approx(nbar[e, d], rel=1e-6, abs=1e-9)
    # dot-product test against the oracle's tangent sweep
    qd = meshgen.adjoint_seed(m.num_nodes, stream=meshgen.STREAM_V)
    qd[:, 5] *= 1e-2
    nd = meshgen.normal(0, meshgen.STREAM_V, np.arange(3 * m.num_edges, dtype=np.uint64)).reshape(-1, 3)
    Rd = oracle.residual_tangent(2, m.edge, q, m.normal, m.dx, m.volume, qd, nd)
    lhs = float(np.sum(lam * Rd))
    rhs = float(np.sum(qbar * qd) + np.sum(nbar * nd))
    assert abs(lhs - rhs) <= 1e-12 * float(np.sum(np.abs(lam * Rd)))
    s.close()
