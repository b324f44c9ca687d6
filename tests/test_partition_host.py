"""Owner-compute partitions on the host (CPU only): recursive coordinate
bisection, the halo plan's local meshes and import / export lists, and the
distributed exchange protocol those lists define, run as two gloo ranks
whose loops are the oracle's."""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen, op2b
from paper_1403_7209_gb300.partition import halo_plan, halo_stats

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return op2b.load(build_if_missing=True)


def lattice_index(m, n):
    """(a, b, c) lattice position of every node of meshgen.lattice(n)."""
    lat = np.empty(m.num_nodes, dtype=np.int64)
    lat[m.new_of_lattice] = np.arange(m.num_nodes)
    return lat % n, (lat // n) % n, lat // (n * n)


def test_rcb_splits_x_then_y_then_z(lib):
    # Sec. 4: the coordinates are split in x, y and z in turn.  The lattice
    # jitter (0.1) is below half the spacing, so the cuts fall between
    # lattice planes and the parts have a closed form.
    n = 8
    m = meshgen.lattice(n)
    a, b, c = lattice_index(m, n)
    part = op2b.op2b_host_partition_rcb(m.coords, 8)
    assert np.array_equal(part, 4 * (a >= 4) + 2 * (b >= 4) + (c >= 4))
    part2 = op2b.op2b_host_partition_rcb(m.coords, 2)
    assert np.array_equal(part2, (a >= 4).astype(np.int32))


def test_rcb_uneven_part_counts(lib):
    # 3 parts of 6^3 = 216 nodes: the first cut keeps floor(216 * 1/3) = 72
    # nodes (planes a = 0, 1) for part 0, the other 144 are cut in y.
    n = 6
    m = meshgen.lattice(n)
    a, b, c = lattice_index(m, n)
    part = op2b.op2b_host_partition_rcb(m.coords, 3)
    assert np.array_equal(part, np.where(a < 2, 0, 1 + (b >= 3)))
    for P in (1, 5, 7, 13, 216):
        p = op2b.op2b_host_partition_rcb(m.coords, P)
        cnt = np.bincount(p, minlength=P)
        assert cnt.sum() == 216 and cnt.min() >= 1
        assert cnt.max() - cnt.min() <= 1 + int(np.ceil(np.log2(P)))


def test_rcb_rejects_bad_counts(lib):
    xyz = np.zeros((4, 3))
    for P in (0, 5):
        with pytest.raises(op2b.Op2bError) as e:
            op2b.op2b_host_partition_rcb(xyz, P)
        assert e.value.code == op2b.EINVAL


def random_graph(N, E, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(0, N, E)
    b = (a + rng.integers(1, N, E)) % N
    return np.stack([a, b], 1).astype(np.int32)


@pytest.mark.parametrize("N,E,P,seed", [(40, 150, 3, 0), (200, 900, 7, 1), (50, 0, 2, 2),
                                        (30, 80, 1, 3), (64, 300, 64, 4)])
def test_halo_plan_matches_brute_force(lib, N, E, P, seed):
    edge = random_graph(N, E, seed) if E else np.zeros((0, 2), np.int32)
    part = np.random.default_rng(seed + 10).integers(0, P, N).astype(np.int32)
    parts = halo_plan(N, edge, part, P)
    owned_seen = np.zeros(N, dtype=np.int64)
    for p, Pp in enumerate(parts):
        z = Pp["sizes"]
        own = np.nonzero(part == p)[0]
        assert z["owned"] == own.size
        assert np.array_equal(Pp["nodes"][:own.size], own)
        owned_seen[own] += 1
        # local edges: exactly the edges with an owned end, in global order
        mine = np.nonzero((part[edge[:, 0]] == p) | (part[edge[:, 1]] == p))[0] if E else []
        assert np.array_equal(Pp["edges"], mine)
        # the local map names the same global ends, same orientation
        if len(mine):
            assert np.array_equal(Pp["nodes"][Pp["local_map"]], edge[mine])
        # halo: the non-owned ends, grouped by owner, increasing id
        ends = np.unique(edge[mine].ravel()) if len(mine) else np.zeros(0, np.int64)
        halo = ends[part[ends] != p]
        key = np.lexsort((halo, part[halo]))
        assert np.array_equal(Pp["nodes"][own.size:], halo[key])
        assert np.array_equal(Pp["halo_owner"], part[halo[key]])
        for g, r, s in zip(Pp["nodes"][own.size:], Pp["halo_owner"], Pp["halo_src"]):
            assert parts[r]["nodes"][s] == g and s < parts[r]["sizes"]["owned"]
        cut = (part[edge[mine, 0]] != part[edge[mine, 1]]).sum() if len(mine) else 0
        assert z["halo_edges"] == cut
        # exports of p to q = q's import rows owned by p, in q's order
        importers = sorted({q for q, Q in enumerate(parts) if np.any(Q["halo_owner"] == p)})
        assert Pp["nbr"].tolist() == importers
        for k, q in enumerate(Pp["nbr"]):
            Q = parts[q]
            rows = Q["halo_owner"] == p
            blk = Pp["exp_idx"][Pp["exp_off"][k]:Pp["exp_off"][k + 1]]
            assert np.array_equal(blk, Q["halo_src"][rows])
    assert np.all(owned_seen == 1)


def test_halo_plan_rejects_bad_input(lib):
    edge = np.array([[0, 1], [1, 2]], dtype=np.int32)
    with pytest.raises(op2b.Op2bError) as e:
        halo_plan(3, edge, np.array([0, 1, 2], np.int32), 2)
    assert e.value.code == op2b.EINVAL
    with pytest.raises(op2b.Op2bError) as e:
        halo_plan(3, np.array([[0, 3]], np.int32), np.zeros(3, np.int32), 1)
    assert e.value.code == op2b.EINVAL


def test_halo_stats_on_the_lattice(lib):
    # Sec. 4.2 (table of halo sizes): the share of halo elements grows with
    # the number of parts.  Split into octants, a part of the periodic
    # lattice reaches the 6 octants that differ from it in one or two
    # coordinates; the one opposite it in all three would need a
    # body-diagonal edge, which the lattice (axis and face diagonals) lacks.
    m = meshgen.lattice(8)
    s2 = halo_stats(halo_plan(m.num_nodes, m.edge, op2b.op2b_host_partition_rcb(m.coords, 2), 2))
    s8 = halo_stats(halo_plan(m.num_nodes, m.edge, op2b.op2b_host_partition_rcb(m.coords, 8), 8))
    assert s2["avg_neighbours"] == 1 and s8["avg_neighbours"] == 6
    assert s8["avg_halo_percent"] > s2["avg_halo_percent"] > 0


# ------------------------------------------------ distributed protocol
def _exchange(dist, P, rank, x):
    """Refresh the halo rows of x (local rows: owned, then halo) from their
    owners: send every importer its export block, receive one block per
    owner, in the plan's orders."""
    n_own = P["sizes"]["owned"]
    reqs, bufs = [], []
    import torch
    for k, q in enumerate(P["nbr"]):
        blk = x[P["exp_idx"][P["exp_off"][k]:P["exp_off"][k + 1]]]
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(blk)), int(q)))
    for r in np.unique(P["halo_owner"]):
        rows = np.nonzero(P["halo_owner"] == r)[0]
        buf = torch.empty((rows.size,) + x.shape[1:], dtype=torch.float64)
        reqs.append(dist.irecv(buf, int(r)))
        bufs.append((rows, buf))
    for rq in reqs:
        rq.wait()
    for rows, buf in bufs:
        x[n_own + rows] = buf.numpy()


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = meshgen.lattice(5)
    q = meshgen.flow_state(m)
    part = op2b.op2b_host_partition_rcb(m.coords, world)
    P = halo_plan(m.num_nodes, m.edge, part, world)[rank]
    nodes, edges, lmap = P["nodes"], P["edges"], P["local_map"]
    n_own = P["sizes"]["owned"]
    nl, dxl, V = m.normal[edges], m.dx[edges], m.volume[nodes]
    x = q[nodes].copy()
    x[n_own:] = np.nan  # the halo comes only from the exchange
    _exchange(dist, P, rank, x)
    dt = oracle.time_step(V, oracle.spectral_radius(lmap, x, nl), 0.5)
    x0 = x.copy()
    for alpha in (0.25, 1.0 / 6.0, 0.375, 0.5, 1.0):
        _exchange(dist, P, rank, x)
        G = oracle.grad_scale(oracle.green_gauss(lmap, x, nl), V)
        G[n_own:] = np.nan
        _exchange(dist, P, rank, G)
        R = oracle.flux2(lmap, x, G, nl, dxl)
        x[:n_own] = oracle.rk_update(x0, R, V, dt, alpha)[:n_own]
        x[n_own:] = np.nan
    out.put((rank, nodes[:n_own].copy(), x[:n_own].copy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_march_like_the_whole_mesh(lib):
    # One RK step on two owner-compute ranks, halos exchanged by the plan's
    # lists: every owned node sees all its edges in global edge order, so
    # the result equals the whole-mesh oracle march bit for bit.
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    qq = ctx.Queue()
    port = 29613
    procs = [ctx.Process(target=_rank, args=(r, 2, port, qq)) for r in range(2)]
    for p in procs:
        p.start()
    res = [qq.get(timeout=300) for _ in range(2)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    m = meshgen.lattice(5)
    q = meshgen.flow_state(m)
    ref, st = oracle.march(2, 1, m.edge, q, m.normal, m.dx, m.volume)
    assert st == 0
    got = np.full_like(ref, np.nan)
    for _, nodes, vals in res:
        got[nodes] = vals
    assert np.array_equal(got, ref)
