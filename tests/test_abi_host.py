"""The C-ABI library without a GPU: it loads, exports every declared entry
point, and its host-only planners are valid (CPU only)."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen, op2b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return op2b.load(build_if_missing=True)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "op2b.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(op2b_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(op2b.EXPORTED)


def test_init_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(op2b.Op2bError) as e:
        op2b.op2b_init(0, 0)
    assert e.value.code == op2b.ECUDA


def test_library_rcm_equals_oracle_rcm(lib):
    for n, seed in ((6, 0), (9, 1), (12, 2)):
        m = meshgen.lattice(n, seed=seed)
        assert np.array_equal(op2b.op2b_host_rcm(m.num_nodes, m.edge),
                              oracle.rcm_order(m.num_nodes, m.edge))
    rng = np.random.default_rng(0)
    edge = rng.integers(0, 300, size=(700, 2))  # irregular, with repeats
    assert np.array_equal(op2b.op2b_host_rcm(300, edge), oracle.rcm_order(300, edge))


@pytest.mark.parametrize("method", [0, 1, 2])
def test_renumber_is_a_bijection_and_sorts_edges(lib, method):
    m = meshgen.lattice(10)
    perm, order = op2b.op2b_host_renumber(m.num_nodes, m.edge, method, seed=5)
    assert np.array_equal(np.sort(perm), np.arange(m.num_nodes))
    assert np.array_equal(np.sort(order), np.arange(m.num_edges))
    e2 = perm[m.edge][order]
    if method == 2:
        assert np.array_equal(order, oracle.renumber.edge_order(m.edge, perm))
        assert oracle.bandwidth(e2) < oracle.bandwidth(m.edge) / 2
    key = np.minimum(e2[:, 0], e2[:, 1]).astype(np.int64) * m.num_nodes + \
        np.maximum(e2[:, 0], e2[:, 1])
    assert np.all(np.diff(key) > 0)


@pytest.mark.parametrize("part", [64, 256, 1000])
def test_block_colouring_is_conflict_free(lib, part):
    m = meshgen.lattice(10)
    perm, order = op2b.op2b_host_renumber(m.num_nodes, m.edge, 2)
    for edge in (m.edge, perm[m.edge][order]):
        col, nc = op2b.op2b_host_colour_blocks(m.num_nodes, edge, part)
        nb = (edge.shape[0] + part - 1) // part
        assert col.shape == (nb,) and np.all((col >= 0) & (col < nc))
        assert set(col.tolist()) == set(range(nc))
        # exhaustive: no node is touched by two blocks of one colour
        owner = {}
        for b in range(nb):
            nodes = set(edge[b * part:(b + 1) * part].ravel().tolist())
            for v in nodes:
                key = (v, int(col[b]))
                assert key not in owner, (v, b, owner.get(key))
                owner[key] = b


def test_node_csr_lists_every_edge_end_once(lib):
    m = meshgen.lattice(7)
    rowptr, ends = op2b.op2b_host_node_csr(m.num_nodes, m.edge)
    assert rowptr[0] == 0 and rowptr[-1] == 2 * m.num_edges
    assert np.array_equal(np.sort(ends), np.arange(2 * m.num_edges))
    for i in range(0, m.num_nodes, 37):
        seg = ends[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(seg) > 0)
        assert np.all(m.edge[seg // 2, seg % 2] == i)
    assert np.all(np.diff(rowptr) == 18)


def test_host_planners_reject_bad_input(lib):
    with pytest.raises(op2b.Op2bError):
        op2b.op2b_host_rcm(3, np.array([[0, 5]]))
    with pytest.raises(op2b.Op2bError):
        op2b.op2b_host_renumber(3, np.array([[0, 1]]), method=9)
    with pytest.raises(op2b.Op2bError):
        op2b.op2b_host_colour_blocks(3, np.array([[0, 1]]), part=0)


@pytest.mark.parametrize("leaf", [1, 4, 64])
def test_library_rcb_equals_oracle_rcb(lib, leaf):
    m = meshgen.lattice(7, seed=2)
    a = op2b.op2b_host_rcb(m.coords, leaf)
    b = oracle.rcb_order(m.coords, leaf)
    assert np.array_equal(a, b)
    assert np.array_equal(np.sort(a), np.arange(m.num_nodes))


def test_rcb_partition_order_is_spatially_local(lib):
    # leaves of the bisection are compact boxes: consecutive new ids stay close
    m = meshgen.lattice(12)
    new = op2b.op2b_host_rcb(m.coords, 1)
    order = np.argsort(new)
    steps = np.linalg.norm(np.diff(m.coords[order], axis=0), axis=1)
    rand = np.linalg.norm(np.diff(m.coords, axis=0), axis=1)
    assert np.median(steps) < 0.25 * np.median(rand)


def test_noalloc_argument_checks_need_no_device(lib):
    """The allocation-free entry point rejects an output that overlaps an
    input and an oversized edge set before it touches the GPU (the
    addresses below are never dereferenced)."""
    N, E, ld = 100, 900, 128
    base = 1 << 40
    q, n, R = base, base + (1 << 30), base + (2 << 30)
    ok = dict(edge_first_ptr=base + (3 << 30), edge_second_ptr=base + (4 << 30),
              rowptr_ptr=base + (5 << 30), ends_ptr=base + (6 << 30))

    def call(q_ptr, n_ptr, R_ptr, e=E):
        op2b.op2b_edge_flux1_noalloc(q_ptr, ld, n_ptr, 1024, ok["edge_first_ptr"],
                                     ok["edge_second_ptr"], ok["rowptr_ptr"], ok["ends_ptr"],
                                     N, e, 1.4, R_ptr, ld, 0)
    # R's last row ends at 8 (5 ld + N) bytes past R: one byte into q is an overlap
    for q_ptr, n_ptr, R_ptr in ((q, n, q), (q, n, n + 8 * 1024), (q + 8 * (5 * ld + N) - 8, n, q),
                                (q, n, q - 8 * (5 * ld + N) + 8)):
        with pytest.raises(op2b.Op2bError) as e:
            call(q_ptr, n_ptr, R_ptr)
        assert e.value.code == op2b.EINVAL
        assert "overlaps" in op2b.op2b_last_error(None)
    with pytest.raises(op2b.Op2bError) as e:
        call(q, n, R, e=op2b.NOALLOC_MAX_EDGES + 1)
    assert e.value.code == op2b.ERANGE
