"""The allocation-free entry point op2b_edge_flux1_noalloc.

It exists for callers that may not allocate device memory (a memory pool
owned by another component, or a time loop in which allocation is not
allowed).  Here it is called through the C ABI with caller-owned tensors,
on two calls in a row on two different meshes, and compared with the
oracle's first-order residual on the library's numbering and with the
context entry point op2b_edge_flux (first order, segmented strategy).  The
second call runs on the scratch array the first call left behind, and
neither the device's free memory (cudaMemGetInfo) nor torch's allocator may change
across it.

This file is named to be collected last.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _inputs(op2b, torch, n):
    from paper_1403_7209_gb300.solver import EdgeSolver
    m = meshgen.lattice(n, seed=n)
    q = meshgen.flow_state(m, seed=n)
    s = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, renumber="rcm")
    s.set_strategy(op2b.LOOP_FLUX1, 0, op2b.STRAT_SEGMENTED)
    s.flux(1)
    torch.cuda.synchronize()
    R_ctx = s.t["R"].clone()
    rowptr, ends = op2b.op2b_host_node_csr(s.N, s.edge)
    dev = {
        "rowptr": torch.from_numpy(rowptr).cuda(),
        "ends": torch.from_numpy(ends.astype(np.int32)).cuda(),
        "m0": torch.from_numpy(np.ascontiguousarray(s.edge[:, 0])).cuda(),
        "m1": torch.from_numpy(np.ascontiguousarray(s.edge[:, 1])).cuda(),
    }
    # the oracle's residual and the scale of every entry (sum of the
    # absolute edge contributions), on the library's numbering
    qn = s.t["q"].cpu().numpy().T
    nn = s.t["n"].cpu().numpy().T
    R_ora, Rabs = oracle.flux1(s.edge, qn, nn, with_abs=True)
    torch.cuda.synchronize()
    return s, R_ctx, R_ora, dev, Rabs


def _call(op2b, torch, s, dev, R):
    op2b.op2b_edge_flux1_noalloc(
        s.t["q"].data_ptr(), s.t["q"].shape[1], s.t["n"].data_ptr(), s.t["n"].shape[1],
        dev["m0"].data_ptr(), dev["m1"].data_ptr(), dev["rowptr"].data_ptr(),
        dev["ends"].data_ptr(), s.N, s.E, 1.4, R.data_ptr(), R.shape[1],
        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()


def _alloc_state(torch):
    st = torch.cuda.memory_stats()
    return (torch.cuda.mem_get_info()[0], st.get("allocation.all.allocated", 0),
            st.get("segment.all.allocated", 0), torch.cuda.memory_reserved())


def test_noalloc_matches_oracle_and_context_entry_point_twice(gpu_lib):
    import torch
    op2b = gpu_lib
    first = _inputs(op2b, torch, 16)    # 36,864 edges
    second = _inputs(op2b, torch, 12)   # 15,552 edges
    outs = [torch.full_like(R_ctx, float("nan")) for _, R_ctx, *_ in (first, second)]
    for k, ((s, R_ctx, R_ora, dev, Rabs), R) in enumerate(zip((first, second), outs)):
        before = _alloc_state(torch)
        _call(op2b, torch, s, dev, R)
        if k == 1:  # the first call may load the module holding the array
            assert _alloc_state(torch) == before, "the second call allocated device memory"
        Rn = R.cpu().numpy().T
        # element by element against the oracle (only the summation order
        # differs) and against the context entry point
        assert float(np.max(np.abs(Rn - R_ora) / (Rabs + 1e-300))) <= TOL
        assert float(np.max(np.abs(Rn - R_ctx.cpu().numpy().T) / (Rabs + 1e-300))) <= TOL
    for s, *_ in (first, second):
        s.close()


def test_noalloc_rejects_oversized_edge_sets(gpu_lib):
    import torch
    op2b = gpu_lib
    R = torch.zeros((6, 4), dtype=torch.float64, device="cuda")
    q = torch.ones((6, 4), dtype=torch.float64, device="cuda")
    E = op2b.NOALLOC_MAX_EDGES + 1
    with pytest.raises(op2b.Op2bError) as e:
        op2b.op2b_edge_flux1_noalloc(q.data_ptr(), 4, q.data_ptr(), E, q.data_ptr(),
                                     q.data_ptr(), q.data_ptr(), q.data_ptr(), 4, E, 1.4,
                                     R.data_ptr(), 4, 0)
    assert e.value.code == op2b.ERANGE
    assert "exceeds the limit" in op2b.op2b_last_error(None)
