"""Measured node-gather rates: the bound of the FP32-mixed stage's passes.

Every node of the 100^3 lattice (RCM numbering, 18 edge ends per node) sums
the packed records (8, 24 or 32 floats) of the other ends of its edges, one
thread per node, 32-byte loads; the same bytes read coalesced set the
scale.  The fused stage's flux pass gathers a 24-float record per edge end,
so its records alone need at least the 24-float gather's time.  With
``OP2B_GATHER_OUT`` set the figures are written there as JSON.  The check
is loose (the gather reaches at least 2 TB/s of useful bytes and does not
beat the coalesced read): the figures are the point.
"""
import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

from paper_1403_7209_gb300 import meshgen

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(gpu_lib, tmp_path_factory):
    out = str(tmp_path_factory.mktemp("gather") / "gather_rate.so")
    subprocess.check_call(["nvcc", "-O3", "-std=c++17", "-gencode",
                           "arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC", "-shared",
                           "-o", out, os.path.join(HERE, "gpu_helpers", "gather_rate.cu")])
    lib = ctypes.CDLL(out)
    lib.run_probe.restype = ctypes.c_float
    lib.run_probe.argtypes = ([ctypes.c_int, ctypes.c_int, ctypes.c_int64] + [ctypes.c_void_p] * 4
                              + [ctypes.c_int, ctypes.c_int])
    return lib


def test_node_gather_rates(gpu_lib, probe):
    import torch
    op2b = gpu_lib
    m = meshgen.lattice(100)
    N = m.num_nodes
    perm, _ = op2b.op2b_host_renumber(N, m.edge, 2, seed=0)
    e = perm[m.edge]
    rp, ends = op2b.op2b_host_node_csr(N, e)
    ends = np.asarray(ends)
    other = np.where(ends & 1, e[ends >> 1, 0], e[ends >> 1, 1]).astype(np.int32)
    d_rp = torch.from_numpy(np.asarray(rp)).cuda()
    d_adj = torch.from_numpy(other).cuda()
    o = torch.empty(N, dtype=torch.float32, device="cuda")
    out = {"mesh": "100^3 lattice, RCM, 18 ends per node", "block": 128}
    for W in (8, 24, 32):
        rec = torch.rand(N * W, dtype=torch.float32, device="cuda")
        for which, nm in ((0, "gather"), (2, "coalesced")):
            ms = probe.run_probe(which, W, N, d_rp.data_ptr(), d_adj.data_ptr(), rec.data_ptr(),
                                 o.data_ptr(), 128, 10)
            assert ms > 0.0
            out["%s_%d_floats" % (nm, W)] = {"ms": ms,
                                             "useful_tb_s": 18 * N * W * 4 / (ms * 1e-3) / 1e12}
    print(json.dumps(out))
    if os.environ.get("OP2B_GATHER_OUT"):
        with open(os.environ["OP2B_GATHER_OUT"], "w") as fh:
            json.dump(out, fh, indent=1)
    for W in (8, 24, 32):
        g, c = out["gather_%d_floats" % W], out["coalesced_%d_floats" % W]
        assert g["useful_tb_s"] >= 2.0, out
        assert g["ms"] >= 0.9 * c["ms"], out
