"""Measured arithmetic rates behind the FP64 roofline of the edge loops.

The FP64 edge loops are bound by the FP64 pipe, and the benchmark's "alu"
roofline divides by its peak: 152 SMs x 2 FP64 fused multiply-adds per
clock x 2 flops x 2.07 GHz = 1.26 TFLOP/s.  This test measures the rates
(4, 8 or 16 independent chains per thread over four launch shapes, the
best of them; CUDA events) with the SM clock sampled by nvidia-smi while
they run, and checks that the best FP64 FMA rate, scaled to 2.07 GHz, lies
within [0.8, 1.05] of that peak (the flux kernel's own FP64 instruction
rate, 0.88 of it, is a lower bound on what the pipe delivers), and that
FP32 FMAs run far faster (the reason for the FP32-mixed and float-float
paths).  With ``OP2B_RATE_OUT`` set the figures are written there as JSON.
"""
import ctypes
import json
import os
import statistics
import subprocess
import threading
import time

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
PEAK_FMA_PER_S = 152 * 2 * 2.07e9  # FP64 FMAs per second at the maximum clock


@pytest.fixture(scope="module")
def rate_lib(gpu_lib, tmp_path_factory):
    out = str(tmp_path_factory.mktemp("rate") / "fp64_rate.so")
    subprocess.check_call(["nvcc", "-O3", "-std=c++17", "-gencode",
                           "arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC",
                           "-shared", "-o", out, os.path.join(HERE, "gpu_helpers", "fp64_rate.cu")])
    lib = ctypes.CDLL(out)
    lib.fp64_rate.argtypes = [ctypes.c_int] * 6
    lib.fp64_rate.restype = ctypes.c_double
    return lib


def _sampled(fn):
    """Run fn() while nvidia-smi samples the SM clock every 20 ms."""
    samples = []
    try:
        p = subprocess.Popen(["nvidia-smi", "-i", "0", "--query-gpu=clocks.sm",
                              "--format=csv,noheader,nounits", "-lms", "20"],
                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        p = None
    if p is not None:
        th = threading.Thread(target=lambda: [samples.append(float(x)) for x in p.stdout
                                              if x.strip().replace(".", "").isdigit()],
                              daemon=True)
        th.start()
        time.sleep(0.3)
    r = fn()
    if p is not None:
        time.sleep(0.1)
        p.terminate()
        p.wait(timeout=5)
    return r, (statistics.median(samples) if samples else None)


def test_fp64_rates(rate_lib):
    import torch
    shapes = [(152 * 8, 256), (152 * 4, 512), (152 * 2, 1024), (152 * 16, 128)]
    names = ["fma", "mul", "add", "div", "sqrt"]
    work = {"fma": 32000, "mul": 32000, "add": 32000, "div": 3200, "sqrt": 3200}  # chain steps

    def best(op, f32, total):
        r, cfg = 0.0, None
        for blocks, threads in shapes:
            for chains in (4, 8, 16):
                v = rate_lib.fp64_rate(op, f32, blocks, threads, total // chains, chains)
                if v > r:
                    r, cfg = v, (blocks, threads, chains)
        return r, cfg

    def run():
        r, cfgs = {}, {}
        for op, nm in enumerate(names):
            r["f64_" + nm], cfgs["f64_" + nm] = best(op, 0, work[nm])
        r["f32_fma"], cfgs["f32_fma"] = best(0, 1, 320000)
        torch.cuda.synchronize()
        return r, cfgs
    (r, cfgs), mhz = _sampled(run)
    assert all(v > 0 for v in r.values()), r
    scale = 2070.0 / mhz if mhz else 1.0
    out = {"ops_per_s": r, "best_launch_blocks_threads_chains": cfgs, "sm_mhz_median": mhz,
           "fp64_fma_tflops": 2 * r["f64_fma"] / 1e12,
           "fp64_fma_tflops_at_2070mhz": 2 * r["f64_fma"] * scale / 1e12,
           "fp64_fma_per_clk_per_sm": r["f64_fma"] / (152 * (mhz or 2070.0) * 1e6),
           "f32_over_f64_fma": r["f32_fma"] / r["f64_fma"]}
    print(json.dumps(out))
    if os.environ.get("OP2B_RATE_OUT"):
        with open(os.environ["OP2B_RATE_OUT"], "w") as fh:
            json.dump(out, fh, indent=1)
    assert 0.8 <= r["f64_fma"] * scale / PEAK_FMA_PER_S <= 1.05, out
    assert r["f32_fma"] / r["f64_fma"] >= 16.0, out
