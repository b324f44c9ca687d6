"""FP32-seeded Newton reciprocal and square root of the FP64 edge kernels,
against correctly rounded IEEE results and their stated error bounds."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def newton(gpu_lib, tmp_path_factory):
    out = str(tmp_path_factory.mktemp("newton") / "newton_check.so")
    subprocess.check_call(["nvcc", "-O3", "-std=c++17", "-gencode",
                           "arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC",
                           "-shared", "-o", out,
                           os.path.join(HERE, "gpu_helpers", "newton_check.cu")])
    lib = ctypes.CDLL(out)
    lib.newton_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                 ctypes.c_int]
    return lib


def run(lib, x, which):
    import torch
    xt = torch.from_numpy(x).cuda()
    ot = torch.empty_like(xt)
    assert lib.newton_check(xt.data_ptr(), ot.data_ptr(), xt.numel(), which) == 0
    return ot.cpu().numpy()


def test_newton_forms_meet_their_error_bounds(newton):
    rng = np.random.default_rng(0)
    # the ranges the kernels see (limiter denominators down to 2e-12,
    # densities and pressures of order 1) plus wide log-uniform samples
    x = np.concatenate([10.0 ** rng.uniform(-30, 30, 200000),
                        rng.uniform(2e-12, 1e-6, 50000), rng.uniform(0.5, 2.0, 50000)])
    rel = lambda a, b: np.abs(a - b) / np.abs(b)
    assert np.all(run(newton, x, 5) == 1.0)  # all seedable
    # two Newton steps: within 2 ulp of the correctly rounded value
    assert np.max(rel(run(newton, x, 0), 1.0 / x)) <= 2.0 ** -51
    assert np.max(rel(run(newton, x, 1), np.sqrt(x))) <= 2.0 ** -51
    assert np.max(rel(run(newton, x, 2), 1.0 / np.sqrt(x))) <= 2.0 ** -51
    # batched inversion (inside [2^-70, 2^70]): a few ulp
    xb = np.concatenate([rng.uniform(2e-12, 1e-6, 50000), rng.uniform(0.5, 2.0, 50000)])
    assert np.max(rel(run(newton, xb, 3), 0.5 / xb)) <= 2.0 ** -49


def test_seedable_range(newton):
    x = np.array([0.0, -1.0, 1e-300, 1e300, 2.0 ** -126, 2.0 ** 126, 1.0, 3e-38,
                  np.inf, np.nan])
    s = run(newton, x, 5)
    assert s.tolist() == [0, 0, 0, 0, 0, 1, 1, 1, 0, 0]


def test_integer_float_to_double_is_exact(newton):
    import torch
    rng = np.random.default_rng(1)
    bits = np.concatenate([rng.integers(0, 2 ** 32, 4_000_000, dtype=np.uint64),
                           np.array([0, 0x80000000, 1, 0x80000001, 0x007fffff, 0x00800000,
                                     0x7f7fffff, 0x7f800000, 0xff800000, 0x7fc00001],
                                    dtype=np.uint64)]).astype(np.uint32)
    newton.f64_exact_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    bt = torch.from_numpy(bits.view(np.int32)).cuda()
    out = torch.empty(bits.size, dtype=torch.float64, device="cuda")
    assert newton.f64_exact_check(bt.data_ptr(), out.data_ptr(), bits.size) == 0
    got = out.cpu().numpy()
    with np.errstate(invalid="ignore"):
        ref = bits.view(np.float32).astype(np.float64)
    same = (got.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(got) & np.isnan(ref))
    assert np.all(same)


def _int_paths(lib, bits, which):
    import torch
    lib.int_paths_check.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_int]
    bt = torch.from_numpy(bits.view(np.int64)).cuda()
    out = torch.empty(bits.size, dtype=torch.float64, device="cuda")
    assert lib.int_paths_check(bt.data_ptr(), out.data_ptr(), bits.size, which) == 0
    return out.cpu().numpy()


def _same(got, ref):
    return (got.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(got) & np.isnan(ref))


def test_increment_conversion_fast_path_is_exact(newton):
    """to_acc: integer re-biasing for zero and normal floats, the general
    integer conversion for subnormal, infinite and NaN ones."""
    rng = np.random.default_rng(2)
    b32 = np.concatenate([rng.integers(0, 2 ** 32, 2_000_000, dtype=np.uint64),
                          np.array([0, 0x80000000, 1, 0x80000001, 0x007fffff, 0x00800000,
                                    0x80800000, 0x7f7fffff, 0x7f800000, 0xff800000,
                                    0x7fc00001], dtype=np.uint64)])
    got = _int_paths(newton, b32, 0)
    with np.errstate(invalid="ignore"):
        ref = b32.astype(np.uint32).view(np.float32).astype(np.float64)
    assert np.all(_same(got, ref))


def test_integer_halving_is_exact(newton):
    """half_exact: exponent decrement for zero and normal x whose half is
    normal, the FP64 multiply for the rest; bitwise x * 0.5 everywhere."""
    rng = np.random.default_rng(3)
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308,
                        4.450147717014403e-308, 4.4501477170144023e-308 * 1.5, 1.0, -3.0,
                        1.7976931348623157e308, np.inf, -np.inf, np.nan, 1e-310],
                       dtype=np.float64).view(np.uint64)
    bits = np.concatenate([rng.integers(0, 2 ** 63, 2_000_000, dtype=np.uint64),
                           rng.integers(0, 2 ** 63, 100_000, dtype=np.uint64) | np.uint64(1 << 63),
                           rng.integers(0, 2 ** 53, 100_000, dtype=np.uint64),  # subnormal / ex 1-2
                           special])
    got = _int_paths(newton, bits, 1)
    with np.errstate(invalid="ignore", over="ignore"):
        ref = bits.view(np.float64) * 0.5
    assert np.all(_same(got, ref))
