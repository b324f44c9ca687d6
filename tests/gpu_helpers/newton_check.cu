// Test helper: evaluates the FP32-seeded Newton reciprocal / square root of
// the edge kernels on an array, for comparison with correctly rounded values.
#include "../../paper_1403_7209_gb300/csrc/edge_math.cuh"

__global__ void k_newton(const double* x, double* out, int64_t n, int which) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = x[i];
  double r = 0.0;
  if (which == 0) r = op2b::recip2(v);
  else if (which == 1) r = op2b::sqrt2(v);
  else if (which == 2) r = op2b::rsqrt2(v);
  else if (which == 3) {
    double d[3] = {v, 1.0 + v, 3.0 * v}, rr[3];
    op2b::batch_reciprocal<3>(d, 0.5, rr);
    r = rr[0];
  }
  else r = op2b::seedable(v) ? 1.0 : 0.0;
  out[i] = r;
}

extern "C" int newton_check(const double* x, double* out, int64_t n, int which) {
  if (n <= 0) return 0;
  k_newton<<<(unsigned)((n + 255) / 256), 256>>>(x, out, n, which);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}

__global__ void k_f64_exact(const unsigned* bits, double* out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = op2b::f64_exact(__int_as_float((int)bits[i]));
}

extern "C" int f64_exact_check(const unsigned* bits, double* out, int64_t n) {
  if (n <= 0) return 0;
  k_f64_exact<<<(unsigned)((n + 255) / 256), 256>>>(bits, out, n);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}

// which = 0: the increments' float -> double conversion (to_acc, with its
// normal-number fast path); which = 1: x / 2 on the integer pipe
// (half_exact), on the bit patterns given (as 64-bit words).
__global__ void k_int_paths(const unsigned long long* bits, double* out, int64_t n, int which) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (which == 0)
    out[i] = op2b::to_acc<double>(__int_as_float((int)(unsigned)bits[i]));
  else
    out[i] = op2b::half_exact(__longlong_as_double((long long)bits[i]));
}

extern "C" int int_paths_check(const unsigned long long* bits, double* out, int64_t n,
                               int which) {
  if (n <= 0) return 0;
  k_int_paths<<<(unsigned)((n + 255) / 256), 256>>>(bits, out, n, which);
  return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
