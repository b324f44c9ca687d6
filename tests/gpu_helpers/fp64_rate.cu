// Test helper: throughput of the arithmetic the FP64 edge loops are built
// from (FP64 fused multiply-add, multiply, add, IEEE division and square
// root) and, for comparison, the FP32 fused multiply-add.  Every thread runs
// C independent dependency chains (C = 4, 8 or 16) so that the pipes, not
// the latencies, bound the rate; the results are stored conditionally so
// that nothing is optimised away.
#include <cuda_runtime.h>

#include <cstdint>

template <int OP, typename T, int C>
__global__ void k_rate(T* out, int iters, T a, T b) {
  T x[C];
#pragma unroll
  for (int k = 0; k < C; k++) x[k] = a + T(threadIdx.x + k) * T(1e-9);
#pragma unroll 2
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int k = 0; k < C; k++) {
      if constexpr (OP == 0) x[k] = fma(x[k], b, a);    // fused multiply-add
      else if constexpr (OP == 1) x[k] = x[k] * b;      // multiply
      else if constexpr (OP == 2) x[k] = x[k] + b;      // add
      else if constexpr (OP == 3) x[k] = a / x[k];      // IEEE division
      else x[k] = sqrt(x[k] + b);                       // IEEE square root
    }
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < C; k++) s += x[k];
  if (s == T(-12345.0)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP, typename T>
static void launch_c(int chains, int blocks, int threads, void* out, int iters, T a, T b) {
  if (chains == 4) k_rate<OP, T, 4><<<blocks, threads>>>((T*)out, iters, a, b);
  else if (chains == 16) k_rate<OP, T, 16><<<blocks, threads>>>((T*)out, iters, a, b);
  else k_rate<OP, T, 8><<<blocks, threads>>>((T*)out, iters, a, b);
}

template <typename T>
static void launch_op(int op, int chains, int blocks, int threads, void* out, int iters, T a,
                      T b) {
  switch (op) {
    case 0: launch_c<0, T>(chains, blocks, threads, out, iters, a, b); break;
    case 1: launch_c<1, T>(chains, blocks, threads, out, iters, a, b); break;
    case 2: launch_c<2, T>(chains, blocks, threads, out, iters, a, b); break;
    case 3: launch_c<3, T>(chains, blocks, threads, out, iters, a, b); break;
    default: launch_c<4, T>(chains, blocks, threads, out, iters, a, b); break;
  }
}

// op: 0 fma, 1 mul, 2 add, 3 div, 4 sqrt; f32: FP32 instead of FP64;
// chains: independent chains per thread (4, 8 or 16).  Returns the
// operations per second (one per chain step per thread; an FMA counts as
// one) measured with CUDA events, or a negative value on error.
extern "C" double fp64_rate(int op, int f32, int blocks, int threads, int iters, int chains) {
  void* out = nullptr;
  if (chains != 4 && chains != 16) chains = 8;
  if (cudaMalloc(&out, (size_t)blocks * threads * 8) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&]() {
    if (f32) launch_op<float>(op, chains, blocks, threads, out, iters, 0.999f, 1.0000001f);
    else launch_op<double>(op, chains, blocks, threads, out, iters, 0.999, 1.0000000001);
  };
  launch();  // warm-up
  cudaEventRecord(e0);
  launch();
  cudaEventRecord(e1);
  double rate = -1.0;
  if (cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess) {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    rate = (double)blocks * threads * iters * chains / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return rate;
}
