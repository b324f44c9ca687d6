// Test helper: the rate at which a GB300 gathers packed node records over a
// mesh's node-sorted adjacency (every node reads the records of the other
// ends of its edges, as the FP32-mixed stage's node passes do), against a
// coalesced read of the same bytes.  It bounds the node-gather passes: their
// records cannot arrive faster than this.
#include <cuda_runtime.h>
#include <cstdint>

__device__ __forceinline__ void ldg8(const float* p, float* v) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7])
      : "l"(p));
}

// W floats per record (8, 24 or 32); thread per node sums the neighbours'
// records over its CSR row
template <int W>
__global__ void k_gather(int64_t N, const int64_t* rowptr, const int32_t* adj, const float* rec,
                         float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float acc[W];
#pragma unroll
    for (int k = 0; k < W; k++) acc[k] = 0.f;
    for (int64_t t = rowptr[i]; t < rowptr[i + 1]; t++) {
      const float* p = rec + (int64_t)adj[t] * W;
      float v[W];
#pragma unroll
      for (int k = 0; k < W / 8; k++) ldg8(p + 8 * k, v + 8 * k);
#pragma unroll
      for (int k = 0; k < W; k++) acc[k] += v[k];
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < W; k++) s += acc[k];
    out[i] = s;
  }
}

// same, but ILP: U ends per iteration (loads first)
template <int W, int U>
__global__ void k_gather_u(int64_t N, const int64_t* rowptr, const int32_t* adj, const float* rec,
                           float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float acc[W];
#pragma unroll
    for (int k = 0; k < W; k++) acc[k] = 0.f;
    const int64_t t0 = rowptr[i], t1 = rowptr[i + 1];
    int64_t t = t0;
    for (; t + U <= t1; t += U) {
      float v[U][W];
#pragma unroll
      for (int u = 0; u < U; u++) {
        const float* p = rec + (int64_t)adj[t + u] * W;
#pragma unroll
        for (int k = 0; k < W / 8; k++) ldg8(p + 8 * k, v[u] + 8 * k);
      }
#pragma unroll
      for (int u = 0; u < U; u++)
#pragma unroll
        for (int k = 0; k < W; k++) acc[k] += v[u][k];
    }
    for (; t < t1; t++) {
      const float* p = rec + (int64_t)adj[t] * W;
      float v[W];
#pragma unroll
      for (int k = 0; k < W / 8; k++) ldg8(p + 8 * k, v + 8 * k);
#pragma unroll
      for (int k = 0; k < W; k++) acc[k] += v[k];
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < W; k++) s += acc[k];
    out[i] = s;
  }
}

// streaming: each thread reads 18 consecutive records of a flat array
// (same bytes as the gather, fully coalesced across threads)
template <int W>
__global__ void k_stream(int64_t N, const float* rec, int64_t nrec, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int r = 0; r < 18; r++) {
      const int64_t idx = ((int64_t)r * N + i) % nrec;
      const float* p = rec + idx * W;
      float v[W];
#pragma unroll
      for (int k = 0; k < W / 8; k++) ldg8(p + 8 * k, v + 8 * k);
#pragma unroll
      for (int k = 0; k < W; k++) s += v[k];
    }
    out[i] = s;
  }
}

extern "C" float run_probe(int which, int W, int64_t N, const int64_t* rowptr,
                           const int32_t* adj, const float* rec, float* out, int block,
                           int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int64_t grid = (N + block - 1) / block;
  auto go = [&]() {
    if (which == 0) {
      if (W == 8) k_gather<8><<<grid, block>>>(N, rowptr, adj, rec, out);
      else if (W == 24) k_gather<24><<<grid, block>>>(N, rowptr, adj, rec, out);
      else k_gather<32><<<grid, block>>>(N, rowptr, adj, rec, out);
    } else if (which == 1) {
      if (W == 8) k_gather_u<8, 4><<<grid, block>>>(N, rowptr, adj, rec, out);
      else if (W == 24) k_gather_u<24, 2><<<grid, block>>>(N, rowptr, adj, rec, out);
      else k_gather_u<32, 2><<<grid, block>>>(N, rowptr, adj, rec, out);
    } else {
      if (W == 8) k_stream<8><<<grid, block>>>(N, rec, N, out);
      else if (W == 24) k_stream<24><<<grid, block>>>(N, rec, N, out);
      else k_stream<32><<<grid, block>>>(N, rec, N, out);
    }
  };
  go();
  cudaEventRecord(e0);
  for (int r = 0; r < reps; r++) go();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return -1.f;
  return ms / reps;
}
