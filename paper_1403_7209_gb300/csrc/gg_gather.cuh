// Green-Gauss sums as a node gather (the "gather" strategy of the
// Green-Gauss loop, in every precision).
//
// Graw_i = sum over node i's edge ends (the node-sorted list of the
// segmented plan) of +-(q_i + q_j) (x) n/2: + at the edge's first end, - at
// its second.  Each node's sums stay in registers and are written once (and
// divided by the node's volume there when the scaling is fused), so
// there is no INC race, no atomic and a fixed order of the ends (bitwise
// reproducible).  SPLIT threads share a node, each summing 6/SPLIT of its
// components (fewer registers per thread, more warps to hide the gathers of
// the other end's q); the end list and normals they read are the same
// addresses, so a warp fetches them once.  With `add` the sums are added
// to G instead of replacing it.
#pragma once
#include <algorithm>

#include "ff_math.cuh"
#include "internal.h"

namespace op2b {

// x * h for h = +-1/2 (exact; for double the sign flip and the halving are
// integer operations, so the FP64 pipe is left to the sums)
__device__ __forceinline__ double gg_scale(double x, float h) {
  return half_exact(h < 0.0f ? neg(x) : x);
}
__device__ __forceinline__ float gg_scale(float x, float h) { return x * h; }
__device__ __forceinline__ ffv gg_scale(ffv x, float h) { return ffv(ff_scale(x.v, h)); }

template <typename T>
__device__ __forceinline__ T gg_zero() {
  return T(0.0f);
}
template <>
__device__ __forceinline__ ffv gg_zero<ffv>() {
  return ffv(make_float2(0.0f, 0.0f));
}

// 1/V in the gradient's type, formed as the scaling loop forms it, so that
// the fused scaling gives the scaling loop's bits
__device__ __forceinline__ void gg_rvol(double V, double& r) { r = 1.0 / V; }
__device__ __forceinline__ void gg_rvol(double V, float& r) { r = (float)(1.0 / V); }
__device__ __forceinline__ void gg_rvol(double V, ffv& r) { r = ffv(ff_recip(ff_of_f64(V))); }

template <typename T, int SPLIT>
__global__ void k_gg_gather(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ ends,
                            const int32_t* __restrict__ m0, const int32_t* __restrict__ m1,
                            const T* __restrict__ q, int64_t ldq, const T* __restrict__ n,
                            int64_t ldn, T* __restrict__ G, int64_t ldG, int64_t N, bool add,
                            const double* __restrict__ vol) {
  constexpr int KC = 6 / SPLIT;
  const int64_t total = N * SPLIT;
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t0 < total;
       t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t0 / SPLIT;
    const int k0 = (int)(t0 - i * SPLIT) * KC;
    T qi[KC], acc[3 * KC];
#pragma unroll
    for (int k = 0; k < KC; k++) qi[k] = ldro(q + (k0 + k) * ldq + i);
#pragma unroll
    for (int c = 0; c < 3 * KC; c++) acc[c] = gg_zero<T>();
    const int64_t t1 = rowptr[i + 1];
    // unrolled so that the dependent loads (end -> edge -> other node ->
    // its q) of several ends are in flight together
#pragma unroll 4
    for (int64_t t = rowptr[i]; t < t1; t++) {
      const int32_t end = ends[t];
      const int64_t e = end >> 1;
      const bool second = end & 1;
      const int64_t j = second ? m0[e] : m1[e];  // the other end
      const float h = second ? -0.5f : 0.5f;      // sign and the 1/2
      T nh[3];
#pragma unroll
      for (int d = 0; d < 3; d++) nh[d] = gg_scale(ldro(n + d * ldn + e), h);
#pragma unroll
      for (int k = 0; k < KC; k++) {
        const T sk = qi[k] + ldro(q + (k0 + k) * ldq + j);
#pragma unroll
        for (int d = 0; d < 3; d++) acc[3 * k + d] = fma(sk, nh[d], acc[3 * k + d]);
      }
    }
    // with vol: G = (sum) / V, the gradient scaling fused into the write
    T r = gg_zero<T>();
    if (vol) gg_rvol(ldro(vol + i), r);
#pragma unroll
    for (int c = 0; c < 3 * KC; c++) {
      T* g = G + (3 * k0 + c) * ldG + i;
      const T v = add ? *g + acc[c] : acc[c];
      *g = vol ? v * r : v;
    }
  }
}

// Launch over the map's node-sorted edge ends; block = 0 picks 128.
template <typename T, int SPLIT>
int launch_gg_gather(Ctx* c, const LoopLaunch& L, int block) {
  DevSegPlan* sp = nullptr;
  if (int rc = c->seg_plan(L.map, &sp)) return rc;
  if (L.N == 0) return OP2B_OK;
  if (block <= 0) block = 128;
  if (block < 32 || block > 1024 || block % 32)
    return c->fail(OP2B_EINVAL, "block size must be a multiple of 32 in [32, 1024]");
  const int64_t grid =
      std::min<int64_t>((L.N * SPLIT + block - 1) / block, 0x7fffffff);  // all blocks, node order
  k_gg_gather<T, SPLIT><<<(unsigned)grid, block, 0, c->stream>>>(
      sp->rowptr, sp->ends, L.m0, L.m1, (const T*)L.q, L.ldq, (const T*)L.n, L.ldn, (T*)L.t0,
      L.ldt0, L.N, !(L.flags & OP2B_ZERO_INC), L.vol);
  return c->launched("green_gauss gather");
}

// Hybrid Green-Gauss (FP64): one launch whose first `gblocks` blocks gather
// components 0..2 of every node (as k_gg_gather, one thread per node, on
// the FP64 pipe) while the remaining blocks scatter components 3..5 edge by
// edge with atomic adds (in the L2's atomic units).  The two halves are
// bound by different units, so running them side by side on every SM
// overlaps the FP64-pipe time of the one with the atomic time of the other.
// Both halves always add into G (the caller zeroes it for OP2B_ZERO_INC).
static __global__ void k_gg_hybrid(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ ends,
                            const int32_t* __restrict__ m0, const int32_t* __restrict__ m1,
                            const double* __restrict__ q, int64_t ldq,
                            const double* __restrict__ n, int64_t ldn, double* __restrict__ G,
                            int64_t ldG, int64_t N, int64_t E, unsigned gblocks) {
  if (blockIdx.x < gblocks) {
    const int64_t stride = (int64_t)gblocks * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
      double qi[3], acc[9];
#pragma unroll
      for (int k = 0; k < 3; k++) qi[k] = ldro(q + k * ldq + i);
#pragma unroll
      for (int c = 0; c < 9; c++) acc[c] = 0.0;
      const int64_t t1 = rowptr[i + 1];
      for (int64_t t = rowptr[i]; t < t1; t++) {
        const int32_t end = ends[t];
        const int64_t e = end >> 1;
        const bool second = end & 1;
        const int64_t j = second ? m0[e] : m1[e];
        double nh[3];
#pragma unroll
        for (int d = 0; d < 3; d++) nh[d] = gg_scale(ldro(n + d * ldn + e), second ? -0.5f : 0.5f);
#pragma unroll
        for (int k = 0; k < 3; k++) {
          const double sk = qi[k] + ldro(q + k * ldq + j);
#pragma unroll
          for (int d = 0; d < 3; d++) acc[3 * k + d] = fma(sk, nh[d], acc[3 * k + d]);
        }
      }
#pragma unroll
      for (int c = 0; c < 9; c++) G[c * ldG + i] += acc[c];
    }
  } else {
    const int64_t stride = (int64_t)(gridDim.x - gblocks) * blockDim.x;
    for (int64_t e = (blockIdx.x - gblocks) * (int64_t)blockDim.x + threadIdx.x; e < E;
         e += stride) {
      const int64_t i = m0[e], j = m1[e];
      const double h[3] = {half_exact(ldro(n + e)), half_exact(ldro(n + ldn + e)),
                           half_exact(ldro(n + 2 * ldn + e))};
#pragma unroll
      for (int k = 3; k < 6; k++) {
        const double sk = ldro(q + k * ldq + i) + ldro(q + k * ldq + j);
#pragma unroll
        for (int d = 0; d < 3; d++) {
          const double v = sk * h[d];
          atomicAdd(G + (3 * k + d) * ldG + i, v);
          atomicAdd(G + (3 * k + d) * ldG + j, neg(v));
        }
      }
    }
  }
}

inline int launch_gg_hybrid(Ctx* c, const LoopLaunch& L, int block) {
  DevSegPlan* sp = nullptr;
  if (int rc = c->seg_plan(L.map, &sp)) return rc;
  if (L.N == 0) return OP2B_OK;
  if (block <= 0) block = 128;
  if (block < 32 || block > 1024 || block % 32)
    return c->fail(OP2B_EINVAL, "block size must be a multiple of 32 in [32, 1024]");
  // both roles resident on every SM at once: an equal number of blocks each
  const int per_sm = std::max(1, 1024 / block);
  const unsigned gblocks = (unsigned)std::min<int64_t>((L.N + block - 1) / block,
                                                       (int64_t)c->sm_count * per_sm / 2);
  const unsigned ablocks = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((L.E + block - 1) / block, (int64_t)c->sm_count * per_sm / 2));
  k_gg_hybrid<<<gblocks + ablocks, block, 0, c->stream>>>(
      sp->rowptr, sp->ends, L.m0, L.m1, (const double*)L.q, L.ldq, (const double*)L.n, L.ldn,
      (double*)L.t0, L.ldt0, L.N, L.E, gblocks);
  return c->launched("green_gauss hybrid");
}

}  // namespace op2b
