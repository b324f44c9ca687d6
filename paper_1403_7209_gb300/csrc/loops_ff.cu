// Float-float edge loop: the second-order flux with its arithmetic in
// float-float (FP32 instructions, ~47 significant bits), reading
// float-float shadows of q, G, n and dx and adding each edge's flux,
// converted to FP64, into the FP64 residual under any strategy.
#include "ff_math.cuh"
#include "launch.cuh"

namespace op2b {

// v = q (6), G (18) of one node as float-float values
struct BodyFlux2FF {
  using TN = float2;
  using TE = double;
  using TA = double;
  static constexpr int NIN = 24, OUT = 6, MODE = MODE_ANTI, DIM0 = 6;
  const float2* q;
  int64_t ldq;
  const float2* G;
  int64_t ldG;
  const float2* n;
  int64_t ldn;
  const float2* dx;
  int64_t lddx;
  GasFF g;
  __device__ __forceinline__ void load(int64_t i, float2* v) const {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ldro(q + k * ldq + i);
#pragma unroll
    for (int c = 0; c < 18; c++) v[6 + c] = ldro(G + c * ldG + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const float2* vi, const float2* vj,
                                       double* oi, double*) const {
    flux2_ff(vi, vj, ldro(dx + e), ldro(dx + lddx + e), ldro(dx + 2 * lddx + e), ldro(n + e),
             ldro(n + ldn + e), ldro(n + 2 * ldn + e), g, oi);
  }
};

// Green-Gauss sums as a node gather: Graw_i = sum over node i's edge ends
// (node-sorted list of the segmented plan) of +-(q_i + q_j) (x) n/2 (+ at
// the edge's first end, - at its second), accumulated in float-float
// registers and written once.  Every node owns its sums, so there is no INC
// race, no atomic and the order of the ends is fixed (bitwise
// reproducible).  SPLIT threads share a node, each summing 6/SPLIT of its
// components (fewer registers per thread, more warps to hide the gathers);
// the end list and normals they read are the same addresses, so a warp
// fetches them once.  With `add` the sums are added to G.
template <int SPLIT>
__global__ void k_gg_ff(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ ends,
                        const int32_t* __restrict__ m0, const int32_t* __restrict__ m1,
                        const float2* __restrict__ q, int64_t ldq, const float2* __restrict__ n,
                        int64_t ldn, float2* __restrict__ G, int64_t ldG, int64_t N, bool add) {
  constexpr int KC = 6 / SPLIT;
  const int64_t total = N * SPLIT;
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t0 < total;
       t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t0 / SPLIT;
    const int k0 = (int)(t0 - i * SPLIT) * KC;
    float2 qi[KC], acc[3 * KC];
#pragma unroll
    for (int k = 0; k < KC; k++) qi[k] = ldro(q + (k0 + k) * ldq + i);
#pragma unroll
    for (int c = 0; c < 3 * KC; c++) acc[c] = make_float2(0.0f, 0.0f);
    const int64_t t1 = rowptr[i + 1];
    for (int64_t t = rowptr[i]; t < t1; t++) {
      const int32_t end = ends[t];
      const int64_t e = end >> 1;
      const bool second = end & 1;
      const int64_t j = second ? m0[e] : m1[e];  // the other end
      const float h = second ? -0.5f : 0.5f;      // exact: sign and the 1/2
      float2 nh[3];
#pragma unroll
      for (int d = 0; d < 3; d++) nh[d] = ff_scale(ldro(n + d * ldn + e), h);
#pragma unroll
      for (int k = 0; k < KC; k++) {
        const float2 sk = ff_add(qi[k], ldro(q + (k0 + k) * ldq + j));
#pragma unroll
        for (int d = 0; d < 3; d++) acc[3 * k + d] = ff_fma(sk, nh[d], acc[3 * k + d]);
      }
    }
#pragma unroll
    for (int c = 0; c < 3 * KC; c++) {
      float2* g = G + (3 * k0 + c) * ldG + i;
      *g = add ? ff_add(*g, acc[c]) : acc[c];
    }
  }
}

// Adjoint of the second-order flux in float-float: v = lam (6), q (6),
// G (18) as float-float shadows; per end qbar (6) then Gbar (18) converted to
// FP64 and accumulated into the FP64 targets; nbar written in FP64.
struct BodyFluxAdjFF {
  using TN = ffv;
  using TE = ffv;
  using TA = double;
  static constexpr int NIN = 30, OUT = 24, MODE = MODE_GEN, DIM0 = 6;
  const ffv* lam;
  int64_t ldl;
  const ffv* q;
  int64_t ldq;
  const ffv* G;
  int64_t ldG;
  const ffv* n;
  int64_t ldn;
  const ffv* dx;
  int64_t lddx;
  double* nbar;
  int64_t ldnb;
  ffv gamma, gm1, eps, two_eps;
  __device__ __forceinline__ void load(int64_t i, ffv* v) const {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ldro(lam + k * ldl + i);
#pragma unroll
    for (int k = 0; k < 6; k++) v[6 + k] = ldro(q + k * ldq + i);
#pragma unroll
    for (int c = 0; c < 18; c++) v[12 + c] = ldro(G + c * ldG + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const ffv* vi, const ffv* vj, ffv* oi,
                                       ffv* oj) const {
    ffv nb[3];
    flux2_adj_t(vi, vj, ldro(dx + e), ldro(dx + lddx + e), ldro(dx + 2 * lddx + e), ldro(n + e),
                ldro(n + ldn + e), ldro(n + 2 * ldn + e), gamma, gm1, eps, two_eps, oi, oj, nb);
    nbar[e] = (double)nb[0];
    nbar[ldnb + e] = (double)nb[1];
    nbar[2 * ldnb + e] = (double)nb[2];
  }
};

int launch_ff(Ctx* c, const LoopLaunch& L, const Strategy& s) {
  if (L.loop == OP2B_LOOP_FLUX2_ADJ) {
    BodyFluxAdjFF b{(const ffv*)L.lam, L.ldl, (const ffv*)L.q, L.ldq, (const ffv*)L.G, L.ldG,
                    (const ffv*)L.n, L.ldn, (const ffv*)L.dx, L.lddx, (double*)L.direct,
                    L.lddirect, ffv(L.gamma), ffv(L.gamma - 1.0), ffv(L.eps), ffv(2.0 * L.eps)};
    Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t1, L.ldt1};
    return run_body(c, b, L, s, tg);
  }
  if (L.loop == OP2B_LOOP_GREEN_GAUSS) {
    DevSegPlan* sp = nullptr;
    if (int rc = c->seg_plan(L.map, &sp)) return rc;
    if (L.N == 0) return OP2B_OK;
    const int block = 128;
    constexpr int SPLIT = 2;
    const int64_t grid = std::min<int64_t>((L.N * SPLIT + block - 1) / block, (int64_t)c->sm_count * 64);
    k_gg_ff<SPLIT><<<(unsigned)grid, block, 0, c->stream>>>(
        sp->rowptr, sp->ends, L.m0, L.m1, (const float2*)L.q, L.ldq, (const float2*)L.n, L.ldn,
        (float2*)L.t0, L.ldt0, L.N, !(L.flags & OP2B_ZERO_INC));
    return c->launched("green_gauss_ff");
  }
  if (L.loop != OP2B_LOOP_FLUX2)
    return c->fail(OP2B_ETYPE, "float-float dats: only the Green-Gauss loop, the second-order flux, "
                               "its adjoint and the viscous flux have float-float variants");
  BodyFlux2FF b{(const float2*)L.q, L.ldq, (const float2*)L.G, L.ldG, (const float2*)L.n, L.ldn,
                (const float2*)L.dx, L.lddx, gas_ff(L.gamma, L.eps)};
  Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
  return run_body(c, b, L, s, tg);
}

}  // namespace op2b
