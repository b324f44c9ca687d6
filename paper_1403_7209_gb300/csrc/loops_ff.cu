// Float-float edge loops (arithmetic on the FP32 units, ~47 significant
// bits, reading float-float shadows of the node and edge data):
//   second-order flux   each edge's flux converted to FP64 and added into
//                       the FP64 residual under any strategy;
//   flux adjoint        the templated reverse sweep (flux2_adj_t) for
//                       float-float, results converted to FP64;
//   flux tangent        the templated forward linearisation (flux2_tan_t),
//                       each edge's Fd converted to FP64;
//   Green-Gauss         the node gather of gg_gather.cuh (float-float sums).
// The viscous flux and the node limiters instantiate their own templates
// for float-float (loops_visc.cu, loops_lim.cu).
#include "ff_math.cuh"
#include "gg_gather.cuh"
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

// Tangent of the second-order flux in float-float: v = q (6), qd (6),
// G (18), Gd (18) as float-float shadows, nd the edge normals' tangent; each
// edge's Fd converted to FP64 and added into the FP64 target.
struct BodyFluxTanFF {
  using TN = ffv;
  using TE = double;
  using TA = double;
  static constexpr int NIN = 48, OUT = 6, MODE = MODE_ANTI, DIM0 = 6;
  const ffv* q;
  int64_t ldq;
  const ffv* qd;
  int64_t ldqd;
  const ffv* G;
  int64_t ldG;
  const ffv* Gd;
  int64_t ldGd;
  const ffv* n;
  int64_t ldn;
  const ffv* nd;
  int64_t ldnd;
  const ffv* dx;
  int64_t lddx;
  ffv gamma, gm1, eps, two_eps;
  __device__ __forceinline__ void load(int64_t i, ffv* v) const {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ldro(q + k * ldq + i);
#pragma unroll
    for (int k = 0; k < 6; k++) v[6 + k] = ldro(qd + k * ldqd + i);
#pragma unroll
    for (int c = 0; c < 18; c++) v[12 + c] = ldro(G + c * ldG + i);
#pragma unroll
    for (int c = 0; c < 18; c++) v[30 + c] = ldro(Gd + c * ldGd + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const ffv* vi, const ffv* vj, double* oi,
                                       double*) const {
    ffv Fd[6];
    flux2_tan_t(vi, vj, ldro(dx + e), ldro(dx + lddx + e), ldro(dx + 2 * lddx + e), ldro(n + e),
                ldro(n + ldn + e), ldro(n + 2 * ldn + e), ldro(nd + e), ldro(nd + ldnd + e),
                ldro(nd + 2 * ldnd + e), gamma, gm1, eps, two_eps, Fd);
#pragma unroll
    for (int k = 0; k < 6; k++) oi[k] = (double)Fd[k];
  }
};

int launch_ff(Ctx* c, const LoopLaunch& L, const Strategy& s) {
  if (L.loop == OP2B_LOOP_FLUX2_TAN) {
    BodyFluxTanFF b{(const ffv*)L.q,  L.ldq,  (const ffv*)L.qd, L.ldqd, (const ffv*)L.G,
                    L.ldG,            (const ffv*)L.Gd,         L.ldGd, (const ffv*)L.n,
                    L.ldn,            (const ffv*)L.nd,         L.ldnd, (const ffv*)L.dx,
                    L.lddx,           ffv(L.gamma),             ffv(L.gamma - 1.0),
                    ffv(L.eps),       ffv(2.0 * L.eps)};
    Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
    return run_body(c, b, L, s, tg);
  }
  if (L.loop == OP2B_LOOP_FLUX2_ADJ) {
    BodyFluxAdjFF b{(const ffv*)L.lam, L.ldl, (const ffv*)L.q, L.ldq, (const ffv*)L.G, L.ldG,
                    (const ffv*)L.n, L.ldn, (const ffv*)L.dx, L.lddx, (double*)L.direct,
                    L.lddirect, ffv(L.gamma), ffv(L.gamma - 1.0), ffv(L.eps), ffv(2.0 * L.eps)};
    Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t1, L.ldt1};
    return run_body(c, b, L, s, tg);
  }
  if (L.loop == OP2B_LOOP_GREEN_GAUSS) return launch_gg_gather<ffv, 2>(c, L, 128);
  if (L.loop != OP2B_LOOP_FLUX2)
    return c->fail(OP2B_ETYPE, "float-float dats: no float-float variant of this loop (Green-Gauss, "
                               "second-order flux, its adjoint and tangent, limited and viscous "
                               "fluxes have one)");
  BodyFlux2FF b{(const float2*)L.q, L.ldq, (const float2*)L.G, L.ldG, (const float2*)L.n, L.ldn,
                (const float2*)L.dx, L.lddx, gas_ff(L.gamma, L.eps)};
  Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
  return run_body(c, b, L, s, tg);
}

}  // namespace op2b
