// Viscous flux (the analogue of the paper's `vfluxedge` loop, Table
// "loopperfmpi"; the paper gives no formula, the library implements the
// textbook Navier-Stokes edge flux):
//
//   node pass   W_i = (u, T, c, grad u / 2, grad T / 2, grad c / 2) from q, G
//   edge loop   face gradient g_f = gbar + ((phi_j - phi_i) - gbar . dx) dx/|dx|^2
//               (gbar the mean of the two nodal gradients) for u, T and c;
//               Fv = (0, tau n, (tau n) . u_f + kappa g_T . n, D g_c . n),
//               tau = mu (g_u + g_u^T - 2/3 div u I), u_f = (u_i + u_j)/2;
//               R_i -= Fv, R_j += Fv.
//
// The primitive variables and their gradients are formed once per node in
// the node pass instead of once per edge end (each node is an end of about
// 18 edges); the gradients are stored halved so that the edge loop's mean is
// one addition.  The FP64 edge loop is bound by the FP64 pipe (one
// reciprocal and about 110 FP64 instructions per edge), the FP32 variant by
// its memory traffic.
#include <algorithm>

#include <type_traits>

#include "ff_math.cuh"
#include "launch.cuh"

namespace op2b {

template <typename T>
__device__ __forceinline__ T recip_dd(T dd);

// ------------------------------------------------------------- node pass
// W layout (dim 20, component-major):
//   0..2 u, 3 T = p/rho, 4 c = q5,
//   5 + 3a + d  (d u_a / d x_d) / 2,  14 + d  (dT/dx_d) / 2,  17 + d  (dc/dx_d) / 2
template <typename T>
__global__ void k_viscous_prims(const T* __restrict__ q, int64_t ldq,
                                const T* __restrict__ G, int64_t ldG,
                                T* __restrict__ W, int64_t ldW, T gm1, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T rho = q[i];
    const T r = recip_dd(rho);
    const T hr = T(0.5) * r;
    T u[3];
#pragma unroll
    for (int a = 0; a < 3; a++) u[a] = q[(1 + a) * ldq + i] * r;
    const T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const T p = gm1 * (q[4 * ldq + i] - T(0.5) * rho * uu);
    const T Tt = p * r;
#pragma unroll
    for (int a = 0; a < 3; a++) W[a * ldW + i] = u[a];
    W[3 * ldW + i] = Tt;
    W[4 * ldW + i] = q[5 * ldq + i];
#pragma unroll
    for (int d = 0; d < 3; d++) {
      const T grho = G[d * ldG + i];
      T udm = T(0);
#pragma unroll
      for (int a = 0; a < 3; a++) {
        const T gm = G[(3 * (1 + a) + d) * ldG + i];
        udm = fma(u[a], gm, udm);
        W[(5 + 3 * a + d) * ldW + i] = (gm - u[a] * grho) * hr;
      }
      const T gp = gm1 * (G[(12 + d) * ldG + i] - udm + T(0.5) * uu * grho);
      W[(14 + d) * ldW + i] = (gp - Tt * grho) * hr;
      W[(17 + d) * ldW + i] = T(0.5) * G[(15 + d) * ldG + i];
    }
  }
}

// ------------------------------------------------------------- edge body
template <typename T>
__device__ __forceinline__ T recip_dd(T dd) {
  if constexpr (std::is_same<T, double>::value)
    return seedable(dd) ? recip2(dd) : 1.0 / dd;
  else if constexpr (std::is_same<T, float>::value)
    return 1.0f / dd;
  else
    return recip(dd);  // float-float
}

// One edge: oi receives -Fv components 1..5 (component 0 is zero and is not
// written); node j receives +Fv (MODE_ANTI).
template <typename T>
struct BodyVisc {
  using TN = T;
  using TE = T;
  using TA = double;
  static constexpr int NIN = 20, OUT = 5, MODE = MODE_ANTI, DIM0 = 5;
  const T* W;
  int64_t ldW;
  const T* n;
  int64_t ldn;
  const T* dx;
  int64_t lddx;
  T mu, kappa, diff;
  __device__ __forceinline__ void load(int64_t i, T* v) const {
#pragma unroll
    for (int c = 0; c < 20; c++) v[c] = ldro(W + c * ldW + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const T* vi, const T* vj, TE* oi,
                                       TE*) const {
    const T x[3] = {ldro(dx + e), ldro(dx + lddx + e), ldro(dx + 2 * lddx + e)};
    const T nn[3] = {ldro(n + e), ldro(n + ldn + e), ldro(n + 2 * ldn + e)};
    const T rdd = recip_dd(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    // face velocity gradient gu[a][d]
    T gu[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      T g[3];
#pragma unroll
      for (int d = 0; d < 3; d++) g[d] = vi[5 + 3 * a + d] + vj[5 + 3 * a + d];
      const T gdx = fma(g[2], x[2], fma(g[1], x[1], g[0] * x[0]));
      const T corr = ((vj[a] - vi[a]) - gdx) * rdd;
#pragma unroll
      for (int d = 0; d < 3; d++) gu[a][d] = fma(corr, x[d], g[d]);
    }
    // normal components of the face gradients of T and c
    const T dxn = fma(x[2], nn[2], fma(x[1], nn[1], x[0] * nn[0]));
    T gn[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const int o = 14 + 3 * s;
      const T g0 = vi[o] + vj[o], g1 = vi[o + 1] + vj[o + 1], g2 = vi[o + 2] + vj[o + 2];
      const T gdx = fma(g2, x[2], fma(g1, x[1], g0 * x[0]));
      const T gnn = fma(g2, nn[2], fma(g1, nn[1], g0 * nn[0]));
      const T corr = ((vj[3 + s] - vi[3 + s]) - gdx) * rdd;
      gn[s] = fma(corr, dxn, gnn);
    }
    // -tau n = -mu ((g_u + g_u^T) n - 2/3 div n)
    const T div23 = T(2.0 / 3.0) * (gu[0][0] + gu[1][1] + gu[2][2]);
    const T nmu = neg(mu);
    T tn[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      T s = neg(div23) * nn[a];
#pragma unroll
      for (int b = 0; b < 3; b++) s = fma(gu[a][b] + gu[b][a], nn[b], s);
      tn[a] = nmu * s;
    }
    // energy: (tau n) . (u_i + u_j)/2 + kappa g_T . n, both negated
    T en = tn[0] * (vi[0] + vj[0]);
    en = fma(tn[1], vi[1] + vj[1], en);
    en = fma(tn[2], vi[2] + vj[2], en);
    oi[0] = tn[0];
    oi[1] = tn[1];
    oi[2] = tn[2];
    oi[3] = fma(T(0.5), en, neg(kappa) * gn[0]);
    oi[4] = neg(diff) * gn[1];
  }
};

int launch_visc(Ctx* c, const LoopLaunch& L, const Strategy& s) {
  // R components 1..5 (component 0 of the viscous flux is zero)
  Targets<double, 5> tg{(double*)L.t0 + L.ldt0, L.ldt0, (double*)L.t0 + L.ldt0, L.ldt0};
  if (L.prec == OP2B_PREC_F64) {
    BodyVisc<double> b{(const double*)L.q, L.ldq, (const double*)L.n, L.ldn,
                       (const double*)L.dx, L.lddx, L.mu, L.kappa, L.diff};
    return run_body(c, b, L, s, tg);
  }
  if (L.prec == OP2B_PREC_FF) {
    BodyVisc<ffv> b{(const ffv*)L.q, L.ldq, (const ffv*)L.n, L.ldn, (const ffv*)L.dx, L.lddx,
                    ffv(L.mu), ffv(L.kappa), ffv(L.diff)};
    return run_body(c, b, L, s, tg);
  }
  BodyVisc<float> b{(const float*)L.q, L.ldq, (const float*)L.n, L.ldn,
                    (const float*)L.dx, L.lddx, (float)L.mu, (float)L.kappa, (float)L.diff};
  return run_body(c, b, L, s, tg);
}

int node_viscous_prims(Ctx* c, const void* q, int64_t ldq, const void* G, int64_t ldG,
                       void* W, int64_t ldW, int type, double gamma, int64_t N) {
  if (N == 0) return OP2B_OK;
  const int block = 256;
  const unsigned grid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((N + block - 1) / block, (int64_t)c->sm_count * 32));
  if (type == OP2B_F64)
    k_viscous_prims<double><<<grid, block, 0, c->stream>>>(
        (const double*)q, ldq, (const double*)G, ldG, (double*)W, ldW, gamma - 1.0, N);
  else if (type == OP2B_FF)
    k_viscous_prims<ffv><<<grid, block, 0, c->stream>>>(
        (const ffv*)q, ldq, (const ffv*)G, ldG, (ffv*)W, ldW, ffv(gamma - 1.0), N);
  else
    k_viscous_prims<float><<<grid, block, 0, c->stream>>>(
        (const float*)q, ldq, (const float*)G, ldG, (float*)W, ldW, (float)(gamma - 1.0), N);
  return c->launched("viscous_prims");
}

}  // namespace op2b
