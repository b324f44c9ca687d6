// Node limiters of the Barth-Jespersen and Venkatakrishnan type and the flux
// with node-limited reconstruction (the alternative to the van Albada edge
// limiter of the second-order flux):
//
//   min/max     qmin_i, qmax_i over node i and its edge neighbours
//   limiter     per edge end, D2 = G_i . d / 2 (d = dx at the first end, -dx
//               at the second), D1 = qmax_i - q_i (D2 > 0) or qmin_i - q_i;
//               phi_e = min(1, D1/D2)  (Barth-Jespersen)  or
//               (D1^2 + eps2 + 2 D1 D2) / (D1^2 + 2 D2^2 + D1 D2 + eps2)
//               (Venkatakrishnan), 1 when D2 = 0; phi_i = min over the ends
//   flux        face states q_i + phi_i D2 at both ends, Rusanov flux
//
// The min/max and the limiter are reductions over each node's edge ends
// whose contributions depend on that node's own data, so they run as
// gathers: one thread per node walks its ends in the node-sorted edge-end
// list (the segmented plan) and keeps the reduction in registers.  Nothing
// is scattered, so there is no race to resolve and the result does not
// depend on the order of the ends.
#include <algorithm>
#include <type_traits>

#include "ff_math.cuh"
#include "launch.cuh"

namespace op2b {

// Doubles in an order-preserving int64 form (IEEE total order; -0 < +0):
// min / max then run on the integer units instead of the FP64 pipe.
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double unkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

// Sign tests and the comparison of two non-negative values: on the bit
// patterns for double (an FP64 comparison issues on the FP64 pipe, which
// GB300 runs at 1/64 of the FP32 rate), plain comparisons otherwise.
__device__ __forceinline__ bool is_zero(double x) {
  return ((__double2hiint(x) & 0x7fffffff) | __double2loint(x)) == 0;
}
__device__ __forceinline__ bool is_pos(double x) {
  return __double2hiint(x) >= 0 && !is_zero(x);
}
__device__ __forceinline__ bool less_nonneg(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}
template <typename T>
__device__ __forceinline__ bool is_zero(T x) {
  return x == T(0);
}
template <typename T>
__device__ __forceinline__ bool is_pos(T x) {
  return x > T(0);
}
template <typename T>
__device__ __forceinline__ bool less_nonneg(T a, T b) {
  return a < b;
}

template <typename T>
struct MinMaxAcc;
template <>
struct MinMaxAcc<double> {
  long long lo, hi;
  __device__ __forceinline__ void init(double v) { lo = hi = okey(v); }
  __device__ __forceinline__ void take(double v) {
    const long long k = okey(v);
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
  __device__ __forceinline__ double min() const { return unkey(lo); }
  __device__ __forceinline__ double max() const { return unkey(hi); }
};
template <>
struct MinMaxAcc<ffv> {
  ffv lo, hi;
  __device__ __forceinline__ void init(ffv v) { lo = hi = v; }
  __device__ __forceinline__ void take(ffv v) {
    lo = v < lo ? v : lo;
    hi = hi < v ? v : hi;
  }
  __device__ __forceinline__ ffv min() const { return lo; }
  __device__ __forceinline__ ffv max() const { return hi; }
};
template <>
struct MinMaxAcc<float> {
  float lo, hi;
  __device__ __forceinline__ void init(float v) { lo = hi = v; }
  __device__ __forceinline__ void take(float v) {
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
  __device__ __forceinline__ float min() const { return lo; }
  __device__ __forceinline__ float max() const { return hi; }
};

template <typename T>
__global__ void k_minmax(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ ends,
                         const int32_t* __restrict__ m0, const int32_t* __restrict__ m1,
                         const T* __restrict__ q, int64_t ldq, T* __restrict__ qmin,
                         int64_t ldmin, T* __restrict__ qmax, int64_t ldmax, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    MinMaxAcc<T> acc[6];
#pragma unroll
    for (int k = 0; k < 6; k++) acc[k].init(q[k * ldq + i]);
    const int64_t t1 = rowptr[i + 1];
    for (int64_t t = rowptr[i]; t < t1; t++) {
      const int32_t end = ends[t];
      const int64_t e = end >> 1;
      const int64_t j = (end & 1) ? m0[e] : m1[e];  // the other end
#pragma unroll
      for (int k = 0; k < 6; k++) acc[k].take(ldro(q + k * ldq + j));
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
      qmin[k * ldmin + i] = acc[k].min();
      qmax[k * ldmax + i] = acc[k].max();
    }
  }
}

// Barth-Jespersen needs only the largest positive and the most negative D2
// of each variable: for D1 >= 0 and D2 > 0 the correctly rounded D1/D2
// decreases as D2 grows, so min over the ends of D1/D2 = D1 / max D2 (and
// likewise on the negative side), two divisions per node and variable.
// Venkatakrishnan keeps the smallest phi_e as a (numerator, denominator)
// pair compared by cross-multiplication (both are >= 0) and divides once.
template <typename T, int KIND>
__global__ void k_limiter(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ ends,
                          const T* __restrict__ dx, int64_t lddx, const T* __restrict__ q,
                          int64_t ldq, const T* __restrict__ G, int64_t ldG,
                          const T* __restrict__ qmin, int64_t ldmin,
                          const T* __restrict__ qmax, int64_t ldmax, T eps2,
                          T* __restrict__ phi, int64_t ldphi, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    T g[18], d1p[6], d1m[6];
#pragma unroll
    for (int c = 0; c < 18; c++) g[c] = G[c * ldG + i];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const T qi = q[k * ldq + i];
      d1p[k] = qmax[k * ldmax + i] - qi;
      d1m[k] = qmin[k * ldmin + i] - qi;
    }
    // Barth-Jespersen: running max / min of D2; Venkatakrishnan: best pair,
    // with the per-node parts D1^2 + eps2 and 2 D1 of both signs formed once
    MinMaxAcc<T> ext[6];
    T bn[6], bd[6], ap[6], am[6], tp[6], tm[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      ext[k].init(T(0));
      bn[k] = T(1);
      bd[k] = T(0);  // ratio +inf: the first end always replaces it
      if constexpr (KIND != OP2B_LIM_BARTH_JESPERSEN) {
        ap[k] = fma(d1p[k], d1p[k], eps2);
        am[k] = fma(d1m[k], d1m[k], eps2);
        tp[k] = d1p[k] + d1p[k];
        tm[k] = d1m[k] + d1m[k];
      }
    }
    const int64_t t1 = rowptr[i + 1];
    for (int64_t t = rowptr[i]; t < t1; t++) {
      const int32_t end = ends[t];
      const int64_t e = end >> 1;
      T h[3] = {halve(ldro(dx + e)), halve(ldro(dx + lddx + e)), halve(ldro(dx + 2 * lddx + e))};
      if (end & 1) {
        h[0] = neg(h[0]);
        h[1] = neg(h[1]);
        h[2] = neg(h[2]);
      }
#pragma unroll
      for (int k = 0; k < 6; k++) {
        const T d2 = fma(g[3 * k + 2], h[2], fma(g[3 * k + 1], h[1], g[3 * k] * h[0]));
        if constexpr (KIND == OP2B_LIM_BARTH_JESPERSEN) {
          ext[k].take(d2);
        } else {
          // D1 takes the sign of D2, so every term below is >= 0; D2 = 0
          // gives phi_e = 1 (selected, not branched)
          const bool pos = is_pos(d2);
          const T d1 = pos ? d1p[k] : d1m[k];
          const T a = pos ? ap[k] : am[k];
          const T num0 = fma(pos ? tp[k] : tm[k], d2, a);
          const T den0 = fma(d2, fma(T(2), d2, d1), a);
          const bool zero = is_zero(d2);
          const T num = zero ? T(1) : num0, den = zero ? T(1) : den0;
          if (less_nonneg(num * bd[k], bn[k] * den)) {
            bn[k] = num;
            bd[k] = den;
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
      T f = T(1);
      if constexpr (KIND == OP2B_LIM_BARTH_JESPERSEN) {
        const T hi = ext[k].max(), lo = ext[k].min();
        if (hi > T(0)) f = fmin(f, d1p[k] / hi);
        if (lo < T(0)) f = fmin(f, d1m[k] / lo);
      } else {
        if (bd[k] != T(0)) f = bn[k] / bd[k];
      }
      phi[k * ldphi + i] = f;
    }
  }
}

// Flux with node-limited reconstruction.  v = q (6), G (18), phi (6).
template <typename T>
struct BodyFlux2Phi {
  using TN = T;
  // float-float: each edge's flux leaves the float-float Rusanov as FP64
  using TE = typename std::conditional<std::is_same<T, ffv>::value, double, T>::type;
  using TA = double;
  static constexpr int NIN = 30, OUT = 6, MODE = MODE_ANTI, DIM0 = 6;
  const T* q;
  int64_t ldq;
  const T* G;
  int64_t ldG;
  const T* phi;
  int64_t ldphi;
  const T* n;
  int64_t ldn;
  const T* dx;
  int64_t lddx;
  Gas<T> g;
  __device__ __forceinline__ void load(int64_t i, T* v) const {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ldro(q + k * ldq + i);
#pragma unroll
    for (int c = 0; c < 18; c++) v[6 + c] = ldro(G + c * ldG + i);
#pragma unroll
    for (int k = 0; k < 6; k++) v[24 + k] = ldro(phi + k * ldphi + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const T* vi, const T* vj, TE* oi,
                                       TE*) const {
    const T h[3] = {T(0.5) * ldro(dx + e), T(0.5) * ldro(dx + lddx + e),
                    T(0.5) * ldro(dx + 2 * lddx + e)};
    T qL[6], qR[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const T ai = fma(vi[8 + 3 * k], h[2], fma(vi[7 + 3 * k], h[1], vi[6 + 3 * k] * h[0]));
      const T aj = fma(vj[8 + 3 * k], h[2], fma(vj[7 + 3 * k], h[1], vj[6 + 3 * k] * h[0]));
      qL[k] = fma(vi[24 + k], ai, vi[k]);
      qR[k] = fma(neg(vj[24 + k]), aj, vj[k]);
    }
    const T nx = ldro(n + e), ny = ldro(n + ldn + e), nz = ldro(n + 2 * ldn + e);
    if constexpr (std::is_same<T, double>::value) {
      rusanov_f64(qL, qR, nx, ny, nz, g, oi);
    } else if constexpr (std::is_same<T, ffv>::value) {
      const GasFF gf{g.gamma.v, g.gm1.v, g.eps.v, g.two_eps.v};
      rusanov_ff(reinterpret_cast<const float2*>(qL), reinterpret_cast<const float2*>(qR), nx.v,
                 ny.v, nz.v, gf, oi);
    } else {
      rusanov(qL, qR, nx, ny, nz, g, oi);
    }
  }
};

int launch_lim(Ctx* c, const LoopLaunch& L, const Strategy& s) {
  Targets<double, 6> tg{(double*)L.t0, L.ldt0, (double*)L.t0, L.ldt0};
  if (L.prec == OP2B_PREC_FF) {
    Gas<ffv> g{ffv(L.gamma), ffv(L.gamma - 1.0), ffv(L.eps), ffv(2.0 * L.eps)};
    BodyFlux2Phi<ffv> b{(const ffv*)L.q,   L.ldq,   (const ffv*)L.G, L.ldG,
                        (const ffv*)L.phi, L.ldphi, (const ffv*)L.n, L.ldn,
                        (const ffv*)L.dx,  L.lddx,  g};
    return run_body(c, b, L, s, tg);
  }
  if (L.prec == OP2B_PREC_F64) {
    Gas<double> g{L.gamma, L.gamma - 1.0, L.eps, 2.0 * L.eps};
    BodyFlux2Phi<double> b{(const double*)L.q,   L.ldq,   (const double*)L.G, L.ldG,
                           (const double*)L.phi, L.ldphi, (const double*)L.n, L.ldn,
                           (const double*)L.dx,  L.lddx,  g};
    return run_body(c, b, L, s, tg);
  }
  Gas<float> g{(float)L.gamma, (float)(L.gamma - 1.0), (float)L.eps, (float)(2.0 * L.eps)};
  BodyFlux2Phi<float> b{(const float*)L.q,   L.ldq,   (const float*)L.G, L.ldG,
                        (const float*)L.phi, L.ldphi, (const float*)L.n, L.ldn,
                        (const float*)L.dx,  L.lddx,  g};
  return run_body(c, b, L, s, tg);
}

static unsigned node_grid(Ctx* c, int64_t N, int block) {
  return (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((N + block - 1) / block, (int64_t)c->sm_count * 32));
}

int node_minmax(Ctx* c, const DevSegPlan& sp, const int32_t* m0, const int32_t* m1, int type,
                const void* q, int64_t ldq, void* qmin, int64_t ldmin, void* qmax, int64_t ldmax,
                int64_t N) {
  if (N == 0) return OP2B_OK;
  const int block = 128;
  if (type == OP2B_F64)
    k_minmax<double><<<node_grid(c, N, block), block, 0, c->stream>>>(
        sp.rowptr, sp.ends, m0, m1, (const double*)q, ldq, (double*)qmin, ldmin,
        (double*)qmax, ldmax, N);
  else if (type == OP2B_FF)
    k_minmax<ffv><<<node_grid(c, N, block), block, 0, c->stream>>>(
        sp.rowptr, sp.ends, m0, m1, (const ffv*)q, ldq, (ffv*)qmin, ldmin, (ffv*)qmax, ldmax,
        N);
  else
    k_minmax<float><<<node_grid(c, N, block), block, 0, c->stream>>>(
        sp.rowptr, sp.ends, m0, m1, (const float*)q, ldq, (float*)qmin, ldmin, (float*)qmax,
        ldmax, N);
  return c->launched("minmax");
}

template <typename T, int KIND>
static void launch_limiter_t(Ctx* c, const DevSegPlan& sp, const LimArgs& a, int64_t N) {
  const int block = 128;
  k_limiter<T, KIND><<<node_grid(c, N, block), block, 0, c->stream>>>(
      sp.rowptr, sp.ends, (const T*)a.dx, a.lddx, (const T*)a.q, a.ldq, (const T*)a.G, a.ldG,
      (const T*)a.qmin, a.ldmin, (const T*)a.qmax, a.ldmax, (T)a.eps2, (T*)a.phi, a.ldphi, N);
}

int node_limiter(Ctx* c, const DevSegPlan& sp, int kind, int type, const LimArgs& a,
                 int64_t N) {
  if (N == 0) return OP2B_OK;
  const bool bj = kind == OP2B_LIM_BARTH_JESPERSEN;
  if (type == OP2B_F64) {
    if (bj) launch_limiter_t<double, OP2B_LIM_BARTH_JESPERSEN>(c, sp, a, N);
    else launch_limiter_t<double, OP2B_LIM_VENKATAKRISHNAN>(c, sp, a, N);
  } else if (type == OP2B_FF) {
    if (bj) launch_limiter_t<ffv, OP2B_LIM_BARTH_JESPERSEN>(c, sp, a, N);
    else launch_limiter_t<ffv, OP2B_LIM_VENKATAKRISHNAN>(c, sp, a, N);
  } else {
    if (bj) launch_limiter_t<float, OP2B_LIM_BARTH_JESPERSEN>(c, sp, a, N);
    else launch_limiter_t<float, OP2B_LIM_VENKATAKRISHNAN>(c, sp, a, N);
  }
  return c->launched("limiter");
}

}  // namespace op2b
