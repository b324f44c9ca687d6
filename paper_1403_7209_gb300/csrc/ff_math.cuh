// Float-float arithmetic and the second-order flux computed in it.
//
// GB300 executes FP64 at 1/64 of its FP32 rate, so an edge loop whose
// arithmetic is FP64 is bound by the FP64 pipe long before HBM.  A
// float-float number is the unevaluated sum hi + lo of two floats with
// |lo| of the order of ulp(hi): about 47 significant bits carried by FP32
// instructions.  The error-free building blocks are Knuth's two-sum, Dekker's
// fast two-sum (|a| >= |b|) and the FMA two-product (p = a b rounded,
// e = fma(a, b, -p) exactly a b - p); the operations follow the
// double-double of Hida, Li and Bailey (2001) with float limbs, in their
// "sloppy" forms: each operation's error is a small multiple of 2^-47 times
// the magnitude of its operands, which keeps the flux within ~1e-14 of the
// FP64 definition relative to the size of its terms.
//
// Storage: one float2 per value (x = hi, y = lo), 8 bytes like a double.
// Range: values of magnitude below 2^-126 convert to zero; values of
// magnitude 2^128 or more become infinite, as do intermediate results
// beyond the float range.
//
// Every primitive uses the explicitly rounded intrinsics (__fadd_rn, ...),
// which the compiler never contracts into FMAs: the error-free transforms
// rely on each operation being rounded exactly as written.
#pragma once
#include <cstdint>

#include "edge_math.cuh"

namespace op2b {

// ------------------------------------------------------------ conversions

// double -> float-float: hi = the top 24 significant bits of x (truncated,
// integer operations), lo = the remaining 29 bits rounded to a float
// (24 significant bits, round to nearest) and scaled exactly.  Relative
// error at most 2^-48 for |x| in [2^-75, 2^128) (below 2^-75 lo may lose
// bits to the float subnormal range); |x| below 2^-126 becomes 0, 2^128 and
// above infinite.
__device__ __forceinline__ float2 ff_of_f64(double x) {
  const unsigned hw = (unsigned)__double2hiint(x);
  const unsigned lw = (unsigned)__double2loint(x);
  const unsigned sign = hw & 0x80000000u;
  const unsigned ax = hw & 0x7fffffffu;
  const unsigned ex = ax >> 20;  // biased double exponent
  // hi: exponent re-biased from 1023 to 127, fraction bits 51..29
  unsigned hb = sign | __funnelshift_l(lw, ax - 0x38000000u, 3);
  // lo = (fraction bits 28..0) x 2^(E-52), E = ex - 1023: the 29-bit
  // integer rounded to a float, times 2^(E-52) -- for small x as
  // 2^(E-52+64) and then 2^-64, so that each factor is a normal float
  const float rem = __uint2float_rn(lw & 0x1fffffffu);
  const bool big = ex >= 949u;
  const float s1 = __uint_as_float((big ? ex - 948u : ex - 884u) << 23);
  float lo = __fmul_rn(__fmul_rn(rem, s1), big ? 1.0f : 0x1p-64f);
  lo = __uint_as_float(__float_as_uint(lo) | sign);
  const unsigned inf_nan = sign | 0x7f800000u |
                           ((ex == 2047u && ((ax & 0xfffffu) | lw)) ? 0x400000u : 0u);
  hb = ex > 1150u ? inf_nan : (ex >= 897u ? hb : sign);
  lo = (ex >= 897u && ex <= 1150u) ? lo : 0.0f;
  return make_float2(__uint_as_float(hb), lo);
}

// float-float -> double: both limbs exactly (integer re-biasing), one FP64
// addition.  The general conversion (subnormal, infinite and NaN limbs) is
// branched to only for the lanes that need it.
__device__ __forceinline__ double f64_of_ff(float2 a) {
  if (normal_or_zero(a.x) && normal_or_zero(a.y))
    return f64_of_normal(a.x) + f64_of_normal(a.y);
  return f64_exact(a.x) + f64_exact(a.y);
}

// ---------------------------------------------------- error-free blocks

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ float2 ff_fast(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// ------------------------------------------------------------ operations

__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  const float2 s = ff_two_sum(a.x, b.x);
  return ff_fast(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}

__device__ __forceinline__ float2 ff_sub(float2 a, float2 b) { return ff_add(a, ff_neg(b)); }

// Products are returned as the pair (p, e) without the final fast two-sum:
// a product cannot cancel, so |e| stays within about 2^-23 |p| (the
// rounding error of p plus the two cross terms), close enough to
// normalised for every operation here, all of which take such pairs (the
// additions renormalise).
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return make_float2(p, e);
}

__device__ __forceinline__ float2 ff_sqr(float2 a) {
  const float p = __fmul_rn(a.x, a.x);
  float e = __fmaf_rn(a.x, a.x, -p);
  e = __fmaf_rn(__fadd_rn(a.x, a.x), a.y, e);
  return make_float2(p, e);
}

// a b + c with one rounding of the leading parts
__device__ __forceinline__ float2 ff_fma(float2 a, float2 b, float2 c) {
  const float p = __fmul_rn(a.x, b.x);
  const float pe = __fmaf_rn(a.x, b.x, -p);
  const float2 s = ff_two_sum(p, c.x);
  float e = __fadd_rn(s.y, __fadd_rn(pe, c.y));
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return ff_fast(s.x, e);
}

// exact scaling by a power of two
__device__ __forceinline__ float2 ff_scale(float2 a, float s) {
  return make_float2(__fmul_rn(a.x, s), __fmul_rn(a.y, s));
}

__device__ __forceinline__ float ff_rcp_seed(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// a / b: FP32 quotient from the reciprocal seed, corrected once with the
// float-float remainder a - b q1 (relative error about 2^-44)
__device__ __forceinline__ float2 ff_div(float2 a, float2 b) {
  const float y = ff_rcp_seed(b.x);
  const float q1 = __fmul_rn(a.x, y);
  const float p = __fmul_rn(b.x, q1);
  const float pe = __fmaf_rn(b.x, q1, -p);
  float r = __fsub_rn(__fsub_rn(a.x, p), pe);
  r = __fadd_rn(r, __fmaf_rn(-b.y, q1, a.y));
  return ff_fast(q1, __fmul_rn(r, y));
}

// a / b as the unnormalised pair (q1, r y): |r y| is about 2^-22 |q1|, close
// enough to normalised for an operand of ff_add, which renormalises with a
// full two-sum (saves the fast two-sum of ff_div)
__device__ __forceinline__ float2 ff_div_raw(float2 a, float2 b) {
  const float y = ff_rcp_seed(b.x);
  const float q1 = __fmul_rn(a.x, y);
  const float p = __fmul_rn(b.x, q1);
  const float pe = __fmaf_rn(b.x, q1, -p);
  float r = __fsub_rn(__fsub_rn(a.x, p), pe);
  r = __fadd_rn(r, __fmaf_rn(-b.y, q1, a.y));
  return make_float2(q1, __fmul_rn(r, y));
}

// 1 / b
__device__ __forceinline__ float2 ff_recip(float2 b) {
  const float y = ff_rcp_seed(b.x);
  const float p = __fmul_rn(b.x, y);
  const float pe = __fmaf_rn(b.x, y, -p);
  float r = __fsub_rn(__fsub_rn(1.0f, p), pe);
  r = __fmaf_rn(-b.y, y, r);
  return ff_fast(y, __fmul_rn(r, y));
}

// sqrt(x), x > 0: FP32 root from the reciprocal square-root seed, corrected
// once with the float-float remainder x - s1^2
__device__ __forceinline__ float2 ff_sqrt(float2 x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.x));
  const float s1 = __fmul_rn(x.x, r);
  const float p = __fmul_rn(s1, s1);
  const float pe = __fmaf_rn(s1, s1, -p);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.x, p), pe), x.y);
  return ff_fast(s1, __fmul_rn(d, __fmul_rn(0.5f, r)));
}

__device__ __forceinline__ float2 ff_abs(float2 a) { return a.x < 0.0f ? ff_neg(a) : a; }

// a >= b by the sign of the renormalised difference: correct for
// unnormalised operands too (products), whose hi parts alone may order
// them wrongly when they are within ~2^-23 of each other
__device__ __forceinline__ bool ff_ge(float2 a, float2 b) {
  return ff_sub(a, b).x >= 0.0f;
}

// host-side split of a double constant
struct GasFF {
  float2 gamma, gm1, eps, two_eps;
};

inline float2 ff_split_host(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

// A float-float value with arithmetic operators, so that loop bodies and
// node loops written for a scalar type T (double, float) also instantiate
// for float-float.  Conversions: from double (device: ff_of_f64; host: the
// rounded split) and to double (f64_of_ff, device only).
struct ffv {
  float2 v;
  ffv() = default;
  __host__ __device__ __forceinline__ explicit ffv(float2 x) : v(x) {}
  __host__ __device__ __forceinline__ explicit ffv(double x) {
#ifdef __CUDA_ARCH__
    v = ff_of_f64(x);
#else
    v = ff_split_host(x);
#endif
  }
  __device__ __forceinline__ explicit operator double() const { return f64_of_ff(v); }
};
__device__ __forceinline__ ffv operator+(ffv a, ffv b) { return ffv(ff_add(a.v, b.v)); }
__device__ __forceinline__ ffv operator-(ffv a, ffv b) { return ffv(ff_sub(a.v, b.v)); }
__device__ __forceinline__ ffv operator-(ffv a) { return ffv(ff_neg(a.v)); }
__device__ __forceinline__ ffv operator*(ffv a, ffv b) { return ffv(ff_mul(a.v, b.v)); }
__device__ __forceinline__ ffv operator/(ffv a, ffv b) { return ffv(ff_div(a.v, b.v)); }
__device__ __forceinline__ ffv& operator+=(ffv& a, ffv b) { return a = a + b; }
// the float-float fma joins the global (double, float) overloads instead of
// hiding them inside this namespace
using ::fma;
__device__ __forceinline__ ffv fma(ffv a, ffv b, ffv c) { return ffv(ff_fma(a.v, b.v, c.v)); }
__device__ __forceinline__ ffv neg(ffv a) { return -a; }
__device__ __forceinline__ ffv recip(ffv a) { return ffv(ff_recip(a.v)); }
using ::sqrt;
using ::fabs;
__device__ __forceinline__ ffv sqrt(ffv a) { return ffv(ff_sqrt(a.v)); }
__device__ __forceinline__ ffv fabs(ffv a) { return ffv(ff_abs(a.v)); }
__device__ __forceinline__ bool operator>=(ffv a, ffv b) { return ff_ge(a.v, b.v); }
// order of float-float values: the sign of the renormalised difference
// (see ff_ge)
__device__ __forceinline__ bool operator<(ffv a, ffv b) { return ff_sub(a.v, b.v).x < 0.0f; }
__device__ __forceinline__ bool operator>(ffv a, ffv b) { return b < a; }
__device__ __forceinline__ bool operator==(ffv a, ffv b) {
  return a.v.x == b.v.x && a.v.y == b.v.y;
}
__device__ __forceinline__ bool operator!=(ffv a, ffv b) { return !(a == b); }
using ::fmin;
__device__ __forceinline__ ffv fmin(ffv a, ffv b) { return b < a ? b : a; }
// sign(x) v with sign(0) = 0
__device__ __forceinline__ ffv sign_times(ffv x, ffv v) {
  return x.v.x > 0.0f ? v : (x.v.x < 0.0f ? -v : ffv(make_float2(0.0f, 0.0f)));
}
__device__ __forceinline__ ffv ffk(float f) { return ffv(make_float2(f, 0.0f)); }
template <>
__device__ __forceinline__ ffv ldro<ffv>(const ffv* p) {
  return ffv(__ldg(reinterpret_cast<const float2*>(p)));
}

inline GasFF gas_ff(double gamma, double eps) {
  return {ff_split_host(gamma), ff_split_host(gamma - 1.0), ff_split_host(eps),
          ff_split_host(2.0 * eps)};
}

// ------------------------------------------------- second-order flux

// Rusanov flux of the face states (as rusanov() / the oracle: F = (f(qL).n +
// f(qR).n)/2 - s (qR - qL)/2, s the larger of |u.n| + a|n| of the two
// states, ties to the left), every operation in float-float; F is returned
// in FP64.
__device__ __forceinline__ void rusanov_ff(const float2* qL, const float2* qR, float2 nx,
                                           float2 ny, float2 nz, const GasFF& g, double* F) {
  const float2 gnn = ff_mul(g.gamma, ff_fma(nz, nz, ff_fma(ny, ny, ff_sqr(nx))));
  float2 f[2][6], lam[2];
#pragma unroll
  for (int sd = 0; sd < 2; sd++) {
    const float2* q = sd ? qR : qL;
    const float2 rr = ff_recip(q[0]);
    const float2 mn = ff_fma(q[3], nz, ff_fma(q[2], ny, ff_mul(q[1], nx)));
    const float2 un = ff_mul(mn, rr);
    const float2 mm = ff_fma(q[3], q[3], ff_fma(q[2], q[2], ff_sqr(q[1])));
    const float2 p = ff_mul(g.gm1, ff_sub(q[4], ff_scale(ff_mul(mm, rr), 0.5f)));
    const float2 x = ff_mul(ff_mul(p, rr), gnn);  // (a |n|)^2
    lam[sd] = ff_add(ff_abs(un), ff_sqrt(x));
    f[sd][0] = mn;
    f[sd][1] = ff_fma(q[1], un, ff_mul(p, nx));
    f[sd][2] = ff_fma(q[2], un, ff_mul(p, ny));
    f[sd][3] = ff_fma(q[3], un, ff_mul(p, nz));
    f[sd][4] = ff_mul(ff_add(q[4], p), un);
    f[sd][5] = ff_mul(q[5], un);
  }
  const float2 s = ff_ge(lam[0], lam[1]) ? lam[0] : lam[1];
#pragma unroll
  for (int k = 0; k < 6; k++)
    F[k] = f64_of_ff(ff_scale(ff_fma(ff_neg(s), ff_sub(qR[k], qL[k]), ff_add(f[0][k], f[1][k])),
                              0.5f));
}

// van Albada-limited reconstruction (phi(a, b) = (a + b)(ab + eps) /
// (a^2 + b^2 + 2 eps), the same rational function as van_albada()) and the
// Rusanov flux of the face states.  vi, vj: q (6) then G (18, component
// 3k+d) of the two ends; dx = x_j - x_i.
__device__ __forceinline__ void flux2_ff(const float2* vi, const float2* vj, float2 dx,
                                         float2 dy, float2 dz, float2 nx, float2 ny, float2 nz,
                                         const GasFF& g, double* F) {
  float2 qL[6], qR[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const float2 b = ff_sub(vj[k], vi[k]);
    const float2 ai = ff_fma(vi[8 + 3 * k], dz, ff_fma(vi[7 + 3 * k], dy, ff_mul(vi[6 + 3 * k], dx)));
    const float2 aj = ff_fma(vj[8 + 3 * k], dz, ff_fma(vj[7 + 3 * k], dy, ff_mul(vj[6 + 3 * k], dx)));
    const float2 b2e = ff_fma(b, b, g.two_eps);
    const float2 phi_i = ff_div_raw(ff_mul(ff_add(ai, b), ff_fma(ai, b, g.eps)), ff_fma(ai, ai, b2e));
    const float2 phi_j = ff_div_raw(ff_mul(ff_add(aj, b), ff_fma(aj, b, g.eps)), ff_fma(aj, aj, b2e));
    qL[k] = ff_add(vi[k], ff_scale(phi_i, 0.5f));
    qR[k] = ff_sub(vj[k], ff_scale(phi_j, 0.5f));
  }
  rusanov_ff(qL, qR, nx, ny, nz, g, F);
}

// ------------------------------------------- adjoint of the second-order flux
// The reverse sweep of flux2 (the same steps as flux2_adj_f64: face states
// recomputed from q, G, n, dx, the Rusanov flux reversed side by side, the
// van Albada limiter's partial derivatives), written for a scalar type T
// with operators and instantiated for float-float.  Plain reciprocals and
// square roots instead of the FP64 batching; non-smooth points as in the
// FP64 sweep: d|x|/dx = sign(x) (0 at 0), the max picks L on ties.

template <typename T>
struct SideStateT {
  T rr, un, mm, p, a, ra;  // 1/rho, u.n, |m|^2, p, sound speed, 1/a
};

template <typename T>
__device__ __forceinline__ T side_state_t(const T* q, T nx, T ny, T nz, T rr, T nn, T gamma,
                                          T gm1, SideStateT<T>& s) {
  s.rr = rr;
  s.un = fma(q[3], nz, fma(q[2], ny, q[1] * nx)) * rr;
  s.mm = fma(q[3], q[3], fma(q[2], q[2], q[1] * q[1]));
  s.p = gm1 * (q[4] - ffk(0.5f) * s.mm * rr);
  s.a = sqrt(gamma * s.p * rr);
  s.ra = recip(s.a);
  return fabs(s.un) + s.a * nn;  // wave speed
}

// fb = adjoint of f(q).n (6), lamb = adjoint of the side's wave speed
template <typename T>
__device__ __forceinline__ void side_reverse_t(const T* q, T nx, T ny, T nz,
                                               const SideStateT<T>& s, T nn, T rn, T gamma,
                                               T gm1, const T* fb, T lamb, T* qb, T* nb) {
  const T half = ffk(0.5f);
  T unb = sign_times(s.un, lamb);
  const T ab = lamb * nn;
  const T rnb = lamb * s.a * rn;  // d|n|/dn = n / |n|
#pragma unroll
  for (int k = 0; k < 6; k++) {
    qb[k] = fma(fb[k], s.un, qb[k]);
    unb = fma(fb[k], q[k], unb);
  }
  unb = fma(fb[4], s.p, unb);
  T pb = fma(fb[3], nz, fma(fb[2], ny, fma(fb[1], nx, fb[4] * s.un)));
  pb = fma(half * gamma * ab, s.rr * s.ra, pb);  // a = sqrt(gamma p / rho)
  const T gpb = gm1 * pb;
  const T ur = unb * s.rr;
  const T gpr = gpb * s.rr;
  const T n3[3] = {nx, ny, nz};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    nb[d] = fma(fb[1 + d], s.p, fma(rnb, n3[d], fma(ur, q[1 + d], nb[d])));
    qb[1 + d] = fma(-gpr, q[1 + d], fma(ur, n3[d], qb[1 + d]));
  }
  qb[4] = qb[4] + gpb;
  // rho enters through 1/rho in u.n, p and a
  qb[0] = qb[0] + fma(half * gpr, s.mm * s.rr, fma(-(half * ab), s.a * s.rr, -(ur * s.un)));
}

template <typename T>
__device__ __forceinline__ void rusanov_reverse_t(const T* qL, const T* qR, T nx, T ny, T nz,
                                                  T gamma, T gm1, const T* w, T* qLb, T* qRb,
                                                  T* nb) {
  const T half = ffk(0.5f);
  const T nn = sqrt(fma(nz, nz, fma(ny, ny, nx * nx)));
  const T rn = recip(nn);
  SideStateT<T> sL, sR;
  const T lL = side_state_t(qL, nx, ny, nz, recip(qL[0]), nn, gamma, gm1, sL);
  const T lR = side_state_t(qR, nx, ny, nz, recip(qR[0]), nn, gamma, gm1, sR);
  const bool left = lL >= lR;
  const T hs = half * (left ? lL : lR);
  T fb[6];
  T sb = ffk(0.0f);
#pragma unroll
  for (int k = 0; k < 6; k++) {
    fb[k] = half * w[k];
    sb = fma(w[k], qR[k] - qL[k], sb);
    qRb[k] = fma(-hs, w[k], qRb[k]);
    qLb[k] = fma(hs, w[k], qLb[k]);
  }
  sb = -(half * sb);
  const T zero = ffk(0.0f);
  side_reverse_t(qL, nx, ny, nz, sL, nn, rn, gamma, gm1, fb, left ? sb : zero, qLb, nb);
  side_reverse_t(qR, nx, ny, nz, sR, nn, rn, gamma, gm1, fb, left ? zero : sb, qRb, nb);
}

// Adjoint of the second-order flux of edge (i, j).  vi, vj: lam (6), q (6),
// G (18).  oi, oj: qbar (6) then Gbar (18) of each end; nb: nbar (3).
template <typename T>
__device__ __forceinline__ void flux2_adj_t(const T* vi, const T* vj, T dx, T dy, T dz, T nx,
                                            T ny, T nz, T gamma, T gm1, T eps, T two_eps, T* oi,
                                            T* oj, T* nb) {
  const T half = ffk(0.5f);
  const T* qi = vi + 6;
  const T* qj = vj + 6;
  const T* Gi = vi + 12;
  const T* Gj = vj + 12;
  T qL[6], qR[6], pa[12], pb[12];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const T b = qj[k] - qi[k];
    const T be = fma(b, b, eps);
    const T b2e = fma(b, b, two_eps);
    const T b2 = b + b;
    const T a[2] = {fma(Gi[3 * k + 2], dz, fma(Gi[3 * k + 1], dy, Gi[3 * k] * dx)),
                    fma(Gj[3 * k + 2], dz, fma(Gj[3 * k + 1], dy, Gj[3 * k] * dx))};
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
      const T x = a[sd];
      const T rd = recip(fma(x, x, b2e));
      const T phi = (x + b) * fma(x, b, eps) * rd;
      // d phi / da = (b^2 + eps + 2a(b - phi)) / D,
      // d phi / db = (a^2 + eps + 2b(a - phi)) / D
      pa[2 * k + sd] = fma(x + x, b - phi, be) * rd;
      pb[2 * k + sd] = fma(b2, x - phi, fma(x, x, eps)) * rd;
      if (sd == 0) qL[k] = fma(half, phi, qi[k]);
      else qR[k] = fma(-half, phi, qj[k]);
    }
  }
  T w[6], qLb[6], qRb[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    w[k] = vi[k] - vj[k];
    qLb[k] = ffk(0.0f);
    qRb[k] = ffk(0.0f);
  }
  nb[0] = nb[1] = nb[2] = ffk(0.0f);
  rusanov_reverse_t(qL, qR, nx, ny, nz, gamma, gm1, w, qLb, qRb, nb);
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const T phib = half * qLb[k], phjb = -(half * qRb[k]);
    const T aib = phib * pa[2 * k], ajb = phjb * pa[2 * k + 1];
    const T bb = fma(phib, pb[2 * k], phjb * pb[2 * k + 1]);
    oi[k] = qLb[k] - bb;
    oj[k] = qRb[k] + bb;
    oi[6 + 3 * k] = aib * dx;
    oi[7 + 3 * k] = aib * dy;
    oi[8 + 3 * k] = aib * dz;
    oj[6 + 3 * k] = ajb * dx;
    oj[7 + 3 * k] = ajb * dy;
    oj[8 + 3 * k] = ajb * dz;
  }
}

// ------------------------------------------- tangent of the second-order flux
// Forward-mode linearisation in the direction (qd, Gd, nd), dx fixed: the
// same steps as flux2_tan_f64 (side by side: f(q).n, its tangent, the wave
// speed and its tangent; the limiter's partial derivatives), written for a
// scalar type T with operators and instantiated for float-float.
// Non-smooth points as in the FP64 sweep: d|x|/dx = sign(x) (0 at 0), the
// max picks L on ties.

template <typename T>
__device__ __forceinline__ void side_tangent_t(const T* q, const T* qd, T nx, T ny, T nz, T ndx,
                                               T ndy, T ndz, T rr, T nn, T nnd, T gamma, T gm1,
                                               T* f, T* fd, T& lam, T& lamd) {
  const T half = ffk(0.5f);
  const T mn = fma(q[3], nz, fma(q[2], ny, q[1] * nx));
  const T mnd = fma(qd[3], nz, fma(qd[2], ny, fma(qd[1], nx,
                fma(q[3], ndz, fma(q[2], ndy, q[1] * ndx)))));
  const T un = mn * rr;
  const T und = fma(-un, qd[0], mnd) * rr;  // (mnd - un rhod) / rho
  const T mm = fma(q[3], q[3], fma(q[2], q[2], q[1] * q[1]));
  const T mmd = ffk(2.0f) * fma(q[3], qd[3], fma(q[2], qd[2], q[1] * qd[1]));
  const T hgm1 = half * gm1;
  const T p = gm1 * (q[4] - half * mm * rr);
  // pd = (gamma-1) (Ed - mmd/(2 rho) + mm rhod / (2 rho^2))
  const T pd = fma(gm1, qd[4], hgm1 * rr * fma(mm * rr, qd[0], -mmd));
  const T a = sqrt(gamma * p * rr);
  const T ra = recip(a);
  // 2 a ad = (gamma pd - a^2 rhod) / rho
  const T ad = half * ra * rr * fma(-(a * a), qd[0], gamma * pd);
  lam = fabs(un) + a * nn;
  lamd = sign_times(un, und) + fma(ad, nn, a * nnd);
#pragma unroll
  for (int k = 0; k < 6; k++) {
    f[k] = q[k] * un;
    fd[k] = fma(qd[k], un, q[k] * und);
  }
  const T n3[3] = {nx, ny, nz}, nd3[3] = {ndx, ndy, ndz};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    f[1 + d] = fma(p, n3[d], f[1 + d]);
    fd[1 + d] = fma(pd, n3[d], fma(p, nd3[d], fd[1 + d]));
  }
  f[4] = fma(p, un, f[4]);
  fd[4] = fma(pd, un, fma(p, und, fd[4]));
}

template <typename T>
__device__ __forceinline__ void rusanov_tangent_t(const T* qL, const T* qLd, const T* qR,
                                                  const T* qRd, T nx, T ny, T nz, T ndx, T ndy,
                                                  T ndz, T gamma, T gm1, T* Fd) {
  const T half = ffk(0.5f);
  const T nn = sqrt(fma(nz, nz, fma(ny, ny, nx * nx)));
  const T rn = recip(nn);
  const T nnd = fma(nz, ndz, fma(ny, ndy, nx * ndx)) * rn;
  T fL[6], fLd[6], fR[6], fRd[6], lL, lLd, lR, lRd;
  side_tangent_t(qL, qLd, nx, ny, nz, ndx, ndy, ndz, recip(qL[0]), nn, nnd, gamma, gm1, fL, fLd,
                 lL, lLd);
  side_tangent_t(qR, qRd, nx, ny, nz, ndx, ndy, ndz, recip(qR[0]), nn, nnd, gamma, gm1, fR, fRd,
                 lR, lRd);
  const bool left = lL >= lR;
  const T hs = half * (left ? lL : lR), hsd = half * (left ? lLd : lRd);
#pragma unroll
  for (int k = 0; k < 6; k++)
    Fd[k] = fma(half, fLd[k] + fRd[k], -fma(hsd, qR[k] - qL[k], hs * (qRd[k] - qLd[k])));
}

// vi, vj: q (6), qd (6), G (18), Gd (18); Fd: the flux's tangent (6)
template <typename T>
__device__ __forceinline__ void flux2_tan_t(const T* vi, const T* vj, T dx, T dy, T dz, T nx,
                                            T ny, T nz, T ndx, T ndy, T ndz, T gamma, T gm1,
                                            T eps, T two_eps, T* Fd) {
  const T half = ffk(0.5f);
  const T *qi = vi, *qid = vi + 6, *Gi = vi + 12, *Gid = vi + 30;
  const T *qj = vj, *qjd = vj + 6, *Gj = vj + 12, *Gjd = vj + 30;
  T qL[6], qR[6], qLd[6], qRd[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const T b = qj[k] - qi[k];
    const T bd = qjd[k] - qid[k];
    const T be = fma(b, b, eps);
    const T b2e = fma(b, b, two_eps);
    const T b2 = b + b;
    const T a[2] = {fma(Gi[3 * k + 2], dz, fma(Gi[3 * k + 1], dy, Gi[3 * k] * dx)),
                    fma(Gj[3 * k + 2], dz, fma(Gj[3 * k + 1], dy, Gj[3 * k] * dx))};
    const T ad[2] = {fma(Gid[3 * k + 2], dz, fma(Gid[3 * k + 1], dy, Gid[3 * k] * dx)),
                     fma(Gjd[3 * k + 2], dz, fma(Gjd[3 * k + 1], dy, Gjd[3 * k] * dx))};
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
      const T x = a[sd];
      const T rd = recip(fma(x, x, b2e));
      const T phi = (x + b) * fma(x, b, eps) * rd;
      const T pa = fma(x + x, b - phi, be) * rd;
      const T pb = fma(b2, x - phi, fma(x, x, eps)) * rd;
      const T phid = fma(pa, ad[sd], pb * bd);
      if (sd == 0) {
        qL[k] = fma(half, phi, qi[k]);
        qLd[k] = fma(half, phid, qid[k]);
      } else {
        qR[k] = fma(-half, phi, qj[k]);
        qRd[k] = fma(-half, phid, qjd[k]);
      }
    }
  }
  rusanov_tangent_t(qL, qLd, qR, qRd, nx, ny, nz, ndx, ndy, ndz, gamma, gm1, Fd);
}

}  // namespace op2b
