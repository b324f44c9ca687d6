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
// Range: values of magnitude below 2^-126 convert to zero, below 2^-103 to
// hi alone (24 bits); values of magnitude 2^128 or more become infinite, as
// do intermediate results beyond the float range.
//
// Every primitive uses the explicitly rounded intrinsics (__fadd_rn, ...),
// which the compiler never contracts into FMAs: the error-free transforms
// rely on each operation being rounded exactly as written.
#pragma once
#include <cstdint>

#include "edge_math.cuh"

namespace op2b {

// ------------------------------------------------------------ conversions

// double -> float-float with integer operations only: hi = the top 24
// significant bits (truncated), lo = the next 23 bits.  Relative error
// below 2^-46 for |x| in [2^-103, 2^128).
__device__ __forceinline__ float2 ff_of_f64(double x) {
  const unsigned hw = (unsigned)__double2hiint(x);
  const unsigned lw = (unsigned)__double2loint(x);
  const unsigned sign = hw & 0x80000000u;
  const unsigned ax = hw & 0x7fffffffu;
  const unsigned ex = ax >> 20;  // biased double exponent
  // hi: exponent re-biased from 1023 to 127, fraction bits 51..29
  unsigned hb = sign | __funnelshift_l(lw, ax - 0x38000000u, 3);
  // lo = (fraction bits 28..6) x 2^(E-46), E = ex - 1023: built as
  // (2^(E-23) + m 2^(E-46)) - 2^(E-23), an exact float subtraction
  const unsigned m = (lw >> 6) & 0x7fffffu;
  const unsigned eb = (ex - 919u) << 23;
  const float f1 = __uint_as_float(sign | eb | m);
  const float f2 = __uint_as_float(sign | eb);
  float lo = __fsub_rn(f1, f2);
  const unsigned inf_nan = sign | 0x7f800000u |
                           ((ex == 2047u && ((ax & 0xfffffu) | lw)) ? 0x400000u : 0u);
  hb = ex > 1150u ? inf_nan : (ex >= 897u ? hb : sign);
  lo = (ex >= 920u && ex <= 1150u) ? lo : 0.0f;
  return make_float2(__uint_as_float(hb), lo);
}

// Exact float -> double for zero and normal floats only (integer
// re-biasing, no special cases).
__device__ __forceinline__ double f64_of_normal(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u, mag = b & 0x7fffffffu;
  const unsigned hi = mag ? (sign | ((mag >> 3) + 0x38000000u)) : sign;
  return __hiloint2double((int)hi, (int)(mag << 29));
}
__device__ __forceinline__ bool normal_or_zero(float f) {
  const unsigned mag = __float_as_uint(f) & 0x7fffffffu;
  return mag - 0x00800000u < 0x7f000000u || mag == 0u;
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

__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return ff_fast(p, e);
}

__device__ __forceinline__ float2 ff_sqr(float2 a) {
  const float p = __fmul_rn(a.x, a.x);
  float e = __fmaf_rn(a.x, a.x, -p);
  e = __fmaf_rn(__fadd_rn(a.x, a.x), a.y, e);
  return ff_fast(p, e);
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

// a >= b (hi parts first, then lo)
__device__ __forceinline__ bool ff_ge(float2 a, float2 b) {
  return a.x > b.x || (a.x == b.x && a.y >= b.y);
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

}  // namespace op2b
