// Per-edge arithmetic of the loops: Euler/Rusanov flux, van Albada-limited
// reconstruction, Green-Gauss contributions and the hand-written adjoints.
// Templated on the arithmetic type T (double, or float for the mixed path).
#pragma once
#include <cstdint>

namespace op2b {

template <typename T>
struct Gas {
  T gamma;    // ratio of specific heats
  T gm1;      // gamma - 1
  T eps;      // van Albada epsilon
  T two_eps;  // 2 eps
};

template <typename T>
__device__ __forceinline__ T ldro(const T* p) {
  return __ldg(p);
}

// -x by flipping the sign bit on the integer pipe (an FP64 negation that is
// not folded into another instruction would cost an FP64-pipe add)
__device__ __forceinline__ double neg(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}
__device__ __forceinline__ float neg(float x) {
  return __int_as_float(__float_as_int(x) ^ (int)0x80000000);
}

// x / 2 exactly, on the integer pipe for zero and for normal x whose half is
// normal (exponent field 2..2046: decrement it); the rest (subnormal, the
// smallest normals, infinity, NaN) takes the FP64 multiply.
__device__ __forceinline__ double half_exact(double x) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const unsigned ex = ((unsigned)hi >> 20) & 0x7ffu;
  const bool norm = ex - 2u < 2045u;
  const bool zero = ((hi & 0x7fffffff) | lo) == 0;
  if (__builtin_expect(norm || zero, 1))
    return norm ? __hiloint2double(hi - 0x00100000, lo) : x;
  return x * 0.5;
}

// x / 2 in the loop's arithmetic type (exact; integer route for double)
template <typename T>
__device__ __forceinline__ T halve(T x) {
  return T(0.5) * x;
}
template <>
__device__ __forceinline__ double halve<double>(double x) {
  return half_exact(x);
}

// Exact float -> double on the integer pipe (the conversion instruction runs
// at the FP64 rate): re-bias the exponent and move the mantissa.  Zero,
// subnormal, infinite and NaN inputs are handled with integer selects too,
// so no FP64-pipe instruction is issued on any path.
__device__ __forceinline__ double f64_exact(float f) {
  const unsigned b = (unsigned)__float_as_int(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned mag = b & 0x7fffffffu;
  // normal: exponent + (1023 - 127), mantissa moved up by 29 bits
  unsigned hi = sign | ((mag >> 3) + 0x38000000u);
  unsigned lo = mag << 29;
  // subnormal: normalise the mantissa (value m * 2^-149, m < 2^23)
  const int lz = __clz((int)mag) - 8;  // shift that brings the top bit to bit 23
  const unsigned mn = mag << (lz & 31);
  const unsigned hs = sign | ((unsigned)(897 - lz) << 20) | ((mn & 0x7fffffu) >> 3);
  const unsigned ls = mn << 29;
  // infinity / NaN: all-ones exponent, payload kept
  const unsigned hn = sign | 0x7ff00000u | ((mag & 0x7fffffu) >> 3);
  const bool normal = mag - 0x00800000u < 0x7f000000u;  // exponent field 1..254
  const bool inf_nan = mag >= 0x7f800000u;
  const bool zero = mag == 0u;
  hi = normal ? hi : (inf_nan ? hn : (zero ? sign : hs));
  lo = normal ? lo : (inf_nan ? lo : (zero ? 0u : ls));
  return __hiloint2double((int)hi, (int)lo);
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

// value of a per-edge result in the accumulation type of its target; a
// float goes the short integer route unless it is subnormal, infinite or NaN
template <typename TA, typename TE>
__device__ __forceinline__ TA to_acc(TE x) {
  if constexpr (sizeof(TA) == 8 && sizeof(TE) == 4) {
    if (__builtin_expect(normal_or_zero(x), 1)) return f64_of_normal(x);
    return f64_exact(x);
  } else {
    return (TA)x;
  }
}

// Quotient of the flux arithmetic: the IEEE division for double (and the
// float-float division for float-float); for float the reciprocal-based
// quotient __fdividef (within 2 ulp for divisors of magnitude below 2^126:
// the limiter denominators are at least 2 eps and the densities of order
// one), a fraction of the instructions of the IEEE float division.  The
// FP32 path's error budget (1e-5 of the residual) is set by its 24-bit
// arithmetic, not by these last-bit differences.
template <typename T>
__device__ __forceinline__ T quot(T a, T b) {
  return a / b;
}
template <>
__device__ __forceinline__ float quot<float>(float a, float b) {
  return __fdividef(a, b);
}

// Euler flux Jacobian d(f(q).n)/dq (row r = flux component, column c =
// conserved variable), scaled by h and written to out[6r + c]: with
// u = m/rho, u_n = u.n, k = |u|^2/2, H = (E + p)/rho, c = q_5/rho,
//   row 0: (0, n, 0, 0)
//   row 1+a: (-u_a u_n + (g-1) k n_a, u_n e_a + u_a n - (g-1) n_a u, (g-1) n_a, 0)
//   row 4: (u_n ((g-1) k - H), H n - (g-1) u_n u, g u_n, 0)
//   row 5: (-c u_n, c n, 0, u_n).
__device__ __forceinline__ void flux_jacobian_f64(const double* q, const double* nv,
                                                  const Gas<double>& g, double h, double* out) {
  const double rr = 1.0 / q[0];
  const double u[3] = {q[1] * rr, q[2] * rr, q[3] * rr};
  const double un = u[0] * nv[0] + u[1] * nv[1] + u[2] * nv[2];
  const double k = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const double p = g.gm1 * (q[4] - q[0] * k);
  const double H = (q[4] + p) * rr;
  const double cs = q[5] * rr;
  out[0] = 0.0;
#pragma unroll
  for (int b = 0; b < 3; b++) out[1 + b] = h * nv[b];
  out[4] = 0.0;
  out[5] = 0.0;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    double* row = out + 6 * (1 + a);
    row[0] = h * (g.gm1 * k * nv[a] - u[a] * un);
#pragma unroll
    for (int b = 0; b < 3; b++)
      row[1 + b] = h * ((a == b ? un : 0.0) + u[a] * nv[b] - g.gm1 * nv[a] * u[b]);
    row[4] = h * g.gm1 * nv[a];
    row[5] = 0.0;
  }
  out[24] = h * un * (g.gm1 * k - H);
#pragma unroll
  for (int b = 0; b < 3; b++) out[25 + b] = h * (H * nv[b] - g.gm1 * un * u[b]);
  out[28] = h * g.gamma * un;
  out[29] = 0.0;
  out[30] = -h * cs * un;
#pragma unroll
  for (int b = 0; b < 3; b++) out[31 + b] = h * cs * nv[b];
  out[34] = 0.0;
  out[35] = h * un;
}

// Euler flux through the face of normal n, and the state's largest wave
// speed |u.n| + a|n| (a = sqrt(gamma p / rho); nn2 = |n|^2).
template <typename T>
__device__ __forceinline__ void euler_side(const T* q, T nx, T ny, T nz,
                                           T nn2, const Gas<T>& g, T* f,
                                           T& lam) {
  T rr = quot(T(1), q[0]);
  T un = (q[1] * nx + q[2] * ny + q[3] * nz) * rr;
  T mm = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  T p = g.gm1 * (q[4] - T(0.5) * mm * rr);
  T an = sqrt(g.gamma * p * rr * nn2);
  lam = fabs(un) + an;
  f[0] = q[0] * un;
  f[1] = q[1] * un + p * nx;
  f[2] = q[2] * un + p * ny;
  f[3] = q[3] * un + p * nz;
  f[4] = (q[4] + p) * un;
  f[5] = q[5] * un;
}

// Rusanov flux F = (f(qL)+f(qR))/2 - s (qR - qL)/2, s = max wave speed
// (ties take the left state).
template <typename T>
__device__ __forceinline__ void rusanov(const T* qL, const T* qR, T nx, T ny,
                                        T nz, const Gas<T>& g, T* F) {
  T nn2 = nx * nx + ny * ny + nz * nz;
  T fL[6], fR[6], lL, lR;
  euler_side(qL, nx, ny, nz, nn2, g, fL, lL);
  euler_side(qR, nx, ny, nz, nn2, g, fR, lR);
  T hs = T(0.5) * (lL >= lR ? lL : lR);
#pragma unroll
  for (int k = 0; k < 6; k++) F[k] = T(0.5) * (fL[k] + fR[k]) - hs * (qR[k] - qL[k]);
}

// van Albada limiter phi(a, b) = (a(b^2+eps) + b(a^2+eps)) / (a^2+b^2+2eps),
// evaluated as (a + b)(ab + eps) / (a^2 + (b^2 + 2 eps)): the same rational
// function, with the b-only part b2e = b^2 + 2 eps shared by both ends.
template <typename T>
__device__ __forceinline__ T van_albada(T a, T b, T eps, T b2e) {
  return quot((a + b) * fma(a, b, eps), fma(a, a, b2e));
}

// Limited linear reconstruction of the two face states.  vi, vj: q (6)
// then G (18, component 3k+d) of the two ends; dx = x_j - x_i.
template <typename T>
__device__ __forceinline__ void reconstruct(const T* vi, const T* vj, T dx,
                                            T dy, T dz, const Gas<T>& g,
                                            T* qL, T* qR) {
#pragma unroll
  for (int k = 0; k < 6; k++) {
    T b = vj[k] - vi[k];
    T ai = vi[6 + 3 * k] * dx + vi[7 + 3 * k] * dy + vi[8 + 3 * k] * dz;
    T aj = vj[6 + 3 * k] * dx + vj[7 + 3 * k] * dy + vj[8 + 3 * k] * dz;
    T b2e = fma(b, b, g.two_eps);
    qL[k] = vi[k] + T(0.5) * van_albada(ai, b, g.eps, b2e);
    qR[k] = vj[k] - T(0.5) * van_albada(aj, b, g.eps, b2e);
  }
}

// ------------------------------------------------- FP64 second-order flux
// GB300 runs FP64 at 1/64 of the FP32 rate (2 FMA per clock per SM) and a
// division or square root costs about ten FMA slots, so the FP64 flux is
// bound by its FP64 instruction count.  This version computes the same
// formulas as reconstruct() + rusanov() with fewer FP64 instructions:
//  * the 12 limiter denominators are inverted together (prefix products,
//    one reciprocal, back-substitution: Montgomery's batch inversion), and so
//    are the two face densities; that one reciprocal and the square roots
//    start from FP32 seeds refined by two Newton steps in FP64 (recip2,
//    sqrt2 below), so every value keeps full double precision and the
//    residual stays smooth at rounding level (finite differences of it are
//    meaningful down to h ~ 1e-7);
//  * the factors 1/2 are folded into those reciprocals;
//  * the larger of the two wave speeds is chosen by an integer comparison
//    of their bit patterns (both are >= 0, so the order is the same).
// Batching is used only when every denominator lies in [2^-70, 2^70], so no
// prefix product can overflow or underflow; otherwise each is divided.

// FP32-seeded Newton-Raphson reciprocal and square root for the FP64 pipe.
// The seed comes from the FP32 special-function unit (rcp.approx /
// rsqrt.approx, about 2^-22 relative error including the truncation of the
// argument); the conversions between double and float are done with
// integer operations on the bit patterns, so no FP64-pipe instruction is
// spent on them.  Each Newton step in FP64 squares the relative error
// (about 2^-44 after one), so two steps reach full double precision.  Valid for positive
// arguments whose FP32 image is a normal number with a normal reciprocal
// (exponent field of the double in [898, 1149]); callers check seedable().
__device__ __forceinline__ bool seedable(double x) {
  const unsigned e = ((unsigned)__double2hiint(x) >> 20);  // sign bit must be 0
  return e - 898u <= 251u;
}
__device__ __forceinline__ float f32_of_f64(double x) {  // truncating, x > 0
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  return __int_as_float(((hi - 0x38000000) << 3) | (int)(lo >> 29));
}
__device__ __forceinline__ double f64_of_f32(float f) {  // exact, f > 0 normal
  const int b = __float_as_int(f);
  return __hiloint2double((b >> 3) + 0x38000000, b << 29);
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// 1 / d with two Newton steps (full precision)
__device__ __forceinline__ double recip2(double d) {
  const double y0 = f64_of_f32(rcp_approx(f32_of_f64(d)));
  const double y1 = fma(y0, fma(-d, y0, 1.0), y0);
  return fma(y1, fma(-d, y1, 1.0), y1);
}
// sqrt(x) with two Newton steps (full precision)
__device__ __forceinline__ double sqrt2(double x) {
  const float r = rsqrt_approx(f32_of_f64(x));
  const double r0 = f64_of_f32(r);
  const double r1 = fma(f64_of_f32(0.5f * r), fma(-x * r0, r0, 1.0), r0);
  const double t = x * r1;
  const double hh = fma(-t, 0.5 * r1, 0.5);  // (1 - x r1^2) / 2
  return fma(t, hh, t);
}

// 1/sqrt(x) with two Newton steps (full precision)
__device__ __forceinline__ double rsqrt2(double x) {
  const float r = rsqrt_approx(f32_of_f64(x));
  const double r0 = f64_of_f32(r);
  const double r1 = fma(f64_of_f32(0.5f * r), fma(-x * r0, r0, 1.0), r0);
  return fma(0.5 * r1, fma(-x * r1, r1, 1.0), r1);
}

// Largest wave speed |u.n| + a|n| of one state (a = sqrt(gamma p / rho),
// nn2 = |n|^2) with the FP32-seeded Newton reciprocal and square root (full
// double precision) where the arguments allow, else the IEEE operations.
__device__ __forceinline__ double wave_speed_f64(const double* q, double nx, double ny,
                                                 double nz, double nn2, const Gas<double>& g) {
  const double rr = seedable(q[0]) ? recip2(q[0]) : 1.0 / q[0];
  const double un = fma(q[3], nz, fma(q[2], ny, q[1] * nx)) * rr;
  const double mm = fma(q[3], q[3], fma(q[2], q[2], q[1] * q[1]));
  const double p = g.gm1 * fma(-0.5 * mm, rr, q[4]);
  const double a2n = g.gamma * p * rr * nn2;
  const double an = seedable(a2n) ? sqrt2(a2n) : sqrt(a2n);
  return fabs(un) + an;
}

// The larger wave speed of an edge from its two ends' (u_x, u_y, u_z, a):
// max(|u_i.n| + a_i|n|, |u_j.n| + a_j|n|), ties to the first end.
__device__ __forceinline__ double edge_wave_speed(const double* wi, const double* wj, double nx,
                                                  double ny, double nz) {
  const double nn2 = fma(nz, nz, fma(ny, ny, nx * nx));
  const double nn = seedable(nn2) ? sqrt2(nn2) : sqrt(nn2);
  const double lL = fma(wi[3], nn, fabs(fma(wi[2], nz, fma(wi[1], ny, wi[0] * nx))));
  const double lR = fma(wj[3], nn, fabs(fma(wj[2], nz, fma(wj[1], ny, wj[0] * nx))));
  return lL >= lR ? lL : lR;
}

__device__ __forceinline__ bool exp_in_range(double x, int lim) {
  // |x| in [2^-lim, 2^lim] (x finite, nonzero)
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
  return (unsigned)(e + lim) <= (unsigned)(2 * lim);
}

// r[k] = scale / d[k] for K values
template <int K>
__device__ __forceinline__ void batch_reciprocal(const double* d, double scale,
                                                 double* r) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < K; k++) ok &= exp_in_range(d[k], 70);
  if (ok) {
    double p[K];
    p[0] = d[0];
#pragma unroll
    for (int k = 1; k < K; k++) p[k] = p[k - 1] * d[k];
    const double pk = p[K - 1];
    double inv;
    if (seedable(pk)) {
      inv = recip2(pk);  // a normal double within the float exponent range
      // scale = 1/2 exactly: decrement the exponent on the integer pipe
      if (scale == 0.5)
        inv = __hiloint2double(__double2hiint(inv) - 0x00100000, __double2loint(inv));
      else if (scale != 1.0)
        inv *= scale;
    } else {
      inv = scale / pk;
    }
#pragma unroll
    for (int k = K - 1; k > 0; k--) {
      r[k] = inv * p[k - 1];
      inv = inv * d[k];
    }
    r[0] = inv;
  } else {
#pragma unroll
    for (int k = 0; k < K; k++) r[k] = scale / d[k];
  }
}

__device__ __forceinline__ double max_nonneg(double a, double b) {
  // both >= 0: IEEE order equals the order of the bit patterns; ties -> a
  return __double_as_longlong(a) >= __double_as_longlong(b) ? a : b;
}

// |x| as a float for ranking: truncated, 0 below the float range, +inf
// above it (integer operations only; relative error < 2^-23 in range).
__device__ __forceinline__ float abs_f32_rank(double x) {
  const int hi = __double2hiint(x) & 0x7fffffff;
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned e = (unsigned)hi >> 20;
  const float f = __int_as_float(((hi - 0x38000000) << 3) | (int)(lo >> 29));
  return e < 897u ? 0.0f : (e > 1150u ? __int_as_float(0x7f800000) : f);
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Rusanov flux of the face states (qL, qR) in FP64.  Everything is computed
// at half scale -- 1/(2 rho), u.n/2, p/2, (a|n|/2)^2, the half fluxes and
// s/2 -- which is exact (powers of two), so that
// F = f(qL).n/2 + f(qR).n/2 - (s/2)(qR - qL) needs no final halving.  The
// two densities are inverted together.  The larger wave speed s is found
// by ranking the two sides with FP32 estimates (error < 2^-20) and taking
// the FP64 square root of the larger side only; when the estimates are
// within 2^-14 of each other both sides are computed exactly and the
// larger is picked by an integer comparison of the bit patterns (ties take
// the left state), so s is always the exact larger value.  The two sides'
// fluxes are summed as they are formed (q_L u_L + q_R u_R + (p_L + p_R) n
// in one chain of multiply-adds) instead of side by side.
__device__ __forceinline__ void rusanov_f64(const double* qL, const double* qR,
                                            double nx, double ny, double nz,
                                            const Gas<double>& g, double* F) {
  const double gnn = g.gamma * fma(nz, nz, fma(ny, ny, nx * nx));
  double rho[2] = {qL[0], qR[0]}, rr[2];
  batch_reciprocal<2>(rho, 0.5, rr);  // rr = 1 / (2 rho)
  const double hgm1 = 0.5 * g.gm1;
  double mn[2], un[2], ph[2], e4[2], uh[2], x[2];
  float rank[2];
#pragma unroll
  for (int sd = 0; sd < 2; sd++) {
    const double* q = sd ? qR : qL;
    mn[sd] = fma(q[3], nz, fma(q[2], ny, q[1] * nx));
    un[sd] = mn[sd] * rr[sd];  // u.n / 2
    const double mm = fma(q[3], q[3], fma(q[2], q[2], q[1] * q[1]));
    ph[sd] = fma(-hgm1 * mm, rr[sd], hgm1 * q[4]);  // p / 2
    e4[sd] = fma(2.0, ph[sd], q[4]);                // rho E + p
    x[sd] = ph[sd] * rr[sd] * gnn;                  // (a |n| / 2)^2
    uh[sd] = fabs(un[sd]);
    rank[sd] = abs_f32_rank(un[sd]) +
               (seedable(x[sd]) ? sqrt_approx(f32_of_f64(x[sd])) : 0.0f);
  }
  double s;
  const bool ranked = seedable(x[0]) && seedable(x[1]) &&
                      (rank[0] > rank[1] * 1.00006104f || rank[1] > rank[0] * 1.00006104f);
  if (ranked) {
    const bool r = rank[1] > rank[0];
    const double xs = r ? x[1] : x[0];
    s = (r ? uh[1] : uh[0]) + sqrt2(xs);
  } else {
    const double l0 = uh[0] + (seedable(x[0]) ? sqrt2(x[0]) : sqrt(x[0]));
    const double l1 = uh[1] + (seedable(x[1]) ? sqrt2(x[1]) : sqrt(x[1]));
    s = max_nonneg(l0, l1);
  }
  // the two sides' half fluxes summed directly:
  // f_k(L) + f_k(R) = q_k,L un_L + q_k,R un_R (+ (ph_L + ph_R) n for the momenta)
  const double php = ph[0] + ph[1];
  const double n3[3] = {nx, ny, nz};
  F[0] = fma(-s, qR[0] - qL[0], 0.5 * (mn[0] + mn[1]));
#pragma unroll
  for (int d = 0; d < 3; d++)
    F[1 + d] = fma(-s, qR[1 + d] - qL[1 + d],
                   fma(qL[1 + d], un[0], fma(qR[1 + d], un[1], php * n3[d])));
  F[4] = fma(-s, qR[4] - qL[4], fma(e4[0], un[0], e4[1] * un[1]));
  F[5] = fma(-s, qR[5] - qL[5], fma(qL[5], un[0], qR[5] * un[1]));
}

// vi, vj: q (6) then G (18, component 3k+d); F: the Rusanov flux of the
// limited face states.
__device__ __forceinline__ void flux2_f64(const double* vi, const double* vj,
                                          double dx, double dy, double dz,
                                          double nx, double ny, double nz,
                                          const Gas<double>& g, double* F) {
  double num[12], den[12], rec[12];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const double b = vj[k] - vi[k];
    const double ai = fma(vi[8 + 3 * k], dz, fma(vi[7 + 3 * k], dy, vi[6 + 3 * k] * dx));
    const double aj = fma(vj[8 + 3 * k], dz, fma(vj[7 + 3 * k], dy, vj[6 + 3 * k] * dx));
    const double b2e = fma(b, b, g.two_eps);
    num[2 * k] = (ai + b) * fma(ai, b, g.eps);
    den[2 * k] = fma(ai, ai, b2e);
    num[2 * k + 1] = (aj + b) * fma(aj, b, g.eps);
    den[2 * k + 1] = fma(aj, aj, b2e);
  }
  batch_reciprocal<12>(den, 0.5, rec);  // rec = 1 / (2 den)
  double qL[6], qR[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    qL[k] = fma(num[2 * k], rec[2 * k], vi[k]);
    qR[k] = fma(-num[2 * k + 1], rec[2 * k + 1], vj[k]);
  }
  rusanov_f64(qL, qR, nx, ny, nz, g, F);
}

// ---------------------------------------------------------------- adjoint

__device__ __forceinline__ double sgn(double x) {
  return (double)((x > 0.0) - (x < 0.0));
}

// Reverse of one side of the Rusanov flux.  fb: adjoint of f(q).n (6),
// lamb: adjoint of the side's wave speed.  Accumulates qb (6), nb (3).
__device__ __forceinline__ void euler_side_reverse(
    const double* q, double nx, double ny, double nz, const Gas<double>& g,
    const double* fb, double lamb, double* qb, double& nbx, double& nby,
    double& nbz) {
  double rr = 1.0 / q[0];
  double un = (q[1] * nx + q[2] * ny + q[3] * nz) * rr;
  double mm = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  double p = g.gm1 * (q[4] - 0.5 * mm * rr);
  double a = sqrt(g.gamma * p * rr);
  double nn = sqrt(nx * nx + ny * ny + nz * nz);
  // lam = |un| + a |n|
  double unb = sgn(un) * lamb;
  double ab = lamb * nn;
  double nnb = lamb * a;
  // f_k = q_k un (+ p n_d for k = 1..3, + p un for k = 4)
  double pb = fb[1] * nx + fb[2] * ny + fb[3] * nz + fb[4] * un;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    qb[k] += fb[k] * un;
    unb += fb[k] * q[k];
  }
  unb += fb[4] * p;
  double rnn = nnb / nn;
  nbx += fb[1] * p + rnn * nx;
  nby += fb[2] * p + rnn * ny;
  nbz += fb[3] * p + rnn * nz;
  // a = sqrt(gamma p / rho)
  pb += ab * g.gamma * rr / (2.0 * a);
  double rhob = -0.5 * ab * a * rr;
  // p = (gamma-1)(E - |m|^2 / (2 rho))
  double gpb = g.gm1 * pb;
  qb[4] += gpb;
  rhob += 0.5 * gpb * mm * rr * rr;
  // un = (m . n) / rho
  double ur = unb * rr;
  qb[1] += ur * nx - gpb * q[1] * rr;
  qb[2] += ur * ny - gpb * q[2] * rr;
  qb[3] += ur * nz - gpb * q[3] * rr;
  nbx += ur * q[1];
  nby += ur * q[2];
  nbz += ur * q[3];
  rhob -= ur * un;
  qb[0] += rhob;
}

// Reverse of the Rusanov flux for adjoint weights w = dJ/dF.
__device__ __forceinline__ void rusanov_reverse(
    const double* qL, const double* qR, double nx, double ny, double nz,
    const Gas<double>& g, const double* w, double* qLb, double* qRb,
    double& nbx, double& nby, double& nbz) {
  double nn2 = nx * nx + ny * ny + nz * nz;
  double fL[6], fR[6], lL, lR;
  euler_side(qL, nx, ny, nz, nn2, g, fL, lL);
  euler_side(qR, nx, ny, nz, nn2, g, fR, lR);
  bool left = lL >= lR;
  double s = left ? lL : lR;
  double fb[6], sb = 0.0;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    fb[k] = 0.5 * w[k];
    sb -= 0.5 * w[k] * (qR[k] - qL[k]);
    qRb[k] -= 0.5 * s * w[k];
    qLb[k] += 0.5 * s * w[k];
  }
  euler_side_reverse(qL, nx, ny, nz, g, fb, left ? sb : 0.0, qLb, nbx, nby, nbz);
  euler_side_reverse(qR, nx, ny, nz, g, fb, left ? 0.0 : sb, qRb, nbx, nby, nbz);
}

// van Albada value and partial derivatives
__device__ __forceinline__ void van_albada_d(double a, double b, double eps,
                                             double b2e, double& phi,
                                             double& pa, double& pb) {
  double s = a + b;
  double t = fma(a, b, eps);
  double rd = 1.0 / fma(a, a, b2e);
  phi = s * t * rd;
  // d/da: (b^2 + eps + 2ab - 2a phi)/D, d/db: (a^2 + eps + 2ab - 2b phi)/D
  pa = (fma(b, b, eps) + 2.0 * a * b - 2.0 * a * phi) * rd;
  pb = (fma(a, a, eps) + 2.0 * a * b - 2.0 * b * phi) * rd;
}

// ------------------------------------------ FP64 adjoint, fewer FP64 ops
// The same reverse sweep as rusanov_reverse() / van_albada_d(), arranged for
// the FP64 pipe: batched reciprocals as in flux2_f64(), one
// reciprocal square root giving both a and 1/a (and |n|, 1/|n|), no forward fluxes
// (the reverse sweep needs only the wave speeds and the primitive
// quantities), and sign / max taken from the bit patterns.

// sign(x) * v, with sign(0) = 0
__device__ __forceinline__ double sign_times(double x, double v) {
  const long long b = __double_as_longlong(x);
  if ((b << 1) == 0) return 0.0;
  return b < 0 ? -v : v;
}

struct SideState {
  double rr, un, mm, p, a, ra;  // 1/rho, u.n, |m|^2, p, sound speed, 1/a
};

__device__ __forceinline__ double side_state(const double* q, double nx,
                                             double ny, double nz, double rr,
                                             double nn, const Gas<double>& g,
                                             double hgm1, SideState& s) {
  s.rr = rr;
  s.un = fma(q[3], nz, fma(q[2], ny, q[1] * nx)) * rr;
  s.mm = fma(q[3], q[3], fma(q[2], q[2], q[1] * q[1]));
  s.p = fma(-hgm1 * s.mm, rr, g.gm1 * q[4]);
  const double a2 = g.gamma * s.p * rr;
  s.ra = seedable(a2) ? rsqrt2(a2) : rsqrt(a2);
  s.a = a2 * s.ra;
  return fabs(s.un) + s.a * nn;  // wave speed
}

// fb = adjoint of f(q).n (6), lamb = adjoint of the wave speed.
__device__ __forceinline__ void side_reverse_f64(
    const double* q, double nx, double ny, double nz, const SideState& s,
    double nn, double rn, const Gas<double>& g, const double* fb, double lamb,
    double* qb, double* nb) {
  double unb = sign_times(s.un, lamb);
  const double ab = lamb * nn;
  const double rnb = lamb * s.a * rn;  // d|n|/dn = n / |n|
#pragma unroll
  for (int k = 0; k < 6; k++) {
    qb[k] = fma(fb[k], s.un, qb[k]);
    unb = fma(fb[k], q[k], unb);
  }
  unb = fma(fb[4], s.p, unb);
  double pb = fma(fb[3], nz, fma(fb[2], ny, fma(fb[1], nx, fb[4] * s.un)));
  pb = fma(0.5 * g.gamma * ab, s.rr * s.ra, pb);  // a = sqrt(gamma p / rho)
  const double gpb = g.gm1 * pb;
  const double ur = unb * s.rr;
  const double gpr = gpb * s.rr;
  const double n3[3] = {nx, ny, nz};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    nb[d] = fma(fb[1 + d], s.p, fma(rnb, n3[d], fma(ur, q[1 + d], nb[d])));
    qb[1 + d] = fma(-gpr, q[1 + d], fma(ur, n3[d], qb[1 + d]));
  }
  qb[4] += gpb;
  // rho enters through 1/rho in u.n, p and a
  const double rhob =
      fma(0.5 * gpr, s.mm * s.rr, fma(-0.5 * ab, s.a * s.rr, -ur * s.un));
  qb[0] += rhob;
}

// Reverse of the Rusanov flux: w = dJ/dF; accumulates qLb, qRb (6), nb (3).
__device__ __forceinline__ void rusanov_reverse_f64(
    const double* qL, const double* qR, double nx, double ny, double nz,
    const Gas<double>& g, const double* w, double* qLb, double* qRb,
    double* nb) {
  const double nn2 = fma(nz, nz, fma(ny, ny, nx * nx));
  const double rn = seedable(nn2) ? rsqrt2(nn2) : rsqrt(nn2);
  const double nn = nn2 * rn;
  double rho[2] = {qL[0], qR[0]}, rr[2];
  batch_reciprocal<2>(rho, 1.0, rr);
  const double hgm1 = 0.5 * g.gm1;
  SideState sL, sR;
  const double lL = side_state(qL, nx, ny, nz, rr[0], nn, g, hgm1, sL);
  const double lR = side_state(qR, nx, ny, nz, rr[1], nn, g, hgm1, sR);
  const bool left = __double_as_longlong(lL) >= __double_as_longlong(lR);
  const double hs = 0.5 * (left ? lL : lR);
  double fb[6], sb = 0.0;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    fb[k] = 0.5 * w[k];
    sb = fma(w[k], qR[k] - qL[k], sb);
    qRb[k] = fma(-hs, w[k], qRb[k]);
    qLb[k] = fma(hs, w[k], qLb[k]);
  }
  sb *= -0.5;
  side_reverse_f64(qL, nx, ny, nz, sL, nn, rn, g, fb, left ? sb : 0.0, qLb, nb);
  side_reverse_f64(qR, nx, ny, nz, sR, nn, rn, g, fb, left ? 0.0 : sb, qRb, nb);
}

// Adjoint of the second-order flux of edge (i, j).  vi, vj: lam (6), q (6),
// G (18).  oi, oj: qbar (6) then Gbar (18) of each end; nb: nbar (3).
__device__ __forceinline__ void flux2_adj_f64(const double* vi,
                                              const double* vj, double dx,
                                              double dy, double dz, double nx,
                                              double ny, double nz,
                                              const Gas<double>& g, double* oi,
                                              double* oj, double* nb) {
  const double* qi = vi + 6;
  const double* qj = vj + 6;
  const double* Gi = vi + 12;
  const double* Gj = vj + 12;
  double a[12], num[12], den[12], rd[12], bk[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const double b = qj[k] - qi[k];
    bk[k] = b;
    a[2 * k] = fma(Gi[3 * k + 2], dz, fma(Gi[3 * k + 1], dy, Gi[3 * k] * dx));
    a[2 * k + 1] = fma(Gj[3 * k + 2], dz, fma(Gj[3 * k + 1], dy, Gj[3 * k] * dx));
    const double b2e = fma(b, b, g.two_eps);
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
      const double x = a[2 * k + sd];
      num[2 * k + sd] = (x + b) * fma(x, b, g.eps);
      den[2 * k + sd] = fma(x, x, b2e);
    }
  }
  batch_reciprocal<12>(den, 1.0, rd);
  // d phi / da = 2 P / D with P = a(b - phi) + (b^2 + eps)/2,
  // d phi / db = 2 Q / D with Q = b(a - phi) + (a^2 + eps)/2;
  // the factor 2 cancels the 1/2 of the face states; P and Q are kept
  // divided by D
  double qL[6], qR[6], P[12], Q[12];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const double b = bk[k];
    const double hbe = 0.5 * fma(b, b, g.eps);
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
      const int c = 2 * k + sd;
      const double x = a[c];
      const double phi = num[c] * rd[c];
      P[c] = fma(x, b - phi, hbe) * rd[c];
      Q[c] = fma(b, x - phi, fma(0.5 * x, x, 0.5 * g.eps)) * rd[c];
      if (sd == 0) qL[k] = fma(0.5, phi, qi[k]);
      else qR[k] = fma(-0.5, phi, qj[k]);
    }
  }
  double w[6], qLb[6], qRb[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    w[k] = vi[k] - vj[k];
    qLb[k] = 0.0;
    qRb[k] = 0.0;
  }
  rusanov_reverse_f64(qL, qR, nx, ny, nz, g, w, qLb, qRb, nb);
#pragma unroll
  for (int k = 0; k < 6; k++) {
    // phi_i bar = qLb/2, phi_j bar = -qRb/2
    const double aib = qLb[k] * P[2 * k], ajb = neg(qRb[k] * P[2 * k + 1]);
    const double bb = fma(qLb[k], Q[2 * k], neg(qRb[k] * Q[2 * k + 1]));
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

// ------------------------------------------------------ tangent (forward)
// Forward-mode linearisation of the flux in the direction (qd, Gd, nd):
// Fd = dF/dq . qd + dF/dG . Gd + dF/dn . nd (dx fixed).  Non-smooth points
// as in the reverse sweep: d|x|/dx = sign(x) (0 at 0), the max picks L on
// ties.

// one side: f(q).n and its tangent, the wave speed and its tangent
__device__ __forceinline__ void side_tangent_f64(
    const double* q, const double* qd, double nx, double ny, double nz,
    double ndx, double ndy, double ndz, double rr, double nn, double nnd,
    const Gas<double>& g, double* f, double* fd, double& lam, double& lamd) {
  const double mn = fma(q[3], nz, fma(q[2], ny, q[1] * nx));
  const double mnd = fma(qd[3], nz, fma(qd[2], ny, fma(qd[1], nx,
                     fma(q[3], ndz, fma(q[2], ndy, q[1] * ndx)))));
  const double un = mn * rr;
  const double und = fma(-un, qd[0], mnd) * rr;  // (mnd - un rhod) / rho
  const double mm = fma(q[3], q[3], fma(q[2], q[2], q[1] * q[1]));
  const double mmd = 2.0 * fma(q[3], qd[3], fma(q[2], qd[2], q[1] * qd[1]));
  const double hgm1 = 0.5 * g.gm1;
  const double p = fma(-hgm1 * mm, rr, g.gm1 * q[4]);
  // pd = (gamma-1) (Ed - mmd/(2 rho) + mm rhod / (2 rho^2))
  const double pd = g.gm1 * qd[4] + hgm1 * rr * fma(mm * rr, qd[0], -mmd);
  const double a2 = g.gamma * p * rr;
  const double ra = seedable(a2) ? rsqrt2(a2) : rsqrt(a2);
  const double a = a2 * ra;
  // 2 a ad = (gamma pd - a^2 rhod) / rho
  const double ad = 0.5 * ra * rr * fma(-a2, qd[0], g.gamma * pd);
  lam = fabs(un) + a * nn;
  lamd = sign_times(un, und) + fma(ad, nn, a * nnd);
#pragma unroll
  for (int k = 0; k < 6; k++) {
    f[k] = q[k] * un;
    fd[k] = fma(qd[k], un, q[k] * und);
  }
  const double n3[3] = {nx, ny, nz}, nd3[3] = {ndx, ndy, ndz};
#pragma unroll
  for (int d = 0; d < 3; d++) {
    f[1 + d] = fma(p, n3[d], f[1 + d]);
    fd[1 + d] = fma(pd, n3[d], fma(p, nd3[d], fd[1 + d]));
  }
  f[4] = fma(p, un, f[4]);
  fd[4] = fma(pd, un, fma(p, und, fd[4]));
}

// Fd of the Rusanov flux for face states (qL, qR) with tangents (qLd, qRd)
__device__ __forceinline__ void rusanov_tangent_f64(
    const double* qL, const double* qLd, const double* qR, const double* qRd,
    double nx, double ny, double nz, double ndx, double ndy, double ndz,
    const Gas<double>& g, double* Fd) {
  const double nn2 = fma(nz, nz, fma(ny, ny, nx * nx));
  const double rn = seedable(nn2) ? rsqrt2(nn2) : rsqrt(nn2);
  const double nn = nn2 * rn;
  const double nnd = fma(nz, ndz, fma(ny, ndy, nx * ndx)) * rn;
  double rho[2] = {qL[0], qR[0]}, rr[2];
  batch_reciprocal<2>(rho, 1.0, rr);
  double fL[6], fLd[6], fR[6], fRd[6], lL, lLd, lR, lRd;
  side_tangent_f64(qL, qLd, nx, ny, nz, ndx, ndy, ndz, rr[0], nn, nnd, g, fL, fLd, lL, lLd);
  side_tangent_f64(qR, qRd, nx, ny, nz, ndx, ndy, ndz, rr[1], nn, nnd, g, fR, fRd, lR, lRd);
  const bool left = __double_as_longlong(lL) >= __double_as_longlong(lR);
  const double hs = 0.5 * (left ? lL : lR), hsd = 0.5 * (left ? lLd : lRd);
#pragma unroll
  for (int k = 0; k < 6; k++)
    Fd[k] = fma(0.5, fLd[k] + fRd[k], -fma(hsd, qR[k] - qL[k], hs * (qRd[k] - qLd[k])));
}

// Tangent of the second-order flux.  vi, vj: q (6), qd (6), G (18), Gd (18).
__device__ __forceinline__ void flux2_tan_f64(const double* vi, const double* vj,
                                              double dx, double dy, double dz,
                                              double nx, double ny, double nz,
                                              double ndx, double ndy, double ndz,
                                              const Gas<double>& g, double* Fd) {
  const double *qi = vi, *qid = vi + 6, *Gi = vi + 12, *Gid = vi + 30;
  const double *qj = vj, *qjd = vj + 6, *Gj = vj + 12, *Gjd = vj + 30;
  double a[12], ad[12], num[12], den[12], rd[12], bk[6], bdk[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const double b = qj[k] - qi[k];
    bk[k] = b;
    bdk[k] = qjd[k] - qid[k];
    a[2 * k] = fma(Gi[3 * k + 2], dz, fma(Gi[3 * k + 1], dy, Gi[3 * k] * dx));
    a[2 * k + 1] = fma(Gj[3 * k + 2], dz, fma(Gj[3 * k + 1], dy, Gj[3 * k] * dx));
    ad[2 * k] = fma(Gid[3 * k + 2], dz, fma(Gid[3 * k + 1], dy, Gid[3 * k] * dx));
    ad[2 * k + 1] = fma(Gjd[3 * k + 2], dz, fma(Gjd[3 * k + 1], dy, Gjd[3 * k] * dx));
    const double b2e = fma(b, b, g.two_eps);
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
      const double x = a[2 * k + sd];
      num[2 * k + sd] = (x + b) * fma(x, b, g.eps);
      den[2 * k + sd] = fma(x, x, b2e);
    }
  }
  batch_reciprocal<12>(den, 1.0, rd);
  double qL[6], qR[6], qLd[6], qRd[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const double b = bk[k], bd = bdk[k];
    const double be = fma(b, b, g.eps);
    const double b2 = b + b;
#pragma unroll
    for (int sd = 0; sd < 2; sd++) {
      const int c = 2 * k + sd;
      const double x = a[c];
      const double phi = num[c] * rd[c];
      const double pa = fma(x + x, b - phi, be) * rd[c];
      const double pb = fma(b2, x - phi, fma(x, x, g.eps)) * rd[c];
      const double phid = fma(pa, ad[c], pb * bd);
      if (sd == 0) {
        qL[k] = fma(0.5, phi, qi[k]);
        qLd[k] = fma(0.5, phid, qid[k]);
      } else {
        qR[k] = fma(-0.5, phi, qj[k]);
        qRd[k] = fma(-0.5, phid, qjd[k]);
      }
    }
  }
  rusanov_tangent_f64(qL, qLd, qR, qRd, nx, ny, nz, ndx, ndy, ndz, g, Fd);
}

}  // namespace op2b
