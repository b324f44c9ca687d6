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

// Euler flux through the face of normal n, and the state's largest wave
// speed |u.n| + a|n| (a = sqrt(gamma p / rho); nn2 = |n|^2).
template <typename T>
__device__ __forceinline__ void euler_side(const T* q, T nx, T ny, T nz,
                                           T nn2, const Gas<T>& g, T* f,
                                           T& lam) {
  T rr = T(1) / q[0];
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
  return (a + b) * fma(a, b, eps) / fma(a, a, b2e);
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

}  // namespace op2b
