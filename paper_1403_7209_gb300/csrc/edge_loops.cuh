// The loop bodies ("user kernels" in the paper's terms, Sec. 3.1) and the
// three race-resolution strategies that drive them over an edge set.
//
// A loop body P declares:
//   TN  type of the node/edge data it reads and computes in
//   TE  type of its per-edge results,  TA  type of the INC targets
//   NIN values read per end node, OUT results per end node
//   MODE  MODE_ANTI: node j receives -(node i's result) (fluxes)
//         MODE_SYM:  node j receives the same result     (spectral radius)
//         MODE_GEN:  node j has its own OUT results       (adjoints)
//   DIM0  how many of the OUT components go to the first INC dat (the rest
//         go to the second)
//   load(node, v[NIN])  and  edge(e, vi, vj, oi, oj)
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "edge_math.cuh"

namespace op2b {

enum { MODE_ANTI = 0, MODE_SYM = 1, MODE_GEN = 2 };

template <typename TA, int DIM0>
struct Targets {
  TA* p0;
  int64_t ld0;
  TA* p1;
  int64_t ld1;
  __device__ __forceinline__ TA* at(int c, int64_t node) const {
    return c < DIM0 ? p0 + (int64_t)c * ld0 + node
                    : p1 + (int64_t)(c - DIM0) * ld1 + node;
  }
};

// ------------------------------------------------------------ loop bodies

// Green-Gauss: oi[3k+d] = (q_i,k + q_j,k) (n_d / 2); node j gets -oi.
template <typename T>
struct BodyGG {
  using TN = T;
  using TE = T;
  using TA = T;
  static constexpr int NIN = 6, OUT = 18, MODE = MODE_ANTI, DIM0 = 18;
  const T* q;
  int64_t ldq;
  const T* n;
  int64_t ldn;
  __device__ __forceinline__ void load(int64_t i, T* v) const {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ldro(q + k * ldq + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const T* vi, const T* vj,
                                       TE* oi, TE*) const {
    T hx = halve(ldro(n + e)), hy = halve(ldro(n + ldn + e)), hz = halve(ldro(n + 2 * ldn + e));
#pragma unroll
    for (int k = 0; k < 6; k++) {
      T s = vi[k] + vj[k];
      oi[3 * k] = s * hx;
      oi[3 * k + 1] = s * hy;
      oi[3 * k + 2] = s * hz;
    }
  }
  // Packed form for the strategies that keep per-edge results: the 6 sums
  // q_i + q_j and n/2 (9 values instead of 18 products); the outer product
  // is formed while summing per node (18 FMAs per edge end).
  static constexpr int PACK = 9;
  __device__ __forceinline__ void pack(int64_t e, const T* vi, const T* vj,
                                       TE* st) const {
#pragma unroll
    for (int k = 0; k < 6; k++) st[k] = vi[k] + vj[k];
    st[6] = halve(ldro(n + e));
    st[7] = halve(ldro(n + ldn + e));
    st[8] = halve(ldro(n + 2 * ldn + e));
  }
  template <class Get>
  __device__ __forceinline__ static void unpack_add(Get get, bool second,
                                                    TA* acc) {
    const T h[3] = {second ? neg(get(6)) : get(6), second ? neg(get(7)) : get(7),
                    second ? neg(get(8)) : get(8)};
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const T s = get(k);
#pragma unroll
      for (int d = 0; d < 3; d++) acc[3 * k + d] = fma(s, h[d], acc[3 * k + d]);
    }
  }
};

// First-order Rusanov flux of the two node states.
template <typename T>
struct BodyFlux1 {
  using TN = T;
  using TE = T;
  using TA = double;
  static constexpr int NIN = 6, OUT = 6, MODE = MODE_ANTI, DIM0 = 6;
  const T* q;
  int64_t ldq;
  const T* n;
  int64_t ldn;
  Gas<T> g;
  __device__ __forceinline__ void load(int64_t i, T* v) const {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ldro(q + k * ldq + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const T* vi, const T* vj,
                                       TE* oi, TE*) const {
    rusanov(vi, vj, ldro(n + e), ldro(n + ldn + e), ldro(n + 2 * ldn + e), g,
            oi);
  }
};

// Second-order flux: limited reconstruction then Rusanov.  v = q (6), G (18).
template <typename T>
struct BodyFlux2 {
  using TN = T;
  using TE = T;
  using TA = double;
  static constexpr int NIN = 24, OUT = 6, MODE = MODE_ANTI, DIM0 = 6;
  const T* q;
  int64_t ldq;
  const T* G;
  int64_t ldG;
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
  }
  __device__ __forceinline__ void edge(int64_t e, const T* vi, const T* vj,
                                       TE* oi, TE*) const {
    if constexpr (sizeof(T) == 8) {
      flux2_f64(vi, vj, ldro(dx + e), ldro(dx + lddx + e), ldro(dx + 2 * lddx + e),
                ldro(n + e), ldro(n + ldn + e), ldro(n + 2 * ldn + e), g, oi);
    } else {
      T qL[6], qR[6];
      reconstruct(vi, vj, ldro(dx + e), ldro(dx + lddx + e),
                  ldro(dx + 2 * lddx + e), g, qL, qR);
      rusanov(qL, qR, ldro(n + e), ldro(n + ldn + e), ldro(n + 2 * ldn + e), g,
              oi);
    }
  }
};

// Block-Jacobi blocks: the first end gets (A(q_i, n) + s I)/2, the second
// (-A(q_j, n) + s I)/2, s the Rusanov wave speed of the two node states.
struct BodyJacobi {
  using TN = double;
  using TE = double;
  using TA = double;
  static constexpr int NIN = 6, OUT = 36, MODE = MODE_GEN, DIM0 = 36;
  const double* q;
  int64_t ldq;
  const double* n;
  int64_t ldn;
  Gas<double> g;
  __device__ __forceinline__ void load(int64_t i, double* v) const {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ldro(q + k * ldq + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const double* vi, const double* vj,
                                       double* oi, double* oj) const {
    const double nv[3] = {ldro(n + e), ldro(n + ldn + e), ldro(n + 2 * ldn + e)};
    const double nn2 = fma(nv[2], nv[2], fma(nv[1], nv[1], nv[0] * nv[0]));
    const double lL = wave_speed_f64(vi, nv[0], nv[1], nv[2], nn2, g);
    const double lR = wave_speed_f64(vj, nv[0], nv[1], nv[2], nn2, g);
    const double hs = 0.5 * (lL >= lR ? lL : lR);
    flux_jacobian_f64(vi, nv, g, 0.5, oi);
    flux_jacobian_f64(vj, nv, g, -0.5, oj);
#pragma unroll
    for (int r = 0; r < 6; r++) {
      oi[7 * r] += hs;
      oj[7 * r] += hs;
    }
  }
};

// Sums of the factored block-Jacobi blocks: (s, n) to the first end,
// (s, -n) to the second, s the Rusanov wave speed of the two node states.
// v = (u_x, u_y, u_z, a) of each node (the wave-primitive node pass).
struct BodyJacobiSums {
  using TN = double;
  using TE = double;
  using TA = double;
  static constexpr int NIN = 4, OUT = 4, MODE = MODE_GEN, DIM0 = 4;
  const double* w;
  int64_t ldw;
  const double* n;
  int64_t ldn;
  Gas<double> g;
  __device__ __forceinline__ void load(int64_t i, double* v) const {
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = ldro(w + k * ldw + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const double* vi, const double* vj,
                                       double* oi, double* oj) const {
    const double nx = ldro(n + e), ny = ldro(n + ldn + e), nz = ldro(n + 2 * ldn + e);
    oi[0] = oj[0] = edge_wave_speed(vi, vj, nx, ny, nz);
    oi[1] = nx;
    oi[2] = ny;
    oi[3] = nz;
    oj[1] = neg(nx);
    oj[2] = neg(ny);
    oj[3] = neg(nz);
  }
};

// Spectral radius: s_e = max wave speed of the two node states, to both.
// v = (u_x, u_y, u_z, a) of each node (the wave-primitive node pass).
struct BodySpectral {
  using TN = double;
  using TE = double;
  using TA = double;
  static constexpr int NIN = 4, OUT = 1, MODE = MODE_SYM, DIM0 = 1;
  const double* w;
  int64_t ldw;
  const double* n;
  int64_t ldn;
  Gas<double> g;
  __device__ __forceinline__ void load(int64_t i, double* v) const {
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = ldro(w + k * ldw + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const double* vi,
                                       const double* vj, double* oi,
                                       double*) const {
    oi[0] = edge_wave_speed(vi, vj, ldro(n + e), ldro(n + ldn + e), ldro(n + 2 * ldn + e));
  }
};

// Adjoint of the flux loop.  v = lam (6), q (6) [, G (18)].  Results:
// qbar (6) then Gbar (18, order 2) for each end; nbar written directly.
template <int ORDER>
struct BodyFluxAdj {
  using TN = double;
  using TE = double;
  using TA = double;
  static constexpr int NIN = ORDER == 1 ? 12 : 30;
  static constexpr int OUT = ORDER == 1 ? 6 : 24;
  static constexpr int MODE = MODE_GEN, DIM0 = 6;
  const double* lam;
  int64_t ldl;
  const double* q;
  int64_t ldq;
  const double* G;
  int64_t ldG;
  const double* n;
  int64_t ldn;
  const double* dx;
  int64_t lddx;
  double* nbar;
  int64_t ldnb;
  Gas<double> g;
  __device__ __forceinline__ void load(int64_t i, double* v) const {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ldro(lam + k * ldl + i);
#pragma unroll
    for (int k = 0; k < 6; k++) v[6 + k] = ldro(q + k * ldq + i);
    if constexpr (ORDER == 2) {
#pragma unroll
      for (int c = 0; c < 18; c++) v[12 + c] = ldro(G + c * ldG + i);
    }
  }
  __device__ __forceinline__ void edge(int64_t e, const double* vi,
                                       const double* vj, double* oi,
                                       double* oj) const {
    const double nx = ldro(n + e), ny = ldro(n + ldn + e), nz = ldro(n + 2 * ldn + e);
    double nb[3] = {0.0, 0.0, 0.0};
    if constexpr (ORDER == 1) {
      double w[6];
#pragma unroll
      for (int k = 0; k < 6; k++) {
        w[k] = vi[k] - vj[k];
        oi[k] = 0.0;
        oj[k] = 0.0;
      }
      rusanov_reverse_f64(vi + 6, vj + 6, nx, ny, nz, g, w, oi, oj, nb);
    } else {
      flux2_adj_f64(vi, vj, ldro(dx + e), ldro(dx + lddx + e), ldro(dx + 2 * lddx + e), nx,
                    ny, nz, g, oi, oj, nb);
    }
    const double nbx = nb[0], nby = nb[1], nbz = nb[2];
    nbar[e] = nbx;
    nbar[ldnb + e] = nby;
    nbar[2 * ldnb + e] = nbz;
  }
};

// Adjoint of Green-Gauss.  v = Gbar (18), q (6).  Both ends receive
// sum_d (Gbar_i - Gbar_j)[k][d] n_d / 2; nbar_e += direct.
struct BodyGGAdj {
  using TN = double;
  using TE = double;
  using TA = double;
  static constexpr int NIN = 24, OUT = 6, MODE = MODE_SYM, DIM0 = 6;
  const double* Gb;
  int64_t ldGb;
  const double* q;
  int64_t ldq;
  const double* n;
  int64_t ldn;
  double* nbar;
  int64_t ldnb;
  __device__ __forceinline__ void load(int64_t i, double* v) const {
#pragma unroll
    for (int c = 0; c < 18; c++) v[c] = ldro(Gb + c * ldGb + i);
#pragma unroll
    for (int k = 0; k < 6; k++) v[18 + k] = ldro(q + k * ldq + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const double* vi,
                                       const double* vj, double* oi,
                                       double*) const {
    double hx = half_exact(ldro(n + e)), hy = half_exact(ldro(n + ldn + e)),
           hz = half_exact(ldro(n + 2 * ldn + e));
    double nbx = 0.0, nby = 0.0, nbz = 0.0;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      double dxk = vi[3 * k] - vj[3 * k];
      double dyk = vi[3 * k + 1] - vj[3 * k + 1];
      double dzk = vi[3 * k + 2] - vj[3 * k + 2];
      oi[k] = dxk * hx + dyk * hy + dzk * hz;
      double hq = half_exact(vi[18 + k] + vj[18 + k]);
      nbx += hq * dxk;
      nby += hq * dyk;
      nbz += hq * dzk;
    }
    nbar[e] += nbx;
    nbar[ldnb + e] += nby;
    nbar[2 * ldnb + e] += nbz;
  }
};

// Tangent of Green-Gauss: v = q (6), qd (6);
// oi[3k+d] = (qd_i + qd_j)_k n_d / 2 + (q_i + q_j)_k nd_d / 2, node j gets -oi.
struct BodyGGTan {
  using TN = double;
  using TE = double;
  using TA = double;
  static constexpr int NIN = 12, OUT = 18, MODE = MODE_ANTI, DIM0 = 18;
  const double* q;
  int64_t ldq;
  const double* qd;
  int64_t ldqd;
  const double* n;
  int64_t ldn;
  const double* nd;
  int64_t ldnd;
  __device__ __forceinline__ void load(int64_t i, double* v) const {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ldro(q + k * ldq + i);
#pragma unroll
    for (int k = 0; k < 6; k++) v[6 + k] = ldro(qd + k * ldqd + i);
  }
  __device__ __forceinline__ void edge(int64_t e, const double* vi, const double* vj,
                                       double* oi, double*) const {
    const double h[3] = {half_exact(ldro(n + e)), half_exact(ldro(n + ldn + e)),
                         half_exact(ldro(n + 2 * ldn + e))};
    const double hd[3] = {half_exact(ldro(nd + e)), half_exact(ldro(nd + ldnd + e)),
                          half_exact(ldro(nd + 2 * ldnd + e))};
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const double sv = vi[k] + vj[k], sd = vi[6 + k] + vj[6 + k];
#pragma unroll
      for (int d = 0; d < 3; d++) oi[3 * k + d] = fma(sd, h[d], sv * hd[d]);
    }
  }
};

// Tangent of the flux loop.  v = q (6), qd (6) [, G (18), Gd (18)].
template <int ORDER>
struct BodyFluxTan {
  using TN = double;
  using TE = double;
  using TA = double;
  static constexpr int NIN = ORDER == 1 ? 12 : 48;
  static constexpr int OUT = 6, MODE = MODE_ANTI, DIM0 = 6;
  const double* q;
  int64_t ldq;
  const double* qd;
  int64_t ldqd;
  const double* G;
  int64_t ldG;
  const double* Gd;
  int64_t ldGd;
  const double* n;
  int64_t ldn;
  const double* nd;
  int64_t ldnd;
  const double* dx;
  int64_t lddx;
  Gas<double> g;
  __device__ __forceinline__ void load(int64_t i, double* v) const {
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = ldro(q + k * ldq + i);
#pragma unroll
    for (int k = 0; k < 6; k++) v[6 + k] = ldro(qd + k * ldqd + i);
    if constexpr (ORDER == 2) {
#pragma unroll
      for (int c = 0; c < 18; c++) v[12 + c] = ldro(G + c * ldG + i);
#pragma unroll
      for (int c = 0; c < 18; c++) v[30 + c] = ldro(Gd + c * ldGd + i);
    }
  }
  __device__ __forceinline__ void edge(int64_t e, const double* vi, const double* vj,
                                       double* oi, double*) const {
    const double nx = ldro(n + e), ny = ldro(n + ldn + e), nz = ldro(n + 2 * ldn + e);
    const double ndx = ldro(nd + e), ndy = ldro(nd + ldnd + e), ndz = ldro(nd + 2 * ldnd + e);
    if constexpr (ORDER == 1) {
      rusanov_tangent_f64(vi, vi + 6, vj, vj + 6, nx, ny, nz, ndx, ndy, ndz, g, oi);
    } else {
      flux2_tan_f64(vi, vj, ldro(dx + e), ldro(dx + lddx + e), ldro(dx + 2 * lddx + e), nx, ny,
                    nz, ndx, ndy, ndz, g, oi);
    }
  }
};

// --------------------------------------------------------------- strategies

// (1) one thread per edge, atomic adds into the INC targets.
template <class P>
__global__ void k_atomic(P ph, const int32_t* __restrict__ m0,
                         const int32_t* __restrict__ m1, int64_t E,
                         Targets<typename P::TA, P::DIM0> tg) {
  using TN = typename P::TN;
  using TE = typename P::TE;
  using TA = typename P::TA;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += stride) {
    int64_t i = m0[e], j = m1[e];
    TN vi[P::NIN], vj[P::NIN];
    ph.load(i, vi);
    ph.load(j, vj);
    TE oi[P::OUT], oj[P::MODE == MODE_GEN ? P::OUT : 1];
    ph.edge(e, vi, vj, oi, oj);
#pragma unroll
    for (int c = 0; c < P::OUT; c++) {
      TA a = to_acc<TA>(oi[c]);
      atomicAdd(tg.at(c, i), a);
      if constexpr (P::MODE == MODE_ANTI) atomicAdd(tg.at(c, j), neg(a));
      if constexpr (P::MODE == MODE_SYM) atomicAdd(tg.at(c, j), a);
      if constexpr (P::MODE == MODE_GEN) atomicAdd(tg.at(c, j), to_acc<TA>(oj[c]));
    }
  }
}

// (5) owner-compute: thread per node v over the edges whose lower-numbered
// end is v (CSR own_ptr / own_idx).  The owner's node data is loaded once
// and its sum kept in registers, flushed with one atomic add per component;
// only the other end of each edge receives atomic adds.
template <class P>
__global__ void k_owner(P ph, const int32_t* __restrict__ m0,
                        const int32_t* __restrict__ m1, int64_t N,
                        const int64_t* __restrict__ own_ptr,
                        const int32_t* __restrict__ own_idx,
                        Targets<typename P::TA, P::DIM0> tg) {
  using TN = typename P::TN;
  using TE = typename P::TE;
  using TA = typename P::TA;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += stride) {
    const int64_t t0 = own_ptr[v], t1 = own_ptr[v + 1];
    if (t0 == t1) continue;
    TN vv[P::NIN];
    ph.load(v, vv);
    TA acc[P::OUT];
#pragma unroll
    for (int c = 0; c < P::OUT; c++) acc[c] = TA(0);
    // the next owned edge's id and ends are fetched one iteration ahead, so
    // only the other end's data load is left on each iteration's path
    int64_t e = own_idx[t0];
    int64_t i = m0[e], j = m1[e];
    for (int64_t t = t0; t < t1; t++) {
      const int64_t en = t + 1 < t1 ? (int64_t)own_idx[t + 1] : e;
      const int64_t in = m0[en], jn = m1[en];
      const bool first = (i == v);
      const int64_t w = first ? j : i;
      TN vw[P::NIN];
      ph.load(w, vw);
      // the edge's own orientation whichever end v is: the operands are
      // selected and the body runs once (a branch between two calls would
      // run both bodies in a warp whose threads own edges of both
      // orientations)
      TN va[P::NIN], vb[P::NIN];
#pragma unroll
      for (int k = 0; k < P::NIN; k++) {
        va[k] = first ? vv[k] : vw[k];
        vb[k] = first ? vw[k] : vv[k];
      }
      TE oi[P::OUT], oj[P::MODE == MODE_GEN ? P::OUT : 1];
      ph.edge(e, va, vb, oi, oj);
#pragma unroll
      for (int c = 0; c < P::OUT; c++) {
        const TA a = to_acc<TA>(oi[c]);
        TA b;  // the second end's increment
        if constexpr (P::MODE == MODE_ANTI) b = neg(a);
        else if constexpr (P::MODE == MODE_SYM) b = a;
        else b = to_acc<TA>(oj[c]);
        acc[c] += first ? a : b;
        atomicAdd(tg.at(c, w), first ? b : a);
      }
      e = en;
      i = in;
      j = jn;
    }
#pragma unroll
    for (int c = 0; c < P::OUT; c++) atomicAdd(tg.at(c, v), acc[c]);
  }
}

// (6) redundant gather: thread per node over its edge ends (the node-sorted
// list of the segmented plan); every edge is computed at both of its ends,
// each time in the edge's own orientation (first end, second end), so the
// two evaluations are bitwise identical and the INC stays exactly
// antisymmetric (MODE_ANTI) or symmetric (MODE_SYM).  Each node's sum is
// kept in registers and written once: no race, no atomics, a fixed order
// (bitwise reproducible), at twice the arithmetic.  For bodies without
// per-edge (direct) outputs.  With `add` the sums are added to the targets.
template <class P, class = void>
struct HasDirectOutput {
  static constexpr bool value = false;
};
template <class P>
struct HasDirectOutput<P, std::void_t<decltype(&P::nbar)>> {
  static constexpr bool value = true;
};

template <class P>
__global__ void k_gather_nodes(P ph, const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ ends, const int32_t* __restrict__ m0,
                               const int32_t* __restrict__ m1, int64_t N,
                               Targets<typename P::TA, P::DIM0> tg, bool add) {
  using TN = typename P::TN;
  using TE = typename P::TE;
  using TA = typename P::TA;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    TN vs[P::NIN];
    ph.load(i, vs);
    TA acc[P::OUT];
#pragma unroll
    for (int c = 0; c < P::OUT; c++) acc[c] = TA(0);
    const int64_t t0 = rowptr[i], t1 = rowptr[i + 1];
    // the next end's edge and other node are fetched one iteration ahead
    int32_t end = t0 < t1 ? ends[t0] : 0;
    int64_t o = t0 < t1 ? (end & 1 ? m0[end >> 1] : m1[end >> 1]) : 0;
    for (int64_t t = t0; t < t1; t++) {
      const int64_t e = end >> 1;
      const bool second = end & 1;
      const int32_t endn = t + 1 < t1 ? ends[t + 1] : end;
      const int64_t on = endn & 1 ? m0[endn >> 1] : m1[endn >> 1];
      TN vo[P::NIN];
      ph.load(o, vo);
      // the edge's own orientation whichever end this is (no divergence:
      // the operands are selected, the body runs once)
      TN va[P::NIN], vb[P::NIN];
#pragma unroll
      for (int k = 0; k < P::NIN; k++) {
        va[k] = second ? vo[k] : vs[k];
        vb[k] = second ? vs[k] : vo[k];
      }
      TE oi[P::OUT], oj[P::MODE == MODE_GEN ? P::OUT : 1];
      ph.edge(e, va, vb, oi, oj);
#pragma unroll
      for (int c = 0; c < P::OUT; c++) {
        const TA a = to_acc<TA>(oi[c]);
        if constexpr (P::MODE == MODE_ANTI) acc[c] += second ? neg(a) : a;
        else if constexpr (P::MODE == MODE_SYM) acc[c] += a;
        else acc[c] += second ? to_acc<TA>(oj[c]) : a;
      }
      end = endn;
      o = on;
    }
#pragma unroll
    for (int c = 0; c < P::OUT; c++) {
      TA* p = tg.at(c, i);
      *p = add ? *p + acc[c] : acc[c];
    }
  }
}

// Device view of a block plan (mini-partitions + colours).
struct BlockView {
  const int32_t* cblocks;  // blocks of the colour being launched (null: all
                           // blocks in order, for the atomic flush)
  int64_t nblk;
  int32_t part;
  int32_t ucap;            // staging capacity (max distinct nodes per block)
  const int32_t* bn_off;
  const int32_t* bnodes;
  const uint32_t* eloc;
  const int32_t* lrow;
  const uint16_t* lent;
};

__host__ __device__ constexpr int64_t align16(int64_t b) {
  return (b + 15) & ~(int64_t)15;
}

template <class P>
__host__ __device__ constexpr int outs_per_edge() {
  return P::MODE == MODE_GEN ? 2 * P::OUT : P::OUT;
}

// Bodies with a packed per-edge form (PACK, pack(), unpack_add())
template <class P, class = void>
struct HasPack {
  static constexpr bool value = false;
};
template <class P>
struct HasPack<P, std::void_t<decltype(P::PACK)>> {
  static constexpr bool value = true;
};

// values kept per edge by the colour and segmented strategies
template <class P>
__host__ __device__ constexpr int stored_per_edge() {
  if constexpr (HasPack<P>::value) return P::PACK;
  else return outs_per_edge<P>();
}

// Edge-major stride of the segmented strategy's per-edge buffer: the stored
// values of one edge are contiguous and padded to a multiple of 16 bytes,
// so the node phase reads an edge's values from one or two sectors with
// vector loads (a component-major buffer would touch one sector per value).
template <class P>
__host__ __device__ constexpr int ebuf_stride() {
  constexpr int per16 = 16 / (int)sizeof(typename P::TE);
  return (stored_per_edge<P>() + per16 - 1) / per16 * per16;
}

// copy n values of type T between 16-byte aligned buffers in 16-byte words
template <typename T, int N>
__device__ __forceinline__ void copy16(T* __restrict__ dst, const T* __restrict__ src) {
  static_assert((N * sizeof(T)) % 16 == 0, "16-byte multiple");
#pragma unroll
  for (int k = 0; k < (int)(N * sizeof(T) / 16); k++)
    reinterpret_cast<float4*>(dst)[k] = reinterpret_cast<const float4*>(src)[k];
}

template <class P, bool STAGED>
__host__ int64_t colour_smem_bytes(int32_t part, int32_t ucap) {
  int64_t b = align16((int64_t)stored_per_edge<P>() * part * sizeof(typename P::TE));
  if (STAGED) b += (int64_t)P::NIN * ucap * sizeof(typename P::TN);
  return b;
}

// (2) block colouring: one CTA per edge block of the launched colour.  The
// block's results are kept in shared memory and summed per distinct node
// over the block-local edge-end lists, then added into the targets with
// plain read-modify-writes (no two blocks of a colour share a node).  With
// STAGED the READ data of the block's distinct nodes is first gathered
// into shared memory and the edges read it from there.
// (4) block-atomic (ATOMIC_FLUSH): the same kernel over all blocks in one
// launch, flushing each block's per-node sums with atomic adds: one atomic
// per (block, node, component) instead of one per edge end.
template <class P, bool STAGED, bool ATOMIC_FLUSH = false>
__global__ void k_colour(P ph, const int32_t* __restrict__ m0,
                         const int32_t* __restrict__ m1, int64_t E,
                         BlockView bv, Targets<typename P::TA, P::DIM0> tg) {
  using TN = typename P::TN;
  using TE = typename P::TE;
  using TA = typename P::TA;
  constexpr int OUTS = stored_per_edge<P>();
  extern __shared__ __align__(16) unsigned char smem[];
  const int part = bv.part;
  TE* sOut = reinterpret_cast<TE*>(smem);
  TN* sIn = reinterpret_cast<TN*>(smem + align16((int64_t)OUTS * part * sizeof(TE)));
  for (int64_t bi = blockIdx.x; bi < bv.nblk; bi += gridDim.x) {
    const int64_t b = bv.cblocks ? bv.cblocks[bi] : bi;
    const int64_t e0 = b * part;
    const int ne = (int)min((int64_t)part, E - e0);
    const int64_t u0 = bv.bn_off[b];
    const int U = (int)(bv.bn_off[b + 1] - u0);
    if constexpr (STAGED) {
      for (int u = threadIdx.x; u < U; u += blockDim.x) {
        TN v[P::NIN];
        ph.load(bv.bnodes[u0 + u], v);
#pragma unroll
        for (int k = 0; k < P::NIN; k++) sIn[k * bv.ucap + u] = v[k];
      }
      __syncthreads();
    }
    for (int el = threadIdx.x; el < ne; el += blockDim.x) {
      const int64_t e = e0 + el;
      TN vi[P::NIN], vj[P::NIN];
      if constexpr (STAGED) {
        uint32_t l = bv.eloc[e];
        int li = (int)(l & 0xffffu), lj = (int)(l >> 16);
#pragma unroll
        for (int k = 0; k < P::NIN; k++) {
          vi[k] = sIn[k * bv.ucap + li];
          vj[k] = sIn[k * bv.ucap + lj];
        }
      } else {
        ph.load(m0[e], vi);
        ph.load(m1[e], vj);
      }
      if constexpr (HasPack<P>::value) {
        TE st[P::PACK];
        ph.pack(e, vi, vj, st);
#pragma unroll
        for (int c = 0; c < P::PACK; c++) sOut[c * part + el] = st[c];
      } else {
        TE oi[P::OUT], oj[P::MODE == MODE_GEN ? P::OUT : 1];
        ph.edge(e, vi, vj, oi, oj);
#pragma unroll
        for (int c = 0; c < P::OUT; c++) sOut[c * part + el] = oi[c];
        if constexpr (P::MODE == MODE_GEN) {
#pragma unroll
          for (int c = 0; c < P::OUT; c++) sOut[(P::OUT + c) * part + el] = oj[c];
        }
      }
    }
    __syncthreads();
    const int32_t* lr = bv.lrow + u0 + b;
    const uint16_t* le = bv.lent + 2 * e0;
    for (int u = threadIdx.x; u < U; u += blockDim.x) {
      TA acc[P::OUT];
#pragma unroll
      for (int c = 0; c < P::OUT; c++) acc[c] = TA(0);
      const int r1 = lr[u + 1];
      for (int t = lr[u]; t < r1; t++) {
        const int ent = le[t];
        const int el = ent >> 1;
        const bool second = ent & 1;
        if constexpr (HasPack<P>::value) {
          P::unpack_add([&](int c) { return sOut[c * part + el]; }, second, acc);
        } else if constexpr (P::MODE == MODE_GEN) {
          const int base = second ? P::OUT : 0;
#pragma unroll
          for (int c = 0; c < P::OUT; c++) acc[c] += to_acc<TA>(sOut[(base + c) * part + el]);
        } else {
#pragma unroll
          for (int c = 0; c < P::OUT; c++) {
            TA v = to_acc<TA>(sOut[c * part + el]);
            if constexpr (P::MODE == MODE_ANTI) acc[c] += second ? neg(v) : v;
            else acc[c] += v;
          }
        }
      }
      const int64_t node = bv.bnodes[u0 + u];
#pragma unroll
      for (int c = 0; c < P::OUT; c++) {
        TA* p = tg.at(c, node);
        if constexpr (ATOMIC_FLUSH) atomicAdd(p, acc[c]);
        else *p = *p + acc[c];
      }
    }
    __syncthreads();
  }
}

// (3) sorted segmented reduction, phase 1: each edge's results to a global
// buffer (OUTS x E, component-major).
template <class P>
__global__ void k_seg_edges(P ph, const int32_t* __restrict__ m0,
                            const int32_t* __restrict__ m1, int64_t E,
                            typename P::TE* __restrict__ ebuf) {
  using TN = typename P::TN;
  using TE = typename P::TE;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E;
       e += stride) {
    TN vi[P::NIN], vj[P::NIN];
    ph.load(m0[e], vi);
    ph.load(m1[e], vj);
    constexpr int SP = ebuf_stride<P>();
    __align__(16) TE st[SP];
#pragma unroll
    for (int c = 0; c < SP; c++) st[c] = TE(0);
    if constexpr (HasPack<P>::value) {
      ph.pack(e, vi, vj, st);
    } else {
      TE oj[P::MODE == MODE_GEN ? P::OUT : 1];
      ph.edge(e, vi, vj, st, oj);
      if constexpr (P::MODE == MODE_GEN) {
#pragma unroll
        for (int c = 0; c < P::OUT; c++) st[P::OUT + c] = oj[c];
      }
    }
    copy16<TE, SP>(ebuf + e * SP, st);
  }
}

// Phase 2 for bodies with a packed per-edge form (Green-Gauss).  Every
// node's sums are written once: added to the targets with `add`, else
// written over them (no zeroing pass needed), and with `vol` multiplied by
// the node's 1/V as they are written -- the gradient scaling fused into the
// write, formed as the scaling loop forms it (1/V in FP64, then rounded to
// the target type), so the result is bitwise the two loops'.
template <class P>
__global__ void k_seg_nodes_packed(const int64_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ ends, int64_t N,
                                   int64_t E, const typename P::TE* __restrict__ ebuf,
                                   Targets<typename P::TA, P::DIM0> tg,
                                   const double* __restrict__ vol, bool add) {
  using TA = typename P::TA;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += stride) {
    TA acc[P::OUT];
#pragma unroll
    for (int c = 0; c < P::OUT; c++) acc[c] = TA(0);
    constexpr int SP = ebuf_stride<P>();
    const int64_t r1 = rowptr[i + 1];
    for (int64_t t = rowptr[i]; t < r1; t++) {
      const int32_t end = ends[t];
      __align__(16) typename P::TE st[SP];
      copy16<typename P::TE, SP>(st, ebuf + (int64_t)(end >> 1) * SP);
      P::unpack_add([&](int c) { return st[c]; }, (end & 1) != 0, acc);
    }
    const TA r = vol ? (TA)(1.0 / vol[i]) : TA(1);
#pragma unroll
    for (int c = 0; c < P::OUT; c++) {
      TA* p = tg.at(c, i);
      const TA v = add ? *p + acc[c] : acc[c];
      *p = vol ? v * r : v;
    }
  }
}

// Phase 2: the edge ends are sorted by node (CSR); each node's segment is
// summed by one thread in edge order and added into the targets.  The
// per-edge buffer is edge-major (see ebuf_stride()).  A
// warp-cooperative scan would cost log2(32) = 5 adds per end instead of 1,
// which the FP64 pipe cannot spare, so segments are reduced one per lane.
template <typename TE, typename TA, int OUT, int MODE, int DIM0>
__global__ void k_seg_nodes(const int64_t* __restrict__ rowptr,
                            const int32_t* __restrict__ ends, int64_t N,
                            int64_t E, const TE* __restrict__ ebuf,
                            Targets<TA, DIM0> tg) {
  // edge-major buffer, stride as ebuf_stride(): OUTS values padded to 16 B
  constexpr int OUTS = MODE == MODE_GEN ? 2 * OUT : OUT;
  constexpr int per16 = 16 / (int)sizeof(TE);
  constexpr int SP = (OUTS + per16 - 1) / per16 * per16;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += stride) {
    TA acc[OUT];
#pragma unroll
    for (int c = 0; c < OUT; c++) acc[c] = TA(0);
    const int64_t r1 = rowptr[i + 1];
    for (int64_t t = rowptr[i]; t < r1; t++) {
      const int32_t end = ends[t];
      const int64_t e = end >> 1;
      const bool second = end & 1;
      if constexpr (MODE == MODE_GEN) {
        // only this end's half: OUT values at offset 0 or OUT
        static_assert((OUT * sizeof(TE)) % 16 == 0, "halves must be 16-byte aligned");
        __align__(16) TE st[OUT];
        copy16<TE, OUT>(st, ebuf + e * SP + (second ? OUT : 0));
#pragma unroll
        for (int c = 0; c < OUT; c++) acc[c] += to_acc<TA>(st[c]);
      } else {
        __align__(16) TE st[SP];
        copy16<TE, SP>(st, ebuf + e * SP);
#pragma unroll
        for (int c = 0; c < OUT; c++) {
          TA v = to_acc<TA>(st[c]);
          if constexpr (MODE == MODE_ANTI) acc[c] += second ? neg(v) : v;
          else acc[c] += v;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < OUT; c++) {
      TA* p = tg.at(c, i);
      *p = *p + acc[c];
    }
  }
}

}  // namespace op2b
