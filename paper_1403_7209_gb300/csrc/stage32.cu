// op2b_stage_mixed: one second-order explicit Runge-Kutta stage in the
// FP32-mixed precision, fused into two node passes over packed FP32 node
// records.
//
// The stage is the paper's sequence of parallel loops -- the Green-Gauss
// edge loop with the gradient scaling, the limited Rusanov flux edge loop
// and the node update (Sec. 2's Runge-Kutta march, Table "loopperfmpi":
// accumedges, ifluxedge, updatek) -- with FP32 node data, gradients,
// normals and flux arithmetic and an FP64 residual and update.
//
// Why it is laid out this way on GB300.  Gathering a node's 24 FP32 values
// from structure-of-arrays dats touches 24 separate 32-byte sectors; the
// packed record (q then G, 96 bytes: three sectors, three 32-byte loads) cuts
// the L2 traffic of every gather by 8x.  Accumulating the edge fluxes into
// FP64 needs 12 FP64 additions per edge, which GB300's FP64 pipe (2 per
// clock per SM) cannot absorb -- 108M per stage on the 1M-node lattice,
// longer than the stage's whole HBM floor -- and FP64 atomics at the L2 are
// slower still.  So both passes are node gathers (no atomics, no race, a
// fixed summation order, bitwise reproducible) and each node's flux sum is
// carried as an unevaluated pair of floats built with Knuth's error-free
// two-sum, converted exactly to FP64 once per node: the pair holds the sum
// of the FP32 fluxes to about 2^-48 of its running magnitude.
//
//   pass 1 (Green-Gauss, 1 thread per node): G_i = (1/V_i) sum over the
//     node's edge ends of (q_i + q_j) (x) (+-n/2), written into the record's
//     G part (and into an optional FP32 G dat);
//   pass 2 (flux + update, 1 thread per node): for every edge end the edge's
//     flux with the node as the first end (the edge reversed at its second
//     end, which gives bitwise minus the first end's value, so the residual
//     stays exactly antisymmetric), summed; then R_i in FP64 and
//     q_i = q0_i - alpha (dt_i / V_i) R_i, written to q (FP64), to the other
//     record buffer's q part (FP32) and optionally to R and q0.
#include <algorithm>
#include <string>

#include "edge_math.cuh"
#include "f32x2.cuh"
#include "host_plan.h"
#include "internal.h"

namespace op2b {

namespace {

// floats per node record: q (6), then G dimension-major: dq_k/dx for
// k = 0..5, then dq_k/dy, then dq_k/dz (so that the gradients of two
// consecutive components are adjacent, as the paired FP32 instructions of
// the flux pass want them)
constexpr int REC = 24;
constexpr int GX = 6, GY = 12, GZ = 18;

template <typename T>
__device__ __forceinline__ float f32_of(T x) {
  return (float)x;
}

// the staged passes' adjacency, sliced-ELL with local ids: for slot s with
// node-sorted end t = sell_end[s] (-1: padding), adjn_s = {lother[t], +-n/2},
// adje_s = {2 lother[t] + side, 2e + side}
template <typename TN>
__global__ void k_s32_adjacency_sell(const int32_t* __restrict__ sell_end, int64_t nslots,
                                     const int32_t* __restrict__ ends,
                                     const int32_t* __restrict__ lother,
                                     const TN* __restrict__ n, int64_t ldn,
                                     int4* __restrict__ adjn_s, int2* __restrict__ adje_s) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslots;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = sell_end[s];
    if (t < 0) {
      adjn_s[s] = make_int4(-1, 0, 0, 0);
      adje_s[s] = make_int2(-1, 0);
      continue;
    }
    const int32_t end = ends[t];
    const int64_t e = end >> 1;
    const bool second = end & 1;
    const int32_t lj = lother[t];
    const float h = second ? -0.5f : 0.5f;
    const float hx = f32_of(n[e]) * h, hy = f32_of(n[ldn + e]) * h, hz = f32_of(n[2 * ldn + e]) * h;
    adjn_s[s] = make_int4(lj, __float_as_int(hx), __float_as_int(hy), __float_as_int(hz));
    adje_s[s] = make_int2(2 * lj + (int)second, end);
  }
}

// per edge: {n_x, n_y, n_z, dx_x}, {dx_y, dx_z, 0, 0} in FP32 (32 bytes, one sector)
template <typename TN, typename TD>
__global__ void k_s32_geometry(int64_t E, const TN* __restrict__ n, int64_t ldn,
                               const TD* __restrict__ dx, int64_t lddx, float4* __restrict__ geo) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    geo[2 * e] = make_float4(f32_of(n[e]), f32_of(n[ldn + e]), f32_of(n[2 * ldn + e]), f32_of(dx[e]));
    geo[2 * e + 1] = make_float4(f32_of(dx[lddx + e]), f32_of(dx[2 * lddx + e]), 0.0f, 0.0f);
  }
}

// The direct passes' adjacency, sliced-ELL: the k-th end of node i (in the
// node-sorted order) at slot ell_off[i / 32] + 32 k + i % 32, so that the
// ends a warp's 32 nodes read together are contiguous.  Per slot
// adjn_l = {other end j, +-n/2 (FP32 bits)} (Green-Gauss pass) and
// ende = {j (bits), s n, s dx, 0} with s = -1 at the edge's second end, the
// edge already reversed (flux pass; 32 bytes, one sector).
template <typename TN, typename TD>
__global__ void k_s32_adjacency_ell(const int32_t* __restrict__ ends, int64_t nends,
                                    const int64_t* __restrict__ rowptr,
                                    const int64_t* __restrict__ ell_off,
                                    const int32_t* __restrict__ m0, const int32_t* __restrict__ m1,
                                    const TN* __restrict__ n, int64_t ldn,
                                    const TD* __restrict__ dx, int64_t lddx,
                                    int4* __restrict__ adjn_l, float4* __restrict__ ende) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nends;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t end = ends[t];
    const int64_t e = end >> 1;
    const bool second = end & 1;
    const int32_t i = second ? m1[e] : m0[e];
    const int32_t j = second ? m0[e] : m1[e];
    const int64_t s = ell_off[i >> 5] + 32 * (t - rowptr[i]) + (i & 31);
    const float nx = f32_of(n[e]), ny = f32_of(n[ldn + e]), nz = f32_of(n[2 * ldn + e]);
    const float h = second ? -0.5f : 0.5f;
    adjn_l[s] = make_int4(j, __float_as_int(nx * h), __float_as_int(ny * h),
                          __float_as_int(nz * h));
    const float dxx = f32_of(dx[e]), dxy = f32_of(dx[lddx + e]), dxz = f32_of(dx[2 * lddx + e]);
    if (second) {
      ende[2 * s] = make_float4(__int_as_float(j), -nx, -ny, -nz);
      ende[2 * s + 1] = make_float4(-dxx, -dxy, -dxz, 0.0f);
    } else {
      ende[2 * s] = make_float4(__int_as_float(j), nx, ny, nz);
      ende[2 * s + 1] = make_float4(dxx, dxy, dxz, 0.0f);
    }
  }
}

// record q part <- (float) q
__global__ void k_s32_pack_q(int64_t N, const double* __restrict__ q, int64_t ldq,
                             float* __restrict__ rec) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 6; k++) rec[i * REC + k] = (float)q[k * ldq + i];
  }
}

// 32 bytes (8 floats) from a 32-byte aligned address in one load
__device__ __forceinline__ void ldg8(const float* __restrict__ p, float* v) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7])
      : "l"(p));
}

// the same through the coherent path: for records whose other bytes the
// running kernel writes (the Green-Gauss pass writes the G parts while it
// reads the q parts)
__device__ __forceinline__ void ld8(const float* p, float* v) {
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                 "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}

// a node record (96 bytes at a multiple of 96: 32-byte aligned) in three loads
__device__ __forceinline__ void load_rec(const float* __restrict__ p, float* v) {
#pragma unroll
  for (int k = 0; k < 3; k++) ldg8(p + 8 * k, v + 8 * k);
}

__device__ __forceinline__ float rcp_f(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_f(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ f2 rcp2(f2 a) { return mk2(rcp_f(a.x), rcp_f(a.y)); }

struct GasPairs {
  f2 gm1, gamma, eps, two_eps;
};

// van Albada phi(a, b) = (a + b)(ab + eps) / (a^2 + (b^2 + 2 eps)) on two
// components at once (b2e = b^2 + 2 eps); the quotient as the product with
// the FP32 special-function reciprocal
__device__ __forceinline__ f2 van_albada2(f2 a, f2 b, f2 eps, f2 b2e) {
  const f2 num = mul2(add2(a, b), fma2(a, b, eps));
  return mul2(num, rcp2(fma2(a, a, b2e)));
}

// The second-order flux of one edge in FP32 on paired instructions: the
// limited reconstruction on component pairs (0,1), (2,3), (4,5), the Euler
// fluxes of the two face states on (left, right) pairs, the Rusanov
// combination per component.  va / vb: the first and the second end's
// records (q, then G dimension-major); g0 = (n, dx_x), g1 = (dx_y, dx_z).
__device__ __forceinline__ void flux2_pairs(const float* va, const float* vb, float4 g0,
                                            float4 g1, GasPairs g, float* F) {
  const f2 dx2 = splat2(g0.w), dy2 = splat2(g1.x), dz2 = splat2(g1.y);
  float qL[6], qR[6];
#pragma unroll
  for (int k = 0; k < 6; k += 2) {
    const f2 a = mk2(va[k], va[k + 1]), b = mk2(vb[k], vb[k + 1]);
    const f2 jump = sub2(b, a);
    const f2 ai = fma2(mk2(va[GZ + k], va[GZ + k + 1]), dz2,
                       fma2(mk2(va[GY + k], va[GY + k + 1]), dy2,
                            mul2(mk2(va[GX + k], va[GX + k + 1]), dx2)));
    const f2 aj = fma2(mk2(vb[GZ + k], vb[GZ + k + 1]), dz2,
                       fma2(mk2(vb[GY + k], vb[GY + k + 1]), dy2,
                            mul2(mk2(vb[GX + k], vb[GX + k + 1]), dx2)));
    const f2 b2e = fma2(jump, jump, g.two_eps);
    const f2 l = fma2(splat2(0.5f), van_albada2(ai, jump, g.eps, b2e), a);
    const f2 r = fma2(splat2(-0.5f), van_albada2(aj, jump, g.eps, b2e), b);
    qL[k] = l.x;
    qL[k + 1] = l.y;
    qR[k] = r.x;
    qR[k + 1] = r.y;
  }
  // Euler flux f(q).n and wave speed |u.n| + a|n| of both face states
  const float nx = g0.x, ny = g0.y, nz = g0.z;
  const float nn2 = fmaf(nz, nz, fmaf(ny, ny, nx * nx));
  const f2 rho = mk2(qL[0], qR[0]), m1 = mk2(qL[1], qR[1]), m2 = mk2(qL[2], qR[2]);
  const f2 m3 = mk2(qL[3], qR[3]), en = mk2(qL[4], qR[4]), cs = mk2(qL[5], qR[5]);
  const f2 rr = rcp2(rho);
  const f2 nx2 = splat2(nx), ny2 = splat2(ny), nz2 = splat2(nz);
  const f2 un = mul2(fma2(m3, nz2, fma2(m2, ny2, mul2(m1, nx2))), rr);
  const f2 mm = fma2(m3, m3, fma2(m2, m2, mul2(m1, m1)));
  const f2 p = mul2(g.gm1, fma2(mul2(splat2(-0.5f), mm), rr, en));
  const f2 a2n = mul2(mul2(mul2(g.gamma, p), rr), splat2(nn2));
  const float lL = fabsf(un.x) + sqrt_f(a2n.x), lR = fabsf(un.y) + sqrt_f(a2n.y);
  const float hs = 0.5f * (lL >= lR ? lL : lR);
  const f2 f0 = mul2(rho, un);
  const f2 f1 = fma2(m1, un, mul2(p, nx2));
  const f2 f2_ = fma2(m2, un, mul2(p, ny2));
  const f2 f3 = fma2(m3, un, mul2(p, nz2));
  const f2 f4 = mul2(add2(en, p), un);
  const f2 f5 = mul2(cs, un);
  const f2 f[6] = {f0, f1, f2_, f3, f4, f5};
#pragma unroll
  for (int k = 0; k < 6; k++) F[k] = fmaf(-hs, qR[k] - qL[k], 0.5f * (f[k].x + f[k].y));
}

// Pass 2: every edge end evaluates its edge's flux with its own node as the
// first end -- for a node that is the edge's second end the edge reversed:
// n -> -n, dx -> -dx, which gives exactly -F of the edge's own orientation
// (every operation of the flux is odd or even in those signs and rounds
// symmetrically), the second end's share -- so the node's record is loaded
// once and no operand is selected.  The shares are summed with two-sum
// pairs, then the FP64 residual and the node update.

// one edge end: the node's record vi, the other end's record vj, the edge
// geometry (n, dx; 32 bytes) and the end's side; adds the share to (hi, lo)
// an edge's geometry (n, dx) as two 16-byte words, loaded in one 32-byte load
struct Geo {
  float4 a, b;
};
__device__ __forceinline__ Geo ldg_geo(const float* __restrict__ p) {
  Geo g;
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(g.a.x), "=f"(g.a.y), "=f"(g.a.z), "=f"(g.a.w), "=f"(g.b.x), "=f"(g.b.y),
        "=f"(g.b.z), "=f"(g.b.w)
      : "l"(p));
  return g;
}

__device__ __forceinline__ void flux_end_g(const float* vi, const float* vj, Geo gv,
                                           bool second, GasPairs gas, f2* hi, f2* lo) {
  float4 g0 = gv.a, g1 = make_float4(gv.b.x, gv.b.y, 0.f, 0.f);
  if (second) {  // the edge reversed
    g0 = make_float4(neg(g0.x), neg(g0.y), neg(g0.z), neg(g0.w));
    g1 = make_float4(neg(g1.x), neg(g1.y), 0.0f, 0.0f);
  }
  float F[6];
  flux2_pairs(vi, vj, g0, g1, gas, F);
#pragma unroll
  for (int k = 0; k < 3; k++) two_sum_acc2(hi[k], lo[k], mk2(F[2 * k], F[2 * k + 1]));
}

// R_i from the pair sums (each float converted exactly, one FP64 add) and the
// update of components [k0, k1) of node i
__device__ __forceinline__ void finish_node(int64_t i, const f2* hi, const f2* lo, int k0, int k1,
                                            float* __restrict__ rout, double* __restrict__ q0,
                                            int64_t ld0, double* __restrict__ q, int64_t ldq,
                                            const double* __restrict__ V,
                                            const double* __restrict__ dt, double alpha,
                                            double* __restrict__ R, int64_t ldR, bool store_q0) {
  const double a = alpha * (dt[i] / V[i]);
#pragma unroll
  for (int k = 0; k < 6; k++) {
    if (k < k0 || k >= k1) continue;
    const float h = k & 1 ? hi[k >> 1].y : hi[k >> 1].x;
    const float l = k & 1 ? lo[k >> 1].y : lo[k >> 1].x;
    const double Rk = to_acc<double>(h) + to_acc<double>(l);
    const double v = q0[k * ld0 + i] - a * Rk;
    q[k * ldq + i] = v;
    rout[i * REC + k] = (float)v;
    if (R) R[k * ldR + i] = Rk;
    if (store_q0) q0[k * ld0 + i] = v;
  }
}

// the adjacency is read once per stage: loaded without allocating in L1,
// which the node records use
__device__ __forceinline__ int4 ld_stream4(const int4* p) {
  int4 a;
  asm("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
      : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w)
      : "l"(p));
  return a;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int NPEND>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(NPEND) : "memory");
}

// Direct form of both passes: one thread per node, CTAs of 128 consecutive
// nodes, every other end's record (or q part) gathered from global memory
// through the sliced-ELL adjacency (the k-th ends of a warp's 32 nodes read
// in one coalesced load).

// Pass 1: Green-Gauss with the scaling: each end's other node's q comes in
// one 32-byte load (the record's first 8 floats: q and two G values, unused,
// which other threads may be writing: coherent loads).  Same operations in
// the same order as the FP32 Green-Gauss node gather, so the same bits.
// The pass waits on its gathers; six ends per unrolled iteration keep
// several gathers in flight per thread (4% faster per stage than two).  A
// minimum of 7 blocks per SM gives it 72 registers (measured: 1.5% faster
// per stage than with no minimum, 66 registers; minima of 8, 9 or 1 blocks,
// 64, 56 or 108 registers, slower).
__global__ void __launch_bounds__(128, 7) k_s32_green_gauss(
    int64_t N, const int64_t* __restrict__ rowptr, const int64_t* __restrict__ ell_off,
    const int4* __restrict__ adjn_l, float* __restrict__ rec, const double* __restrict__ V,
    float* __restrict__ Gout, int64_t ldG) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float qi[8];
    ld8(rec + i * REC, qi);
    float acc[18];
#pragma unroll
    for (int c = 0; c < 18; c++) acc[c] = 0.0f;
    const int64_t deg = rowptr[i + 1] - rowptr[i];
    const int4* a_i = adjn_l + ell_off[i >> 5] + (i & 31);
#pragma unroll 6
    for (int64_t k = 0; k < deg; k++) {
      const int4 a = ld_stream4(a_i + 32 * k);
      float qj[8];
      ld8(rec + (int64_t)a.x * REC, qj);
      const float h[3] = {__int_as_float(a.y), __int_as_float(a.z), __int_as_float(a.w)};
#pragma unroll
      for (int c = 0; c < 6; c++) {
        const float sc = qi[c] + qj[c];
#pragma unroll
        for (int d = 0; d < 3; d++) acc[3 * c + d] = fmaf(sc, h[d], acc[3 * c + d]);
      }
    }
    const float r = (float)(1.0 / V[i]);
    float gd[18];  // the record's G part, dimension-major: gd[6 d + k] = G[3 k + d]
#pragma unroll
    for (int c = 0; c < 18; c++) {  // c = 3 k + d
      const float v = acc[c] * r;
      gd[6 * (c % 3) + c / 3] = v;
      if (Gout) Gout[c * ldG + i] = v;
    }
    float* g = rec + i * REC;
    *reinterpret_cast<float2*>(g + GX) = make_float2(gd[0], gd[1]);
#pragma unroll
    for (int k = 0; k < 4; k++)
      *reinterpret_cast<float4*>(g + GX + 2 + 4 * k) =
          make_float4(gd[2 + 4 * k], gd[3 + 4 * k], gd[4 + 4 * k], gd[5 + 4 * k]);
  }
}

// Pass 2: flux + update.  Per end a 32-byte end record {j, s n, s dx} (the
// edge already reversed at its second end) and the other node's record.
// The end records stream from DRAM; each thread copies them by cp.async
// into its own ring of kRing shared-memory slots, kRing - 1 ends ahead of
// their use, so that an end waits only for its node-record gather, not for
// the DRAM read of the index that gather needs.  At most 80 registers
// (6 CTAs of 128 per SM).
constexpr int kFluxBlock = 128;
constexpr int kRing = 4;

__global__ void __launch_bounds__(kFluxBlock, 6) k_s32_flux_update(
    int64_t N, const int64_t* __restrict__ rowptr, const int64_t* __restrict__ ell_off,
    const float* __restrict__ ende, const float* __restrict__ rin, float* __restrict__ rout,
    double* __restrict__ q0, int64_t ld0, double* __restrict__ q, int64_t ldq,
    const double* __restrict__ V, const double* __restrict__ dt, double alpha,
    double* __restrict__ R, int64_t ldR, bool store_q0, GasPairs gas) {
  constexpr int PD = kRing, B = kFluxBlock;
  // word h of ring slot s of thread t at ring[2 (s B + t) + h]: each slot
  // holds the warp's 32 end records as they lie in global memory (a
  // thread's two 16-byte words adjacent).  Measured: with each word's 32
  // threads contiguous instead (no bank conflicts on the reads) the copies
  // made 2.3x the L2 requests and the stage ran 11% slower.
  __shared__ float4 ring[PD * 2 * B];
  float4* my = ring + 2 * threadIdx.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float vi[REC];
    load_rec(rin + i * REC, vi);
    f2 hi[3], lo[3];
#pragma unroll
    for (int k = 0; k < 3; k++) hi[k] = lo[k] = splat2(0.0f);
    const int deg = (int)(rowptr[i + 1] - rowptr[i]);
    const float* e_i = ende + 8 * (ell_off[i >> 5] + (i & 31));
#pragma unroll
    for (int s = 0; s < PD - 1; s++) {
      if (s < deg) {
        cp_async16(my + 2 * s * B, e_i + 256 * s);
        cp_async16(my + 2 * s * B + 1, e_i + 256 * s + 4);
      }
      cp_async_commit();  // one group per end, empty past the row's end
    }
    int sw = PD - 1, sr = 0;  // the ring slots written and read next
    const float* src = e_i + 256 * (PD - 1);  // end k + PD - 1 (read only below deg)
#pragma unroll 1
    for (int k = 0; k < deg; k++) {
      if (k + PD - 1 < deg) {
        cp_async16(my + 2 * sw * B, src);
        cp_async16(my + 2 * sw * B + 1, src + 4);
      }
      cp_async_commit();
      src += 256;
      sw = sw == PD - 1 ? 0 : sw + 1;
      cp_async_wait_group<PD - 1>();  // end k's group is complete
      Geo g;
      g.a = my[2 * sr * B];
      g.b = my[2 * sr * B + 1];
      sr = sr == PD - 1 ? 0 : sr + 1;
      float vj[REC];
      load_rec(rin + (int64_t)__float_as_int(g.a.x) * REC, vj);
      float F[6];
      flux2_pairs(vi, vj, make_float4(g.a.y, g.a.z, g.a.w, g.b.x),
                  make_float4(g.b.y, g.b.z, 0.0f, 0.0f), gas, F);
#pragma unroll
      for (int c = 0; c < 3; c++) two_sum_acc2(hi[c], lo[c], mk2(F[2 * c], F[2 * c + 1]));
    }
    cp_async_wait_all();
    finish_node(i, hi, lo, 0, 6, rout, q0, ld0, q, ldq, V, dt, alpha, R, ldR, store_q0);
  }
}

// ------------------------------------------------------------ staged form
// One CTA per block of B consecutive nodes, one thread per node.  The
// records of the block's neighbourhood (its own nodes, then every other
// node its ends reach: the node-block plan) are first copied into shared
// memory by asynchronous 16-byte copies (cp.async: every copy in flight at
// once, no register round trip), so that an end reads its other node's
// record there -- each record is read from global memory once per block
// instead of once per edge end.  The ends are read sliced-ELL (the k-th
// ends of a warp's 32 nodes at consecutive addresses, coalesced) and carry
// the other node's local id.  Several CTAs per SM overlap one block's
// copies with another block's arithmetic.

constexpr int SREC4 = 7;  // 16-byte words per record slot in shared memory
                          // (112 bytes: an odd multiple of 16, so that the
                          // 16-byte reads of eight slots fall in different
                          // bank groups)
constexpr int SQ4 = 3;    // 16-byte words per q slot of the Green-Gauss pass

// Pass 1, staged: q parts of the neighbourhood in shared memory; adjn_s =
// {local id of the other node (-1: padding), +-n/2 (FP32 bits)} sliced-ELL.
// The same operations in the same order as the direct form, so the same bits.
__global__ void __launch_bounds__(128) k_s32_green_gauss_sell(
    int64_t N, int32_t B, const int64_t* __restrict__ uoff, const int32_t* __restrict__ uniq,
    const int64_t* __restrict__ sell_off, const int4* __restrict__ adjn_s,
    float* __restrict__ rec, const double* __restrict__ V, float* __restrict__ Gout,
    int64_t ldG) {
  extern __shared__ float4 sq[];
  const int64_t b = blockIdx.x;
  const int64_t u0 = uoff[b];
  const int U = (int)(uoff[b + 1] - u0);
  for (int u = threadIdx.x; u < U; u += blockDim.x) {
    const float* src = rec + (int64_t)uniq[u0 + u] * REC;
    cp_async16(sq + u * SQ4, src);
    cp_async8(sq + u * SQ4 + 1, src + 4);
  }
  cp_async_wait_all();
  __syncthreads();
  const int li = threadIdx.x;
  const int64_t i = b * B + li;
  if (li >= B || i >= N) return;
  const float* sqf = reinterpret_cast<const float*>(sq);
  float qi[6];
#pragma unroll
  for (int k = 0; k < 6; k++) qi[k] = sqf[li * 4 * SQ4 + k];
  float acc[18];
#pragma unroll
  for (int c = 0; c < 18; c++) acc[c] = 0.0f;
  const int64_t sl = i >> 5;
  const int64_t base = sell_off[sl] + (i & 31);
  const int K = (int)((sell_off[sl + 1] - sell_off[sl]) >> 5);
  int4 a = K > 0 ? __ldg(adjn_s + base) : make_int4(-1, 0, 0, 0);
  for (int k = 0; k < K; k++) {
    const int4 an = k + 1 < K ? __ldg(adjn_s + base + 32 * (k + 1)) : make_int4(-1, 0, 0, 0);
    if (a.x >= 0) {
      const float* qj = sqf + a.x * 4 * SQ4;
      const float h[3] = {__int_as_float(a.y), __int_as_float(a.z), __int_as_float(a.w)};
#pragma unroll
      for (int c = 0; c < 6; c++) {
        const float sc = qi[c] + qj[c];
#pragma unroll
        for (int d = 0; d < 3; d++) acc[3 * c + d] = fmaf(sc, h[d], acc[3 * c + d]);
      }
    }
    a = an;
  }
  const float r = (float)(1.0 / V[i]);
  float gd[18];  // the record's G part, dimension-major: gd[6 d + k] = G[3 k + d]
#pragma unroll
  for (int c = 0; c < 18; c++) {  // c = 3 k + d
    const float v = acc[c] * r;
    gd[6 * (c % 3) + c / 3] = v;
    if (Gout) Gout[c * ldG + i] = v;
  }
  // floats 6..23 of the record: one 8-byte and four 16-byte stores
  float* g = rec + i * REC;
  *reinterpret_cast<float2*>(g + GX) = make_float2(gd[0], gd[1]);
#pragma unroll
  for (int k = 0; k < 4; k++)
    *reinterpret_cast<float4*>(g + GX + 2 + 4 * k) =
        make_float4(gd[2 + 4 * k], gd[3 + 4 * k], gd[4 + 4 * k], gd[5 + 4 * k]);
}

// Pass 2, staged: records of the neighbourhood in shared memory; adje_s =
// {2 (local id of the other node) + side (-1: padding), 2e + side}
// sliced-ELL.  Two threads per node: the CTA's first B threads take the
// node's even-numbered ends, the other B the odd ones (each warp still reads
// the ends of 32 consecutive nodes from consecutive addresses); the second
// half leaves its pair sums in shared memory and the first combines them
// exactly (two-sum) and updates the node.  The other end's record is read
// from shared memory where the arithmetic needs it (few registers, more
// warps); each end's geometry is fetched one end ahead and its entry two
// ahead, so that their latency hides behind the arithmetic of the current end.
__global__ void __launch_bounds__(256, 3) k_s32_flux_update_sell(
    int64_t N, int32_t B, const int64_t* __restrict__ uoff, const int32_t* __restrict__ uniq,
    const int64_t* __restrict__ sell_off, const int2* __restrict__ adje_s,
    const float* __restrict__ geo, const float* __restrict__ rin, float* __restrict__ rout,
    double* __restrict__ q0, int64_t ld0, double* __restrict__ q, int64_t ldq,
    const double* __restrict__ V, const double* __restrict__ dt, double alpha,
    double* __restrict__ R, int64_t ldR, bool store_q0, GasPairs gas) {
  extern __shared__ float4 srec[];
  const int64_t b = blockIdx.x;
  const int64_t u0 = uoff[b];
  const int U = (int)(uoff[b + 1] - u0);
  const float4* rin4 = reinterpret_cast<const float4*>(rin);
  for (int f = threadIdx.x; f < 6 * U; f += blockDim.x) {
    const int u = f / 6, k = f - 6 * u;
    cp_async16(srec + u * SREC4 + k, rin4 + (int64_t)uniq[u0 + u] * (REC / 4) + k);
  }
  cp_async_wait_all();
  __syncthreads();
  const float* sf = reinterpret_cast<const float*>(srec);
  float* spart = reinterpret_cast<float*>(srec + U * SREC4);  // B x 12 floats
  const int half = threadIdx.x >= B;
  const int li = threadIdx.x - half * B;
  const int64_t i = b * B + li;
  const bool live = i < N;
  f2 hi[3], lo[3];
#pragma unroll
  for (int k = 0; k < 3; k++) hi[k] = lo[k] = splat2(0.0f);
  if (live) {
    float vi[REC];
    const float4* si = srec + li * SREC4;
#pragma unroll
    for (int k = 0; k < REC / 4; k++) {
      const float4 x = si[k];
      vi[4 * k] = x.x;
      vi[4 * k + 1] = x.y;
      vi[4 * k + 2] = x.z;
      vi[4 * k + 3] = x.w;
    }
    const int64_t sl = i >> 5;
    const int64_t base = sell_off[sl] + (i & 31);
    const int K = (int)((sell_off[sl + 1] - sell_off[sl]) >> 5);
    const int2 pad = make_int2(-1, 0);
    int2 a0 = half < K ? __ldg(adje_s + base + 32 * half) : pad;
    int2 a1 = half + 2 < K ? __ldg(adje_s + base + 32 * (half + 2)) : pad;
    // padding entries (x < 0) read edge 0's geometry (in bounds), unused
    Geo g0 = ldg_geo(geo + 8 * (int64_t)(a0.x >= 0 ? a0.y >> 1 : 0));
    for (int k = half; k < K; k += 2) {
      const int2 a2 = k + 4 < K ? __ldg(adje_s + base + 32 * (k + 4)) : pad;
      const Geo g1 = ldg_geo(geo + 8 * (int64_t)(a1.x >= 0 ? a1.y >> 1 : 0));
      if (a0.x >= 0) flux_end_g(vi, sf + (a0.x >> 1) * 4 * SREC4, g0, a0.x & 1, gas, hi, lo);
      a0 = a1;
      a1 = a2;
      g0 = g1;
    }
    if (half) {
#pragma unroll
      for (int k = 0; k < 3; k++) {
        spart[li * 12 + 4 * k] = hi[k].x;
        spart[li * 12 + 4 * k + 1] = hi[k].y;
        spart[li * 12 + 4 * k + 2] = lo[k].x;
        spart[li * 12 + 4 * k + 3] = lo[k].y;
      }
    }
  }
  __syncthreads();
  if (half || !live) return;
#pragma unroll
  for (int k = 0; k < 3; k++) {  // the two halves' pairs, combined exactly
    const f2 oh = mk2(spart[li * 12 + 4 * k], spart[li * 12 + 4 * k + 1]);
    const f2 ol = mk2(spart[li * 12 + 4 * k + 2], spart[li * 12 + 4 * k + 3]);
    f2 h = hi[k], l = splat2(0.0f);
    two_sum_acc2(h, l, oh);
    hi[k] = h;
    lo[k] = add2(add2(lo[k], ol), l);
  }
  finish_node(i, hi, lo, 0, 6, rout, q0, ld0, q, ldq, V, dt, alpha, R, ldR, store_q0);
}

unsigned grid_all(int64_t work, int block) {
  const int64_t g = (work + block - 1) / block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 0x7fffffff));
}

unsigned grid_of(const Ctx& c, int64_t work, int block) {
  const int64_t g = (work + block - 1) / block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)c.sm_count * 64));
}

void free_stage32(Stage32Plan& p) {
  cudaFree(p.uoff);
  cudaFree(p.uniq);
  cudaFree(p.lother);
  cudaFree(p.sell_off);
  cudaFree(p.sell_end);
  cudaFree(p.adjn_s);
  cudaFree(p.adje_s);
  cudaFree(p.geo);
  cudaFree(p.ell_off);
  cudaFree(p.adjn_l);
  cudaFree(p.ende);
  cudaFree(p.rec[0]);
  cudaFree(p.rec[1]);
  p = Stage32Plan();
}

template <typename T>
int alloc(Ctx& c, T** p, size_t count) {
  if (cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return c.fail(OP2B_ENOMEM, "stage_mixed: allocation of the packed records failed");
  }
  return OP2B_OK;
}

template <typename T>
int upload(Ctx& c, T** p, const std::vector<T>& v) {
  int rc = alloc(c, p, v.size());
  if (rc) return rc;
  if (!v.empty() && cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) !=
                        cudaSuccess)
    return c.fail(OP2B_ECUDA, "stage_mixed: upload of the staging plan failed");
  return OP2B_OK;
}

int check_dat(Ctx& c, op2b_dat d, int dim, op2b_set set, bool f64_only, bool f32_only,
              const char* role) {
  const std::string at = std::string("stage_mixed: ") + role;
  if (d < 0 || d >= (op2b_dat)c.dats.size()) return c.fail(OP2B_EINVAL, at + ": bad dat");
  const DatRec& r = c.dats[d];
  if (r.set != set) return c.fail(OP2B_ESET, at + ": dat on the wrong set");
  if (r.dim != dim) return c.fail(OP2B_EDIM, at + ": dim " + std::to_string(r.dim) + ", expected " +
                                                 std::to_string(dim));
  if (f64_only && r.type != OP2B_F64) return c.fail(OP2B_ETYPE, at + ": must be F64");
  if (f32_only && r.type != OP2B_F32) return c.fail(OP2B_ETYPE, at + ": must be F32");
  if (!f64_only && !f32_only && r.type != OP2B_F64 && r.type != OP2B_F32)
    return c.fail(OP2B_ETYPE, at + ": must be F64 or F32");
  return OP2B_OK;
}

// shared memory per CTA of the staged passes for a neighbourhood of U nodes
size_t smem_gg(int64_t U) { return (size_t)U * SQ4 * 16; }
size_t smem_flux(int64_t U, int32_t B) { return (size_t)U * SREC4 * 16 + (size_t)B * 12 * 4; }
// the staged passes run only where at least two CTAs fit on an SM
constexpr size_t kStageSmemLimit = 100 * 1024;
constexpr int kStageBlocks[3] = {128, 64, 32};

// The sliced-ELL offsets of the direct passes from the map's node degrees:
// slice s (nodes 32 s .. 32 s + 31) holds width_s = its largest degree
// rows of 32 slots.
void ell_offsets(const MapRec& m, int64_t N, int64_t E, std::vector<int64_t>* off) {
  std::vector<int32_t> deg((size_t)N, 0);
  for (int64_t e = 0; e < E; e++) {
    deg[m.host[2 * e]]++;
    deg[m.host[2 * e + 1]]++;
  }
  const int64_t S = (N + 31) / 32;
  off->assign((size_t)S + 1, 0);
  for (int64_t sl = 0; sl < S; sl++) {
    int32_t w = 0;
    for (int64_t i = 32 * sl; i < std::min<int64_t>(N, 32 * sl + 32); i++) w = std::max(w, deg[i]);
    (*off)[sl + 1] = (*off)[sl] + 32 * (int64_t)w;
  }
}

// The node-block staging plan, on the host from the map in its current
// numbering: the largest block size whose every neighbourhood fits
// kStageSmemLimit, or none (p.staged stays false).
int build_staging(Ctx& c, const MapRec& m, int64_t N, int64_t E, Stage32Plan& p) {
  p.staged = false;
  if (N == 0 || E == 0) return OP2B_OK;
  std::vector<int32_t> m0((size_t)E), m1((size_t)E);
  for (int64_t e = 0; e < E; e++) {
    m0[e] = m.host[2 * e];
    m1[e] = m.host[2 * e + 1];
  }
  std::vector<int64_t> rowptr;
  std::vector<int32_t> ends;
  node_csr(N, E, m0.data(), m1.data(), &rowptr, &ends);
  NodeBlockPlan bp;
  bool ok = false;
  for (int B : kStageBlocks) {
    build_node_block_plan(N, m0.data(), m1.data(), rowptr, ends, B, &bp);
    if (smem_flux(bp.max_unique, B) <= kStageSmemLimit) {
      ok = true;
      break;
    }
  }
  if (!ok) return OP2B_OK;
  int rc;
  if ((rc = upload(c, &p.uoff, bp.uoff)) || (rc = upload(c, &p.uniq, bp.uniq)) ||
      (rc = upload(c, &p.lother, bp.lother)) || (rc = upload(c, &p.sell_off, bp.sell_off)) ||
      (rc = upload(c, &p.sell_end, bp.sell_end)) ||
      (rc = alloc(c, &p.adjn_s, bp.sell_end.size())) ||
      (rc = alloc(c, &p.adje_s, bp.sell_end.size())) || (rc = alloc(c, &p.geo, (size_t)2 * E)))
    return rc;
  p.staged = true;
  p.B = bp.B;
  p.nblocks = bp.nblocks;
  p.max_unique = bp.max_unique;
  p.nslots = (int64_t)bp.sell_end.size();
  return OP2B_OK;
}

template <typename TN, typename TD>
void launch_adjacency_ell(Ctx& c, const DevSegPlan& sp, int64_t nends, const int32_t* m0,
                          const int32_t* m1, const DatRec& n, const DatRec& dx, Stage32Plan& p) {
  k_s32_adjacency_ell<TN, TD><<<grid_of(c, nends, 256), 256, 0, c.stream>>>(
      sp.ends, nends, sp.rowptr, p.ell_off, m0, m1, (const TN*)n.ptr, n.ld, (const TD*)dx.ptr,
      dx.ld, p.adjn_l, p.ende);
}

// the staged passes' sliced-ELL adjacency (local ids) and edge geometry
template <typename TN, typename TD>
void launch_staged_adjacency(Ctx& c, const DevSegPlan& sp, int64_t E, const DatRec& n,
                             const DatRec& dx, Stage32Plan& p) {
  k_s32_adjacency_sell<TN><<<grid_of(c, p.nslots, 256), 256, 0, c.stream>>>(
      p.sell_end, p.nslots, sp.ends, p.lother, (const TN*)n.ptr, n.ld, p.adjn_s, p.adje_s);
  k_s32_geometry<TN, TD><<<grid_of(c, E, 256), 256, 0, c.stream>>>(
      E, (const TN*)n.ptr, n.ld, (const TD*)dx.ptr, dx.ld, p.geo);
}

}  // namespace

int stage32_free_all(Ctx& c) {
  for (auto& kv : c.s32plans) free_stage32(kv.second);
  c.s32plans.clear();
  return OP2B_OK;
}

}  // namespace op2b

using namespace op2b;

extern "C" int op2b_stage_mixed(op2b_ctx h, op2b_map map, op2b_dat q0, op2b_dat q, op2b_dat V,
                                op2b_dat dt, op2b_dat n, op2b_dat dx, op2b_dat R, op2b_dat G,
                                double alpha, double gamma, double eps_lim, int32_t flags) {
  if (!h) {
    set_thread_error("stage_mixed: null context");
    return OP2B_EINVAL;
  }
  Ctx& c = h->c;
  if (map < 0 || map >= (op2b_map)c.maps.size()) return c.fail(OP2B_EINVAL, "stage_mixed: bad map");
  MapRec& m = c.maps[map];
  if (m.arity != 2) return c.fail(OP2B_EINVAL, "stage_mixed: the map must have arity 2");
  if (flags & ~(OP2B_STAGE_SYNC | OP2B_STAGE_STORE_Q0 | OP2B_STAGE_SYNC_MESH | OP2B_STAGE_STAGED))
    return c.fail(OP2B_EINVAL, "stage_mixed: unknown flag");
  if (!(gamma > 1.0) || !(eps_lim > 0.0) || !(alpha == alpha))
    return c.fail(OP2B_EINVAL, "stage_mixed: need gamma > 1, eps_lim > 0 and a finite alpha");
  const op2b_set nodes = m.to, edges = m.from;
  int rc;
  if ((rc = check_dat(c, q0, 6, nodes, true, false, "q0")) ||
      (rc = check_dat(c, q, 6, nodes, true, false, "q")) ||
      (rc = check_dat(c, V, 1, nodes, true, false, "V")) ||
      (rc = check_dat(c, dt, 1, nodes, true, false, "dt")) ||
      (rc = check_dat(c, n, 3, edges, false, false, "n")) ||
      (rc = check_dat(c, dx, 3, edges, false, false, "dx")) ||
      (R >= 0 && (rc = check_dat(c, R, 6, nodes, true, false, "R"))) ||
      (G >= 0 && (rc = check_dat(c, G, 18, nodes, false, true, "G"))))
    return rc;
  if (q0 == q) return c.fail(OP2B_EINVAL, "stage_mixed: q0 and q must be different dats");
  const int64_t N = c.sets[nodes].size, E = c.sets[edges].size;
  DevSegPlan* sp = nullptr;
  if ((rc = c.seg_plan(map, &sp))) return rc;
  const DatRec &dn = c.dats[n], &ddx = c.dats[dx], &dq = c.dats[q];
  auto it = c.s32plans.find(map);
  if (it != c.s32plans.end() && it->second.map_version != m.version) {
    cudaStreamSynchronize(c.stream);
    free_stage32(it->second);
    c.s32plans.erase(it);
    it = c.s32plans.end();
  }
  bool sync_geo = (flags & OP2B_STAGE_SYNC_MESH) != 0, sync_q = (flags & OP2B_STAGE_SYNC) != 0;
  if (it == c.s32plans.end()) {
    Stage32Plan p;
    p.map_version = m.version;
    p.N = N;
    p.E = E;
    std::vector<int64_t> eoff;
    ell_offsets(m, N, E, &eoff);
    p.nell = eoff.back();
    if ((rc = upload(c, &p.ell_off, eoff)) || (rc = alloc(c, &p.adjn_l, (size_t)p.nell)) ||
        (rc = alloc(c, &p.ende, (size_t)2 * p.nell)) || (rc = alloc(c, &p.rec[0], (size_t)REC * N)) ||
        (rc = alloc(c, &p.rec[1], (size_t)REC * N))) {
      free_stage32(p);
      return rc;
    }
    it = c.s32plans.emplace(map, p).first;
    sync_geo = sync_q = true;
  }
  Stage32Plan& p = it->second;
  if ((flags & OP2B_STAGE_STAGED) && !p.staging_planned) {
    // the node-block staging plan, built on the first request
    if ((rc = build_staging(c, m, N, E, p))) return rc;
    p.staging_planned = true;
    sync_geo = true;  // its adjacency is built with the geometry
  }
  if (p.n_src != dn.ptr || p.n_type != dn.type || p.dx_src != ddx.ptr || p.dx_type != ddx.type)
    sync_geo = true;
  if (p.q_src != dq.ptr) sync_q = true;
  const int32_t* m0 = m.dev;
  const int32_t* m1 = m.dev + E;
  if (sync_geo && E > 0) {
    const bool n64 = dn.type == OP2B_F64, dx64 = ddx.type == OP2B_F64;
    if (n64 && dx64) launch_adjacency_ell<double, double>(c, *sp, 2 * E, m0, m1, dn, ddx, p);
    else if (n64) launch_adjacency_ell<double, float>(c, *sp, 2 * E, m0, m1, dn, ddx, p);
    else if (dx64) launch_adjacency_ell<float, double>(c, *sp, 2 * E, m0, m1, dn, ddx, p);
    else launch_adjacency_ell<float, float>(c, *sp, 2 * E, m0, m1, dn, ddx, p);
    if ((rc = c.launched("stage_mixed adjacency"))) return rc;
    if (p.staged) {
      if (n64 && dx64) launch_staged_adjacency<double, double>(c, *sp, E, dn, ddx, p);
      else if (n64) launch_staged_adjacency<double, float>(c, *sp, E, dn, ddx, p);
      else if (dx64) launch_staged_adjacency<float, double>(c, *sp, E, dn, ddx, p);
      else launch_staged_adjacency<float, float>(c, *sp, E, dn, ddx, p);
      if ((rc = c.launched("stage_mixed staged adjacency"))) return rc;
    }
  }
  p.n_src = dn.ptr;
  p.n_type = dn.type;
  p.dx_src = ddx.ptr;
  p.dx_type = ddx.type;
  if (N == 0) return OP2B_OK;
  float* rin = p.rec[p.cur];
  float* rout = p.rec[p.cur ^ 1];
  if (sync_q) {
    k_s32_pack_q<<<grid_of(c, N, 256), 256, 0, c.stream>>>(N, (const double*)dq.ptr, dq.ld, rin);
    if ((rc = c.launched("stage_mixed pack"))) return rc;
  }
  p.q_src = dq.ptr;
  const bool staged = p.staged && (flags & OP2B_STAGE_STAGED);
  const DatRec* dG = G >= 0 ? &c.dats[G] : nullptr;
  float* pG = dG ? (float*)dG->ptr : nullptr;
  const int64_t ldG = dG ? dG->ld : 0;
  const double* pV = (const double*)c.dats[V].ptr;
  const double* pdt = (const double*)c.dats[dt].ptr;
  const DatRec* dR = R >= 0 ? &c.dats[R] : nullptr;
  double* pR = dR ? (double*)dR->ptr : nullptr;
  const int64_t ldR = dR ? dR->ld : 0;
  const DatRec& d0 = c.dats[q0];
  const bool sq0 = (flags & OP2B_STAGE_STORE_Q0) != 0;
  GasPairs gas{splat2((float)(gamma - 1.0)), splat2((float)gamma), splat2((float)eps_lim),
               splat2((float)(2.0 * eps_lim))};
  if (staged) {
    const size_t s1 = smem_gg(p.max_unique), s2 = smem_flux(p.max_unique, p.B);
    if (cudaFuncSetAttribute(k_s32_green_gauss_sell, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)s1) != cudaSuccess ||
        cudaFuncSetAttribute(k_s32_flux_update_sell, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)s2) != cudaSuccess)
      return c.fail(OP2B_ECUDA, "stage_mixed: cudaFuncSetAttribute failed");
    k_s32_green_gauss_sell<<<(unsigned)p.nblocks, p.B, s1, c.stream>>>(
        N, p.B, p.uoff, p.uniq, p.sell_off, p.adjn_s, rin, pV, pG, ldG);
    if ((rc = c.launched("stage_mixed green_gauss"))) return rc;
    k_s32_flux_update_sell<<<(unsigned)p.nblocks, 2 * p.B, s2, c.stream>>>(
        N, p.B, p.uoff, p.uniq, p.sell_off, p.adje_s, (const float*)p.geo, rin, rout,
        (double*)d0.ptr, d0.ld, (double*)dq.ptr, dq.ld, pV, pdt, alpha, pR, ldR, sq0, gas);
  } else {
    // one node per thread, every block launched: the blocks are dispatched in
    // node order, so the nodes in flight form one moving window of the mesh
    // whose neighbours stay in L2 (a grid capped at 64 blocks per SM, each
    // block striding over the whole mesh, measured 6.7% slower per stage at
    // 200^3)
    k_s32_green_gauss<<<grid_all(N, 128), 128, 0, c.stream>>>(N, sp->rowptr, p.ell_off,
                                                                 p.adjn_l, rin, pV, pG, ldG);
    if ((rc = c.launched("stage_mixed green_gauss"))) return rc;
    k_s32_flux_update<<<grid_all(N, kFluxBlock), kFluxBlock, 0, c.stream>>>(
        N, sp->rowptr, p.ell_off, (const float*)p.ende, rin, rout, (double*)d0.ptr, d0.ld,
        (double*)dq.ptr, dq.ld, pV, pdt, alpha, pR, ldR, sq0, gas);
  }
  if ((rc = c.launched("stage_mixed flux_update"))) return rc;
  p.cur ^= 1;
  return OP2B_OK;
}
