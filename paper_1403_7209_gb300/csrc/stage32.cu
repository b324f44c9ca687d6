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
// packed record (q then G, 96 bytes: three sectors, six 16-byte loads) cuts
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
//   pass 1 (Green-Gauss, 2 threads per node): G_i = (1/V_i) sum over the
//     node's edge ends of (q_i + q_j) (x) (+-n/2), written into the record's
//     G part (and into an optional FP32 G dat);
//   pass 2 (flux + update, 1 thread per node): for every edge end the edge's
//     flux in its own orientation (first end, second end: the two ends of an
//     edge compute bitwise the same value, so the residual stays exactly
//     antisymmetric), summed with sign; then R_i in FP64 and
//     q_i = q0_i - alpha (dt_i / V_i) R_i, written to q (FP64), to the other
//     record buffer's q part (FP32) and optionally to R and q0.
#include <algorithm>
#include <string>

#include "edge_math.cuh"
#include "internal.h"

namespace op2b {

namespace {

constexpr int REC = 24;  // floats per node record: q (6) then G (18)

// Knuth's two-sum: hi + lo += x with the rounding error of the addition
// kept in lo (exact: s + err == hi + x)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += err;
}

template <typename T>
__device__ __forceinline__ float f32_of(T x) {
  return (float)x;
}

// per edge end t (the segmented plan's node-sorted ends, value 2e + side):
// adjn[t] = {other end j, +-n_e/2 (FP32 bits)} for the Green-Gauss pass,
// adje[t] = {j, 2e + side} for the flux pass
template <typename TN>
__global__ void k_s32_adjacency(const int32_t* __restrict__ ends, int64_t nends,
                                const int32_t* __restrict__ m0, const int32_t* __restrict__ m1,
                                const TN* __restrict__ n, int64_t ldn, int4* __restrict__ adjn,
                                int2* __restrict__ adje) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nends;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t end = ends[t];
    const int64_t e = end >> 1;
    const bool second = end & 1;
    const int32_t j = second ? m0[e] : m1[e];
    const float h = second ? -0.5f : 0.5f;
    const float hx = f32_of(n[e]) * h, hy = f32_of(n[ldn + e]) * h, hz = f32_of(n[2 * ldn + e]) * h;
    adjn[t] = make_int4(j, __float_as_int(hx), __float_as_int(hy), __float_as_int(hz));
    adje[t] = make_int2(j, end);
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

// record q part <- (float) q
__global__ void k_s32_pack_q(int64_t N, const double* __restrict__ q, int64_t ldq,
                             float* __restrict__ rec) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 6; k++) rec[i * REC + k] = (float)q[k * ldq + i];
  }
}

// Pass 1: Green-Gauss with the scaling, two threads per node (components
// 0-2 and 3-5 of q, so G entries 0-8 and 9-17).  Same operations in the
// same order as the FP32 Green-Gauss node gather, so the same bits.
__global__ void __launch_bounds__(128) k_s32_green_gauss(
    int64_t N, const int64_t* __restrict__ rowptr, const int4* __restrict__ adjn,
    float* __restrict__ rec, const double* __restrict__ V, float* __restrict__ Gout,
    int64_t ldG) {
  for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t0 < 2 * N;
       t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t0 >> 1;
    const int h = (int)(t0 & 1);
    const int k0 = 3 * h;
    const float* qi = rec + i * REC + k0;
    const float qi0 = __ldg(qi), qi1 = __ldg(qi + 1), qi2 = __ldg(qi + 2);
    float acc[9];
#pragma unroll
    for (int c = 0; c < 9; c++) acc[c] = 0.0f;
    const int64_t t1 = rowptr[i + 1];
#pragma unroll 4
    for (int64_t t = rowptr[i]; t < t1; t++) {
      const int4 a = __ldg(adjn + t);
      const float* qj = rec + (int64_t)a.x * REC + k0;
      const float hx = __int_as_float(a.y), hy = __int_as_float(a.z), hz = __int_as_float(a.w);
      const float s0 = qi0 + __ldg(qj), s1 = qi1 + __ldg(qj + 1), s2 = qi2 + __ldg(qj + 2);
      acc[0] = fmaf(s0, hx, acc[0]);
      acc[1] = fmaf(s0, hy, acc[1]);
      acc[2] = fmaf(s0, hz, acc[2]);
      acc[3] = fmaf(s1, hx, acc[3]);
      acc[4] = fmaf(s1, hy, acc[4]);
      acc[5] = fmaf(s1, hz, acc[5]);
      acc[6] = fmaf(s2, hx, acc[6]);
      acc[7] = fmaf(s2, hy, acc[7]);
      acc[8] = fmaf(s2, hz, acc[8]);
    }
    const float r = (float)(1.0 / V[i]);
    float* g = rec + i * REC + 6 + 9 * h;
#pragma unroll
    for (int c = 0; c < 9; c++) {
      const float v = acc[c] * r;
      g[c] = v;
      if (Gout) Gout[(9 * h + c) * ldG + i] = v;
    }
  }
}

__device__ __forceinline__ void load_rec(const float* __restrict__ p, float* v) {
  const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < REC / 4; k++) {
    const float4 x = __ldg(p4 + k);
    v[4 * k] = x.x;
    v[4 * k + 1] = x.y;
    v[4 * k + 2] = x.z;
    v[4 * k + 3] = x.w;
  }
}

// Pass 2: the flux of every edge end in the edge's own orientation (the
// FP32 reconstruction and Rusanov flux of the mixed flux loop), summed per
// node with two-sum pairs, then the FP64 residual and the node update.
__global__ void __launch_bounds__(128) k_s32_flux_update(
    int64_t N, const int64_t* __restrict__ rowptr, const int2* __restrict__ adje,
    const float4* __restrict__ geo, const float* __restrict__ rin, float* __restrict__ rout,
    double* __restrict__ q0, int64_t ld0, double* __restrict__ q, int64_t ldq,
    const double* __restrict__ V, const double* __restrict__ dt, double alpha,
    double* __restrict__ R, int64_t ldR, bool store_q0, Gas<float> gas) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float hi[6], lo[6];
#pragma unroll
    for (int k = 0; k < 6; k++) hi[k] = lo[k] = 0.0f;
    const int64_t t1 = rowptr[i + 1];
    for (int64_t t = rowptr[i]; t < t1; t++) {
      const int2 a = __ldg(adje + t);
      const int64_t e = a.y >> 1;
      const bool second = a.y & 1;
      const int64_t first_node = second ? (int64_t)a.x : i;
      const int64_t second_node = second ? i : (int64_t)a.x;
      float va[REC], vb[REC];
      load_rec(rin + first_node * REC, va);
      load_rec(rin + second_node * REC, vb);
      const float4 g0 = __ldg(geo + 2 * e), g1 = __ldg(geo + 2 * e + 1);
      float qL[6], qR[6], F[6];
      reconstruct(va, vb, g0.w, g1.x, g1.y, gas, qL, qR);
      rusanov(qL, qR, g0.x, g0.y, g0.z, gas, F);
#pragma unroll
      for (int k = 0; k < 6; k++) two_sum_acc(hi[k], lo[k], second ? neg(F[k]) : F[k]);
    }
    const double a = alpha * (dt[i] / V[i]);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const double Rk = to_acc<double>(hi[k]) + to_acc<double>(lo[k]);
      const double v = q0[k * ld0 + i] - a * Rk;
      q[k * ldq + i] = v;
      rout[i * REC + k] = (float)v;
      if (R) R[k * ldR + i] = Rk;
      if (store_q0) q0[k * ld0 + i] = v;
    }
  }
}

unsigned grid_of(const Ctx& c, int64_t work, int block) {
  const int64_t g = (work + block - 1) / block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)c.sm_count * 64));
}

void free_stage32(Stage32Plan& p) {
  cudaFree(p.adjn);
  cudaFree(p.adje);
  cudaFree(p.geo);
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

template <typename TN>
void launch_adjacency(Ctx& c, const DevSegPlan& sp, int64_t nends, const int32_t* m0,
                      const int32_t* m1, const DatRec& n, Stage32Plan& p) {
  k_s32_adjacency<TN><<<grid_of(c, nends, 256), 256, 0, c.stream>>>(
      sp.ends, nends, m0, m1, (const TN*)n.ptr, n.ld, p.adjn, p.adje);
}

template <typename TN, typename TD>
void launch_geometry(Ctx& c, int64_t E, const DatRec& n, const DatRec& dx, Stage32Plan& p) {
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
  if (flags & ~(OP2B_STAGE_SYNC | OP2B_STAGE_STORE_Q0))
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
  bool sync_geo = (flags & OP2B_STAGE_SYNC) != 0, sync_q = sync_geo;
  if (it == c.s32plans.end()) {
    Stage32Plan p;
    p.map_version = m.version;
    p.N = N;
    p.E = E;
    if ((rc = alloc(c, &p.adjn, (size_t)2 * E)) || (rc = alloc(c, &p.adje, (size_t)2 * E)) ||
        (rc = alloc(c, &p.geo, (size_t)2 * E)) || (rc = alloc(c, &p.rec[0], (size_t)REC * N)) ||
        (rc = alloc(c, &p.rec[1], (size_t)REC * N))) {
      free_stage32(p);
      return rc;
    }
    it = c.s32plans.emplace(map, p).first;
    sync_geo = sync_q = true;
  }
  Stage32Plan& p = it->second;
  if (p.n_src != dn.ptr || p.n_type != dn.type || p.dx_src != ddx.ptr || p.dx_type != ddx.type)
    sync_geo = true;
  if (p.q_src != dq.ptr) sync_q = true;
  const int32_t* m0 = m.dev;
  const int32_t* m1 = m.dev + E;
  if (sync_geo && E > 0) {
    if (dn.type == OP2B_F64) launch_adjacency<double>(c, *sp, 2 * E, m0, m1, dn, p);
    else launch_adjacency<float>(c, *sp, 2 * E, m0, m1, dn, p);
    if ((rc = c.launched("stage_mixed adjacency"))) return rc;
    if (dn.type == OP2B_F64 && ddx.type == OP2B_F64) launch_geometry<double, double>(c, E, dn, ddx, p);
    else if (dn.type == OP2B_F64) launch_geometry<double, float>(c, E, dn, ddx, p);
    else if (ddx.type == OP2B_F64) launch_geometry<float, double>(c, E, dn, ddx, p);
    else launch_geometry<float, float>(c, E, dn, ddx, p);
    if ((rc = c.launched("stage_mixed geometry"))) return rc;
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
  const DatRec* dG = G >= 0 ? &c.dats[G] : nullptr;
  k_s32_green_gauss<<<grid_of(c, 2 * N, 128), 128, 0, c.stream>>>(
      N, sp->rowptr, p.adjn, rin, (const double*)c.dats[V].ptr, dG ? (float*)dG->ptr : nullptr,
      dG ? dG->ld : 0);
  if ((rc = c.launched("stage_mixed green_gauss"))) return rc;
  Gas<float> gas{(float)gamma, (float)(gamma - 1.0), (float)eps_lim, (float)(2.0 * eps_lim)};
  const DatRec* dR = R >= 0 ? &c.dats[R] : nullptr;
  const DatRec& d0 = c.dats[q0];
  k_s32_flux_update<<<grid_of(c, N, 128), 128, 0, c.stream>>>(
      N, sp->rowptr, p.adje, p.geo, rin, rout, (double*)d0.ptr, d0.ld, (double*)dq.ptr, dq.ld,
      (const double*)c.dats[V].ptr, (const double*)c.dats[dt].ptr, alpha,
      dR ? (double*)dR->ptr : nullptr, dR ? dR->ld : 0, (flags & OP2B_STAGE_STORE_Q0) != 0, gas);
  if ((rc = c.launched("stage_mixed flux_update"))) return rc;
  p.cur ^= 1;
  return OP2B_OK;
}
