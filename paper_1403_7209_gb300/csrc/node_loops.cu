// Direct node loops (no map): gradient scaling, local time step, the
// Runge-Kutta stage update, fills, copies and the gathers that apply a
// renumbering to a dat.  Grid-stride loops over nodes; every component
// array is read and written with unit stride.
#include <algorithm>

#include "ff_math.cuh"
#include "internal.h"

namespace op2b {

static unsigned grid_for(Ctx* c, int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)c->sm_count * 32));
}

// G <- G * (1/V): one division per node, 18 multiplies
template <typename T>
__global__ void k_grad_scale(T* __restrict__ G, int64_t ld,
                             const double* __restrict__ V, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    T r = (T)(1.0 / V[i]);
#pragma unroll
    for (int c = 0; c < 18; c++) G[c * ld + i] *= r;
  }
}

// float-float G <- G * (1/V): the reciprocal of V in float-float, 18
// float-float multiplies
__global__ void k_grad_scale_ff(float2* __restrict__ G, int64_t ld, const double* __restrict__ V,
                                int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 r = ff_recip(ff_of_f64(V[i]));
#pragma unroll
    for (int c = 0; c < 18; c++) G[c * ld + i] = ff_mul(G[c * ld + i], r);
  }
}

int node_grad_scale(Ctx* c, void* G, int type, int64_t ldG, const double* V,
                    int64_t N) {
  if (N == 0) return OP2B_OK;
  if (type == OP2B_F64)
    k_grad_scale<double><<<grid_for(c, N, 256), 256, 0, c->stream>>>((double*)G, ldG, V, N);
  else if (type == OP2B_FF)
    k_grad_scale_ff<<<grid_for(c, N, 256), 256, 0, c->stream>>>((float2*)G, ldG, V, N);
  else
    k_grad_scale<float><<<grid_for(c, N, 256), 256, 0, c->stream>>>((float*)G, ldG, V, N);
  return c->launched("grad_scale");
}

__global__ void k_time_step(const double* __restrict__ V,
                            const double* __restrict__ lam, double cfl,
                            double* __restrict__ dt, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    dt[i] = cfl * V[i] / lam[i];
}

int node_time_step(Ctx* c, const double* V, const double* lam, double cfl,
                   double* dt, int64_t N) {
  if (N == 0) return OP2B_OK;
  k_time_step<<<grid_for(c, N, 256), 256, 0, c->stream>>>(V, lam, cfl, dt, N);
  return c->launched("time_step");
}

// q = q0 - alpha (dt/V) R, with the shadow of q (FP32 or float-float) when
// sh != null
template <typename TS>
__global__ void k_update(const double* __restrict__ q0, int64_t ld0,
                         double* __restrict__ q, int64_t ldq,
                         const double* __restrict__ R, int64_t ldR,
                         const double* __restrict__ V,
                         const double* __restrict__ dt, double alpha,
                         TS* __restrict__ sh, int64_t ldsh, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double a = alpha * (dt[i] / V[i]);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      double v = q0[k * ld0 + i] - a * R[k * ldR + i];
      q[k * ldq + i] = v;
      if (sh) {
        if constexpr (sizeof(TS) == 4) sh[k * ldsh + i] = (float)v;
        else sh[k * ldsh + i] = ff_of_f64(v);
      }
    }
  }
}

int node_update(Ctx* c, const double* q0, int64_t ld0, double* q, int64_t ldq,
                const double* R, int64_t ldR, const double* V,
                const double* dt, double alpha, void* shadow, int shadow_type,
                int64_t ldsh, int64_t N) {
  if (N == 0) return OP2B_OK;
  const unsigned g = grid_for(c, N, 256);
  if (shadow && shadow_type == OP2B_FF)
    k_update<float2><<<g, 256, 0, c->stream>>>(q0, ld0, q, ldq, R, ldR, V, dt, alpha,
                                               (float2*)shadow, ldsh, N);
  else
    k_update<float><<<g, 256, 0, c->stream>>>(q0, ld0, q, ldq, R, ldR, V, dt, alpha,
                                              (float*)shadow, ldsh, N);
  return c->launched("update");
}

// transpose of the stage update with respect to q0 and R:
// qbar += sbar,  lam = -alpha (dt/V) sbar
__global__ void k_update_adjoint(const double* __restrict__ sb, int64_t ldsb,
                                 double* __restrict__ qb, int64_t ldqb,
                                 double* __restrict__ lam, int64_t ldl,
                                 const double* __restrict__ V,
                                 const double* __restrict__ dt, double alpha, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = -alpha * (dt[i] / V[i]);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const double v = sb[k * ldsb + i];
      qb[k * ldqb + i] += v;
      lam[k * ldl + i] = a * v;
    }
  }
}

int node_update_adjoint(Ctx* c, const double* sb, int64_t ldsb, double* qb, int64_t ldqb,
                        double* lam, int64_t ldl, const double* V, const double* dt,
                        double alpha, int64_t N) {
  if (N == 0) return OP2B_OK;
  k_update_adjoint<<<grid_for(c, N, 256), 256, 0, c->stream>>>(sb, ldsb, qb, ldqb, lam, ldl, V,
                                                               dt, alpha, N);
  return c->launched("update_adjoint");
}

// y += a x, component-wise
__global__ void k_axpy(double* __restrict__ y, int64_t ldy, double a,
                       const double* __restrict__ x, int64_t ldx, int dim, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < dim; k++) y[k * ldy + i] = fma(a, x[k * ldx + i], y[k * ldy + i]);
}

int node_axpy(Ctx* c, double* y, int64_t ldy, double a, const double* x, int64_t ldx, int dim,
              int64_t n) {
  if (n == 0 || dim == 0) return OP2B_OK;
  k_axpy<<<grid_for(c, n, 256), 256, 0, c->stream>>>(y, ldy, a, x, ldx, dim, n);
  return c->launched("axpy");
}

template <typename T>
__global__ void k_fill(T* __restrict__ p, int64_t ld, int dim, int64_t n,
                       T v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < dim; k++) p[k * ld + i] = v;
}

int node_fill(Ctx* c, void* p, int type, int64_t ld, int dim, int64_t n,
              double value) {
  if (n == 0 || dim == 0) return OP2B_OK;
  unsigned g = grid_for(c, n, 256);
  if (type == OP2B_F64)
    k_fill<double><<<g, 256, 0, c->stream>>>((double*)p, ld, dim, n, value);
  else if (type == OP2B_F32)
    k_fill<float><<<g, 256, 0, c->stream>>>((float*)p, ld, dim, n, (float)value);
  else if (type == OP2B_FF)
    k_fill<float2><<<g, 256, 0, c->stream>>>((float2*)p, ld, dim, n, ff_split_host(value));
  else
    k_fill<int32_t><<<g, 256, 0, c->stream>>>((int32_t*)p, ld, dim, n, (int32_t)value);
  return c->launched("fill");
}

template <typename TD, typename TS>
__global__ void k_copy(TD* __restrict__ d, int64_t ldd,
                       const TS* __restrict__ s, int64_t lds, int dim,
                       int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < dim; k++) d[k * ldd + i] = (TD)s[k * lds + i];
}

// double -> float-float and back (ff_of_f64 / f64_of_ff)
__global__ void k_copy_ff(float2* __restrict__ d, int64_t ldd, const double* __restrict__ s,
                          int64_t lds, int dim, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < dim; k++) d[k * ldd + i] = ff_of_f64(s[k * lds + i]);
}
__global__ void k_copy_from_ff(double* __restrict__ d, int64_t ldd, const float2* __restrict__ s,
                               int64_t lds, int dim, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < dim; k++) d[k * ldd + i] = f64_of_ff(s[k * lds + i]);
}

int node_copy(Ctx* c, void* dst, int dtype, int64_t ldd, const void* src,
              int stype, int64_t lds, int dim, int64_t n) {
  if (n == 0 || dim == 0) return OP2B_OK;
  unsigned g = grid_for(c, n, 256);
  if (dtype == OP2B_F64 && stype == OP2B_F64)
    k_copy<double, double><<<g, 256, 0, c->stream>>>((double*)dst, ldd, (const double*)src, lds, dim, n);
  else if (dtype == OP2B_F32 && stype == OP2B_F64)
    k_copy<float, double><<<g, 256, 0, c->stream>>>((float*)dst, ldd, (const double*)src, lds, dim, n);
  else if (dtype == OP2B_F64 && stype == OP2B_F32)
    k_copy<double, float><<<g, 256, 0, c->stream>>>((double*)dst, ldd, (const float*)src, lds, dim, n);
  else if (dtype == OP2B_F32 && stype == OP2B_F32)
    k_copy<float, float><<<g, 256, 0, c->stream>>>((float*)dst, ldd, (const float*)src, lds, dim, n);
  else if (dtype == OP2B_FF && stype == OP2B_F64)
    k_copy_ff<<<g, 256, 0, c->stream>>>((float2*)dst, ldd, (const double*)src, lds, dim, n);
  else if (dtype == OP2B_F64 && stype == OP2B_FF)
    k_copy_from_ff<<<g, 256, 0, c->stream>>>((double*)dst, ldd, (const float2*)src, lds, dim, n);
  else if (dtype == OP2B_FF && stype == OP2B_FF)
    k_copy<double, double><<<g, 256, 0, c->stream>>>((double*)dst, ldd, (const double*)src, lds, dim, n);
  else if (dtype == OP2B_I32 && stype == OP2B_I32)
    k_copy<int32_t, int32_t><<<g, 256, 0, c->stream>>>((int32_t*)dst, ldd, (const int32_t*)src, lds, dim, n);
  else
    return c->fail(OP2B_ETYPE, "dat_copy: unsupported type pair");
  return c->launched("copy");
}

template <typename T>
__global__ void k_gather(T* __restrict__ out, const T* __restrict__ in,
                         int64_t ld, int dim, const int64_t* __restrict__ idx,
                         int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t s = idx[t];
    for (int k = 0; k < dim; k++) out[k * ld + t] = in[k * ld + s];
  }
}

int node_gather(Ctx* c, void* out, const void* in, int esize, int64_t ld,
                int dim, const int64_t* idx, int64_t n) {
  if (n == 0 || dim == 0) return OP2B_OK;
  unsigned g = grid_for(c, n, 256);
  if (esize == 8)
    k_gather<uint64_t><<<g, 256, 0, c->stream>>>((uint64_t*)out, (const uint64_t*)in, ld, dim, idx, n);
  else if (esize == 4)
    k_gather<uint32_t><<<g, 256, 0, c->stream>>>((uint32_t*)out, (const uint32_t*)in, ld, dim, idx, n);
  else
    return c->fail(OP2B_EINVAL, "gather: element size must be 4 or 8");
  return c->launched("gather");
}

// ------------------------------------------------------ global reductions
// Two passes in a fixed order (per-block partials over contiguous chunks,
// then one block over the partials), so the result does not depend on
// scheduling: bitwise reproducible.

template <int OP>
__device__ __forceinline__ double red_init() {
  return OP == OP2B_RED_MIN ? INFINITY : 0.0;
}
template <int OP>
__device__ __forceinline__ double red_take(double acc, double v) {  // one value
  if constexpr (OP == OP2B_RED_SUM) return acc + v;
  else if constexpr (OP == OP2B_RED_L2) return fma(v, v, acc);
  else if constexpr (OP == OP2B_RED_MAXABS) return fmax(acc, fabs(v));
  else return fmin(acc, v);
}
template <int OP>
__device__ __forceinline__ double red_merge(double a, double b) {  // two partials
  if constexpr (OP == OP2B_RED_SUM || OP == OP2B_RED_L2) return a + b;
  else if constexpr (OP == OP2B_RED_MAXABS) return fmax(a, b);
  else return fmin(a, b);
}

template <int OP, int T>
__device__ __forceinline__ double block_tree(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int w = T / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = red_merge<OP>(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

template <int OP, int T>
__global__ void k_reduce_partial(const double* __restrict__ x, int64_t ld, int dim, int64_t n,
                                 int64_t chunk, double* __restrict__ part) {
  __shared__ double sh[T];
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = min(n, lo + chunk);
  for (int k = 0; k < dim; k++) {
    double acc = red_init<OP>();
    for (int64_t i = lo + threadIdx.x; i < hi; i += T) acc = red_take<OP>(acc, x[k * ld + i]);
    double r = block_tree<OP, T>(acc, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * dim + k] = r;
  }
}

template <int OP, int T>
__global__ void k_reduce_final(const double* __restrict__ part, int nb, int dim,
                               double* __restrict__ out) {
  __shared__ double sh[T];
  for (int k = 0; k < dim; k++) {
    double acc = red_init<OP>();
    for (int b = threadIdx.x; b < nb; b += T) acc = red_merge<OP>(acc, part[(int64_t)b * dim + k]);
    double r = block_tree<OP, T>(acc, sh);
    if (threadIdx.x == 0) out[k] = (OP == OP2B_RED_L2) ? sqrt(r) : r;
  }
}

template <int OP>
static int reduce_op(Ctx* c, const double* x, int64_t ld, int dim, int64_t n, double* out) {
  constexpr int T = 256;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (n + 2047) / 2048));
  const int64_t chunk = (n + nb - 1) / nb;
  void* part = nullptr;
  int rc = c->need_scratch((size_t)nb * dim * sizeof(double), &part);
  if (rc) return rc;
  k_reduce_partial<OP, T><<<nb, T, 0, c->stream>>>(x, ld, dim, n, std::max<int64_t>(chunk, 1),
                                                    (double*)part);
  if ((rc = c->launched("reduce partial"))) return rc;
  k_reduce_final<OP, T><<<1, T, 0, c->stream>>>((const double*)part, nb, dim, out);
  return c->launched("reduce final");
}

// Block-Jacobi inverse: p = m^{-1} (6 x 6, row-major) by Gauss-Jordan
// elimination with partial pivoting (the largest |pivot| of the column, the
// first on ties), in place: the pivot column is replaced by the inverse's
// column as it is eliminated (6 x 6 storage and 216 multiply-adds, half of
// the eliminations on [m | I]), the row exchanges are undone on the columns
// at the end.  Every index is a compile-time constant (exchanges are done
// with selects), so the values stay in registers.
__device__ __forceinline__ void gj_invert6(const double* m, double* p) {
  double a[6][6];
#pragma unroll
  for (int r = 0; r < 6; r++)
#pragma unroll
    for (int c = 0; c < 6; c++) a[r][c] = m[6 * r + c];
  int pv[6];
#pragma unroll
  for (int k = 0; k < 6; k++) {
    int piv = k;
    double best = fabs(a[k][k]);
#pragma unroll
    for (int r = k + 1; r < 6; r++) {
      const double v = fabs(a[r][k]);
      piv = v > best ? r : piv;
      best = v > best ? v : best;
    }
    pv[k] = piv;
#pragma unroll
    for (int r = k + 1; r < 6; r++) {
      const bool sw = piv == r;
#pragma unroll
      for (int c = 0; c < 6; c++) {
        const double t = a[k][c];
        a[k][c] = sw ? a[r][c] : t;
        a[r][c] = sw ? t : a[r][c];
      }
    }
    const double inv = 1.0 / a[k][k];
    a[k][k] = 1.0;
#pragma unroll
    for (int c = 0; c < 6; c++) a[k][c] *= inv;
#pragma unroll
    for (int r = 0; r < 6; r++) {
      if (r == k) continue;
      const double f = a[r][k];
      a[r][k] = 0.0;
#pragma unroll
      for (int c = 0; c < 6; c++) a[r][c] = fma(-f, a[k][c], a[r][c]);
    }
  }
  // undo the row exchanges on the columns, the last one first
#pragma unroll
  for (int kk = 0; kk < 6; kk++) {
    const int k = 5 - kk;
#pragma unroll
    for (int c2 = 0; c2 < 6; c2++) {  // constant bounds keep a[][] in registers
      const bool sw = c2 > k && pv[k] == c2;
#pragma unroll
      for (int r = 0; r < 6; r++) {
        const double t = a[r][k];
        a[r][k] = sw ? a[r][c2] : t;
        a[r][c2] = sw ? t : a[r][c2];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 6; r++)
#pragma unroll
    for (int c = 0; c < 6; c++) p[6 * r + c] = a[r][c];
}

__global__ void k_block_invert(const double* __restrict__ M, int64_t ldM, double* __restrict__ P,
                               int64_t ldP, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double m[36], p[36];
#pragma unroll
    for (int c = 0; c < 36; c++) m[c] = M[c * ldM + i];
    gj_invert6(m, p);
#pragma unroll
    for (int c = 0; c < 36; c++) P[c * ldP + i] = p[c];
  }
}

// Factored blocks: M_i = (Lambda_i I + A(q_i, S_i)) / 2 from the node's
// sums S = (Lambda, S_x, S_y, S_z); writes M and/or P = M^{-1} (null skips).
__global__ void k_jacobi_from_sums(const double* __restrict__ q, int64_t ldq,
                                   const double* __restrict__ S, int64_t ldS,
                                   double* __restrict__ M, int64_t ldM, double* __restrict__ P,
                                   int64_t ldP, Gas<double> g, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double qi[6], m[36];
#pragma unroll
    for (int k = 0; k < 6; k++) qi[k] = q[k * ldq + i];
    const double sv[3] = {S[ldS + i], S[2 * ldS + i], S[3 * ldS + i]};
    flux_jacobian_f64(qi, sv, g, 0.5, m);
    const double hl = 0.5 * S[i];
#pragma unroll
    for (int r = 0; r < 6; r++) m[7 * r] += hl;
    if (M) {
#pragma unroll
      for (int c = 0; c < 36; c++) M[c * ldM + i] = m[c];
    }
    if (P) {
      double p[36];
      gj_invert6(m, p);
#pragma unroll
      for (int c = 0; c < 36; c++) P[c * ldP + i] = p[c];
    }
  }
}

int node_jacobi_from_sums(Ctx* c, const double* q, int64_t ldq, const double* S, int64_t ldS,
                          double* M, int64_t ldM, double* P, int64_t ldP, double gamma,
                          int64_t N) {
  if (N == 0) return OP2B_OK;
  Gas<double> g{gamma, gamma - 1.0, 0.0, 0.0};
  k_jacobi_from_sums<<<grid_for(c, N, 128), 128, 0, c->stream>>>(q, ldq, S, ldS, M, ldM, P, ldP,
                                                                 g, N);
  return c->launched("jacobi_from_sums");
}

int node_block_invert(Ctx* c, const double* M, int64_t ldM, double* P, int64_t ldP, int64_t N) {
  if (N == 0) return OP2B_OK;
  k_block_invert<<<grid_for(c, N, 128), 128, 0, c->stream>>>(M, ldM, P, ldP, N);
  return c->launched("block_invert");
}

// Preconditioned stage: q = q0 - alpha_sigma P R per node.
__global__ void k_update_precond(const double* __restrict__ q0, int64_t ld0,
                                 double* __restrict__ q, int64_t ldq,
                                 const double* __restrict__ R, int64_t ldR,
                                 const double* __restrict__ P, int64_t ldP, double as,
                                 int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double r[6], out[6];
#pragma unroll
    for (int k = 0; k < 6; k++) r[k] = R[k * ldR + i];
#pragma unroll
    for (int row = 0; row < 6; row++) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < 6; k++) acc = fma(P[(6 * row + k) * ldP + i], r[k], acc);
      out[row] = fma(-as, acc, q0[row * ld0 + i]);
    }
#pragma unroll
    for (int row = 0; row < 6; row++) q[row * ldq + i] = out[row];
  }
}

int node_update_precond(Ctx* c, const double* q0, int64_t ld0, double* q, int64_t ldq,
                        const double* R, int64_t ldR, const double* P, int64_t ldP, double as,
                        int64_t N) {
  if (N == 0) return OP2B_OK;
  k_update_precond<<<grid_for(c, N, 256), 256, 0, c->stream>>>(q0, ld0, q, ldq, R, ldR, P, ldP,
                                                               as, N);
  return c->launched("update_precond");
}

// Per-node wave primitives for the wave-speed loops: u = m/rho and the
// sound speed a = sqrt(gamma p / rho), so that an edge needs only
// |u.n| + a|n| of each end (FP32-seeded Newton reciprocal and square root
// where the arguments allow).
__global__ void k_wave_prims(const double* __restrict__ q, int64_t ldq, double* __restrict__ W,
                             double gamma, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v[6];
#pragma unroll
    for (int k = 0; k < 6; k++) v[k] = q[k * ldq + i];
    const double rr = seedable(v[0]) ? recip2(v[0]) : 1.0 / v[0];
    const double u0 = v[1] * rr, u1 = v[2] * rr, u2 = v[3] * rr;
    const double mm = fma(v[3], v[3], fma(v[2], v[2], v[1] * v[1]));
    const double p = (gamma - 1.0) * fma(-0.5 * mm, rr, v[4]);
    const double a2 = gamma * p * rr;
    W[i] = u0;
    W[N + i] = u1;
    W[2 * N + i] = u2;
    W[3 * N + i] = seedable(a2) ? sqrt2(a2) : sqrt(a2);
  }
}

int node_wave_prims(Ctx* c, const double* q, int64_t ldq, double* W, double gamma, int64_t N) {
  if (N == 0) return OP2B_OK;
  k_wave_prims<<<grid_for(c, N, 256), 256, 0, c->stream>>>(q, ldq, W, gamma, N);
  return c->launched("wave_prims");
}

int node_reduce(Ctx* c, const double* x, int64_t ld, int dim, int64_t n, int op, double* out) {
  switch (op) {
    case OP2B_RED_SUM: return reduce_op<OP2B_RED_SUM>(c, x, ld, dim, n, out);
    case OP2B_RED_L2: return reduce_op<OP2B_RED_L2>(c, x, ld, dim, n, out);
    case OP2B_RED_MAXABS: return reduce_op<OP2B_RED_MAXABS>(c, x, ld, dim, n, out);
    case OP2B_RED_MIN: return reduce_op<OP2B_RED_MIN>(c, x, ld, dim, n, out);
    default: return c->fail(OP2B_EINVAL, "dat_reduce: unknown operation");
  }
}

}  // namespace op2b
