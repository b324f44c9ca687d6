// Owner-compute partitions of an edge mesh (the paper's distributed-memory
// execution, Sec. 2 and 3.2: each process owns a part of the nodes, runs
// every edge with an owned end and refreshes its halo -- the non-owned ends
// of those edges -- from their owners before a loop reads them; Sec. 4: the
// parts come from recursive coordinate bisection).
//
// Host side: RCB partitioning and the halo plan (local meshes, import and
// export lists), exported as plain host functions.  Device side: the halo
// exchange of a dat between parts that live on one GPU, one gather kernel
// over every (importer, owner) pair: dst[c][di] = src[c][si].
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

using namespace op2b;

struct op2b_halo_s {
  std::vector<HaloPart> parts;
};

// One (importer, owner) pair of an exchange: the dat rows of both parts.
struct ExSeg {
  const void* src;
  void* dst;
  int64_t sld, dld;
};

struct op2b_exchange_s {
  int32_t type = OP2B_F64, dim = 0;
  int64_t n = 0;             // entries (halo rows) over all pairs
  ExSeg* seg = nullptr;      // device, one per pair
  int32_t* eseg = nullptr;   // device, pair of every entry
  int32_t* sidx = nullptr;   // device, source row of every entry
  int32_t* didx = nullptr;   // device, destination row of every entry
};

namespace {

int host_fail(int code, const std::string& msg) {
  set_thread_error(msg);
  return code;
}

template <typename T>
__global__ void k_exchange(const ExSeg* __restrict__ seg, const int32_t* __restrict__ eseg,
                           const int32_t* __restrict__ sidx, const int32_t* __restrict__ didx,
                           int64_t n, int dim) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const ExSeg s = seg[eseg[t]];
    const T* __restrict__ src = (const T*)s.src;
    T* __restrict__ dst = (T*)s.dst;
    const int64_t si = sidx[t], di = didx[t];
    for (int c = 0; c < dim; c++) dst[c * s.dld + di] = src[c * s.sld + si];
  }
}

template <typename T>
int dev_upload(T** dst, const T* src, size_t count) {
  if (cudaMalloc((void**)dst, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    return OP2B_ENOMEM;
  }
  if (count && cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return OP2B_ECUDA;
  return OP2B_OK;
}

void free_exchange(op2b_exchange_s* x) {
  cudaFree(x->seg);
  cudaFree(x->eseg);
  cudaFree(x->sidx);
  cudaFree(x->didx);
  delete x;
}

}  // namespace

// ------------------------------------------------------------- host plans

extern "C" int op2b_host_partition_rcb(int64_t N, const double* xyz, int32_t nparts,
                                       int32_t* part) {
  if (N < 0 || (N > 0 && (!xyz || !part)) || N > INT32_MAX)
    return host_fail(OP2B_EINVAL, "partition_rcb: bad arguments");
  if (nparts < 1 || (int64_t)nparts > std::max<int64_t>(N, 1))
    return host_fail(OP2B_EINVAL, "partition_rcb: nparts must be in [1, max(N, 1)]");
  try {
    if (!rcb_parts(N, xyz, nparts, part)) return host_fail(OP2B_EINVAL, "partition_rcb failed");
  } catch (const std::bad_alloc&) {
    return host_fail(OP2B_ENOMEM, "partition_rcb: out of host memory");
  }
  return OP2B_OK;
}

extern "C" int op2b_halo_create(int64_t N, int64_t E, const int32_t* edge, const int32_t* part,
                                int32_t nparts, op2b_halo* out) {
  if (!out || N < 0 || E < 0 || (E > 0 && !edge) || (N > 0 && !part) || nparts < 1)
    return host_fail(OP2B_EINVAL, "halo_create: bad arguments");
  *out = nullptr;
  try {
    auto* h = new op2b_halo_s();
    std::string err;
    if (!build_halo_plan(N, E, edge, part, nparts, &h->parts, &err)) {
      delete h;
      return host_fail(OP2B_EINVAL, "halo_create: " + err);
    }
    *out = h;
  } catch (const std::bad_alloc&) {
    return host_fail(OP2B_ENOMEM, "halo_create: out of host memory");
  }
  return OP2B_OK;
}

extern "C" int op2b_halo_sizes(op2b_halo h, int32_t p, int64_t* sizes) {
  if (!h || !sizes || p < 0 || p >= (int32_t)h->parts.size())
    return host_fail(OP2B_EINVAL, "halo_sizes: bad handle, part or pointer");
  const HaloPart& q = h->parts[p];
  sizes[0] = q.n_owned;
  sizes[1] = (int64_t)q.nodes.size() - q.n_owned;
  sizes[2] = (int64_t)q.edges.size();
  sizes[3] = (int64_t)q.nbr.size();
  sizes[4] = (int64_t)q.exp_idx.size();
  sizes[5] = q.halo_edges;
  return OP2B_OK;
}

extern "C" int op2b_halo_part(op2b_halo h, int32_t p, int32_t* nodes, int32_t* edges,
                              int32_t* local_map, int32_t* halo_owner, int32_t* halo_src,
                              int32_t* nbr, int64_t* exp_off, int32_t* exp_idx) {
  if (!h || p < 0 || p >= (int32_t)h->parts.size())
    return host_fail(OP2B_EINVAL, "halo_part: bad handle or part");
  const HaloPart& q = h->parts[p];
  auto put = [](auto* dst, const auto& v) {
    if (dst && !v.empty()) std::copy(v.begin(), v.end(), dst);
  };
  put(nodes, q.nodes);
  put(edges, q.edges);
  put(local_map, q.lmap);
  put(halo_owner, q.halo_owner);
  put(halo_src, q.halo_src);
  put(nbr, q.nbr);
  put(exp_off, q.exp_off);
  put(exp_idx, q.exp_idx);
  return OP2B_OK;
}

extern "C" int op2b_halo_destroy(op2b_halo h) {
  delete h;
  return OP2B_OK;
}

// ------------------------------------------------------ device exchange

extern "C" int op2b_exchange_create(op2b_ctx h, int32_t type, int32_t dim, int32_t nseg,
                                    const void* const* src, const int64_t* src_ld,
                                    void* const* dst, const int64_t* dst_ld,
                                    const int64_t* count, const int32_t* src_idx,
                                    const int32_t* dst_idx, op2b_exchange* out) {
  if (!h) return host_fail(OP2B_EINVAL, "exchange_create: null context");
  Ctx* c = &h->c;
  if (!out) return c->fail(OP2B_EINVAL, "exchange_create: null output");
  *out = nullptr;
  if (type != OP2B_F64 && type != OP2B_F32 && type != OP2B_FF)
    return c->fail(OP2B_ETYPE, "exchange_create: type must be F64, F32 or FF");
  if (dim < 1 || dim > 64) return c->fail(OP2B_EDIM, "exchange_create: dim must be in [1, 64]");
  if (nseg < 0 || (nseg > 0 && (!src || !src_ld || !dst || !dst_ld || !count)))
    return c->fail(OP2B_EINVAL, "exchange_create: bad segment arrays");
  int64_t n = 0;
  for (int32_t s = 0; s < nseg; s++) {
    if (count[s] < 0) return c->fail(OP2B_EINVAL, "exchange_create: negative count");
    if (count[s] > 0 && (!src[s] || !dst[s] || src_ld[s] < 1 || dst_ld[s] < 1))
      return c->fail(OP2B_EINVAL, "exchange_create: segment " + std::to_string(s) +
                                      " has a null pointer or a bad leading dimension");
    n += count[s];
  }
  if (n > INT32_MAX) return c->fail(OP2B_ERANGE, "exchange_create: too many entries");
  if (n > 0 && (!src_idx || !dst_idx))
    return c->fail(OP2B_EINVAL, "exchange_create: null index arrays");
  std::vector<int32_t> eseg(n);
  std::vector<ExSeg> segs(nseg);
  int64_t t = 0;
  for (int32_t s = 0; s < nseg; s++) {
    segs[s] = {src[s], dst[s], src_ld[s], dst_ld[s]};
    for (int64_t k = 0; k < count[s]; k++, t++) {
      // every row stays inside its dat: indices below the leading dimension
      if (src_idx[t] < 0 || src_idx[t] >= src_ld[s] || dst_idx[t] < 0 || dst_idx[t] >= dst_ld[s])
        return c->fail(OP2B_EINVAL, "exchange_create: entry " + std::to_string(t) +
                                        " indexes outside its dat");
      eseg[t] = s;
    }
  }
  auto* x = new op2b_exchange_s();
  x->type = type;
  x->dim = dim;
  x->n = n;
  int rc = dev_upload(&x->seg, segs.data(), segs.size());
  if (rc == OP2B_OK) rc = dev_upload(&x->eseg, eseg.data(), eseg.size());
  if (rc == OP2B_OK) rc = dev_upload(&x->sidx, src_idx, (size_t)n);
  if (rc == OP2B_OK) rc = dev_upload(&x->didx, dst_idx, (size_t)n);
  if (rc != OP2B_OK) {
    free_exchange(x);
    return c->fail(rc, "exchange_create: device allocation or upload failed");
  }
  *out = x;
  return OP2B_OK;
}

extern "C" int op2b_exchange_run(op2b_ctx h, op2b_exchange x) {
  if (!h) return host_fail(OP2B_EINVAL, "exchange_run: null context");
  Ctx* c = &h->c;
  if (!x) return c->fail(OP2B_EINVAL, "exchange_run: null exchange");
  if (x->n == 0) return OP2B_OK;
  const int block = 256;
  const int64_t want = (x->n + block - 1) / block;
  const int grid = (int)std::min<int64_t>(want, (int64_t)c->sm_count * 8);
  if (x->type == OP2B_F64 || x->type == OP2B_FF)  // 8-byte rows, copied bitwise
    k_exchange<double><<<grid, block, 0, c->stream>>>(x->seg, x->eseg, x->sidx, x->didx, x->n,
                                                       x->dim);
  else
    k_exchange<float><<<grid, block, 0, c->stream>>>(x->seg, x->eseg, x->sidx, x->didx, x->n,
                                                      x->dim);
  return c->launched("halo exchange");
}

extern "C" int op2b_exchange_destroy(op2b_ctx h, op2b_exchange x) {
  if (!x) return OP2B_OK;
  if (h) cudaStreamSynchronize(h->c.stream);
  free_exchange(x);
  return OP2B_OK;
}
