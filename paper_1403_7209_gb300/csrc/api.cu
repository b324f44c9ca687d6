// The op2b C ABI: contexts, sets / maps / dats (Sec. 3.1 of the paper),
// renumbering (Sec. 4), argument validation of the parallel loops, the
// execution plans and the autotuner (Sec. 4.1).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <thread>

#include "internal.h"

using namespace op2b;

static thread_local std::string g_init_err;

void op2b::set_thread_error(const std::string& msg) { g_init_err = msg; }

#define OP2B_VERSION_STR "op2b 0.1 (sm_103a)"

static const char* kLoopName[OP2B_NUM_LOOPS] = {
    "green_gauss", "flux1", "flux2", "spectral", "flux1_adj", "flux2_adj", "gg_adj",
    "flux1_tan", "flux2_tan", "gg_tan", "viscous", "flux2_phi", "jacobi", "jacobi_sums"};

// ------------------------------------------------------------------ Ctx
namespace op2b {

int Ctx::launched(const char* what) {
  launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(OP2B_ECUDA, std::string("kernel launch (") + what + "): " + cudaGetErrorString(e));
  return OP2B_OK;
}

int Ctx::need_scratch(size_t bytes, void** out) {
  if (bytes > scratch_bytes) {
    if (scratch) {
      cudaStreamSynchronize(stream);
      cudaFree(scratch);
      scratch = nullptr;
      scratch_bytes = 0;
    }
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(OP2B_ENOMEM, "scratch allocation of " + std::to_string(bytes) + " B failed");
    }
    scratch_bytes = bytes;
  }
  *out = scratch;
  return OP2B_OK;
}

int Ctx::need_aux(size_t bytes, void** out) {
  if (bytes > aux_bytes) {
    if (aux) {
      cudaStreamSynchronize(stream);
      cudaFree(aux);
      aux = nullptr;
      aux_bytes = 0;
    }
    if (cudaMalloc(&aux, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(OP2B_ENOMEM, "aux allocation of " + std::to_string(bytes) + " B failed");
    }
    aux_bytes = bytes;
  }
  *out = aux;
  return OP2B_OK;
}

template <typename T>
static int upload(Ctx* c, T** dst, const std::vector<T>& v) {
  size_t b = std::max<size_t>(1, v.size() * sizeof(T));
  if (cudaMalloc((void**)dst, b) != cudaSuccess) {
    cudaGetLastError();
    return c->fail(OP2B_ENOMEM, "plan allocation failed");
  }
  if (!v.empty() && cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return c->fail(OP2B_ECUDA, "plan upload failed");
  return OP2B_OK;
}

static void free_block_plan(DevBlockPlan& p) {
  cudaFree(p.bn_off);
  cudaFree(p.bnodes);
  cudaFree(p.lrow);
  cudaFree(p.cblocks);
  cudaFree(p.eloc);
  cudaFree(p.lent);
  p = DevBlockPlan();
}

static void free_seg_plan(DevSegPlan& p) {
  cudaFree(p.rowptr);
  cudaFree(p.ends);
  p = DevSegPlan();
}

static void split_map(const MapRec& m, std::vector<int32_t>& m0, std::vector<int32_t>& m1) {
  int64_t E = (int64_t)m.host.size() / 2;
  m0.resize(E);
  m1.resize(E);
  for (int64_t e = 0; e < E; e++) {
    m0[e] = m.host[2 * e];
    m1[e] = m.host[2 * e + 1];
  }
}

int Ctx::block_plan(int map, int32_t part, DevBlockPlan** out) {
  if (part <= 0) part = 512;
  if (part > 8192) return fail(OP2B_EINVAL, "partition size must be <= 8192");
  MapRec& m = maps[map];
  // a partition never needs to be longer than the edge set
  const int64_t E = sets[m.from].size;
  if (E < part) part = (int32_t)std::max<int64_t>(1, E);
  auto key = std::make_pair(map, (int)part);
  auto it = bplans.find(key);
  if (it != bplans.end() && it->second.map_version == m.version) {
    *out = &it->second;
    return OP2B_OK;
  }
  if (it != bplans.end()) {
    cudaStreamSynchronize(stream);
    free_block_plan(it->second);
  }
  std::vector<int32_t> m0, m1;
  split_map(m, m0, m1);
  BlockPlan hp;
  std::string e;
  if (!build_block_plan(sets[m.to].size, (int64_t)m0.size(), m0.data(), m1.data(), part, &hp, &e))
    return fail(OP2B_EPLAN, e);
  DevBlockPlan& d = bplans[key];
  d.map_version = m.version;
  d.part = part;
  d.nblocks = hp.nblocks;
  d.ncolours = hp.ncolours;
  d.max_unique = hp.max_unique;
  d.avg_unique = hp.avg_unique;
  d.coff = hp.coff;
  d.min_per_colour = hp.nblocks;
  d.max_per_colour = 0;
  for (int32_t k = 0; k < hp.ncolours; k++) {
    int64_t nbk = hp.coff[k + 1] - hp.coff[k];
    d.min_per_colour = std::min(d.min_per_colour, nbk);
    d.max_per_colour = std::max(d.max_per_colour, nbk);
  }
  int rc;
  if ((rc = upload(this, &d.bn_off, hp.bn_off)) || (rc = upload(this, &d.bnodes, hp.bnodes)) ||
      (rc = upload(this, &d.eloc, hp.eloc)) || (rc = upload(this, &d.lrow, hp.lrow)) ||
      (rc = upload(this, &d.lent, hp.lent)) || (rc = upload(this, &d.cblocks, hp.cblocks))) {
    free_block_plan(d);
    bplans.erase(key);
    return rc;
  }
  *out = &d;
  return OP2B_OK;
}

int Ctx::seg_plan(int map, DevSegPlan** out) {
  MapRec& m = maps[map];
  auto it = splans.find(map);
  if (it != splans.end() && it->second.map_version == m.version) {
    *out = &it->second;
    return OP2B_OK;
  }
  if (it != splans.end()) {
    cudaStreamSynchronize(stream);
    free_seg_plan(it->second);
  }
  std::vector<int32_t> m0, m1;
  split_map(m, m0, m1);
  if ((int64_t)m0.size() * 2 >= ((int64_t)1 << 31))
    return fail(OP2B_ERANGE, "segmented plan: more than 2^30 edges");
  std::vector<int64_t> rp;
  std::vector<int32_t> ends;
  node_csr(sets[m.to].size, (int64_t)m0.size(), m0.data(), m1.data(), &rp, &ends);
  DevSegPlan& d = splans[map];
  d.map_version = m.version;
  int rc;
  if ((rc = upload(this, &d.rowptr, rp)) || (rc = upload(this, &d.ends, ends))) {
    free_seg_plan(d);
    splans.erase(map);
    return rc;
  }
  *out = &d;
  return OP2B_OK;
}

int Ctx::own_plan(int map, DevOwnPlan** out) {
  MapRec& m = maps[map];
  auto it = oplans.find(map);
  if (it != oplans.end() && it->second.map_version == m.version) {
    *out = &it->second;
    return OP2B_OK;
  }
  if (it != oplans.end()) {
    cudaStreamSynchronize(stream);
    cudaFree(it->second.ptr);
    cudaFree(it->second.idx);
    it->second = DevOwnPlan();
  }
  std::vector<int32_t> m0, m1;
  split_map(m, m0, m1);
  std::vector<int64_t> ptr;
  std::vector<int32_t> idx;
  owner_csr(sets[m.to].size, (int64_t)m0.size(), m0.data(), m1.data(), &ptr, &idx);
  DevOwnPlan& d = oplans[map];
  d.map_version = m.version;
  int rc;
  if ((rc = upload(this, &d.ptr, ptr)) || (rc = upload(this, &d.idx, idx))) {
    cudaFree(d.ptr);
    cudaFree(d.idx);
    oplans.erase(map);
    return rc;
  }
  *out = &d;
  return OP2B_OK;
}

}  // namespace op2b

// ------------------------------------------------------------- lifecycle
#define CTX_CHECK(c)                                  \
  do {                                                \
    if (!(c)) return OP2B_EINVAL;                     \
  } while (0)

extern "C" const char* op2b_version(void) { return OP2B_VERSION_STR; }

extern "C" int op2b_init(op2b_ctx* out, int32_t device, void* stream) {
  if (!out) return OP2B_EINVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    g_init_err = std::string("no usable CUDA device: ") +
                 (e != cudaSuccess ? cudaGetErrorString(e) : "device index out of range");
    return OP2B_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    g_init_err = "cudaSetDevice failed";
    return OP2B_ECUDA;
  }
  auto* h = new (std::nothrow) op2b_ctx_s();
  if (!h) return OP2B_ENOMEM;
  Ctx& c = h->c;
  c.device = device;
  c.stream = (cudaStream_t)stream;
  cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c.smem_optin = (size_t)optin;
  // defaults: FP64 atomics everywhere until told or tuned otherwise
  for (int l = 0; l < OP2B_NUM_LOOPS; l++)
    for (int p = 0; p < OP2B_NUM_PREC; p++) c.strat[l][p] = Strategy();
  *out = h;
  return OP2B_OK;
}

extern "C" int op2b_finalize(op2b_ctx h) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  cudaStreamSynchronize(c.stream);
  for (auto& kv : c.bplans) free_block_plan(kv.second);
  for (auto& kv : c.splans) free_seg_plan(kv.second);
  for (auto& kv : c.oplans) {
    cudaFree(kv.second.ptr);
    cudaFree(kv.second.idx);
  }
  stage32_free_all(c);
  for (auto& m : c.maps) cudaFree(m.dev);
  cudaFree(c.scratch);
  cudaFree(c.aux);
  delete h;
  return OP2B_OK;
}

extern "C" int op2b_set_stream(op2b_ctx h, void* stream) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  cudaStream_t ns = (cudaStream_t)stream;
  if (ns == c.stream) return OP2B_OK;
  // Every loop shares the context's scratch, aux buffer and plans: work
  // launched on the new stream must not start before the work already
  // queued on the old one, so the new stream waits for an event recorded on
  // the old stream at the switch.
  cudaEvent_t ev;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return c.fail(OP2B_ECUDA, "set_stream: event creation failed");
  }
  cudaError_t e = cudaEventRecord(ev, c.stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ns, ev, 0);
  cudaEventDestroy(ev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return c.fail(OP2B_ECUDA, std::string("set_stream: ordering after the old stream failed: ") +
                                  cudaGetErrorString(e));
  }
  c.stream = ns;
  return OP2B_OK;
}

extern "C" const char* op2b_last_error(op2b_ctx h) {
  return h ? h->c.err.c_str() : g_init_err.c_str();
}

extern "C" int64_t op2b_launch_count(op2b_ctx h) { return h ? h->c.launches : -1; }

// ---------------------------------------------------------- declarations
extern "C" int op2b_decl_set(op2b_ctx h, int64_t size, const char* name, op2b_set* out) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!out || size < 0) return c.fail(OP2B_EINVAL, "decl_set: bad size or output");
  if (size >= ((int64_t)1 << 31) - 1) return c.fail(OP2B_ERANGE, "decl_set: sets are limited to 2^31-2 elements");
  c.sets.push_back({size, name ? name : ""});
  *out = (op2b_set)(c.sets.size() - 1);
  return OP2B_OK;
}

static bool valid_set(Ctx& c, op2b_set s) { return s >= 0 && s < (op2b_set)c.sets.size(); }
static bool valid_map(Ctx& c, op2b_map m) { return m >= 0 && m < (op2b_map)c.maps.size(); }
static bool valid_dat(Ctx& c, op2b_dat d) { return d >= 0 && d < (op2b_dat)c.dats.size(); }

static int upload_map(Ctx& c, MapRec& m) {
  int64_t F = c.sets[m.from].size;
  std::vector<int32_t> soa((size_t)F * m.arity);
  for (int64_t e = 0; e < F; e++)
    for (int k = 0; k < m.arity; k++) soa[(size_t)k * F + e] = m.host[(size_t)e * m.arity + k];
  if (!m.dev) {
    if (cudaMalloc((void**)&m.dev, std::max<size_t>(1, soa.size() * 4)) != cudaSuccess) {
      cudaGetLastError();
      return c.fail(OP2B_ENOMEM, "map allocation failed");
    }
  }
  if (!soa.empty() && cudaMemcpy(m.dev, soa.data(), soa.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return c.fail(OP2B_ECUDA, "map upload failed");
  return OP2B_OK;
}

extern "C" int op2b_decl_map(op2b_ctx h, op2b_set from, op2b_set to, int32_t arity,
                             const int32_t* data, const char* name, op2b_map* out) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!out || !valid_set(c, from) || !valid_set(c, to) || arity < 1 || arity > 16)
    return c.fail(OP2B_EINVAL, "decl_map: bad set, arity or output");
  int64_t F = c.sets[from].size, T = c.sets[to].size;
  if (F > 0 && !data) return c.fail(OP2B_EINVAL, "decl_map: null data");
  MapRec m;
  m.from = from;
  m.to = to;
  m.arity = arity;
  m.name = name ? name : "";
  m.host.assign(data, data + (size_t)F * arity);
  for (int32_t v : m.host)
    if (v < 0 || v >= T) return c.fail(OP2B_EINVAL, "decl_map: index outside the to-set");
  int rc = upload_map(c, m);
  if (rc) {
    cudaFree(m.dev);
    return rc;
  }
  c.maps.push_back(std::move(m));
  *out = (op2b_map)(c.maps.size() - 1);
  return OP2B_OK;
}

static int esize(int type) { return (type == OP2B_F64 || type == OP2B_FF) ? 8 : 4; }

extern "C" int op2b_decl_dat(op2b_ctx h, op2b_set set, int32_t dim, int32_t type, void* ptr,
                             int64_t ld, const char* name, op2b_dat* out) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!out || !valid_set(c, set) || dim < 1 || dim > 64)
    return c.fail(OP2B_EINVAL, "decl_dat: bad set, dim or output");
  if (type != OP2B_F64 && type != OP2B_F32 && type != OP2B_I32 && type != OP2B_FF)
    return c.fail(OP2B_ETYPE, "decl_dat: unknown type");
  int64_t n = c.sets[set].size;
  if (ld == 0) ld = n;
  if (ld < n) return c.fail(OP2B_EINVAL, "decl_dat: ld smaller than the set size");
  if (!ptr && n > 0) return c.fail(OP2B_EINVAL, "decl_dat: null device pointer");
  c.dats.push_back({set, dim, type, ptr, ld, name ? name : ""});
  *out = (op2b_dat)(c.dats.size() - 1);
  return OP2B_OK;
}

extern "C" int op2b_rebind_dat(op2b_ctx h, op2b_dat d, void* ptr) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!valid_dat(c, d)) return c.fail(OP2B_EINVAL, "rebind_dat: bad dat");
  if (!ptr && c.sets[c.dats[d].set].size > 0) return c.fail(OP2B_EINVAL, "rebind_dat: null pointer");
  c.dats[d].ptr = ptr;
  return OP2B_OK;
}

extern "C" int op2b_fetch_map(op2b_ctx h, op2b_map m, int32_t* out) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!valid_map(c, m) || !out) return c.fail(OP2B_EINVAL, "fetch_map: bad map or output");
  std::copy(c.maps[m].host.begin(), c.maps[m].host.end(), out);
  return OP2B_OK;
}

// ----------------------------------------------------------- renumbering
static int permute_dat(Ctx& c, DatRec& d, const int64_t* idx_dev, int64_t n) {
  if (n == 0) return OP2B_OK;
  int es = esize(d.type);
  void* tmp = nullptr;
  int rc = c.need_scratch((size_t)d.dim * d.ld * es, &tmp);
  if (rc) return rc;
  if ((rc = node_gather(&c, tmp, d.ptr, es, d.ld, d.dim, idx_dev, n))) return rc;
  if (cudaMemcpy2DAsync(d.ptr, d.ld * es, tmp, d.ld * es, n * es, d.dim, cudaMemcpyDeviceToDevice,
                        c.stream) != cudaSuccess)
    return c.fail(OP2B_ECUDA, "renumber: copy back failed");
  return OP2B_OK;
}

// Apply a node permutation (new id of each old node) and the matching edge
// order to the maps and to every dat on the two sets of map `mid`.
static int apply_renumbering(Ctx& c, op2b_map mid, const std::vector<int32_t>& nperm,
                             const std::vector<int64_t>& order) {
  MapRec& m = c.maps[mid];
  const op2b_set eset = m.from, nset = m.to;
  const int64_t N = c.sets[nset].size, E = c.sets[eset].size;
  std::vector<int64_t> old_of_new(N), new_edge(E);
  for (int64_t i = 0; i < N; i++) old_of_new[nperm[i]] = i;
  for (int64_t t = 0; t < E; t++) new_edge[order[t]] = t;
  int rc = OP2B_OK;
  // maps: reorder rows of maps from a renumbered set, relabel entries into one
  for (auto& mm : c.maps) {
    if (!(mm.from == eset || mm.from == nset || mm.to == nset || mm.to == eset)) continue;
    std::vector<int32_t> nh(mm.host.size());
    int64_t F = c.sets[mm.from].size;
    for (int64_t r = 0; r < F; r++) {
      int64_t src = r;
      if (mm.from == eset) src = order[r];
      else if (mm.from == nset) src = old_of_new[r];
      for (int k = 0; k < mm.arity; k++) {
        int64_t v = mm.host[(size_t)src * mm.arity + k];
        if (mm.to == nset) v = nperm[v];
        else if (mm.to == eset) v = new_edge[v];
        nh[(size_t)r * mm.arity + k] = (int32_t)v;
      }
    }
    mm.host.swap(nh);
    mm.version++;
    if ((rc = upload_map(c, mm))) return rc;
  }
  // dats on the two sets, through the scratch buffer
  int64_t* idx = nullptr;
  if (cudaMalloc((void**)&idx, std::max<int64_t>(1, std::max(N, E)) * 8) != cudaSuccess) {
    cudaGetLastError();
    return c.fail(OP2B_ENOMEM, "renumber: index allocation failed");
  }
  if (N > 0) cudaMemcpy(idx, old_of_new.data(), N * 8, cudaMemcpyHostToDevice);
  for (auto& d : c.dats)
    if (d.set == nset && (rc = permute_dat(c, d, idx, N))) break;
  if (!rc) {
    cudaStreamSynchronize(c.stream);
    if (E > 0) cudaMemcpy(idx, order.data(), E * 8, cudaMemcpyHostToDevice);
    if (eset != nset)
      for (auto& d : c.dats)
        if (d.set == eset && (rc = permute_dat(c, d, idx, E))) break;
  }
  cudaStreamSynchronize(c.stream);
  cudaFree(idx);
  return rc;
}

extern "C" int op2b_renumber(op2b_ctx h, op2b_map mid, int32_t method, uint64_t seed,
                             int32_t* node_perm_out, int64_t* edge_order_out) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!valid_map(c, mid) || c.maps[mid].arity != 2)
    return c.fail(OP2B_EINVAL, "renumber: needs an arity-2 map");
  MapRec& m = c.maps[mid];
  const int64_t N = c.sets[m.to].size, E = c.sets[m.from].size;
  std::vector<int32_t> nperm(N);
  std::vector<int64_t> order(E);
  int rc = op2b_host_renumber(N, E, m.host.data(), method, seed, nperm.data(), order.data());
  if (rc) return c.fail(rc, "renumber: bad method or map");
  if ((rc = apply_renumbering(c, mid, nperm, order))) return rc;
  if (node_perm_out) std::copy(nperm.begin(), nperm.end(), node_perm_out);
  if (edge_order_out) std::copy(order.begin(), order.end(), edge_order_out);
  return OP2B_OK;
}

extern "C" int op2b_renumber_rcb(op2b_ctx h, op2b_map mid, op2b_dat coords, int32_t leaf,
                                 int32_t* node_perm_out, int64_t* edge_order_out) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!valid_map(c, mid) || c.maps[mid].arity != 2)
    return c.fail(OP2B_EINVAL, "renumber_rcb: needs an arity-2 map");
  if (leaf < 1) return c.fail(OP2B_EINVAL, "renumber_rcb: leaf must be >= 1");
  MapRec& m = c.maps[mid];
  if (!valid_dat(c, coords)) return c.fail(OP2B_EINVAL, "renumber_rcb: bad coordinate dat");
  const DatRec& x = c.dats[coords];
  if (x.set != m.to) return c.fail(OP2B_ESET, "renumber_rcb: coordinates must live on the nodes");
  if (x.dim != 3) return c.fail(OP2B_EDIM, "renumber_rcb: coordinates need dim 3");
  if (x.type != OP2B_F64) return c.fail(OP2B_ETYPE, "renumber_rcb: coordinates must be F64");
  const int64_t N = c.sets[m.to].size, E = c.sets[m.from].size;
  std::vector<double> soa((size_t)3 * x.ld), xyz((size_t)3 * N);
  cudaStreamSynchronize(c.stream);
  if (N > 0 && cudaMemcpy(soa.data(), x.ptr, soa.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return c.fail(OP2B_ECUDA, "renumber_rcb: coordinate copy failed");
  for (int64_t i = 0; i < N; i++)
    for (int d = 0; d < 3; d++) xyz[3 * i + d] = soa[(size_t)d * x.ld + i];
  std::vector<int32_t> nperm(N);
  std::vector<int64_t> order(E);
  if (!op2b::rcb(N, xyz.data(), leaf, nperm.data()))
    return c.fail(OP2B_EINVAL, "renumber_rcb: bad input");
  op2b::edge_order(N, E, m.host.data(), nperm.data(), order.data());
  int rc = apply_renumbering(c, mid, nperm, order);
  if (rc) return rc;
  if (node_perm_out) std::copy(nperm.begin(), nperm.end(), node_perm_out);
  if (edge_order_out) std::copy(order.begin(), order.end(), edge_order_out);
  return OP2B_OK;
}

// ------------------------------------------------------ argument checks
namespace {

// expected argument: map entry (0/1) or -1 for direct; access; dim;
// type class: 'P' the loop's precision, 'D' always F64
struct Spec {
  int idx;
  int acc;
  int dim;
  char tcls;
};

struct Checked {
  int map = -1;
  int prec = OP2B_PREC_F64;
  int64_t N = 0, E = 0;
};

int check_args(Ctx& c, const char* loop, const op2b_arg* a, int nargs, const Spec* sp, int ns,
               Checked* out) {
  if (!a || nargs != ns)
    return c.fail(OP2B_EINVAL, std::string(loop) + ": expected " + std::to_string(ns) + " arguments");
  int map = -1, ptype = -1;
  for (int k = 0; k < ns; k++) {
    if (!valid_dat(c, a[k].dat))
      return c.fail(OP2B_EINVAL, std::string(loop) + ": argument " + std::to_string(k) + " is not a dat");
    if (sp[k].idx >= 0) {
      if (a[k].map == OP2B_ID || !valid_map(c, a[k].map))
        return c.fail(OP2B_EINVAL, std::string(loop) + ": argument " + std::to_string(k) + " needs a map");
      if (map < 0) map = a[k].map;
      if (a[k].map != map)
        return c.fail(OP2B_EINVAL, std::string(loop) + ": all indirect arguments must use one map");
    }
  }
  if (map < 0) return c.fail(OP2B_EINVAL, std::string(loop) + ": no indirect argument");
  const MapRec& m = c.maps[map];
  if (m.arity != 2) return c.fail(OP2B_EINVAL, std::string(loop) + ": the map must have arity 2");
  for (int k = 0; k < ns; k++) {
    const op2b_arg& x = a[k];
    const DatRec& d = c.dats[x.dat];
    std::string at = std::string(loop) + ": argument " + std::to_string(k) + " (" + d.name + ")";
    if (sp[k].idx >= 0) {
      if (x.idx != sp[k].idx) return c.fail(OP2B_EINVAL, at + ": wrong map index");
      if (d.set != m.to) return c.fail(OP2B_ESET, at + ": dat is not on the map's to-set");
      if (x.acc == OP2B_WRITE || x.acc == OP2B_RW)
        return c.fail(OP2B_EACCESS, at + ": WRITE/RW through a map is not allowed (use INC)");
    } else {
      if (x.map != OP2B_ID || x.idx != -1) return c.fail(OP2B_EINVAL, at + ": expected a direct argument");
      if (d.set != m.from) return c.fail(OP2B_ESET, at + ": dat is not on the loop's set");
      if (x.acc == OP2B_INC) return c.fail(OP2B_EACCESS, at + ": INC on a direct argument");
    }
    if (x.acc != sp[k].acc) return c.fail(OP2B_EACCESS, at + ": wrong access mode");
    if (d.dim != sp[k].dim)
      return c.fail(OP2B_EDIM, at + ": dim " + std::to_string(d.dim) + ", expected " + std::to_string(sp[k].dim));
    if (sp[k].tcls == 'D') {
      if (d.type != OP2B_F64) return c.fail(OP2B_ETYPE, at + ": must be F64");
    } else {
      if (d.type != OP2B_F64 && d.type != OP2B_F32 && d.type != OP2B_FF)
        return c.fail(OP2B_ETYPE, at + ": must be F64, F32 or FF");
      if (ptype < 0) ptype = d.type;
      if (d.type != ptype) return c.fail(OP2B_ETYPE, at + ": mixed F64/F32/FF data");
    }
  }
  // the two ends of an indirect dat (adjacent entries 0 and 1) are one dat
  for (int k = 0; k + 1 < ns; k++)
    if (sp[k].idx == 0 && sp[k + 1].idx == 1 && a[k].dat != a[k + 1].dat)
      return c.fail(OP2B_EINVAL, std::string(loop) + ": map entries 0 and 1 of one argument use different dats");
  out->map = map;
  out->prec = ptype == OP2B_F32 ? OP2B_PREC_F32 : (ptype == OP2B_FF ? OP2B_PREC_FF : OP2B_PREC_F64);
  out->N = c.sets[m.to].size;
  out->E = c.sets[m.from].size;
  return OP2B_OK;
}

const DatRec& D(Ctx& c, const op2b_arg& a) { return c.dats[a.dat]; }

std::string tune_key(const LoopLaunch& L, bool det) {
  return std::string(kLoopName[L.loop]) + ":p" + std::to_string(L.prec) + ":N" + std::to_string(L.N) +
         ":E" + std::to_string(L.E) + (det ? ":det" : "");
}

// whether the Green-Gauss launch writes every node's finished sums itself
// (the node gather, and the node phase of the segmented strategy): its
// targets then need no zeroing, and it divides by the volumes as it writes;
// otherwise the scaling loop runs after it
static bool gg_writes_all(const LoopLaunch& L, const Strategy& s) {
  return L.loop == OP2B_LOOP_GREEN_GAUSS &&
         (L.prec == OP2B_PREC_FF || s.strategy == OP2B_STRAT_GATHER ||
          s.strategy == OP2B_STRAT_SEGMENTED);
}
static bool gg_scale_fused(const LoopLaunch& L, const Strategy& s) { return gg_writes_all(L, s); }

static int launch_loop(Ctx& c, const LoopLaunch& L, const Strategy& s) {
  if (L.loop == OP2B_LOOP_VISCOUS) return launch_visc(&c, L, s);  // F64, F32 or FF
  if (L.loop == OP2B_LOOP_FLUX2_PHI) return launch_lim(&c, L, s);  // F64, F32 or FF
  if (L.prec == OP2B_PREC_FF) return launch_ff(&c, L, s);  // GG, FLUX2, FLUX2_ADJ (checked there)
  if (L.loop == OP2B_LOOP_JACOBI || L.loop == OP2B_LOOP_JACOBI_SUMS) return launch_f64(&c, L, s);
  if (L.loop >= OP2B_LOOP_FLUX1_ADJ) return launch_adj(&c, L, s);
  return L.prec == OP2B_PREC_F32 ? launch_f32(&c, L, s) : launch_f64(&c, L, s);
}

int dispatch(Ctx& c, const LoopLaunch& L, const Strategy& s) {
  int rc = launch_loop(c, L, s);
  if (rc == OP2B_OK && L.vol && L.loop == OP2B_LOOP_GREEN_GAUSS && !gg_scale_fused(L, s)) {
    const int type = L.prec == OP2B_PREC_F32 ? OP2B_F32 : OP2B_F64;
    rc = node_grad_scale(&c, L.t0, type, L.ldt0, L.vol, L.N);
  }
  return rc;
}

// wait for an event with a host-side deadline
int wait_deadline(Ctx& c, cudaEvent_t ev, double ms) {
  auto t0 = std::chrono::steady_clock::now();
  while (true) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return OP2B_OK;
    if (e != cudaErrorNotReady) return c.fail(OP2B_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
    double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (el > ms) return c.fail(OP2B_ETIMEOUT, "autotune: candidate exceeded its deadline");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

std::vector<Strategy> candidates(const LoopLaunch& L, bool det) {
  std::vector<Strategy> v;
  for (int b : {128, 256, 512}) {
    if (det) break;
    Strategy s;
    s.strategy = OP2B_STRAT_ATOMIC;
    s.block = b;
    v.push_back(s);
  }
  for (int part : {256, 512, 1024, 2048})
    for (int st : {0, 1}) {
      Strategy s;
      s.strategy = OP2B_STRAT_COLOUR;
      s.part = part;
      s.block = std::min(part, 256);
      s.staged = st;
      v.push_back(s);
    }
  for (int b : {128, 256}) {
    Strategy s;
    s.strategy = OP2B_STRAT_SEGMENTED;
    s.block = b;
    v.push_back(s);
  }
  if (!det && L.loop == OP2B_LOOP_GREEN_GAUSS && L.prec == OP2B_PREC_F64)
    for (int b : {128, 256}) {
      Strategy s;
      s.strategy = OP2B_STRAT_HYBRID;
      s.block = b;
      v.push_back(s);
    }
  if (L.loop != OP2B_LOOP_FLUX1_ADJ && L.loop != OP2B_LOOP_FLUX2_ADJ && L.loop != OP2B_LOOP_GG_ADJ)
    for (int b : {128, 256}) {
      Strategy s;
      s.strategy = OP2B_STRAT_GATHER;
      s.block = b;
      v.push_back(s);
    }
  if (!det)
    for (int b : {128, 256}) {
      Strategy s;
      s.strategy = OP2B_STRAT_OWNER;
      s.block = b;
      v.push_back(s);
    }
  if (!det)
    for (int part : {512, 1024, 2048})
      for (int st : {0, 1}) {
        Strategy s;
        s.strategy = OP2B_STRAT_BLOCK_ATOMIC;
        s.part = part;
        s.block = 256;
        s.staged = st;
        v.push_back(s);
      }
  return v;
}

// Time every candidate on scratch copies of the outputs; keep the fastest.
int autotune(Ctx& c, const LoopLaunch& L, size_t b0, size_t b1, size_t bd, bool det,
             Strategy* best) {
  LoopLaunch T = L;
  void *t0 = nullptr, *t1 = nullptr, *td = nullptr;
  auto alloc = [&](size_t b, void** p) {
    if (!b) return true;
    if (cudaMalloc(p, b) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    cudaMemsetAsync(*p, 0, b, c.stream);
    return true;
  };
  if (!alloc(b0, &t0) || !alloc(b1, &t1) || !alloc(bd, &td)) {
    cudaFree(t0);
    cudaFree(t1);
    cudaFree(td);
    return c.fail(OP2B_ENOMEM, "autotune: scratch outputs");
  }
  T.t0 = t0;
  T.t1 = t1 ? t1 : t0;
  T.direct = td;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best_ms = 1e300;
  int rc = OP2B_OK, found = 0;
  std::string timings;
  for (const Strategy& s : candidates(L, det)) {
    int r = dispatch(c, T, s);  // warm-up (also builds the plan)
    // skip candidates that cannot run here: a block too large for shared
    // memory or registers (ERANGE), or a colouring that needs too many
    // colours (EPLAN, e.g. under a random numbering)
    if (r == OP2B_ERANGE || r == OP2B_EPLAN) continue;
    if (r) {
      rc = r;
      break;
    }
    cudaEventRecord(e0, c.stream);
    const int reps = 3;
    // the zeroing of the targets that run_loop does before this strategy is
    // part of its cost
    const bool zero = (L.flags & OP2B_ZERO_INC) && !gg_writes_all(L, s);
    for (int k = 0; k < reps && !r; k++) {
      if (zero) {
        if (b0) cudaMemsetAsync(t0, 0, b0, c.stream);
        if (b1) cudaMemsetAsync(t1, 0, b1, c.stream);
      }
      r = dispatch(c, T, s);
    }
    cudaEventRecord(e1, c.stream);
    if (r) {
      rc = r;
      break;
    }
    if ((r = wait_deadline(c, e1, c.tune_deadline_ms))) {
      rc = r;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    double per = ms / reps;
    char buf[96];
    snprintf(buf, sizeof buf, "%s[%d, %d, %d, %d, %.4f]", timings.empty() ? "" : ", ", s.strategy,
             s.block, s.part, s.staged, per);
    timings += buf;
    if (per < best_ms) {
      best_ms = per;
      *best = s;
      best->tuned_ms = per;
      found = 1;
    }
  }
  if (rc == OP2B_ETIMEOUT) {
    // let the candidate finish before its scratch outputs are freed
    cudaStreamSynchronize(c.stream);
  } else {
    cudaStreamSynchronize(c.stream);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(t0);
  cudaFree(t1);
  cudaFree(td);
  if (rc) return rc;
  if (!found) return c.fail(OP2B_EPLAN, "autotune: no candidate could run");
  best->timings = timings;
  return OP2B_OK;
}

size_t dat_bytes(Ctx& c, const DatRec& d) { return (size_t)d.dim * d.ld * esize(d.type); }

// strategy lookup / tuning, optional zeroing, then the launch
int run_loop(Ctx& c, LoopLaunch& L, int flags, const DatRec* z0, const DatRec* z1,
             const DatRec* direct) {
  L.flags = flags;
  // the float-float Green-Gauss loop is a node gather: it writes (or adds)
  // each node's sums itself and has no strategy to choose
  if (L.prec == OP2B_PREC_FF && L.loop == OP2B_LOOP_GREEN_GAUSS) return launch_ff(&c, L, Strategy());
  Strategy& s = c.strat[L.loop][L.prec];
  if (s.strategy == OP2B_STRAT_AUTO || s.strategy == OP2B_STRAT_AUTO_DET) {
    const bool det = s.strategy == OP2B_STRAT_AUTO_DET;
    auto it = c.tuned.find(tune_key(L, det));
    Strategy best;
    if (it != c.tuned.end()) {
      best = it->second;
    } else {
      int rc = autotune(c, L, z0 ? dat_bytes(c, *z0) : 0, z1 ? dat_bytes(c, *z1) : 0,
                        direct ? dat_bytes(c, *direct) : 0, det, &best);
      if (rc) return rc;
      c.tuned[tune_key(L, det)] = best;
    }
    s = best;
  }
  // the Green-Gauss node gather and segmented node phase write every node's
  // 18 sums, so their targets need no zeroing first
  if ((flags & OP2B_ZERO_INC) && !gg_writes_all(L, s)) {
    int rc;
    if (z0 && (rc = node_fill(&c, z0->ptr, z0->type, z0->ld, z0->dim, L.N, 0.0))) return rc;
    if (z1 && (rc = node_fill(&c, z1->ptr, z1->type, z1->ld, z1->dim, L.N, 0.0))) return rc;
  }
  return dispatch(c, L, s);
}

}  // namespace

// ------------------------------------------------------------ edge loops
static int node_dat(Ctx& c, op2b_dat d, int dim, int type, op2b_set set, const char* what);

static int green_gauss_impl(op2b_ctx h, const op2b_arg* a, int32_t nargs, op2b_dat V,
                            int32_t flags, const char* what) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  static const Spec sp[5] = {{0, OP2B_READ, 6, 'P'}, {1, OP2B_READ, 6, 'P'}, {-1, OP2B_READ, 3, 'P'},
                             {0, OP2B_INC, 18, 'P'}, {1, OP2B_INC, 18, 'P'}};
  Checked ck;
  int rc = check_args(c, what, a, nargs, sp, 5, &ck);
  if (rc) return rc;
  const double* vol = nullptr;
  if (V >= 0) {
    if ((rc = node_dat(c, V, 1, OP2B_F64, c.maps[ck.map].to, what))) return rc;
    vol = (const double*)c.dats[V].ptr;
  }
  LoopLaunch L;
  L.loop = OP2B_LOOP_GREEN_GAUSS;
  L.prec = ck.prec;
  L.map = ck.map;
  L.N = ck.N;
  L.E = ck.E;
  L.m0 = c.maps[ck.map].dev;
  L.m1 = c.maps[ck.map].dev + ck.E;
  L.q = D(c, a[0]).ptr;
  L.ldq = D(c, a[0]).ld;
  L.n = D(c, a[2]).ptr;
  L.ldn = D(c, a[2]).ld;
  L.t0 = D(c, a[3]).ptr;
  L.ldt0 = D(c, a[3]).ld;
  L.vol = vol;
  return run_loop(c, L, flags, &D(c, a[3]), nullptr, nullptr);
}

static int jacobi_loop(op2b_ctx h, const op2b_arg* a, int32_t nargs, double gamma,
                       int32_t flags, bool sums) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  const char* w = sums ? "jacobi_sums" : "jacobi_blocks";
  if (!(gamma > 1.0)) return c.fail(OP2B_EINVAL, std::string(w) + ": need gamma > 1");
  const int dim = sums ? 4 : 36;
  const Spec sp[5] = {{0, OP2B_READ, 6, 'D'}, {1, OP2B_READ, 6, 'D'}, {-1, OP2B_READ, 3, 'D'},
                      {0, OP2B_INC, dim, 'D'}, {1, OP2B_INC, dim, 'D'}};
  Checked ck;
  int rc = check_args(c, w, a, nargs, sp, 5, &ck);
  if (rc) return rc;
  LoopLaunch L;
  L.loop = sums ? OP2B_LOOP_JACOBI_SUMS : OP2B_LOOP_JACOBI;
  L.prec = OP2B_PREC_F64;
  L.map = ck.map;
  L.N = ck.N;
  L.E = ck.E;
  L.m0 = c.maps[ck.map].dev;
  L.m1 = c.maps[ck.map].dev + ck.E;
  L.gamma = gamma;
  L.q = D(c, a[0]).ptr;
  L.ldq = D(c, a[0]).ld;
  if (sums) {  // the sums need only each node's (u, a), formed once per node
    void* W = nullptr;
    if ((rc = c.need_aux((size_t)4 * std::max<int64_t>(ck.N, 1) * sizeof(double), &W))) return rc;
    if ((rc = node_wave_prims(&c, (const double*)L.q, L.ldq, (double*)W, gamma, ck.N))) return rc;
    L.q = W;
    L.ldq = ck.N;
  }
  L.n = D(c, a[2]).ptr;
  L.ldn = D(c, a[2]).ld;
  L.t0 = D(c, a[3]).ptr;
  L.ldt0 = D(c, a[3]).ld;
  return run_loop(c, L, flags, &D(c, a[3]), nullptr, nullptr);
}

extern "C" int op2b_jacobi_blocks(op2b_ctx h, const op2b_arg* a, int32_t nargs, double gamma,
                                  int32_t flags) {
  return jacobi_loop(h, a, nargs, gamma, flags, false);
}

extern "C" int op2b_jacobi_sums(op2b_ctx h, const op2b_arg* a, int32_t nargs, double gamma,
                                int32_t flags) {
  return jacobi_loop(h, a, nargs, gamma, flags, true);
}

extern "C" int op2b_green_gauss(op2b_ctx h, const op2b_arg* a, int32_t nargs, int32_t flags) {
  return green_gauss_impl(h, a, nargs, -1, flags, "green_gauss");
}

extern "C" int op2b_green_gauss_scaled(op2b_ctx h, const op2b_arg* a, int32_t nargs, op2b_dat V,
                                       int32_t flags) {
  return green_gauss_impl(h, a, nargs, V, flags, "green_gauss_scaled");
}

extern "C" int op2b_edge_flux(op2b_ctx h, const op2b_arg* a, int32_t nargs, const op2b_flux_params* p) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!p || (p->order != 1 && p->order != 2)) return c.fail(OP2B_EINVAL, "edge_flux: order must be 1 or 2");
  if (!(p->gamma > 1.0) || !(p->eps_lim > 0.0)) return c.fail(OP2B_EINVAL, "edge_flux: need gamma > 1, eps > 0");
  static const Spec s1[5] = {{0, OP2B_READ, 6, 'P'}, {1, OP2B_READ, 6, 'P'}, {-1, OP2B_READ, 3, 'P'},
                             {0, OP2B_INC, 6, 'D'}, {1, OP2B_INC, 6, 'D'}};
  static const Spec s2[8] = {{0, OP2B_READ, 6, 'P'},  {1, OP2B_READ, 6, 'P'},  {0, OP2B_READ, 18, 'P'},
                             {1, OP2B_READ, 18, 'P'}, {-1, OP2B_READ, 3, 'P'}, {-1, OP2B_READ, 3, 'P'},
                             {0, OP2B_INC, 6, 'D'},   {1, OP2B_INC, 6, 'D'}};
  Checked ck;
  int rc = p->order == 1 ? check_args(c, "edge_flux", a, nargs, s1, 5, &ck)
                         : check_args(c, "edge_flux", a, nargs, s2, 8, &ck);
  if (rc) return rc;
  LoopLaunch L;
  L.loop = p->order == 1 ? OP2B_LOOP_FLUX1 : OP2B_LOOP_FLUX2;
  L.prec = ck.prec;
  L.order = p->order;
  L.map = ck.map;
  L.N = ck.N;
  L.E = ck.E;
  L.m0 = c.maps[ck.map].dev;
  L.m1 = c.maps[ck.map].dev + ck.E;
  L.gamma = p->gamma;
  L.eps = p->eps_lim;
  L.q = D(c, a[0]).ptr;
  L.ldq = D(c, a[0]).ld;
  const op2b_arg* R;
  if (p->order == 1) {
    L.n = D(c, a[2]).ptr;
    L.ldn = D(c, a[2]).ld;
    R = &a[3];
  } else {
    L.G = D(c, a[2]).ptr;
    L.ldG = D(c, a[2]).ld;
    L.n = D(c, a[4]).ptr;
    L.ldn = D(c, a[4]).ld;
    L.dx = D(c, a[5]).ptr;
    L.lddx = D(c, a[5]).ld;
    R = &a[6];
  }
  L.t0 = D(c, *R).ptr;
  L.ldt0 = D(c, *R).ld;
  return run_loop(c, L, p->flags, &D(c, *R), nullptr, nullptr);
}

extern "C" int op2b_edge_flux_limited(op2b_ctx h, const op2b_arg* a, int32_t nargs,
                                      const op2b_flux_params* p) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!p || !(p->gamma > 1.0)) return c.fail(OP2B_EINVAL, "edge_flux_limited: need gamma > 1");
  static const Spec sp[10] = {{0, OP2B_READ, 6, 'P'},  {1, OP2B_READ, 6, 'P'},  {0, OP2B_READ, 18, 'P'},
                              {1, OP2B_READ, 18, 'P'}, {0, OP2B_READ, 6, 'P'},  {1, OP2B_READ, 6, 'P'},
                              {-1, OP2B_READ, 3, 'P'}, {-1, OP2B_READ, 3, 'P'}, {0, OP2B_INC, 6, 'D'},
                              {1, OP2B_INC, 6, 'D'}};
  Checked ck;
  int rc = check_args(c, "edge_flux_limited", a, nargs, sp, 10, &ck);
  if (rc) return rc;
  LoopLaunch L;
  L.loop = OP2B_LOOP_FLUX2_PHI;
  L.prec = ck.prec;
  L.order = 2;
  L.map = ck.map;
  L.N = ck.N;
  L.E = ck.E;
  L.m0 = c.maps[ck.map].dev;
  L.m1 = c.maps[ck.map].dev + ck.E;
  L.gamma = p->gamma;
  L.eps = p->eps_lim;
  L.q = D(c, a[0]).ptr;
  L.ldq = D(c, a[0]).ld;
  L.G = D(c, a[2]).ptr;
  L.ldG = D(c, a[2]).ld;
  L.phi = D(c, a[4]).ptr;
  L.ldphi = D(c, a[4]).ld;
  L.n = D(c, a[6]).ptr;
  L.ldn = D(c, a[6]).ld;
  L.dx = D(c, a[7]).ptr;
  L.lddx = D(c, a[7]).ld;
  L.t0 = D(c, a[8]).ptr;
  L.ldt0 = D(c, a[8]).ld;
  return run_loop(c, L, p->flags, &D(c, a[8]), nullptr, nullptr);
}

extern "C" int op2b_viscous_flux(op2b_ctx h, const op2b_arg* a, int32_t nargs,
                                 const op2b_visc_params* p) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!p || !(p->gamma > 1.0) || !(p->mu >= 0.0) || !(p->prandtl > 0.0) || !(p->diff >= 0.0))
    return c.fail(OP2B_EINVAL, "viscous_flux: need gamma > 1, mu >= 0, prandtl > 0, diff >= 0");
  static const Spec sp[6] = {{0, OP2B_READ, 20, 'P'},  {1, OP2B_READ, 20, 'P'},
                             {-1, OP2B_READ, 3, 'P'},  {-1, OP2B_READ, 3, 'P'},
                             {0, OP2B_INC, 6, 'D'},    {1, OP2B_INC, 6, 'D'}};
  Checked ck;
  int rc = check_args(c, "viscous_flux", a, nargs, sp, 6, &ck);
  if (rc) return rc;
  LoopLaunch L;
  L.loop = OP2B_LOOP_VISCOUS;
  L.prec = ck.prec;
  L.map = ck.map;
  L.N = ck.N;
  L.E = ck.E;
  L.m0 = c.maps[ck.map].dev;
  L.m1 = c.maps[ck.map].dev + ck.E;
  L.gamma = p->gamma;
  L.mu = p->mu;
  L.kappa = p->mu * p->gamma / ((p->gamma - 1.0) * p->prandtl);
  L.diff = p->diff;
  L.q = D(c, a[0]).ptr;
  L.ldq = D(c, a[0]).ld;
  L.n = D(c, a[2]).ptr;
  L.ldn = D(c, a[2]).ld;
  L.dx = D(c, a[3]).ptr;
  L.lddx = D(c, a[3]).ld;
  L.t0 = D(c, a[4]).ptr;
  L.ldt0 = D(c, a[4]).ld;
  return run_loop(c, L, p->flags, &D(c, a[4]), nullptr, nullptr);
}

extern "C" int op2b_spectral_radius(op2b_ctx h, const op2b_arg* a, int32_t nargs, double gamma,
                                    int32_t flags) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  static const Spec sp[5] = {{0, OP2B_READ, 6, 'D'}, {1, OP2B_READ, 6, 'D'}, {-1, OP2B_READ, 3, 'D'},
                             {0, OP2B_INC, 1, 'D'}, {1, OP2B_INC, 1, 'D'}};
  Checked ck;
  int rc = check_args(c, "spectral_radius", a, nargs, sp, 5, &ck);
  if (rc) return rc;
  if (!(gamma > 1.0)) return c.fail(OP2B_EINVAL, "spectral_radius: need gamma > 1");
  LoopLaunch L;
  L.loop = OP2B_LOOP_SPECTRAL;
  L.prec = OP2B_PREC_F64;
  L.map = ck.map;
  L.N = ck.N;
  L.E = ck.E;
  L.m0 = c.maps[ck.map].dev;
  L.m1 = c.maps[ck.map].dev + ck.E;
  L.gamma = gamma;
  // the edge loop reads each node's (u, a), formed once per node
  void* W = nullptr;
  if ((rc = c.need_aux((size_t)4 * std::max<int64_t>(ck.N, 1) * sizeof(double), &W))) return rc;
  if ((rc = node_wave_prims(&c, (const double*)D(c, a[0]).ptr, D(c, a[0]).ld, (double*)W, gamma,
                            ck.N)))
    return rc;
  L.q = W;
  L.ldq = ck.N;
  L.n = D(c, a[2]).ptr;
  L.ldn = D(c, a[2]).ld;
  L.t0 = D(c, a[3]).ptr;
  L.ldt0 = D(c, a[3]).ld;
  return run_loop(c, L, flags, &D(c, a[3]), nullptr, nullptr);
}

extern "C" int op2b_edge_flux_adjoint(op2b_ctx h, const op2b_arg* a, int32_t nargs,
                                      const op2b_flux_params* p) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!p || (p->order != 1 && p->order != 2)) return c.fail(OP2B_EINVAL, "edge_flux_adjoint: order must be 1 or 2");
  if (!(p->gamma > 1.0) || !(p->eps_lim > 0.0))
    return c.fail(OP2B_EINVAL, "edge_flux_adjoint: need gamma > 1, eps > 0");
  static const Spec s1[8] = {{0, OP2B_READ, 6, 'D'},  {1, OP2B_READ, 6, 'D'}, {0, OP2B_READ, 6, 'D'},
                             {1, OP2B_READ, 6, 'D'},  {-1, OP2B_READ, 3, 'D'}, {0, OP2B_INC, 6, 'D'},
                             {1, OP2B_INC, 6, 'D'},   {-1, OP2B_WRITE, 3, 'D'}};
  static const Spec s2[13] = {{0, OP2B_READ, 6, 'P'},   {1, OP2B_READ, 6, 'P'},  {0, OP2B_READ, 6, 'P'},
                              {1, OP2B_READ, 6, 'P'},   {0, OP2B_READ, 18, 'P'}, {1, OP2B_READ, 18, 'P'},
                              {-1, OP2B_READ, 3, 'P'},  {-1, OP2B_READ, 3, 'P'}, {0, OP2B_INC, 6, 'D'},
                              {1, OP2B_INC, 6, 'D'},    {0, OP2B_INC, 18, 'D'},  {1, OP2B_INC, 18, 'D'},
                              {-1, OP2B_WRITE, 3, 'D'}};
  Checked ck;
  int rc = p->order == 1 ? check_args(c, "edge_flux_adjoint", a, nargs, s1, 8, &ck)
                         : check_args(c, "edge_flux_adjoint", a, nargs, s2, 13, &ck);
  if (rc) return rc;
  if (ck.prec == OP2B_PREC_F32)
    return c.fail(OP2B_ETYPE, "edge_flux_adjoint: READ dats must be F64 (or FF for order 2)");
  LoopLaunch L;
  L.loop = p->order == 1 ? OP2B_LOOP_FLUX1_ADJ : OP2B_LOOP_FLUX2_ADJ;
  L.prec = ck.prec;
  L.order = p->order;
  L.map = ck.map;
  L.N = ck.N;
  L.E = ck.E;
  L.m0 = c.maps[ck.map].dev;
  L.m1 = c.maps[ck.map].dev + ck.E;
  L.gamma = p->gamma;
  L.eps = p->eps_lim;
  L.lam = D(c, a[0]).ptr;
  L.ldl = D(c, a[0]).ld;
  L.q = D(c, a[2]).ptr;
  L.ldq = D(c, a[2]).ld;
  const DatRec *z0, *z1 = nullptr, *dir;
  if (p->order == 1) {
    L.n = D(c, a[4]).ptr;
    L.ldn = D(c, a[4]).ld;
    z0 = &D(c, a[5]);
    dir = &D(c, a[7]);
  } else {
    L.G = D(c, a[4]).ptr;
    L.ldG = D(c, a[4]).ld;
    L.n = D(c, a[6]).ptr;
    L.ldn = D(c, a[6]).ld;
    L.dx = D(c, a[7]).ptr;
    L.lddx = D(c, a[7]).ld;
    z0 = &D(c, a[8]);
    z1 = &D(c, a[10]);
    dir = &D(c, a[12]);
    L.t1 = z1->ptr;
    L.ldt1 = z1->ld;
  }
  L.t0 = z0->ptr;
  L.ldt0 = z0->ld;
  L.direct = dir->ptr;
  L.lddirect = dir->ld;
  return run_loop(c, L, p->flags, z0, z1, dir);
}

extern "C" int op2b_green_gauss_adjoint(op2b_ctx h, const op2b_arg* a, int32_t nargs, int32_t flags) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  static const Spec sp[8] = {{0, OP2B_READ, 18, 'D'}, {1, OP2B_READ, 18, 'D'}, {0, OP2B_READ, 6, 'D'},
                             {1, OP2B_READ, 6, 'D'},  {-1, OP2B_READ, 3, 'D'}, {0, OP2B_INC, 6, 'D'},
                             {1, OP2B_INC, 6, 'D'},   {-1, OP2B_RW, 3, 'D'}};
  Checked ck;
  int rc = check_args(c, "green_gauss_adjoint", a, nargs, sp, 8, &ck);
  if (rc) return rc;
  LoopLaunch L;
  L.loop = OP2B_LOOP_GG_ADJ;
  L.prec = OP2B_PREC_F64;
  L.map = ck.map;
  L.N = ck.N;
  L.E = ck.E;
  L.m0 = c.maps[ck.map].dev;
  L.m1 = c.maps[ck.map].dev + ck.E;
  L.Gb = D(c, a[0]).ptr;
  L.ldGb = D(c, a[0]).ld;
  L.q = D(c, a[2]).ptr;
  L.ldq = D(c, a[2]).ld;
  L.n = D(c, a[4]).ptr;
  L.ldn = D(c, a[4]).ld;
  L.t0 = D(c, a[5]).ptr;
  L.ldt0 = D(c, a[5]).ld;
  L.direct = D(c, a[7]).ptr;
  L.lddirect = D(c, a[7]).ld;
  return run_loop(c, L, flags, &D(c, a[5]), nullptr, &D(c, a[7]));
}

extern "C" int op2b_green_gauss_tangent(op2b_ctx h, const op2b_arg* a, int32_t nargs, int32_t flags) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  static const Spec sp[8] = {{0, OP2B_READ, 6, 'D'},  {1, OP2B_READ, 6, 'D'},  {0, OP2B_READ, 6, 'D'},
                             {1, OP2B_READ, 6, 'D'},  {-1, OP2B_READ, 3, 'D'}, {-1, OP2B_READ, 3, 'D'},
                             {0, OP2B_INC, 18, 'D'},  {1, OP2B_INC, 18, 'D'}};
  Checked ck;
  int rc = check_args(c, "green_gauss_tangent", a, nargs, sp, 8, &ck);
  if (rc) return rc;
  LoopLaunch L;
  L.loop = OP2B_LOOP_GG_TAN;
  L.prec = OP2B_PREC_F64;
  L.map = ck.map;
  L.N = ck.N;
  L.E = ck.E;
  L.m0 = c.maps[ck.map].dev;
  L.m1 = c.maps[ck.map].dev + ck.E;
  L.q = D(c, a[0]).ptr;
  L.ldq = D(c, a[0]).ld;
  L.qd = D(c, a[2]).ptr;
  L.ldqd = D(c, a[2]).ld;
  L.n = D(c, a[4]).ptr;
  L.ldn = D(c, a[4]).ld;
  L.nd = D(c, a[5]).ptr;
  L.ldnd = D(c, a[5]).ld;
  L.t0 = D(c, a[6]).ptr;
  L.ldt0 = D(c, a[6]).ld;
  return run_loop(c, L, flags, &D(c, a[6]), nullptr, nullptr);
}

extern "C" int op2b_edge_flux_tangent(op2b_ctx h, const op2b_arg* a, int32_t nargs,
                                      const op2b_flux_params* p) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!p || (p->order != 1 && p->order != 2)) return c.fail(OP2B_EINVAL, "edge_flux_tangent: order must be 1 or 2");
  if (!(p->gamma > 1.0) || !(p->eps_lim > 0.0))
    return c.fail(OP2B_EINVAL, "edge_flux_tangent: need gamma > 1, eps > 0");
  static const Spec s1[8] = {{0, OP2B_READ, 6, 'D'},  {1, OP2B_READ, 6, 'D'},  {0, OP2B_READ, 6, 'D'},
                             {1, OP2B_READ, 6, 'D'},  {-1, OP2B_READ, 3, 'D'}, {-1, OP2B_READ, 3, 'D'},
                             {0, OP2B_INC, 6, 'D'},   {1, OP2B_INC, 6, 'D'}};
  static const Spec s2[13] = {{0, OP2B_READ, 6, 'P'},   {1, OP2B_READ, 6, 'P'},  {0, OP2B_READ, 6, 'P'},
                              {1, OP2B_READ, 6, 'P'},   {0, OP2B_READ, 18, 'P'}, {1, OP2B_READ, 18, 'P'},
                              {0, OP2B_READ, 18, 'P'},  {1, OP2B_READ, 18, 'P'}, {-1, OP2B_READ, 3, 'P'},
                              {-1, OP2B_READ, 3, 'P'},  {-1, OP2B_READ, 3, 'P'}, {0, OP2B_INC, 6, 'D'},
                              {1, OP2B_INC, 6, 'D'}};
  Checked ck;
  int rc = p->order == 1 ? check_args(c, "edge_flux_tangent", a, nargs, s1, 8, &ck)
                         : check_args(c, "edge_flux_tangent", a, nargs, s2, 13, &ck);
  if (rc) return rc;
  if (ck.prec == OP2B_PREC_F32)
    return c.fail(OP2B_ETYPE, "edge_flux_tangent: READ dats must be F64 (or FF for order 2)");
  LoopLaunch L;
  L.loop = p->order == 1 ? OP2B_LOOP_FLUX1_TAN : OP2B_LOOP_FLUX2_TAN;
  L.prec = ck.prec;
  L.order = p->order;
  L.map = ck.map;
  L.N = ck.N;
  L.E = ck.E;
  L.m0 = c.maps[ck.map].dev;
  L.m1 = c.maps[ck.map].dev + ck.E;
  L.gamma = p->gamma;
  L.eps = p->eps_lim;
  L.q = D(c, a[0]).ptr;
  L.ldq = D(c, a[0]).ld;
  L.qd = D(c, a[2]).ptr;
  L.ldqd = D(c, a[2]).ld;
  const op2b_arg* R;
  if (p->order == 1) {
    L.n = D(c, a[4]).ptr;
    L.ldn = D(c, a[4]).ld;
    L.nd = D(c, a[5]).ptr;
    L.ldnd = D(c, a[5]).ld;
    R = &a[6];
  } else {
    L.G = D(c, a[4]).ptr;
    L.ldG = D(c, a[4]).ld;
    L.Gd = D(c, a[6]).ptr;
    L.ldGd = D(c, a[6]).ld;
    L.n = D(c, a[8]).ptr;
    L.ldn = D(c, a[8]).ld;
    L.nd = D(c, a[9]).ptr;
    L.ldnd = D(c, a[9]).ld;
    L.dx = D(c, a[10]).ptr;
    L.lddx = D(c, a[10]).ld;
    R = &a[11];
  }
  L.t0 = D(c, *R).ptr;
  L.ldt0 = D(c, *R).ld;
  return run_loop(c, L, p->flags, &D(c, *R), nullptr, nullptr);
}

// ------------------------------------------------------------ node loops
static int node_dat(Ctx& c, op2b_dat d, int dim, int type, op2b_set set, const char* what) {
  if (!valid_dat(c, d)) return c.fail(OP2B_EINVAL, std::string(what) + ": bad dat");
  const DatRec& r = c.dats[d];
  if (set >= 0 && r.set != set) return c.fail(OP2B_ESET, std::string(what) + ": dats on different sets");
  if (dim > 0 && r.dim != dim) return c.fail(OP2B_EDIM, std::string(what) + ": wrong dim (" + r.name + ")");
  if (type >= 0 && r.type != type) return c.fail(OP2B_ETYPE, std::string(what) + ": wrong type (" + r.name + ")");
  return OP2B_OK;
}

static int grad_scale_impl(op2b_ctx h, op2b_dat G, op2b_dat V, const char* what) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  int rc;
  if ((rc = node_dat(c, G, 18, -1, -1, what))) return rc;
  const DatRec& g = c.dats[G];
  const bool fwd = std::string(what) == "grad_scale";
  if (g.type != OP2B_F64 && g.type != OP2B_F32 && !(fwd && g.type == OP2B_FF))
    return c.fail(OP2B_ETYPE, std::string(what) + (fwd ? ": G must be F64, F32 or FF" : ": G must be F64 or F32"));
  if ((rc = node_dat(c, V, 1, OP2B_F64, g.set, what))) return rc;
  return node_grad_scale(&c, g.ptr, g.type, g.ld, (const double*)c.dats[V].ptr, c.sets[g.set].size);
}

extern "C" int op2b_block_invert(op2b_ctx h, op2b_dat M, op2b_dat P) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  const char* w = "block_invert";
  int rc;
  if ((rc = node_dat(c, M, 36, OP2B_F64, -1, w))) return rc;
  if ((rc = node_dat(c, P, 36, OP2B_F64, c.dats[M].set, w))) return rc;
  if (M == P) return c.fail(OP2B_EINVAL, "block_invert: M and P must be distinct dats");
  const DatRec &m = c.dats[M], &p = c.dats[P];
  return node_block_invert(&c, (const double*)m.ptr, m.ld, (double*)p.ptr, p.ld, c.sets[m.set].size);
}

extern "C" int op2b_jacobi_from_sums(op2b_ctx h, op2b_dat q, op2b_dat S, op2b_dat M, op2b_dat P,
                                     double gamma) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  const char* w = "jacobi_from_sums";
  if (!(gamma > 1.0)) return c.fail(OP2B_EINVAL, "jacobi_from_sums: need gamma > 1");
  int rc;
  if ((rc = node_dat(c, q, 6, OP2B_F64, -1, w))) return rc;
  const op2b_set set = c.dats[q].set;
  if ((rc = node_dat(c, S, 4, OP2B_F64, set, w))) return rc;
  if (M >= 0 && (rc = node_dat(c, M, 36, OP2B_F64, set, w))) return rc;
  if (P >= 0 && (rc = node_dat(c, P, 36, OP2B_F64, set, w))) return rc;
  if (M >= 0 && M == P) return c.fail(OP2B_EINVAL, "jacobi_from_sums: M and P must be distinct dats");
  const DatRec &dq = c.dats[q], &ds = c.dats[S];
  double* mp = M >= 0 ? (double*)c.dats[M].ptr : nullptr;
  double* pp = P >= 0 ? (double*)c.dats[P].ptr : nullptr;
  return node_jacobi_from_sums(&c, (const double*)dq.ptr, dq.ld, (const double*)ds.ptr, ds.ld, mp,
                               M >= 0 ? c.dats[M].ld : 0, pp, P >= 0 ? c.dats[P].ld : 0, gamma,
                               c.sets[set].size);
}

extern "C" int op2b_node_update_precond(op2b_ctx h, op2b_dat q0, op2b_dat q, op2b_dat R,
                                        op2b_dat P, double alpha_sigma) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  const char* w = "node_update_precond";
  int rc;
  if ((rc = node_dat(c, q0, 6, OP2B_F64, -1, w))) return rc;
  const op2b_set set = c.dats[q0].set;
  if ((rc = node_dat(c, q, 6, OP2B_F64, set, w)) || (rc = node_dat(c, R, 6, OP2B_F64, set, w)) ||
      (rc = node_dat(c, P, 36, OP2B_F64, set, w)))
    return rc;
  if (R == q) return c.fail(OP2B_EINVAL, "node_update_precond: R and q must be distinct dats");
  const DatRec &a = c.dats[q0], &b = c.dats[q], &r = c.dats[R], &p = c.dats[P];
  return node_update_precond(&c, (const double*)a.ptr, a.ld, (double*)b.ptr, b.ld,
                             (const double*)r.ptr, r.ld, (const double*)p.ptr, p.ld, alpha_sigma,
                             c.sets[set].size);
}

extern "C" int op2b_grad_scale(op2b_ctx h, op2b_dat G, op2b_dat V) {
  return grad_scale_impl(h, G, V, "grad_scale");
}

extern "C" int op2b_grad_scale_adjoint(op2b_ctx h, op2b_dat Gb, op2b_dat V) {
  return grad_scale_impl(h, Gb, V, "grad_scale_adjoint");
}

// dats of a node gather over `map`: on the map's to-set, one type (F64/F32)
static int gather_dat(Ctx& c, op2b_dat d, int dim, int type, op2b_set set, const char* what) {
  if (!valid_dat(c, d)) return c.fail(OP2B_EINVAL, std::string(what) + ": bad dat");
  const DatRec& r = c.dats[d];
  if (r.set != set) return c.fail(OP2B_ESET, std::string(what) + ": " + r.name + " is on the wrong set");
  if (r.dim != dim) return c.fail(OP2B_EDIM, std::string(what) + ": wrong dim (" + r.name + ")");
  if (r.type != type) return c.fail(OP2B_ETYPE, std::string(what) + ": mixed types (" + r.name + ")");
  return OP2B_OK;
}

extern "C" int op2b_node_minmax(op2b_ctx h, op2b_map map, op2b_dat q, op2b_dat qmin, op2b_dat qmax) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  const char* w = "node_minmax";
  if (!valid_map(c, map) || c.maps[map].arity != 2) return c.fail(OP2B_EINVAL, "node_minmax: need an arity-2 map");
  if (!valid_dat(c, q)) return c.fail(OP2B_EINVAL, "node_minmax: bad dat");
  const int type = c.dats[q].type;
  if (type != OP2B_F64 && type != OP2B_F32 && type != OP2B_FF)
    return c.fail(OP2B_ETYPE, "node_minmax: F64, F32 or FF dats");
  const MapRec& m = c.maps[map];
  int rc;
  if ((rc = gather_dat(c, q, 6, type, m.to, w)) || (rc = gather_dat(c, qmin, 6, type, m.to, w)) ||
      (rc = gather_dat(c, qmax, 6, type, m.to, w)))
    return rc;
  if (qmin == q || qmax == q || qmin == qmax)
    return c.fail(OP2B_EINVAL, "node_minmax: q, qmin and qmax must be distinct dats");
  DevSegPlan* sp = nullptr;
  if ((rc = c.seg_plan(map, &sp))) return rc;
  const int64_t E = c.sets[m.from].size;
  return node_minmax(&c, *sp, m.dev, m.dev + E, type, c.dats[q].ptr, c.dats[q].ld, c.dats[qmin].ptr,
                     c.dats[qmin].ld, c.dats[qmax].ptr, c.dats[qmax].ld, c.sets[m.to].size);
}

extern "C" int op2b_node_limiter(op2b_ctx h, op2b_map map, int32_t kind, double eps2, op2b_dat q,
                                 op2b_dat G, op2b_dat dx, op2b_dat qmin, op2b_dat qmax, op2b_dat phi) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  const char* w = "node_limiter";
  if (kind != OP2B_LIM_BARTH_JESPERSEN && kind != OP2B_LIM_VENKATAKRISHNAN)
    return c.fail(OP2B_EINVAL, "node_limiter: unknown limiter");
  if (!(eps2 >= 0.0)) return c.fail(OP2B_EINVAL, "node_limiter: eps2 must be >= 0");
  if (!valid_map(c, map) || c.maps[map].arity != 2) return c.fail(OP2B_EINVAL, "node_limiter: need an arity-2 map");
  if (!valid_dat(c, q)) return c.fail(OP2B_EINVAL, "node_limiter: bad dat");
  const int type = c.dats[q].type;
  if (type != OP2B_F64 && type != OP2B_F32 && type != OP2B_FF)
    return c.fail(OP2B_ETYPE, "node_limiter: F64, F32 or FF dats");
  const MapRec& m = c.maps[map];
  int rc;
  if ((rc = gather_dat(c, q, 6, type, m.to, w)) || (rc = gather_dat(c, G, 18, type, m.to, w)) ||
      (rc = gather_dat(c, qmin, 6, type, m.to, w)) || (rc = gather_dat(c, qmax, 6, type, m.to, w)) ||
      (rc = gather_dat(c, phi, 6, type, m.to, w)) || (rc = gather_dat(c, dx, 3, type, m.from, w)))
    return rc;
  if (phi == q || phi == qmin || phi == qmax)
    return c.fail(OP2B_EINVAL, "node_limiter: phi must not be an input dat");
  DevSegPlan* sp = nullptr;
  if ((rc = c.seg_plan(map, &sp))) return rc;
  LimArgs la;
  la.q = c.dats[q].ptr;
  la.ldq = c.dats[q].ld;
  la.G = c.dats[G].ptr;
  la.ldG = c.dats[G].ld;
  la.dx = c.dats[dx].ptr;
  la.lddx = c.dats[dx].ld;
  la.qmin = c.dats[qmin].ptr;
  la.ldmin = c.dats[qmin].ld;
  la.qmax = c.dats[qmax].ptr;
  la.ldmax = c.dats[qmax].ld;
  la.phi = c.dats[phi].ptr;
  la.ldphi = c.dats[phi].ld;
  la.eps2 = eps2;
  return node_limiter(&c, *sp, kind, type, la, c.sets[m.to].size);
}

extern "C" int op2b_viscous_prims(op2b_ctx h, op2b_dat q, op2b_dat G, op2b_dat W, double gamma) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  int rc;
  if ((rc = node_dat(c, q, 6, -1, -1, "viscous_prims"))) return rc;
  const DatRec& rq = c.dats[q];
  if (rq.type != OP2B_F64 && rq.type != OP2B_F32 && rq.type != OP2B_FF)
    return c.fail(OP2B_ETYPE, "viscous_prims: q must be F64, F32 or FF");
  if ((rc = node_dat(c, G, 18, rq.type, rq.set, "viscous_prims")) ||
      (rc = node_dat(c, W, 20, rq.type, rq.set, "viscous_prims")))
    return rc;
  if (!(gamma > 1.0)) return c.fail(OP2B_EINVAL, "viscous_prims: need gamma > 1");
  const DatRec &rg = c.dats[G], &rw = c.dats[W];
  return node_viscous_prims(&c, rq.ptr, rq.ld, rg.ptr, rg.ld, rw.ptr, rw.ld, rq.type, gamma,
                            c.sets[rq.set].size);
}

extern "C" int op2b_time_step(op2b_ctx h, op2b_dat V, op2b_dat lam, double cfl, op2b_dat dt) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  int rc;
  if ((rc = node_dat(c, V, 1, OP2B_F64, -1, "time_step"))) return rc;
  op2b_set s = c.dats[V].set;
  if ((rc = node_dat(c, lam, 1, OP2B_F64, s, "time_step")) || (rc = node_dat(c, dt, 1, OP2B_F64, s, "time_step")))
    return rc;
  if (!(cfl > 0.0)) return c.fail(OP2B_EINVAL, "time_step: cfl must be positive");
  return node_time_step(&c, (const double*)c.dats[V].ptr, (const double*)c.dats[lam].ptr, cfl,
                        (double*)c.dats[dt].ptr, c.sets[s].size);
}

extern "C" int op2b_node_update(op2b_ctx h, op2b_dat q0, op2b_dat q, op2b_dat R, op2b_dat V, op2b_dat dt,
                                double alpha, op2b_dat q32) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  int rc;
  if ((rc = node_dat(c, q0, 6, OP2B_F64, -1, "node_update"))) return rc;
  op2b_set s = c.dats[q0].set;
  if ((rc = node_dat(c, q, 6, OP2B_F64, s, "node_update")) || (rc = node_dat(c, R, 6, OP2B_F64, s, "node_update")) ||
      (rc = node_dat(c, V, 1, OP2B_F64, s, "node_update")) || (rc = node_dat(c, dt, 1, OP2B_F64, s, "node_update")))
    return rc;
  void* psh = nullptr;
  int tsh = OP2B_F32;
  int64_t ldsh = 0;
  if (q32 >= 0) {
    if ((rc = node_dat(c, q32, 6, -1, s, "node_update"))) return rc;
    tsh = c.dats[q32].type;
    if (tsh != OP2B_F32 && tsh != OP2B_FF)
      return c.fail(OP2B_ETYPE, "node_update: the shadow of q must be F32 or FF");
    psh = c.dats[q32].ptr;
    ldsh = c.dats[q32].ld;
  }
  return node_update(&c, (const double*)c.dats[q0].ptr, c.dats[q0].ld, (double*)c.dats[q].ptr, c.dats[q].ld,
                     (const double*)c.dats[R].ptr, c.dats[R].ld, (const double*)c.dats[V].ptr,
                     (const double*)c.dats[dt].ptr, alpha, psh, tsh, ldsh, c.sets[s].size);
}

extern "C" int op2b_node_update_adjoint(op2b_ctx h, op2b_dat sbar, op2b_dat qbar, op2b_dat lam,
                                        op2b_dat V, op2b_dat dt, double alpha) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  int rc;
  const char* w = "node_update_adjoint";
  if ((rc = node_dat(c, sbar, 6, OP2B_F64, -1, w))) return rc;
  op2b_set s = c.dats[sbar].set;
  if ((rc = node_dat(c, qbar, 6, OP2B_F64, s, w)) || (rc = node_dat(c, lam, 6, OP2B_F64, s, w)) ||
      (rc = node_dat(c, V, 1, OP2B_F64, s, w)) || (rc = node_dat(c, dt, 1, OP2B_F64, s, w)))
    return rc;
  if (sbar == qbar || sbar == lam || qbar == lam)
    return c.fail(OP2B_EINVAL, "node_update_adjoint: sbar, qbar and lam must be distinct dats");
  return node_update_adjoint(&c, (const double*)c.dats[sbar].ptr, c.dats[sbar].ld,
                             (double*)c.dats[qbar].ptr, c.dats[qbar].ld, (double*)c.dats[lam].ptr,
                             c.dats[lam].ld, (const double*)c.dats[V].ptr,
                             (const double*)c.dats[dt].ptr, alpha, c.sets[s].size);
}

extern "C" int op2b_dat_axpy(op2b_ctx h, op2b_dat y, double a, op2b_dat x) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!valid_dat(c, y) || !valid_dat(c, x)) return c.fail(OP2B_EINVAL, "dat_axpy: bad dat");
  const DatRec &dy = c.dats[y], &dx = c.dats[x];
  if (dy.set != dx.set) return c.fail(OP2B_ESET, "dat_axpy: dats on different sets");
  if (dy.dim != dx.dim) return c.fail(OP2B_EDIM, "dat_axpy: dims differ");
  if (dy.type != OP2B_F64 || dx.type != OP2B_F64) return c.fail(OP2B_ETYPE, "dat_axpy: F64 dats only");
  return node_axpy(&c, (double*)dy.ptr, dy.ld, a, (const double*)dx.ptr, dx.ld, dy.dim,
                   c.sets[dy.set].size);
}

extern "C" int op2b_dat_fill(op2b_ctx h, op2b_dat d, double value) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!valid_dat(c, d)) return c.fail(OP2B_EINVAL, "dat_fill: bad dat");
  const DatRec& r = c.dats[d];
  return node_fill(&c, r.ptr, r.type, r.ld, r.dim, c.sets[r.set].size, value);
}

extern "C" int op2b_dat_reduce(op2b_ctx h, op2b_dat d, int32_t op, double* out_dev) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!valid_dat(c, d)) return c.fail(OP2B_EINVAL, "dat_reduce: bad dat");
  const DatRec& r = c.dats[d];
  if (r.type != OP2B_F64) return c.fail(OP2B_ETYPE, "dat_reduce: F64 dats only");
  if (!out_dev) return c.fail(OP2B_EINVAL, "dat_reduce: null output");
  if (op < OP2B_RED_SUM || op > OP2B_RED_MIN) return c.fail(OP2B_EINVAL, "dat_reduce: unknown operation");
  return node_reduce(&c, (const double*)r.ptr, r.ld, r.dim, c.sets[r.set].size, op, out_dev);
}

extern "C" int op2b_dat_copy(op2b_ctx h, op2b_dat dst, op2b_dat src) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!valid_dat(c, dst) || !valid_dat(c, src)) return c.fail(OP2B_EINVAL, "dat_copy: bad dat");
  const DatRec &d = c.dats[dst], &s = c.dats[src];
  if (d.set != s.set) return c.fail(OP2B_ESET, "dat_copy: dats on different sets");
  if (d.dim != s.dim) return c.fail(OP2B_EDIM, "dat_copy: dims differ");
  return node_copy(&c, d.ptr, d.type, d.ld, s.ptr, s.type, s.ld, d.dim, c.sets[d.set].size);
}

// ------------------------------------------------ planner and autotuner
extern "C" int op2b_set_strategy(op2b_ctx h, int32_t loop, int32_t prec, int32_t strategy, int32_t block,
                                 int32_t part, int32_t staged) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (loop < 0 || loop >= OP2B_NUM_LOOPS || (prec < 0 || prec >= OP2B_NUM_PREC))
    return c.fail(OP2B_EINVAL, "set_strategy: bad loop or precision");
  if (strategy < OP2B_STRAT_AUTO || strategy > OP2B_STRAT_HYBRID)
    return c.fail(OP2B_EINVAL, "set_strategy: bad strategy");
  if (strategy == OP2B_STRAT_HYBRID && (loop != OP2B_LOOP_GREEN_GAUSS || prec != OP2B_PREC_F64))
    return c.fail(OP2B_EINVAL, "set_strategy: the hybrid strategy serves the FP64 Green-Gauss loop only");
  if (strategy == OP2B_STRAT_GATHER &&
      (loop == OP2B_LOOP_FLUX1_ADJ || loop == OP2B_LOOP_FLUX2_ADJ || loop == OP2B_LOOP_GG_ADJ))
    return c.fail(OP2B_EINVAL, "set_strategy: the gather strategy needs a loop without per-edge outputs");
  if (block != 0 && (block < 32 || block > 1024 || block % 32))
    return c.fail(OP2B_EINVAL, "set_strategy: block must be a multiple of 32 in [32, 1024]");
  if (part != 0 && (part < 64 || part > 8192)) return c.fail(OP2B_EINVAL, "set_strategy: part must be in [64, 8192]");
  Strategy s;
  s.strategy = strategy;
  s.block = block ? block : 256;
  s.part = part ? part : 512;
  s.staged = staged ? 1 : 0;
  c.strat[loop][prec] = s;
  return OP2B_OK;
}

extern "C" int op2b_set_tune_deadline(op2b_ctx h, double ms) {
  CTX_CHECK(h);
  if (!(ms > 0.0)) return h->c.fail(OP2B_EINVAL, "set_tune_deadline: must be positive");
  h->c.tune_deadline_ms = ms;
  return OP2B_OK;
}

extern "C" int op2b_save_tuning(op2b_ctx h, const char* path) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!path) return c.fail(OP2B_EINVAL, "save_tuning: null path");
  std::ofstream f(path);
  if (!f) return c.fail(OP2B_EINVAL, std::string("save_tuning: cannot write ") + path);
  f << "{\n";
  size_t k = 0;
  for (auto& kv : c.tuned) {
    const Strategy& s = kv.second;
    char line[512];
    snprintf(line, sizeof line,
             "  \"%s\": {\"strategy\": %d, \"block\": %d, \"part\": %d, \"staged\": %d, \"ms\": %.6f",
             kv.first.c_str(), s.strategy, s.block, s.part, s.staged, s.tuned_ms);
    f << line;
    if (!s.timings.empty()) f << ", \"candidates\": [" << s.timings << "]";
    f << "}" << (++k < c.tuned.size() ? "," : "") << "\n";
  }
  f << "}\n";
  return f.good() ? OP2B_OK : c.fail(OP2B_EINVAL, "save_tuning: write failed");
}

extern "C" int op2b_load_tuning(op2b_ctx h, const char* path) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (!path) return c.fail(OP2B_EINVAL, "load_tuning: null path");
  std::ifstream f(path);
  if (!f) return c.fail(OP2B_EINVAL, std::string("load_tuning: cannot read ") + path);
  std::string line;
  while (std::getline(f, line)) {
    char key[256];
    Strategy s;
    if (sscanf(line.c_str(),
               " \"%255[^\"]\": {\"strategy\": %d, \"block\": %d, \"part\": %d, \"staged\": %d, \"ms\": %lf}",
               key, &s.strategy, &s.block, &s.part, &s.staged, &s.tuned_ms) == 6) {
      if (s.strategy < OP2B_STRAT_ATOMIC || s.strategy == OP2B_STRAT_AUTO_DET ||
          s.strategy > OP2B_STRAT_HYBRID)
        return c.fail(OP2B_EINVAL, "load_tuning: bad strategy in table");
      c.tuned[key] = s;
    }
  }
  return OP2B_OK;
}

extern "C" int op2b_plan_stats(op2b_ctx h, int32_t loop, int32_t prec, op2b_map map, op2b_plan_stats_t* out) {
  CTX_CHECK(h);
  Ctx& c = h->c;
  if (loop < 0 || loop >= OP2B_NUM_LOOPS || (prec < 0 || prec >= OP2B_NUM_PREC) || !out || !valid_map(c, map))
    return c.fail(OP2B_EINVAL, "plan_stats: bad loop, precision, map or output");
  const Strategy& s = c.strat[loop][prec];
  memset(out, 0, sizeof *out);
  out->strategy = s.strategy;
  out->block = s.block;
  out->part = s.part;
  out->staged = s.staged;
  out->tuned_ms = s.tuned_ms;
  DevBlockPlan* bp = nullptr;
  int rc = c.block_plan(map, s.part, &bp);
  if (rc == OP2B_EPLAN) {  // no colouring at this partition size: say so
    out->nblocks = -1;
    out->ncolours = -1;
    return OP2B_OK;
  }
  if (rc) return rc;
  out->nblocks = bp->nblocks;
  out->ncolours = bp->ncolours;
  out->min_blocks_per_colour = bp->min_per_colour;
  out->max_blocks_per_colour = bp->max_per_colour;
  out->max_unique_nodes = bp->max_unique;
  out->avg_unique_nodes = bp->avg_unique;
  return OP2B_OK;
}

// ---------------------------------------------------- host-only planners
extern "C" int op2b_host_rcm(int64_t N, int64_t E, const int32_t* edge, int32_t* new_of_old) {
  if (N < 0 || E < 0 || (E > 0 && !edge) || (N > 0 && !new_of_old)) return OP2B_EINVAL;
  return op2b::rcm(N, E, edge, new_of_old) ? OP2B_OK : OP2B_EINVAL;
}

extern "C" int op2b_host_renumber(int64_t N, int64_t E, const int32_t* edge, int32_t method, uint64_t seed,
                                  int32_t* new_of_old, int64_t* order) {
  if (N < 0 || E < 0 || (E > 0 && !edge) || (N > 0 && !new_of_old) || (E > 0 && !order)) return OP2B_EINVAL;
  for (int64_t e = 0; e < 2 * E; e++)
    if (edge[e] < 0 || edge[e] >= N) return OP2B_EINVAL;
  if (method == 0) {
    for (int64_t i = 0; i < N; i++) new_of_old[i] = (int32_t)i;
  } else if (method == 1) {
    op2b::random_perm(N, seed, new_of_old);
  } else if (method == 2) {
    if (!op2b::rcm(N, E, edge, new_of_old)) return OP2B_EINVAL;
  } else {
    return OP2B_EINVAL;
  }
  op2b::edge_order(N, E, edge, new_of_old, order);
  return OP2B_OK;
}

extern "C" int op2b_host_colour_blocks(int64_t N, int64_t E, const int32_t* edge, int32_t part,
                                       int32_t* block_colour, int64_t* ncolours) {
  if (N < 0 || E < 0 || (E > 0 && (!edge || !block_colour)) || !ncolours || part < 1 || part > 32767)
    return OP2B_EINVAL;
  std::vector<int32_t> m0(E), m1(E);
  for (int64_t e = 0; e < E; e++) {
    m0[e] = edge[2 * e];
    m1[e] = edge[2 * e + 1];
    if (m0[e] < 0 || m0[e] >= N || m1[e] < 0 || m1[e] >= N) return OP2B_EINVAL;
  }
  op2b::BlockPlan p;
  std::string err;
  if (!op2b::build_block_plan(N, E, m0.data(), m1.data(), part, &p, &err)) return OP2B_EPLAN;
  std::copy(p.colour.begin(), p.colour.end(), block_colour);
  *ncolours = p.ncolours;
  return OP2B_OK;
}

extern "C" int op2b_host_rcb(int64_t N, const double* xyz, int32_t leaf, int32_t* new_of_old) {
  if (N < 0 || leaf < 1 || (N > 0 && (!xyz || !new_of_old))) return OP2B_EINVAL;
  return op2b::rcb(N, xyz, leaf, new_of_old) ? OP2B_OK : OP2B_EINVAL;
}

extern "C" int op2b_host_node_csr(int64_t N, int64_t E, const int32_t* edge, int64_t* rowptr, int64_t* ends) {
  if (N < 0 || E < 0 || (E > 0 && (!edge || !ends)) || !rowptr) return OP2B_EINVAL;
  std::vector<int32_t> m0(E), m1(E);
  for (int64_t e = 0; e < E; e++) {
    m0[e] = edge[2 * e];
    m1[e] = edge[2 * e + 1];
    if (m0[e] < 0 || m0[e] >= N || m1[e] < 0 || m1[e] >= N) return OP2B_EINVAL;
  }
  std::vector<int64_t> rp;
  std::vector<int32_t> en;
  op2b::node_csr(N, E, m0.data(), m1.data(), &rp, &en);
  std::copy(rp.begin(), rp.end(), rowptr);
  for (int64_t t = 0; t < 2 * E; t++) ends[t] = en[t];
  return OP2B_OK;
}
