// op2b_edge_flux1_noalloc: the first-order flux edge loop with the sorted
// segmented strategy, for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc: a solver embedded in a host program
// whose device memory is one arena owned by someone else, a real-time loop
// that must not allocate between time steps, or code running where a new
// allocation is not allowed.  The context entry points allocate plans and a
// growable scratch buffer on demand, so they cannot serve these callers.
// This entry point takes every input and the output from the caller and
// keeps its per-edge scratch in a fixed array compiled into the library.
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "edge_loops.cuh"
#include "internal.h"

namespace {

// Largest edge set the entry point accepts.
constexpr int64_t kMaxEdges = OP2B_NOALLOC_MAX_EDGES;

// Per-edge fluxes, 6 doubles per edge, edge-major (6 x kMaxEdges doubles =
// 12 MiB).  A GPU reserves this array when the module holding it is loaded
// there -- at the first call on that device under lazy module loading (the
// CUDA default), at context creation under eager loading -- and keeps it
// until the process exits.
static __device__ __align__(256) double g_flux_scratch[6 * kMaxEdges];

std::mutex g_mu;
std::vector<double*> g_scratch_addr;  // device address per device id

// The array's device address on the current device.  In host code the
// symbol g_flux_scratch is only a stand-in, so the address is asked for
// once per device, with that device current, and cached.
int scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if ((int)g_scratch_addr.size() <= dev) g_scratch_addr.resize(dev + 1, nullptr);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_flux_scratch);
    if (e != cudaSuccess || !p) {
      op2b::set_thread_error(std::string("edge_flux1_noalloc: cudaGetSymbolAddress failed: ") +
                             cudaGetErrorString(e));
      return OP2B_ECUDA;
    }
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return OP2B_OK;
}

__global__ void k_zero_rows(double* __restrict__ R, int64_t ld, int dim, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < dim; k++) R[k * ld + i] = 0.0;
}

int fail(int code, const std::string& msg) {
  op2b::set_thread_error("edge_flux1_noalloc: " + msg);
  return code;
}

// Do the byte ranges [a, a + na) and [b, b + nb) overlap?
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  if (!a || !b || na == 0 || nb == 0) return false;
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

// bytes spanned by `dim` rows of `n` doubles at leading dimension ld
size_t span(int dim, int64_t ld, int64_t n) {
  return n > 0 ? ((size_t)(dim - 1) * (size_t)ld + (size_t)n) * sizeof(double) : 0;
}

}  // namespace

extern "C" int op2b_edge_flux1_noalloc(const double* q, int64_t ldq, const double* n, int64_t ldn,
                                       const int32_t* edge_first, const int32_t* edge_second,
                                       const int64_t* rowptr, const int32_t* ends, int64_t N,
                                       int64_t E, double gamma, double* R, int64_t ldR,
                                       void* stream) {
  if (N < 0 || E < 0) return fail(OP2B_EINVAL, "negative size");
  if (E > kMaxEdges)
    return fail(OP2B_ERANGE, "edge set of " + std::to_string(E) + " edges exceeds the limit of " +
                                 std::to_string(kMaxEdges));
  if (N >= ((int64_t)1 << 31) - 1) return fail(OP2B_ERANGE, "node set too large");
  if (!(gamma > 1.0)) return fail(OP2B_EINVAL, "gamma must exceed 1");
  if (ldq < N || ldR < N || ldn < E) return fail(OP2B_EINVAL, "leading dimension below the set size");
  if (N > 0 && (!q || !R || !rowptr)) return fail(OP2B_EINVAL, "null node pointer");
  if (E > 0 && (!n || !edge_first || !edge_second || !ends)) return fail(OP2B_EINVAL, "null edge pointer");
  // R is zeroed before the edge phase reads q and n: an output that shares
  // memory with an input would be read after it was overwritten
  const size_t bR = span(6, ldR, N);
  if (overlaps(R, bR, q, span(6, ldq, N)) || overlaps(R, bR, n, span(3, ldn, E)))
    return fail(OP2B_EINVAL, "R overlaps q or n");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(OP2B_ECUDA, "no current CUDA device");
  double* scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int block = 256;
  const int64_t cap = (int64_t)std::max(sms, 1) * 32;
  if (N > 0) {
    // R receives the sum: the node phase adds into it, so it starts at zero
    unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + block - 1) / block, cap));
    k_zero_rows<<<g, block, 0, st>>>(R, ldR, 6, N);
  }
  static_assert(op2b::ebuf_stride<op2b::BodyFlux1<double>>() == 6, "scratch holds 6 per edge");
  if (E > 0) {
    // the edge phase writes all 6 x E scratch entries that the node phase
    // reads, so the array's previous contents never matter
    op2b::Gas<double> gas{gamma, gamma - 1.0, 1e-12, 2e-12};
    op2b::BodyFlux1<double> body{q, ldq, n, ldn, gas};
    unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((E + block - 1) / block, cap));
    op2b::k_seg_edges<op2b::BodyFlux1<double>><<<g, block, 0, st>>>(body, edge_first, edge_second,
                                                                    E, scratch);
    op2b::Targets<double, 6> tg{R, ldR, R, ldR};
    unsigned gn = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + block - 1) / block, cap));
    op2b::k_seg_nodes<double, double, 6, op2b::MODE_ANTI, 6>
        <<<gn, block, 0, st>>>(rowptr, ends, N, E, scratch, tg);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(OP2B_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return OP2B_OK;
}
