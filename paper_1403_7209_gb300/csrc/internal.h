// Internal state of an op2b context and the launch interface between the
// C ABI (api.cu) and the per-loop kernel instantiations (loops_*.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/op2b.h"
#include "host_plan.h"

namespace op2b {

struct SetRec {
  int64_t size;
  std::string name;
};

struct MapRec {
  op2b_set from, to;
  int32_t arity;
  std::vector<int32_t> host;  // element-major copy
  int32_t* dev = nullptr;     // SoA on the device: entry k at dev[k*from+e]
  std::string name;
  uint64_t version = 0;       // bumped on renumbering (invalidates plans)
};

struct DatRec {
  op2b_set set;
  int32_t dim, type;
  void* ptr;
  int64_t ld;
  std::string name;
};

// device copy of a BlockPlan
struct DevBlockPlan {
  uint64_t map_version = ~0ull;
  int32_t part = 0;
  int64_t nblocks = 0;
  int32_t ncolours = 0;
  int64_t max_unique = 0;
  double avg_unique = 0.0;
  std::vector<int64_t> coff;
  int64_t min_per_colour = 0, max_per_colour = 0;
  int32_t *bn_off = nullptr, *bnodes = nullptr, *lrow = nullptr,
          *cblocks = nullptr;
  uint32_t* eloc = nullptr;
  uint16_t* lent = nullptr;
};

struct DevSegPlan {
  uint64_t map_version = ~0ull;
  int64_t* rowptr = nullptr;
  int32_t* ends = nullptr;
};

struct DevOwnPlan {
  uint64_t map_version = ~0ull;
  int64_t* ptr = nullptr;  // N+1
  int32_t* idx = nullptr;  // E edges, grouped by lower-numbered end
};

// Packed FP32 records of the fused mixed-precision stage (stage32.cu), per
// map: the edge ends' adjacency, sliced-ELL (per 32-node slice: width = the
// slice's largest degree, ell_off = 32 x the widths' prefix sums; per slot
// the other node's id with +-n/2 for the Green-Gauss pass, with the signed
// edge geometry for the flux pass) and two node-record buffers (q then G,
// 24 floats per node), the current one holding the state's FP32 copy.
// Where the node-block staging plan fits (staged), the adjacency sliced-ELL
// with the other node's local id in its block's neighbourhood and the
// edges' geometry (n, dx; 32 bytes per edge).
struct Stage32Plan {
  uint64_t map_version = ~0ull;
  int64_t N = 0, E = 0;
  int64_t nell = 0;
  int64_t* ell_off = nullptr;  // per slice + 1
  int4* adjn_l = nullptr;      // per slot: {j, +-n/2}
  float4* ende = nullptr;      // per slot, two words: {j, s n}, {s dx, 0}
  float4* geo = nullptr;       // staged passes only
  float* rec[2] = {nullptr, nullptr};
  int cur = 0;
  // the dats the geometry and the records were packed from
  const void *n_src = nullptr, *dx_src = nullptr, *q_src = nullptr;
  int n_type = -1, dx_type = -1;
  // staging plan (blocks of B nodes and their neighbourhoods), built on
  // the first call that asks for the staged passes
  bool staging_planned = false;
  bool staged = false;
  int32_t B = 0;
  int64_t nblocks = 0, max_unique = 0, nslots = 0;
  int64_t* uoff = nullptr;      // nblocks+1
  int32_t* uniq = nullptr;      // neighbourhood node ids
  int32_t* lother = nullptr;    // per end (node-sorted): the other node's local id
  int64_t* sell_off = nullptr;  // per 32-node slice + 1
  int32_t* sell_end = nullptr;  // per slot: node-sorted end index or -1
  int4* adjn_s = nullptr;       // sliced-ELL adjacency of the staged passes
  int2* adje_s = nullptr;
};

struct Strategy {
  int32_t strategy = OP2B_STRAT_ATOMIC;
  int32_t block = 256;
  int32_t part = 512;
  int32_t staged = 0;
  double tuned_ms = 0.0;
  std::string timings;  // every candidate the tuner ran, "[strategy, block, part, staged, ms], ..."
};

// Everything a loop launch needs; pointers are device pointers.
struct LoopLaunch {
  int loop = 0, prec = 0, order = 1;
  int flags = 0;  // the call's OP2B_* loop flags
  int map = -1;  // the edge->node map (plan lookup)
  int64_t N = 0, E = 0;
  const int32_t* m0 = nullptr;  // first end of every edge
  const int32_t* m1 = nullptr;  // second end
  // READ data
  const void *q = nullptr, *G = nullptr, *n = nullptr, *dx = nullptr,
             *lam = nullptr, *Gb = nullptr;
  int64_t ldq = 0, ldG = 0, ldn = 0, lddx = 0, ldl = 0, ldGb = 0;
  // tangent directions
  const void *qd = nullptr, *Gd = nullptr, *nd = nullptr;
  int64_t ldqd = 0, ldGd = 0, ldnd = 0;
  // INC targets (first and second dat) and direct output
  void *t0 = nullptr, *t1 = nullptr, *direct = nullptr;
  int64_t ldt0 = 0, ldt1 = 0, lddirect = 0;
  double gamma = 1.4, eps = 1e-12;
  double mu = 0.0, kappa = 0.0, diff = 0.0;  // viscous flux coefficients
  const void* phi = nullptr;                  // node limiter (FLUX2_PHI)
  int64_t ldphi = 0;
  // Green-Gauss: node volumes; when set, the sums are divided by them (the
  // gradient scaling, fused into the node gather, else run after the loop)
  const double* vol = nullptr;
};

// Arguments of the node limiter (device pointers, leading dimensions).
struct LimArgs {
  const void *q = nullptr, *G = nullptr, *dx = nullptr, *qmin = nullptr, *qmax = nullptr;
  void* phi = nullptr;
  int64_t ldq = 0, ldG = 0, lddx = 0, ldmin = 0, ldmax = 0, ldphi = 0;
  double eps2 = 0.0;
};

struct Ctx;

// Text returned by op2b_last_error(NULL) on this thread (set by entry points
// that have no context).
void set_thread_error(const std::string& msg);

// Run one edge loop with strategy s (plans and scratch taken from ctx).
// loops_f64.cu: GREEN_GAUSS, FLUX1, FLUX2, SPECTRAL in FP64;
// loops_f32.cu: GREEN_GAUSS, FLUX1, FLUX2 with FP32 arithmetic;
// loops_adj.cu: FLUX1_ADJ, FLUX2_ADJ, GG_ADJ and the tangents FLUX1_TAN,
// FLUX2_TAN, GG_TAN.
int launch_f64(Ctx* c, const LoopLaunch& L, const Strategy& s);
int launch_f32(Ctx* c, const LoopLaunch& L, const Strategy& s);
// loops_ff.cu: FLUX2 with float-float arithmetic (float-float READ dats)
int launch_ff(Ctx* c, const LoopLaunch& L, const Strategy& s);
int launch_adj(Ctx* c, const LoopLaunch& L, const Strategy& s);
// loops_lim.cu: FLUX2_PHI (FP64 or FP32) and the node min/max and limiter
int launch_lim(Ctx* c, const LoopLaunch& L, const Strategy& s);
// loops_visc.cu: VISCOUS (FP64 or FP32 arithmetic) and its node pass
int launch_visc(Ctx* c, const LoopLaunch& L, const Strategy& s);
int node_viscous_prims(Ctx* c, const void* q, int64_t ldq, const void* G, int64_t ldG,
                       void* W, int64_t ldW, int type, double gamma, int64_t N);
int node_minmax(Ctx* c, const DevSegPlan& sp, const int32_t* m0, const int32_t* m1, int type,
                const void* q, int64_t ldq, void* qmin, int64_t ldmin, void* qmax, int64_t ldmax,
                int64_t N);
int node_limiter(Ctx* c, const DevSegPlan& sp, int kind, int type, const LimArgs& a, int64_t N);

// Frees every fused-stage plan of the context (stage32.cu).
int stage32_free_all(Ctx& c);

// Direct node loops (node_loops.cu).
int node_grad_scale(Ctx* c, void* G, int type, int64_t ldG, const double* V,
                    int64_t N);
int node_block_invert(Ctx* c, const double* M, int64_t ldM, double* P, int64_t ldP, int64_t N);
// W = (u_x, u_y, u_z, a) per node from q (SoA, ld N), a = sqrt(gamma p / rho)
int node_wave_prims(Ctx* c, const double* q, int64_t ldq, double* W, double gamma, int64_t N);
int node_jacobi_from_sums(Ctx* c, const double* q, int64_t ldq, const double* S, int64_t ldS,
                          double* M, int64_t ldM, double* P, int64_t ldP, double gamma,
                          int64_t N);
int node_update_precond(Ctx* c, const double* q0, int64_t ld0, double* q, int64_t ldq,
                        const double* R, int64_t ldR, const double* P, int64_t ldP, double as,
                        int64_t N);
int node_time_step(Ctx* c, const double* V, const double* lam, double cfl,
                   double* dt, int64_t N);
int node_update(Ctx* c, const double* q0, int64_t ld0, double* q, int64_t ldq,
                const double* R, int64_t ldR, const double* V,
                const double* dt, double alpha, void* shadow, int shadow_type,
                int64_t ldsh, int64_t N);
int node_update_adjoint(Ctx* c, const double* sb, int64_t ldsb, double* qb, int64_t ldqb,
                        double* lam, int64_t ldl, const double* V, const double* dt,
                        double alpha, int64_t N);
int node_axpy(Ctx* c, double* y, int64_t ldy, double a, const double* x, int64_t ldx, int dim,
              int64_t n);
int node_fill(Ctx* c, void* p, int type, int64_t ld, int dim, int64_t n,
              double value);
int node_copy(Ctx* c, void* dst, int dtype, int64_t ldd, const void* src,
              int stype, int64_t lds, int dim, int64_t n);
// per-component reduction of an FP64 SoA dat into out[dim] (device)
int node_reduce(Ctx* c, const double* x, int64_t ld, int dim, int64_t n, int op, double* out);
// out[k*ld + t] = in[k*ld + idx[t]] for t < n (elements of `esize` bytes)
int node_gather(Ctx* c, void* out, const void* in, int esize, int64_t ld,
                int dim, const int64_t* idx, int64_t n);

struct Ctx {
  int device = 0;
  int sm_count = 0;
  size_t smem_optin = 0;
  cudaStream_t stream = nullptr;
  std::vector<SetRec> sets;
  std::vector<MapRec> maps;
  std::vector<DatRec> dats;
  std::string err;
  Strategy strat[OP2B_NUM_LOOPS][OP2B_NUM_PREC];
  std::map<std::pair<int, int>, DevBlockPlan> bplans;  // (map, part)
  std::map<int, DevSegPlan> splans;                    // map
  std::map<int, DevOwnPlan> oplans;                    // map
  std::map<int, Stage32Plan> s32plans;                 // map
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  // node-pass results an edge loop reads (apart from `scratch`, which the
  // loop's own strategy may use)
  void* aux = nullptr;
  size_t aux_bytes = 0;
  double tune_deadline_ms = 20000.0;
  int64_t launches = 0;
  std::map<std::string, Strategy> tuned;  // persistent table

  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
  // check the last launch; count it
  int launched(const char* what);
  // scratch of at least `bytes` (grows, never shrinks)
  int need_scratch(size_t bytes, void** out);
  int need_aux(size_t bytes, void** out);
  // plans (built or rebuilt on demand)
  int block_plan(int map, int32_t part, DevBlockPlan** out);
  int seg_plan(int map, DevSegPlan** out);
  int own_plan(int map, DevOwnPlan** out);
};

}  // namespace op2b

// The opaque handle of the C ABI.
struct op2b_ctx_s {
  op2b::Ctx c;
};
