/*
 * op2b: edge loops of an edge-based unstructured finite-volume solver on
 * one GB300 (sm_103a), behind a C ABI in the set / map / dat / parallel-loop
 * model of the paper (Reguly et al., "Acceleration of a Full-scale
 * Industrial CFD Application with OP2", Sec. 3.1 "The OP2 API",
 * Fig. "declOP2" and Fig. "OP2loop").
 *
 * Conventions for every entry point:
 *  - return 0 (OP2B_OK) or a negative OP2B_E* code; no C++ exception ever
 *    crosses the ABI; the text of the last error of a context is returned by
 *    op2b_last_error().
 *  - device pointers are borrowed: the caller allocates and frees the device
 *    memory behind every dat (it must outlive the dat's use).  The library
 *    owns its copies of the maps, its execution plans and its scratch.
 *  - work is launched asynchronously on the context's stream; launch errors
 *    are reported with OP2B_ECUDA, never by aborting.
 *  - dats are structure-of-arrays: component k of element i lives at
 *    ptr[k * ld + i], ld >= set size (Sec. 4.1.2 of the paper: SoA gave
 *    +40% on the GPU).  Maps are element-major on input, as in Fig.
 *    "declOP2" (entry k of element e at data[e * arity + k]) and 0-based.
 *  - loops take OP2-style argument lists (dat, map index, map, access).
 *    A direct argument has map = OP2B_ID and idx = -1.  The INC race on
 *    indirectly incremented dats is resolved by the strategy chosen for the
 *    loop (block colouring, FP64/FP32 atomics or sorted segmented
 *    reductions, Sec. 4.1 "execution plan"), set by op2b_set_strategy() or
 *    picked by the autotuner on measured time.
 */
#ifndef OP2B_H
#define OP2B_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define OP2B_OK 0
#define OP2B_EINVAL (-1)   /* bad handle, null pointer, bad size or flag */
#define OP2B_EDIM (-2)     /* dat dimension does not match the loop */
#define OP2B_ETYPE (-3)    /* dat element type does not match the loop */
#define OP2B_EACCESS (-4)  /* wrong access mode (e.g. INC on a direct arg) */
#define OP2B_ESET (-5)     /* dat lives on another set than the map/loop */
#define OP2B_ENOMEM (-6)   /* device or host allocation failed */
#define OP2B_ECUDA (-7)    /* a CUDA call or kernel launch failed */
#define OP2B_ETIMEOUT (-8) /* an autotuner candidate exceeded its deadline */
#define OP2B_EPLAN (-9)    /* an execution plan could not be built */
#define OP2B_ERANGE (-10)  /* a size exceeds what the library supports */

typedef struct op2b_ctx_s* op2b_ctx;
typedef int32_t op2b_set;
typedef int32_t op2b_map;
typedef int32_t op2b_dat;

/* access descriptors (Fig. "OP2loop": OP_READ, OP_WRITE, OP_RW, OP_INC) */
#define OP2B_READ 1
#define OP2B_WRITE 2
#define OP2B_RW 3
#define OP2B_INC 4

/* element types */
#define OP2B_F64 0
#define OP2B_F32 1
#define OP2B_I32 2
/* float-float: a value is the unevaluated sum hi + lo of two floats (hi
 * first, 8 bytes per element like a double; about 47 significant bits).
 * Shadows of F64 dats for the float-float flux (op2b_edge_flux); made by
 * op2b_dat_copy (F64 -> FF: hi = the top 24 significant bits, lo = the
 * remaining bits rounded to a float, relative error at most 2^-48;
 * magnitudes below 2^-126 become 0, 2^128 and above infinite) and by
 * op2b_node_update's shadow output. */
#define OP2B_FF 3

/* the identity "map" of a direct argument (OP_ID in the paper) */
#define OP2B_ID (-1)

/* one loop argument, like op_arg_dat(dat, idx, map, dim, type, access) */
typedef struct {
  op2b_dat dat;
  int32_t idx; /* which map entry (0 or 1 for an edge->node map); -1 direct */
  op2b_map map;
  int32_t acc; /* OP2B_READ / WRITE / RW / INC */
} op2b_arg;

/* loop identifiers, for strategies, the autotuner and plan statistics */
#define OP2B_LOOP_GREEN_GAUSS 0
#define OP2B_LOOP_FLUX1 1
#define OP2B_LOOP_FLUX2 2
#define OP2B_LOOP_SPECTRAL 3
#define OP2B_LOOP_FLUX1_ADJ 4
#define OP2B_LOOP_FLUX2_ADJ 5
#define OP2B_LOOP_GG_ADJ 6
#define OP2B_LOOP_FLUX1_TAN 7
#define OP2B_LOOP_FLUX2_TAN 8
#define OP2B_LOOP_GG_TAN 9
#define OP2B_LOOP_VISCOUS 10
#define OP2B_LOOP_FLUX2_PHI 11
#define OP2B_LOOP_JACOBI 12
#define OP2B_LOOP_JACOBI_SUMS 13
#define OP2B_NUM_LOOPS 14

/* arithmetic variant of a loop: all-FP64, or FP32 node data and arithmetic
 * (the INC precision is then fixed by the loop: FP64 residuals, FP32
 * gradients) */
#define OP2B_PREC_F64 0
#define OP2B_PREC_F32 1
/* FF node and edge data (float-float shadows) and float-float arithmetic:
 * the Green-Gauss loop (FF sums), the second-order flux, the node-limited
 * flux and the viscous flux (FP64 R), the flux adjoint and tangent (FP64
 * results) */
#define OP2B_PREC_FF 2
#define OP2B_NUM_PREC 3

/* race-resolution strategies (Sec. 4.1: mini-partitions with block
 * colouring; the other two are not in the paper) */
#define OP2B_STRAT_AUTO 0      /* autotune on the next call, then reuse */
#define OP2B_STRAT_ATOMIC 1    /* one thread per edge, atomic adds */
#define OP2B_STRAT_COLOUR 2    /* coloured edge blocks, shared-memory sums */
#define OP2B_STRAT_SEGMENTED 3 /* per-edge results, then per-node sums over
                                  the node-sorted edge ends */
#define OP2B_STRAT_BLOCK_ATOMIC 5 /* edge blocks in one launch, shared-memory
                                     sums per distinct node, one atomic add per
                                     (block, node, component) */
#define OP2B_STRAT_OWNER 6     /* thread per node over the edges whose lower-
                                  numbered end it is: that end's data loaded
                                  once and its sum kept in registers; atomic
                                  adds for the other end only */
#define OP2B_STRAT_GATHER 7    /* thread per node over the node's sorted
                                  edge ends, sums kept in registers and
                                  written once (no scatter, no race, no
                                  atomics); every edge is evaluated at both
                                  ends in its own orientation (bitwise the
                                  same result), so it costs twice the edge
                                  arithmetic -- except for Green-Gauss, whose
                                  gather forms each end's share directly.
                                  Not for the adjoint loops (per-edge
                                  outputs) */
#define OP2B_STRAT_HYBRID 8    /* FP64 Green-Gauss only: one launch in which
                                  half the blocks gather components 0-2 per
                                  node (FP64 pipe) while the other half
                                  scatter components 3-5 with atomic adds
                                  (L2 atomic units), so the two bounds
                                  overlap */
#define OP2B_STRAT_AUTO_DET 4  /* autotune among the deterministic strategies
                                  only (colour, segmented, gather): their sums
                                  run in a fixed order, so results are
                                  bitwise reproducible from run to run, which
                                  finite-difference uses of the loops need;
                                  the atomic strategy's order is not fixed */

/* loop flags */
#define OP2B_ZERO_INC 1 /* zero the INC targets first (they receive the sum) */

typedef struct {
  int32_t order;  /* 1: first order (q_i, q_j); 2: limited reconstruction */
  int32_t flags;  /* OP2B_ZERO_INC */
  double gamma;   /* ratio of specific heats */
  double eps_lim; /* van Albada epsilon (absolute) */
} op2b_flux_params;

/* coefficients of the viscous flux (op2b_viscous_flux) */
typedef struct {
  int32_t flags;    /* OP2B_ZERO_INC */
  int32_t reserved; /* 0 */
  double gamma;     /* ratio of specific heats (> 1) */
  double mu;        /* dynamic viscosity (>= 0) */
  double prandtl;   /* Prandtl number (> 0); heat conductivity
                       kappa = mu gamma / ((gamma - 1) prandtl) */
  double diff;      /* diffusivity of the passive scalar (>= 0) */
} op2b_visc_params;

typedef struct {
  int32_t strategy, block, part, staged; /* what the loop runs with */
  int64_t nblocks;     /* edge blocks (mini-partitions) of the plan */
  int64_t ncolours;    /* block colours */
  int64_t min_blocks_per_colour, max_blocks_per_colour;
  int64_t max_unique_nodes; /* largest number of distinct nodes of a block */
  double avg_unique_nodes;  /* mean distinct nodes per block */
  double tuned_ms;     /* autotuner's best time (0 if not tuned) */
} op2b_plan_stats_t;

/* ------------------------------------------------------------ lifecycle */
/* Create a context on CUDA device `device`, launching on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
int op2b_init(op2b_ctx* out, int32_t device, void* cuda_stream);
/* Free every library-owned allocation of the context. */
int op2b_finalize(op2b_ctx ctx);
/* Launch subsequent work on another stream (a cudaStream_t; NULL is the
 * legacy default stream).  The context's loops share its scratch buffers
 * and plans, so the switch orders the new stream after the work already
 * queued on the old one (an event recorded on the old stream, waited for on
 * the new one): work the context launched before the call finishes before
 * any it launches after.  Work that other code queues on the old stream
 * later is not ordered.  OP2B_ECUDA if the event cannot be recorded or
 * waited for; the context then keeps the old stream. */
int op2b_set_stream(op2b_ctx ctx, void* cuda_stream);
/* Text of the context's last error ("" if none).  Valid until the next
 * call on the context.  With ctx == NULL: the last init failure. */
const char* op2b_last_error(op2b_ctx ctx);
const char* op2b_version(void);

/* --------------------------------------------------------- declarations
 * Sec. 3.1, Fig. "declOP2": sets, maps between sets and data on sets. */

/* A named iteration space of `size` elements (size >= 0). */
int op2b_decl_set(op2b_ctx ctx, int64_t size, const char* name, op2b_set* out);
/* A map from every element of `from` to `arity` elements of `to`;
 * host_data holds from.size * arity 0-based indices, element-major.  The
 * data is copied (host and device).  Indices outside [0, to.size) give
 * OP2B_EINVAL.  Only arity 2 maps can drive the edge loops. */
int op2b_decl_map(op2b_ctx ctx, op2b_set from, op2b_set to, int32_t arity,
                  const int32_t* host_data, const char* name, op2b_map* out);
/* Data of `dim` components per element of `set` in caller-owned device
 * memory (SoA with leading dimension ld >= set size; ld = 0 means the set
 * size).  type is OP2B_F64, OP2B_F32 or OP2B_I32. */
int op2b_decl_dat(op2b_ctx ctx, op2b_set set, int32_t dim, int32_t type,
                  void* device_ptr, int64_t ld, const char* name,
                  op2b_dat* out);
/* Point a dat at another buffer of the same shape (e.g. a new tensor). */
int op2b_rebind_dat(op2b_ctx ctx, op2b_dat dat, void* device_ptr);
/* Copy the map's current (possibly renumbered) table to host memory,
 * element-major, from.size * arity entries. */
int op2b_fetch_map(op2b_ctx ctx, op2b_map map, int32_t* host_out);

/* ---------------------------------------------------------- renumbering
 * Sec. 4: renumbering the sets for cache locality (+17% for Hydra).
 * method: 0 none (edges are still sorted), 1 random (seeded SplitMix64),
 * 2 reverse Cuthill-McKee.  The node permutation is applied in place to
 * every dat declared on the map's to-set, and the edge order (edges sorted
 * by (min end, max end), orientation kept) to every dat on its from-set,
 * through a library scratch buffer.  node_perm_out (host, nullable) gets
 * new id of each old node; edge_order_out (host, nullable) the old index
 * of each new edge.  Plans of the map are rebuilt on their next use. */
int op2b_renumber(op2b_ctx ctx, op2b_map edge2node, int32_t method,
                  uint64_t seed, int32_t* node_perm_out,
                  int64_t* edge_order_out);

/* Partition-order renumbering by recursive coordinate bisection (Sec. 4:
 * the paper's RCB partitioner, used here as a node ordering): coords is an
 * F64 dim-3 dat on the map's to-set; sets of more than `leaf` nodes are
 * split at the median of their longest coordinate extent (ties: lowest
 * axis; nodes ordered by (coordinate, id)), lower half first; a leaf keeps
 * id order.  Applied to the dats and maps exactly like op2b_renumber. */
int op2b_renumber_rcb(op2b_ctx ctx, op2b_map edge2node, op2b_dat coords,
                      int32_t leaf, int32_t* node_perm_out,
                      int64_t* edge_order_out);

/* ----------------------------------------------------------- edge loops
 * Sec. 3.1, Fig. "OP2loop": a loop over the edge set that reads node data
 * through an arity-2 edge->node map and increments both end nodes (INC).
 * All indirect arguments must use the same map.  With OP2B_ZERO_INC the
 * INC dats are zeroed first; otherwise the loop adds to them.  The loop's
 * precision (OP2B_PREC_F64 / F32 / FF) is the type of its READ node dats. */

/* Green-Gauss gradient sums, per edge (i, j) with normal n:
 *   Graw_i[k][d] += (q_i,k + q_j,k)/2 * n_d,  Graw_j[k][d] -= the same.
 * args (5): q idx 0 READ, q idx 1 READ (node, dim 6), n OP2B_ID READ
 * (edge, dim 3), G idx 0 INC, G idx 1 INC (node, dim 18, component 3k+d).
 * All five of one type (F64, or F32 with FP32 sums, or FF: float-float
 * arithmetic and sums).  The FF loop always runs as a node gather -- one
 * thread per node over its edge ends sorted by node, the sums kept in
 * registers and written once -- so it has no race to resolve, ignores the
 * loop's strategy and is bitwise reproducible. */
int op2b_green_gauss(op2b_ctx ctx, const op2b_arg* args, int32_t nargs,
                     int32_t flags);

/* ------------------------------------------------ block-Jacobi blocks
 * Sec. 2: Hydra's Runge-Kutta march is block-Jacobi preconditioned; Table
 * "loopperfmpi": the per-node blocks are inverted in a direct loop
 * (`invjacs`).  The paper gives neither the block nor the scheme; here the
 * block of node i is the diagonal block of the Jacobian of the first-order
 * Rusanov residual with every edge's wave speed s_e held fixed:
 *   M_i += ( A(q_i, n) + s_e I)/2  at the first end of edge e,
 *   M_j += (-A(q_j, n) + s_e I)/2  at the second,
 * A(q, n) = d(f(q).n)/dq the Euler flux Jacobian (6 x 6 with the passive
 * scalar), s_e = max(|u_i.n| + a_i|n|, |u_j.n| + a_j|n|).
 * args (5): q idx 0 READ, q idx 1 READ (node, dim 6), n OP2B_ID READ (edge,
 * dim 3), M idx 0 INC, M idx 1 INC (node, dim 36, component 6r + c = row r,
 * column c), all F64 (else OP2B_ETYPE).  An edge loop like the others: any
 * strategy, tuned as OP2B_LOOP_JACOBI. */
int op2b_jacobi_blocks(op2b_ctx ctx, const op2b_arg* args, int32_t nargs, double gamma,
                       int32_t flags);

/* The same blocks in factored form.  A(q, n) is linear in n, so
 *   M_i = (Lambda_i I + A(q_i, S_i)) / 2,  Lambda_i = sum_e s_e,
 *   S_i = sum_e (+n_e at the first end, -n_e at the second):
 * op2b_jacobi_sums is the edge loop of the four sums -- args (5): q idx 0
 * READ, q idx 1 READ (node, dim 6), n OP2B_ID READ (edge, dim 3), S idx 0
 * INC, S idx 1 INC (node, dim 4: Lambda, S_x, S_y, S_z), all F64; tuned as
 * OP2B_LOOP_JACOBI_SUMS -- and op2b_jacobi_from_sums the node loop that forms
 * each block from q and S and writes it to M and/or its inverse (as
 * op2b_block_invert) to P (a dat handle < 0 skips that output; M, P dim 36
 * F64 and q dim 6, S dim 4 F64, all on one set).  Equal to
 * op2b_jacobi_blocks up to rounding, with 4 instead of 36 sums per edge end. */
int op2b_jacobi_sums(op2b_ctx ctx, const op2b_arg* args, int32_t nargs, double gamma,
                     int32_t flags);
int op2b_jacobi_from_sums(op2b_ctx ctx, op2b_dat q, op2b_dat S, op2b_dat M, op2b_dat P,
                          double gamma);

/* P_i = M_i^{-1} for every node (direct loop): Gauss-Jordan elimination in
 * place with partial pivoting (largest |pivot| of the column, the first on
 * ties), in FP64 registers.  M, P: node dats, dim 36, F64, on one set, P
 * distinct from M (else OP2B_EINVAL); M is not modified.  A block with a
 * zero pivot gets a non-finite P (no error is reported for it). */
int op2b_block_invert(op2b_ctx ctx, op2b_dat M, op2b_dat P);

/* Preconditioned stage (direct loop): q = q0 - alpha_sigma P R per node
 * (P dim 36 as above; q0, q, R dim 6); all F64 on one set.  q may be q0;
 * R must differ from q (else OP2B_EINVAL).  With P from op2b_block_invert
 * and alpha_sigma = alpha_k sigma this is the block-Jacobi preconditioned
 * form of op2b_node_update. */
int op2b_node_update_precond(op2b_ctx ctx, op2b_dat q0, op2b_dat q, op2b_dat R, op2b_dat P,
                             double alpha_sigma);

/* Green-Gauss gradients with the scaling by the node volume (Sec. 4.1.1's
 * direct loop op2b_grad_scale) applied to the sums: G = (G_in + sums) / V,
 * G_in = 0 with OP2B_ZERO_INC.  args as op2b_green_gauss; V: node dat,
 * dim 1, F64, on the map's to-set (else OP2B_ESET / OP2B_EDIM /
 * OP2B_ETYPE).  Under the node gather (the FF loop, or OP2B_STRAT_GATHER)
 * each node's sums are multiplied by its 1/V as they are written, formed
 * exactly as op2b_grad_scale forms it, so the result is bitwise that of
 * op2b_green_gauss followed by op2b_grad_scale, in one pass over G; the
 * other strategies run the scaling loop after the edge loop. */
int op2b_green_gauss_scaled(op2b_ctx ctx, const op2b_arg* args, int32_t nargs,
                            op2b_dat V, int32_t flags);

/* Rusanov edge flux (Euler, 6 conserved variables incl. a passive scalar):
 *   R_i += F(qL, qR, n),  R_j -= F(qL, qR, n).
 * order 1: qL = q_i, qR = q_j.  args (5): q 0 READ, q 1 READ, n ID READ,
 *   R 0 INC, R 1 INC.
 * order 2: van Albada-limited linear reconstruction
 *   qL = q_i + phi(G_i.dx, q_j - q_i)/2,  qR = q_j - phi(G_j.dx, q_j - q_i)/2.
 *   args (8): q 0 READ, q 1 READ, G 0 READ, G 1 READ, n ID READ,
 *   dx ID READ (edge, dim 3), R 0 INC, R 1 INC.
 * R is always F64 (dim 6).  q, G, n, dx are all F64 or all F32; with F32 the
 * flux arithmetic is FP32 and each edge's flux is converted to FP64 before
 * it is added into R.  Order 2 also takes all four as FF (float-float)
 * shadows: every operation of the reconstruction and the flux is then done
 * in float-float on the FP32 units (about 2^-47 per operation relative to
 * its operands; the flux stays within ~1e-14 of the FP64 definition
 * relative to its terms, values within the FF range), and each edge's flux
 * is converted to FP64 before it is added into R.  Other loops reject FF
 * dats with OP2B_ETYPE. */
int op2b_edge_flux(op2b_ctx ctx, const op2b_arg* args, int32_t nargs,
                   const op2b_flux_params* prm);

/* Spectral radius for the local time step:
 *   Lam_i += s_e, Lam_j += s_e,  s_e = max over the two end states of
 *   |u.n| + a|n|.
 * args (5): q 0 READ, q 1 READ (F64 dim 6), n ID READ (F64), Lam 0 INC,
 * Lam 1 INC (F64 dim 1). */
int op2b_spectral_radius(op2b_ctx ctx, const op2b_arg* args, int32_t nargs,
                         double gamma, int32_t flags);

/* Adjoint (transpose) of the flux loop for J = lam . R:
 * per edge w = lam_i - lam_j; the face states are recomputed from the node
 * data and the flux Jacobian-transpose products are scattered to both ends.
 * order 1 args (8): lam 0 READ, lam 1 READ, q 0 READ, q 1 READ, n ID READ,
 *   qbar 0 INC, qbar 1 INC, nbar ID WRITE.
 * order 2 args (13): lam 0, lam 1, q 0, q 1, G 0, G 1 (READ), n ID READ,
 *   dx ID READ, qbar 0 INC, qbar 1 INC, Gbar 0 INC, Gbar 1 INC (dim 18),
 *   nbar ID WRITE (edge, dim 3).  All F64; or, order 2 only, the eight READ
 *   dats FF (float-float shadows): the reverse sweep then runs in
 *   float-float arithmetic on the FP32 units and its per-edge results are
 *   converted to FP64 for qbar, Gbar (INC) and nbar (WRITE), all F64.  The
 *   float-float sweep's error is about 1e-12 of max |qbar| per component
 *   (the sweep's terms cancel by about two orders of magnitude). */
int op2b_edge_flux_adjoint(op2b_ctx ctx, const op2b_arg* args, int32_t nargs,
                           const op2b_flux_params* prm);

/* Adjoint of the Green-Gauss loop: with d = Gbar_i - Gbar_j (unscaled),
 *   qbar_i,k += sum_d d[k][d] n_d / 2,  qbar_j,k += the same,
 *   nbar_e[d] += sum_k (q_i,k + q_j,k)/2 d[k][d].
 * args (8): Gbar 0 READ, Gbar 1 READ (dim 18), q 0 READ, q 1 READ,
 * n ID READ, qbar 0 INC, qbar 1 INC, nbar ID RW.  All F64. */
int op2b_green_gauss_adjoint(op2b_ctx ctx, const op2b_arg* args,
                             int32_t nargs, int32_t flags);

/* Tangent-linear (forward-mode) loops: the Jacobian-vector products
 * dR = dR/dq . qd + dR/dn . nd that Newton-Krylov solvers need (dx and V
 * fixed).  Non-smooth points as in the adjoint: d|x|/dx = sign(x), 0 at 0;
 * the max picks the left state on ties.
 * Green-Gauss tangent: Gd_i += ((qd_i + qd_j) (x) n + (q_i + q_j) (x) nd)/2,
 *   Gd_j -= the same.  args (8): q 0 READ, q 1 READ, qd 0 READ, qd 1 READ
 *   (dim 6), n ID READ, nd ID READ (dim 3), Gd 0 INC, Gd 1 INC (dim 18).
 *   Scale with op2b_grad_scale afterwards, as for G.
 * Flux tangent: Rd_i += dF, Rd_j -= dF.
 *   order 1 args (8): q 0, q 1, qd 0, qd 1 (READ), n ID READ, nd ID READ,
 *     Rd 0 INC, Rd 1 INC.
 *   order 2 args (13): q 0, q 1, qd 0, qd 1, G 0, G 1, Gd 0, Gd 1 (READ,
 *     G and Gd scaled), n ID READ, nd ID READ, dx ID READ, Rd 0 INC,
 *     Rd 1 INC.  All F64; or, for op2b_edge_flux_tangent order 2, the
 *     eleven READ dats FF (float-float shadows): the linearisation then
 *     runs in float-float arithmetic and each edge's Fd is converted to
 *     FP64 before it is added into Rd (F64). */
int op2b_green_gauss_tangent(op2b_ctx ctx, const op2b_arg* args, int32_t nargs,
                             int32_t flags);
int op2b_edge_flux_tangent(op2b_ctx ctx, const op2b_arg* args, int32_t nargs,
                           const op2b_flux_params* prm);

/* Node-limited second-order flux: the alternative to the van Albada edge
 * limiter (the paper does not name Hydra's limiter; these are the two
 * textbook node limiters, Barth & Jespersen 1989 and Venkatakrishnan 1995).
 * Three steps per residual evaluation, after the gradients G:
 *
 * op2b_node_minmax: qmin_i / qmax_i = min / max of q over node i and the
 *   nodes that share an edge of `map` with it.  q, qmin, qmax: dim 6 on the
 *   map's to-set, all F64, all F32 or all FF, qmin and qmax distinct from q.
 *
 * op2b_node_limiter: for every end of every edge at node i, with d = dx at
 *   the edge's first end and -dx at its second, D2 = G_i . d / 2 (the
 *   unlimited extrapolation to the edge midpoint) and D1 = qmax_i - q_i if
 *   D2 > 0, qmin_i - q_i if D2 < 0;
 *     OP2B_LIM_BARTH_JESPERSEN  phi_e = min(1, D1 / D2),
 *     OP2B_LIM_VENKATAKRISHNAN  phi_e = (D1^2 + eps2 + 2 D1 D2) /
 *                                       (D1^2 + 2 D2^2 + D1 D2 + eps2),
 *   phi_e = 1 if D2 = 0, and phi_i = min over the node's edge ends (1 for a
 *   node without edges).  Venkatakrishnan's phi may exceed 1 slightly (it is
 *   1 at D2/D1 = 0 and 1/2 and above 1 in between); eps2 >= 0 smooths it
 *   (eps2 = (K h)^3 in Venkatakrishnan's notation).  q, qmin, qmax, phi dim
 *   6 and G dim 18 on the to-set, dx dim 3 on the from-set (edges), all F64,
 *   all F32 or all FF (float-float arithmetic); phi distinct from the inputs.
 *
 * op2b_edge_flux_limited: R_i += F(qL, qR, n), R_j -= F, with face states
 *   qL = q_i + phi_i (G_i . dx)/2, qR = q_j - phi_j (G_j . dx)/2 and the
 *   Rusanov flux of op2b_edge_flux.  args (10): q 0, q 1, G 0, G 1, phi 0,
 *   phi 1 (READ), n ID READ, dx ID READ, R 0 INC, R 1 INC (F64 dim 6).
 *   prm->order is ignored; prm->eps_lim unused.  q, G, phi, n, dx all F64,
 *   or all F32 with FP32 arithmetic, or all FF with float-float arithmetic;
 *   with F32 or FF each edge's flux is converted to FP64 before it is added
 *   into R.
 *
 * The two node loops run as gathers over the node-sorted edge ends (no
 * atomics, results independent of the order of the ends). */
#define OP2B_LIM_BARTH_JESPERSEN 1
#define OP2B_LIM_VENKATAKRISHNAN 2
int op2b_node_minmax(op2b_ctx ctx, op2b_map map, op2b_dat q, op2b_dat qmin,
                     op2b_dat qmax);
int op2b_node_limiter(op2b_ctx ctx, op2b_map map, int32_t kind, double eps2,
                      op2b_dat q, op2b_dat G, op2b_dat dx, op2b_dat qmin,
                      op2b_dat qmax, op2b_dat phi);
int op2b_edge_flux_limited(op2b_ctx ctx, const op2b_arg* args, int32_t nargs,
                           const op2b_flux_params* prm);

/* Viscous flux, the analogue of the paper's `vfluxedge` loop (named in
 * Table "loopperfmpi" as the most expensive loop of the solver, Sec. 4; the
 * paper does not give its formula, this is the textbook Navier-Stokes edge
 * flux).  Two steps:
 *
 * op2b_viscous_prims: direct node loop, W from q (dim 6) and the scaled
 *   conserved gradients G (dim 18, component 3k+d):
 *     W[0..2] = u = m / rho,  W[3] = T = p / rho,  W[4] = c = q5,
 *     W[5 + 3a + d] = (d u_a / d x_d) / 2,  W[14 + d] = (dT/dx_d) / 2,
 *     W[17 + d] = (dc/dx_d) / 2   (gradients halved),
 *   by the quotient rule (grad u_a = (grad m_a - u_a grad rho) / rho,
 *   grad p = (gamma-1)(grad E - u . grad m + |u|^2/2 grad rho),
 *   grad T = (grad p - T grad rho) / rho).  q, G, W (dim 20) all F64, all
 *   F32 or all FF (float-float arithmetic) on one set.
 *
 * op2b_viscous_flux: edge loop, per edge (i, j) with normal n and
 *   dx = x_j - x_i: for phi in (u_x, u_y, u_z, T, c) the face gradient
 *     g = gbar + ((phi_j - phi_i) - gbar . dx) dx / |dx|^2,
 *   gbar the mean of the two nodal gradients; then
 *     Fv = (0, tau n, (tau n) . (u_i + u_j)/2 + kappa g_T . n, diff g_c . n),
 *     tau = mu (g_u + g_u^T - 2/3 (div u) I),
 *   and R_i -= Fv, R_j += Fv (with OP2B_ZERO_INC R is zeroed first;
 *   otherwise the viscous flux is added to R, e.g. onto the inviscid flux).
 *   args (6): W 0 READ, W 1 READ (dim 20), n ID READ, dx ID READ (edge,
 *   dim 3), R 0 INC, R 1 INC (F64 dim 6).  W, n, dx all F64, or all F32
 *   with FP32 arithmetic, or all FF with float-float arithmetic; with F32
 *   or FF each edge's flux is converted to FP64 before it is added into R.
 *   |dx| must be nonzero. */
int op2b_viscous_prims(op2b_ctx ctx, op2b_dat q, op2b_dat G, op2b_dat W,
                       double gamma);
int op2b_viscous_flux(op2b_ctx ctx, const op2b_arg* args, int32_t nargs,
                      const op2b_visc_params* prm);

/* ------------------------------------------- fused FP32-mixed RK stage
 * One second-order explicit Runge-Kutta stage of Sec. 2's march -- the
 * Green-Gauss edge loop with the gradient scaling, the van Albada-limited
 * Rusanov flux edge loop and the node update (Table "loopperfmpi":
 * accumedges, ifluxedge, updatek) -- in the FP32-mixed precision: FP32 node
 * state, gradients, normals and flux arithmetic, FP64 residual and update.
 * The same arithmetic as op2b_green_gauss_scaled + op2b_edge_flux (order 2)
 * + op2b_node_update on F32 dats, fused into two node passes over packed
 * FP32 node records (q then G, 96 bytes per node) that the library keeps
 * between calls:
 *   Green-Gauss: G_i = (1/V_i) sum over the node's edge ends of
 *     (q_i + q_j) (x) (+-n_e/2), summed in FP32 (the same bits as the FP32
 *     node gather);
 *   flux and update: every edge end evaluates its edge's flux with its own
 *     node as the first end -- at the edge's second end the edge reversed
 *     (n -> -n, dx -> -dx), which gives bitwise minus the first end's value,
 *     so the residual is exactly antisymmetric -- the node sums them with
 *     Knuth's two-sum into a pair of floats (the sum to about 2^-48 of its
 *     running magnitude), converts the pair exactly to FP64 once: R_i; then
 *     q_i = q0_i - alpha (dt_i / V_i) R_i in FP64.
 * No atomics: the result is bitwise reproducible.
 *
 * map: the edge->node map (arity 2).  q0, q, V, dt: F64 node dats (dim 6,
 * 6, 1, 1); q is read (as its FP32 record) and overwritten with the new
 * state; q0 is read (and with OP2B_STAGE_STORE_Q0 overwritten by the new
 * state too, which saves the copy that starts the next step).  n, dx: edge
 * dats of dim 3, F64 or F32 (converted to FP32).  R: F64 node dat of dim 6
 * receiving the residual, or -1.  G: F32 node dat of dim 18 receiving the
 * scaled gradients, or -1.  gamma > 1, eps_lim > 0 as in op2b_flux_params.
 *
 * The records carry the state from one call to the next: the library packs
 * them from q on the first call for a map, after a renumbering, when q is a
 * different buffer, and whenever flags holds OP2B_STAGE_SYNC -- pass it
 * after changing q by any other means.  It packs the edge ends' adjacency
 * and geometry (n and dx in FP32, the edge reversed at its second end) on
 * the first call, when n or dx is a different buffer or type, and with
 * OP2B_STAGE_SYNC_MESH (after changing their values).
 *
 * Two forms of the passes, the same bits.  By default one thread per node
 * walks the node's edge ends, laid out sliced-ELL (the k-th ends of 32
 * consecutive nodes contiguous: 16 bytes per end for the Green-Gauss pass,
 * 32 for the flux pass), and gathers each other node's record from global
 * memory (three 32-byte loads); the flux pass streams its 32-byte end
 * records through a small shared-memory ring a few ends ahead.  With
 * OP2B_STAGE_STAGED the library plans, on the host at the first such call,
 * blocks of B consecutive nodes (B = 128, else 64 or 32) and the distinct
 * nodes each block's edge ends reach; where every such neighbourhood fits
 * 100 KB of shared memory at 112 bytes per record, both passes run one CTA
 * per node block that first copies the neighbourhood's records into shared
 * memory (asynchronous copies), and the ends read the records there (the
 * paper's staging of a block's indirect data, Sec. 4.1.2); elsewhere the
 * flag has no effect.  A numbering with compact blocks (recursive
 * coordinate bisection) needs about 0.2 records per edge end; on GB300 the
 * gathering form measured faster on the lattices tried, hence the default.
 * Library-owned memory per map: 48 bytes per edge end (sliced-ELL slots,
 * padded per 32-node slice to its largest degree) and 192 per node (plus,
 * once staged, 36 per end, 32 per edge and the neighbourhood lists).
 * Errors: OP2B_EINVAL (bad map, flag, q0 == q, coefficients), OP2B_ESET /
 * OP2B_EDIM / OP2B_ETYPE (dats), OP2B_ENOMEM, OP2B_ECUDA. */
#define OP2B_STAGE_SYNC 1
#define OP2B_STAGE_STORE_Q0 2
#define OP2B_STAGE_SYNC_MESH 4
/* stage each node block's neighbourhood in shared memory (see above) */
#define OP2B_STAGE_STAGED 8
int op2b_stage_mixed(op2b_ctx ctx, op2b_map map, op2b_dat q0, op2b_dat q, op2b_dat V,
                     op2b_dat dt, op2b_dat n, op2b_dat dx, op2b_dat R, op2b_dat G,
                     double alpha, double gamma, double eps_lim, int32_t flags);

/* ----------------------------------------------------------- node loops
 * Direct loops over the node set (no map). */

/* G <- G / V (G dim 18 F64, F32 or FF, RW; V dim 1 F64, READ). */
int op2b_grad_scale(op2b_ctx ctx, op2b_dat G, op2b_dat V);
/* Reverse of the scaling: Gbar <- Gbar / V. */
int op2b_grad_scale_adjoint(op2b_ctx ctx, op2b_dat Gbar, op2b_dat V);
/* dt_i = cfl V_i / Lam_i (all F64 dim 1). */
int op2b_time_step(op2b_ctx ctx, op2b_dat V, op2b_dat lam, double cfl,
                   op2b_dat dt);
/* Runge-Kutta stage update q = q0 - alpha (dt/V) R (F64 dim 6, F64 dim 1);
 * q32 (F32 or FF dim 6, or -1) receives the FP32 or float-float shadow of
 * the new q. */
int op2b_node_update(op2b_ctx ctx, op2b_dat q0, op2b_dat q, op2b_dat R,
                     op2b_dat V, op2b_dat dt, double alpha, op2b_dat q32);
/* Transpose of op2b_node_update with respect to q0 and R, the step of the
 * reverse sweep through one Runge-Kutta stage (Sec. 2's explicit march,
 * with dt fixed): qbar += sbar and lam = -alpha (dt/V) sbar, where sbar is
 * the adjoint of the stage's output state, qbar accumulates the adjoint of
 * the step's initial state q0, and lam is the weight that the residual's
 * adjoint loops then take (J = lam . R).  sbar, qbar, lam F64 dim 6 (three
 * distinct dats), V, dt F64 dim 1, all on one set. */
int op2b_node_update_adjoint(op2b_ctx ctx, op2b_dat sbar, op2b_dat qbar,
                             op2b_dat lam, op2b_dat V, op2b_dat dt,
                             double alpha);
/* y += a x, component-wise (F64 dats of one set and dim; a node or an edge
 * set), e.g. to accumulate the normals' adjoint over the stages. */
int op2b_dat_axpy(op2b_ctx ctx, op2b_dat y, double a, op2b_dat x);
/* Global reductions (the residual norms and global time step that an
 * explicit solver monitors each stage; the paper's `updatek` loop ends in a
 * global reduction, Table "loopperfmpi", and Sec. 4.2 finds reductions
 * latency-bound at scale).  out_dev (caller-owned device memory, dim
 * doubles) receives per component: OP2B_RED_SUM the sum, OP2B_RED_L2
 * sqrt(sum x^2), OP2B_RED_MAXABS max |x|, OP2B_RED_MIN the minimum, over
 * the elements of the dat's set.  F64 dats only.  Two passes in a fixed
 * order: the result is bitwise reproducible.  Asynchronous on the stream. */
#define OP2B_RED_SUM 0
#define OP2B_RED_L2 1
#define OP2B_RED_MAXABS 2
#define OP2B_RED_MIN 3
int op2b_dat_reduce(op2b_ctx ctx, op2b_dat dat, int32_t op, double* out_dev);
/* Set every component of a dat to `value`. */
int op2b_dat_fill(op2b_ctx ctx, op2b_dat dat, double value);
/* dst = src component-wise (same set and dim; F64 <-> F32 and F64 <-> FF
 * conversions). */
int op2b_dat_copy(op2b_ctx ctx, op2b_dat dst, op2b_dat src);

/* ------------------------------------------------ planner and autotuner
 * Sec. 4.1: the execution plan (mini-partitions, block colours) is built
 * once per loop and reused; block sizes were autotuned into a lookup table
 * (Sec. 4.1.2).  Here the tuner also picks the race-resolution strategy. */

/* Fix the strategy of (loop, prec) (OP2B_STRAT_*).  block: threads per CTA (32..1024,
 * 0 = default); part: edges per block for OP2B_STRAT_COLOUR (64..8192,
 * 0 = default); staged: stage each block's node data in shared memory
 * (COLOUR and BLOCK_ATOMIC; ignored elsewhere).  OP2B_STRAT_AUTO makes the
 * next call of the loop time the candidates (writing into scratch copies of
 * its INC dats) and keep the fastest. */
int op2b_set_strategy(op2b_ctx ctx, int32_t loop, int32_t prec,
                      int32_t strategy, int32_t block, int32_t part,
                      int32_t staged);
/* Deadline for one autotuner candidate in milliseconds (default 20000);
 * a candidate that has not finished by then gives OP2B_ETIMEOUT. */
int op2b_set_tune_deadline(op2b_ctx ctx, double ms);
/* Save / load the tuned strategies as a JSON object keyed by loop,
 * precision and set sizes. */
int op2b_save_tuning(op2b_ctx ctx, const char* path);
int op2b_load_tuning(op2b_ctx ctx, const char* path);
/* Strategy and plan statistics of (loop, prec) on `map` (block-plan fields
 * are -1 when no colouring exists at the loop's partition size). */
int op2b_plan_stats(op2b_ctx ctx, int32_t loop, int32_t prec, op2b_map map,
                    op2b_plan_stats_t* out);
/* Number of kernels the context has launched so far. */
int64_t op2b_launch_count(op2b_ctx ctx);

/* ------------------------------------------- allocation-free entry point
 * The paper has no counterpart to this call.  It serves callers that must
 * not allocate device memory (their memory is a pool owned by someone
 * else, or allocation is forbidden inside their time loop): it needs no
 * context, calls no cudaMalloc, cudaFree or allocating library routine, and
 * keeps its per-edge scratch in one array compiled into the library.
 *
 * Computes the first-order Rusanov residual R (overwritten, F64 SoA dim 6,
 * leading dimension ldR >= N): R_i = sum of F(q_i, q_j, n_e) over edges
 * leaving i minus the sum over edges entering i, with the sorted segmented
 * strategy.  Inputs (device pointers, caller-owned): q (F64 SoA dim 6, ldq),
 * n (F64 SoA dim 3 over the edges, ldn >= E), edge_first / edge_second (the
 * two ends of every edge, int32, 0-based), rowptr (N+1 int64) and ends (2E
 * int32, value 2e + side) of the edge ends sorted by node, as produced by
 * op2b_host_node_csr.  Launches on `stream` (a cudaStream_t) on the current
 * device and returns without waiting.
 *
 * R must not share memory with q or n (OP2B_EINVAL): it is zeroed before
 * the inputs are read.
 *
 * Limits and sharing: E must not exceed OP2B_NOALLOC_MAX_EDGES (larger sets
 * give OP2B_ERANGE and launch nothing).  The scratch array (6 x that many
 * doubles, 12 MiB) exists once per device for the life of the process and
 * every call uses it, so calls whose work overlaps on the GPU (concurrent
 * streams, or several host threads) race on it; serialise them.  A device
 * reserves the array when the library's module is loaded on it: under lazy
 * module loading (the CUDA default) that is this entry point's first call
 * on the device, under eager loading the creation of the CUDA context.  The
 * first call also looks up the array's device address and caches it.  Make
 * that first call at set-up -- before a memory pool takes the device's free
 * memory (else the reservation can fail with OP2B_ECUDA) and before any
 * stream capture; later calls allocate nothing.  On error
 * op2b_last_error(NULL) gives the reason. */
#define OP2B_NOALLOC_MAX_EDGES 262144
int op2b_edge_flux1_noalloc(const double* q, int64_t ldq, const double* n,
                            int64_t ldn, const int32_t* edge_first,
                            const int32_t* edge_second, const int64_t* rowptr,
                            const int32_t* ends, int64_t N, int64_t E,
                            double gamma, double* R, int64_t ldR,
                            void* stream);

/* ------------------------------------------ owner-compute partitions
 * The paper's distributed-memory execution (Sec. 3.2: OP2's MPI back-end
 * follows OPlus's owner-compute model; Sec. 2: OPlus's halo updates): the nodes are split
 * into parts; a part owns its nodes, executes every edge with an owned end
 * (a cut edge runs in both of its parts) and, before a loop reads node data
 * through the map, refreshes its halo -- the non-owned ends of its edges --
 * from the owners.  The results of a part are then final on its owned
 * nodes; halo rows hold partial sums and are overwritten by the next
 * exchange.
 *
 * Recursive coordinate bisection into nparts parts (Sec. 4: the mesh's 3-D
 * coordinates are split in x, y and z in turn until there is one part per
 * process).  xyz: host, N x 3 node-major.  part (host, N): part of each node.
 * A range meant for k parts is ordered by (coordinate on axis depth mod 3,
 * node id) and cut after floor(size * floor(k/2) / k) nodes, so part sizes
 * differ by at most one node per level.  Needs 1 <= nparts <= max(N, 1);
 * otherwise OP2B_EINVAL.  No context, no GPU. */
int op2b_host_partition_rcb(int64_t N, const double* xyz, int32_t nparts,
                            int32_t* part);

/* Halo plan of a node partition (host only; no context, no GPU).
 * edge: E x 2 element-major (0-based); part: N values in [0, nparts).
 * Per part p the plan holds its local mesh -- local node l is global node
 * nodes[l]: the n_owned owned nodes in increasing id, then the halo nodes
 * grouped by owner (increasing part), increasing id within a group -- its
 * edges (global ids with an owned end, increasing), the local edge->node
 * map (2 per edge, ends in the edge's own orientation), the import list
 * (owner and owner-local id of each halo node) and the export list (the
 * importers, increasing, and per importer the owned local ids it receives,
 * in that importer's halo order: export list of p for q = the q-side import
 * rows that name p, row by row).  Errors: OP2B_EINVAL (a part id or an edge
 * end out of range; text from op2b_last_error(NULL)), OP2B_ENOMEM.  The
 * handle owns host memory until op2b_halo_destroy. */
typedef struct op2b_halo_s* op2b_halo;
int op2b_halo_create(int64_t N, int64_t E, const int32_t* edge,
                     const int32_t* part, int32_t nparts, op2b_halo* out);
/* sizes[6] of part p: owned nodes, halo nodes, local edges, importers
 * (neighbours this part sends to), exported rows, local edges with a
 * non-owned end (the redundantly executed ones). */
int op2b_halo_sizes(op2b_halo h, int32_t p, int64_t* sizes);
/* Copy part p's lists into caller arrays (host; any may be NULL to skip):
 * nodes (owned + halo), edges (local edges), local_map (2 x local edges),
 * halo_owner and halo_src (halo nodes), nbr (importers), exp_off
 * (importers + 1), exp_idx (exported rows). */
int op2b_halo_part(op2b_halo h, int32_t p, int32_t* nodes, int32_t* edges,
                   int32_t* local_map, int32_t* halo_owner, int32_t* halo_src,
                   int32_t* nbr, int64_t* exp_off, int32_t* exp_idx);
int op2b_halo_destroy(op2b_halo h);

/* Halo exchange of one dat between parts held on the context's GPU (the
 * halo update of Sec. 2, between parts in one device's memory):
 * for every segment s (one per importer/owner pair) and entry k of it,
 * dst[s][c * dst_ld[s] + dst_idx[t]] = src[s][c * src_ld[s] + src_idx[t]]
 * for c < dim, t running over the entries of all segments in order
 * (count[s] per segment).  src / dst: device pointers of SoA dats of `type`
 * (F64, F32 or FF) whose leading dimensions are src_ld / dst_ld; the pointers
 * are captured at creation (re-create the exchange after moving a dat).
 * Indices must lie in [0, ld) of their dat (checked on the host at
 * creation: OP2B_EINVAL).  Rows of one exchange must not be both read and
 * written.  Index lists are host arrays, copied to the device; the handle
 * owns that device memory until op2b_exchange_destroy (which waits for the
 * context's stream).  op2b_exchange_run launches one kernel on the
 * context's stream. */
typedef struct op2b_exchange_s* op2b_exchange;
int op2b_exchange_create(op2b_ctx ctx, int32_t type, int32_t dim, int32_t nseg,
                         const void* const* src, const int64_t* src_ld,
                         void* const* dst, const int64_t* dst_ld,
                         const int64_t* count, const int32_t* src_idx,
                         const int32_t* dst_idx, op2b_exchange* out);
int op2b_exchange_run(op2b_ctx ctx, op2b_exchange x);
int op2b_exchange_destroy(op2b_ctx ctx, op2b_exchange x);

/* ------------------------------------------------ host-only planners
 * Pure host functions (no context, no GPU), exported for validation. */

/* Reverse Cuthill-McKee: new id of every node.  edge: E x 2 element-major. */
int op2b_host_rcm(int64_t N, int64_t E, const int32_t* edge,
                  int32_t* new_of_old);
/* Node permutation of `method` (as op2b_renumber) and the resulting edge
 * order (old index of each new edge). */
int op2b_host_renumber(int64_t N, int64_t E, const int32_t* edge,
                       int32_t method, uint64_t seed, int32_t* new_of_old,
                       int64_t* edge_order);
/* Block colouring of consecutive edge blocks of `part` edges: colour of
 * each of the ceil(E/part) blocks; *ncolours receives the colour count. */
int op2b_host_colour_blocks(int64_t N, int64_t E, const int32_t* edge,
                            int32_t part, int32_t* block_colour,
                            int64_t* ncolours);
/* Recursive coordinate bisection order (as op2b_renumber_rcb) from host
 * coordinates xyz (N x 3, node-major). */
int op2b_host_rcb(int64_t N, const double* xyz, int32_t leaf,
                  int32_t* new_of_old);
/* Node-sorted edge ends: rowptr (N+1) and ends (2E, value 2e + side). */
int op2b_host_node_csr(int64_t N, int64_t E, const int32_t* edge,
                       int64_t* rowptr, int64_t* ends);

#ifdef __cplusplus
}
#endif
#endif /* OP2B_H */
