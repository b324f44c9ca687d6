// Generic launcher: runs a loop body with the chosen race-resolution
// strategy on the context's stream.
#pragma once
#include <algorithm>

#include "edge_loops.cuh"
#include "internal.h"

namespace op2b {

// ERANGE when `block` threads exceed what the kernel's register use allows
template <typename K>
static int check_block(Ctx* c, K kern, int block) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess)
    return c->fail(OP2B_ECUDA, "cudaFuncGetAttributes failed");
  if (block > fa.maxThreadsPerBlock)
    return c->fail(OP2B_ERANGE, "block of " + std::to_string(block) + " threads exceeds the kernel's limit of " +
                                    std::to_string(fa.maxThreadsPerBlock));
  return OP2B_OK;
}

template <class P, bool STAGED, bool ATOMIC_FLUSH>
static int run_colour(Ctx* c, const P& ph, const LoopLaunch& L,
                      const Strategy& s, Targets<typename P::TA, P::DIM0> tg) {
  DevBlockPlan* bp = nullptr;
  int rc = c->block_plan(L.map, s.part, &bp);
  if (rc) return rc;
  const int32_t ucap = STAGED ? (int32_t)bp->max_unique : 0;
  const int64_t smem = colour_smem_bytes<P, STAGED>(bp->part, ucap);
  if (smem > (int64_t)c->smem_optin)
    return c->fail(OP2B_ERANGE, "colour plan: " + std::to_string(smem) +
                                    " B of shared memory per block exceeds the device limit");
  auto kern = k_colour<P, STAGED, ATOMIC_FLUSH>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return c->fail(OP2B_ECUDA, "cudaFuncSetAttribute (shared memory) failed");
  const int block = s.block > 0 ? s.block : 256;
  if ((rc = check_block(c, kern, block))) return rc;
  if constexpr (ATOMIC_FLUSH) {  // every block in one launch
    BlockView bv;
    bv.cblocks = nullptr;
    bv.nblk = bp->nblocks;
    bv.part = bp->part;
    bv.ucap = ucap;
    bv.bn_off = bp->bn_off;
    bv.bnodes = bp->bnodes;
    bv.eloc = bp->eloc;
    bv.lrow = bp->lrow;
    bv.lent = bp->lent;
    if (bv.nblk == 0) return OP2B_OK;
    unsigned grid = (unsigned)std::min<int64_t>(bv.nblk, (int64_t)1 << 30);
    kern<<<grid, block, smem, c->stream>>>(ph, L.m0, L.m1, L.E, bv, tg);
    return c->launched("block-atomic");
  } else {
    for (int32_t col = 0; col < bp->ncolours; col++) {
      BlockView bv;
      bv.cblocks = bp->cblocks + bp->coff[col];
      bv.nblk = bp->coff[col + 1] - bp->coff[col];
      bv.part = bp->part;
      bv.ucap = ucap;
      bv.bn_off = bp->bn_off;
      bv.bnodes = bp->bnodes;
      bv.eloc = bp->eloc;
      bv.lrow = bp->lrow;
      bv.lent = bp->lent;
      if (bv.nblk == 0) continue;
      unsigned grid = (unsigned)std::min<int64_t>(bv.nblk, (int64_t)1 << 30);
      kern<<<grid, block, smem, c->stream>>>(ph, L.m0, L.m1, L.E, bv, tg);
      if ((rc = c->launched("colour"))) return rc;
    }
  }
  return OP2B_OK;
}

// Grid of a node-parallel kernel (one node per thread): every block is
// launched, so that blocks are dispatched in node order and the nodes in
// flight form one moving window of the mesh whose neighbours stay in L2.
// (A grid capped at 64 blocks per SM makes each resident block stride over
// the whole mesh: measured 3.4% slower for the FP32-mixed stage's owner and
// gather loops at 200^3.  The edge-parallel atomic kernels keep the cap:
// without it the FP64 stage measured 0.2% slower.)
static inline int64_t full_grid(int64_t n, int block) {
  return std::min<int64_t>((n + block - 1) / block, 0x7fffffff);
}

template <class P>
static int run_body(Ctx* c, const P& ph, const LoopLaunch& L,
                    const Strategy& s, Targets<typename P::TA, P::DIM0> tg) {
  if (L.E == 0) return OP2B_OK;
  const int block = s.block > 0 ? s.block : 256;
  if (block < 32 || block > 1024 || block % 32)
    return c->fail(OP2B_EINVAL, "block size must be a multiple of 32 in [32, 1024]");
  const int64_t cap = (int64_t)c->sm_count * 64;
  switch (s.strategy) {
    case OP2B_STRAT_ATOMIC: {
      if (int rc = check_block(c, k_atomic<P>, block)) return rc;
      int64_t grid = std::min<int64_t>((L.E + block - 1) / block, cap);
      k_atomic<P><<<(unsigned)grid, block, 0, c->stream>>>(ph, L.m0, L.m1, L.E, tg);
      return c->launched("atomic");
    }
    case OP2B_STRAT_COLOUR:
      return s.staged ? run_colour<P, true, false>(c, ph, L, s, tg)
                      : run_colour<P, false, false>(c, ph, L, s, tg);
    case OP2B_STRAT_OWNER: {
      DevOwnPlan* op = nullptr;
      int rc = c->own_plan(L.map, &op);
      if (rc) return rc;
      if ((rc = check_block(c, k_owner<P>, block))) return rc;
      // node-parallel: every block launched (see full_grid)
      int64_t grid = full_grid(L.N, block);
      if (grid == 0) return OP2B_OK;
      k_owner<P><<<(unsigned)grid, block, 0, c->stream>>>(ph, L.m0, L.m1, L.N, op->ptr, op->idx, tg);
      return c->launched("owner");
    }
    case OP2B_STRAT_BLOCK_ATOMIC:
      return s.staged ? run_colour<P, true, true>(c, ph, L, s, tg)
                      : run_colour<P, false, true>(c, ph, L, s, tg);
    case OP2B_STRAT_SEGMENTED: {
      DevSegPlan* sp = nullptr;
      int rc = c->seg_plan(L.map, &sp);
      if (rc) return rc;
      using TE = typename P::TE;
      if ((rc = check_block(c, k_seg_edges<P>, block))) return rc;
      const size_t bytes = (size_t)ebuf_stride<P>() * L.E * sizeof(TE);
      void* buf = nullptr;
      if ((rc = c->need_scratch(bytes, &buf))) return rc;
      int64_t grid = std::min<int64_t>((L.E + block - 1) / block, cap);
      k_seg_edges<P><<<(unsigned)grid, block, 0, c->stream>>>(ph, L.m0, L.m1, L.E, (TE*)buf);
      if ((rc = c->launched("segmented edges"))) return rc;
      int64_t gridn = std::min<int64_t>((L.N + block - 1) / block, cap);
      if (gridn == 0) return OP2B_OK;
      if constexpr (HasPack<P>::value)  // writes every node (scaling fused when L.vol)
        k_seg_nodes_packed<P><<<(unsigned)gridn, block, 0, c->stream>>>(
            sp->rowptr, sp->ends, L.N, L.E, (const TE*)buf, tg, L.vol,
            !(L.flags & OP2B_ZERO_INC));
      else
        k_seg_nodes<TE, typename P::TA, P::OUT, P::MODE, P::DIM0>
            <<<(unsigned)gridn, block, 0, c->stream>>>(sp->rowptr, sp->ends, L.N, L.E,
                                                       (const TE*)buf, tg);
      return c->launched("segmented nodes");
    }
    case OP2B_STRAT_GATHER: {
      if constexpr (HasDirectOutput<P>::value) {
        return c->fail(OP2B_EINVAL, "the gather strategy needs a loop without per-edge outputs");
      } else {
        DevSegPlan* sp = nullptr;
        int rc = c->seg_plan(L.map, &sp);
        if (rc) return rc;
        if ((rc = check_block(c, k_gather_nodes<P>, block))) return rc;
        int64_t grid = full_grid(L.N, block);
        if (grid == 0) return OP2B_OK;
        k_gather_nodes<P><<<(unsigned)grid, block, 0, c->stream>>>(
            ph, sp->rowptr, sp->ends, L.m0, L.m1, L.N, tg, !(L.flags & OP2B_ZERO_INC));
        return c->launched("gather");
      }
    }
    default:
      return c->fail(OP2B_EINVAL, "unknown strategy");
  }
}

}  // namespace op2b
