// Host-side planners of the op2b library: renumbering, edge ordering, edge
// block plans with block colouring, and node-sorted edge ends.  Pure C++,
// no CUDA; the device copies are made by the context (api.cu).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace op2b {

// Reverse Cuthill-McKee (Cuthill & McKee 1969, reversal by George 1971):
// component starts at the unvisited node of least (degree, id); a node's
// unvisited neighbours are queued in increasing (degree, id) order; the
// visit order is reversed.  Returns false on bad input.
bool rcm(int64_t N, int64_t E, const int32_t* edge, int32_t* new_of_old);

// A uniformly random relabelling from SplitMix64 keys (Steele, Lea and
// Flood 2014): node k gets the rank of key(seed, k) (ties by k).
void random_perm(int64_t N, uint64_t seed, int32_t* new_of_old);

// Recursive coordinate bisection order: a set of more than `leaf` nodes is
// split at its median along the axis of largest extent (ties: lowest axis),
// nodes ordered by (coordinate, id) with the lower half first; a leaf lists
// its nodes by id.  new_of_old[node] = position in that order.
bool rcb(int64_t N, const double* xyz, int32_t leaf, int32_t* new_of_old);

// Old edge index of each new edge once the ends are relabelled: ordered by
// (min end, max end), ties in input order (two stable counting sorts).
void edge_order(int64_t N, int64_t E, const int32_t* edge,
                const int32_t* new_of_old, int64_t* order);

// Edge-block (mini-partition) plan over the edges in their current order:
// block b = edges [b*part, min(E, (b+1)*part)).
struct BlockPlan {
  int32_t part = 0;
  int64_t nblocks = 0;
  int32_t ncolours = 0;
  int64_t max_unique = 0;
  double avg_unique = 0.0;
  std::vector<int32_t> bn_off;   // nblocks+1: offsets into bnodes
  std::vector<int32_t> bnodes;   // distinct nodes of each block, ascending
  std::vector<uint32_t> eloc;    // per edge: local i | local j << 16
  std::vector<int32_t> lrow;     // per block U_b+1 offsets (at bn_off[b]+b)
  std::vector<uint16_t> lent;    // per block 2*ne entries: local edge*2+side
  std::vector<int32_t> colour;   // colour of each block
  std::vector<int32_t> cblocks;  // block ids grouped by colour
  std::vector<int64_t> coff;     // ncolours+1 offsets into cblocks
};

// Build the plan; the greedy colouring gives each block the smallest
// colour that no earlier block sharing a node holds (at most 256 colours).
bool build_block_plan(int64_t N, int64_t E, const int32_t* m0,
                      const int32_t* m1, int32_t part, BlockPlan* out,
                      std::string* err);

// Edge ends sorted by node (counting sort, ends of one node by edge
// index): rowptr N+1, ends 2E with value 2*e + side.
void node_csr(int64_t N, int64_t E, const int32_t* m0, const int32_t* m1,
              std::vector<int64_t>* rowptr, std::vector<int32_t>* ends);

// Edges grouped by their lower-numbered end (counting sort, edge order
// kept within a node): ptr N+1, idx E.
void owner_csr(int64_t N, int64_t E, const int32_t* m0, const int32_t* m1,
               std::vector<int64_t>* ptr, std::vector<int32_t>* idx);

// Owner-compute partitioning (the paper's distributed-memory model, Sec. 2 and 3.2:
// every partition owns a set of nodes, executes every edge that has an
// owned end -- redundantly where an edge is cut -- and imports the halo,
// the non-owned ends of those edges, from their owners).
//
// Recursive coordinate bisection into `nparts` parts (Sec. 4: the
// coordinates are split in x, y and z in turn until there are as many
// parts as processes).  A range of nodes meant for k parts is ordered by
// (coordinate on the axis of its depth, id) and cut after
// floor(size * floor(k/2) / k) nodes; the lower part gets the lower part
// numbers.  1 <= nparts <= max(N, 1).
bool rcb_parts(int64_t N, const double* xyz, int32_t nparts, int32_t* part);

struct HaloPart {
  int64_t n_owned = 0;
  // local node -> global node: owned nodes in increasing id, then the halo
  // grouped by owner (increasing part), increasing id within a group
  std::vector<int32_t> nodes;
  std::vector<int32_t> edges;       // global edge ids with an owned end, increasing
  std::vector<int32_t> lmap;        // 2 per local edge: local ids of its ends
  std::vector<int32_t> halo_owner;  // per halo node: owning part
  std::vector<int32_t> halo_src;    // per halo node: its local id in the owner
  std::vector<int32_t> nbr;         // parts that import from this one, increasing
  std::vector<int64_t> exp_off;     // nbr.size()+1 offsets into exp_idx
  std::vector<int32_t> exp_idx;     // owned local ids sent to each importer,
                                    // in the importer's halo order
  int64_t halo_edges = 0;           // local edges with a non-owned end
};

// Local meshes and the exchange lists of a node partition.
bool build_halo_plan(int64_t N, int64_t E, const int32_t* edge, const int32_t* part,
                     int32_t nparts, std::vector<HaloPart>* out, std::string* err);

// Node-block neighbourhoods (the staging plan of the fused mixed stage):
// blocks of B consecutive nodes; per block the distinct nodes its nodes'
// edge ends reach -- the block's own nodes first (local id = node - block
// start), then the others in increasing id -- and per edge end (in the
// node-sorted order of node_csr) the local id of the end's other node.
//
// The ends are also laid out sliced-ELL (slices of 32 consecutive nodes, one
// per warp; B is a multiple of 32): the k-th end of the slice's lane l at
// sell_off[slice] + 32 k + l, for k below the slice's largest degree, so
// that a warp reads the k-th ends of its 32 nodes from consecutive
// addresses; sell_end holds the end's index in the node-sorted order, -1
// where a lane's node has fewer ends.
struct NodeBlockPlan {
  int32_t B = 0;
  int64_t nblocks = 0;
  int64_t max_unique = 0;
  std::vector<int64_t> uoff;      // nblocks+1 offsets into uniq
  std::vector<int32_t> uniq;      // global node ids
  std::vector<int32_t> lother;    // per end: local id of the other node
  std::vector<int64_t> sell_off;  // per slice (ceil(N/32)) + 1
  std::vector<int32_t> sell_end;  // per slot: node-sorted end index or -1
};
void build_node_block_plan(int64_t N, const int32_t* m0, const int32_t* m1,
                           const std::vector<int64_t>& rowptr, const std::vector<int32_t>& ends,
                           int32_t B, NodeBlockPlan* out);

// Hardware threads to use for host planning.
int host_threads();

}  // namespace op2b
