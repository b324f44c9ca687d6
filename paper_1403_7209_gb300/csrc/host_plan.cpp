// Host planners: renumbering, edge ordering, block plans, node-sorted ends.
#include "host_plan.h"

#include <algorithm>
#include <numeric>
#include <string>
#include <thread>

namespace op2b {

int host_threads() {
  unsigned t = std::thread::hardware_concurrency();
  if (t == 0) t = 4;
  return (int)std::min<unsigned>(t, 32);
}

// Run f(lo, hi) over [0, n) split into contiguous chunks on host threads.
template <class F>
static void parallel_for(int64_t n, F f) {
  int T = host_threads();
  if (n < 4096 || T == 1) {
    f((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + T - 1) / T;
  for (int t = 0; t < T; t++) {
    int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back([=] { f(lo, hi); });
  }
  for (auto& x : th) x.join();
}

bool rcm(int64_t N, int64_t E, const int32_t* edge, int32_t* new_of_old) {
  if (N < 0 || E < 0) return false;
  if (N == 0) return true;
  // undirected adjacency with duplicates and self loops removed
  std::vector<int64_t> off(N + 1, 0);
  for (int64_t e = 0; e < E; e++) {
    int64_t i = edge[2 * e], j = edge[2 * e + 1];
    if (i < 0 || i >= N || j < 0 || j >= N) return false;
    if (i == j) continue;
    off[i + 1]++;
    off[j + 1]++;
  }
  for (int64_t v = 0; v < N; v++) off[v + 1] += off[v];
  std::vector<int32_t> adj(off[N]);
  {
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    for (int64_t e = 0; e < E; e++) {
      int32_t i = edge[2 * e], j = edge[2 * e + 1];
      if (i == j) continue;
      adj[pos[i]++] = j;
      adj[pos[j]++] = i;
    }
  }
  std::vector<int32_t> deg(N);
  parallel_for(N, [&](int64_t lo, int64_t hi) {
    for (int64_t v = lo; v < hi; v++) {
      auto b = adj.begin() + off[v], en = adj.begin() + off[v + 1];
      std::sort(b, en);
      deg[v] = (int32_t)(std::unique(b, en) - b);
    }
  });
  // component starts in (degree, id) order: stable counting sort by degree
  int32_t maxdeg = 0;
  for (int64_t v = 0; v < N; v++) maxdeg = std::max(maxdeg, deg[v]);
  std::vector<int64_t> dc(maxdeg + 2, 0);
  for (int64_t v = 0; v < N; v++) dc[deg[v] + 1]++;
  for (int32_t d = 0; d <= maxdeg; d++) dc[d + 1] += dc[d];
  std::vector<int32_t> starts(N);
  for (int64_t v = 0; v < N; v++) starts[dc[deg[v]]++] = (int32_t)v;

  std::vector<uint8_t> seen(N, 0);
  std::vector<int32_t> order;  // breadth-first visit order, used as queue
  order.reserve(N);
  std::vector<uint64_t> fresh;
  int64_t si = 0, head = 0;
  while ((int64_t)order.size() < N) {
    while (seen[starts[si]]) si++;
    int32_t s = starts[si];
    seen[s] = 1;
    order.push_back(s);
    while (head < (int64_t)order.size()) {
      int32_t v = order[head++];
      fresh.clear();
      for (int64_t t = off[v]; t < off[v] + deg[v]; t++) {
        int32_t w = adj[t];
        if (!seen[w]) fresh.push_back(((uint64_t)(uint32_t)deg[w] << 32) | (uint32_t)w);
      }
      std::sort(fresh.begin(), fresh.end());
      for (uint64_t k : fresh) {
        int32_t w = (int32_t)(k & 0xffffffffu);
        seen[w] = 1;
        order.push_back(w);
      }
    }
  }
  for (int64_t k = 0; k < N; k++) new_of_old[order[N - 1 - k]] = (int32_t)k;
  return true;
}

bool rcb(int64_t N, const double* xyz, int32_t leaf, int32_t* new_of_old) {
  if (N < 0 || leaf < 1) return false;
  std::vector<int32_t> ids(N);
  for (int64_t i = 0; i < N; i++) ids[i] = (int32_t)i;
  int64_t next = 0;
  // explicit stack of [lo, hi) ranges; the lower half is processed first
  std::vector<std::pair<int64_t, int64_t>> st;
  st.push_back({0, N});
  while (!st.empty()) {
    auto [lo, hi] = st.back();
    st.pop_back();
    if (hi - lo <= leaf) {
      std::sort(ids.begin() + lo, ids.begin() + hi);
      for (int64_t k = lo; k < hi; k++) new_of_old[ids[k]] = (int32_t)(next++);
      continue;
    }
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t k = lo; k < hi; k++)
      for (int d = 0; d < 3; d++) {
        double v = xyz[3 * (int64_t)ids[k] + d];
        mn[d] = std::min(mn[d], v);
        mx[d] = std::max(mx[d], v);
      }
    int ax = 0;
    for (int d = 1; d < 3; d++)
      if (mx[d] - mn[d] > mx[ax] - mn[ax]) ax = d;
    const int64_t mid = lo + (hi - lo) / 2;
    std::nth_element(ids.begin() + lo, ids.begin() + mid, ids.begin() + hi,
                     [&](int32_t a, int32_t b) {
                       double ca = xyz[3 * (int64_t)a + ax], cb = xyz[3 * (int64_t)b + ax];
                       return ca < cb || (ca == cb && a < b);
                     });
    st.push_back({mid, hi});
    st.push_back({lo, mid});
  }
  return true;
}

static inline uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void random_perm(int64_t N, uint64_t seed, int32_t* new_of_old) {
  const uint64_t G = 0x9E3779B97F4A7C15ull;
  const uint64_t stream = 8;  // the library's renumbering stream
  uint64_t base = splitmix_mix(seed * G + stream);
  std::vector<std::pair<uint64_t, int32_t>> key(N);
  for (int64_t k = 0; k < N; k++)
    key[k] = {splitmix_mix(base + (uint64_t)(k + 1) * G), (int32_t)k};
  std::sort(key.begin(), key.end());
  for (int64_t r = 0; r < N; r++) new_of_old[key[r].second] = (int32_t)r;
}

void edge_order(int64_t N, int64_t E, const int32_t* edge,
                const int32_t* new_of_old, int64_t* order) {
  std::vector<int32_t> lo(E), hi(E);
  for (int64_t e = 0; e < E; e++) {
    int32_t a = new_of_old ? new_of_old[edge[2 * e]] : edge[2 * e];
    int32_t b = new_of_old ? new_of_old[edge[2 * e + 1]] : edge[2 * e + 1];
    lo[e] = std::min(a, b);
    hi[e] = std::max(a, b);
  }
  // LSD: stable counting sort by hi, then by lo
  std::vector<int64_t> cnt(N + 1), tmp(E);
  std::fill(cnt.begin(), cnt.end(), 0);
  for (int64_t e = 0; e < E; e++) cnt[hi[e] + 1]++;
  for (int64_t v = 0; v < N; v++) cnt[v + 1] += cnt[v];
  for (int64_t e = 0; e < E; e++) tmp[cnt[hi[e]]++] = e;
  std::fill(cnt.begin(), cnt.end(), 0);
  for (int64_t e = 0; e < E; e++) cnt[lo[e] + 1]++;
  for (int64_t v = 0; v < N; v++) cnt[v + 1] += cnt[v];
  for (int64_t t = 0; t < E; t++) {
    int64_t e = tmp[t];
    order[cnt[lo[e]]++] = e;
  }
}

bool build_block_plan(int64_t N, int64_t E, const int32_t* m0,
                      const int32_t* m1, int32_t part, BlockPlan* P,
                      std::string* err) {
  if (part < 1 || part > 32767) {
    *err = "block plan: part must be in [1, 32767]";
    return false;
  }
  P->part = part;
  P->nblocks = (E + part - 1) / part;
  const int64_t nb = P->nblocks;
  std::vector<std::vector<int32_t>> uniq(nb);
  parallel_for(nb, [&](int64_t lo, int64_t hi) {
    for (int64_t b = lo; b < hi; b++) {
      int64_t e0 = b * part, e1 = std::min(E, e0 + part);
      auto& u = uniq[b];
      u.reserve(2 * (e1 - e0));
      for (int64_t e = e0; e < e1; e++) {
        u.push_back(m0[e]);
        u.push_back(m1[e]);
      }
      std::sort(u.begin(), u.end());
      u.erase(std::unique(u.begin(), u.end()), u.end());
    }
  });
  P->bn_off.assign(nb + 1, 0);
  int64_t tot = 0, mx = 0;
  for (int64_t b = 0; b < nb; b++) {
    P->bn_off[b] = (int32_t)tot;
    tot += (int64_t)uniq[b].size();
    mx = std::max<int64_t>(mx, (int64_t)uniq[b].size());
  }
  if (tot + nb >= ((int64_t)1 << 31)) {
    *err = "block plan: too many block-local nodes for 32-bit offsets";
    return false;
  }
  P->bn_off[nb] = (int32_t)tot;
  P->max_unique = mx;
  P->avg_unique = nb ? (double)tot / (double)nb : 0.0;
  P->bnodes.resize(tot);
  P->eloc.resize(E);
  P->lrow.resize(tot + nb);
  P->lent.resize(2 * E);
  parallel_for(nb, [&](int64_t lo, int64_t hi) {
    std::vector<int32_t> cnt;
    for (int64_t b = lo; b < hi; b++) {
      const auto& u = uniq[b];
      int64_t U = (int64_t)u.size();
      std::copy(u.begin(), u.end(), P->bnodes.begin() + P->bn_off[b]);
      int64_t e0 = b * part, e1 = std::min(E, e0 + part);
      cnt.assign(U + 1, 0);
      for (int64_t e = e0; e < e1; e++) {
        uint32_t li = (uint32_t)(std::lower_bound(u.begin(), u.end(), m0[e]) - u.begin());
        uint32_t lj = (uint32_t)(std::lower_bound(u.begin(), u.end(), m1[e]) - u.begin());
        P->eloc[e] = li | (lj << 16);
        cnt[li + 1]++;
        cnt[lj + 1]++;
      }
      for (int64_t k = 0; k < U; k++) cnt[k + 1] += cnt[k];
      int32_t* lr = P->lrow.data() + P->bn_off[b] + b;
      for (int64_t k = 0; k <= U; k++) lr[k] = cnt[k];
      uint16_t* le = P->lent.data() + 2 * e0;
      for (int64_t e = e0; e < e1; e++) {
        uint32_t l = P->eloc[e];
        uint16_t el = (uint16_t)(e - e0);
        le[cnt[l & 0xffff]++] = (uint16_t)(el * 2 + 0);
        le[cnt[l >> 16]++] = (uint16_t)(el * 2 + 1);
      }
    }
  });
  // greedy block colouring, 64 colours per pass
  P->colour.assign(nb, -1);
  std::vector<uint64_t> mask(N);
  int64_t left = nb;
  int32_t base = 0;
  while (left > 0) {
    if (base >= 256) {
      *err = "block plan: more than 256 block colours";
      return false;
    }
    std::fill(mask.begin(), mask.end(), 0ull);
    for (int64_t b = 0; b < nb; b++) {
      if (P->colour[b] >= 0) continue;
      const int32_t* nd = P->bnodes.data() + P->bn_off[b];
      int64_t U = P->bn_off[b + 1] - P->bn_off[b];
      uint64_t used = 0;
      for (int64_t k = 0; k < U; k++) used |= mask[nd[k]];
      if (used == ~0ull) continue;  // try in the next pass
      int c = __builtin_ctzll(~used);
      P->colour[b] = base + c;
      for (int64_t k = 0; k < U; k++) mask[nd[k]] |= (1ull << c);
      left--;
    }
    base += 64;
  }
  int32_t nc = 0;
  for (int64_t b = 0; b < nb; b++) nc = std::max(nc, P->colour[b] + 1);
  P->ncolours = nc;
  P->coff.assign(nc + 1, 0);
  for (int64_t b = 0; b < nb; b++) P->coff[P->colour[b] + 1]++;
  for (int32_t c = 0; c < nc; c++) P->coff[c + 1] += P->coff[c];
  P->cblocks.resize(nb);
  std::vector<int64_t> pos(P->coff.begin(), P->coff.end() - 1);
  for (int64_t b = 0; b < nb; b++) P->cblocks[pos[P->colour[b]]++] = (int32_t)b;
  return true;
}

void node_csr(int64_t N, int64_t E, const int32_t* m0, const int32_t* m1,
              std::vector<int64_t>* rowptr, std::vector<int32_t>* ends) {
  rowptr->assign(N + 1, 0);
  auto& rp = *rowptr;
  for (int64_t e = 0; e < E; e++) {
    rp[m0[e] + 1]++;
    rp[m1[e] + 1]++;
  }
  for (int64_t v = 0; v < N; v++) rp[v + 1] += rp[v];
  ends->resize(2 * E);
  std::vector<int64_t> pos(rp.begin(), rp.end() - 1);
  for (int64_t e = 0; e < E; e++) {
    (*ends)[pos[m0[e]]++] = (int32_t)(2 * e);
    (*ends)[pos[m1[e]]++] = (int32_t)(2 * e + 1);
  }
}

void owner_csr(int64_t N, int64_t E, const int32_t* m0, const int32_t* m1,
               std::vector<int64_t>* ptr, std::vector<int32_t>* idx) {
  ptr->assign(N + 1, 0);
  auto& p = *ptr;
  for (int64_t e = 0; e < E; e++) p[std::min(m0[e], m1[e]) + 1]++;
  for (int64_t v = 0; v < N; v++) p[v + 1] += p[v];
  idx->resize(E);
  std::vector<int64_t> pos(p.begin(), p.end() - 1);
  for (int64_t e = 0; e < E; e++) (*idx)[pos[std::min(m0[e], m1[e])]++] = (int32_t)e;
}

bool rcb_parts(int64_t N, const double* xyz, int32_t nparts, int32_t* part) {
  if (N < 0 || nparts < 1 || (int64_t)nparts > std::max<int64_t>(N, 1)) return false;
  std::vector<int32_t> ids(N);
  for (int64_t i = 0; i < N; i++) ids[i] = (int32_t)i;
  struct Range {
    int64_t lo, hi;
    int32_t p0, k, depth;
  };
  std::vector<Range> st;
  st.push_back({0, N, 0, nparts, 0});
  while (!st.empty()) {
    const Range r = st.back();
    st.pop_back();
    if (r.k == 1) {
      for (int64_t t = r.lo; t < r.hi; t++) part[ids[t]] = r.p0;
      continue;
    }
    const int ax = r.depth % 3;
    const int32_t kl = r.k / 2;
    const int64_t cut = r.lo + (r.hi - r.lo) * kl / r.k;
    std::nth_element(ids.begin() + r.lo, ids.begin() + cut, ids.begin() + r.hi,
                     [&](int32_t a, int32_t b) {
                       const double ca = xyz[3 * (int64_t)a + ax], cb = xyz[3 * (int64_t)b + ax];
                       return ca < cb || (ca == cb && a < b);
                     });
    st.push_back({cut, r.hi, r.p0 + kl, r.k - kl, r.depth + 1});
    st.push_back({r.lo, cut, r.p0, kl, r.depth + 1});
  }
  return true;
}

bool build_halo_plan(int64_t N, int64_t E, const int32_t* edge, const int32_t* part,
                     int32_t nparts, std::vector<HaloPart>* out, std::string* err) {
  if (N < 0 || E < 0 || nparts < 1 || N > INT32_MAX || E > INT32_MAX) {
    *err = "bad sizes";
    return false;
  }
  for (int64_t i = 0; i < N; i++)
    if (part[i] < 0 || part[i] >= nparts) {
      *err = "node " + std::to_string(i) + " has part " + std::to_string(part[i]) +
             " outside [0, " + std::to_string(nparts) + ")";
      return false;
    }
  for (int64_t e = 0; e < 2 * E; e++)
    if (edge[e] < 0 || edge[e] >= N) {
      *err = "edge " + std::to_string(e / 2) + " has an end outside the node set";
      return false;
    }
  std::vector<HaloPart>& P = *out;
  P.assign(nparts, HaloPart());
  // local id of every node in its owner: rank among the owner's nodes
  std::vector<int32_t> own_local(N);
  for (int64_t i = 0; i < N; i++) {
    HaloPart& h = P[part[i]];
    own_local[i] = (int32_t)h.n_owned++;
    h.nodes.push_back((int32_t)i);
  }
  // edges with an owned end, and the (owner, node) pairs of the halo
  std::vector<std::vector<std::pair<int32_t, int32_t>>> halo(nparts);
  for (int64_t e = 0; e < E; e++) {
    const int32_t a = edge[2 * e], b = edge[2 * e + 1];
    const int32_t pa = part[a], pb = part[b];
    P[pa].edges.push_back((int32_t)e);
    if (pb != pa) {
      P[pb].edges.push_back((int32_t)e);
      halo[pa].push_back({pb, b});
      halo[pb].push_back({pa, a});
    }
  }
  std::vector<int32_t> halo_local(N, -1);
  for (int32_t p = 0; p < nparts; p++) {
    HaloPart& h = P[p];
    auto& hv = halo[p];
    std::sort(hv.begin(), hv.end());
    hv.erase(std::unique(hv.begin(), hv.end()), hv.end());
    h.halo_owner.resize(hv.size());
    h.halo_src.resize(hv.size());
    for (size_t k = 0; k < hv.size(); k++) {
      const int32_t r = hv[k].first, g = hv[k].second;
      halo_local[g] = (int32_t)(h.n_owned + (int64_t)k);
      h.nodes.push_back(g);
      h.halo_owner[k] = r;
      h.halo_src[k] = own_local[g];
      // part r exports g to p; p increases in this loop, so every
      // exporter's importer list stays sorted
      HaloPart& o = P[r];
      if (o.nbr.empty() || o.nbr.back() != p) {
        o.nbr.push_back(p);
        o.exp_off.push_back((int64_t)o.exp_idx.size());
      }
      o.exp_idx.push_back(own_local[g]);
    }
    h.lmap.resize(2 * h.edges.size());
    for (size_t t = 0; t < h.edges.size(); t++) {
      const int64_t e = h.edges[t];
      bool cut = false;
      for (int s = 0; s < 2; s++) {
        const int32_t g = edge[2 * e + s];
        if (part[g] == p) {
          h.lmap[2 * t + s] = own_local[g];
        } else {
          h.lmap[2 * t + s] = halo_local[g];
          cut = true;
        }
      }
      h.halo_edges += cut;
    }
    for (size_t k = 0; k < hv.size(); k++) halo_local[hv[k].second] = -1;
    hv.clear();
    hv.shrink_to_fit();
  }
  for (auto& h : P) h.exp_off.push_back((int64_t)h.exp_idx.size());
  return true;
}

}  // namespace op2b

namespace op2b {

void build_node_block_plan(int64_t N, const int32_t* m0, const int32_t* m1,
                           const std::vector<int64_t>& rowptr, const std::vector<int32_t>& ends,
                           int32_t B, NodeBlockPlan* out) {
  NodeBlockPlan& p = *out;
  p = NodeBlockPlan();
  p.B = B;
  p.nblocks = (N + B - 1) / B;
  p.uoff.assign((size_t)p.nblocks + 1, 0);
  p.lother.assign(ends.size(), 0);
  std::vector<int64_t> stamp((size_t)N, -1);
  std::vector<int32_t> local((size_t)N, 0);
  std::vector<int32_t> extra;
  for (int64_t b = 0; b < p.nblocks; b++) {
    const int64_t n0 = b * B, n1 = std::min<int64_t>(N, n0 + B);
    p.uoff[b] = (int64_t)p.uniq.size();
    for (int64_t v = n0; v < n1; v++) {
      stamp[v] = b;
      local[v] = (int32_t)(v - n0);
      p.uniq.push_back((int32_t)v);
    }
    extra.clear();
    for (int64_t t = rowptr[n0]; t < rowptr[n1]; t++) {
      const int32_t end = ends[t];
      const int32_t j = (end & 1) ? m0[end >> 1] : m1[end >> 1];
      if (stamp[j] != b) {
        stamp[j] = b;
        extra.push_back(j);
      }
    }
    std::sort(extra.begin(), extra.end());
    for (size_t k = 0; k < extra.size(); k++) {
      local[extra[k]] = (int32_t)(n1 - n0 + k);
      p.uniq.push_back(extra[k]);
    }
    for (int64_t t = rowptr[n0]; t < rowptr[n1]; t++) {
      const int32_t end = ends[t];
      p.lother[t] = local[(end & 1) ? m0[end >> 1] : m1[end >> 1]];
    }
    p.max_unique = std::max<int64_t>(p.max_unique, (int64_t)p.uniq.size() - p.uoff[b]);
  }
  p.uoff[p.nblocks] = (int64_t)p.uniq.size();
  const int64_t nslices = (N + 31) / 32;
  p.sell_off.assign((size_t)nslices + 1, 0);
  for (int64_t sl = 0; sl < nslices; sl++) {
    int64_t kmax = 0;
    for (int64_t v = sl * 32; v < std::min<int64_t>(N, sl * 32 + 32); v++)
      kmax = std::max<int64_t>(kmax, rowptr[v + 1] - rowptr[v]);
    p.sell_off[sl + 1] = p.sell_off[sl] + 32 * kmax;
  }
  p.sell_end.assign((size_t)p.sell_off[nslices], -1);
  for (int64_t v = 0; v < N; v++) {
    const int64_t base = p.sell_off[v / 32] + (v % 32);
    for (int64_t t = rowptr[v]; t < rowptr[v + 1]; t++)
      p.sell_end[base + 32 * (t - rowptr[v])] = (int32_t)t;
  }
}

}  // namespace op2b
