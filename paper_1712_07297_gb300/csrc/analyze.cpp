// Host analysis: recursive coordinate bisection (Alg. 1, partition step),
// block pattern A_B of a level (Eq. quotient) with the distance-2 clusters
// where fill-in can appear (Sec. 2.3), and the greedy distance-2 colouring
// that turns the independence rule of Sec. 3.2 into batches of clusters.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <queue>

#include "common.h"

namespace hs {

int round_up(int x, int a) { return (x + a - 1) / a * a; }

int rcb_leaves(int64_t n, const double* coords, int dim, int leaf,
               std::vector<std::vector<int64_t>>& leaves) {
  int depth = 0;
  while ((n + (int64_t(1) << depth) - 1) / (int64_t(1) << depth) > leaf) depth++;
  std::vector<std::vector<int64_t>> nodes(1);
  nodes[0].resize(n);
  std::iota(nodes[0].begin(), nodes[0].end(), int64_t(0));
  for (int d = 0; d < depth; d++) {
    std::vector<std::vector<int64_t>> nxt;
    nxt.reserve(nodes.size() * 2);
    for (auto& idx : nodes) {
      if (idx.empty()) {
        nxt.emplace_back();
        nxt.emplace_back();
        continue;
      }
      // longest bounding-box axis, lowest axis on ties; without coordinates
      // the global index is the only coordinate
      int ax = 0;
      if (coords) {
        double best = -1.0;
        for (int a = 0; a < dim; a++) {
          double lo = coords[idx[0] * dim + a], hi = lo;
          for (int64_t p : idx) {
            double c = coords[p * dim + a];
            lo = std::min(lo, c);
            hi = std::max(hi, c);
          }
          if (hi - lo > best) {
            best = hi - lo;
            ax = a;
          }
        }
      }
      std::vector<int64_t> ord = idx;
      if (coords) {
        std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
          double ca = coords[a * dim + ax], cb = coords[b * dim + ax];
          return ca < cb || (ca == cb && a < b);
        });
      } else {
        std::sort(ord.begin(), ord.end());
      }
      size_t half = ord.size() / 2;
      nxt.emplace_back(ord.begin(), ord.begin() + half);
      nxt.emplace_back(ord.begin() + half, ord.end());
    }
    nodes.swap(nxt);
  }
  for (auto& v : nodes) std::sort(v.begin(), v.end());
  leaves.swap(nodes);
  return depth;
}

int64_t LevelPattern::find(int i, int j) const {
  auto b = col.begin() + ptr[i], e = col.begin() + ptr[i + 1];
  auto it = std::lower_bound(b, e, j);
  if (it == e || *it != j) return -1;
  return it - col.begin();
}

void build_level_pattern(LevelPattern& L, const std::vector<std::vector<int>>& adj) {
  const int nc = L.nclu;
  L.ld.resize(nc);
  L.voff.assign(nc + 1, 0);
  for (int i = 0; i < nc; i++) {
    L.ld[i] = std::max(4, round_up(L.m[i], 4));
    L.voff[i + 1] = L.voff[i] + L.m[i];
  }
  // distance-2 sets and the pattern rows
  L.ptr.assign(nc + 1, 0);
  L.col.clear();
  L.kind.clear();
  std::vector<int> mark(nc, -1);
  std::vector<std::vector<int>> d2(nc);
  for (int i = 0; i < nc; i++) {
    mark[i] = i;
    for (int j : adj[i]) mark[j] = i;
    std::vector<int> row;
    for (int j : adj[i])
      for (int q : adj[j])
        if (mark[q] != i) {
          mark[q] = i;
          d2[i].push_back(q);
        }
    std::sort(d2[i].begin(), d2[i].end());
    // merge self, neighbours, distance 2 into one sorted row
    std::vector<std::pair<int, int8_t>> ent;
    ent.emplace_back(i, 0);
    for (int j : adj[i]) ent.emplace_back(j, 1);
    for (int j : d2[i]) ent.emplace_back(j, 2);
    std::sort(ent.begin(), ent.end());
    for (auto& e : ent) {
      L.col.push_back(e.first);
      L.kind.push_back(e.second);
    }
    L.ptr[i + 1] = (int)L.col.size();
  }
  L.off.resize(L.col.size());
  int64_t o = 0;
  for (int i = 0; i < nc; i++)
    for (int p = L.ptr[i]; p < L.ptr[i + 1]; p++) {
      L.off[p] = o;
      o += int64_t(L.ld[i]) * std::max(L.m[L.col[p]], 1);
    }
  L.arena_elems = std::max<int64_t>(o, 1);
  // greedy distance-2 colouring in smallest-last order: remove the cluster
  // with the fewest remaining distance-<=2 neighbours (ties: lowest index)
  // until none is left; colour in reverse removal order, each cluster taking
  // the smallest colour unused by its coloured distance-<=2 neighbours
  std::vector<int> deg(nc), order;
  order.reserve(nc);
  for (int i = 0; i < nc; i++) deg[i] = L.ptr[i + 1] - L.ptr[i] - 1;  // row minus self
  std::priority_queue<std::pair<int, int>, std::vector<std::pair<int, int>>,
                      std::greater<std::pair<int, int>>>
      heap;
  for (int i = 0; i < nc; i++) heap.emplace(deg[i], i);
  std::vector<char> removed(nc, 0);
  while (!heap.empty()) {
    const auto [d, i] = heap.top();
    heap.pop();
    if (removed[i] || d != deg[i]) continue;  // a stale entry
    removed[i] = 1;
    order.push_back(i);
    for (int p = L.ptr[i]; p < L.ptr[i + 1]; p++) {
      const int j = L.col[p];
      if (j != i && !removed[j]) heap.emplace(--deg[j], j);
    }
  }
  std::reverse(order.begin(), order.end());
  L.colour.assign(nc, -1);
  int ncol = 0;
  std::vector<int> used(1, -1);
  for (int i : order) {
    for (int p = L.ptr[i]; p < L.ptr[i + 1]; p++) {
      int j = L.col[p];
      if (j != i && L.colour[j] >= 0) {
        if ((int)used.size() <= L.colour[j]) used.resize(L.colour[j] + 1, -1);
        used[L.colour[j]] = i;
      }
    }
    int c = 0;
    while (c < (int)used.size() && used[c] == i) c++;
    L.colour[i] = c;
    ncol = std::max(ncol, c + 1);
  }
  L.classes.assign(ncol, {});
  for (int i = 0; i < nc; i++) L.classes[L.colour[i]].push_back(i);
}

}  // namespace hs
