// rcm_host.h -- reverse Cuthill-McKee ordering on the host (plan set-up of the block-Jacobi
// preconditioner, Section 5.8: the matrix is reordered with RCM before the blocks are
// taken).  The paper gives no variant, so the rules are fixed here:
//   * the graph is the structure of A + A^T without the diagonal; deg(v) = number of
//     distinct neighbours; vertices are ranked by (deg, index);
//   * components are started in the order of their lowest-ranked vertex s; the start
//     vertex is the pseudo-peripheral vertex of the George-Liu iteration from s (root r =
//     s; x = lowest-ranked vertex of the last BFS level of r; if x's level structure is
//     deeper, r = x and repeat; else x is the start);
//   * the Cuthill-McKee BFS appends the unvisited neighbours of each dequeued vertex in
//     rank order; the whole order is reversed.  perm[new] = old.
// O(nnz log) time, O(nnz) memory.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace gm {

struct RcmGraph {
  int n = 0;
  std::vector<int64_t> off;  // n+1
  std::vector<int> adj;      // sorted, unique neighbour lists
  std::vector<int> deg;
  bool rank_less(int a, int b) const { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; }
};

// Symmetrised neighbour lists of a CSR structure (row_ptr/col_idx validated by the caller).
inline void rcm_graph(int n, const int32_t* rp, const int32_t* ci, RcmGraph& g) {
  g.n = n;
  std::vector<int64_t> cnt(n + 1, 0);
  for (int i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] != i) {
        ++cnt[i + 1];
        ++cnt[ci[p] + 1];
      }
  for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> raw(cnt[n]);
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  for (int i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int j = ci[p];
      if (j != i) {
        raw[fill[i]++] = j;
        raw[fill[j]++] = i;
      }
    }
  g.off.assign(n + 1, 0);
  g.deg.assign(n, 0);
  g.adj.clear();
  g.adj.reserve(raw.size());
  for (int i = 0; i < n; ++i) {
    auto b = raw.begin() + cnt[i], e = raw.begin() + cnt[i + 1];
    std::sort(b, e);
    e = std::unique(b, e);
    g.adj.insert(g.adj.end(), b, e);
    g.off[i + 1] = (int64_t)g.adj.size();
    g.deg[i] = (int)(e - b);
  }
}

// BFS level structure of root's component: returns the number of levels and leaves the
// last level in `last`.  `mark` holds a stamp per vertex (stamp must be fresh).
inline int rcm_levels(const RcmGraph& g, int root, std::vector<int>& mark, int stamp,
                      std::vector<int>& cur, std::vector<int>& nxt, std::vector<int>& last) {
  cur.assign(1, root);
  mark[root] = stamp;
  int depth = 1;
  while (true) {
    nxt.clear();
    for (int u : cur)
      for (int64_t p = g.off[u]; p < g.off[u + 1]; ++p) {
        const int v = g.adj[p];
        if (mark[v] != stamp) {
          mark[v] = stamp;
          nxt.push_back(v);
        }
      }
    if (nxt.empty()) {
      last = cur;
      return depth;
    }
    cur.swap(nxt);
    ++depth;
  }
}

// perm[new] = old for the n vertices.
inline void rcm_order(int n, const int32_t* rp, const int32_t* ci, int32_t* perm) {
  RcmGraph g;
  rcm_graph(n, rp, ci, g);
  std::vector<int> byrank(n);
  for (int i = 0; i < n; ++i) byrank[i] = i;
  std::sort(byrank.begin(), byrank.end(), [&](int a, int b) { return g.rank_less(a, b); });
  std::vector<int> mark(n, 0), cur, nxt, last, nb;
  std::vector<char> visited(n, 0);
  std::vector<int> order;
  order.reserve(n);
  int stamp = 0;
  auto lowest = [&](const std::vector<int>& vs) {
    int best = vs[0];
    for (int v : vs)
      if (g.rank_less(v, best)) best = v;
    return best;
  };
  for (int s : byrank) {
    if (visited[s]) continue;
    // George-Liu pseudo-peripheral vertex of s's component
    int depth_r = rcm_levels(g, s, mark, ++stamp, cur, nxt, last);
    int x;
    while (true) {
      x = lowest(last);
      std::vector<int> last_x;
      const int depth_x = rcm_levels(g, x, mark, ++stamp, cur, nxt, last_x);
      if (depth_x > depth_r) {
        depth_r = depth_x;
        last.swap(last_x);
      } else {
        break;
      }
    }
    // Cuthill-McKee BFS from x
    size_t head = order.size();
    visited[x] = 1;
    order.push_back(x);
    while (head < order.size()) {
      const int u = order[head++];
      nb.clear();
      for (int64_t p = g.off[u]; p < g.off[u + 1]; ++p) {
        const int v = g.adj[p];
        if (!visited[v]) {
          visited[v] = 1;
          nb.push_back(v);
        }
      }
      std::sort(nb.begin(), nb.end(), [&](int a, int b) { return g.rank_less(a, b); });
      order.insert(order.end(), nb.begin(), nb.end());
    }
  }
  for (int i = 0; i < n; ++i) perm[i] = order[n - 1 - i];
}

}  // namespace gm
