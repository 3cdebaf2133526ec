// Symbolic analysis for the sparse LDL^T of K = [I A^T; A -I] (host code; see ldl.h).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <exception>
#include <map>
#include <set>
#include <numeric>
#include <thread>

#include "../../include/pogs.h"
#include "ldl.h"

namespace pogs {
namespace {

// Undirected graph of K without the diagonal: x_j -- y_i for every nonzero A_ij.  eid[p] is the
// CSR index of the A entry behind adjacency entry p.
struct Graph {
  int N = 0;
  std::vector<int> off, adj, eid;
};

Graph build_graph(int m, int n, const int* rp, const int* ci) {
  Graph g;
  g.N = n + m;
  std::vector<int> deg(g.N, 0);
  for (int i = 0; i < m; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      ++deg[ci[p]];
      ++deg[n + i];
    }
  g.off.assign(g.N + 1, 0);
  for (int v = 0; v < g.N; ++v) g.off[v + 1] = g.off[v] + deg[v];
  g.adj.resize(g.off[g.N]);
  g.eid.resize(g.off[g.N]);
  std::vector<int> pos(g.off.begin(), g.off.end() - 1);
  for (int i = 0; i < m; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      g.eid[pos[ci[p]]] = p;
      g.adj[pos[ci[p]]++] = n + i;   // x_j's neighbours: rows in increasing order
      g.eid[pos[n + i]] = p;
      g.adj[pos[n + i]++] = ci[p];   // y_i's neighbours: columns in increasing order
    }
  return g;
}

// Runs f(bounds[w], bounds[w + 1], w) for every w on its own host thread (w = 0 on the calling
// thread, and any chunk whose thread cannot be started); returns the first nonzero code, in chunk
// order.  A chunk that throws (an allocation failure) reports POGS_ERR_OOM instead.
template <class F>
int parallel_ranges(const std::vector<int>& bounds, F f) {
  const int nw = (int)bounds.size() - 1;
  if (nw < 1) return 0;
  std::vector<int> rc(nw, 0);
  auto chunk = [&](int w) {
    try {
      rc[w] = f(bounds[w], bounds[w + 1], w);
    } catch (...) {
      rc[w] = POGS_ERR_OOM;
    }
  };
  std::vector<std::thread> th;
  int started = 1;
  try {
    for (; started < nw; ++started) th.emplace_back(chunk, started);
  } catch (...) {   // no more threads: the remaining chunks run here
  }
  chunk(0);
  for (int w = started; w < nw; ++w) chunk(w);
  for (auto& t : th) t.join();
  for (int r : rc)
    if (r) return r;
  return 0;
}

// parallel_ranges over [0, count) cut into up to 16 equal contiguous chunks of at least `grain`
// items (one chunk on the calling thread when count is small).
template <class F>
int parallel_chunks(int count, int grain, F f) {
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nw = std::min({16, hw, std::max(1, count / std::max(1, grain))});
  std::vector<int> bounds(nw + 1);
  for (int w = 0; w <= nw; ++w) bounds[w] = (int)((int64_t)count * w / nw);
  return parallel_ranges(bounds, f);
}

// Cut [0, cost.size()) into at most `parts` contiguous ranges of about equal total cost.
std::vector<int> balanced_bounds(const std::vector<int64_t>& cost, int parts) {
  int64_t total = 0;
  for (int64_t c : cost) total += c;
  std::vector<int> b{0};
  int64_t acc = 0;
  for (int i = 0; i < (int)cost.size(); ++i) {
    acc += cost[i];
    if ((int)b.size() < parts && acc * parts >= total * (int64_t)b.size() && i + 1 < (int)cost.size()) b.push_back(i + 1);
  }
  b.push_back((int)cost.size());
  return b;
}

// Nested dissection by breadth-first level structures.  A connected part is split at the level
// that holds the middle node of a BFS from a pseudo-peripheral node; that level is a vertex
// separator and is ordered after both halves.  Disconnected parts are ordered one after another,
// parts of at most kLeaf nodes in their given order.  Nodes of very high degree (dense rows or
// columns of A, such as the coupling rows of a block-angular matrix) are taken out first and
// ordered last.
class Dissection {
 public:
  static constexpr int kLeaf = 8;
  // Below a separator the two halves touch disjoint nodes (a half's neighbours lie in that half or
  // in separators already ordered), so halves of at least kParallelMin nodes each are ordered on two
  // threads, down to par_depth_ levels of the recursion; the result is the same as in one thread.
  static constexpr int kParallelMin = 16384;
  explicit Dissection(const Graph& g) : g_(g), tag_(g.N, 0) {
    const unsigned hw = std::thread::hardware_concurrency();
    while (par_depth_ < 4 && (2u << par_depth_) <= hw) ++par_depth_;
  }

  std::vector<int> order() {
    const int N = g_.N;
    std::vector<int> out;
    out.reserve(N);
    if (N == 0) return out;
    const double avg = (double)g_.adj.size() / N;
    const int dense_deg = std::max(64, (int)(10.0 * avg));
    std::vector<int> rest, dense;
    for (int v = 0; v < N; ++v) (g_.off[v + 1] - g_.off[v] > dense_deg ? dense : rest).push_back(v);
    for (int v : dense) tag_[v] = -1;   // excluded from every part
    dissect(rest, out, 0);
    for (int v : dense) out.push_back(v);
    return out;
  }

 private:
  const Graph& g_;
  std::vector<int> tag_;
  std::atomic<int> cur_{0};
  int par_depth_ = 0;

  int new_tag() { return cur_.fetch_add(1, std::memory_order_relaxed) + 1; }

  // Level structure of a BFS: the nodes in visiting order, and the start of each level in it
  // (lo.back() == q.size()).
  struct Levels {
    std::vector<int> q, lo;
    int count() const { return (int)lo.size() - 1; }
    const int* begin(int l) const { return q.data() + lo[l]; }
    const int* end(int l) const { return q.data() + lo[l + 1]; }
  };

  // BFS over the nodes tagged t from s (neighbours in adjacency order, level by level).  Visited
  // nodes are tagged `seen`; with restore they get t back at the end.
  void bfs(int s, int t, int seen, bool restore, Levels& L) {
    L.q.clear();
    L.lo.clear();
    L.q.push_back(s);
    tag_[s] = seen;
    size_t b = 0;
    while (b < L.q.size()) {
      const size_t e = L.q.size();
      L.lo.push_back((int)b);
      for (size_t k = b; k < e; ++k) {
        const int v = L.q[k];
        for (int p = g_.off[v]; p < g_.off[v + 1]; ++p) {
          const int u = g_.adj[p];
          if (tag_[u] == t) {
            tag_[u] = seen;
            L.q.push_back(u);
          }
        }
      }
      b = e;
    }
    L.lo.push_back((int)L.q.size());
    if (restore)
      for (int v : L.q) tag_[v] = t;
  }

  // Appends the order of `nodes` (increasing node numbers) to out.
  void dissect(const std::vector<int>& nodes, std::vector<int>& out, int depth) {
    if ((int)nodes.size() <= kLeaf) {
      out.insert(out.end(), nodes.begin(), nodes.end());
      return;
    }
    const int t = new_tag();
    for (int v : nodes) tag_[v] = t;
    // connected parts, each moved to a tag of its own as it is found
    std::vector<std::vector<int>> parts;
    std::vector<int> ptag;
    Levels levels;
    int tpart = t;
    for (int v : nodes) {
      if (tag_[v] != t) continue;
      tpart = new_tag();
      bfs(v, t, tpart, false, levels);
      parts.push_back(levels.q);
      ptag.push_back(tpart);
    }
    if (parts.size() > 1) {
      // each part in increasing node order: one walk over the (increasing) input; the parts' tags
      // increase in the order the parts were found
      for (auto& part : parts) part.clear();
      for (int v : nodes) parts[std::lower_bound(ptag.begin(), ptag.end(), tag_[v]) - ptag.begin()].push_back(v);
      for (auto& part : parts) dissect(part, out, depth);
      return;
    }
    // one connected part (tag tpart): pseudo-peripheral start, the last node of a BFS, repeated
    // while the depth grows
    int start = *levels.begin(levels.count() - 1);
    int bfs_depth = levels.count();
    Levels l2;
    for (int it = 0; it < 4; ++it) {
      bfs(start, tpart, new_tag(), true, l2);
      if (l2.count() <= bfs_depth) break;
      bfs_depth = l2.count();
      std::swap(levels, l2);
      start = *levels.begin(levels.count() - 1);
    }
    if (levels.count() < 3) {         // nearly a clique: no useful separator
      out.insert(out.end(), nodes.begin(), nodes.end());
      return;
    }
    const int half = (int)nodes.size() / 2;
    int acc = 0, L = 1;
    for (int l = 0; l < levels.count(); ++l) {
      acc += levels.lo[l + 1] - levels.lo[l];
      if (acc > half) {
        L = l;
        break;
      }
    }
    L = std::max(1, std::min(L, levels.count() - 2));
    // levels [0, L) | level L (the separator) | levels (L, end), each in increasing node order
    const int t1 = new_tag(), ts = new_tag();
    for (const int* v = levels.begin(0); v != levels.begin(L); ++v) tag_[*v] = t1;
    for (const int* v = levels.begin(L); v != levels.end(L); ++v) tag_[*v] = ts;
    std::vector<int> p1, p2, sep;
    p1.reserve(levels.lo[L]);
    sep.reserve(levels.lo[L + 1] - levels.lo[L]);
    p2.reserve(nodes.size() - levels.lo[L + 1]);
    for (int v : nodes) (tag_[v] == t1 ? p1 : tag_[v] == ts ? sep : p2).push_back(v);
    levels = Levels();
    l2 = Levels();
    std::vector<int> out1;
    std::exception_ptr err1;   // an exception of the other thread, rethrown here after the join
    std::thread th;
    if (depth < par_depth_ && (int)p1.size() >= kParallelMin && (int)p2.size() >= kParallelMin) {
      try {
        th = std::thread([&] {
          try {
            dissect(p1, out1, depth + 1);
          } catch (...) {
            err1 = std::current_exception();
          }
        });
      } catch (...) {   // no thread available: order both halves here
      }
    }
    if (!th.joinable()) {
      dissect(p1, out, depth + 1);
      dissect(p2, out, depth + 1);
    } else {
      std::vector<int> out2;
      try {
        dissect(p2, out2, depth + 1);
      } catch (...) {
        th.join();
        throw;
      }
      th.join();
      if (err1) std::rethrow_exception(err1);
      out.insert(out.end(), out1.begin(), out1.end());
      out.insert(out.end(), out2.begin(), out2.end());
    }
    out.insert(out.end(), sep.begin(), sep.end());
  }
};

}  // namespace

namespace {

int analyze(int m, int n, const int* rp, const int* ci, LdlSymbolic& S) {
  if (m < 1 || n < 1 || !rp || !ci || rp[0] != 0) return POGS_ERR_ARG;
  for (int i = 0; i < m; ++i) {
    if (rp[i + 1] < rp[i]) return POGS_ERR_ARG;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] < 0 || ci[p] >= n || (p > rp[i] && ci[p] <= ci[p - 1])) return POGS_ERR_ARG;
  }
  S = LdlSymbolic();
  S.n = n;
  S.m = m;
  const int N = S.N = n + m;
  Graph pg;   // the graph in the new numbering (neighbours of each node in their order in g)
  {
    const Graph g = build_graph(m, n, rp, ci);
    // ---- ordering -----------------------------------------------------------------------------
    S.perm = Dissection(g).order();
    S.iperm.assign(N, -1);
    for (int k = 0; k < N; ++k) S.iperm[S.perm[k]] = k;
    pg.N = N;
    pg.off.assign(N + 1, 0);
    for (int k = 0; k < N; ++k) pg.off[k + 1] = pg.off[k] + (g.off[S.perm[k] + 1] - g.off[S.perm[k]]);
    pg.adj.resize(g.adj.size());
    pg.eid.resize(g.eid.size());
    parallel_chunks(N, 8192, [&](int b, int e, int) -> int {
      for (int k = b; k < e; ++k) {
        const int v = S.perm[k];
        for (int p = g.off[v], q = pg.off[k]; p < g.off[v + 1]; ++p, ++q) {
          pg.adj[q] = S.iperm[g.adj[p]];
          pg.eid[q] = g.eid[p];
        }
      }
      return 0;
    });
  }
  // ---- elimination tree (ancestor links with path compression) ------------------------------
  S.parent.assign(N, -1);
  {
    std::vector<int> anc(N, -1);
    for (int k = 0; k < N; ++k) {
      for (int p = pg.off[k]; p < pg.off[k + 1]; ++p) {
        int i = pg.adj[p];
        while (i != -1 && i < k) {
          const int next = anc[i];
          anc[i] = k;
          if (next == -1) S.parent[i] = k;
          i = next;
        }
      }
    }
  }
  // ---- column counts ----------------------------------------------------------------------------
  // cc(j) = |struct(j)| + 1 is the number of row subtrees T_r(i) (the columns k with L_ik != 0, a
  // subtree of the elimination tree rooted at i) that contain j.  Each T_r(i) is given weight +1 at
  // every leaf, -1 at the lowest common ancestor of each pair of leaves adjacent in postorder and -1
  // at parent(i); the weights summed over the subtree of j then count the row subtrees through j
  // (Gilbert, Ng and Peyton's row/column count method).  Leaves are found in one postorder sweep
  // (k is a leaf of T_r(i) when no earlier member of T_r(i) lies in the subtree of k), ancestors by
  // a disjoint-set forest of the finished nodes.
  S.colcount.resize(N);
  {
    std::vector<int> head(N, -1), nxt(N, -1), post, first(N, -1);
    post.reserve(N);
    for (int j = N - 1; j >= 0; --j)
      if (S.parent[j] >= 0) {
        nxt[j] = head[S.parent[j]];
        head[S.parent[j]] = j;
      }
    std::vector<int> stack;
    for (int r = 0; r < N; ++r) {
      if (S.parent[r] >= 0) continue;
      stack.push_back(r);
      while (!stack.empty()) {
        const int v = stack.back(), c = head[v];
        if (c >= 0) {
          head[v] = nxt[c];
          stack.push_back(c);
        } else {
          stack.pop_back();
          post.push_back(v);
        }
      }
    }
    for (int k = 0; k < N; ++k)
      for (int u = post[k]; u >= 0 && first[u] < 0; u = S.parent[u]) first[u] = k;
    std::vector<int> delta(N, 0), maxfirst(N, -1), prevleaf(N, -1), uf(N);
    std::iota(uf.begin(), uf.end(), 0);
    auto find = [&](int x) {
      int r = x;
      while (uf[r] != r) r = uf[r];
      while (uf[x] != r) {
        const int nx = uf[x];
        uf[x] = r;
        x = nx;
      }
      return r;
    };
    for (int k = 0; k < N; ++k) {
      const int j = post[k];
      if (S.parent[j] >= 0) --delta[S.parent[j]];
      for (int p = pg.off[j]; p < pg.off[j + 1]; ++p) {
        const int i = pg.adj[p];
        if (i <= j || first[j] <= maxfirst[i]) continue;
        ++delta[j];              // j is a leaf of T_r(i)
        maxfirst[i] = first[j];
        if (prevleaf[i] >= 0) --delta[find(prevleaf[i])];
        prevleaf[i] = j;
      }
      if (maxfirst[j] < first[j]) ++delta[j];   // T_r(j) = {j}
      if (S.parent[j] >= 0) uf[j] = S.parent[j];
    }
    for (int k = 0; k < N; ++k) {
      const int j = post[k];
      if (S.parent[j] >= 0) delta[S.parent[j]] += delta[j];
      S.colcount[j] = delta[j] - 1;
    }
  }
  // ---- supernodes: fundamental, then chains merged while small and with little zero fill ------
  std::vector<int> nkids(N, 0);
  for (int j = 0; j < N; ++j)
    if (S.parent[j] >= 0) ++nkids[S.parent[j]];
  std::vector<int> sfirst, swidth;
  for (int j = 0; j < N;) {
    int l = j;
    while (l + 1 < N && S.parent[l] == l + 1 && nkids[l + 1] == 1 && S.colcount[l] == S.colcount[l + 1] + 1) ++l;
    sfirst.push_back(j);
    swidth.push_back(l - j + 1);
    j = l + 1;
  }
  // merge supernode s into the next one when it is that one's only child, the two are contiguous
  // and small, and the zeros added to s's columns stay below half of the merged panel
  {
    std::vector<int> f2, w2;
    int i = 0;
    const int cnt = (int)sfirst.size();
    while (i < cnt) {
      int f = sfirst[i], w = swidth[i];
      while (i + 1 < cnt) {
        const int l = f + w - 1, fp = sfirst[i + 1], wp = swidth[i + 1];
        if (S.parent[l] != fp || nkids[fp] != 1 || w + wp > 32) break;
        const int64_t hp = S.colcount[fp + wp - 1];
        const int64_t h_s = S.colcount[l];
        // each of s's w columns grows from (its own) to wp + hp rows below the merged block
        const int64_t zeros = (int64_t)w * (wp + hp - h_s);
        const int64_t panel = (int64_t)(w + wp) * (w + wp + hp);
        if (2 * zeros > panel) break;
        w += wp;
        ++i;
      }
      f2.push_back(f);
      w2.push_back(w);
      ++i;
    }
    sfirst.swap(f2);
    swidth.swap(w2);
  }
  const int ns = S.ns = (int)sfirst.size();
  S.first = sfirst;
  S.width = swidth;
  std::vector<int> col2sn(N);
  for (int s = 0; s < ns; ++s)
    for (int j = sfirst[s]; j < sfirst[s] + swidth[s]; ++j) col2sn[j] = s;
  S.sparent.assign(ns, -1);
  for (int s = 0; s < ns; ++s) {
    const int p = S.parent[sfirst[s] + swidth[s] - 1];
    S.sparent[s] = p >= 0 ? col2sn[p] : -1;
  }
  // children lists (increasing), levels (leaves 0, parent = 1 + max over children)
  S.child_off.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s)
    if (S.sparent[s] >= 0) ++S.child_off[S.sparent[s] + 1];
  for (int s = 0; s < ns; ++s) S.child_off[s + 1] += S.child_off[s];
  S.child.resize(S.child_off[ns]);
  {
    std::vector<int> pos(S.child_off.begin(), S.child_off.end() - 1);
    for (int s = 0; s < ns; ++s)
      if (S.sparent[s] >= 0) S.child[pos[S.sparent[s]]++] = s;
  }
  S.level.assign(ns, 0);
  for (int s = 0; s < ns; ++s)   // children have smaller indices than their parent
    if (S.sparent[s] >= 0) S.level[S.sparent[s]] = std::max(S.level[S.sparent[s]], S.level[s] + 1);
  S.levels = ns ? 1 + *std::max_element(S.level.begin(), S.level.end()) : 0;
  S.level_off.assign(S.levels + 1, 0);
  for (int s = 0; s < ns; ++s) ++S.level_off[S.level[s] + 1];
  for (int l = 0; l < S.levels; ++l) S.level_off[l + 1] += S.level_off[l];
  S.level_nodes.resize(ns);
  {
    std::vector<int> pos(S.level_off.begin(), S.level_off.end() - 1);
    for (int s = 0; s < ns; ++s) S.level_nodes[pos[S.level[s]]++] = s;
  }
  // ---- row structures of the supernodes -------------------------------------------------------
  // The columns of a supernode form a chain of the elimination tree, so the subtree of its last
  // column l is its own columns plus the subtrees of its child supernodes' last columns, and
  // struct(l) = {i > l : i a neighbour of one of its columns, or a row of a child supernode}.
  S.row_off.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) S.row_off[s + 1] = S.row_off[s] + S.colcount[sfirst[s] + swidth[s] - 1];
  S.rows.resize(S.row_off[ns]);
  // Supernodes of one level of the supernodal tree are independent (their children lie in lower
  // levels): the levels from the leaves up, while they hold many supernodes, are done on several
  // threads, each with its own marker array; the rest in index order on this thread (children
  // before parents, and a supernode's children's rows are usually still in cache).
  std::vector<std::vector<int>> marks(16), tmps(16);
  // The rows of s in increasing order: its columns' later neighbours (sorted), then each child's
  // rows not yet present, a sorted run merged in (with many children, one sort at the end).
  auto rows_of = [&](int s, std::vector<int>& mark, std::vector<int>& tmp) -> int {
    const int f = sfirst[s], l = f + swidth[s] - 1;
    const bool merge = S.child_off[s + 1] - S.child_off[s] <= 16;
    tmp.clear();
    for (int j = f; j <= l; ++j)
      for (int p = pg.off[j]; p < pg.off[j + 1]; ++p) {
        const int i = pg.adj[p];
        if (i > l && mark[i] != s) {
          mark[i] = s;
          tmp.push_back(i);
        }
      }
    if (merge) std::sort(tmp.begin(), tmp.end());
    for (int c = S.child_off[s]; c < S.child_off[s + 1]; ++c) {
      const int ch = S.child[c];
      const size_t mid = tmp.size();
      for (int a = S.row_off[ch]; a < S.row_off[ch + 1]; ++a) {
        const int i = S.rows[a];
        if (i > l && mark[i] != s) {
          mark[i] = s;
          tmp.push_back(i);
        }
      }
      if (merge && mid > 0 && mid < tmp.size()) std::inplace_merge(tmp.begin(), tmp.begin() + mid, tmp.end());
    }
    if ((int)tmp.size() != S.row_off[s + 1] - S.row_off[s]) return POGS_ERR_ARG;   // counts disagree: cannot happen
    if (!merge) std::sort(tmp.begin(), tmp.end());
    std::copy(tmp.begin(), tmp.end(), S.rows.begin() + S.row_off[s]);
    return 0;
  };
  int wide = 0;   // levels [0, wide) done in parallel
  for (; wide < S.levels && S.level_off[wide + 1] - S.level_off[wide] >= 2048; ++wide) {
    const int lb = S.level_off[wide];
    const int rc = parallel_chunks(S.level_off[wide + 1] - lb, 1024, [&](int b, int e, int wk) -> int {
      if (marks[wk].empty()) marks[wk].assign(N, -1);
      for (int k = lb + b; k < lb + e; ++k) {
        const int r = rows_of(S.level_nodes[k], marks[wk], tmps[wk]);
        if (r) return r;
      }
      return 0;
    });
    if (rc) return rc;
  }
  if (marks[0].empty()) marks[0].assign(N, -1);
  for (int s = 0; s < ns; ++s)
    if (S.level[s] >= wide) {
      const int r = rows_of(s, marks[0], tmps[0]);
      if (r) return r;
    }
  // ---- index maps: children's rows in the parent's front; original entries of K -----------------
  // Supernode by supernode, fpos holds the front position of each of its rows (own columns first,
  // then its row structure) while its children's rows and its original entries are looked up.
  S.rel_off.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) S.rel_off[s + 1] = S.rel_off[s] + (S.sparent[s] >= 0 ? S.row_off[s + 1] - S.row_off[s] : 0);
  S.rel.resize(S.rel_off[ns]);
  // entries per supernode (each own column's diagonal and its neighbours below it), then every
  // supernode's entries at its offset, supernodes in contiguous chunks on several threads
  S.asm_off.assign(ns + 1, 0);
  parallel_chunks(ns, 1024, [&](int b, int e, int) -> int {
    for (int s = b; s < e; ++s) {
      int c = 0;
      for (int j = sfirst[s]; j < sfirst[s] + swidth[s]; ++j) {
        ++c;
        for (int p = pg.off[j]; p < pg.off[j + 1]; ++p) c += pg.adj[p] > j;
      }
      S.asm_off[s + 1] = c;
    }
    return 0;
  });
  for (int s = 0; s < ns; ++s) S.asm_off[s + 1] += S.asm_off[s];
  S.asm_pos.assign(S.asm_off[ns], 0);
  S.asm_src.assign(S.asm_off[ns], 0);
  std::vector<int64_t> cost(ns);   // a supernode's share: its entries, rows and children's rows
  for (int s = 0; s < ns; ++s) {
    cost[s] = (S.asm_off[s + 1] - S.asm_off[s]) + 2 * (S.row_off[s + 1] - S.row_off[s]) + swidth[s];
    for (int c = S.child_off[s]; c < S.child_off[s + 1]; ++c) cost[s] += S.row_off[S.child[c] + 1] - S.row_off[S.child[c]];
  }
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int mrc = parallel_ranges(balanced_bounds(cost, std::min({16, hw, std::max(1, ns / 1024)})),
                                  [&](int b, int e, int wk) -> int {
    std::vector<int>& fpos = marks[wk];   // front position of each row of the current supernode
    if (fpos.empty()) fpos.assign(N, -1);
    std::fill(fpos.begin(), fpos.end(), -1);
    for (int s = b; s < e; ++s) {
      const int f = sfirst[s], w = swidth[s];
      const int nf = w + (S.row_off[s + 1] - S.row_off[s]);
      for (int j = f; j < f + w; ++j) fpos[j] = j - f;
      for (int a = S.row_off[s]; a < S.row_off[s + 1]; ++a) fpos[S.rows[a]] = w + (a - S.row_off[s]);
      for (int c = S.child_off[s]; c < S.child_off[s + 1]; ++c) {
        const int ch = S.child[c];
        for (int a = S.row_off[ch]; a < S.row_off[ch + 1]; ++a) {
          const int loc = fpos[S.rows[a]];
          if (loc < 0) return POGS_ERR_ARG;   // cannot happen for an elimination tree
          S.rel[S.rel_off[ch] + (a - S.row_off[ch])] = loc;
        }
      }
      int t = S.asm_off[s];
      for (int j = f; j < f + w; ++j) {
        const int lc = j - f;
        S.asm_pos[t] = lc * nf + lc;
        S.asm_src[t++] = S.perm[j] < n ? -1 : -2;
        for (int p = pg.off[j]; p < pg.off[j + 1]; ++p) {
          const int i = pg.adj[p];
          if (i <= j) continue;
          const int lr = fpos[i];
          if (lr < 0) return POGS_ERR_ARG;
          S.asm_pos[t] = lr * nf + lc;
          S.asm_src[t++] = pg.eid[p];   // the A entry linking the two unknowns
        }
      }
      for (int j = f; j < f + w; ++j) fpos[j] = -1;
      for (int a = S.row_off[s]; a < S.row_off[s + 1]; ++a) fpos[S.rows[a]] = -1;
    }
    return 0;
  });
  if (mrc) return mrc;
  // ---- storage ----------------------------------------------------------------------------------
  S.panel_off.assign(ns + 1, 0);
  S.upd_off.assign(ns, 0);
  S.front_off.assign(ns, 0);
  S.vec_off.assign(ns + 1, 0);
  S.nnz_l = 0;
  S.max_front = 0;
  S.smem_front_max = 0;
  auto nf_of = [&](int s) { return (int64_t)swidth[s] + (S.row_off[s + 1] - S.row_off[s]); };
  for (int s = 0; s < ns; ++s) {
    const int64_t w = swidth[s], h = S.row_off[s + 1] - S.row_off[s], nf = w + h;
    S.panel_off[s + 1] = S.panel_off[s] + nf * w;
    S.vec_off[s + 1] = S.vec_off[s] + (int)h;
    S.nnz_l += w * (w - 1) / 2 + w * h;
    S.max_front = std::max<int>(S.max_front, (int)nf);
    if (nf <= LdlSymbolic::kSmemFront) S.smem_front_max = std::max<int>(S.smem_front_max, (int)nf);
  }
  // shared-memory fronts first within each level; global fronts get scratch offsets
  S.level_split.assign(S.levels, 0);
  S.front_max = 0;
  for (int l = 0; l < S.levels; ++l) {
    auto b = S.level_nodes.begin() + S.level_off[l], e = S.level_nodes.begin() + S.level_off[l + 1];
    std::stable_partition(b, e, [&](int s) { return nf_of(s) <= LdlSymbolic::kSmemFront; });
    int64_t acc = 0;
    int split = S.level_off[l + 1];
    for (int k = S.level_off[l]; k < S.level_off[l + 1]; ++k) {
      const int s = S.level_nodes[k];
      if (nf_of(s) <= LdlSymbolic::kSmemFront) continue;
      split = std::min(split, k);
      S.front_off[s] = acc;
      acc += nf_of(s) * nf_of(s);
    }
    S.level_split[l] = split;
    S.front_max = std::max(S.front_max, acc);
  }
  // update matrices: an arena with best-fit reuse (the smallest free block that holds the
  // update, lowest offset among equals; free neighbours merge).  The update of s is written at
  // level(s) and read at level(parent(s)); its space is free again from the level after that.
  {
    std::map<int64_t, int64_t> free_by_off;            // offset -> size
    std::set<std::pair<int64_t, int64_t>> free_by_size;  // (size, offset)
    int64_t end = 0;
    std::vector<std::vector<int>> release_after(S.levels + 1);
    auto insert = [&](int64_t off, int64_t size) {
      free_by_off[off] = size;
      free_by_size.insert({size, off});
    };
    auto erase = [&](std::map<int64_t, int64_t>::iterator it) {
      free_by_size.erase({it->second, it->first});
      return free_by_off.erase(it);
    };
    auto take = [&](int64_t size) -> int64_t {
      auto fit = free_by_size.lower_bound({size, INT64_MIN});
      if (fit == free_by_size.end()) {
        const int64_t off = end;
        end += size;
        return off;
      }
      const int64_t off = fit->second, rest = fit->first - size;
      erase(free_by_off.find(off));
      if (rest > 0) insert(off + size, rest);
      return off;
    };
    auto give = [&](int64_t off, int64_t size) {
      auto nx = free_by_off.lower_bound(off);
      if (nx != free_by_off.end() && off + size == nx->first) {
        size += nx->second;
        nx = erase(nx);
      }
      if (nx != free_by_off.begin()) {
        auto pv = std::prev(nx);
        if (pv->first + pv->second == off) {
          off = pv->first;
          size += pv->second;
          erase(pv);
        }
      }
      insert(off, size);
    };
    for (int l = 0; l < S.levels; ++l) {
      if (l > 0)   // read at level l - 1, which has completed before level l starts
        for (int s : release_after[l - 1]) {
          const int64_t h = S.row_off[s + 1] - S.row_off[s];
          give(S.upd_off[s], h * h);
        }
      for (int k = S.level_off[l]; k < S.level_off[l + 1]; ++k) {
        const int s = S.level_nodes[k];
        const int64_t h = S.row_off[s + 1] - S.row_off[s];
        if (h == 0 || S.sparent[s] < 0) continue;
        S.upd_off[s] = take(h * h);
        release_after[S.level[S.sparent[s]]].push_back(s);
      }
    }
    S.upd_total = end;
  }
  S.panel_total = S.panel_off[ns];
  S.vec_total = S.vec_off[ns];
  return 0;
}

}  // namespace

int ldl_analyze(int m, int n, const int* rp, const int* ci, LdlSymbolic& S) {
  try {
    return analyze(m, n, rp, ci, S);
  } catch (...) {   // host memory exhausted (the analysis allocates all its work arrays)
    S = LdlSymbolic();
    return POGS_ERR_OOM;
  }
}

}  // namespace pogs

// ---- C ABI: the symbolic analysis alone (host only, no device work) ------------------------------
extern "C" int pogs_ldl_analyze(int64_t m, int64_t n, const int* rowptr, const int* colind, int64_t* stats,
                                int* perm, int* colcount) {
  if (m < 1 || n < 1 || m + n > (int64_t)1 << 30 || !rowptr || !colind) return POGS_ERR_ARG;
  pogs::LdlSymbolic S;
  const int rc = pogs::ldl_analyze((int)m, (int)n, rowptr, colind, S);
  if (rc != 0) return rc;
  if (stats) {
    stats[0] = S.N;
    stats[1] = S.nnz_l;
    stats[2] = S.ns;
    stats[3] = S.levels;
    stats[4] = S.max_front;
    stats[5] = S.panel_total;
    stats[6] = S.upd_total;
    stats[7] = S.front_max;
  }
  if (perm) std::memcpy(perm, S.perm.data(), sizeof(int) * S.N);
  if (colcount) std::memcpy(colcount, S.colcount.data(), sizeof(int) * S.N);
  return 0;
}
