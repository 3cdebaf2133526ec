// Symbolic analysis for the sparse LDL^T of K = [I A^T; A -I] (host code; see ldl.h).
#include <algorithm>
#include <cstring>
#include <map>
#include <set>
#include <numeric>

#include "../../include/pogs.h"
#include "ldl.h"

namespace pogs {
namespace {

// Undirected graph of K without the diagonal: x_j -- y_i for every nonzero A_ij.
struct Graph {
  int N = 0;
  std::vector<int> off, adj;
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
  std::vector<int> pos(g.off.begin(), g.off.end() - 1);
  for (int i = 0; i < m; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      g.adj[pos[ci[p]]++] = n + i;   // x_j's neighbours: rows in increasing order
      g.adj[pos[n + i]++] = ci[p];   // y_i's neighbours: columns in increasing order
    }
  return g;
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
  explicit Dissection(const Graph& g) : g_(g), tag_(g.N, 0), lvl_(g.N, -1) {}

  std::vector<int> order() {
    const int N = g_.N;
    out_.clear();
    out_.reserve(N);
    if (N == 0) return out_;
    const double avg = (double)g_.adj.size() / N;
    const int dense_deg = std::max(64, (int)(10.0 * avg));
    std::vector<int> rest, dense;
    for (int v = 0; v < N; ++v) (g_.off[v + 1] - g_.off[v] > dense_deg ? dense : rest).push_back(v);
    ++cur_;
    for (int v : dense) tag_[v] = -1;   // excluded from every part
    dissect(rest);
    for (int v : dense) out_.push_back(v);
    return out_;
  }

 private:
  const Graph& g_;
  std::vector<int> tag_, lvl_, out_;
  int cur_ = 0;

  // Level structure of a BFS: the nodes in visiting order, and the start of each level in it
  // (lo.back() == q.size()).
  struct Levels {
    std::vector<int> q, lo;
    int count() const { return (int)lo.size() - 1; }
    const int* begin(int l) const { return q.data() + lo[l]; }
    const int* end(int l) const { return q.data() + lo[l + 1]; }
  };

  // BFS over the nodes tagged t from s (neighbours in adjacency order, level by level).
  void bfs(int s, int t, Levels& L) {
    L.q.clear();
    L.lo.clear();
    L.q.push_back(s);
    lvl_[s] = 0;
    size_t b = 0;
    while (b < L.q.size()) {
      const size_t e = L.q.size();
      L.lo.push_back((int)b);
      const int next = (int)L.lo.size();
      for (size_t k = b; k < e; ++k) {
        const int v = L.q[k];
        for (int p = g_.off[v]; p < g_.off[v + 1]; ++p) {
          const int u = g_.adj[p];
          if (tag_[u] == t && lvl_[u] < 0) {
            lvl_[u] = next;
            L.q.push_back(u);
          }
        }
      }
      b = e;
    }
    L.lo.push_back((int)L.q.size());
    for (int v : L.q) lvl_[v] = -1;
  }

  void dissect(const std::vector<int>& nodes) {
    if ((int)nodes.size() <= kLeaf) {
      for (int v : nodes) out_.push_back(v);
      return;
    }
    const int t = ++cur_;
    for (int v : nodes) tag_[v] = t;
    // connected parts, each moved to a tag of its own as it is found
    std::vector<std::vector<int>> parts;
    Levels levels;
    int tpart = t;
    for (int v : nodes) {
      if (tag_[v] != t) continue;
      bfs(v, t, levels);
      std::vector<int> part(levels.q);
      tpart = ++cur_;
      for (int u : part) tag_[u] = tpart;
      parts.push_back(std::move(part));
    }
    if (parts.size() > 1) {
      for (auto& part : parts) {
        std::sort(part.begin(), part.end());
        dissect(part);
      }
      return;
    }
    // one connected part (tag tpart): pseudo-peripheral start, the last node of a BFS, repeated
    // while the depth grows
    int start = *levels.begin(levels.count() - 1);
    int depth = levels.count();
    Levels l2;
    for (int it = 0; it < 4; ++it) {
      bfs(start, tpart, l2);
      if (l2.count() <= depth) break;
      depth = l2.count();
      std::swap(levels, l2);
      start = *levels.begin(levels.count() - 1);
    }
    if (levels.count() < 3) {         // nearly a clique: no useful separator
      std::vector<int> v(nodes);
      std::sort(v.begin(), v.end());
      for (int u : v) out_.push_back(u);
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
    std::vector<int> p1(levels.begin(0), levels.begin(L)), p2(levels.begin(L + 1), levels.end(levels.count() - 1)),
        sep(levels.begin(L), levels.end(L));
    std::sort(p1.begin(), p1.end());
    std::sort(p2.begin(), p2.end());
    std::sort(sep.begin(), sep.end());
    dissect(p1);
    dissect(p2);
    for (int v : sep) out_.push_back(v);
  }
};

// Position of value x in the sorted range [b, e), or -1.
int find_sorted(const int* b, const int* e, int x) {
  const int* p = std::lower_bound(b, e, x);
  return (p != e && *p == x) ? (int)(p - b) : -1;
}

}  // namespace

int ldl_analyze(int m, int n, const int* rp, const int* ci, LdlSymbolic& S) {
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
  const Graph g = build_graph(m, n, rp, ci);
  // ---- ordering -------------------------------------------------------------------------------
  S.perm = Dissection(g).order();
  S.iperm.assign(N, -1);
  for (int k = 0; k < N; ++k) S.iperm[S.perm[k]] = k;
  // ---- elimination tree (ancestor links with path compression) ------------------------------
  S.parent.assign(N, -1);
  {
    std::vector<int> anc(N, -1);
    for (int k = 0; k < N; ++k) {
      const int v = S.perm[k];
      for (int p = g.off[v]; p < g.off[v + 1]; ++p) {
        int i = S.iperm[g.adj[p]];
        while (i != -1 && i < k) {
          const int next = anc[i];
          anc[i] = k;
          if (next == -1) S.parent[i] = k;
          i = next;
        }
      }
    }
  }
  // ---- column structures: struct(j) = higher neighbours of j  U  struct(children) \ {j} -------
  std::vector<std::vector<int>> st(N);
  {
    std::vector<std::vector<int>> kids(N);
    for (int j = 0; j < N; ++j)
      if (S.parent[j] >= 0) kids[S.parent[j]].push_back(j);
    std::vector<int> mark(N, -1);
    for (int j = 0; j < N; ++j) {
      std::vector<int>& s = st[j];
      const int v = S.perm[j];
      for (int p = g.off[v]; p < g.off[v + 1]; ++p) {
        const int i = S.iperm[g.adj[p]];
        if (i > j && mark[i] != j) {
          mark[i] = j;
          s.push_back(i);
        }
      }
      for (int c : kids[j])
        for (int i : st[c])
          if (i > j && mark[i] != j) {
            mark[i] = j;
            s.push_back(i);
          }
      std::sort(s.begin(), s.end());
    }
  }
  S.colcount.resize(N);
  for (int j = 0; j < N; ++j) S.colcount[j] = (int)st[j].size();
  // ---- supernodes: fundamental, then chains merged while small and with little zero fill ------
  std::vector<int> nkids(N, 0);
  for (int j = 0; j < N; ++j)
    if (S.parent[j] >= 0) ++nkids[S.parent[j]];
  std::vector<int> sfirst, swidth;
  for (int j = 0; j < N;) {
    int l = j;
    while (l + 1 < N && S.parent[l] == l + 1 && nkids[l + 1] == 1 && st[l].size() == st[l + 1].size() + 1) ++l;
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
        const int64_t hp = (int64_t)st[fp + wp - 1].size();
        const int64_t h_s = (int64_t)st[l].size();
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
  S.row_off.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) S.row_off[s + 1] = S.row_off[s] + (int)st[sfirst[s] + swidth[s] - 1].size();
  S.rows.resize(S.row_off[ns]);
  for (int s = 0; s < ns; ++s) {
    const auto& r = st[sfirst[s] + swidth[s] - 1];
    std::copy(r.begin(), r.end(), S.rows.begin() + S.row_off[s]);
  }
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
  // ---- index maps: children's rows in the parent's front; original entries of K -----------------
  auto local = [&](int s, int i) -> int {   // front position of row i (new index) in supernode s
    const int f = sfirst[s], w = swidth[s];
    if (i >= f && i < f + w) return i - f;
    const int a = find_sorted(S.rows.data() + S.row_off[s], S.rows.data() + S.row_off[s + 1], i);
    return a < 0 ? -1 : w + a;
  };
  S.rel_off.assign(ns + 1, 0);
  for (int s = 0; s < ns; ++s) S.rel_off[s + 1] = S.rel_off[s] + (S.sparent[s] >= 0 ? S.row_off[s + 1] - S.row_off[s] : 0);
  S.rel.resize(S.rel_off[ns]);
  for (int s = 0; s < ns; ++s) {
    const int p = S.sparent[s];
    if (p < 0) continue;
    for (int a = S.row_off[s]; a < S.row_off[s + 1]; ++a) {
      const int loc = local(p, S.rows[a]);
      if (loc < 0) return POGS_ERR_ARG;   // cannot happen for an elimination tree
      S.rel[S.rel_off[s] + (a - S.row_off[s])] = loc;
    }
  }
  S.asm_off.assign(ns + 1, 0);
  S.asm_pos.clear();
  S.asm_src.clear();
  for (int s = 0; s < ns; ++s) {
    const int f = sfirst[s], w = swidth[s];
    const int nf = w + (S.row_off[s + 1] - S.row_off[s]);
    for (int j = f; j < f + w; ++j) {
      const int v = S.perm[j];
      const int lc = j - f;
      S.asm_pos.push_back(lc * nf + lc);
      S.asm_src.push_back(v < n ? -1 : -2);
      for (int p = g.off[v]; p < g.off[v + 1]; ++p) {
        const int u = g.adj[p];
        const int i = S.iperm[u];
        if (i <= j) continue;
        const int lr = local(s, i);
        if (lr < 0) return POGS_ERR_ARG;
        // the A entry linking x_col and y_row
        const int row = v < n ? u - n : v - n;
        const int col = v < n ? v : u;
        const int k = find_sorted(ci + rp[row], ci + rp[row + 1], col);
        S.asm_pos.push_back(lr * nf + lc);
        S.asm_src.push_back(rp[row] + k);
      }
    }
    S.asm_off[s + 1] = (int)S.asm_pos.size();
  }
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
