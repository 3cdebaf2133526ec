// Sparse LDL^T of the quasi-definite KKT matrix of the graph projection (Section 3.5, the direct
// method for sparse A with factorization caching).
//
//   K = [ I   A^T ]     (N = n + m; unknowns x (n) first, then y (m))
//       [ A   -I  ]
//
// K is quasi-definite (a positive definite block, a negative definite block), so P K P^T = L D L^T
// exists for every symmetric permutation P with D diagonal (positive on the x block, negative on
// the y block, in exact arithmetic); the ordering can therefore be chosen for sparsity alone,
// before any value is known.  One factorization serves both projections:
//   K [x; y] = [r; 0]    gives x = (I + A^T A)^{-1} r     (tall reduced update),
//   K [u; v] = [0; -r]   gives v = (I + A A^T)^{-1} r     (fat reduced update).
//
// Host side (this header, ldl.cu): nested-dissection ordering of the graph of K, elimination tree,
// column structures, supernodes (fundamental, then merged along chains), the level of each
// supernode in the supernodal tree, and the index maps of the multifrontal method.  Device side
// (ldl.cu): the numeric factorization, one kernel launch per level with one CTA per frontal
// matrix, and the two triangular solves, again one launch per level.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace pogs {

struct LdlSymbolic {
  int n = 0, m = 0, N = 0;
  std::vector<int> perm;      // new index -> old index (old: x_j = j, y_i = n + i)
  std::vector<int> iperm;     // old -> new
  std::vector<int> parent;    // elimination tree over columns (new indices), -1 at roots
  std::vector<int> colcount;  // nonzeros of column j of L below the diagonal (structural)
  // supernodes: columns [first, first + width) share the row structure rows[row_off[s] ..) below them
  int ns = 0;
  std::vector<int> first, width, row_off, rows, sparent, level;
  std::vector<int> child_off, child;      // children of each supernode, increasing
  std::vector<int> level_off, level_nodes;
  std::vector<int> rel_off, rel;          // for supernode c: front positions of its rows in its parent
  // original entries of K per supernode: front position (row * nf + col) and source (CSR index of
  // the A entry, or -1 for +1 on the x diagonal, -2 for -1 on the y diagonal)
  std::vector<int> asm_off, asm_pos, asm_src;
  std::vector<int64_t> panel_off;         // nf x w doubles per supernode (rows: own columns, then R_s)
  // h x h doubles per supernode (update matrix), placed in one arena: an update lives from its
  // supernode's level to its parent's level, and the space is reused after that
  std::vector<int64_t> upd_off;
  // fronts of more than kSmemFront rows are assembled in global scratch (nf x nf doubles at
  // front_off inside the level's region); smaller ones in shared memory.  Within each level the
  // shared-memory fronts come first: level_split[l] is the position of the first global one.
  static constexpr int kSmemFront = 96;
  std::vector<int64_t> front_off;
  std::vector<int> level_split;
  std::vector<int> vec_off;               // h entries per supernode (update vectors of the solve)
  int64_t panel_total = 0, upd_total = 0, front_max = 0, nnz_l = 0;
  int vec_total = 0, max_front = 0, levels = 0, smem_front_max = 0;
};

// The numeric factor on the device, cached in a handle (Section 3.5, factorization caching).
struct LdlFactor {
  int N = 0, n = 0, m = 0, ns = 0, levels = 0, max_front = 0;
  int64_t panel_entries = 0;
  std::vector<int> level_off;             // host copy: supernodes per level (launch sizes)
  std::vector<int> level_threads;         // host copy: solve threads per CTA of each level (32, 64 or 128)
  int *perm = nullptr, *first = nullptr, *width = nullptr, *row_off = nullptr, *rows = nullptr;
  int *child_off = nullptr, *child = nullptr, *level_nodes = nullptr, *rel_off = nullptr, *rel = nullptr;
  int* vec_off = nullptr;
  int64_t* panel_off = nullptr;
  double* panel = nullptr;                // per supernode nf x w: rows < w X11 = L11^{-1} below the diagonal
                                          // (unit diagonal implied) and D on it, rows >= w L21
  double* y = nullptr;                    // N: the solve's work vector (new order)
  double* uvec = nullptr;                 // update vectors of the forward solve
  int64_t device_bytes = 0;
  std::vector<void*> allocs;
  void release(cudaStream_t s);
};

// Numeric factorization P K P^T = L D L^T on `stream` with the values of A (CSR values on the
// device, in the order of the pattern given to ldl_analyze).  Builds F (device arrays owned by
// F until release).  err (device int) receives POGS_ERR_NUMERIC on a zero or non-finite pivot.
int ldl_factor(const LdlSymbolic& S, const float* va, LdlFactor& F, int* err, cudaStream_t stream);

// out = (I + A^T A)^{-1} v (tall: in = v on the x unknowns) or (I + A A^T)^{-1} v (fat: -v on the
// y unknowns), applied through the epilogue `epi` (EpiR codes, kernels.h) element by element.
struct EpiArgs;
void ldl_apply(const LdlFactor& F, bool tall, const float* v, int epi, const EpiArgs& ep, cudaStream_t stream);
int ldl_launches(const LdlFactor& F);    // kernel launches of one ldl_apply

// Symbolic analysis of K for the m x n pattern of A given in CSR (rowptr m + 1, colind sorted and
// unique within each row, host arrays).  Returns 0, POGS_ERR_ARG on a malformed pattern, or
// POGS_ERR_OOM when host memory runs out.
int ldl_analyze(int m, int n, const int* rowptr, const int* colind, LdlSymbolic& S);

}  // namespace pogs
