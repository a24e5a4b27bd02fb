/*
 * oracle.c -- plain, slow FP64 CPU oracle for the sparsity-aware SpMM path of SHIRO
 * (Zhuang et al., "SHIRO: Near-Optimal Communication Strategies for Distributed Sparse Matrix
 * Multiplication", ICS 2026).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may call it.  It shares no code, header or table with the CUDA library; the two are compared
 * on the same seeded inputs.
 *
 * What it computes (notation of Tab. 1):
 *   - the tile grid A^(p,q): row block p = rows [rb[p], rb[p+1]), column block q = columns
 *     [cb[q], cb[q+1]) (Sec. 2.2 partitions A, B and C into row blocks; the sub-block A^(p,q) of
 *     Tab. 1 is the part of A^(p,:) whose columns are owned by process q);
 *   - Cols(A^(p,q)), the unique column indices of the nonzeros of the tile, in ascending order
 *     (Tab. 1, Eq. 2), and Rows(A^(p,q)) (Tab. 1, Eq. 3);
 *   - the remapped index of every nonzero: its position in its tile's Cols (the packed B rows are
 *     consumed by the receiver, Sec. 5.1 stages 3 and 5);
 *   - the volumes V_block = K_q * N * sz (Eq. 1) and V_col = |Cols| * N * sz (Eq. 2);
 *   - the pack of B rows named by Cols (Sec. 5.1 stage 3) -- a plain row copy;
 *   - C = A B (Sec. 2.1) summed in FP64, both directly from B and through the packed rows;
 *   - the backward pieces dB = A^T dC and dA_ij = <dC_i,:, B_j,:> on A's pattern, and the
 *     CSR transpose with rows of A^T in ascending order of A's row index;
 *   - the per-element scale S = |A| |B| and the scaled error |C - C64| / S that turns a result
 *     into pass or fail (the tolerance is stated on C = A B, Sec. 2.1);
 *   - the maximum matching of a tile's row-column graph, whose size is the minimum vertex cover
 *     mu of the joint row-column strategy (Sec. 5.3, Eq. 7-8; Koenig's theorem);
 *   - the minimum weighted vertex cover of that graph through the flow network and minimum cut
 *     of Sec. 5.3.3.
 *
 * Every loop is the definition written out: no blocking, fusion or reordering.  Floating-point
 * sums are taken in CSR order in FP64.  Build with -ffp-contract=off so every product and sum is
 * rounded on its own, the same on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Uniform block boundaries: block p starts at p * ceil(n / P), clamped to n (the last block takes
 * the remainder; trailing blocks may be empty). */
void oracle_uniform_bounds(int64_t n, int32_t P, int64_t* bounds) {
  int64_t b = (n + P - 1) / P;
  for (int32_t p = 0; p <= P; ++p) {
    int64_t v = (int64_t)p * b;
    bounds[p] = v < n ? v : n;
  }
}

/* Index of the block that contains x (bounds ascending, bounds[0] <= x < bounds[P]). */
static int32_t block_of(int64_t x, const int64_t* bounds, int32_t P) {
  for (int32_t p = 0; p < P; ++p)
    if (x >= bounds[p] && x < bounds[p + 1]) return p;
  return -1;
}

/*
 * oracle_plan: for every tile t = p * Pc + q (or t = p when diag_only, where the only tile of row
 * block p is (p, p)) compute
 *   tile_nnz[t], tile_nrows[t] = |Rows(A^(p,q))|, tile_ncols[t] = |Cols(A^(p,q))|,
 *   tile_cols_ptr[t] = sum of |Cols| of the tiles before t (exclusive scan, T+1 entries),
 *   cols_sorted[tile_cols_ptr[t] + u] = u-th smallest distinct column of tile t,
 *   colidx_local[e] = position of col[e] in its tile's cols_sorted segment.
 * cols_cap is the capacity of cols_sorted.  Returns 0, or -1 if a column is out of range, a
 * nonzero lies outside its row block's tile in diag_only mode, or cols_cap is too small.
 */
int oracle_plan(int64_t M, int64_t K, const int64_t* rowptr, const int32_t* col, int32_t Pr,
                int32_t Pc, const int64_t* rb, const int64_t* cb, int diag_only, int64_t* tile_nnz,
                int64_t* tile_nrows, int64_t* tile_ncols, int64_t* tile_cols_ptr,
                int32_t* cols_sorted, int64_t cols_cap, int32_t* colidx_local) {
  (void)M;
  int32_t T = diag_only ? Pr : Pr * Pc;
  int64_t total = 0;
  tile_cols_ptr[0] = 0;
  for (int32_t t = 0; t < T; ++t) {
    int32_t p = diag_only ? t : t / Pc;
    int32_t q = diag_only ? t : t % Pc;
    int64_t c0 = cb[q], width = cb[q + 1] - cb[q];
    char* present = (char*)calloc((size_t)(width > 0 ? width : 1), 1);
    int64_t* rank = (int64_t*)malloc(sizeof(int64_t) * (size_t)(width > 0 ? width : 1));
    int64_t nnz_t = 0, rows_t = 0;
    for (int64_t i = rb[p]; i < rb[p + 1]; ++i) {
      int row_hit = 0;
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        int64_t j = col[e];
        if (j < 0 || j >= K) { free(present); free(rank); return -1; }
        if (j >= c0 && j < c0 + width) {
          present[j - c0] = 1;
          ++nnz_t;
          row_hit = 1;
        } else if (diag_only) {
          free(present); free(rank); return -1;
        }
      }
      rows_t += row_hit;
    }
    int64_t u = 0;
    for (int64_t j = 0; j < width; ++j) {
      if (present[j]) {
        if (total + u >= cols_cap) { free(present); free(rank); return -1; }
        cols_sorted[total + u] = (int32_t)(c0 + j);
        rank[j] = u;
        ++u;
      }
    }
    for (int64_t i = rb[p]; i < rb[p + 1]; ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        int64_t j = col[e];
        if (j >= c0 && j < c0 + width) colidx_local[e] = (int32_t)rank[j - c0];
      }
    tile_nnz[t] = nnz_t;
    tile_nrows[t] = rows_t;
    tile_ncols[t] = u;
    total += u;
    tile_cols_ptr[t + 1] = total;
    free(present);
    free(rank);
  }
  return 0;
}

/* Volumes of Eq. 1, Eq. 2 and Eq. 3 for every tile, in bytes, for N columns: B elements of sz
 * bytes (the block B^(q) for Eq. 1, the rows named by Cols for Eq. 2) and partial C elements of
 * szc bytes (one partial row per row of Rows for Eq. 3).  With local_diag the diagonal tiles are
 * the local computation of Sec. 2.2 and communicate nothing (0 bytes). */
void oracle_volumes(int32_t Pr, int32_t Pc, int diag_only, int local_diag, const int64_t* cb,
                    const int64_t* tile_ncols, const int64_t* tile_nrows, int32_t N, int32_t sz,
                    int32_t szc, int64_t* v_block, int64_t* v_col, int64_t* v_row) {
  int32_t T = diag_only ? Pr : Pr * Pc;
  for (int32_t t = 0; t < T; ++t) {
    int32_t p = diag_only ? t : t / Pc;
    int32_t q = diag_only ? t : t % Pc;
    v_block[t] = (cb[q + 1] - cb[q]) * (int64_t)N * sz;
    v_col[t] = tile_ncols[t] * (int64_t)N * sz;
    v_row[t] = tile_nrows[t] * (int64_t)N * szc;
    if (local_diag && p == q) v_block[t] = v_col[t] = v_row[t] = 0;
  }
}

/* Pack (Sec. 5.1 stage 3): Bpack row r is B row src[r].  Rows are elem_bytes * N bytes wide;
 * ldb and ldp are row strides in elements. */
void oracle_pack(const void* B, int64_t ldb, int32_t N, int32_t elem_bytes, const int32_t* src,
                 int64_t nrows, void* Bpack, int64_t ldp) {
  const char* b = (const char*)B;
  char* o = (char*)Bpack;
  for (int64_t r = 0; r < nrows; ++r)
    memcpy(o + r * ldp * elem_bytes, b + (int64_t)src[r] * ldb * elem_bytes,
           (size_t)N * (size_t)elem_bytes);
}

/* C = A B in FP64 (Sec. 2.1): C[i,k] = sum over the nonzeros e of row i, in CSR order, of
 * val[e] * B[col[e], k].  rows == NULL computes every row; otherwise only rows[0..nrows) and
 * C is nrows x N (row r of C is matrix row rows[r]). */
void oracle_spmm(int64_t M, const int64_t* rowptr, const int32_t* col, const double* val,
                 const double* B, int64_t ldb, int32_t N, const int64_t* rows, int64_t nrows,
                 double* C, int64_t ldc) {
  int64_t n = rows ? nrows : M;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < n; ++r) {
    int64_t i = rows ? rows[r] : r;
    double* c = C + r * ldc;
    for (int32_t k = 0; k < N; ++k) c[k] = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const double a = val[e];
      const double* b = B + (int64_t)col[e] * ldb;
      for (int32_t k = 0; k < N; ++k) c[k] += a * b[k];
    }
  }
}

/* The same product read through the packed rows (Sec. 5.1 stages 3 and 5): the nonzero e of tile
 * t reads Bpack row pack_ptr[t] + colidx_local[e]; when local_diag is set, nonzeros of the
 * diagonal tiles (p == q, the "local computation" of Sec. 2.2) read B[col[e]] directly.
 * Tile of e: p = block of row i in rb, q = block of col[e] in cb (t = p for diag_only). */
void oracle_spmm_packed(int64_t M, const int64_t* rowptr, const int32_t* col, const double* val,
                        int32_t Pr, int32_t Pc, const int64_t* rb, const int64_t* cb,
                        int diag_only, int local_diag, const int64_t* pack_ptr,
                        const int32_t* colidx_local, const double* Bpack, int64_t ldp,
                        const double* B, int64_t ldb, int32_t N, double* C, int64_t ldc) {
  (void)M;
#pragma omp parallel for schedule(dynamic, 64)
  for (int32_t p = 0; p < Pr; ++p) {
    for (int64_t i = rb[p]; i < rb[p + 1]; ++i) {
      double* c = C + i * ldc;
      for (int32_t k = 0; k < N; ++k) c[k] = 0.0;
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        int32_t q = block_of(col[e], cb, Pc);
        int32_t t = diag_only ? p : p * Pc + q;
        const double* b;
        if (local_diag && q == p)
          b = B + (int64_t)col[e] * ldb;
        else
          b = Bpack + (pack_ptr[t] + colidx_local[e]) * ldp;
        const double a = val[e];
        for (int32_t k = 0; k < N; ++k) c[k] += a * b[k];
      }
    }
  }
}

/* Error scale of the tolerance: S[i,k] = sum_e |val[e]| * |B[col[e], k]| (FP64). */
void oracle_abs_scale(int64_t M, const int64_t* rowptr, const int32_t* col, const double* val,
                      const double* B, int64_t ldb, int32_t N, const int64_t* rows,
                      int64_t nrows, double* S, int64_t lds) {
  int64_t n = rows ? nrows : M;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < n; ++r) {
    int64_t i = rows ? rows[r] : r;
    double* s = S + r * lds;
    for (int32_t k = 0; k < N; ++k) s[k] = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const double a = fabs(val[e]);
      const double* b = B + (int64_t)col[e] * ldb;
      for (int32_t k = 0; k < N; ++k) s[k] += a * fabs(b[k]);
    }
  }
}

/* The tolerance of every parity comparison (the per-element scaled error of a result against
 * the FP64 definition of C = A B, Sec. 2.1): for element (i, k) of an nrows x N result,
 *   err_ik = |C_ik - C64_ik| / S_ik,   S_ik = sum_j |a_ij| |b_jk|   (from oracle_abs_scale),
 * and where S_ik == 0 every term of the sum is 0, so C_ik must be exactly 0 (err 0) or the
 * element fails (err +inf).  A NaN in C fails too.  Returns the maximum over all elements;
 * row_max (nullable) receives the maximum of each row.  C, C64 and S are row-major with row
 * strides ldc, ld64 and lds. */
double oracle_scaled_error(int64_t nrows, int32_t N, const double* C, int64_t ldc,
                           const double* C64, int64_t ld64, const double* S, int64_t lds,
                           double* row_max) {
  double worst = 0.0;
  for (int64_t i = 0; i < nrows; ++i) {
    double rmax = 0.0;
    for (int32_t k = 0; k < N; ++k) {
      const double c = C[i * ldc + k];
      const double s = S[i * lds + k];
      const double d = fabs(c - C64[i * ld64 + k]);
      double r;
      if (isnan(d)) r = INFINITY;
      else if (s == 0.0) r = (c == 0.0) ? 0.0 : INFINITY;
      else r = d / s;
      if (r > rmax) rmax = r;
    }
    if (row_max) row_max[i] = rmax;
    if (rmax > worst) worst = rmax;
  }
  return worst;
}

/* dB = A^T dC (the gradient of C = A B with respect to B): dB[j,k] = sum over nonzeros e with
 * col[e] == j of val[e] * dC[row(e), k], accumulated in row-major order of A. */
void oracle_spmm_t(int64_t M, int64_t K, const int64_t* rowptr, const int32_t* col,
                   const double* val, const double* dC, int64_t lddc, int32_t N, double* dB,
                   int64_t lddb) {
  for (int64_t j = 0; j < K; ++j)
    for (int32_t k = 0; k < N; ++k) dB[j * lddb + k] = 0.0;
  for (int64_t i = 0; i < M; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      double* d = dB + (int64_t)col[e] * lddb;
      const double* g = dC + i * lddc;
      for (int32_t k = 0; k < N; ++k) d[k] += val[e] * g[k];
    }
}

/* dA on the pattern of A (sampled dense-dense product): out[e] = sum_k dC[row(e),k] * B[col(e),k]. */
void oracle_sddmm(int64_t M, const int64_t* rowptr, const int32_t* col, const double* dC,
                  int64_t lddc, const double* B, int64_t ldb, int32_t N, double* out) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < M; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      double s = 0.0;
      const double* g = dC + i * lddc;
      const double* b = B + (int64_t)col[e] * ldb;
      for (int32_t k = 0; k < N; ++k) s += g[k] * b[k];
      out[e] = s;
    }
}

/* CSR of A^T (K x M): row j of A^T lists the nonzeros of column j of A in ascending row order
 * (ties, i.e. duplicate entries, in CSR order).  perm[eT] is the A-index of entry eT. */
void oracle_transpose(int64_t M, int64_t K, const int64_t* rowptr, const int32_t* col,
                      int64_t* rowptrT, int32_t* colT, int64_t* perm) {
  for (int64_t j = 0; j <= K; ++j) rowptrT[j] = 0;
  for (int64_t e = 0; e < rowptr[M]; ++e) rowptrT[col[e] + 1] += 1;
  for (int64_t j = 0; j < K; ++j) rowptrT[j + 1] += rowptrT[j];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(K > 0 ? K : 1));
  for (int64_t j = 0; j < K; ++j) fill[j] = rowptrT[j];
  for (int64_t i = 0; i < M; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      int64_t pos = fill[col[e]]++;
      colT[pos] = (int32_t)i;
      perm[pos] = e;
    }
  free(fill);
}

/* Size of a maximum matching of the bipartite graph with left vertices 0..nL-1 (a tile's rows),
 * right vertices 0..nR-1 (its columns) and edges adj[ptr[u] .. ptr[u+1]) of left vertex u (its
 * nonzeros).  By Koenig's theorem this is the size mu of a minimum vertex cover, the optimum of
 * Eq. 4-6 with uniform costs (Sec. 5.3.1 reduction, Sec. 5.4 uniform case).  Kuhn's method: for
 * every left vertex, search an augmenting path depth first (explicit stack); levels remember the
 * right vertex they were reached through so the path can be flipped. */
int64_t oracle_max_matching(int32_t nL, int32_t nR, const int64_t* ptr, const int32_t* adj) {
  int32_t* matchR = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nR > 0 ? nR : 1));
  int64_t* seen = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nR > 0 ? nR : 1));
  int32_t* su = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nL > 0 ? nL : 1));
  int64_t* sk = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nL > 0 ? nL : 1));
  int32_t* sv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nL > 0 ? nL : 1));
  for (int32_t v = 0; v < nR; ++v) {
    matchR[v] = -1;
    seen[v] = -1;
  }
  int64_t size = 0;
  for (int32_t root = 0; root < nL; ++root) {
    int32_t d = 0;
    su[0] = root;
    sk[0] = ptr[root];
    while (d >= 0) {
      const int32_t u = su[d];
      if (sk[d] == ptr[u + 1]) {
        --d;
        continue;
      }
      const int32_t v = adj[sk[d]++];
      if (seen[v] == root) continue;
      seen[v] = root;
      if (matchR[v] < 0) {
        matchR[v] = u;
        for (int32_t l = d - 1; l >= 0; --l) matchR[sv[l]] = su[l];
        ++size;
        break;
      }
      sv[d] = v;
      ++d;
      su[d] = matchR[v];
      sk[d] = ptr[su[d]];
    }
  }
  free(matchR);
  free(seen);
  free(su);
  free(sk);
  free(sv);
  return size;
}

/* Minimum weighted vertex cover of the bipartite row-column graph of a tile (Sec. 5.3.2: Eq. 4-6
 * with a cost per vertex, w_row[u] for sending partial row c_u, w_col[v] for sending row b_v).
 * Sec. 5.3.3 turns it into a minimum s-t cut: the source feeds row u with capacity w_row[u],
 * every nonzero (u, v) links row u to column v with unbounded capacity, column v feeds the sink
 * with capacity w_col[v].  The maximum flow is found here by shortest augmenting paths
 * (Edmonds-Karp; the paper's Dinic reaches the same flow value), and the cut is read off the set Z
 * of vertices reachable from the source in the residual network: a row outside Z or a column
 * inside Z is selected.  Z is the same for every maximum flow (it is the smallest source side of
 * a minimum cut), so the selection is unique.  Rows without edges are never selected.
 * cover_row (nL bytes) and cover_col (nR bytes) receive the selection; returns the maximum
 * flow, which equals the selection's total cost (max-flow min-cut).  Costs must be >= 0 with a
 * sum below 2^62. */
int64_t oracle_min_weight_cover(int32_t nL, int32_t nR, const int64_t* ptr, const int32_t* adj,
                                const int64_t* w_row, const int64_t* w_col, uint8_t* cover_row,
                                uint8_t* cover_col) {
  const int64_t UNBOUNDED = (int64_t)1 << 62;
  const int64_t E = ptr[nL];
  const int32_t n = nL + nR + 2, s = 0, t = nL + nR + 1;
  const int64_t m = 2 * ((int64_t)nL + E + nR); /* every arc and its residual twin */
  int32_t* to = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int64_t* cap = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* via = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  for (int32_t x = 0; x < n; ++x) head[x] = -1;
  int64_t a = 0;
  /* arc 2k goes forward with the capacity, arc 2k+1 is its twin with none: twin(e) = e ^ 1 */
#define ORACLE_ARC(x, y, c)                                   \
  do {                                                        \
    to[a] = (y); cap[a] = (c); next[a] = head[x]; head[x] = a; ++a; \
    to[a] = (x); cap[a] = 0; next[a] = head[y]; head[y] = a; ++a;   \
  } while (0)
  for (int32_t u = 0; u < nL; ++u) ORACLE_ARC(s, 1 + u, w_row[u]);
  for (int32_t u = 0; u < nL; ++u)
    for (int64_t k = ptr[u]; k < ptr[u + 1]; ++k) ORACLE_ARC(1 + u, 1 + nL + adj[k], UNBOUNDED);
  for (int32_t v = 0; v < nR; ++v) ORACLE_ARC(1 + nL + v, t, w_col[v]);
#undef ORACLE_ARC
  int64_t flow = 0;
  for (;;) {
    /* breadth-first search for a shortest path with residual capacity */
    for (int32_t x = 0; x < n; ++x) via[x] = -2;
    via[s] = -1;
    int32_t qh = 0, qt = 0;
    queue[qt++] = s;
    while (qh < qt && via[t] == -2) {
      const int32_t x = queue[qh++];
      for (int64_t e = head[x]; e >= 0; e = next[e])
        if (cap[e] > 0 && via[to[e]] == -2) {
          via[to[e]] = e;
          queue[qt++] = to[e];
        }
    }
    if (via[t] == -2) break;
    int64_t b = UNBOUNDED;
    for (int32_t x = t; x != s; x = to[via[x] ^ 1])
      if (cap[via[x]] < b) b = cap[via[x]];
    for (int32_t x = t; x != s; x = to[via[x] ^ 1]) {
      cap[via[x]] -= b;
      cap[via[x] ^ 1] += b;
    }
    flow += b;
  }
  /* Z: reachable from the source through arcs with residual capacity (via[] != -2 after the last
   * search, which ran to exhaustion because the sink was not reached) */
  for (int32_t u = 0; u < nL; ++u) cover_row[u] = (uint8_t)(via[1 + u] == -2 && ptr[u + 1] > ptr[u]);
  for (int32_t v = 0; v < nR; ++v) cover_col[v] = (uint8_t)(via[1 + nL + v] != -2);
  free(to);
  free(cap);
  free(next);
  free(head);
  free(via);
  free(queue);
  return flow;
}
