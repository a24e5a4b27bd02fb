// joint.cu -- the joint row-column strategy (Sec. 5.2-5.3): per tile, a minimum vertex cover of
// the bipartite graph whose left vertices are the tile's rows, right vertices its columns and
// edges its nonzeros.  With uniform costs (Sec. 5.4) the cover size mu equals the maximum matching
// (Koenig's theorem), found by Hopcroft-Karp; the cover is read off the alternating reachability
// from unmatched rows.  A nonzero whose column is in the cover is column-based (its B row is sent,
// Eq. 2); every other nonzero has its row in the cover and is row-based (a partial C row is sent,
// Eq. 3).  Offline host work, as in the paper; tiles are solved in parallel threads.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace shiro {

namespace {

// Bipartite graph: left vertex u has right neighbours adj[ptr[u] .. ptr[u+1]).
struct Bipartite {
  int32_t nL = 0, nR = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> adj;
};

// Hopcroft-Karp with iterative DFS; returns the matching size and fills pairL / pairR.
int64_t hopcroft_karp(const Bipartite& g, std::vector<int32_t>& pairL, std::vector<int32_t>& pairR) {
  const int32_t INF = INT32_MAX;
  pairL.assign(g.nL, -1);
  pairR.assign(g.nR, -1);
  std::vector<int32_t> dist(g.nL), queue(g.nL), stack(g.nL);
  std::vector<int64_t> it(g.nL);
  int64_t matching = 0;
  while (true) {
    // BFS layers from the free left vertices.
    int32_t qh = 0, qt = 0;
    bool found = false;
    for (int32_t u = 0; u < g.nL; ++u) {
      if (pairL[u] < 0 && g.ptr[u + 1] > g.ptr[u]) {
        dist[u] = 0;
        queue[qt++] = u;
      } else {
        dist[u] = INF;
      }
    }
    while (qh < qt) {
      const int32_t u = queue[qh++];
      for (int64_t k = g.ptr[u]; k < g.ptr[u + 1]; ++k) {
        const int32_t w = pairR[g.adj[k]];
        if (w < 0) {
          found = true;
        } else if (dist[w] == INF) {
          dist[w] = dist[u] + 1;
          queue[qt++] = w;
        }
      }
    }
    if (!found) break;
    // DFS along the layers from every free left vertex (iterative, one path at a time).
    for (int32_t u = 0; u < g.nL; ++u) it[u] = g.ptr[u];
    for (int32_t root = 0; root < g.nL; ++root) {
      if (pairL[root] >= 0 || dist[root] != 0) continue;
      int32_t sp = 0;
      stack[sp++] = root;
      bool augmented = false;
      while (sp > 0 && !augmented) {
        const int32_t u = stack[sp - 1];
        bool advanced = false;
        while (it[u] < g.ptr[u + 1]) {
          const int32_t v = g.adj[it[u]];
          const int32_t w = pairR[v];
          if (w < 0) {
            // Augment along the stack: stack[s] takes the right vertex its iterator points at.
            for (int32_t s = sp - 1; s >= 0; --s) {
              const int32_t x = stack[s];
              const int32_t y = g.adj[it[x]];
              pairL[x] = y;
              pairR[y] = x;
            }
            augmented = true;
            ++matching;
            break;
          }
          if (dist[w] == dist[u] + 1) {
            stack[sp++] = w;
            advanced = true;
            break;
          }
          ++it[u];
        }
        if (augmented) break;
        if (!advanced) {
          dist[u] = INF;  // dead end: drop it from this phase
          --sp;
          if (sp > 0) ++it[stack[sp - 1]];
        }
      }
    }
  }
  return matching;
}

// Koenig: Z = vertices reachable from free left vertices by alternating paths (non-matching edges
// left -> right, matching edges right -> left); cover = (left not in Z) + (right in Z).
void koenig_cover(const Bipartite& g, const std::vector<int32_t>& pairL,
                  const std::vector<int32_t>& pairR, std::vector<char>& coverL,
                  std::vector<char>& coverR) {
  std::vector<char> zL(g.nL, 0), zR(g.nR, 0);
  std::vector<int32_t> queue;
  queue.reserve(g.nL);
  for (int32_t u = 0; u < g.nL; ++u)
    if (pairL[u] < 0) {
      zL[u] = 1;
      queue.push_back(u);
    }
  for (size_t h = 0; h < queue.size(); ++h) {
    const int32_t u = queue[h];
    for (int64_t k = g.ptr[u]; k < g.ptr[u + 1]; ++k) {
      const int32_t v = g.adj[k];
      if (zR[v] || pairL[u] == v) continue;
      zR[v] = 1;
      const int32_t w = pairR[v];
      if (w >= 0 && !zL[w]) {
        zL[w] = 1;
        queue.push_back(w);
      }
    }
  }
  coverL.assign(g.nL, 0);
  coverR.assign(g.nR, 0);
  for (int32_t u = 0; u < g.nL; ++u) coverL[u] = (!zL[u] && g.ptr[u + 1] > g.ptr[u]) ? 1 : 0;
  for (int32_t v = 0; v < g.nR; ++v) coverR[v] = zR[v];
}

}  // namespace

}  // namespace shiro

using namespace shiro;

extern "C" shiro_status shiro_plan_joint(shiro_plan_t P, int64_t* tile_mu,
                                         int64_t* tile_cover_rows, int64_t* tile_cover_cols,
                                         uint8_t* nnz_row_based, void* stream) {
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nnz = P->nnz;
  std::vector<int32_t> col(nnz > 0 ? nnz : 1), local(nnz > 0 ? nnz : 1);
  if (nnz > 0)
    SHIRO_CUDA(cudaMemcpyAsync(col.data(), P->col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, s));
  SHIRO_CUDA(cudaStreamSynchronize(s));
  const bool diag = P->flags & SHIRO_PLAN_DIAG_ONLY;
  const bool local_diag = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  const int32_t T = P->T, Pc = P->geo.Pc;
  // Column block of every column and the rank of a column inside its tile's Cols.
  auto col_block_h = [&](int64_t j) {
    return (int32_t)(std::upper_bound(P->cb.begin(), P->cb.end(), j) - P->cb.begin() - 1);
  };
  std::vector<int32_t> cols_sorted(P->total_cols > 0 ? P->total_cols : 1);
  if (P->total_cols > 0) {
    SHIRO_CUDA(cudaMemcpyAsync(cols_sorted.data(), P->d_cols_sorted,
                               sizeof(int32_t) * P->total_cols, cudaMemcpyDeviceToHost, s));
    SHIRO_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<int32_t> tile_of(nnz > 0 ? nnz : 1);
  for (int32_t p = 0; p < P->geo.Pr; ++p)
    for (int64_t i = P->rb[p]; i < P->rb[p + 1]; ++i)
      for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e) {
        const int32_t q = diag ? p : col_block_h(col[e]);
        const int32_t t = diag ? p : p * Pc + q;
        tile_of[e] = t;
        const int32_t* c0 = cols_sorted.data() + P->tile_cols_ptr[t];
        const int32_t* c1 = cols_sorted.data() + P->tile_cols_ptr[t + 1];
        local[e] = (int32_t)(std::lower_bound(c0, c1, col[e]) - c0);
      }
  std::vector<int64_t> mu(T, 0), crows(T, 0), ccols(T, 0);
  std::vector<uint8_t> side(nnz > 0 ? nnz : 1, 0);
  std::atomic<int32_t> next{0};
  auto worker = [&]() {
    while (true) {
      const int32_t t = next.fetch_add(1);
      if (t >= T) break;
      const int32_t p = diag ? t : t / Pc, q = diag ? t : t % Pc;
      if (local_diag && p == q) continue;  // local tile: nothing is communicated
      Bipartite g;
      g.nL = (int32_t)(P->rb[p + 1] - P->rb[p]);
      g.nR = (int32_t)P->tile_ncols[t];
      g.ptr.assign(g.nL + 1, 0);
      for (int32_t u = 0; u < g.nL; ++u) {
        const int64_t i = P->rb[p] + u;
        int64_t cnt = 0;
        for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e) cnt += tile_of[e] == t;
        g.ptr[u + 1] = g.ptr[u] + cnt;
      }
      g.adj.resize(g.ptr[g.nL]);
      for (int32_t u = 0; u < g.nL; ++u) {
        const int64_t i = P->rb[p] + u;
        int64_t k = g.ptr[u];
        for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e)
          if (tile_of[e] == t) g.adj[k++] = local[e];
      }
      std::vector<int32_t> pairL, pairR;
      mu[t] = hopcroft_karp(g, pairL, pairR);
      std::vector<char> coverL, coverR;
      koenig_cover(g, pairL, pairR, coverL, coverR);
      int64_t nr = 0, nc = 0;
      for (char c : coverL) nr += c;
      for (char c : coverR) nc += c;
      crows[t] = nr;
      ccols[t] = nc;
      for (int32_t u = 0; u < g.nL; ++u) {
        const int64_t i = P->rb[p] + u;
        for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e)
          if (tile_of[e] == t) side[e] = coverR[local[e]] ? 0 : 1;
      }
    }
  };
  const unsigned nt = std::max(1u, std::min(std::thread::hardware_concurrency(), (unsigned)T));
  std::vector<std::thread> pool;
  for (unsigned k = 1; k < nt; ++k) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  if (tile_mu) memcpy(tile_mu, mu.data(), sizeof(int64_t) * T);
  if (tile_cover_rows) memcpy(tile_cover_rows, crows.data(), sizeof(int64_t) * T);
  if (tile_cover_cols) memcpy(tile_cover_cols, ccols.data(), sizeof(int64_t) * T);
  if (nnz_row_based && nnz > 0) memcpy(nnz_row_based, side.data(), (size_t)nnz);
  return SHIRO_OK;
}

namespace {

// Host copies of the planned matrix's columns and values (FP32 or FP64 as raw bytes).
shiro_status fetch_csr(const shiro_plan_s* P, std::vector<int32_t>& col, std::vector<char>& val,
                       cudaStream_t s) {
  const size_t vs = dtype_size(P->vdt);
  col.resize(P->nnz > 0 ? P->nnz : 1);
  val.resize((P->nnz > 0 ? P->nnz : 1) * vs);
  if (P->nnz > 0) {
    SHIRO_CUDA(cudaMemcpyAsync(col.data(), P->col, sizeof(int32_t) * P->nnz,
                               cudaMemcpyDeviceToHost, s));
    SHIRO_CUDA(cudaMemcpyAsync(val.data(), P->val, vs * P->nnz, cudaMemcpyDeviceToHost, s));
  }
  SHIRO_CUDA(cudaStreamSynchronize(s));
  return SHIRO_OK;
}

}  // namespace

extern "C" shiro_status shiro_joint_split_sizes(shiro_plan_t P, const uint8_t* nnz_row_based,
                                                int64_t* col_nnz, int64_t* split_rows,
                                                int64_t* split_nnz) {
  if (!P || (!nnz_row_based && P->nnz > 0)) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null argument");
  if (P->flags & SHIRO_PLAN_TRANSPOSE) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "not for TRANSPOSE plans");
  int64_t cn = 0, rn = 0, rows = 0;
  for (int64_t e = 0; e < P->nnz; ++e) {
    if (nnz_row_based[e]) ++rn; else ++cn;
  }
  // Count distinct (tile, row) pairs among the row-based nonzeros.
  std::vector<int32_t> col;
  std::vector<char> val;
  if (rn > 0) {
    SHIRO_TRY(fetch_csr(P, col, val, nullptr));
    const bool diag = P->flags & SHIRO_PLAN_DIAG_ONLY;
    for (int32_t p = 0; p < P->geo.Pr; ++p)
      for (int64_t i = P->rb[p]; i < P->rb[p + 1]; ++i) {
        std::vector<int32_t> qs;
        for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e)
          if (nnz_row_based[e]) {
            const int32_t q = diag ? p : (int32_t)(std::upper_bound(P->cb.begin(), P->cb.end(), (int64_t)col[e]) - P->cb.begin() - 1);
            qs.push_back(q);
          }
        std::sort(qs.begin(), qs.end());
        rows += std::unique(qs.begin(), qs.end()) - qs.begin();
      }
  }
  if (col_nnz) *col_nnz = cn;
  if (split_rows) *split_rows = rows;
  if (split_nnz) *split_nnz = rn;
  return SHIRO_OK;
}

extern "C" shiro_status shiro_joint_split(shiro_plan_t P, const uint8_t* nnz_row_based,
                                          int64_t* col_rowptr, int32_t* col_col, void* col_val,
                                          int64_t* rs_rowptr, int32_t* rs_col, void* rs_val,
                                          int64_t* agg_rowptr, int32_t* agg_col, void* agg_val,
                                          void* stream) {
  if (!P || (!nnz_row_based && P->nnz > 0)) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null argument");
  if (P->flags & SHIRO_PLAN_TRANSPOSE) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "not for TRANSPOSE plans");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> col;
  std::vector<char> val;
  SHIRO_TRY(fetch_csr(P, col, val, s));
  const size_t vs = dtype_size(P->vdt);
  const bool diag = P->flags & SHIRO_PLAN_DIAG_ONLY;
  const int32_t Pc = P->geo.Pc;
  // A_col: the column-based nonzeros of every row, in order.
  std::vector<int64_t> crp(P->M + 1, 0);
  std::vector<int32_t> ccol;
  std::vector<char> cval;
  // Split rows: (tile, row) pairs ordered by tile, then row; their row-based nonzeros in order.
  struct Split { int32_t t; int64_t i; };
  std::vector<Split> splits;
  for (int32_t p = 0; p < P->geo.Pr; ++p)
    for (int64_t i = P->rb[p]; i < P->rb[p + 1]; ++i)
      for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e) {
        if (!nnz_row_based[e]) continue;
        const int32_t q = diag ? p : (int32_t)(std::upper_bound(P->cb.begin(), P->cb.end(), (int64_t)col[e]) - P->cb.begin() - 1);
        const int32_t t = diag ? p : p * Pc + q;
        if (splits.empty() || splits.back().t != t || splits.back().i != i) splits.push_back({t, i});
      }
  std::stable_sort(splits.begin(), splits.end(), [](const Split& a, const Split& b) {
    return a.t != b.t ? a.t < b.t : a.i < b.i;
  });
  splits.erase(std::unique(splits.begin(), splits.end(),
                           [](const Split& a, const Split& b) { return a.t == b.t && a.i == b.i; }),
               splits.end());
  for (int64_t i = 0; i < P->M; ++i) {
    for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e)
      if (!nnz_row_based[e]) {
        ccol.push_back(col[e]);
        cval.insert(cval.end(), val.begin() + e * vs, val.begin() + (e + 1) * vs);
      }
    crp[i + 1] = (int64_t)ccol.size();
  }
  std::vector<int64_t> rrp(splits.size() + 1, 0);
  std::vector<int32_t> rcol;
  std::vector<char> rval;
  for (size_t k = 0; k < splits.size(); ++k) {
    const int64_t i = splits[k].i;
    const int32_t t = splits[k].t;
    for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e) {
      if (!nnz_row_based[e]) continue;
      const int32_t p = diag ? t : t / Pc;
      const int32_t q = diag ? p : (int32_t)(std::upper_bound(P->cb.begin(), P->cb.end(), (int64_t)col[e]) - P->cb.begin() - 1);
      if ((diag ? p : p * Pc + q) != t) continue;
      rcol.push_back(col[e]);
      rval.insert(rval.end(), val.begin() + e * vs, val.begin() + (e + 1) * vs);
    }
    rrp[k + 1] = (int64_t)rcol.size();
  }
  // Aggregation: row i of C gathers its split rows in split order (tile order), weight one.
  std::vector<int64_t> arp(P->M + 1, 0);
  for (const Split& sp : splits) arp[sp.i + 1] += 1;
  for (int64_t i = 0; i < P->M; ++i) arp[i + 1] += arp[i];
  std::vector<int32_t> acol(splits.size() > 0 ? splits.size() : 1);
  {
    std::vector<int64_t> fill(arp.begin(), arp.end() - 1);
    for (size_t k = 0; k < splits.size(); ++k) acol[fill[splits[k].i]++] = (int32_t)k;
  }
  std::vector<char> aval(splits.size() * vs);
  for (size_t k = 0; k < splits.size(); ++k) {
    if (P->vdt == SHIRO_F64) { const double one = 1.0; memcpy(&aval[k * vs], &one, vs); }
    else { const float one = 1.0f; memcpy(&aval[k * vs], &one, vs); }
  }
  auto h2d = [&](void* dst, const void* src, size_t bytes) -> shiro_status {
    if (bytes && dst) SHIRO_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    return SHIRO_OK;
  };
  SHIRO_TRY(h2d(col_rowptr, crp.data(), sizeof(int64_t) * crp.size()));
  SHIRO_TRY(h2d(col_col, ccol.data(), sizeof(int32_t) * ccol.size()));
  SHIRO_TRY(h2d(col_val, cval.data(), cval.size()));
  SHIRO_TRY(h2d(rs_rowptr, rrp.data(), sizeof(int64_t) * rrp.size()));
  SHIRO_TRY(h2d(rs_col, rcol.data(), sizeof(int32_t) * rcol.size()));
  SHIRO_TRY(h2d(rs_val, rval.data(), rval.size()));
  SHIRO_TRY(h2d(agg_rowptr, arp.data(), sizeof(int64_t) * arp.size()));
  SHIRO_TRY(h2d(agg_col, acol.data(), sizeof(int32_t) * splits.size()));
  SHIRO_TRY(h2d(agg_val, aval.data(), aval.size()));
  SHIRO_CUDA(cudaStreamSynchronize(s));
  return SHIRO_OK;
}
