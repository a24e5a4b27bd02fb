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


// Minimum weighted vertex cover through the minimum s-t cut of Sec. 5.3.3: source -> row u with
// capacity w_row[u], row -> column with unbounded capacity for every edge, column v -> sink with
// capacity w_col[v].  Dinic's algorithm (BFS level graph, blocking flow by an iterative DFS that
// retreats to the first saturated arc after each augmentation).  The cover is read off the set Z
// reachable from the source in the final residual network (rows outside Z, columns inside Z):
// that set is the same for every maximum flow, so the selection does not depend on the search
// order.  Returns the maximum flow (= the cover's cost).
struct FlowNet {
  int32_t n = 0;
  std::vector<int64_t> first;  // arcs of node x: [first[x], first[x+1])
  std::vector<int32_t> to;
  std::vector<int64_t> twin;
  std::vector<int64_t> cap;
};

int64_t dinic_cover(const Bipartite& g, const std::vector<int64_t>& w_row,
                    const std::vector<int64_t>& w_col, std::vector<char>& coverL,
                    std::vector<char>& coverR) {
  const int64_t UNBOUNDED = (int64_t)1 << 62;
  const int32_t nL = g.nL, nR = g.nR, s = 0, t = nL + nR + 1;
  FlowNet f;
  f.n = nL + nR + 2;
  // Arc counts per node: s has nL, row u has 1 + deg(u), column v has in-degree + 1, t has nR.
  std::vector<int64_t> deg(f.n + 1, 0);
  deg[s] = nL;
  for (int32_t u = 0; u < nL; ++u) deg[1 + u] = 1 + (g.ptr[u + 1] - g.ptr[u]);
  for (int32_t v = 0; v < nR; ++v) deg[1 + nL + v] = 1;
  for (int64_t k = 0; k < g.ptr[nL]; ++k) deg[1 + nL + g.adj[k]] += 1;
  deg[t] = nR;
  f.first.assign(f.n + 1, 0);
  for (int32_t x = 0; x < f.n; ++x) f.first[x + 1] = f.first[x] + deg[x];
  const int64_t m = f.first[f.n];
  f.to.resize(m);
  f.twin.resize(m);
  f.cap.resize(m);
  std::vector<int64_t> fill(f.first.begin(), f.first.end() - 1);
  auto arc = [&](int32_t x, int32_t y, int64_t c) {
    const int64_t a = fill[x]++, b = fill[y]++;
    f.to[a] = y; f.cap[a] = c; f.twin[a] = b;
    f.to[b] = x; f.cap[b] = 0; f.twin[b] = a;
  };
  for (int32_t u = 0; u < nL; ++u) arc(s, 1 + u, w_row[u]);
  for (int32_t u = 0; u < nL; ++u)
    for (int64_t k = g.ptr[u]; k < g.ptr[u + 1]; ++k) arc(1 + u, 1 + nL + g.adj[k], UNBOUNDED);
  for (int32_t v = 0; v < nR; ++v) arc(1 + nL + v, t, w_col[v]);

  std::vector<int32_t> level(f.n), queue(f.n);
  std::vector<int64_t> it(f.n), path;
  path.reserve(64);
  auto bfs = [&]() {
    std::fill(level.begin(), level.end(), -1);
    int32_t qh = 0, qt = 0;
    level[s] = 0;
    queue[qt++] = s;
    while (qh < qt) {
      const int32_t x = queue[qh++];
      for (int64_t a = f.first[x]; a < f.first[x + 1]; ++a)
        if (f.cap[a] > 0 && level[f.to[a]] < 0) {
          level[f.to[a]] = level[x] + 1;
          queue[qt++] = f.to[a];
        }
    }
    return level[t] >= 0;
  };
  int64_t flow = 0;
  while (bfs()) {
    for (int32_t x = 0; x < f.n; ++x) it[x] = f.first[x];
    path.clear();
    int32_t x = s;
    while (true) {
      if (x == t) {
        int64_t b = UNBOUNDED;
        for (int64_t a : path) b = std::min(b, f.cap[a]);
        size_t cut = path.size();
        for (size_t k = 0; k < path.size(); ++k) {
          f.cap[path[k]] -= b;
          f.cap[f.twin[path[k]]] += b;
          if (f.cap[path[k]] == 0 && cut == path.size()) cut = k;
        }
        flow += b;
        // Retreat to the tail of the first saturated arc and continue the blocking flow there.
        x = f.to[f.twin[path[cut]]];
        path.resize(cut);
        continue;
      }
      bool advanced = false;
      for (; it[x] < f.first[x + 1]; ++it[x]) {
        const int64_t a = it[x];
        if (f.cap[a] > 0 && level[f.to[a]] == level[x] + 1) {
          path.push_back(a);
          x = f.to[a];
          advanced = true;
          break;
        }
      }
      if (advanced) continue;
      if (x == s) break;
      level[x] = -1;  // dead end for the rest of this phase
      const int64_t a = path.back();
      path.pop_back();
      x = f.to[f.twin[a]];
      ++it[x];
    }
  }
  // Z: reachable from the source through arcs with residual capacity.
  std::vector<char> z(f.n, 0);
  int32_t qh = 0, qt = 0;
  z[s] = 1;
  queue[qt++] = s;
  while (qh < qt) {
    const int32_t x = queue[qh++];
    for (int64_t a = f.first[x]; a < f.first[x + 1]; ++a)
      if (f.cap[a] > 0 && !z[f.to[a]]) {
        z[f.to[a]] = 1;
        queue[qt++] = f.to[a];
      }
  }
  coverL.assign(nL, 0);
  coverR.assign(nR, 0);
  for (int32_t u = 0; u < nL; ++u) coverL[u] = (!z[1 + u] && g.ptr[u + 1] > g.ptr[u]) ? 1 : 0;
  for (int32_t v = 0; v < nR; ++v) coverR[v] = z[1 + nL + v];
  return flow;
}

}  // namespace

}  // namespace shiro

using namespace shiro;

namespace {

// Host view of the plan's tiles: the tile and the rank in its tile's Cols of every nonzero.
struct TileIndex {
  std::vector<int32_t> col, local, tile_of, cols_sorted;
};

shiro_status tile_index(const shiro_plan_s* P, TileIndex& X, cudaStream_t s) {
  const int64_t nnz = P->nnz;
  X.col.assign(nnz > 0 ? nnz : 1, 0);
  X.local.assign(nnz > 0 ? nnz : 1, 0);
  X.tile_of.assign(nnz > 0 ? nnz : 1, 0);
  X.cols_sorted.assign(P->total_cols > 0 ? P->total_cols : 1, 0);
  if (nnz > 0)
    SHIRO_CUDA(cudaMemcpyAsync(X.col.data(), P->col, sizeof(int32_t) * nnz,
                               cudaMemcpyDeviceToHost, s));
  if (P->total_cols > 0)
    SHIRO_CUDA(cudaMemcpyAsync(X.cols_sorted.data(), P->d_cols_sorted,
                               sizeof(int32_t) * P->total_cols, cudaMemcpyDeviceToHost, s));
  SHIRO_CUDA(cudaStreamSynchronize(s));
  const bool diag = P->flags & SHIRO_PLAN_DIAG_ONLY;
  const int32_t Pc = P->geo.Pc;
  for (int32_t p = 0; p < P->geo.Pr; ++p)
    for (int64_t i = P->rb[p]; i < P->rb[p + 1]; ++i)
      for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e) {
        const int32_t q = diag ? p : (int32_t)(std::upper_bound(P->cb.begin(), P->cb.end(),
                                                                (int64_t)X.col[e]) - P->cb.begin() - 1);
        const int32_t t = diag ? p : p * Pc + q;
        X.tile_of[e] = t;
        const int32_t* c0 = X.cols_sorted.data() + P->tile_cols_ptr[t];
        const int32_t* c1 = X.cols_sorted.data() + P->tile_cols_ptr[t + 1];
        X.local[e] = (int32_t)(std::lower_bound(c0, c1, X.col[e]) - c0);
      }
  return SHIRO_OK;
}

// The bipartite graph of tile t: left = the row block's rows (local ids), right = the tile's Cols
// positions, one edge per nonzero.
Bipartite tile_bipartite(const shiro_plan_s* P, const TileIndex& X, int32_t t) {
  const bool diag = P->flags & SHIRO_PLAN_DIAG_ONLY;
  const int32_t p = diag ? t : t / P->geo.Pc;
  Bipartite g;
  g.nL = (int32_t)(P->rb[p + 1] - P->rb[p]);
  g.nR = (int32_t)P->tile_ncols[t];
  g.ptr.assign(g.nL + 1, 0);
  for (int32_t u = 0; u < g.nL; ++u) {
    const int64_t i = P->rb[p] + u;
    int64_t cnt = 0;
    for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e) cnt += X.tile_of[e] == t;
    g.ptr[u + 1] = g.ptr[u] + cnt;
  }
  g.adj.resize(g.ptr[g.nL]);
  for (int32_t u = 0; u < g.nL; ++u) {
    const int64_t i = P->rb[p] + u;
    int64_t k = g.ptr[u];
    for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e)
      if (X.tile_of[e] == t) g.adj[k++] = X.local[e];
  }
  return g;
}

// Runs solve(t, g, coverL, coverR) -> cost on every communicated tile in parallel host threads
// and gathers per-tile costs, cover sizes and the side of every nonzero (1 = row-based).
template <class Solve>
void solve_tiles(const shiro_plan_s* P, const TileIndex& X, Solve solve, int64_t* tile_cost,
                 int64_t* tile_cover_rows, int64_t* tile_cover_cols, uint8_t* nnz_row_based) {
  const int32_t T = P->T;
  const bool diag = P->flags & SHIRO_PLAN_DIAG_ONLY;
  const bool local_diag = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  std::vector<int64_t> cost(T, 0), crows(T, 0), ccols(T, 0);
  std::vector<uint8_t> side(P->nnz > 0 ? P->nnz : 1, 0);
  std::atomic<int32_t> next{0};
  auto worker = [&]() {
    while (true) {
      const int32_t t = next.fetch_add(1);
      if (t >= T) break;
      const int32_t p = diag ? t : t / P->geo.Pc, q = diag ? t : t % P->geo.Pc;
      if (local_diag && p == q) continue;  // local tile: nothing is communicated
      const Bipartite g = tile_bipartite(P, X, t);
      std::vector<char> coverL, coverR;
      cost[t] = solve(t, g, coverL, coverR);
      int64_t nr = 0, nc = 0;
      for (char c : coverL) nr += c;
      for (char c : coverR) nc += c;
      crows[t] = nr;
      ccols[t] = nc;
      for (int32_t u = 0; u < g.nL; ++u) {
        const int64_t i = P->rb[p] + u;
        for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e)
          if (X.tile_of[e] == t) side[e] = coverR[X.local[e]] ? 0 : 1;
      }
    }
  };
  const unsigned nt = std::max(1u, std::min(std::thread::hardware_concurrency(), (unsigned)T));
  std::vector<std::thread> pool;
  for (unsigned k = 1; k < nt; ++k) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  if (tile_cost) memcpy(tile_cost, cost.data(), sizeof(int64_t) * T);
  if (tile_cover_rows) memcpy(tile_cover_rows, crows.data(), sizeof(int64_t) * T);
  if (tile_cover_cols) memcpy(tile_cover_cols, ccols.data(), sizeof(int64_t) * T);
  if (nnz_row_based && P->nnz > 0) memcpy(nnz_row_based, side.data(), (size_t)P->nnz);
}

}  // namespace

extern "C" shiro_status shiro_plan_joint(shiro_plan_t P, int64_t* tile_mu,
                                         int64_t* tile_cover_rows, int64_t* tile_cover_cols,
                                         uint8_t* nnz_row_based, void* stream) {
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  TileIndex X;
  SHIRO_TRY(tile_index(P, X, (cudaStream_t)stream));
  auto solve = [](int32_t, const Bipartite& g, std::vector<char>& cl, std::vector<char>& cr) {
    std::vector<int32_t> pairL, pairR;
    const int64_t mu = hopcroft_karp(g, pairL, pairR);
    koenig_cover(g, pairL, pairR, cl, cr);
    return mu;
  };
  solve_tiles(P, X, solve, tile_mu, tile_cover_rows, tile_cover_cols, nnz_row_based);
  return SHIRO_OK;
}

extern "C" shiro_status shiro_plan_joint_weighted(shiro_plan_t P, const int64_t* w_row,
                                                  const int64_t* w_col, int64_t w_row_all,
                                                  int64_t w_col_all, int64_t* tile_cost,
                                                  int64_t* tile_cover_rows,
                                                  int64_t* tile_cover_cols,
                                                  uint8_t* nnz_row_based, void* stream) {
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  // Costs must be >= 0 and every tile's total below 2^62 (the unbounded arc capacity).
  const int64_t LIMIT = ((int64_t)1 << 62) / 4;
  if (!w_row && (w_row_all < 0 || w_row_all > LIMIT / std::max<int64_t>(1, P->M)))
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "row cost out of range");
  if (!w_col && (w_col_all < 0 || w_col_all > LIMIT / std::max<int64_t>(1, P->K)))
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "column cost out of range");
  int64_t sum = 0;
  if (w_row)
    for (int64_t i = 0; i < P->M; ++i) {
      if (w_row[i] < 0 || w_row[i] > LIMIT) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "row cost out of range");
      sum += w_row[i];
      if (sum > LIMIT) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "row costs sum too large");
    }
  sum = 0;
  if (w_col)
    for (int64_t j = 0; j < P->K; ++j) {
      if (w_col[j] < 0 || w_col[j] > LIMIT) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "column cost out of range");
      sum += w_col[j];
      if (sum > LIMIT) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "column costs sum too large");
    }
  TileIndex X;
  SHIRO_TRY(tile_index(P, X, (cudaStream_t)stream));
  const bool diag = P->flags & SHIRO_PLAN_DIAG_ONLY;
  auto solve = [&](int32_t t, const Bipartite& g, std::vector<char>& cl, std::vector<char>& cr) {
    const int32_t p = diag ? t : t / P->geo.Pc;
    std::vector<int64_t> wr(g.nL), wc(g.nR);
    for (int32_t u = 0; u < g.nL; ++u) wr[u] = w_row ? w_row[P->rb[p] + u] : w_row_all;
    const int32_t* cols = X.cols_sorted.data() + P->tile_cols_ptr[t];
    for (int32_t v = 0; v < g.nR; ++v) wc[v] = w_col ? w_col[cols[v]] : w_col_all;
    return dinic_cover(g, wr, wc, cl, cr);
  };
  solve_tiles(P, X, solve, tile_cost, tile_cover_rows, tile_cover_cols, nnz_row_based);
  return SHIRO_OK;
}

extern "C" shiro_status shiro_plan_row_based(shiro_plan_t P, int64_t* tile_rows,
                                             uint8_t* nnz_row_based, void* stream) {
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  TileIndex X;
  SHIRO_TRY(tile_index(P, X, (cudaStream_t)stream));
  // Every row of a communicated tile that holds a nonzero is selected, no column (Eq. 3).
  auto solve = [](int32_t, const Bipartite& g, std::vector<char>& cl, std::vector<char>& cr) {
    cl.assign(g.nL, 0);
    cr.assign(g.nR, 0);
    int64_t n = 0;
    for (int32_t u = 0; u < g.nL; ++u) {
      cl[u] = g.ptr[u + 1] > g.ptr[u] ? 1 : 0;
      n += cl[u];
    }
    return n;
  };
  solve_tiles(P, X, solve, tile_rows, nullptr, nullptr, nnz_row_based);
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
