// plan_kernels.cuh -- device kernels of the plan (sparsity analysis, Sec. 5.1 stage 1).
//
// Cols(A^(p,q)) (Tab. 1, Eq. 2) is found with one presence bitmap per tile: bit c of tile t is set
// when some nonzero of the tile has column cb[q] + c.  Every tile's bitmap starts on a word
// boundary, so an exclusive scan of the words' popcounts gives, for every set bit, its global
// position in the concatenation of the tiles' ascending Cols lists; the remap of a nonzero is the
// scan value of its word plus the popcount of the lower bits.  Rows(A^(p,q)) (Eq. 3) uses a second
// bitmap per tile over the tile's rows.
#pragma once

#include "internal.cuh"

namespace shiro {

constexpr int kScanItems = 16;
constexpr int kScanThreads = 256;
constexpr int64_t kScanTile = (int64_t)kScanItems * kScanThreads;  // 4096

__global__ void k_validate_rowptr(const int64_t* __restrict__ rowptr, int64_t M, int64_t nnz,
                                  int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (i == 0 && (rowptr[0] != 0 || rowptr[M] != nnz)) atomicOr(status, ST_BAD_ROWPTR);
  for (; i < M; i += stride)
    if (rowptr[i] > rowptr[i + 1]) atomicOr(status, ST_BAD_ROWPTR);
}

__global__ void k_validate_cols(const int32_t* __restrict__ col, int64_t nnz, int64_t K,
                                int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < nnz; i += stride)
    if (col[i] < 0 || col[i] >= K) atomicOr(status, ST_BAD_COL);
}

// Marks the column and row bitmaps and counts nonzeros per tile.  One warp per row.
template <bool DIAG>
__global__ void __launch_bounds__(256) k_mark(const int64_t* __restrict__ rowptr,
                                              const int32_t* __restrict__ col, Geometry g,
                                              const int64_t* __restrict__ woff,
                                              uint32_t* bitmap,
                                              const int64_t* __restrict__ rwoff,
                                              uint32_t* rbitmap, unsigned long long* tile_nnz,
                                              int32_t T, int* status) {
  extern __shared__ unsigned int s_cnt[];
  const bool smem = T <= 4096;
  if (smem)
    for (int t = threadIdx.x; t < T; t += blockDim.x) s_cnt[t] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < g.M;
       i += warps) {
    const int32_t p = row_block(g, i);
    const int64_t r_local = i - g.rb[p];
    const int64_t e_end = rowptr[i + 1];
    for (int64_t e0 = rowptr[i]; e0 < e_end; e0 += 32) {
      const int64_t e = e0 + lane;
      int32_t t = -1;
      if (e < e_end) {
        const int64_t j = col[e];
        if (j < 0 || j >= g.K) {
          atomicOr(status, ST_BAD_COL);
        } else {
          int32_t q;
          if (DIAG) {
            q = p;
            if (j < g.cb[p] || j >= g.cb[p + 1]) { atomicOr(status, ST_OFF_DIAG); q = -1; }
          } else {
            q = col_block(g, j);
          }
          if (q >= 0) {
            t = DIAG ? p : p * g.Pc + q;
            const int64_t c = j - g.cb[q];
            uint32_t* w = bitmap + woff[t] + (c >> 5);
            const uint32_t bit = 1u << (c & 31);
            if (!(*(volatile uint32_t*)w & bit)) atomicOr(w, bit);
          }
        }
      }
      const unsigned active = __ballot_sync(0xffffffffu, true);
      const unsigned peers = __match_any_sync(active, t);
      const int leader = __ffs(peers) - 1;
      if (t >= 0 && lane == leader) {
        const unsigned cnt = __popc(peers);
        if (smem) atomicAdd(&s_cnt[t], cnt); else atomicAdd(&tile_nnz[t], (unsigned long long)cnt);
        uint32_t* rw = rbitmap + rwoff[t] + (r_local >> 5);
        const uint32_t rbit = 1u << (r_local & 31);
        if (!(*(volatile uint32_t*)rw & rbit)) atomicOr(rw, rbit);
      }
    }
  }
  __syncthreads();
  if (smem)
    for (int t = threadIdx.x; t < T; t += blockDim.x)
      if (s_cnt[t]) atomicAdd(&tile_nnz[t], (unsigned long long)s_cnt[t]);
}

// ---- exclusive scan of an int64 array in place (3 kernels) ----
// s_warp must hold 33 entries: one per warp plus the block total.

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t x, int64_t* s_warp,
                                                        int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    int64_t v = lane < nw ? s_warp[lane] : 0;
    int64_t vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < nw) s_warp[lane] = vi - v;
    if (lane == nw - 1) s_warp[32] = vi;
  }
  __syncthreads();
  const int64_t r = s_warp[warp] + inc - x;
  if (total) *total = s_warp[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int64_t* __restrict__ a,
                                                              int64_t n, int64_t* bsum) {
  __shared__ int64_t s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += a[base + k];
  int64_t tot;
  block_exclusive_scan(s, s_warp, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(int64_t* bsum, int64_t nb, int* status,
                                                   int64_t limit) {
  __shared__ int64_t s_warp[33];
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < nb ? bsum[i] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_scan(v, s_warp, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    bsum[nb] = carry;
    if (limit > 0 && carry > limit) atomicOr(status, ST_OVERFLOW);
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(int64_t* a, int64_t n,
                                                            const int64_t* __restrict__ bsum) {
  __shared__ int64_t s_warp[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? a[base + k] : 0;
    s += v[k];
  }
  int64_t ex = bsum[blockIdx.x] + block_exclusive_scan(s, s_warp, nullptr);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) {
      a[base + k] = ex;
      ex += v[k];
    }
}

__global__ void k_popc_words(const uint32_t* __restrict__ bm, int64_t W, int64_t* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i <= W; i += stride) out[i] = i < W ? __popc(bm[i]) : 0;
}

// |Rows| of every tile: popcount of its row bitmap.  One warp per tile.
__global__ void k_tile_rows(const uint32_t* __restrict__ rbm, const int64_t* __restrict__ rwoff,
                            int32_t T, unsigned long long* nrows) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < T;
       t += warps) {
    unsigned long long s = 0;
    for (int64_t w = rwoff[t] + lane; w < rwoff[t + 1]; w += 32) s += __popc(rbm[w]);
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrows[t] = s;
  }
}

__global__ void k_tile_cols_ptr(const int64_t* __restrict__ wprefix,
                                const int64_t* __restrict__ woff, int32_t T, int64_t* out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= T) out[t] = wprefix[woff[t]];
}

// Writes Cols of every tile in ascending order, and the gather list of packed tiles.
__global__ void k_emit_cols(const uint32_t* __restrict__ bm, int64_t W,
                            const int64_t* __restrict__ woff, int32_t T, Geometry g,
                            const int64_t* __restrict__ wprefix,
                            const int64_t* __restrict__ tile_cols_ptr,
                            const int64_t* __restrict__ pack_ptr, int local_diag,
                            int32_t* cols_sorted, int32_t* pack_src) {
  int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; w < W; w += stride) {
    uint32_t bits = bm[w];
    if (!bits) continue;
    const int32_t t = find_block(woff, T, w);
    const int32_t p = g.diag_only ? t : t / g.Pc;
    const int32_t q = g.diag_only ? t : t % g.Pc;
    const int64_t c0 = g.cb[q] + (w - woff[t]) * 32;
    int64_t pos = wprefix[w];
    const bool packed = pack_src != cols_sorted;
    const bool is_local = local_diag && p == q;
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      const int32_t c = (int32_t)(c0 + b);
      cols_sorted[pos] = c;
      if (packed && !is_local) pack_src[pack_ptr[t] + (pos - tile_cols_ptr[t])] = c;
      ++pos;
    }
  }
}

// remap[e]: packed row of nonzero e (or -1 - col for local diagonal tiles);
// colidx[e]: position of col[e] in its tile's Cols.  Either output may be null.
template <bool DIAG>
__global__ void __launch_bounds__(256) k_remap(const int64_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ col, Geometry g,
                                               const int64_t* __restrict__ woff,
                                               const uint32_t* __restrict__ bm,
                                               const int64_t* __restrict__ wprefix,
                                               const int64_t* __restrict__ tile_cols_ptr,
                                               const int64_t* __restrict__ pack_ptr,
                                               int local_diag, int32_t* remap, int32_t* colidx) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < g.M;
       i += warps) {
    const int32_t p = row_block(g, i);
    const int64_t e_end = rowptr[i + 1];
    for (int64_t e = rowptr[i] + lane; e < e_end; e += 32) {
      const int64_t j = col[e];
      const int32_t q = DIAG ? p : col_block(g, j);
      const int32_t t = DIAG ? p : p * g.Pc + q;
      const int64_t c = j - g.cb[q];
      const int64_t w = woff[t] + (c >> 5);
      const uint32_t lower = bm[w] & ((1u << (c & 31)) - 1u);
      const int64_t local = wprefix[w] - tile_cols_ptr[t] + __popc(lower);
      if (colidx) colidx[e] = (int32_t)local;
      if (remap) remap[e] = (local_diag && p == q) ? (int32_t)(-1 - j) : (int32_t)(pack_ptr[t] + local);
    }
  }
}

// ---- CSR transpose by a stable LSD radix sort of the column indices ----

constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 8;
constexpr int64_t kRadixTile = (int64_t)kRadixThreads * kRadixRounds;  // 2048

// Column of the first nonzero of each chunk item (schedule ordering).
__global__ void k_chunk_first_col(const Item* __restrict__ items, int64_t n,
                                  const int32_t* __restrict__ col, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = col[items[i].e0];
}

__global__ void k_row_ids(const int64_t* __restrict__ rowptr, int64_t M, int32_t* rowid) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < M;
       i += warps)
    for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) rowid[e] = (int32_t)i;
}

__global__ void k_iota_copy(const int32_t* __restrict__ col, int64_t n, uint32_t* keys,
                            int32_t* vals) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) {
    keys[i] = (uint32_t)col[i];
    vals[i] = (int32_t)i;
  }
}

__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                              int64_t n, int shift,
                                                              int64_t nblocks, int64_t* hist) {
  __shared__ unsigned int s_hist[256];
  s_hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int r = 0; r < kRadixRounds; ++r) {
    const int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
    if (i < n) atomicAdd(&s_hist[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_hist[threadIdx.x];
}

// Stable scatter: elements keep their input order among equal digits.
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    const uint32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in, int64_t n,
    int shift, int64_t nblocks, const int64_t* __restrict__ offsets, uint32_t* keys_out,
    int32_t* vals_out) {
  __shared__ int64_t s_base[256];
  __shared__ int s_wcnt[kRadixThreads / 32][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  s_base[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int r = 0; r < kRadixRounds; ++r) {
    for (int w = 0; w < kRadixThreads / 32; ++w) s_wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
    const bool valid = i < n;
    const uint32_t key = valid ? keys_in[i] : 0u;
    const int d = valid ? (int)((key >> shift) & 255u) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt_mask);
    if (valid && rank == 0) s_wcnt[warp][d] = __popc(peers);
    __syncthreads();
    int run = 0;
    for (int w = 0; w < kRadixThreads / 32; ++w) {
      const int c = s_wcnt[w][threadIdx.x];
      s_wcnt[w][threadIdx.x] = run;
      run += c;
    }
    __syncthreads();
    if (valid) {
      const int64_t pos = s_base[d] + s_wcnt[warp][d] + rank;
      keys_out[pos] = key;
      vals_out[pos] = vals_in[i];
    }
    __syncthreads();
    s_base[threadIdx.x] += run;
    __syncthreads();
  }
}

// rowptrT[j] = first position of key j in the sorted keys (K + 1 entries).
__global__ void k_rowptr_from_sorted(const uint32_t* __restrict__ keys, int64_t n, int64_t K,
                                     int64_t* rowptrT) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i <= n; i += stride) {
    const int64_t prev = i == 0 ? -1 : (int64_t)keys[i - 1];
    const int64_t cur = i == n ? K : (int64_t)keys[i];
    for (int64_t j = prev + 1; j <= cur; ++j) rowptrT[j] = i;
  }
}

template <typename TV>
__global__ void k_gather_transpose(const int32_t* __restrict__ perm32,
                                   const int32_t* __restrict__ rowid,
                                   const TV* __restrict__ val, int64_t n, int32_t* colT,
                                   TV* valT, int64_t* perm64) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) {
    const int32_t e = perm32[i];
    if (colT) colT[i] = rowid[e];
    if (valT) valT[i] = val[e];
    if (perm64) perm64[i] = e;
  }
}

template <typename TV>
__global__ void k_gather_values(const int64_t* __restrict__ perm, const TV* __restrict__ val,
                                int64_t n, TV* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) out[i] = val[perm[i]];
}

// ---- batch: concatenate G graphs into one block-diagonal CSR ----

struct GraphDesc {
  const int64_t* rowptr;
  const int32_t* col;
  const void* val;
  int64_t M, nnz, roff, coff, eoff;
};

template <typename TV>
__global__ void k_concat(const GraphDesc* __restrict__ gd, int32_t G, int64_t* rowptr,
                         int32_t* col, TV* val) {
  for (int32_t g = blockIdx.x; g < G; g += gridDim.x) {
    const GraphDesc d = gd[g];
    for (int64_t i = threadIdx.x; i < d.M; i += blockDim.x)
      rowptr[d.roff + i] = d.rowptr[i] + d.eoff;
    const TV* v = (const TV*)d.val;
    for (int64_t e = threadIdx.x; e < d.nnz; e += blockDim.x) {
      col[d.eoff + e] = (int32_t)(d.col[e] + d.coff);
      val[d.eoff + e] = v[e];
    }
    if (g == G - 1 && threadIdx.x == 0) rowptr[d.roff + d.M] = d.eoff + d.nnz;
  }
}

}  // namespace shiro
