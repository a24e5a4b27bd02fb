// spmm_ring.cuh -- the SpMM work loop with every gathered B row landing in a per-warp ring of R
// shared-memory row slots, refilled R rows ahead of their use by per-lane asynchronous copies.
//
// Lane l copies (cp.async, 4-16 bytes) only its own slice of every row and later reads back only
// that slice, so a lane waits only for its own copies (cp.async.wait_group, one commit group per
// G rows) and no barrier or cross-lane wait exists; the warp accumulates the oldest G rows and
// refills their slots with the rows R positions on, so R rows stay in flight without holding
// registers.  The (index, value) pairs of two batches of 32
// sit in shared memory (the copies of the rows R positions on read their indices there); the
// pairs of the batch after those are held in lane registers.  Rows are summed in the same order
// as the register-gather loop, so C is bit-identical to it.
#pragma once

#include "internal.cuh"
#include "vec.cuh"

namespace shiro {

template <typename TV, typename TB, int VEC, int NCH, int R, int G>
struct LRingLayout {
  static constexpr int PIECE = VEC * (int)sizeof(TB);  // bytes per lane per chunk
  static constexpr int ROW = 32 * PIECE * NCH;         // bytes of one row (N * sz)
  static constexpr int NG = R / G;
  static constexpr int PAIRS = 64 * (int)sizeof(Pair<TV>);
  static constexpr int WARP = (R * ROW + PAIRS + 127) / 128 * 128;
  static_assert(R % G == 0 && NG >= 2 && R <= 32 && 32 % G == 0, "ring shape");
};

template <typename TV, typename TB, int VEC, int NCH, int R, int G, bool LOCAL>
__device__ __forceinline__ void spmm_span_lring(const SpmmParams<TV, TB>& p, char* wsm,
                                                int64_t base, int total, int32_t r0, int nr,
                                                int rel, bool nonempty,
                                                typename AccOf<TB>::T (&acc)[NCH][VEC],
                                                int lane) {
  using TA = typename AccOf<TB>::T;
  using L = LRingLayout<TV, TB, VEC, NCH, R, G>;
  if (total <= 0) return;
  Pair<TV>* sp = reinterpret_cast<Pair<TV>*>(wsm + R * L::ROW);
  const uint32_t s_slots = (uint32_t)__cvta_generic_to_shared(wsm) + lane * L::PIECE;
  const TB* my_slots = reinterpret_cast<const TB*>(wsm) + lane * VEC;
  __syncwarp();
  {
    Pair<TV> pr;
    pr.idx = lane < total ? __ldcs(p.remap + base + lane) : 0;
    pr.val = lane < total ? __ldcs(p.val + base + lane) : (TV)0;
    sp[lane] = pr;
  }
  int32_t nidx = 0;
  TV nval = 0;
  if (32 + lane < total) {
    nidx = __ldcs(p.remap + base + 32 + lane);
    nval = __ldcs(p.val + base + 32 + lane);
  }
  __syncwarp();
  int ib = 0;  // batches up to ib are staged in shared memory
  // Copies of rows k*G .. k*G+G-1 (those below total) as one commit group (empty past the end,
  // so that every wait below keeps the same constant count).
  auto issue = [&](int k) {
    const int t0 = k * G;
    if (t0 < total && (t0 >> 5) > ib) {
      // The copies enter batch ib + 1: stage its pairs (batch ib - 1, two back, is consumed).
      ib = t0 >> 5;
      __syncwarp();
      Pair<TV> pr;
      pr.idx = nidx;
      pr.val = nval;
      sp[(ib & 1) * 32 + lane] = pr;
      nidx = 0;
      nval = 0;
      if (32 * (ib + 1) + lane < total) {
        nidx = __ldcs(p.remap + base + 32 * (ib + 1) + lane);
        nval = __ldcs(p.val + base + 32 * (ib + 1) + lane);
      }
      __syncwarp();
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int t = t0 + g;
      if (t < total) {
        const int32_t idx = sp[t & 63].idx;
        const TB* row;
        if (LOCAL && idx < 0)
          row = p.B + (uint64_t)(uint32_t)(-1 - idx) * (uint64_t)p.ldb;
        else
          row = p.Bpack + (uint64_t)(uint32_t)idx * (uint64_t)p.ldp;
        const uint32_t dst = s_slots + (uint32_t)(t % R) * L::ROW;
#pragma unroll
        for (int c = 0; c < NCH; ++c)
          cp_async<L::PIECE>(dst + c * 32 * L::PIECE, row + c * 32 * VEC + lane * VEC);
      }
    }
    cp_async_commit();
  };
#pragma unroll 1
  for (int k = 0; k < L::NG; ++k) issue(k);
  const int ngroups = (total + G - 1) / G;
  int cb = -1;
  unsigned endmask = 0;
#pragma unroll 1
  for (int k = 0; k < ngroups; ++k) {
    cp_async_wait<L::NG - 1>();
    const int t0 = k * G;
    if ((t0 >> 5) != cb) {
      cb = t0 >> 5;
      const int q = rel - 1 - 32 * cb;
      const unsigned bit = (lane < nr && nonempty && q >= 0 && q < 32) ? (1u << q) : 0u;
      endmask = __reduce_or_sync(0xffffffffu, bit);
    }
    const int n = min(G, total - t0);
    const unsigned ends = (endmask >> (t0 & 31)) & ((1u << G) - 1u);
    if (n == G && ends == 0) {
      TA b[G][NCH][VEC];
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int c = 0; c < NCH; ++c)
          load_vec<TB, VEC, false>(
              my_slots + ((t0 + g) % R) * (L::ROW / (int)sizeof(TB)) + c * 32 * VEC, b[g][c]);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const TA a = (TA)sp[(t0 + g) & 63].val;
#pragma unroll
        for (int c = 0; c < NCH; ++c)
#pragma unroll
          for (int v = 0; v < VEC; ++v) acc[c][v] = fma(a, b[g][c][v], acc[c][v]);
      }
    } else {
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (g < n) {
          const TA a = (TA)sp[(t0 + g) & 63].val;
#pragma unroll
          for (int c = 0; c < NCH; ++c) {
            TA b[VEC];
            load_vec<TB, VEC, false>(
                my_slots + ((t0 + g) % R) * (L::ROW / (int)sizeof(TB)) + c * 32 * VEC, b);
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] = fma(a, b[v], acc[c][v]);
          }
          if ((ends >> g) & 1u) {
            const unsigned who = __ballot_sync(0xffffffffu, lane < nr && rel == t0 + g + 1);
            flush_row<TV, TB, VEC, NCH, false>(p, r0 + __ffs(who) - 1, acc, lane);
          }
        }
      }
    }
    issue(k + L::NG);
  }
  cp_async_wait<0>();
  __syncwarp();
}

template <typename TV, typename TB, int VEC, int NCH, int R, int G, bool LOCAL>
__global__ void __launch_bounds__(256) k_spmm_lring(const SpmmParams<TV, TB> p) {
  extern __shared__ __align__(128) char smem[];
  using L = LRingLayout<TV, TB, VEC, NCH, R, G>;
  using TA = typename AccOf<TB>::T;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  char* wsm = smem + warp * L::WARP;
  if ((int64_t)blockIdx.x < p.chunk_blocks) {
    const int64_t step = (int64_t)p.chunk_blocks * wpb;
    for (int64_t it = (int64_t)blockIdx.x * wpb + warp; it < p.n_chunk_items; it += step) {
      const Item item = p.items[it];
      const int32_t slot = -item.tag - 1;
      const int64_t row_end = __ldg(p.rowptr + item.row + 1);
      const int total = (int)min((int64_t)p.chunk, row_end - item.e0);
      TA acc[NCH][VEC];
#pragma unroll
      for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[c][v] = 0;
      spmm_span_lring<TV, TB, VEC, NCH, R, G, LOCAL>(p, wsm, item.e0, total, item.row, 0, 0,
                                                     false, acc, lane);
      finish_chunk<TV, TB, VEC, NCH, false>(p, slot, acc, lane);
    }
  } else {
    const int64_t nb = (int64_t)gridDim.x - p.chunk_blocks;
    const int64_t step = p.persistent ? nb * wpb : p.n_items;
    for (int64_t it = p.n_chunk_items + ((int64_t)blockIdx.x - p.chunk_blocks) * wpb + warp;
         it < p.n_items; it += step) {
      const Item item = p.items[it];
      const int32_t r0 = item.row, nr = item.tag;
      const int64_t rp = lane < nr ? __ldg(p.rowptr + r0 + lane + 1) : 0;
      const int rel = (int)(rp - item.e0);
      const int prev = __shfl_up_sync(0xffffffffu, rel, 1);
      const bool nonempty = lane < nr && rel > (lane ? prev : 0);
      const int total = __shfl_sync(0xffffffffu, rel, nr - 1);
      TA acc[NCH][VEC];
#pragma unroll
      for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[c][v] = 0;
      if (!p.accumulate) {
        unsigned empty = __ballot_sync(0xffffffffu, lane < nr && !nonempty);
        while (empty) {
          const int l = __ffs(empty) - 1;
          empty &= empty - 1;
          flush_row<TV, TB, VEC, NCH, false>(p, r0 + l, acc, lane);
        }
      }
      spmm_span_lring<TV, TB, VEC, NCH, R, G, LOCAL>(p, wsm, item.e0, total, r0, nr, rel,
                                                     nonempty, acc, lane);
    }
  }
}

}  // namespace shiro
