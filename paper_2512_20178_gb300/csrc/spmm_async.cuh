// spmm_async.cuh -- the SpMM work loop with the B-row gathers staged through shared memory by
// asynchronous copies (cp.async), two stages of BATCH rows per warp.
//
// Every lane copies only its own VEC-element slice of each gathered row (4, 8 or 16 bytes) and
// later reads back only that slice, so the staged data needs no cross-lane synchronisation and
// `cp.async.wait_group` (a wait on the lane's own copies) cannot stall forever.  Bytes in flight no
// longer cost registers: a warp keeps up to 2 * BATCH rows outstanding while it accumulates the
// previous batch.  The (index, value) pairs of a batch are shared through shared memory.
#pragma once

#include "internal.cuh"
#include "vec.cuh"

namespace shiro {

template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t smem, const void* gmem) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem), "l"(gmem), "n"(BYTES)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Read back VEC elements of a staged slice (shared memory, same layout as global).
template <typename TB, int VEC>
__device__ __forceinline__ void lds_vec(const TB* p, typename AccOf<TB>::T (&out)[VEC]) {
  load_vec<TB, VEC, false>(p, out);
}

template <typename TV, typename TB, int VEC, int NCH, int BATCH>
struct AsyncLayout {
  static constexpr int PIECE = VEC * (int)sizeof(TB);      // bytes per lane per chunk
  static constexpr int ROW = 32 * PIECE * NCH;             // bytes of one staged row
  static constexpr int STAGE = BATCH * ROW;
  static constexpr int PAIRS = 32 * (int)sizeof(Pair<TV>);
  static constexpr int WARP = 2 * STAGE + 2 * PAIRS;       // shared bytes per warp
};

// Accumulates nonzeros [base, base + total) exactly like spmm_span, with staged gathers.
template <typename TV, typename TB, int VEC, int NCH, int BATCH, bool LOCAL>
__device__ __forceinline__ void spmm_span_async(const SpmmParams<TV, TB>& p, char* wsm,
                                                int64_t base, int total, int32_t r0, int nr,
                                                int rel, bool nonempty,
                                                typename AccOf<TB>::T (&acc)[NCH][VEC], int lane) {
  using TA = typename AccOf<TB>::T;
  using L = AsyncLayout<TV, TB, VEC, NCH, BATCH>;
  static_assert(BATCH <= 32, "a batch is at most one index load per lane");
  char* stage_base = wsm;
  Pair<TV>* pairs = reinterpret_cast<Pair<TV>*>(wsm + 2 * L::STAGE);
  const uint32_t s_stage = (uint32_t)__cvta_generic_to_shared(stage_base);
  const int nb = (total + BATCH - 1) / BATCH;

  // Index/value registers hold the pairs of the next batch to be staged.
  int32_t nidx = 0;
  TV nval = 0;
  if (lane < BATCH && lane < total) {
    nidx = __ldcs(p.remap + base + lane);
    nval = __ldcs(p.val + base + lane);
  }
  // Stage batch k: publish its pairs, then every lane copies its slices of the batch's rows.
  auto issue = [&](int k) {
    const int s = k & 1;
    const int off = k * BATCH;
    const int n = min(BATCH, total - off);
    Pair<TV> pr;
    pr.idx = nidx;
    pr.val = nval;
    if (lane < BATCH) pairs[s * 32 + lane] = pr;
    const int32_t my_idx = nidx;
    const int nxt = off + BATCH + lane;
    if (lane < BATCH && nxt < total) {
      nidx = __ldcs(p.remap + base + nxt);
      nval = __ldcs(p.val + base + nxt);
    }
    // Row indices come from the lanes' registers by shuffle, fully unrolled, so the copies of a
    // batch issue back to back instead of one dependent index read per row.
    const uint32_t dst0 = s_stage + s * L::STAGE + lane * L::PIECE;
#pragma unroll
    for (int j = 0; j < BATCH; ++j) {
      const int32_t idx = __shfl_sync(0xffffffffu, my_idx, j);
      if (j < n) {
        const TB* row;
        if (LOCAL && idx < 0)
          row = p.B + (uint64_t)(uint32_t)(-1 - idx) * (uint32_t)p.ldb;
        else
          row = p.Bpack + (uint64_t)(uint32_t)idx * (uint32_t)p.ldp;
#pragma unroll
        for (int c = 0; c < NCH; ++c)
          cp_async<L::PIECE>(dst0 + j * L::ROW + c * 32 * L::PIECE,
                             row + c * 32 * VEC + lane * VEC);
      }
    }
    cp_async_commit();
    __syncwarp();
  };

  if (nb > 0) issue(0);
  for (int k = 0; k < nb; ++k) {
    if (k + 1 < nb) {
      issue(k + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    const int s = k & 1;
    const int off = k * BATCH;
    const int n = min(BATCH, total - off);
    const int q = rel - 1 - off;
    const unsigned bit = (lane < nr && nonempty && q >= 0 && q < 32) ? (1u << q) : 0u;
    const unsigned endmask = __reduce_or_sync(0xffffffffu, bit);
    const TB* slot = reinterpret_cast<const TB*>(stage_base + s * L::STAGE) + lane * VEC;
    const Pair<TV>* pk = pairs + s * 32;
#pragma unroll 4
    for (int j = 0; j < n; ++j) {
      const TA a = (TA)pk[j].val;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        TA b[VEC];
        lds_vec<TB, VEC>(slot + (j * L::ROW + c * 32 * L::PIECE) / (int)sizeof(TB), b);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[c][v] = fma(a, b[v], acc[c][v]);
      }
      if ((endmask >> j) & 1u) {
        const unsigned who = __ballot_sync(0xffffffffu, lane < nr && rel == off + j + 1);
        flush_row<TV, TB, VEC, NCH, false>(p, r0 + __ffs(who) - 1, acc, lane);
      }
    }
    __syncwarp();
  }
}

template <typename TV, typename TB, int VEC, int NCH, int BATCH, bool LOCAL>
__device__ __forceinline__ void run_group_async(const SpmmParams<TV, TB>& p, char* wsm,
                                                const Item& item, int lane) {
  using TA = typename AccOf<TB>::T;
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
  spmm_span_async<TV, TB, VEC, NCH, BATCH, LOCAL>(p, wsm, item.e0, total, r0, nr, rel, nonempty,
                                                  acc, lane);
}

template <typename TV, typename TB, int VEC, int NCH, int BATCH, bool LOCAL>
__device__ __forceinline__ void run_chunk_async(const SpmmParams<TV, TB>& p, char* wsm,
                                                const Item& item, int lane) {
  using TA = typename AccOf<TB>::T;
  const int32_t i = item.row;
  const int32_t slot = -item.tag - 1;
  const int64_t row_end = __ldg(p.rowptr + i + 1);
  const int total = (int)min((int64_t)p.chunk, row_end - item.e0);
  TA acc[NCH][VEC];
#pragma unroll
  for (int c = 0; c < NCH; ++c)
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[c][v] = 0;
  spmm_span_async<TV, TB, VEC, NCH, BATCH, LOCAL>(p, wsm, item.e0, total, i, 0, 0, false, acc,
                                                  lane);
  finish_chunk<TV, TB, VEC, NCH, false>(p, slot, acc, lane);
}

template <typename TV, typename TB, int VEC, int NCH, int BATCH, bool LOCAL>
__global__ void __launch_bounds__(256) k_spmm_async(const SpmmParams<TV, TB> p) {
  extern __shared__ __align__(16) char smem[];
  using L = AsyncLayout<TV, TB, VEC, NCH, BATCH>;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  char* wsm = smem + warp * L::WARP;
  if ((int64_t)blockIdx.x < p.chunk_blocks) {
    const int64_t step = (int64_t)p.chunk_blocks * wpb;
    for (int64_t it = (int64_t)blockIdx.x * wpb + warp; it < p.n_chunk_items; it += step) {
      const Item item = p.items[it];
      run_chunk_async<TV, TB, VEC, NCH, BATCH, LOCAL>(p, wsm, item, lane);
    }
  } else {
    const int64_t nb = (int64_t)gridDim.x - p.chunk_blocks;
    const int64_t step = p.persistent ? nb * wpb : p.n_items;
    for (int64_t it = p.n_chunk_items + ((int64_t)blockIdx.x - p.chunk_blocks) * wpb + warp;
         it < p.n_items; it += step) {
      const Item item = p.items[it];
      run_group_async<TV, TB, VEC, NCH, BATCH, LOCAL>(p, wsm, item, lane);
    }
  }
}

}  // namespace shiro
