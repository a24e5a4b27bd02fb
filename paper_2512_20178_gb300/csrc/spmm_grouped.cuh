// spmm_grouped.cuh -- SpMM for narrow rows (128 or 256 bytes): the warp splits into G lane groups
// of 32 / G lanes, every lane holding a 16-byte slice of a row, and the groups take interleaved
// nonzeros of the same row (group g: nonzeros g, g + G, g + 2G, ...).  One warp load then gathers
// G rows instead of one, so a warp keeps G * U rows in flight.  At the end of a row the G partial
// sums are combined by a butterfly over the groups (shuffle xor 16, 8 ... 32 / G) and written once;
// the order is fixed, so results are deterministic (but not bit-identical to the one-row-per-warp
// pipelines, whose per-row order is sequential).
#pragma once

#include "internal.cuh"
#include "vec.cuh"

namespace shiro {

template <typename TA, int VEC, int G>
__device__ __forceinline__ void group_allreduce(TA (&acc)[VEC]) {
#pragma unroll
  for (int off = 16; off >= 32 / G; off >>= 1)
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
}

// Writes the row held by group 0 (lanes 0 .. 32/G - 1) and clears every lane's accumulator.
template <typename TV, typename TB, int VEC, int G>
__device__ __forceinline__ void flush_row_grouped(const SpmmParams<TV, TB>& p, int32_t r,
                                                  typename AccOf<TB>::T (&acc)[VEC], int lane) {
  using TA = typename AccOf<TB>::T;
  if (lane < 32 / G) {
    TA* c = p.C + (int64_t)r * p.ldc + lane * VEC;
    if (p.accumulate) {
      TA old[VEC];
      load_acc_cg<TA, VEC>(c, old);
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[v] += old[v];
    }
    store_vec<TA, VEC, true>(c, acc);
  }
#pragma unroll
  for (int v = 0; v < VEC; ++v) acc[v] = 0;
}

// Accumulates this lane group's share of nonzeros [e0, e1) of one row into acc.
template <typename TV, typename TB, int VEC, int G, int U, bool LOCAL>
__device__ __forceinline__ void grouped_row(const SpmmParams<TV, TB>& p, int64_t e0, int64_t e1,
                                            typename AccOf<TB>::T (&acc)[VEC], int g, int sub) {
  using TA = typename AccOf<TB>::T;
  for (int64_t e = e0 + g; e < e1; e += (int64_t)G * U) {
    TA b[U][VEC];
    TV a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t ee = e + (int64_t)u * G;
      if (ee < e1) {
        const int32_t idx = __ldcs(p.remap + ee);
        a[u] = __ldcs(p.val + ee);
        const TB* row;
        if (LOCAL && idx < 0)
          row = p.B + (uint64_t)(uint32_t)(-1 - idx) * (uint32_t)p.ldb;
        else
          row = p.Bpack + (uint64_t)(uint32_t)idx * (uint32_t)p.ldp;
        load_vec<TB, VEC, true>(row + sub * VEC, b[u]);
      } else {
        a[u] = 0;
#pragma unroll
        for (int v = 0; v < VEC; ++v) b[u][v] = 0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[v] = fma((TA)a[u], b[u][v], acc[v]);
  }
}

template <typename TV, typename TB, int VEC, int G, int U, bool LOCAL>
__global__ void __launch_bounds__(256, 4) k_spmm_grouped(const SpmmParams<TV, TB> p) {
  using TA = typename AccOf<TB>::T;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int g = lane / (32 / G);    // lane group
  const int sub = lane % (32 / G);  // slice of the row held by this lane
  TA acc[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) acc[v] = 0;
  if ((int64_t)blockIdx.x < p.chunk_blocks) {
    const int64_t step = (int64_t)p.chunk_blocks * wpb;
    for (int64_t it = (int64_t)blockIdx.x * wpb + warp; it < p.n_chunk_items; it += step) {
      const Item item = p.items[it];
      const int32_t slot = -item.tag - 1;
      const int64_t row_end = __ldg(p.rowptr + item.row + 1);
      const int64_t e1 = min(item.e0 + (int64_t)p.chunk, row_end);
      grouped_row<TV, TB, VEC, G, U, LOCAL>(p, item.e0, e1, acc, g, sub);
      group_allreduce<TA, VEC, G>(acc);
      // Partial of this chunk (group 0), arrival count, ordered sum by the last chunk.
      TA* part = p.scratch + (int64_t)slot * p.N + lane * VEC;
      if (lane < 32 / G) store_acc_cg<TA, VEC>(part, acc);
      // Release (fence, then a warp barrier before lane 0's arrival count) and acquire (lane 0
      // fences after the count, a warp barrier before any lane reads the other partials).
      __threadfence();
      __syncwarp();
      const int32_t lr = __ldg(p.slot_lr + slot);
      const LongRow L = p.lr[lr];
      int old = 0;
      if (lane == 0) {
        __threadfence();
        old = atomicAdd(p.counters + lr, 1);
        __threadfence();
      }
      __syncwarp();
      old = __shfl_sync(0xffffffffu, old, 0);
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[v] = 0;
      if (old == L.nchunks - 1) {
        __threadfence();
        if (lane < 32 / G) {
          for (int32_t s = 0; s < L.nchunks; ++s) {
            TA t[VEC];
            load_acc_cg<TA, VEC>(p.scratch + (int64_t)(L.slot0 + s) * p.N + lane * VEC, t);
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] += t[v];
          }
        }
        flush_row_grouped<TV, TB, VEC, G>(p, L.row, acc, lane);
        if (lane == 0) p.counters[lr] = 0;
      } else if (old >= L.nchunks) {
        if (lane == 0) atomicOr(p.status, ST_COUNTER);
      }
    }
  } else {
    const int64_t nb = (int64_t)gridDim.x - p.chunk_blocks;
    const int64_t step = p.persistent ? nb * wpb : p.n_items;
    for (int64_t it = p.n_chunk_items + ((int64_t)blockIdx.x - p.chunk_blocks) * wpb + warp;
         it < p.n_items; it += step) {
      const Item item = p.items[it];
      const int32_t r0 = item.row, nr = item.tag;
      const int64_t rp = lane < nr ? __ldg(p.rowptr + r0 + lane + 1) : 0;
      int64_t start = item.e0;
      for (int l = 0; l < nr; ++l) {
        const int64_t end = __shfl_sync(0xffffffffu, rp, l);
        if (end > start) {
          grouped_row<TV, TB, VEC, G, U, LOCAL>(p, start, end, acc, g, sub);
          group_allreduce<TA, VEC, G>(acc);
          flush_row_grouped<TV, TB, VEC, G>(p, r0 + l, acc, lane);
        } else if (!p.accumulate) {
          flush_row_grouped<TV, TB, VEC, G>(p, r0 + l, acc, lane);
        }
        start = end;
      }
    }
  }
}

}  // namespace shiro
