// spmm_bulk.cuh -- the SpMM work loop with every gathered B row moved into shared memory by one
// TMA bulk copy (cp.async.bulk, completion counted in bytes on an mbarrier), two stages of BATCH
// rows per warp.
//
// Lane j of a warp issues the copy of the j-th row of a batch (the whole N * sz bytes, contiguous in
// the packed buffer), so a batch of 32 rows is one warp instruction and up to 2 * BATCH rows per
// warp are in flight without holding registers.  Lane 0 arms the stage's mbarrier with the batch's
// byte count before the copies are issued; the warp waits on the barrier's phase parity.  Every
// wait is bounded: if a phase does not complete within the limit the warp sets ST_TIMEOUT in the
// plan's status word, waits once more (bounded) for its copies, and stops.
#pragma once

#include "internal.cuh"
#include "vec.cuh"

namespace shiro {

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
      "r"(bytes)
      : "memory");
}

// True once the phase with the given parity has completed; false after the iteration limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < (1 << 20); ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "r"(1000u)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

template <typename TV, typename TB, int VEC, int NCH, int BATCH>
struct BulkLayout {
  static constexpr int ROW = 32 * VEC * NCH * (int)sizeof(TB);  // bytes of one row (N * sz)
  static constexpr int STAGE = BATCH * ROW;
  static constexpr int PAIRS = 32 * (int)sizeof(Pair<TV>);
  static constexpr int WARP = 2 * STAGE + 2 * PAIRS + 16;       // + two mbarriers
};

// Per-warp pipeline state: the two stage barriers and how many times each has been armed.
struct BulkState {
  uint32_t bar0;
  uint32_t uses[2];
  bool ok;
};

template <typename TV, typename TB, int VEC, int NCH, int BATCH, bool LOCAL>
__device__ __forceinline__ void spmm_span_bulk(const SpmmParams<TV, TB>& p, char* wsm,
                                               BulkState& bst, int64_t base, int total,
                                               int32_t r0, int nr, int rel, bool nonempty,
                                               typename AccOf<TB>::T (&acc)[NCH][VEC], int lane) {
  using TA = typename AccOf<TB>::T;
  using L = BulkLayout<TV, TB, VEC, NCH, BATCH>;
  static_assert(BATCH <= 32, "a batch is at most one row per lane");
  Pair<TV>* pairs = reinterpret_cast<Pair<TV>*>(wsm + 2 * L::STAGE);
  const uint32_t s_stage = (uint32_t)__cvta_generic_to_shared(wsm);
  const int nb = (total + BATCH - 1) / BATCH;
  int32_t nidx = 0;
  TV nval = 0;
  if (lane < BATCH && lane < total) {
    nidx = __ldcs(p.remap + base + lane);
    nval = __ldcs(p.val + base + lane);
  }
  auto issue = [&](int k) {
    const int s = k & 1;
    const int n = min(BATCH, total - k * BATCH);
    Pair<TV> pr;
    pr.idx = nidx;
    pr.val = nval;
    if (lane < BATCH) pairs[s * 32 + lane] = pr;
    const uint32_t bar = bst.bar0 + 8 * s;
    if (lane == 0) mbar_arrive_expect(bar, (uint32_t)(n * L::ROW));
    __syncwarp();
    if (lane < n) {
      const TB* row;
      if (LOCAL && nidx < 0)
        row = p.B + (uint64_t)(uint32_t)(-1 - nidx) * (uint32_t)p.ldb;
      else
        row = p.Bpack + (uint64_t)(uint32_t)nidx * (uint32_t)p.ldp;
      bulk_copy(s_stage + s * L::STAGE + lane * L::ROW, row, L::ROW, bar);
    }
    const int nxt = (k + 1) * BATCH + lane;
    if (lane < BATCH && nxt < total) {
      nidx = __ldcs(p.remap + base + nxt);
      nval = __ldcs(p.val + base + nxt);
    }
  };
  if (nb > 0) issue(0);
  for (int k = 0; k < nb && bst.ok; ++k) {
    if (k + 1 < nb) issue(k + 1);
    const int s = k & 1;
    const uint32_t parity = bst.uses[s] & 1u;
    bst.uses[s]++;
    if (!mbar_wait(bst.bar0 + 8 * s, parity)) {
      if (lane == 0) atomicOr(p.status, ST_TIMEOUT);
      if (k + 1 < nb) mbar_wait(bst.bar0 + 8 * ((k + 1) & 1), bst.uses[(k + 1) & 1] & 1u);
      bst.ok = false;
      break;
    }
    const int off = k * BATCH;
    const int n = min(BATCH, total - off);
    const int q = rel - 1 - off;
    const unsigned bit = (lane < nr && nonempty && q >= 0 && q < 32) ? (1u << q) : 0u;
    const unsigned endmask = __reduce_or_sync(0xffffffffu, bit);
    const TB* slot = reinterpret_cast<const TB*>(wsm + s * L::STAGE) + lane * VEC;
    const Pair<TV>* pk = pairs + s * 32;
#pragma unroll 4
    for (int j = 0; j < n; ++j) {
      const TA a = (TA)pk[j].val;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        TA b[VEC];
        load_vec<TB, VEC, false>(slot + j * (L::ROW / (int)sizeof(TB)) + c * 32 * VEC, b);
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
__global__ void __launch_bounds__(256) k_spmm_bulk(const SpmmParams<TV, TB> p) {
  extern __shared__ __align__(128) char smem[];
  using L = BulkLayout<TV, TB, VEC, NCH, BATCH>;
  using TA = typename AccOf<TB>::T;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  char* wsm = smem + warp * L::WARP;
  BulkState bst;
  bst.bar0 = (uint32_t)__cvta_generic_to_shared(wsm + 2 * L::STAGE + 2 * L::PAIRS);
  bst.uses[0] = bst.uses[1] = 0;
  bst.ok = true;
  if (lane == 0) {
    mbar_init(bst.bar0, 1);
    mbar_init(bst.bar0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  if ((int64_t)blockIdx.x < p.chunk_blocks) {
    const int64_t step = (int64_t)p.chunk_blocks * wpb;
    for (int64_t it = (int64_t)blockIdx.x * wpb + warp; it < p.n_chunk_items && bst.ok;
         it += step) {
      const Item item = p.items[it];
      const int32_t slot = -item.tag - 1;
      const int64_t row_end = __ldg(p.rowptr + item.row + 1);
      const int total = (int)min((int64_t)p.chunk, row_end - item.e0);
      TA acc[NCH][VEC];
#pragma unroll
      for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[c][v] = 0;
      spmm_span_bulk<TV, TB, VEC, NCH, BATCH, LOCAL>(p, wsm, bst, item.e0, total, item.row, 0, 0,
                                                     false, acc, lane);
      if (bst.ok) finish_chunk<TV, TB, VEC, NCH, false>(p, slot, acc, lane);
    }
  } else {
    const int64_t nb = (int64_t)gridDim.x - p.chunk_blocks;
    const int64_t step = p.persistent ? nb * wpb : p.n_items;
    for (int64_t it = p.n_chunk_items + ((int64_t)blockIdx.x - p.chunk_blocks) * wpb + warp;
         it < p.n_items && bst.ok; it += step) {
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
      spmm_span_bulk<TV, TB, VEC, NCH, BATCH, LOCAL>(p, wsm, bst, item.e0, total, r0, nr, rel,
                                                     nonempty, acc, lane);
    }
  }
}

}  // namespace shiro
