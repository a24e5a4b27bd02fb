// spmm_kernels.cuh -- local SpMM over the packed B rows with aggregation over the tiles of a row
// block (Sec. 2.2 stages 3-4, Sec. 5.1 stage 5): the kernels and their launchers.  Each storage
// type instantiates them in a translation unit of its own (spmm_f32.cu, spmm_bf16.cu,
// spmm_f64.cu) so that the three compile in parallel; spmm.cu holds the C entry points.
//
// Design (HBM-bound gather, not a dense contraction, so no tensor cores):
//   * one warp per work item; a dense row of B/C is spread over the 32 lanes in 4-16 byte
//     vectors, so every B-row gather is one fully coalesced 128-512 byte warp load;
//   * short rows are grouped into items and walked as one flat stream of nonzeros, so the
//     U gathers of a batch are in flight together even when rows hold 1-3 nonzeros; the group's
//     row pointers sit in lane registers (no dependent loads at row boundaries);
//   * rows longer than long_row_nnz (power-law hubs) are cut into chunks whose FP32 partial sums
//     go to scratch; the last chunk to arrive adds them in chunk order (deterministic, no float
//     atomics, bounded FP32 summation length) and writes the C row;
//   * all tiles of a row are summed in one pass in the row's stored order (ascending column
//     blocks for column-sorted rows), so C is written once with streaming stores.
#pragma once

#include <algorithm>
#include <cstring>

#include "internal.cuh"
#include "vec.cuh"

namespace shiro {

constexpr unsigned FULL_MASK = 0xffffffffu;

template <typename TV, typename TB>
struct SpmmParams {
  using TA = typename AccOf<TB>::T;
  const int64_t* rowptr;
  const int32_t* remap;
  const TV* val;
  const TB* Bpack;
  int64_t ldp;
  const TB* B;
  int64_t ldb;
  int32_t N;
  TA* C;
  int64_t ldc;
  const Item* items;
  int64_t n_items;
  TA* scratch;
  const int32_t* slot_lr;
  const LongRow* lr;
  int32_t* counters;
  int64_t n_chunk_items;
  int64_t chunk_blocks;
  int32_t chunk;
  int32_t accumulate;
  int32_t persistent;
  int* status;
  int32_t pf_bytes;  // bytes of a row to prefetch into L2 ahead of its gather (0: off)
  int32_t* work;     // item counter of the dynamically scheduled kernel (zeroed before launch)
};

// (index, value) of one nonzero as staged in shared memory; two FP32 entries fill 16 bytes.
template <typename TV> struct Pair { int32_t idx; float val; };
template <> struct Pair<double> { int32_t idx; int32_t pad; double val; };

template <typename TV, typename TB, int VEC, int NCH, bool MASKED>
__device__ __forceinline__ void gather_row(const SpmmParams<TV, TB>& p, const TB* row,
                                           typename AccOf<TB>::T (&b)[NCH][VEC], int lane) {
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int col = c * 32 * VEC + lane * VEC;
    if (!MASKED || col < p.N) {
      load_vec<TB, VEC, true>(row + c * 32 * VEC, b[c]);
    } else {
#pragma unroll
      for (int v = 0; v < VEC; ++v) b[c][v] = 0;
    }
  }
}

template <typename TV, typename TB, int VEC, int NCH, bool MASKED>
__device__ __forceinline__ void gather_raw(
    const SpmmParams<TV, TB>& p, const TB* row,
    typename RawFrag<TB, VEC>::T (&b)[NCH][RawFrag<TB, VEC>::W], int lane) {
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int col = c * 32 * VEC + lane * VEC;
    if (!MASKED || col < p.N) {
      load_raw<TB, VEC>(row + c * 32 * VEC, b[c]);
    } else {
#pragma unroll
      for (int w = 0; w < RawFrag<TB, VEC>::W; ++w) b[c][w] = 0;
    }
  }
}

template <typename TV, typename TB, int VEC, int NCH, bool MASKED>
__device__ __forceinline__ void flush_row(const SpmmParams<TV, TB>& p, int32_t r,
                                          typename AccOf<TB>::T (&acc)[NCH][VEC], int lane) {
  using TA = typename AccOf<TB>::T;
  TA* c = p.C + (int64_t)r * p.ldc;
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
    const int col = ch * 32 * VEC + lane * VEC;
    if (!MASKED || col < p.N) {
      if (p.accumulate) {
        TA old[VEC];
        load_acc_cg<TA, VEC>(c + col, old);
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[ch][v] += old[v];
      }
      store_vec<TA, VEC, true>(c + col, acc[ch]);
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[ch][v] = 0;
  }
}

// Lane-local view of the dense operands: row r of the packed buffer starts at bp + r * ldp
// (32-bit index times 32-bit stride, one wide multiply-add per gather).
template <typename TB>
struct Bases {
  const TB* bp;
  const TB* b;
  uint32_t ldp, ldb;
};

template <typename TV, typename TB, int VEC, int NCH, bool MASKED, int U, bool LOCAL, bool FULL,
          bool ENDS = true>
__device__ __forceinline__ void spmm_batch(const SpmmParams<TV, TB>& p, const Bases<TB>& bs,
                                           const Pair<TV>* sp, int n, int off, int32_t r0, int nr,
                                           int rel, unsigned endmask,
                                           typename AccOf<TB>::T (&acc)[NCH][VEC], int lane,
                                           int32_t nidx = 0, int nnext = 0) {
  using TA = typename AccOf<TB>::T;
  // A full batch walks all 32 staged pairs in steps of U without bounds checks.
  static_assert(32 % U == 0, "U must divide the 32-pair batch");
#pragma unroll 1
  for (int j = 0; j < (FULL ? 32 : n); j += U) {
    typename RawFrag<TB, VEC>::T b[U][NCH][RawFrag<TB, VEC>::W];
    TV a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (FULL || j + u < n) {
        const Pair<TV> pr = sp[j + u];
        a[u] = (TV)pr.val;
        const TB* row;
        if (LOCAL && pr.idx < 0)
          row = bs.b + (uint64_t)(uint32_t)(-1 - pr.idx) * bs.ldb;
        else
          row = bs.bp + (uint64_t)(uint32_t)pr.idx * bs.ldp;
        gather_raw<TV, TB, VEC, NCH, MASKED>(p, row, b[u], lane);
      }
    }
#ifndef SHIRO_SPMM_PF
#define SHIRO_SPMM_PF 2
#endif
    // Kernels that keep only U <= 2 rows of 512 bytes or more in flight per warp (FP32 N >= 256,
    // BF16 N = 256): bring the rows of the step SHIRO_SPMM_PF steps ahead into L2 while this
    // step's gathers are in flight (more requests outstanding to HBM without registers).  With
    // U = 4 the prefetch code costs more issue slots than the misses it hides (measured).
    constexpr bool PF = VEC * NCH * sizeof(TB) >= 16 && U <= 2;
    // BF16 rows (raw words in flight leave registers free) also prefetch across the batch end,
    // from the next batch's indices (one per lane in nidx); FP32 rows would spill for it.
    constexpr bool XB = PF && std::is_same<TB, __nv_bfloat16>::value;
    if (PF && FULL && p.pf_bytes) {
      const int k = j + SHIRO_SPMM_PF * U;
      if (k < 32) {
        // Every lane forms an address; lanes 0 .. U-1 issue (predicated, no branch).
        const int32_t ix = sp[k + (lane & (U - 1))].idx;
        const TB* r = (LOCAL && ix < 0) ? p.B + (uint64_t)(uint32_t)(-1 - ix) * (uint64_t)p.ldb
                                        : p.Bpack + (uint64_t)(uint32_t)ix * (uint64_t)p.ldp;
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.lt.u32 q, %2, %3;\n\t"
            "@q cp.async.bulk.prefetch.L2.global [%0], %1;\n\t}"
            ::"l"(r), "r"(p.pf_bytes), "r"(lane), "r"(U));
      } else if (XB) {
        const int32_t ix = __shfl_sync(FULL_MASK, nidx, (k - 32) + (lane & (U - 1)));
        if (lane < U && (k - 32) + lane < nnext) {
          const TB* r = (LOCAL && ix < 0) ? p.B + (uint64_t)(uint32_t)(-1 - ix) * (uint64_t)p.ldb
                                          : p.Bpack + (uint64_t)(uint32_t)ix * (uint64_t)p.ldp;
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(r), "r"(p.pf_bytes));
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (FULL || j + u < n) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) fma_raw<TB, VEC>(a[u], b[u][c], acc[c]);
        if (ENDS && ((endmask >> (j + u)) & 1u)) {
          // The nonzero at off + j + u ends a non-empty row: the first lane whose row end is here.
          const unsigned who = __ballot_sync(FULL_MASK, lane < nr && rel == off + j + u + 1);
          flush_row<TV, TB, VEC, NCH, MASKED>(p, r0 + __ffs(who) - 1, acc, lane);
        }
      }
    }
  }
}

// Accumulates nonzeros [base, base + total) of rows r0 .. r0 + nr - 1.  Lane l < nr holds the
// end of row r0 + l relative to base in `rel` and whether that row is non-empty; the end of every
// non-empty row is flushed to C as the stream passes it (chunks of long rows pass nr = 0 and
// flush nothing).  The (index, value) pairs of each batch of 32 go through shared memory and the
// next batch's pairs are loaded while the current batch's gathers are in flight.
template <typename TV, typename TB, int VEC, int NCH, bool MASKED, int U, bool LOCAL>
__device__ __forceinline__ void spmm_span(const SpmmParams<TV, TB>& p, const Bases<TB>& bs,
                                          Pair<TV>* sp, int64_t base, int total, int32_t r0,
                                          int nr, int rel, bool nonempty,
                                          typename AccOf<TB>::T (&acc)[NCH][VEC], int lane) {
  int32_t nidx = 0;
  TV nval = 0;
  if (lane < total) {
    nidx = __ldcs(p.remap + base + lane);
    nval = __ldcs(p.val + base + lane);
  }
  for (int off = 0; off < total; off += 32) {
    const int n = min(32, total - off);
    __syncwarp();
    Pair<TV> pr;
    pr.idx = nidx;
    pr.val = nval;
    sp[lane] = pr;
    __syncwarp();
    if (off + 32 + lane < total) {
      nidx = __ldcs(p.remap + base + off + 32 + lane);
      nval = __ldcs(p.val + base + off + 32 + lane);
    }
    const int q = rel - 1 - off;
    const unsigned bit = (lane < nr && nonempty && q >= 0 && q < 32) ? (1u << q) : 0u;
    const unsigned endmask = __reduce_or_sync(FULL_MASK, bit);
    // Full batches with no row end inside (all chunk batches, most batches of long rows) take a
    // copy of the loop without the flush test: fewer instructions between dependent gathers.
    if (n == 32 && endmask == 0)
      spmm_batch<TV, TB, VEC, NCH, MASKED, U, LOCAL, true, false>(p, bs, sp, n, off, r0, nr, rel,
                                                                  endmask, acc, lane, nidx,
                                                                  total - off - 32);
    else if (n == 32)
      spmm_batch<TV, TB, VEC, NCH, MASKED, U, LOCAL, true>(p, bs, sp, n, off, r0, nr, rel, endmask,
                                                           acc, lane, nidx, total - off - 32);
    else
      spmm_batch<TV, TB, VEC, NCH, MASKED, U, LOCAL, false>(p, bs, sp, n, off, r0, nr, rel,
                                                            endmask, acc, lane);
  }
}

template <typename TV, typename TB, int VEC, int NCH, bool MASKED, int U, bool LOCAL>
__device__ __forceinline__ void run_group(const SpmmParams<TV, TB>& p, const Bases<TB>& bs,
                                          Pair<TV>* sp, const Item& item, int lane) {
  using TA = typename AccOf<TB>::T;
  const int32_t r0 = item.row, nr = item.tag;
  const int64_t rp = lane < nr ? __ldg(p.rowptr + r0 + lane + 1) : 0;
  const int rel = (int)(rp - item.e0);
  const int prev = __shfl_up_sync(FULL_MASK, rel, 1);
  const bool nonempty = lane < nr && rel > (lane ? prev : 0);
  const int total = __shfl_sync(FULL_MASK, rel, nr - 1);
  TA acc[NCH][VEC];
#pragma unroll
  for (int c = 0; c < NCH; ++c)
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[c][v] = 0;
  // Empty rows get zeros up front (C += 0 leaves them unchanged when accumulating).
  if (!p.accumulate) {
    unsigned empty = __ballot_sync(FULL_MASK, lane < nr && !nonempty);
    while (empty) {
      const int l = __ffs(empty) - 1;
      empty &= empty - 1;
      flush_row<TV, TB, VEC, NCH, MASKED>(p, r0 + l, acc, lane);
    }
  }
  spmm_span<TV, TB, VEC, NCH, MASKED, U, LOCAL>(p, bs, sp, item.e0, total, r0, nr, rel, nonempty,
                                                acc, lane);
}

// Partial sum of one chunk of a long row, then its arrival count; the last chunk to arrive adds
// the row's partials in chunk order and writes the C row.
template <typename TV, typename TB, int VEC, int NCH, bool MASKED>
__device__ __forceinline__ void finish_chunk(const SpmmParams<TV, TB>& p, int32_t slot,
                                             typename AccOf<TB>::T (&acc)[NCH][VEC], int lane) {
  using TA = typename AccOf<TB>::T;
  TA* part = p.scratch + (int64_t)slot * p.N;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int col = c * 32 * VEC + lane * VEC;
    if (!MASKED || col < p.N) store_acc_cg<TA, VEC>(part + col, acc[c]);
  }
  // Release: every lane's partial is visible device-wide (fence), and the warp barrier orders
  // all lanes' stores and fences before lane 0's arrival count.
  __threadfence();
  __syncwarp();
  const int32_t lr = __ldg(p.slot_lr + slot);
  const LongRow L = p.lr[lr];
  int old = 0;
  if (lane == 0) {
    __threadfence();  // cumulative release of the partials the barrier ordered before lane 0
    old = atomicAdd(p.counters + lr, 1);
    __threadfence();  // acquire side of the last arrival: the other chunks' partials
  }
  __syncwarp();       // orders lane 0's observation before every lane's loads below
  old = __shfl_sync(FULL_MASK, old, 0);
  if (old == L.nchunks - 1) {
    __threadfence();
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[c][v] = 0;
    for (int32_t s = 0; s < L.nchunks; ++s) {
      const TA* q = p.scratch + (int64_t)(L.slot0 + s) * p.N;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int col = c * 32 * VEC + lane * VEC;
        if (!MASKED || col < p.N) {
          TA t[VEC];
          load_acc_cg<TA, VEC>(q + col, t);
#pragma unroll
          for (int v = 0; v < VEC; ++v) acc[c][v] += t[v];
        }
      }
    }
    flush_row<TV, TB, VEC, NCH, MASKED>(p, L.row, acc, lane);
    if (lane == 0) p.counters[lr] = 0;
  } else if (old >= L.nchunks) {
    if (lane == 0) atomicOr(p.status, ST_COUNTER);
  }
}

template <typename TV, typename TB, int VEC, int NCH, bool MASKED, int U, bool LOCAL>
__device__ __forceinline__ void run_chunk(const SpmmParams<TV, TB>& p, const Bases<TB>& bs,
                                          Pair<TV>* sp, const Item& item, int lane) {
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
  spmm_span<TV, TB, VEC, NCH, MASKED, U, LOCAL>(p, bs, sp, item.e0, total, i, 0, 0, false, acc,
                                                lane);
  finish_chunk<TV, TB, VEC, NCH, MASKED>(p, slot, acc, lane);
}

}  // namespace shiro

#include "spmm_async.cuh"
#include "spmm_bulk.cuh"
#include "spmm_grouped.cuh"
#include "spmm_ring.cuh"
#include "spmm_lean.cuh"
#include "spmm_gather4.cuh"
#include "spmm_bwd.cuh"

namespace shiro {

template <int VEC, int NCH, typename TB>
struct Occupancy {
  // Registers per lane held by one gathered row fragment in flight (raw storage words).
  static constexpr int REG =
      RawFrag<TB, VEC>::W * NCH * (int)((sizeof(typename RawFrag<TB, VEC>::T) + 3) / 4);
#ifndef SHIRO_SPMM_U
#define SHIRO_SPMM_U 4
#endif
#ifndef SHIRO_SPMM_U8
#define SHIRO_SPMM_U8 2
#endif
#ifndef SHIRO_SPMM_UW
#define SHIRO_SPMM_UW 2
#endif
  // Accumulators wider than one 4-register fragment (BF16 rows of 256 elements).
  static constexpr bool WIDE_ACC = VEC * NCH * (int)(sizeof(typename AccOf<TB>::T) / 4) > 4;
  static constexpr int U =
      REG >= 16 ? 2 : (REG >= 8 ? SHIRO_SPMM_U8 : (WIDE_ACC ? SHIRO_SPMM_UW : SHIRO_SPMM_U));
  // 64 registers for 4-register fragments (32 warps per SM): measured faster than 80 registers
  // without spills (24 warps), though ptxas spills a few bytes of the long-row epilogue.
#ifndef SHIRO_SPMM_MIN_BLOCKS
#define SHIRO_SPMM_MIN_BLOCKS 4
#endif
#ifndef SHIRO_SPMM_MIN_BLOCKS8
#define SHIRO_SPMM_MIN_BLOCKS8 4
#endif
  static constexpr int MIN_BLOCKS =
      REG <= 4 ? SHIRO_SPMM_MIN_BLOCKS : (REG <= 8 ? SHIRO_SPMM_MIN_BLOCKS8 : 2);
};

// Blocks [0, chunk_blocks) run the chunks of long rows, the others the row groups (the two
// paths share no loop, so each gets its own register allocation).  Items hold the chunks first.
template <typename TV, typename TB, int VEC, int NCH, bool MASKED, int U, bool LOCAL>
__global__ void __launch_bounds__(256, (Occupancy<VEC, NCH, TB>::MIN_BLOCKS))
    k_spmm(const SpmmParams<TV, TB> p) {
  __shared__ Pair<TV> s_pairs[8][32];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  Bases<TB> bs;
  bs.bp = p.Bpack + lane * VEC;
  bs.b = p.B + lane * VEC;
  bs.ldp = (uint32_t)p.ldp;
  bs.ldb = (uint32_t)p.ldb;
  Pair<TV>* sp = s_pairs[warp];
  if ((int64_t)blockIdx.x < p.chunk_blocks) {
    const int64_t step = (int64_t)p.chunk_blocks * wpb;
    for (int64_t it = (int64_t)blockIdx.x * wpb + warp; it < p.n_chunk_items; it += step) {
      const Item item = p.items[it];
      run_chunk<TV, TB, VEC, NCH, MASKED, U, LOCAL>(p, bs, sp, item, lane);
    }
  } else {
    const int64_t nb = (int64_t)gridDim.x - p.chunk_blocks;
    const int64_t step = p.persistent ? nb * wpb : p.n_items;
    for (int64_t it = p.n_chunk_items + ((int64_t)blockIdx.x - p.chunk_blocks) * wpb + warp;
         it < p.n_items; it += step) {
      const Item item = p.items[it];
      run_group<TV, TB, VEC, NCH, MASKED, U, LOCAL>(p, bs, sp, item, lane);
    }
  }
}

// ---- dispatch ----

struct Variant {
  int vec, nch, masked;
};

static bool aligned(const void* ptr, int64_t ld, size_t elem, int vec) {
  const size_t a = std::min<size_t>(16, elem * (size_t)vec);
  return ((uintptr_t)ptr % a) == 0 && ((size_t)ld * elem) % a == 0;
}

// Vector width and chunk count for N columns of storage dtype dt; all operands must honour the
// alignment of the chosen vector width.
static Variant pick_variant(shiro_dtype dt, int32_t N, bool ok16, bool ok8, bool ok4) {
  if (dt == SHIRO_F32) {
    if (ok16 && N % 128 == 0 && (N / 128 == 1 || N / 128 == 2 || N / 128 == 4)) return {4, N / 128, 0};
    if (ok8 && N == 64) return {2, 1, 0};
    if (N == 32) return {1, 1, 0};
  } else if (dt == SHIRO_BF16) {
    if (ok16 && N % 256 == 0 && (N / 256 == 1 || N / 256 == 2)) return {8, N / 256, 0};
    if (ok8 && N == 128) return {4, 1, 0};
    if (ok4 && N == 64) return {2, 1, 0};
    if (N == 32) return {1, 1, 0};
  } else {
    if (ok16 && N % 64 == 0 && (N / 64 == 1 || N / 64 == 2 || N / 64 == 4)) return {2, N / 64, 0};
    if (N == 32) return {1, 1, 0};
  }
  if (N <= 32) return {1, 1, 1};
  if (N <= 128) return {1, 4, 1};
  if (N <= 512) return {1, 16, 1};
  return {0, 0, 0};
}

template <typename TV, typename TB, int VEC, int NCH, int BATCH>
static shiro_status launch_async_batch(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                                       cudaStream_t s) {
  using L = AsyncLayout<TV, TB, VEC, NCH, BATCH>;
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  auto kern = local ? k_spmm_async<TV, TB, VEC, NCH, BATCH, true>
                    : k_spmm_async<TV, TB, VEC, NCH, BATCH, false>;
  const int max_smem = 227 * 1024;
  const int wpc = std::max(1, std::min(P->opts.warps_per_cta, max_smem / L::WARP));
  const int smem = wpc * L::WARP;
  SHIRO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  SpmmParams<TV, TB> q = prm;
  q.n_chunk_items = P->n_slots;
  q.chunk_blocks = (q.n_chunk_items + wpc - 1) / wpc;
  const int64_t n_groups = prm.n_items - q.n_chunk_items;
  int64_t gblocks = (n_groups + wpc - 1) / wpc;
  if (prm.persistent) {
    int per_sm = 0;
    SHIRO_CUDA(blocks_per_sm(&per_sm, kern, wpc * 32, smem));
    gblocks = std::min<int64_t>(gblocks, (int64_t)std::max(per_sm, 1) * P->sm_count);
  }
  const int64_t grid = q.chunk_blocks + gblocks;
  if (grid <= 0) return SHIRO_OK;
  if (grid > INT32_MAX) SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "too many work items");
  kern<<<(unsigned)grid, wpc * 32, smem, s>>>(q);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

template <typename TV, typename TB, int VEC, int NCH>
static shiro_status launch_async(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                                 cudaStream_t s) {
  constexpr int ROW = 32 * VEC * NCH * (int)sizeof(TB);
  int batch = P->opts.stage_rows ? P->opts.stage_rows : 32;
  while (batch > 8 && batch * ROW > 16384) batch /= 2;
  if (batch >= 32 && 32 * ROW <= 16384) return launch_async_batch<TV, TB, VEC, NCH, 32>(P, prm, s);
  if (batch >= 16 && 16 * ROW <= 16384) return launch_async_batch<TV, TB, VEC, NCH, 16>(P, prm, s);
  return launch_async_batch<TV, TB, VEC, NCH, 8>(P, prm, s);
}

template <typename TV, typename TB, int VEC, int NCH, int BATCH>
static shiro_status launch_bulk_batch(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                                      cudaStream_t s) {
  using L = BulkLayout<TV, TB, VEC, NCH, BATCH>;
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  auto kern = local ? k_spmm_bulk<TV, TB, VEC, NCH, BATCH, true>
                    : k_spmm_bulk<TV, TB, VEC, NCH, BATCH, false>;
  const int max_smem = 227 * 1024;
  const int wpc = std::max(1, std::min(P->opts.warps_per_cta, max_smem / L::WARP));
  const int smem = wpc * L::WARP;
  SHIRO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  SpmmParams<TV, TB> q = prm;
  q.n_chunk_items = P->n_slots;
  q.chunk_blocks = (q.n_chunk_items + wpc - 1) / wpc;
  const int64_t n_groups = prm.n_items - q.n_chunk_items;
  int64_t gblocks = (n_groups + wpc - 1) / wpc;
  if (prm.persistent) {
    int per_sm = 0;
    SHIRO_CUDA(blocks_per_sm(&per_sm, kern, wpc * 32, smem));
    gblocks = std::min<int64_t>(gblocks, (int64_t)std::max(per_sm, 1) * P->sm_count);
  }
  const int64_t grid = q.chunk_blocks + gblocks;
  if (grid <= 0) return SHIRO_OK;
  if (grid > INT32_MAX) SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "too many work items");
  kern<<<(unsigned)grid, wpc * 32, smem, s>>>(q);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

template <typename TV, typename TB, int G>
static shiro_status launch_grouped(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                                   cudaStream_t s) {
  constexpr int VEC = 16 / (int)sizeof(TB);
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  auto kern = local ? k_spmm_grouped<TV, TB, VEC, G, 4, true>
                    : k_spmm_grouped<TV, TB, VEC, G, 4, false>;
  const int wpc = P->opts.warps_per_cta;
  SpmmParams<TV, TB> q = prm;
  q.n_chunk_items = P->n_slots;
  q.chunk_blocks = (q.n_chunk_items + wpc - 1) / wpc;
  const int64_t n_groups = prm.n_items - q.n_chunk_items;
  int64_t gblocks = (n_groups + wpc - 1) / wpc;
  if (prm.persistent) {
    int per_sm = 0;
    SHIRO_CUDA(blocks_per_sm(&per_sm, kern, wpc * 32, 0));
    gblocks = std::min<int64_t>(gblocks, (int64_t)std::max(per_sm, 1) * P->sm_count);
  }
  const int64_t grid = q.chunk_blocks + gblocks;
  if (grid <= 0) return SHIRO_OK;
  if (grid > INT32_MAX) SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "too many work items");
  kern<<<(unsigned)grid, wpc * 32, 0, s>>>(q);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

// TMA bulk copies need 16-byte aligned rows whose size is a multiple of 16 bytes.
template <typename TV, typename TB, int VEC, int NCH>
static bool bulk_ok(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm) {
  constexpr int ROW = 32 * VEC * NCH * (int)sizeof(TB);
  if (ROW % 16 || ROW > 4096) return false;
  auto al = [](const void* b, int64_t ld) {
    return ((uintptr_t)b % 16) == 0 && ((uint64_t)ld * sizeof(TB)) % 16 == 0;
  };
  if (!al(prm.Bpack, prm.ldp)) return false;
  if ((P->flags & SHIRO_PLAN_LOCAL_DIAG) && !al(prm.B, prm.ldb)) return false;
  return true;
}

template <typename TV, typename TB, int VEC, int NCH>
static shiro_status launch_bulk(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                                cudaStream_t s) {
  constexpr int ROW = 32 * VEC * NCH * (int)sizeof(TB);
  int batch = P->opts.stage_rows ? P->opts.stage_rows : 32;
  while (batch > 8 && batch * ROW > 16384) batch /= 2;
  if constexpr (32 * ROW <= 16384)
    if (batch >= 32) return launch_bulk_batch<TV, TB, VEC, NCH, 32>(P, prm, s);
  if constexpr (16 * ROW <= 16384)
    if (batch >= 16) return launch_bulk_batch<TV, TB, VEC, NCH, 16>(P, prm, s);
  return launch_bulk_batch<TV, TB, VEC, NCH, 8>(P, prm, s);
}

template <typename TV, typename TB, int VEC, int NCH, int R, int G>
static shiro_status launch_lring_rg(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                                    cudaStream_t s) {
  using L = LRingLayout<TV, TB, VEC, NCH, R, G>;
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  auto kern = local ? k_spmm_lring<TV, TB, VEC, NCH, R, G, true>
                    : k_spmm_lring<TV, TB, VEC, NCH, R, G, false>;
  const int max_smem = 227 * 1024;
  const int wpc = std::max(1, std::min(P->opts.warps_per_cta, max_smem / L::WARP));
  const int smem = wpc * L::WARP;
  SHIRO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  SpmmParams<TV, TB> q = prm;
  q.n_chunk_items = P->n_slots;
  q.chunk_blocks = (q.n_chunk_items + wpc - 1) / wpc;
  const int64_t n_groups = prm.n_items - q.n_chunk_items;
  int64_t gblocks = (n_groups + wpc - 1) / wpc;
  if (prm.persistent) {
    int per_sm = 0;
    SHIRO_CUDA(blocks_per_sm(&per_sm, kern, wpc * 32, smem));
    gblocks = std::min<int64_t>(gblocks, (int64_t)std::max(per_sm, 1) * P->sm_count);
  }
  const int64_t grid = q.chunk_blocks + gblocks;
  if (grid <= 0) return SHIRO_OK;
  if (grid > INT32_MAX) SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "too many work items");
  kern<<<(unsigned)grid, wpc * 32, smem, s>>>(q);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

// Ring depths compiled per row size: 256-byte rows keep 16 or 32 rows (default 16),
// 512-byte rows 8, 12 or 16 (default 8), rows of 1-2 KB 4 or 8 in groups of 2 (default 4).
template <typename TV, typename TB, int VEC, int NCH>
static shiro_status launch_lring(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                                 cudaStream_t s) {
  constexpr int ROW = 32 * VEC * NCH * (int)sizeof(TB);
  const int want = P->opts.stage_rows;
  if constexpr (ROW == 256) {
    if (want == 32) return launch_lring_rg<TV, TB, VEC, NCH, 32, 4>(P, prm, s);
    return launch_lring_rg<TV, TB, VEC, NCH, 16, 4>(P, prm, s);
  } else if constexpr (ROW == 512) {
    if (want == 12) return launch_lring_rg<TV, TB, VEC, NCH, 12, 4>(P, prm, s);
    if (want == 16) return launch_lring_rg<TV, TB, VEC, NCH, 16, 4>(P, prm, s);
    return launch_lring_rg<TV, TB, VEC, NCH, 8, 4>(P, prm, s);
  } else {
    if (want == 8) return launch_lring_rg<TV, TB, VEC, NCH, 8, 2>(P, prm, s);
    return launch_lring_rg<TV, TB, VEC, NCH, 4, 2>(P, prm, s);
  }
}

template <typename TV, typename TB, int VEC, int NCH>
static shiro_status launch_lean(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                                cudaStream_t s) {
  constexpr int U = LeanShape<TB, VEC>::WIDE ? SHIRO_LEAN_UW : Occupancy<VEC, NCH, TB>::U;
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  auto kern = local ? k_spmm_lean<TV, TB, VEC, NCH, U, true>
                    : k_spmm_lean<TV, TB, VEC, NCH, U, false>;
  // Persistent form: explicitly requested, or chosen per row shape by the automatic pipeline.
  const bool dyn = prm.persistent || (P->opts.pipeline == 0 && LeanShape<TB, VEC>::DYN);
  if (dyn)
    kern = local ? k_spmm_lean_dyn<TV, TB, VEC, NCH, U, true>
                 : k_spmm_lean_dyn<TV, TB, VEC, NCH, U, false>;
  SpmmParams<TV, TB> q = prm;
  q.n_chunk_items = P->n_slots;
  q.chunk_blocks = (q.n_chunk_items + 1) / 2;
  int64_t grid = q.chunk_blocks + (prm.n_items - q.n_chunk_items + 1) / 2;
  if (grid <= 0) return SHIRO_OK;
  if (dyn) {
    // Persistent: SMs x resident CTAs, every warp takes the next item from a counter.
    if (prm.n_items > INT32_MAX) SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "too many work items");
    int per_sm = 0;
    SHIRO_CUDA(blocks_per_sm(&per_sm, kern, 64, 0));
    grid = std::min<int64_t>(grid, (int64_t)std::max(per_sm, 1) * P->sm_count);
    q.work = P->d_status + 2;
    SHIRO_CUDA(cudaMemsetAsync(q.work, 0, sizeof(int32_t), s));
  }
  if (grid > INT32_MAX) SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "too many work items");
  kern<<<(unsigned)grid, 64, 0, s>>>(q);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

// Rows of 512 bytes gathered by TMA gather4 into shared memory (pipeline 7): not LOCAL_DIAG
// (every row comes from the packed buffer), the buffer 16-byte aligned with a row stride of a
// multiple of 16 bytes, at least one packed row.
template <typename TV, typename TB, int VEC>
static bool g4_ok(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm) {
  return !(P->flags & SHIRO_PLAN_LOCAL_DIAG) && P->packed_rows > 0 &&
         (int64_t)prm.N * (int64_t)sizeof(TB) == 512 && ((uintptr_t)prm.Bpack % 16) == 0 &&
         ((uint64_t)prm.ldp * sizeof(TB)) % 16 == 0 && tensor_map_encoder() != nullptr;
}

template <typename TV, typename TB, int VEC>
static shiro_status launch_g4(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                              cudaStream_t s) {
  constexpr int D = G4Shape<TB>::D, W = G4Shape<TB>::W;
  using L = G4Layout<TV, D>;
  auto kern = k_spmm_g4<TV, TB, VEC, D, W>;
  if (prm.n_items <= 0) return SHIRO_OK;
  if (prm.n_items > INT32_MAX) SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "too many work items");
  // The packed buffer as R rows of 128 32-bit words, one row per box.
  CUtensorMap tm;
  const cuuint64_t gdim[2] = {128, (cuuint64_t)P->packed_rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)prm.ldp * sizeof(TB)};
  const cuuint32_t box[2] = {128, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = tensor_map_encoder()(
      &tm, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<TB*>(prm.Bpack), gdim, gstride, box,
      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) SHIRO_FAIL(SHIRO_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  const int smem = W * L::WARP;
  SHIRO_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  SHIRO_CUDA(blocks_per_sm(&per_sm, kern, W * 32, (size_t)smem));
  const int64_t grid = std::min<int64_t>((prm.n_items + W - 1) / W,
                                         (int64_t)std::max(per_sm, 1) * P->sm_count);
  SpmmParams<TV, TB> q = prm;
  q.n_chunk_items = P->n_slots;
  q.work = P->d_status + 2;
  SHIRO_CUDA(cudaMemsetAsync(q.work, 0, sizeof(int32_t), s));
  kern<<<(unsigned)grid, W * 32, smem, s>>>(q, tm);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

template <typename TV, typename TB, int VEC, int NCH, bool MASKED>
static shiro_status launch_one(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                               cudaStream_t s) {
  if constexpr (!MASKED && VEC * sizeof(TB) >= 4) {
    constexpr int ROW = 32 * VEC * NCH * (int)sizeof(TB);
    // Per-lane copy ring (pipeline 4) for FP32 / BF16 rows of 256 bytes to 2 KB; with pipeline 0
    // (automatic) rows of 1 KB or more take it (measured faster than register gathers there,
    // slower below).  Pipeline 5 forces register gathers.
    if constexpr (!std::is_same<TB, double>::value && ROW >= 256 && ROW <= 2048 &&
                  (ROW & (ROW - 1)) == 0) {
      if (P->opts.pipeline == 4 || (P->opts.pipeline == 0 && ROW >= 1024))
        return launch_lring<TV, TB, VEC, NCH>(P, prm, s);
    }
    // TMA gather4 ring (pipeline 7), and with pipeline 0 for BF16 rows of 512 bytes outside
    // persistent mode (measured faster there: R-MAT 2^20 0.824 -> 0.771 ms, R-MAT 2^22 avg degree
    // 32 6.00 -> 5.75 ms; FP32 rows of 512 bytes stay on the 48-register gathers, 0.552 against
    // 0.656).
    if constexpr (!std::is_same<TB, double>::value && NCH == 1 && ROW == 512) {
      const bool automatic = std::is_same<TB, __nv_bfloat16>::value && P->opts.pipeline == 0 &&
                             !P->opts.persistent;
      if ((P->opts.pipeline == 7 || automatic) && g4_ok<TV, TB, VEC>(P, prm))
        return launch_g4<TV, TB, VEC>(P, prm, s);
    }
    // Lean register gathers (pipeline 6; 48 registers, 2-warp CTAs; persistent mode takes items
    // from a counter): with pipeline 0 (automatic) rows of 128 to 512 bytes take them outside
    // persistent mode (measured faster there), in the counter form for most row shapes.
    if constexpr (!std::is_same<TB, double>::value && NCH == 1 && ROW >= 128 && ROW <= 512) {
      if (P->opts.pipeline == 6 || (P->opts.pipeline == 0 && !P->opts.persistent))
        return launch_lean<TV, TB, VEC, NCH>(P, prm, s);
    }
    if (P->opts.pipeline == 2 && bulk_ok<TV, TB, VEC, NCH>(P, prm))
      return launch_bulk<TV, TB, VEC, NCH>(P, prm, s);
    if (P->opts.pipeline == 1 || P->opts.pipeline == 2)
      return launch_async<TV, TB, VEC, NCH>(P, prm, s);
  }
  constexpr int U = Occupancy<VEC, NCH, TB>::U;
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  auto kern = local ? k_spmm<TV, TB, VEC, NCH, MASKED, U, true>
                    : k_spmm<TV, TB, VEC, NCH, MASKED, U, false>;
  const int wpc = P->opts.warps_per_cta;
  const int threads = wpc * 32;
  SpmmParams<TV, TB> q = prm;
  q.n_chunk_items = P->n_slots;
  q.chunk_blocks = (q.n_chunk_items + wpc - 1) / wpc;
  const int64_t n_groups = prm.n_items - q.n_chunk_items;
  int64_t gblocks = (n_groups + wpc - 1) / wpc;
  if (prm.persistent) {
    int per_sm = 0;
    SHIRO_CUDA(blocks_per_sm(&per_sm, kern, threads, 0));
    gblocks = std::min<int64_t>(gblocks, (int64_t)std::max(per_sm, 1) * P->sm_count);
  }
  const int64_t grid = q.chunk_blocks + gblocks;
  if (grid <= 0) return SHIRO_OK;
  if (grid > INT32_MAX) SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "too many work items");
  kern<<<(unsigned)grid, threads, 0, s>>>(q);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

template <typename TV, typename TB>
static shiro_status dispatch(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm, Variant v,
                             cudaStream_t s) {
#define SHIRO_CASE(VEC, NCH, MASKED)                                        \
  if (v.vec == VEC && v.nch == NCH && v.masked == MASKED)                   \
    return launch_one<TV, TB, VEC, NCH, MASKED>(P, prm, s);
  if constexpr (std::is_same<TB, float>::value) {
    SHIRO_CASE(4, 1, 0) SHIRO_CASE(4, 2, 0) SHIRO_CASE(4, 4, 0) SHIRO_CASE(2, 1, 0)
    SHIRO_CASE(1, 1, 0)
  } else if constexpr (std::is_same<TB, double>::value) {
    SHIRO_CASE(2, 1, 0) SHIRO_CASE(2, 2, 0) SHIRO_CASE(2, 4, 0) SHIRO_CASE(1, 1, 0)
  } else {
    SHIRO_CASE(8, 1, 0) SHIRO_CASE(8, 2, 0) SHIRO_CASE(4, 1, 0) SHIRO_CASE(2, 1, 0)
    SHIRO_CASE(1, 1, 0)
  }
  SHIRO_CASE(1, 1, 1) SHIRO_CASE(1, 4, 1) SHIRO_CASE(1, 16, 1)
#undef SHIRO_CASE
  SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "no SpMM variant for N=%d", prm.N);
}

template <typename TV, typename TB>
static SpmmParams<TV, TB> make_params(const shiro_plan_s* P, const void* Bpack, int64_t ldp,
                                      const void* B, int64_t ldb, int32_t N, shiro_dtype dt,
                                      void* C, int64_t ldc, uint32_t flags, void* scratch) {
  using TA = typename AccOf<TB>::T;
  SpmmParams<TV, TB> prm{};
  prm.rowptr = P->rowptr;
  prm.remap = P->d_remap;
  prm.val = (const TV*)P->val;
  prm.Bpack = (const TB*)Bpack;
  prm.ldp = ldp;
  prm.B = (const TB*)B;
  prm.ldb = ldb;
  prm.N = N;
  prm.C = (TA*)C;
  prm.ldc = ldc;
  prm.items = P->d_items;
  prm.n_items = P->n_items;
  prm.scratch = (TA*)(scratch ? (void*)(((uintptr_t)scratch + 255) & ~(uintptr_t)255) : nullptr);
  prm.slot_lr = P->d_slot_lr;
  prm.lr = P->d_lr;
  prm.counters = P->d_counters;
  prm.chunk = P->opts.chunk_nnz;
  prm.accumulate = (flags & SHIRO_SPMM_ACCUMULATE) ? 1 : 0;
  prm.persistent = P->opts.persistent;
  prm.status = P->d_status;
  {
    const size_t rb = (size_t)N * dtype_size(dt);
    const bool al16 = ((uintptr_t)Bpack % 16) == 0 && ((size_t)ldp * dtype_size(dt)) % 16 == 0 &&
                      (!(P->flags & SHIRO_PLAN_LOCAL_DIAG) ||
                       (((uintptr_t)B % 16) == 0 && ((size_t)ldb * dtype_size(dt)) % 16 == 0));
    prm.pf_bytes = (rb % 16 == 0 && rb > 0 && rb <= (1u << 20) && al16) ? (int32_t)rb : 0;
  }
  return prm;
}

template <typename TV, typename TB>
static shiro_status spmm_typed(const shiro_plan_s* P, const void* Bpack, int64_t ldp,
                               const void* B, int64_t ldb, int32_t N, shiro_dtype dt, void* C,
                               int64_t ldc, uint32_t flags, void* scratch, cudaStream_t s) {
  using TA = typename AccOf<TB>::T;
  const SpmmParams<TV, TB> prm =
      make_params<TV, TB>(P, Bpack, ldp, B, ldb, N, dt, C, ldc, flags, scratch);
  const size_t esz = dtype_size(dt);
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  auto ok = [&](int vec) {
    bool r = aligned(Bpack, ldp, esz, vec) && aligned(C, ldc, sizeof(TA), vec);
    if (local) r = r && aligned(B, ldb, esz, vec);
    return r;
  };
  if constexpr (!std::is_same<TB, double>::value) {
    // Narrow rows (128 or 256 bytes) split across lane groups (pipeline 3).
    const int64_t row_bytes = (int64_t)N * (int64_t)esz;
    if (P->opts.pipeline == 3 && (row_bytes == 128 || row_bytes == 256) && ok((int)(16 / esz))) {
      if (row_bytes == 128) return launch_grouped<TV, TB, 4>(P, prm, s);
      return launch_grouped<TV, TB, 2>(P, prm, s);
    }
  }
  const int v16 = (int)(16 / esz);
  const Variant v = pick_variant(dt, N, ok(v16), ok(v16 / 2 ? v16 / 2 : 1), ok(v16 / 4 ? v16 / 4 : 1));
  if (!v.vec) SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "N=%d beyond the supported 512 columns", N);
  return dispatch<TV, TB>(P, prm, v, s);
}

template <typename TV, typename TB, int VEC, int NCH>
static shiro_status launch_lean_fused(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                                      const FusedParams<TB>& f, cudaStream_t s) {
  constexpr int U = LeanShape<TB, VEC>::WIDE ? SHIRO_LEAN_UW : Occupancy<VEC, NCH, TB>::U;
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  auto kern = local ? k_spmm_lean_fused<TV, TB, VEC, NCH, U, true>
                    : k_spmm_lean_fused<TV, TB, VEC, NCH, U, false>;
  if (f.n_seq <= 0) return SHIRO_OK;
  int per_sm = 0;
  SHIRO_CUDA(blocks_per_sm(&per_sm, kern, 64, 0));
  const int64_t grid = std::min<int64_t>(((int64_t)f.n_seq + 1) / 2,
                                         (int64_t)std::max(per_sm, 1) * P->sm_count);
  SpmmParams<TV, TB> q = prm;
  q.n_chunk_items = P->n_slots;
  q.work = P->d_status + 2;
  SHIRO_CUDA(cudaMemsetAsync(q.work, 0, sizeof(int32_t), s));
  SHIRO_CUDA(cudaMemsetAsync(f.done, 0, sizeof(int32_t) * (size_t)std::max(P->geo.Pr, 1), s));
  kern<<<(unsigned)grid, 64, 0, s>>>(q, f);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

// Pack + SpMM in one launch (k_spmm_lean_fused): FP32 / BF16 rows of 512 bytes in one fragment per
// lane, pipeline 0 or 6 (BF16 with pipeline 0 only where the gather4 ring cannot run), not
// persistent, operands aligned to the fragment.  *fused = false (nothing launched) otherwise.
template <typename TV, typename TB>
static shiro_status spmm_fused_typed(const shiro_plan_s* P, const void* B, int64_t ldb, int32_t N,
                                     shiro_dtype dt, void* Bpack, int64_t ldp, void* C,
                                     int64_t ldc, uint32_t flags, void* scratch, cudaStream_t s,
                                     bool* fused) {
  using TA = typename AccOf<TB>::T;
  *fused = false;
  if constexpr (std::is_same<TB, double>::value) {
    return SHIRO_OK;
  } else {
    if (P->opts.persistent || (P->opts.pipeline != 0 && P->opts.pipeline != 6)) return SHIRO_OK;
    if (P->n_fseq > INT32_MAX) return SHIRO_OK;
    const SpmmParams<TV, TB> prm =
        make_params<TV, TB>(P, Bpack, ldp, B, ldb, N, dt, C, ldc, flags, scratch);
    const size_t esz = dtype_size(dt);
    // The pack reads B and writes Bpack with the gather's fragments.
    auto ok = [&](int vec) {
      return aligned(Bpack, ldp, esz, vec) && aligned(C, ldc, sizeof(TA), vec) &&
             aligned(B, ldb, esz, vec);
    };
    const int v16 = (int)(16 / esz);
    const Variant v =
        pick_variant(dt, N, ok(v16), ok(v16 / 2 ? v16 / 2 : 1), ok(v16 / 4 ? v16 / 4 : 1));
    if (v.nch != 1 || v.masked) return SHIRO_OK;
    FusedParams<TB> f{P->d_fseq, (int32_t)P->n_fseq, P->d_pchunk, P->d_blk_need,
                      P->d_blk_done, P->d_pack_src, (TB*)Bpack, P->geo};
    // One launch only for rows of 512 bytes (FP32 N = 128, BF16 N = 256), where it measured
    // faster than the two launches (R-MAT 2^20, 4x4 tiles, ms: FP32 N = 128 0.767 -> 0.750; R-MAT
    // 2^22 BF16 N = 256 7.18 -> 7.06); narrower rows measured slower fused (FP32 N = 64 0.479 ->
    // 0.509, BF16 N = 128 0.560 -> 0.565) and take the two launches.
    const int row = N * (int)esz;
    if (row != 512) return SHIRO_OK;
    // BF16 rows of 512 bytes with the automatic pipeline: the pack, then the TMA gather4 ring
    // (pipeline 7), are faster as two launches than this one with register gathers (R-MAT 2^22
    // avg degree 32, N = 256, chunks in column order: 0.98 + 5.29 ms against 6.55 ms).
    if constexpr (!std::is_same<TB, float>::value) {
      if (P->opts.pipeline == 0 && v.vec == 8 && g4_ok<TV, TB, 8>(P, prm)) return SHIRO_OK;
    }
    *fused = true;
    if constexpr (std::is_same<TB, float>::value) {
      if (v.vec == 4) return launch_lean_fused<TV, TB, 4, 1>(P, prm, f, s);
    } else {
      if (v.vec == 8) return launch_lean_fused<TV, TB, 8, 1>(P, prm, f, s);
    }
    *fused = false;
    return SHIRO_OK;
  }
}

template <typename TV, typename TB, int VEC>
static shiro_status launch_lean_bwd(const shiro_plan_s* P, const SpmmParams<TV, TB>& prm,
                                    const FusedParams<TB>& f, const SdParams<TB>& sd,
                                    cudaStream_t s) {
  constexpr int U = LeanShape<TB, VEC>::WIDE ? SHIRO_LEAN_UW : Occupancy<VEC, 1, TB>::U;
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  auto kern = local ? k_spmm_lean_bwd<TV, TB, VEC, U, true> : k_spmm_lean_bwd<TV, TB, VEC, U, false>;
  if (f.n_seq <= 0) return SHIRO_OK;
  int per_sm = 0;
  SHIRO_CUDA(blocks_per_sm(&per_sm, kern, 64, 0));
  const int64_t grid = std::min<int64_t>(((int64_t)f.n_seq + 1) / 2,
                                         (int64_t)std::max(per_sm, 1) * P->sm_count);
  SpmmParams<TV, TB> q = prm;
  q.n_chunk_items = P->n_slots;
  q.work = P->d_status + 2;
  SHIRO_CUDA(cudaMemsetAsync(q.work, 0, sizeof(int32_t), s));
  SHIRO_CUDA(cudaMemsetAsync(f.done, 0, sizeof(int32_t) * (size_t)std::max(P->geo.Pr, 1), s));
  kern<<<(unsigned)grid, 64, 0, s>>>(q, f, sd);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

// The backward in one launch (k_spmm_lean_bwd) on the TRANSPOSE plan PT: dCpack and dB as
// spmm_fused_typed(PT, dC, ...) computes them, plus dA (A's nonzero order) from the same gathers
// and B.  For FP32 / BF16 rows of 256 or 512 bytes with pipeline 0 or 6, not persistent, operands
// and B aligned to the lane's 8- or 16-byte slice; *done = false (nothing launched) otherwise.
template <typename TV, typename TB>
static shiro_status spmm_bwd_typed(const shiro_plan_s* PT, const void* dC, int64_t lddc,
                                   int32_t N, shiro_dtype dt, void* dCpack, int64_t lddp,
                                   void* dB, int64_t lddb, const void* B, int64_t ldb, void* dA,
                                   void* scratch, cudaStream_t s, bool* done) {
  using TA = typename AccOf<TB>::T;
  *done = false;
  if constexpr (std::is_same<TB, double>::value) {
    return SHIRO_OK;
  } else {
    if (PT->opts.persistent || (PT->opts.pipeline != 0 && PT->opts.pipeline != 6)) return SHIRO_OK;
    if (PT->n_fseq > INT32_MAX || !PT->d_perm) return SHIRO_OK;
    const size_t esz = dtype_size(dt);
    const int64_t row = (int64_t)N * (int64_t)esz;
    if (row != 512 && row != 256) return SHIRO_OK;
    const int vec = (int)(row / 32 / (int64_t)esz);  // a 16- or 8-byte slice per lane
    if (!(aligned(dCpack, lddp, esz, vec) && aligned(dB, lddb, sizeof(TA), vec) &&
          aligned(dC, lddc, esz, vec) && aligned(B, ldb, esz, vec)))
      return SHIRO_OK;
    const SpmmParams<TV, TB> prm =
        make_params<TV, TB>(PT, dCpack, lddp, dC, lddc, N, dt, dB, lddb, 0, scratch);
    FusedParams<TB> f{PT->d_fseq, (int32_t)PT->n_fseq, PT->d_pchunk, PT->d_blk_need,
                      PT->d_blk_done, PT->d_pack_src, (TB*)dCpack, PT->geo};
    SdParams<TB> sd{(const TB*)B, (uint32_t)ldb, (float*)dA, PT->d_perm};
    *done = true;
    if constexpr (std::is_same<TB, float>::value)
      return row == 512 ? launch_lean_bwd<TV, TB, 4>(PT, prm, f, sd, s)
                        : launch_lean_bwd<TV, TB, 2>(PT, prm, f, sd, s);
    else
      return row == 512 ? launch_lean_bwd<TV, TB, 8>(PT, prm, f, sd, s)
                        : launch_lean_bwd<TV, TB, 4>(PT, prm, f, sd, s);
  }
}

}  // namespace shiro
