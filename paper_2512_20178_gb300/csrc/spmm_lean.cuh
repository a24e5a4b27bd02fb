// spmm_lean.cuh -- register gathers with a 48-register budget, so that 40 warps fit on an SM
// (2-warp CTAs, 20 per SM) instead of 32: more rows in flight per SM for the same U per warp.
//
// What the 64-register loop keeps in registers and this one does not:
//   * the (index, value) pairs of the next batch: copied straight into the other half of a
//     double-buffered shared-memory batch by cp.async (4-byte copies, no register staging);
//   * the values of the rows in flight: read again from shared memory at the FMA;
//   * per-lane row state: one word, the row's end relative to the item's first nonzero, 0 for
//     rows that end nowhere (empty rows and lanes past the item's rows).
// Rows are summed in the same order as the register-gather and copy pipelines, so C is
// bit-identical to theirs.  k_spmm_lean runs one item per warp; k_spmm_lean_dyn runs SMs x 20
// blocks whose warps take items from a counter in the plan, so that no warp waits for its block's
// other warp.
#pragma once

#include "internal.cuh"
#include "vec.cuh"

namespace shiro {

// 2-warp CTAs resident per SM (65,536 registers / (20 x 64 threads) -> 48 registers per thread).
// Measured against 24 (40 registers) on R-MAT 2^20, 4x4 tiles: 48 registers is as fast or faster
// for FP32 N = 128 and clearly faster for FP32 N = 64 and BF16 N = 128 / 256.
constexpr int LEAN_MIN_BLOCKS = 20;
// BF16 rows of 512 bytes: rows in flight per warp and CTAs per SM.  Measured (ms; R-MAT 2^20 SpMM,
// R-MAT 2^22 avg degree 32 SpMM / pack + SpMM): U = 2, 20 CTAs (48 registers) 0.824, 6.01 / 6.72;
// U = 4, 16 CTAs (64 registers, 40-60 bytes spilled) 0.776, 6.34 / 6.64; U = 2, 16 CTAs 0.826,
// 6.25 / 7.06; U = 4, 12 CTAs 0.789, 6.38 / 7.46.  More rows per warp pay where the gathers hit
// L2 and lose where they go to HBM (the full-size workload), so the default stays.
#ifndef SHIRO_LEAN_MINB_W
#define SHIRO_LEAN_MINB_W 20
#endif
#ifndef SHIRO_LEAN_UW
#define SHIRO_LEAN_UW 2
#endif
// Steps of the batch loop unrolled, per row shape (one step = U gathers, then their FMAs):
// unrolling lets the next step's gathers issue before this step's FMAs, which pays where a step
// is short (narrow rows) and spills where it is long.  R-MAT 2^20, 4x4 tiles, SpMM ms by unroll
// factor 1 / 2 / 4 / 8: FP32 N = 32 0.336 / 0.293 / 0.294 / 0.308; FP32 N = 64 0.370 / 0.381 /
// 0.364; BF16 N = 64 0.359 / 0.356 / 0.316 / 0.366; BF16 N = 128 0.444 / 0.447 / 0.461; FP32 N =
// 128 0.552 / 0.785 (spills).
#ifndef SHIRO_LEAN_DYN_BF16V4
#define SHIRO_LEAN_DYN_BF16V4 0
#endif
#ifndef SHIRO_LU_F32V1
#define SHIRO_LU_F32V1 2
#endif
#ifndef SHIRO_LU_F32V2
#define SHIRO_LU_F32V2 4
#endif
#ifndef SHIRO_LU_BF16V2
#define SHIRO_LU_BF16V2 4
#endif
#ifndef SHIRO_LU_BF16V4
#define SHIRO_LU_BF16V4 1
#endif

// FP32 rows in float4 fragments (16 registers per U = 4 rows in flight) take one loop copy for
// full and partial batches: three copies spill there (112 bytes at 48 registers), and so does a
// copy for full batches with row ends; one copy ran FP32 N = 128 in 0.561 ms against 0.680 (three
// copies) and 0.635 (two).  Other rows take the three copies.
template <typename TB, int VEC>
struct LeanShape {
  static constexpr bool ONE_COPY = std::is_same<TB, float>::value && VEC == 4;
  // The automatic pipeline runs the persistent form (items from a counter) for every row shape
  // but BF16 rows of 256 bytes, measured slower with it (R-MAT 2^20, 4x4 tiles, ms, one item per
  // warp -> counter): FP32 N = 128 0.567 -> 0.554, N = 64 0.391 -> 0.371, N = 32 0.355 -> 0.331,
  // BF16 N = 256 0.815 -> 0.769 (R-MAT 2^22: 6.52 -> 6.16), BF16 N = 128 0.453 -> 0.474.
  static constexpr bool DYN = SHIRO_LEAN_DYN_BF16V4 || !(std::is_same<TB, __nv_bfloat16>::value && VEC == 4);
  static constexpr bool F32 = std::is_same<TB, float>::value;
  // BF16 rows of 512 bytes (eight FP32 accumulators per lane).
  static constexpr bool WIDE = std::is_same<TB, __nv_bfloat16>::value && VEC == 8;
  static constexpr int MIN_BLOCKS = WIDE ? SHIRO_LEAN_MINB_W : LEAN_MIN_BLOCKS;
  static constexpr int UNROLL = F32 ? (VEC == 1 ? SHIRO_LU_F32V1 : VEC == 2 ? SHIRO_LU_F32V2 : 1)
                                    : (VEC == 2 ? SHIRO_LU_BF16V2 : VEC == 4 ? SHIRO_LU_BF16V4 : 1);
};

template <typename TV, typename TB, int VEC, int NCH, int U, bool LOCAL, bool FULL, bool ENDS,
          bool CG = false>
__device__ __forceinline__ void lean_batch(const SpmmParams<TV, TB>& p, const Bases<TB>& bs,
                                           const Pair<TV>* sp, int n, int off, int32_t r0, int rel,
                                           unsigned endmask,
                                           typename AccOf<TB>::T (&acc)[NCH][VEC], int lane) {
  static_assert(32 % U == 0, "U must divide the 32-pair batch");
#pragma unroll LeanShape<TB, VEC>::UNROLL
  for (int j = 0; j < (FULL ? 32 : n); j += U) {
    typename RawFrag<TB, VEC>::T b[U][NCH][RawFrag<TB, VEC>::W];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (FULL || j + u < n) {
        const int32_t idx = sp[j + u].idx;
        // bs holds this lane's slice of row 0 (gather_raw adds only the chunk offsets).
        const TB* row;
        if (LOCAL && idx < 0)
          row = bs.b + (uint64_t)(uint32_t)(-1 - idx) * bs.ldb;
        else
          row = bs.bp + (uint64_t)(uint32_t)idx * bs.ldp;
        if constexpr (CG) {
          // Rows written earlier in the same launch (fused pack + SpMM): read through L2.
#pragma unroll
          for (int c = 0; c < NCH; ++c) load_raw_cg<TB, VEC>(row + c * 32 * VEC, b[u][c]);
        } else {
          gather_raw<TV, TB, VEC, NCH, false>(p, row, b[u], lane);
        }
      }
    }
#ifndef SHIRO_LEAN_PF
#define SHIRO_LEAN_PF 1
#endif
    // Rows of 512 bytes with only U = 2 in flight per warp (BF16 N = 256): bring the rows of the
    // step two ahead into L2 while this step's gathers are in flight (the TMA unit's bulk
    // prefetch: no registers, nothing to wait on), as the 64-register kernel does.  R-MAT 2^22,
    // BF16 N = 256, ms: SpMM 6.19 -> 6.12, fused pack + SpMM 7.05 -> 6.80.  U = 4 at 48 registers
    // (spills) measured 6.92.
    constexpr bool PF = SHIRO_LEAN_PF && VEC * NCH * sizeof(TB) >= 16 && U <= 2;
    if constexpr (PF) {
      const int k = j + 2 * U;
      if (p.pf_bytes && k < (FULL ? 32 : n)) {
        const int32_t ix = sp[min(k + (lane & (U - 1)), (FULL ? 32 : n) - 1)].idx;
        const TB* r = (LOCAL && ix < 0) ? p.B + (uint64_t)(uint32_t)(-1 - ix) * (uint64_t)p.ldb
                                        : p.Bpack + (uint64_t)(uint32_t)ix * (uint64_t)p.ldp;
        if (lane < U) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(r),
                                   "r"(p.pf_bytes));
      }
    }
    // One test per step for row ends among its U nonzeros (most steps have none): a step without
    // one takes the FMAs alone (one copy at 48 registers: 0.617 -> 0.561 ms for FP32 N = 128).
    const unsigned em = ENDS ? (endmask >> j) & ((1u << U) - 1u) : 0u;
    if (em == 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (FULL || j + u < n) {
          const TV a = sp[j + u].val;
#pragma unroll
          for (int c = 0; c < NCH; ++c) fma_raw<TB, VEC>(a, b[u][c], acc[c]);
        }
      }
      continue;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (FULL || j + u < n) {
        const TV a = sp[j + u].val;
#pragma unroll
        for (int c = 0; c < NCH; ++c) fma_raw<TB, VEC>(a, b[u][c], acc[c]);
        if (ENDS && ((em >> u) & 1u)) {
          const unsigned who = __ballot_sync(0xffffffffu, rel == off + j + u + 1);
          flush_row<TV, TB, VEC, NCH, false>(p, r0 + __ffs(who) - 1, acc, lane);
        }
      }
    }
  }
}

// Nonzeros [base, base + total) of rows r0 .. (lane l: rel = end of row r0 + l relative to base
// if that row is non-empty, else 0).  sp holds two batches of 32 pairs.
template <typename TV, typename TB, int VEC, int NCH, int U, bool LOCAL, bool CG = false>
__device__ __forceinline__ void lean_span(const SpmmParams<TV, TB>& p, const Bases<TB>& bs,
                                          Pair<TV>* sp, int64_t base, int total, int32_t r0,
                                          int rel, typename AccOf<TB>::T (&acc)[NCH][VEC],
                                          int lane) {
  if (total <= 0) return;
  __syncwarp();
  if (lane < total) {
    Pair<TV> pr;
    pr.idx = __ldcs(p.remap + base + lane);
    pr.val = __ldcs(p.val + base + lane);
    sp[lane] = pr;
  }
#pragma unroll 1
  for (int off = 0; off < total; off += 32) {
    Pair<TV>* cur = sp + ((off >> 5) & 1) * 32;
    Pair<TV>* nxt = sp + (((off >> 5) + 1) & 1) * 32;
    cp_async_wait<0>();
    __syncwarp();
    // The next batch's pairs land in the other half while this batch's gathers are in flight
    // (that half held the batch before this one, which every lane has finished with).
    if (off + 32 + lane < total) {
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(nxt + lane);
      cp_async<4>(d, p.remap + base + off + 32 + lane);
      cp_async<(int)sizeof(TV)>(d + (uint32_t)offsetof(Pair<TV>, val),
                                p.val + base + off + 32 + lane);
    }
    cp_async_commit();
    const int n = min(32, total - off);
    const int q = rel - 1 - off;
    const unsigned endmask = __reduce_or_sync(0xffffffffu, (q >= 0 && q < 32) ? (1u << q) : 0u);
    if constexpr (LeanShape<TB, VEC>::ONE_COPY) {
      lean_batch<TV, TB, VEC, NCH, U, LOCAL, false, true, CG>(p, bs, cur, n, off, r0, rel,
                                                              endmask, acc, lane);
    } else {
      // Full batches without a row end (all chunk batches, most batches of long rows) take a copy
      // without per-nonzero tests; full batches with row ends a copy without bounds tests.
      if (n == 32 && endmask == 0)
        lean_batch<TV, TB, VEC, NCH, U, LOCAL, true, false, CG>(p, bs, cur, n, off, r0, rel,
                                                                endmask, acc, lane);
      else if (n == 32)
        lean_batch<TV, TB, VEC, NCH, U, LOCAL, true, true, CG>(p, bs, cur, n, off, r0, rel,
                                                               endmask, acc, lane);
      else
        lean_batch<TV, TB, VEC, NCH, U, LOCAL, false, true, CG>(p, bs, cur, n, off, r0, rel,
                                                                endmask, acc, lane);
    }
  }
  cp_async_wait<0>();
}

// Blocks [0, chunk_blocks) run the chunks of long rows, the others the row groups; two warps per
// block, one item per warp (no persistent mode).
template <typename TV, typename TB, int VEC, int NCH, int U, bool LOCAL>
__global__ void __launch_bounds__(64, (LeanShape<TB, VEC>::MIN_BLOCKS))
    k_spmm_lean(const SpmmParams<TV, TB> p) {
  using TA = typename AccOf<TB>::T;
  __shared__ Pair<TV> s_pairs[2][64];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  Pair<TV>* sp = s_pairs[warp];
  Bases<TB> bs;
  bs.bp = p.Bpack + lane * VEC;
  bs.b = p.B + lane * VEC;
  bs.ldp = (uint32_t)p.ldp;
  bs.ldb = (uint32_t)p.ldb;
  TA acc[NCH][VEC];
#pragma unroll
  for (int c = 0; c < NCH; ++c)
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[c][v] = 0;
  if ((int64_t)blockIdx.x < p.chunk_blocks) {
    const int64_t it = (int64_t)blockIdx.x * 2 + warp;
    if (it >= p.n_chunk_items) return;
    const Item item = p.items[it];
    const int64_t row_end = __ldg(p.rowptr + item.row + 1);
    const int total = (int)min((int64_t)p.chunk, row_end - item.e0);
    lean_span<TV, TB, VEC, NCH, U, LOCAL>(p, bs, sp, item.e0, total, item.row, 0, acc, lane);
    finish_chunk<TV, TB, VEC, NCH, false>(p, -item.tag - 1, acc, lane);
  } else {
    const int64_t it = p.n_chunk_items + ((int64_t)blockIdx.x - p.chunk_blocks) * 2 + warp;
    if (it >= p.n_items) return;
    const Item item = p.items[it];
    const int32_t r0 = item.row, nr = item.tag;
    const int64_t rp = lane < nr ? __ldg(p.rowptr + r0 + lane + 1) : 0;
    int rel = (int)(rp - item.e0);
    const int prev = __shfl_up_sync(0xffffffffu, rel, 1);
    const bool nonempty = lane < nr && rel > (lane ? prev : 0);
    const int total = __shfl_sync(0xffffffffu, rel, nr - 1);
    if (!p.accumulate) {
      unsigned empty = __ballot_sync(0xffffffffu, lane < nr && !nonempty);
      while (empty) {
        const int l = __ffs(empty) - 1;
        empty &= empty - 1;
        flush_row<TV, TB, VEC, NCH, false>(p, r0 + l, acc, lane);
      }
    }
    rel = nonempty ? rel : 0;
    lean_span<TV, TB, VEC, NCH, U, LOCAL>(p, bs, sp, item.e0, total, r0, rel, acc, lane);
  }
}

// Persistent form (SMs x resident blocks of two warps): every warp takes the next item from a
// counter (zeroed before the launch) until none is left, chunks of long rows first, so a warp
// whose item ends early does not wait for its block's other warp.  Kept apart from k_spmm_lean:
// a loop around both item paths costs that kernel registers.
template <typename TV, typename TB, int VEC, int NCH, int U, bool LOCAL>
__global__ void __launch_bounds__(64, (LeanShape<TB, VEC>::MIN_BLOCKS))
    k_spmm_lean_dyn(const SpmmParams<TV, TB> p) {
  using TA = typename AccOf<TB>::T;
  __shared__ Pair<TV> s_pairs[2][64];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  Pair<TV>* sp = s_pairs[warp];
  Bases<TB> bs;
  bs.bp = p.Bpack + lane * VEC;
  bs.b = p.B + lane * VEC;
  bs.ldp = (uint32_t)p.ldp;
  bs.ldb = (uint32_t)p.ldb;
  const int n_items = (int)p.n_items, n_chunks = (int)p.n_chunk_items;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(p.work, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n_items) break;
    const Item item = p.items[it];
    TA acc[NCH][VEC];
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[c][v] = 0;
    int32_t r0 = item.row;
    int rel = 0, total;
    if (it < n_chunks) {
      total = (int)min((int64_t)p.chunk, __ldg(p.rowptr + item.row + 1) - item.e0);
    } else {
      const int nr = item.tag;
      const int64_t rp = lane < nr ? __ldg(p.rowptr + r0 + lane + 1) : 0;
      rel = (int)(rp - item.e0);
      const int prev = __shfl_up_sync(0xffffffffu, rel, 1);
      const bool nonempty = lane < nr && rel > (lane ? prev : 0);
      total = __shfl_sync(0xffffffffu, rel, nr - 1);
      if (!p.accumulate) {
        unsigned empty = __ballot_sync(0xffffffffu, lane < nr && !nonempty);
        while (empty) {
          const int l = __ffs(empty) - 1;
          empty &= empty - 1;
          flush_row<TV, TB, VEC, NCH, false>(p, r0 + l, acc, lane);
        }
      }
      rel = nonempty ? rel : 0;
    }
    // One span call for both kinds of item (a chunk has no row end: rel = 0 in every lane).
    lean_span<TV, TB, VEC, NCH, U, LOCAL>(p, bs, sp, item.e0, total, r0, rel, acc, lane);
    if (it < n_chunks) finish_chunk<TV, TB, VEC, NCH, false>(p, -item.tag - 1, acc, lane);
  }
}

// ---- fused pack + SpMM (one launch) ----
//
// The launch walks a plan-built order of work: the pack chunks of row block 0 (Bpack[r] =
// B[pack_src[r]], at most 32 rows each), then for every block p its SpMM items with the pack
// chunks of block p + 1 spread among them.  A warp that takes a pack chunk copies it and counts it
// done for its block (every lane's stores, a fence, a warp barrier, then one atomic: release); a
// warp that takes an item of block p first waits until all of block p's chunks are counted (lane 0
// polls with acquire loads, the warp barrier orders the other lanes after it).  The chunks of a
// block all precede its items in the order, and a warp holding a chunk never waits, so every wait
// ends; each is still bounded, and on expiry the warp sets ST_TIMEOUT and goes on.  Packed rows are
// gathered through L2 (ld.global.cg): other warps of the launch wrote them.  Bpack and C are
// bit-identical to shiro_pack followed by the SpMM (same items, same summation order).
template <typename TB>
struct FusedParams {
  const int32_t* seq;     // >= 0: item index, < 0: pack chunk -code - 1
  int32_t n_seq;
  const int4* pchunk;     // {first packed row, rows, row block, 0}
  const int32_t* need;    // pack chunks per row block
  int32_t* done;          // pack chunks finished per row block (zeroed before the launch)
  const int32_t* pack_src;
  TB* Bpack;              // written by the pack chunks, read by the items
  Geometry geo;
};

constexpr uint32_t kFusedSpinLimit = 1u << 22;  // x 256 ns sleeps: about a second
#ifndef SHIRO_FUSED_PACK_U
#define SHIRO_FUSED_PACK_U 4  // rows a lane copies at once in a pack chunk
#endif
#ifndef SHIRO_FUSED_PACK_STAGED
#define SHIRO_FUSED_PACK_STAGED 1  // pack chunks staged through shared memory (cp.async)
#endif
#ifndef SHIRO_FUSED_PACK_HINT
// Evict-first L2 policy on the pack's B reads and Bpack writes, so that they displace fewer of the
// gathered rows (ms, R-MAT 2^20 FP32 N = 128 0.758 -> 0.751; R-MAT 2^22 BF16 N = 256 6.80 -> 6.78).
#define SHIRO_FUSED_PACK_HINT 1
#endif

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ int ld_acquire_gpu(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename TV, typename TB, int VEC, int NCH, int U>
__device__ __forceinline__ void fused_pack_chunk(const SpmmParams<TV, TB>& p,
                                                 const FusedParams<TB>& f, const int4 c,
                                                 int lane) {
  using RF = RawFrag<TB, VEC>;
  const TB* src0 = p.B + lane * VEC;
  TB* dst0 = f.Bpack + lane * VEC;
  const uint32_t ldb = (uint32_t)p.ldb, ldp = (uint32_t)p.ldp;
  // Lane j holds the source row of the chunk's row j (one coalesced load per chunk).
  const int32_t my_src = lane < c.y ? __ldg(f.pack_src + c.x + lane) : 0;
#pragma unroll 1
  for (int r = 0; r < c.y; r += U) {
    typename RF::T w[U][NCH][RF::W];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (r + u < c.y) {  // warp-uniform
        const int32_t s = __shfl_sync(0xffffffffu, my_src, r + u);
        gather_raw<TV, TB, VEC, NCH, false>(p, src0 + (uint64_t)(uint32_t)s * ldb, w[u], lane);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (r + u < c.y) {
        TB* d = dst0 + (uint64_t)(uint32_t)(c.x + r + u) * ldp;
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) store_raw<TB, VEC>(d + ch * 32 * VEC, w[u][ch]);
      }
    }
  }
  // Release: each lane's stores are fenced, the warp barrier orders them before lane 0, which
  // fences again (cumulative over what the barrier ordered) and counts the chunk.
  __threadfence();
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    atomicAdd(f.done + c.z, 1);
  }
}

// The same copy staged through shared memory by cp.async: the U rows in flight cost no registers
// (each lane reads back only its own slice, so no cross-lane wait is needed), then each lane
// stores its slices.  stage: U rows of 32 * VEC elements for this warp.
template <typename TV, typename TB, int VEC, int U>
__device__ __forceinline__ void fused_pack_chunk_staged(const SpmmParams<TV, TB>& p,
                                                        const FusedParams<TB>& f, const int4 c,
                                                        TB* stage, int lane) {
  constexpr int LB = VEC * (int)sizeof(TB);  // bytes of a lane's slice: 4, 8 or 16
  constexpr int ROW = 32 * VEC;               // elements of a staged row
  const TB* src0 = p.B + lane * VEC;
  TB* dst0 = f.Bpack + lane * VEC;
  const uint32_t ldb = (uint32_t)p.ldb, ldp = (uint32_t)p.ldp;
  const uint32_t st0 = (uint32_t)__cvta_generic_to_shared(stage + lane * VEC);
  const int32_t my_src = lane < c.y ? __ldg(f.pack_src + c.x + lane) : 0;
  const uint64_t pol = SHIRO_FUSED_PACK_HINT ? l2_evict_first_policy() : 0;
#pragma unroll 1
  for (int r = 0; r < c.y; r += U) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (r + u < c.y) {  // warp-uniform
        const int32_t s = __shfl_sync(0xffffffffu, my_src, r + u);
        if constexpr (SHIRO_FUSED_PACK_HINT && LB == 16)
          asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(
                           st0 + (uint32_t)(u * ROW * (int)sizeof(TB))),
                       "l"(src0 + (uint64_t)(uint32_t)s * ldb), "l"(pol)
                       : "memory");
        else
          cp_async<LB>(st0 + (uint32_t)(u * ROW * (int)sizeof(TB)),
                       src0 + (uint64_t)(uint32_t)s * ldb);
      }
    }
    cp_async_commit();
    cp_async_wait<0>();
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (r + u < c.y) {
        const TB* sp = stage + u * ROW + lane * VEC;
        if constexpr (LB == 16) {
          const uint4 v = *reinterpret_cast<const uint4*>(sp);
          uint4* d = reinterpret_cast<uint4*>(dst0 + (uint64_t)(uint32_t)(c.x + r + u) * ldp);
          if constexpr (SHIRO_FUSED_PACK_HINT)
            asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(d),
                         "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "l"(pol)
                         : "memory");
          else
            *d = v;
        } else if constexpr (LB == 8) {
          const uint2 v = *reinterpret_cast<const uint2*>(sp);
          *reinterpret_cast<uint2*>(dst0 + (uint64_t)(uint32_t)(c.x + r + u) * ldp) = v;
        } else {
          const uint32_t v = *reinterpret_cast<const uint32_t*>(sp);
          *reinterpret_cast<uint32_t*>(dst0 + (uint64_t)(uint32_t)(c.x + r + u) * ldp) = v;
        }
      }
    }
  }
  // Release: each lane's stores are fenced, the warp barrier orders them before lane 0, which
  // fences again (cumulative over what the barrier ordered) and counts the chunk.
  __threadfence();
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    atomicAdd(f.done + c.z, 1);
  }
}

template <typename TB>
__device__ __forceinline__ void fused_wait_block(const FusedParams<TB>& f, int32_t blk,
                                                 int* status, int lane) {
  if (lane == 0) {
    const int need = __ldg(f.need + blk);
    uint32_t spins = 0;
    while (ld_acquire_gpu(f.done + blk) < need) {
      if (++spins > kFusedSpinLimit) {
        atomicOr(status, ST_TIMEOUT);
        break;
      }
      __nanosleep(256);
    }
  }
  __syncwarp();
}

template <typename TV, typename TB, int VEC, int NCH, int U, bool LOCAL>
__global__ void __launch_bounds__(64, (LeanShape<TB, VEC>::MIN_BLOCKS))
    k_spmm_lean_fused(const SpmmParams<TV, TB> p, const FusedParams<TB> f) {
  using TA = typename AccOf<TB>::T;
  __shared__ Pair<TV> s_pairs[2][64];
  constexpr int STAGE = SHIRO_FUSED_PACK_STAGED ? SHIRO_FUSED_PACK_U * 32 * VEC : 1;
  __shared__ __align__(16) TB s_stage[2][STAGE];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  Pair<TV>* sp = s_pairs[warp];
  Bases<TB> bs;
  bs.bp = f.Bpack + lane * VEC;
  bs.b = p.B + lane * VEC;
  bs.ldp = (uint32_t)p.ldp;
  bs.ldb = (uint32_t)p.ldb;
  int32_t known = -1;  // highest row block this warp has seen fully packed
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(p.work, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= f.n_seq) break;
    const int32_t code = __ldg(f.seq + it);
    if (code < 0) {
      const int4 c = __ldg(f.pchunk + (-code - 1));
      if constexpr (SHIRO_FUSED_PACK_STAGED && NCH == 1)
        fused_pack_chunk_staged<TV, TB, VEC, SHIRO_FUSED_PACK_U>(p, f, c, s_stage[warp], lane);
      else
        fused_pack_chunk<TV, TB, VEC, NCH, SHIRO_FUSED_PACK_U>(p, f, c, lane);
      continue;
    }
    const Item item = p.items[code];
    // A warp takes its items in launch order, so their row blocks never decrease.
    const int32_t blk = row_block(f.geo, item.row);
    if (blk > known) {
      fused_wait_block<TB>(f, blk, p.status, lane);
      known = blk;
    }
    TA acc[NCH][VEC];
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[c][v] = 0;
    const bool chunk = item.tag <= 0;
    int32_t r0 = item.row;
    int rel = 0, total;
    if (chunk) {
      total = (int)min((int64_t)p.chunk, __ldg(p.rowptr + item.row + 1) - item.e0);
    } else {
      const int nr = item.tag;
      const int64_t rp = lane < nr ? __ldg(p.rowptr + r0 + lane + 1) : 0;
      rel = (int)(rp - item.e0);
      const int prev = __shfl_up_sync(0xffffffffu, rel, 1);
      const bool nonempty = lane < nr && rel > (lane ? prev : 0);
      total = __shfl_sync(0xffffffffu, rel, nr - 1);
      if (!p.accumulate) {
        unsigned empty = __ballot_sync(0xffffffffu, lane < nr && !nonempty);
        while (empty) {
          const int l = __ffs(empty) - 1;
          empty &= empty - 1;
          flush_row<TV, TB, VEC, NCH, false>(p, r0 + l, acc, lane);
        }
      }
      rel = nonempty ? rel : 0;
    }
    lean_span<TV, TB, VEC, NCH, U, LOCAL, true>(p, bs, sp, item.e0, total, r0, rel, acc, lane);
    if (chunk) finish_chunk<TV, TB, VEC, NCH, false>(p, -item.tag - 1, acc, lane);
  }
}

}  // namespace shiro
