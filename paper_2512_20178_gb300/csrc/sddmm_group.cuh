// sddmm_group.cuh -- dA[e] = <dC[row e], B[col e]> by lane groups: the warp's 32 lanes form four
// groups of eight, and each group takes one nonzero per step, so a step finishes four dot
// products with a three-level shuffle reduction inside each group (no cross-group transposition,
// no selects, no partial-sum registers beyond one).
//
// A row of dC / B of RB bytes (128, 256 or 512: FP32 N = 32 / 64 / 128, BF16 N = 64 / 128 / 256) is
// split into 16-byte fragments; lane k of a group owns fragments k, k + 8, ..., so that each load
// instruction moves one contiguous 128-byte line per group.  A lane holds the dC fragments of its
// group's current row (RB / 128 of them) and the B fragments of the nonzero in flight.
//
// Per batch of 32 nonzeros (indices staged in shared memory by cp.async one batch ahead), group g
// takes positions 8g .. 8g + 7 in order, so consecutive nonzeros of a row stay in one group and
// its dC fragments are reloaded only when the row changes; BF16 rows of 512 bytes keep the B
// row of the group's next position in flight as well (SdgShape).  The row of every position comes from
// a warp max-scan over the starts of the item's non-empty rows.  After the eight steps lane j
// holds the sum of position j and dA is written once per batch, coalesced.
//
// Summation order of one dot product: each lane sums every fragment's products in element order
// (one FMA chain per fragment: FP32 N = 128 0.722 -> 0.566 ms against one chain over all), adds
// the fragment sums pairwise, then the eight lanes' sums are added by the butterfly (xor 4, 2, 1)
// -- fixed, so dA is deterministic.
#pragma once

#include "internal.cuh"
#include "sddmm_lean.cuh"
#include "vec.cuh"

namespace shiro {

// Per row shape, the gathers in flight per group and the register budget (2-warp CTAs per SM):
// BF16 rows of 512 bytes keep two B rows in flight per group (the row of step s + 1 is loaded
// before step s's dot) at 64 registers, 16 CTAs per SM; the other shapes one row per group at 48
// registers, 20 CTAs per SM, with the eight steps unrolled.  R-MAT 2^20, 4x4 tiles, ms (one row
// with the steps in a loop -> unrolled -> two rows, 64 registers): FP32 N = 128 0.572 -> 0.554 ->
// 0.621, FP32 N = 64 0.428 -> 0.410 -> 0.449, BF16 N = 256 0.931 -> 0.910 -> 0.807, BF16 N = 128
// 0.507 -> 0.493 -> 0.523; two rows at 48 registers spilled (FP32 N = 128 0.988).
template <typename TB, int L>
struct SdgShape {
  static constexpr int DEPTH = (std::is_same<TB, __nv_bfloat16>::value && L == 4) ? 2 : 1;
  static constexpr int MIN_BLOCKS = DEPTH == 2 ? 16 : 20;
};

// s + <g, b> over one 16-byte fragment of FP32 or BF16 storage, in element order (BF16 widened
// exactly).
template <typename TB>
__device__ __forceinline__ float dot_frag16(const uint4& g, const uint4& b, float s) {
  if constexpr (std::is_same<TB, float>::value) {
    s = fmaf(__uint_as_float(g.x), __uint_as_float(b.x), s);
    s = fmaf(__uint_as_float(g.y), __uint_as_float(b.y), s);
    s = fmaf(__uint_as_float(g.z), __uint_as_float(b.z), s);
    s = fmaf(__uint_as_float(g.w), __uint_as_float(b.w), s);
  } else {
    // One chain in element order (two chains, even and odd elements, measured slower for BF16
    // N = 256: 1.03 -> 1.25 ms on R-MAT 2^20).
    const uint32_t gw[4] = {g.x, g.y, g.z, g.w};
    const uint32_t bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      s = fmaf(bf16_lo(gw[i]), bf16_lo(bw[i]), s);
      s = fmaf(bf16_hi(gw[i]), bf16_hi(bw[i]), s);
    }
  }
  return s;
}

// L 16-byte fragments at stride 128 bytes from p (this lane's slices of a row).
template <int L>
__device__ __forceinline__ void load_frags(const char* p, uint4 (&v)[L]) {
#pragma unroll
  for (int f = 0; f < L; ++f) v[f] = __ldg(reinterpret_cast<const uint4*>(p + f * 128));
}

// One partial per fragment (independent FMA chains, element order within each), added pairwise.
template <typename TB, int L>
__device__ __forceinline__ float grp_dot(const uint4 (&g)[L], const uint4 (&b)[L]) {
  float part[L];
#pragma unroll
  for (int f = 0; f < L; ++f) part[f] = dot_frag16<TB>(g[f], b[f], 0.f);
#pragma unroll
  for (int w = 1; w < L; w <<= 1)
#pragma unroll
    for (int f = 0; f + w < L; f += 2 * w) part[f] += part[f + w];
  return part[0];
}

// One work item (a group of rows or a chunk of a long row).  sidx: 2 x 32 staged indices;
// srow: 32 item-local rows of the batch's positions.
template <typename TB, int L, int DEPTH>
__device__ __forceinline__ void sddmm_grp_item(const SddmmParams<TB>& p, int32_t* sidx,
                                               int32_t* srow, const Item& item, int lane) {
  const bool chunk = item.tag <= 0;
  const int32_t r0 = item.row;
  const int nr = chunk ? 1 : item.tag;
  // End of row r0 + lane relative to the item's first nonzero (monotone over the lanes; an empty
  // row repeats the end before it).
  const int64_t rp = lane < nr ? __ldg(p.rowptr + r0 + lane + 1) : 0;
  const int end = (int)(rp - item.e0);
  int total = __shfl_sync(FULLM, end, nr - 1);
  if (chunk) total = min(total, p.chunk);
  if (total <= 0) return;
  const int up = __shfl_up_sync(FULLM, end, 1);
  const int start = lane ? up : 0;
  const bool starts = !chunk && lane < nr && end > start;  // non-empty row `lane` starts here
  const int grp = lane >> 3, k = lane & 7;
  // Byte offset of this lane's fragment f within a row: (f * 8 + k) * 16.
  const uint32_t lane_off = (uint32_t)k * 16u;
  const uint32_t ldp_b = (uint32_t)p.ldp * (uint32_t)sizeof(TB);
  const uint32_t ldb_b = (uint32_t)p.ldb * (uint32_t)sizeof(TB);
  const char* dC = reinterpret_cast<const char*>(p.dC) + lane_off;
  const char* Bp = reinterpret_cast<const char*>(p.Bpack) + lane_off;
  const char* Bl = reinterpret_cast<const char*>(p.B) + lane_off;
  const uint64_t lddc_b = (uint64_t)p.lddc * sizeof(TB);

  __syncwarp();
  if (lane < total) sidx[lane] = __ldcs(p.remap + item.e0 + lane);
  int carry = -1;  // row of the last position of the previous batch
  int cur = -1;    // row whose dC fragments this lane holds
  uint4 g[L];
#pragma unroll
  for (int f = 0; f < L; ++f) g[f] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 1
  for (int off = 0; off < total; off += 32) {
    const int h = (off >> 5) & 1;
    sd_wait_all();
    __syncwarp();
    if (off + 32 + lane < total)
      sd_cp4((uint32_t)__cvta_generic_to_shared(sidx + (h ^ 1) * 32 + lane),
             p.remap + item.e0 + off + 32 + lane);
    sd_commit();
    // Rows of the batch's positions: mark where non-empty rows start, then a max-scan (rows only
    // grow along the stream), seeded with the row the previous batch ended in.
    int v = 0;
    if (!chunk) {
      srow[lane] = -1;
      __syncwarp();
      if (starts && start >= off && start < off + 32) srow[start - off] = lane;
      __syncwarp();
      v = srow[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(FULLM, v, d);
        if (lane >= d) v = max(v, t);
      }
      v = max(v, carry);
      carry = __shfl_sync(FULLM, v, 31);
      __syncwarp();
    }
    srow[lane] = v;
    __syncwarp();
    const int32_t* ci = sidx + h * 32;
    const int n = min(32, total - off);
    float out = 0.f;
    // This lane's slice of the B row of batch position j (a packed row, or a row of B itself for
    // a LOCAL_DIAG tile) and the dC row of position j, loaded when the row changes.
    auto brow = [&](int j) {
      const int32_t idx = ci[j];
      return idx >= 0 ? Bp + (uint64_t)(uint32_t)idx * ldp_b
                      : Bl + (uint64_t)(uint32_t)(-1 - idx) * ldb_b;
    };
    auto dc_row = [&](int j) {
      const int row = srow[j];
      if (row != cur) {
        const char* dr = dC + (uint64_t)(uint32_t)(r0 + row) * lddc_b;
#pragma unroll
        for (int f = 0; f < L; ++f) g[f] = __ldg(reinterpret_cast<const uint4*>(dr + f * 128));
        cur = row;
      }
    };
    // After step s, lane k == s of each group keeps its group's dot product.
    auto finish = [&](float acc, int s) {
      acc += __shfl_xor_sync(FULLM, acc, 4);
      acc += __shfl_xor_sync(FULLM, acc, 2);
      acc += __shfl_xor_sync(FULLM, acc, 1);
      if (k == s) out = acc;
    };
    if constexpr (DEPTH == 2) {
      // Two gathers in flight per group: the B row of step s + 1 is loaded before step s's dot.
      uint4 bq[2][L];
      if (grp * 8 < n) load_frags<L>(brow(grp * 8), bq[0]);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int j = grp * 8 + s;
        if (s + 1 < 8 && j + 1 < n) load_frags<L>(brow(j + 1), bq[(s + 1) & 1]);
        float acc = 0.f;
        if (j < n) {
          dc_row(j);
          acc = grp_dot<TB, L>(g, bq[s & 1]);
        }
        finish(acc, s);
      }
    } else {
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int j = grp * 8 + s;
        float acc = 0.f;
        if (j < n) {
          dc_row(j);
          uint4 b[L];
          load_frags<L>(brow(j), b);
          acc = grp_dot<TB, L>(g, b);
        }
        finish(acc, s);
      }
    }
    if (lane < n) p.dA[item.e0 + off + lane] = out;
  }
  sd_wait_all();
}

// SMs x resident blocks of two warps; every warp takes the next item from the plan's counter.
template <typename TB, int L>
__global__ void __launch_bounds__(64, (SdgShape<TB, L>::MIN_BLOCKS))
    k_sddmm_grp(const SddmmParams<TB> p) {
  __shared__ __align__(16) int32_t s_idx[2][64];
  __shared__ __align__(16) int32_t s_row[2][32];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(p.work, 1);
    it = __shfl_sync(FULLM, it, 0);
    if ((int64_t)it >= p.n_items) break;
    sddmm_grp_item<TB, L, SdgShape<TB, L>::DEPTH>(p, s_idx[warp], s_row[warp], p.items[it],
                                                   lane);
  }
}

}  // namespace shiro
