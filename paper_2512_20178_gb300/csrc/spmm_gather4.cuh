// spmm_gather4.cuh -- the SpMM over packed rows of 512 bytes (FP32 N = 128, BF16 N = 256) with the
// rows moved into shared memory by 2-D TMA gathers: one cp.async.bulk.tensor ... tile::gather4
// instruction copies the four packed rows named by four row coordinates into a 2 KB stage of the
// warp's ring, completion counted in bytes on the stage's mbarrier (Sec. 5.1 stage 5 over the
// packed buffer of stage 3).
//
// Each warp runs its own pipeline: it takes work items from the plan's counter, stages up to 256
// (index, value) pairs of the item in shared memory, and lane 0 keeps D gathers of four rows in
// flight ahead of the group the warp is multiplying.  The rows in flight cost shared memory, not
// registers (G4Shape: 2 stages of 4 rows per warp, 24-32 warps per SM).  Lane l reads its 16-byte slice of each row from the stage (one
// conflict-free 512-byte read per row) and adds it with the nonzero's value in the nonzeros' stored
// order, so C is bit-identical to the register-gather kernels.  Every wait is bounded: a phase that
// does not complete sets ST_TIMEOUT, the warp waits (bounded) for its gathers in flight and stops.
//
// Tensor map: the packed buffer as a 2-D array of 32-bit words, 128 words per row (one row of 512
// bytes), row stride ldp * sz bytes, box 128 x 1 (a gather box is one row high); the x coordinate of
// every gather is 0, so it starts on a 16-byte boundary.  Plans whose diagonal tiles read B in place
// (LOCAL_DIAG) gather from two arrays and do not take this kernel.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "spmm_bulk.cuh"
#include "vec.cuh"

namespace shiro {

// Stages per warp and warps per CTA, by storage type.  R-MAT 2^20, 4x4 tiles, SpMM ms (FP32
// N = 128 / BF16 N = 256; the 48-register gathers: 0.552 / 0.824): 8 stages x 4 warps 1.370 /
// 1.508; 16 x 2 1.73 / 1.92; 6 x 5 0.857 / 0.961; 4 x 8 0.789 / 0.901; 4 x 6 0.766 / 0.861;
// 3 x 8 0.722 / 0.814; 2 x 8 0.802 / 0.771; 2 x 12 0.656 / 0.780.  R-MAT 2^22 avg degree 32 BF16
// N = 256: 2 x 8 5.75, 2 x 12 5.90 (48-register gathers 6.00).  The warp's groups run one after
// another (wait, read, multiply, refill), so warps per SM matter more than rows in flight.
template <typename TB>
struct G4Shape {
  static constexpr int D = 2;
  static constexpr int W = std::is_same<TB, float>::value ? 12 : 8;
};

// cuTensorMapEncodeTiled of the driver, fetched once through the runtime (no link to libcuda);
// nullptr if the driver does not provide it.
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

template <typename TV, int D>
struct G4Layout {
  static constexpr int ROW = 512;                 // bytes of one packed row
  static constexpr int STAGE = 4 * ROW;           // one gather of four rows
  static constexpr int SEG = 256;                 // pairs of an item staged at a time
  static constexpr int PAIRS = SEG * (int)sizeof(Pair<TV>);
  static constexpr int BARS = 8 * D;
  // Per warp: the ring, the pairs, the barriers, rounded to 1 KB so every stage stays aligned.
  static constexpr int WARP = ((D * STAGE + PAIRS + BARS) + 1023) / 1024 * 1024;
};

__device__ __forceinline__ void g4_gather(uint32_t dst, const CUtensorMap* tm, int32_t r0,
                                          int32_t r1, int32_t r2, int32_t r3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
      : "memory");
}

// Per-warp pipeline state.  issued (lane 0 only) and consumed count gathers over the warp's
// lifetime: gather k uses stage k % D and completes phase k / D of that stage's barrier.
struct G4State {
  const char* ringp;  // the ring (generic address), for the lanes' reads
  uint32_t ring, bar0;
  uint32_t issued, consumed;
  bool ok;
};

// Lane 0: gather group g (pairs 4g .. 4g + 3 of the staged segment of n pairs; a short last group
// repeats its last row, whose copy is not read).
template <typename TV, int D>
__device__ __forceinline__ void g4_issue(const CUtensorMap* tm, const Pair<TV>* pairs, int g,
                                         int n, G4State& st) {
  using L = G4Layout<TV, D>;
  const int j = 4 * g;
  const int last = n - 1;
  const int32_t r0 = pairs[j].idx;
  const int32_t r1 = pairs[min(j + 1, last)].idx;
  const int32_t r2 = pairs[min(j + 2, last)].idx;
  const int32_t r3 = pairs[min(j + 3, last)].idx;
  const uint32_t s = st.issued % D;
  const uint32_t bar = st.bar0 + 8u * s;
  mbar_arrive_expect(bar, (uint32_t)L::STAGE);
  g4_gather(st.ring + s * (uint32_t)L::STAGE, tm, r0, r1, r2, r3, bar);
  ++st.issued;
}

// Nonzeros [base, base + total) of the item whose rows start at r0 (lane l: rel = end of row r0 + l
// relative to base if that row is non-empty, else 0), in segments of SEG staged pairs.
template <typename TV, typename TB, int VEC, int D>
__device__ __forceinline__ void g4_span(const SpmmParams<TV, TB>& p, const CUtensorMap* tm,
                                        Pair<TV>* pairs, G4State& st, int64_t base, int total,
                                        int32_t r0, int rel,
                                        typename AccOf<TB>::T (&acc)[1][VEC], int lane) {
  using L = G4Layout<TV, D>;
  using RF = RawFrag<TB, VEC>;
  static_assert(VEC * (int)sizeof(TB) == 16, "one 16-byte slice of a 512-byte row per lane");
  for (int seg = 0; seg < total && st.ok; seg += L::SEG) {
    const int n = min(L::SEG, total - seg);
    __syncwarp();
    for (int k = lane; k < n; k += 32) {
      Pair<TV> pr;
      pr.idx = __ldcs(p.remap + base + seg + k);
      pr.val = __ldcs(p.val + base + seg + k);
      pairs[k] = pr;
    }
    __syncwarp();
    const int ng = (n + 3) / 4;
    if (lane == 0) {
      // The stages were last read by the lanes (generic proxy) in the previous segment.
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      for (int g = 0; g < min(D, ng); ++g) g4_issue<TV, D>(tm, pairs, g, n, st);
    }
    for (int g = 0; g < ng; ++g) {
      const uint32_t s = st.consumed % D;
      // Warp-uniform verdict, so that no lane goes on alone.
      if (!__all_sync(0xffffffffu, mbar_wait(st.bar0 + 8u * s, (st.consumed / D) & 1u))) {
        st.ok = false;
        break;
      }
      ++st.consumed;
      // This lane's slices of the group's rows, then the FMAs in nonzero order.
      typename RF::T w[4][RF::W];
      const char* stage = st.ringp + s * L::STAGE;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint4 v = *reinterpret_cast<const uint4*>(stage + u * L::ROW + lane * 16);
        if constexpr (std::is_same<TB, float>::value) {
          w[u][0] = __uint_as_float(v.x); w[u][1] = __uint_as_float(v.y);
          w[u][2] = __uint_as_float(v.z); w[u][3] = __uint_as_float(v.w);
        } else {
          w[u][0] = v.x; w[u][1] = v.y; w[u][2] = v.z; w[u][3] = v.w;
        }
      }
      const int j0 = seg + 4 * g;  // item-relative position of the group's first nonzero
      // Rows that end inside this group (at most one per nonzero; warp-uniform).
      unsigned em = __ballot_sync(0xffffffffu, rel > j0 && rel <= j0 + 4);
      if (em == 0 && j0 + 4 <= total) {
#pragma unroll
        for (int u = 0; u < 4; ++u) fma_raw<TB, VEC>(pairs[4 * g + u].val, w[u], acc[0]);
      } else {
        int nl = em ? __ffs(em) - 1 : 0;
        int nend = em ? __shfl_sync(0xffffffffu, rel, nl) - 1 : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (j0 + u < total) {
            fma_raw<TB, VEC>(pairs[4 * g + u].val, w[u], acc[0]);
            if (j0 + u == nend) {
              flush_row<TV, TB, VEC, 1, false>(p, r0 + nl, acc, lane);
              em &= em - 1;
              nl = em ? __ffs(em) - 1 : 0;
              nend = em ? __shfl_sync(0xffffffffu, rel, nl) - 1 : -1;
            }
          }
        }
      }
      // Every lane has read the stage: lane 0 refills it with the gather D groups ahead (the
      // proxy fence orders the generic reads before the asynchronous write).
      __syncwarp();
      if (lane == 0 && g + D < ng) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        g4_issue<TV, D>(tm, pairs, g + D, n, st);
      }
    }
  }
}

// SMs x resident CTAs of W warps; every warp takes the next item from the plan's counter (zeroed
// before the launch), chunks of long rows first.
template <typename TV, typename TB, int VEC, int D, int W>
__global__ void __launch_bounds__(W * 32)
    k_spmm_g4(const SpmmParams<TV, TB> p, const __grid_constant__ CUtensorMap tmap) {
  using L = G4Layout<TV, D>;
  using TA = typename AccOf<TB>::T;
  extern __shared__ __align__(1024) char g4_smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  char* wsm = g4_smem + warp * L::WARP;
  Pair<TV>* pairs = reinterpret_cast<Pair<TV>*>(wsm + D * L::STAGE);
  G4State st;
  st.ringp = wsm;
  st.ring = (uint32_t)__cvta_generic_to_shared(wsm);
  st.bar0 = (uint32_t)__cvta_generic_to_shared(wsm + D * L::STAGE + L::PAIRS);
  st.issued = st.consumed = 0;
  st.ok = true;
  // A tensor copy needs a 128-byte aligned destination: never issue one otherwise.
  if (st.ring % 128u != 0u) {
    if (lane == 0) atomicOr(p.status, ST_OVERFLOW);
    return;
  }
  if (lane == 0) {
    for (int s = 0; s < D; ++s) mbar_init(st.bar0 + 8u * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  const int n_items = (int)p.n_items, n_chunks = (int)p.n_chunk_items;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(p.work, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= n_items) break;
    const Item item = p.items[it];
    TA acc[1][VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[0][v] = 0;
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
          flush_row<TV, TB, VEC, 1, false>(p, r0 + l, acc, lane);
        }
      }
      rel = nonempty ? rel : 0;
    }
    g4_span<TV, TB, VEC, D>(p, &tmap, pairs, st, item.e0, total, r0, rel, acc, lane);
    if (!st.ok) break;
    if (it < n_chunks) finish_chunk<TV, TB, VEC, 1, false>(p, -item.tag - 1, acc, lane);
  }
  if (!st.ok) {
    // A phase did not complete in time: report it, then wait (bounded) for the gathers still in
    // flight so that none lands after the warp has gone.
    if (lane == 0) atomicOr(p.status, ST_TIMEOUT);
    const uint32_t issued = __shfl_sync(0xffffffffu, st.issued, 0);
    for (uint32_t k = st.consumed; k < issued; ++k)
      mbar_wait(st.bar0 + 8u * (k % D), (k / D) & 1u);
  }
}

}  // namespace shiro
