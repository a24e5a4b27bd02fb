// sddmm_lean.cuh -- dA[e] = <dC[row e], B[col e]> with a 48-register budget, so that 40 warps fit
// on an SM (2-warp CTAs, 20 per SM) instead of 32; launched as SMs x 20 blocks whose warps take
// items from a counter.  Two ways to finish the dot products: a 4-wide shuffle butterfly per step
// of 4 nonzeros (four partial registers), or a shared-memory tile:
//
// Per batch of 32 nonzeros every lane forms its slice of each dot product (VEC products of its
// dC slice and the gathered B slice) and stores it into a 32 x 32 shared-memory tile, row = the
// nonzero, column = the lane, XOR-swizzled (column lane ^ row) so that neither the stores of one
// nonzero nor the reads of one row collide on a bank.  After the batch, lane j adds row j's 32
// partials in lane order 0, 1, ..., 31 and writes dA coalesced.  No partial-sum registers are
// held across the batch (the shuffle reduction needs 8), and the batch's indices arrive in shared
// memory by cp.async one batch ahead.  The dC slice of the next non-empty row is loaded one row
// ahead, as in the shuffle-reduction kernel.
#pragma once

#include "internal.cuh"
#include "vec.cuh"

namespace shiro {

constexpr int SD_LEAN_MIN_BLOCKS = 20;  // 2-warp CTAs per SM: 48 registers per thread

__device__ __forceinline__ void sd_cp4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void sd_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void sd_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// s += <g, raw fragment> in element order (BF16 widened exactly).
template <typename TB, int VEC>
__device__ __forceinline__ float dot_raw(const float (&g)[VEC],
                                         const typename RawFrag<TB, VEC>::T (&w)[RawFrag<TB, VEC>::W],
                                         float s) {
  if constexpr (!std::is_same<TB, __nv_bfloat16>::value) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) s = fmaf(g[v], w[v], s);
  } else if constexpr (VEC == 1) {
    s = fmaf(g[0], bf16_lo(w[0]), s);
  } else {
#pragma unroll
    for (int k = 0; k < VEC / 2; ++k) {
      s = fmaf(g[2 * k], bf16_lo(w[k]), s);
      s = fmaf(g[2 * k + 1], bf16_hi(w[k]), s);
    }
  }
  return s;
}

template <typename TB, int VEC>
struct SdLeanShape {
  // Rows in flight per step: 4, or 2 for BF16 rows of 512 bytes (8 elements per lane).
  static constexpr int U = (std::is_same<TB, __nv_bfloat16>::value && VEC == 8) ? 2 : 4;
};

// Dot products of 4 nonzeros, lane slices in part[0..3], summed over the warp: a butterfly over
// lane bits 4, 3 (2 + 1 shuffles) leaves nonzero (lane >> 3) & 3 in every lane, three exchanges
// over bits 2, 1, 0 complete its sum.  Four partials per lane.
__device__ __forceinline__ float reduce4(float (&part)[4], int lane) {
#pragma unroll
  for (int off = 16, half = 2; off >= 8; off >>= 1, half >>= 1) {
    const bool upper = lane & off;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float send = upper ? part[k] : part[k + half];
      const float keep = upper ? part[k + half] : part[k];
      part[k] = keep + __shfl_xor_sync(FULLM, send, off);
    }
  }
  float r = part[0];
  r += __shfl_xor_sync(FULLM, r, 4);
  r += __shfl_xor_sync(FULLM, r, 2);
  r += __shfl_xor_sync(FULLM, r, 1);
  return r;
}

// TILE: partials through the shared-memory tile (sred); else a 4-wide shuffle butterfly per
// step of 4 nonzeros (sred unused).
template <typename TB, int VEC, bool TILE>
__device__ __forceinline__ void sddmm_lean_item(const SddmmParams<TB>& p, int32_t* sidx,
                                                float* sred, const Item& item, int lane) {
  constexpr int U = TILE ? SdLeanShape<TB, VEC>::U : 4;
  const bool chunk = item.tag <= 0;
  const int32_t r0 = item.row;
  const int nr = chunk ? 1 : item.tag;
  const int64_t rp = lane < nr ? __ldg(p.rowptr + r0 + lane + 1) : 0;
  int rel = (int)(rp - item.e0);
  const int prev = __shfl_up_sync(FULLM, rel, 1);
  bool nonempty = lane < nr && rel > (lane ? prev : 0);
  int total = __shfl_sync(FULLM, rel, nr - 1);
  if (chunk) {
    total = min(total, p.chunk);
    rel = total;
    nonempty = lane == 0 && total > 0;
  }
  // Lane l's row state in one word: the end of row r0 + l (relative to e0), 0 if it ends nowhere.
  rel = nonempty ? rel : 0;
  if (total <= 0) return;
  const TB* dC = p.dC + lane * VEC;
  int cur = __ffs(__ballot_sync(FULLM, rel > 0)) - 1;
  const unsigned mn = __ballot_sync(FULLM, rel > __shfl_sync(FULLM, rel, cur));
  int nxt = mn ? __ffs(mn) - 1 : -1;
  float g[VEC], gn[VEC];
  load_vec<TB, VEC, true>(dC + (int64_t)(r0 + cur) * p.lddc, g);
  if (nxt >= 0) load_vec<TB, VEC, true>(dC + (int64_t)(r0 + nxt) * p.lddc, gn);
  __syncwarp();
  if (lane < total) sidx[lane] = __ldcs(p.remap + item.e0 + lane);
#pragma unroll 1
  for (int off = 0; off < total; off += 32) {
    const int h = (off >> 5) & 1;
    sd_wait_all();
    __syncwarp();
    if (off + 32 + lane < total)
      sd_cp4((uint32_t)__cvta_generic_to_shared(sidx + (h ^ 1) * 32 + lane),
             p.remap + item.e0 + off + 32 + lane);
    sd_commit();
    const int32_t* ci = sidx + h * 32;
    const int n = min(32, total - off);
    const int q = rel - 1 - off;
    const unsigned endmask = __reduce_or_sync(FULLM, (q >= 0 && q < 32) ? (1u << q) : 0u);
    float out = 0.f;
#pragma unroll 1
    for (int j = 0; j < n; j += U) {
      typename RawFrag<TB, VEC>::T b[U][RawFrag<TB, VEC>::W];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (j + u < n) {
          const int32_t idx = ci[j + u];
          const TB* row = idx >= 0 ? p.Bpack + (uint64_t)(uint32_t)idx * (uint32_t)p.ldp
                                   : p.B + (uint64_t)(uint32_t)(-1 - idx) * (uint32_t)p.ldb;
          load_raw<TB, VEC>(row + lane * VEC, b[u]);
        }
      }
      const unsigned em = (endmask >> j) & ((1u << U) - 1u);
      float part[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        part[u] = 0.f;
        if (j + u < n) {
          const int t = j + u;
          if constexpr (TILE)
            sred[t * 32 + (lane ^ t)] = dot_raw<TB, VEC>(g, b[u], 0.f);
          else
            part[u] = dot_raw<TB, VEC>(g, b[u], 0.f);
          if ((em >> u) & 1u) {
            // The stream leaves row r0 + cur here: move to the prefetched next row.
            cur = nxt;
            if (cur >= 0) {
#pragma unroll
              for (int v = 0; v < VEC; ++v) g[v] = gn[v];
              const unsigned m = __ballot_sync(FULLM, rel > __shfl_sync(FULLM, rel, cur));
              nxt = m ? __ffs(m) - 1 : -1;
              if (nxt >= 0) load_vec<TB, VEC, true>(dC + (int64_t)(r0 + nxt) * p.lddc, gn);
            }
          }
        }
      }
      if constexpr (!TILE) {
        // Lane t of the batch keeps nonzero t's sum (held by lanes with (lane >> 3) & 3 == t & 3).
        const float r = reduce4(reinterpret_cast<float(&)[4]>(part), lane);
        const float v = __shfl_sync(FULLM, r, (lane & 3) << 3);
        if ((lane >> 2) == (j >> 2)) out = v;
      }
    }
    if constexpr (!TILE) {
      if (lane < n) p.dA[item.e0 + off + lane] = out;
      continue;
    }
    __syncwarp();
    if (lane < n) {
      // Row `lane` of the tile: column c ^ lane holds lane c's partial.
      float t = 0.f;
#pragma unroll
      for (int c = 0; c < 32; ++c) t += sred[lane * 32 + (c ^ lane)];
      p.dA[item.e0 + off + lane] = t;
    }
    __syncwarp();
  }
  sd_wait_all();
}

template <typename TB, int VEC, bool TILE>
__global__ void __launch_bounds__(64, SD_LEAN_MIN_BLOCKS) k_sddmm_lean(const SddmmParams<TB> p) {
  __shared__ __align__(16) int32_t s_idx[2][64];
  __shared__ __align__(16) float s_red[TILE ? 2 : 1][TILE ? 32 * 32 : 1];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  if (!p.work) {
    const int64_t it = (int64_t)blockIdx.x * 2 + warp;
    if (it >= p.n_items) return;
    sddmm_lean_item<TB, VEC, TILE>(p, s_idx[warp], TILE ? s_red[warp] : nullptr, p.items[it],
                                   lane);
    return;
  }
  // Persistent form: every warp takes the next item from the counter until none is left.
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(p.work, 1);
    it = __shfl_sync(FULLM, it, 0);
    if ((int64_t)it >= p.n_items) break;
    sddmm_lean_item<TB, VEC, TILE>(p, s_idx[warp], TILE ? s_red[warp] : nullptr, p.items[it],
                                   lane);
  }
}

}  // namespace shiro
