// spmm_bwd.cuh -- the backward of C = A B in one launch over the TRANSPOSE plan of A (rows of 256
// or 512 bytes):
//   * the pack of dC's rows named by the plan (dCpack[r] = dC[pack_src[r]], Sec. 5.1 stage 3);
//   * dB = A^T dC over the packed rows (the transposed SpMM, Sec. 5.1 stage 5);
//   * dA on A's pattern, dA[e] = <dC[row e, :], B[col e, :]>, from the same gathered dC rows.
// A row j of A^T lists the nonzeros of column j of A; for each of them the warp gathers the dC row
// of the nonzero's row for dB, and that row's dot product with B[j, :] is the nonzero's dA.  B[j]
// is one row per row of A^T (read once, not gathered per nonzero), so the SDDMM's gather of a B
// row per nonzero disappears: the backward makes one pass of row gathers instead of two.
// Work order, pack chunks, the per-block waits and the dB sums are those of k_spmm_lean_fused on
// the same plan, so dB is bit-identical to shiro_pack_spmm on it; dA is summed in its own fixed
// order (two partial sums per lane over the lane's slice, then a tree over the 32 lanes).
#pragma once

#include "spmm_lean.cuh"

namespace shiro {

template <typename TB>
struct SdParams {
  const TB* B;          // the forward operand B, K x N (its rows are the rows of A^T)
  uint32_t ldb;
  float* dA;            // nnz values in A's nonzero order
  const int64_t* perm;  // nonzero e' of A^T -> nonzero of A
};

#ifndef SHIRO_BWD_MINB
// 2-warp CTAs per SM.  Backward ms (R-MAT 2^20, FP32 N = 128 / BF16 N = 256 degree 32) at 16
// (64 registers) 1.178 / 2.472, 18 (56) 1.132 / 2.475, 20 (48, 80-100 bytes spilled) 1.171 /
// 2.523.
#define SHIRO_BWD_MINB 18
#endif

// Measured on R-MAT 2^20 (4x4 tiles), backward ms FP32 N = 128 / BF16 N = 256 (degree 32), with
// (hint, group prefetch) = (0, 1) 1.138 / 2.470, (1, 1) 1.128 / 2.472, (1, 0) 1.125 / 2.480,
// (0, 0) 1.130 / 2.481: all within noise.  Tried and slower: a register copy of the next row's B
// row loaded a row ahead (1.18 / 2.53: spills), and dA written in A^T's order with a separate
// scatter pass to A's order (1.18 / 2.68).
#ifndef SHIRO_BWD_HINT
#define SHIRO_BWD_HINT 1  // evict-first L2 policy on the streamed pattern, nonzero ids and B rows
#endif
#ifndef SHIRO_BWD_GROUP_PF
#define SHIRO_BWD_GROUP_PF 1  // a group's B rows brought into L2 when the group starts
#endif

__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}

// cp.async of BYTES (4 or 8) with an L2 cache policy.
template <int BYTES>
__device__ __forceinline__ void cp_async_hint(uint32_t smem, const void* gmem, uint64_t pol) {
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %3;\n" ::"r"(smem),
               "l"(gmem), "n"(BYTES), "l"(pol)
               : "memory");
}

// The lane's 16- or 8-byte slice of a B row as floats.  B's rows are read once per row of A^T (a
// long row's chunks read it again, mostly from L2); with SHIRO_BWD_HINT the read carries an
// evict-first L2 policy so that it displaces fewer of the gathered dC rows.
template <typename TB, int VEC>
__device__ __forceinline__ void load_b_row(const TB* p, float (&f)[VEC]) {
  constexpr int WORDS = VEC * (int)sizeof(TB) / 4;
  static_assert(WORDS == 4 || WORDS == 2, "16- or 8-byte slices");
  if constexpr (SHIRO_BWD_HINT) {
    uint32_t w[WORDS];
    if constexpr (WORDS == 4)
      asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;\n"
                   : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                   : "l"(p), "l"(evict_first_policy()));
    else
      asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;\n"
                   : "=r"(w[0]), "=r"(w[1])
                   : "l"(p), "l"(evict_first_policy()));
    if constexpr (std::is_same<TB, float>::value) {
#pragma unroll
      for (int v = 0; v < WORDS; ++v) f[v] = __uint_as_float(w[v]);
    } else {
#pragma unroll
      for (int k = 0; k < WORDS; ++k) {
        f[2 * k] = bf16_lo(w[k]);
        f[2 * k + 1] = bf16_hi(w[k]);
      }
    }
  } else {
    load_vec<TB, VEC, true>(p, f);
  }
}

// Sum over the lane's VEC elements of dC * B: two partial sums (even and odd elements, paired
// FMAs), added at the end.
template <typename TB, int VEC>
__device__ __forceinline__ float dot_raw(const typename RawFrag<TB, VEC>::T (&w)[RawFrag<TB, VEC>::W],
                                         const float (&bj)[VEC]) {
  if constexpr (VEC >= 2) {
    float2 d = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < VEC / 2; ++k) {
      float2 x;
      if constexpr (std::is_same<TB, __nv_bfloat16>::value)
        x = make_float2(bf16_lo(w[k]), bf16_hi(w[k]));
      else
        x = make_float2(w[2 * k], w[2 * k + 1]);
      d = __ffma2_rn(x, make_float2(bj[2 * k], bj[2 * k + 1]), d);
    }
    return d.x + d.y;
  } else if constexpr (std::is_same<TB, __nv_bfloat16>::value) {
    return bf16_lo(w[0]) * bj[0];
  } else {
    return w[0] * bj[0];
  }
}

// Warp sums of U values per lane, scattered: lane l ends with the sum over all 32 lanes of
// d[l / (32 / U)].  The first rounds halve the values each lane carries (a lane keeps the half
// its partner sends away), the last ones are plain butterflies: 6 shuffles for U = 4 where four
// separate butterflies take 20.
template <int U>
__device__ __forceinline__ float reduce_scatter(const float (&d)[U], int lane) {
  static_assert(U == 1 || U == 2 || U == 4, "U of 1, 2 or 4");
  float k;
  int first;
  if constexpr (U == 4) {
    const bool hi = lane & 16;
    float k0 = hi ? d[2] : d[0], k1 = hi ? d[3] : d[1];
    const float s0 = hi ? d[0] : d[2], s1 = hi ? d[1] : d[3];
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    const bool h8 = lane & 8;
    k = h8 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
    first = 4;
  } else if constexpr (U == 2) {
    const bool hi = lane & 16;
    k = hi ? d[1] : d[0];
    k += __shfl_xor_sync(0xffffffffu, hi ? d[0] : d[1], 16);
    first = 8;
  } else {
    k = d[0];
    first = 16;
  }
#pragma unroll
  for (int o = first; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  return k;
}

// One batch of up to 32 nonzeros (pairs in sp, A's nonzero ids in spm): the dB accumulation of
// lean_batch plus every nonzero's dA.  bj holds B's row for the row of the current nonzero; at a
// row end the next non-empty row's B row replaces it.
template <typename TV, typename TB, int VEC, int U, bool LOCAL, bool FULL, bool ENDS>
__device__ __forceinline__ void bwd_batch(const SpmmParams<TV, TB>& p, const SdParams<TB>& sd,
                                          const Bases<TB>& bs, const Pair<TV>* sp,
                                          const int64_t* spm, int n, int off, int32_t r0, int rel,
                                          unsigned endmask, float (&acc)[1][VEC],
                                          float (&bj)[VEC], int lane) {
  constexpr int G = 32 / U;  // lanes that end with one nonzero's dA
#pragma unroll 1
  for (int j = 0; j < (FULL ? 32 : n); j += U) {
    typename RawFrag<TB, VEC>::T b[U][1][RawFrag<TB, VEC>::W];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (FULL || j + u < n) {
        const int32_t idx = sp[j + u].idx;
        const TB* row;
        if (LOCAL && idx < 0)
          row = bs.b + (uint64_t)(uint32_t)(-1 - idx) * bs.ldb;
        else
          row = bs.bp + (uint64_t)(uint32_t)idx * bs.ldp;
        load_raw_cg<TB, VEC>(row, b[u][0]);  // packed rows written earlier in this launch
      }
    }
    constexpr bool PF = SHIRO_LEAN_PF && VEC * sizeof(TB) >= 16 && U <= 2;
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
    float d[U];
    const unsigned em = ENDS ? (endmask >> j) & ((1u << U) - 1u) : 0u;
    if (em == 0) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        d[u] = 0.f;
        if (FULL || j + u < n) {
          fma_raw<TB, VEC>(sp[j + u].val, b[u][0], acc[0]);
          d[u] = dot_raw<TB, VEC>(b[u][0], bj);
        }
      }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        d[u] = 0.f;
        if (FULL || j + u < n) {
          fma_raw<TB, VEC>(sp[j + u].val, b[u][0], acc[0]);
          d[u] = dot_raw<TB, VEC>(b[u][0], bj);
          if ((em >> u) & 1u) {
            const int pos = off + j + u + 1;
            const unsigned who = __ballot_sync(0xffffffffu, rel == pos);
            flush_row<TV, TB, VEC, 1, false>(p, r0 + __ffs(who) - 1, acc, lane);
            // The next nonzero's row: the first lane whose row ends beyond this position.
            const unsigned nx = __ballot_sync(0xffffffffu, rel > pos);
            if (nx)
              load_b_row<TB, VEC>(sd.B + (uint64_t)(uint32_t)(r0 + __ffs(nx) - 1) * sd.ldb +
                                      lane * VEC, bj);
          }
        }
      }
    }
    const float t = reduce_scatter<U>(d, lane);
    const int u = lane / G;
    if ((lane & (G - 1)) == 0 && (FULL || j + u < n)) sd.dA[spm[j + u]] = t;
  }
}

// Nonzeros [base, base + total) of rows r0 .. (rel as in lean_span), pairs and A's nonzero ids of
// two batches in sp / spm.
template <typename TV, typename TB, int VEC, int U, bool LOCAL>
__device__ __forceinline__ void bwd_span(const SpmmParams<TV, TB>& p, const SdParams<TB>& sd,
                                         const Bases<TB>& bs, Pair<TV>* sp, int64_t* spm,
                                         int64_t base, int total, int32_t r0, int rel,
                                         float (&acc)[1][VEC], int lane) {
  if (total <= 0) return;
  // The row of the first nonzero: the first non-empty row of a group, or the chunk's row.
  const unsigned ne = __ballot_sync(0xffffffffu, rel > 0);
  const int32_t row = ne ? r0 + __ffs(ne) - 1 : r0;
  // The group's later rows are needed one after another: bring their B rows into L2 now.
  if (SHIRO_BWD_GROUP_PF && p.pf_bytes && rel > 0 && r0 + lane != row)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                     sd.B + (uint64_t)(uint32_t)(r0 + lane) * sd.ldb),
                 "r"(p.pf_bytes));
  float bj[VEC];
  load_b_row<TB, VEC>(sd.B + (uint64_t)(uint32_t)row * sd.ldb + lane * VEC, bj);
  __syncwarp();
  if (lane < total) {
    Pair<TV> pr;
    pr.idx = __ldcs(p.remap + base + lane);
    pr.val = __ldcs(p.val + base + lane);
    sp[lane] = pr;
    spm[lane] = __ldcs(sd.perm + base + lane);
  }
#pragma unroll 1
  for (int off = 0; off < total; off += 32) {
    const int h = (off >> 5) & 1;
    Pair<TV>* cur = sp + h * 32;
    Pair<TV>* nxt = sp + (h ^ 1) * 32;
    cp_async_wait<0>();
    __syncwarp();
    if (off + 32 + lane < total) {
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(nxt + lane);
      const uint32_t dm = (uint32_t)__cvta_generic_to_shared(spm + (h ^ 1) * 32 + lane);
      if constexpr (SHIRO_BWD_HINT) {
        // The pattern and the nonzero ids are read once.
        const uint64_t pol = evict_first_policy();
        cp_async_hint<4>(d, p.remap + base + off + 32 + lane, pol);
        cp_async_hint<(int)sizeof(TV)>(d + (uint32_t)offsetof(Pair<TV>, val),
                                       p.val + base + off + 32 + lane, pol);
        cp_async_hint<8>(dm, sd.perm + base + off + 32 + lane, pol);
      } else {
        cp_async<4>(d, p.remap + base + off + 32 + lane);
        cp_async<(int)sizeof(TV)>(d + (uint32_t)offsetof(Pair<TV>, val),
                                  p.val + base + off + 32 + lane);
        cp_async<8>(dm, sd.perm + base + off + 32 + lane);
      }
    }
    cp_async_commit();
    const int n = min(32, total - off);
    const int q = rel - 1 - off;
    const unsigned endmask = __reduce_or_sync(0xffffffffu, (q >= 0 && q < 32) ? (1u << q) : 0u);
    if (n == 32 && endmask == 0)
      bwd_batch<TV, TB, VEC, U, LOCAL, true, false>(p, sd, bs, cur, spm + h * 32, n, off, r0, rel,
                                                    endmask, acc, bj, lane);
    else
      bwd_batch<TV, TB, VEC, U, LOCAL, false, true>(p, sd, bs, cur, spm + h * 32, n, off, r0, rel,
                                                    endmask, acc, bj, lane);
  }
  cp_async_wait<0>();
}

// One launch: the launch order, pack chunks and per-block waits of k_spmm_lean_fused (p and f
// describe the TRANSPOSE plan with dC as its B operand), plus dA through sd.
template <typename TV, typename TB, int VEC, int U, bool LOCAL>
__global__ void __launch_bounds__(64, SHIRO_BWD_MINB)
    k_spmm_lean_bwd(const SpmmParams<TV, TB> p, const FusedParams<TB> f, const SdParams<TB> sd) {
  __shared__ Pair<TV> s_pairs[2][64];
  __shared__ int64_t s_perm[2][64];
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
      if constexpr (SHIRO_FUSED_PACK_STAGED)
        fused_pack_chunk_staged<TV, TB, VEC, SHIRO_FUSED_PACK_U>(p, f, c, s_stage[warp], lane);
      else
        fused_pack_chunk<TV, TB, VEC, 1, SHIRO_FUSED_PACK_U>(p, f, c, lane);
      continue;
    }
    const Item item = p.items[code];
    const int32_t blk = row_block(f.geo, item.row);
    if (blk > known) {
      fused_wait_block<TB>(f, blk, p.status, lane);
      known = blk;
    }
    float acc[1][VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[0][v] = 0;
    const bool chunk = item.tag <= 0;
    const int32_t r0 = item.row;
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
          flush_row<TV, TB, VEC, 1, false>(p, r0 + l, acc, lane);
        }
      }
      rel = nonempty ? rel : 0;
    }
    bwd_span<TV, TB, VEC, U, LOCAL>(p, sd, bs, sp, s_perm[warp], item.e0, total, r0, rel, acc,
                                    lane);
    if (chunk) finish_chunk<TV, TB, VEC, 1, false>(p, -item.tag - 1, acc, lane);
  }
}

}  // namespace shiro
