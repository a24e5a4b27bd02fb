// sddmm.cu -- gradient of C = A B with respect to A's stored values, dA[e] = <dC[row e], B[col e]>
// (a sampled dense-dense product on A's pattern, reading B through the packed rows), and the
// backward entry point that adds dB = A^T dC through the transposed plan.
//
// One warp per work item (the SpMM schedule).  BF16 rows of 256 or 512 bytes and FP32 rows of 256
// or 512 bytes take the 48-register kernels of sddmm_lean.cuh.  The kernel here takes the other shapes,
// persistent mode and pipeline 5: a batch of up to 32
// nonzeros is taken as four sub-batches of 8, every lane forms its slice of the 8 dot products, a
// butterfly reduction (4+2+1 shuffles, then 2) completes them, and one more shuffle hands nonzero
// j of the batch to lane j, which writes dA coalesced once per batch.
#include <algorithm>

#include "internal.cuh"
#include "vec.cuh"

namespace shiro {

constexpr unsigned FULLM = 0xffffffffu;

template <typename TB>
struct SddmmParams {
  using TA = typename AccOf<TB>::T;
  const int64_t* rowptr;
  const int32_t* remap;
  const TB* dC;
  int64_t lddc;
  const TB* Bpack;
  int64_t ldp;
  const TB* B;
  int64_t ldb;
  int32_t N;
  TA* dA;
  const Item* items;
  int64_t n_items;
  int32_t chunk;
  int32_t persistent;
  int32_t* work;  // item counter of the persistent 48-register kernels (zeroed before launch)
};

template <typename TB, int VEC, int NCH, bool MASKED>
__device__ __forceinline__ void load_frag(const TB* row, int32_t N, int lane,
                                          typename AccOf<TB>::T (&f)[NCH][VEC]) {
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    const int col = c * 32 * VEC + lane * VEC;
    if (!MASKED || col < N) {
      load_vec<TB, VEC, true>(row + col, f[c]);
    } else {
#pragma unroll
      for (int v = 0; v < VEC; ++v) f[c][v] = 0;
    }
  }
}

// Dot products of 8 nonzeros, lane slices in part[0..7], summed over the warp: a butterfly over
// lane bits 4, 3, 2 (4 + 2 + 1 shuffles) leaves nonzero (lane >> 2) in every lane, and two more
// exchanges (lane bits 1, 0) complete its sum.  Eight partials per lane instead of 32.
template <typename TA>
__device__ __forceinline__ TA reduce8(TA (&part)[8], int lane) {
#pragma unroll
  for (int off = 16, half = 4; off >= 4; off >>= 1, half >>= 1) {
    const bool upper = lane & off;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const TA send = upper ? part[k] : part[k + half];
      const TA keep = upper ? part[k + half] : part[k];
      part[k] = keep + __shfl_xor_sync(FULLM, send, off);
    }
  }
  TA r = part[0];
  r += __shfl_xor_sync(FULLM, r, 2);
  r += __shfl_xor_sync(FULLM, r, 1);
  return r;
}

// Row of the stream position `pos` (relative to the item start) and the next non-empty row after
// it: lane l < nr holds the end of row r0 + l in `rel`.
__device__ __forceinline__ int next_nonempty_row(int rel, bool nonempty, int nr, int pos,
                                                 int lane) {
  const unsigned m = __ballot_sync(FULLM, lane < nr && nonempty && rel > pos);
  return m ? __ffs(m) - 1 : -1;
}

// One batch of up to 32 staged nonzeros as four sub-batches of 8; returns, in lane l, the dot
// product of nonzero l of the batch.  cur / nxt and g / gn track the current and the next
// non-empty row and their dC slices across row ends.
template <typename TB, int VEC, int NCH, bool MASKED, int U, bool FULL, bool ENDS>
__device__ __forceinline__ typename AccOf<TB>::T sddmm_batch(
    const SddmmParams<TB>& p, const int32_t* s_idx, int n, unsigned endmask, int32_t r0, int nr,
    int rel, bool nonempty, int& cur, int& nxt, typename AccOf<TB>::T (&g)[NCH][VEC],
    typename AccOf<TB>::T (&gn)[NCH][VEC], int lane) {
  using TA = typename AccOf<TB>::T;
  static_assert(8 % U == 0, "U must divide the 8-nonzero sub-batch");
  TA out = 0;
#pragma unroll 1
  for (int sb = 0; sb < (FULL ? 32 : n); sb += 8) {
    TA part[8];
#pragma unroll
    for (int j = 0; j < 8; j += U) {
      TA b[U][NCH][VEC];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (FULL || sb + j + u < n) {
          const int32_t idx = s_idx[sb + j + u];
          const TB* row = idx >= 0 ? p.Bpack + (uint64_t)(uint32_t)idx * (uint32_t)p.ldp
                                   : p.B + (uint64_t)(uint32_t)(-1 - idx) * (uint32_t)p.ldb;
          load_frag<TB, VEC, NCH, MASKED>(row, p.N, lane, b[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        TA s = 0;
        if (FULL || sb + j + u < n) {
#pragma unroll
          for (int c = 0; c < NCH; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) s = fma(g[c][v], b[u][c][v], s);
          if (ENDS && ((endmask >> (sb + j + u)) & 1u)) {
            // The stream leaves row r0 + cur here: move to the prefetched next row.
            cur = nxt;
            if (cur >= 0) {
#pragma unroll
              for (int c = 0; c < NCH; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) g[c][v] = gn[c][v];
              nxt = next_nonempty_row(rel, nonempty, nr, __shfl_sync(FULLM, rel, cur), lane);
              if (nxt >= 0)
                load_frag<TB, VEC, NCH, MASKED>(p.dC + (int64_t)(r0 + nxt) * p.lddc, p.N, lane,
                                                gn);
            }
          }
        }
        part[j + u] = s;
      }
    }
    const TA r = reduce8<TA>(part, lane);
    const TA v = __shfl_sync(FULLM, r, (lane & 7) << 2);
    if ((lane >> 3) == (sb >> 3)) out = v;
  }
  return out;
}

template <typename TB, int VEC, int NCH, bool MASKED, int U>
__device__ __forceinline__ void sddmm_item(const SddmmParams<TB>& p, int32_t* s_idx,
                                           const Item& item, int lane) {
  using TA = typename AccOf<TB>::T;
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
  // dC slice of the current row and, one row ahead, of the next non-empty row.
  int cur = next_nonempty_row(rel, nonempty, nr, 0, lane);
  if (cur < 0) return;
  int nxt = next_nonempty_row(rel, nonempty, nr, __shfl_sync(FULLM, rel, cur), lane);
  TA g[NCH][VEC], gn[NCH][VEC];
  load_frag<TB, VEC, NCH, MASKED>(p.dC + (int64_t)(r0 + cur) * p.lddc, p.N, lane, g);
  if (nxt >= 0) load_frag<TB, VEC, NCH, MASKED>(p.dC + (int64_t)(r0 + nxt) * p.lddc, p.N, lane, gn);
  int32_t nidx = lane < total ? __ldcs(p.remap + item.e0 + lane) : 0;
  for (int off = 0; off < total; off += 32) {
    const int n = min(32, total - off);
    __syncwarp();
    s_idx[lane] = nidx;
    __syncwarp();
    if (off + 32 + lane < total) nidx = __ldcs(p.remap + item.e0 + off + 32 + lane);
    const int q = rel - 1 - off;
    const unsigned bit = (lane < nr && nonempty && q >= 0 && q < 32) ? (1u << q) : 0u;
    const unsigned endmask = __reduce_or_sync(FULLM, bit);
    // Full batches with no row end inside take a copy of the loop without per-nonzero tests.
    const TA out = (n == 32 && endmask == 0)
        ? sddmm_batch<TB, VEC, NCH, MASKED, U, true, false>(p, s_idx, n, endmask, r0, nr, rel,
                                                            nonempty, cur, nxt, g, gn, lane)
        : sddmm_batch<TB, VEC, NCH, MASKED, U, false, true>(p, s_idx, n, endmask, r0, nr, rel,
                                                            nonempty, cur, nxt, g, gn, lane);
    if (lane < n) p.dA[item.e0 + off + lane] = out;
  }
}

template <int VEC, int NCH, typename TB>
struct SddmmOcc {
  static constexpr int REG = VEC * NCH * (int)(sizeof(typename AccOf<TB>::T) / 4);
#ifdef SHIRO_SDDMM_U
  static constexpr int U = REG >= 16 ? 2 : SHIRO_SDDMM_U;
#else
  static constexpr int U = REG >= 16 ? 2 : 4;
#endif
  // 64 registers (32 warps per SM) measured faster than 80, despite a few spilled bytes.
#ifdef SHIRO_SDDMM_MIN_BLOCKS
  static constexpr int MIN_BLOCKS = REG <= 4 ? SHIRO_SDDMM_MIN_BLOCKS : 2;
#else
  static constexpr int MIN_BLOCKS = REG <= 4 ? 4 : 2;
#endif
};

template <typename TB, int VEC, int NCH, bool MASKED, int U>
__global__ void __launch_bounds__(256, (SddmmOcc<VEC, NCH, TB>::MIN_BLOCKS))
    k_sddmm(const SddmmParams<TB> p) {
  __shared__ int32_t s_idx[8][32];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  int64_t it = (int64_t)blockIdx.x * wpb + warp;
  const int64_t step = p.persistent ? (int64_t)gridDim.x * wpb : p.n_items;
  for (; it < p.n_items; it += step) {
    const Item item = p.items[it];
    sddmm_item<TB, VEC, NCH, MASKED, U>(p, s_idx[warp], item, lane);
  }
}

}  // namespace shiro

#include "sddmm_lean.cuh"
#include "sddmm_group.cuh"

namespace shiro {

template <typename TB, int VEC, int NCH, bool MASKED>
static shiro_status sddmm_launch(const shiro_plan_s* P, const SddmmParams<TB>& prm,
                                 cudaStream_t s) {
  // Lane groups (sddmm_group.cuh), the default for FP32 / BF16 rows of 128, 256 or 512 bytes with
  // 16-byte aligned rows, outside persistent mode: eight lanes per nonzero, four nonzeros per warp
  // step, items from a counter in the plan.
  if constexpr (!MASKED && NCH == 1 && !std::is_same<TB, double>::value) {
    constexpr int RB = 32 * VEC * (int)sizeof(TB);
    if constexpr (RB == 128 || RB == 256 || RB == 512) {
      auto al16 = [](const void* ptr, int64_t ld) {
        return ((uintptr_t)ptr % 16) == 0 && ((uint64_t)ld * sizeof(TB)) % 16 == 0;
      };
      const bool ok16 = al16(prm.Bpack, prm.ldp) && al16(prm.dC, prm.lddc) &&
                        (!(P->flags & SHIRO_PLAN_LOCAL_DIAG) || al16(prm.B, prm.ldb));
      if (!prm.persistent && P->opts.pipeline == 0 && ok16) {
        if (prm.n_items > INT32_MAX) SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "too many work items");
        int per_sm = 0;
        SHIRO_CUDA(blocks_per_sm(&per_sm, k_sddmm_grp<TB, RB / 128>, 64, 0));
        const int64_t grid = std::min<int64_t>((prm.n_items + 1) / 2,
                                               (int64_t)std::max(per_sm, 1) * P->sm_count);
        if (grid <= 0) return SHIRO_OK;
        SddmmParams<TB> q = prm;
        q.work = P->d_status + 2;
        SHIRO_CUDA(cudaMemsetAsync(q.work, 0, sizeof(int32_t), s));
        k_sddmm_grp<TB, RB / 128><<<(unsigned)grid, 64, 0, s>>>(q);
        SHIRO_CUDA(cudaGetLastError());
        return SHIRO_OK;
      }
    }
  }
  // 48-register kernels outside persistent mode and pipeline 5: BF16 rows of 256 or 512 bytes and
  // FP32 rows of 256 bytes (N = 64) with the shared-memory tile reduction, FP32 rows of 512 bytes
  // (N = 128) with the 4-wide shuffle butterfly (the tile with pipeline 6).  Measured on R-MAT
  // 2^20, 4x4 tiles, with items from a counter (ms; 64-register kernel -> tile / butterfly):
  // BF16 N = 256 1.81 -> 1.02 / 1.02, BF16 N = 128 0.92 -> 0.82 / 0.82, FP32 N = 128
  // 0.93 -> 0.82 / 0.75 (the tile competes with the gathers for L1 bandwidth), FP32 N = 64
  // 0.78 -> 0.72 / 0.78.
  if constexpr (!MASKED && NCH == 1 && !std::is_same<TB, double>::value &&
                VEC * sizeof(TB) >= 8) {
    constexpr bool BF = std::is_same<TB, __nv_bfloat16>::value;
    // Pipeline 3 (or 0 when the rows are not 16-byte aligned) takes the butterfly for FP32 rows
    // of 512 bytes; pipeline 6 and the other rows take the tile.
    const bool tile = BF || VEC == 2 || P->opts.pipeline == 6;
    const bool shfl = !BF && VEC == 4 && P->opts.pipeline != 6;  // FP32 N = 128 rows
    if (!prm.persistent && P->opts.pipeline != 5 && (tile || shfl)) {  // pipelines 0, 3, 6
      int64_t grid = (prm.n_items + 1) / 2;
      if (grid <= 0) return SHIRO_OK;
      if (grid > INT32_MAX || prm.n_items > INT32_MAX)
        SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "too many work items");
      // SMs x resident blocks; the warps take items from a counter in the plan (measured against
      // one item per warp, ms: FP32 N = 128 0.92 -> 0.75, BF16 N = 256 1.21 -> 1.02, BF16
      // N = 128 0.88 -> 0.82, FP32 N = 64 with the tile 0.79 -> 0.72).
      SddmmParams<TB> q = prm;
      int per_sm = 0;
      if (tile)
        SHIRO_CUDA(blocks_per_sm(&per_sm, k_sddmm_lean<TB, VEC, true>, 64, 0));
      else
        SHIRO_CUDA(blocks_per_sm(&per_sm, k_sddmm_lean<TB, VEC, (BF || VEC != 4)>, 64, 0));
      grid = std::min<int64_t>(grid, (int64_t)std::max(per_sm, 1) * P->sm_count);
      q.work = P->d_status + 2;
      SHIRO_CUDA(cudaMemsetAsync(q.work, 0, sizeof(int32_t), s));
      if (tile)
        k_sddmm_lean<TB, VEC, true><<<(unsigned)grid, 64, 0, s>>>(q);
      else if constexpr (!BF && VEC == 4)
        k_sddmm_lean<TB, VEC, false><<<(unsigned)grid, 64, 0, s>>>(q);
      SHIRO_CUDA(cudaGetLastError());
      return SHIRO_OK;
    }
  }
  constexpr int U = SddmmOcc<VEC, NCH, TB>::U;
  const int wpc = std::min(P->opts.warps_per_cta, 8);
  int64_t grid = (prm.n_items + wpc - 1) / wpc;
  if (prm.persistent) grid = std::min<int64_t>(grid, (int64_t)P->sm_count * 8);
  if (grid <= 0) return SHIRO_OK;
  k_sddmm<TB, VEC, NCH, MASKED, U><<<(unsigned)grid, wpc * 32, 0, s>>>(prm);
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

static bool al(const void* ptr, int64_t ld, size_t elem, int vec) {
  const size_t a = std::min<size_t>(16, elem * (size_t)vec);
  return ((uintptr_t)ptr % a) == 0 && ((size_t)ld * elem) % a == 0;
}

template <typename TB>
static shiro_status sddmm_typed(const shiro_plan_s* P, const void* dC, int64_t lddc,
                                const void* Bpack, int64_t ldp, const void* B, int64_t ldb,
                                int32_t N, void* dA, cudaStream_t s) {
  SddmmParams<TB> prm{};
  prm.rowptr = P->rowptr;
  prm.remap = P->d_remap;
  prm.dC = (const TB*)dC;
  prm.lddc = lddc;
  prm.Bpack = (const TB*)Bpack;
  prm.ldp = ldp;
  prm.B = (const TB*)B;
  prm.ldb = ldb;
  prm.N = N;
  prm.dA = (typename AccOf<TB>::T*)dA;
  prm.items = P->d_items;
  prm.n_items = P->n_items;
  prm.chunk = P->opts.chunk_nnz;
  prm.persistent = P->opts.persistent;
  const size_t esz = sizeof(TB);
  const bool local = P->flags & SHIRO_PLAN_LOCAL_DIAG;
  auto ok = [&](int vec) {
    bool r = al(Bpack, ldp, esz, vec) && al(dC, lddc, esz, vec);
    if (local) r = r && al(B, ldb, esz, vec);
    return r;
  };
#define SHIRO_SD(VEC, NCH, MASKED) return sddmm_launch<TB, VEC, NCH, MASKED>(P, prm, s);
  if constexpr (std::is_same<TB, float>::value) {
    if (N == 128 && ok(4)) SHIRO_SD(4, 1, false)
    if (N == 256 && ok(4)) SHIRO_SD(4, 2, false)
    if (N == 64 && ok(2)) SHIRO_SD(2, 1, false)
  } else if constexpr (std::is_same<TB, double>::value) {
    if (N == 64 && ok(2)) SHIRO_SD(2, 1, false)
    if (N == 128 && ok(2)) SHIRO_SD(2, 2, false)
  } else {
    if (N == 256 && ok(8)) SHIRO_SD(8, 1, false)
    if (N == 128 && ok(4)) SHIRO_SD(4, 1, false)
    if (N == 64 && ok(2)) SHIRO_SD(2, 1, false)
  }
  if (N == 32) SHIRO_SD(1, 1, false)
  if (N <= 32) SHIRO_SD(1, 1, true)
  if (N <= 128) SHIRO_SD(1, 4, true)
  if (N <= 512) SHIRO_SD(1, 16, true)
#undef SHIRO_SD
  SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "N=%d beyond the supported 512 columns", N);
}

shiro_status launch_sddmm(const shiro_plan_s* P, const void* dC, int64_t lddc, const void* Bpack,
                          int64_t ldp, const void* B, int64_t ldb, int32_t N, shiro_dtype dt,
                          void* dA, cudaStream_t s) {
  if (N < 0 || lddc < N || ldp < N) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "bad N or leading dimension");
  // The gathers multiply a 32-bit row index by a 32-bit row stride.
  if (ldp > (int64_t)UINT32_MAX || ldb > (int64_t)UINT32_MAX)
    SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "leading dimensions of B / Bpack above 2^32 - 1 elements");
  if (P->nnz == 0) return SHIRO_OK;
  if (!dA || !dC) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null dA or dC");
  if (!Bpack && P->packed_rows > 0) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null Bpack");
  if ((P->flags & SHIRO_PLAN_LOCAL_DIAG) && (!B || ldb < N))
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "LOCAL_DIAG plan needs B with ldb >= N");
  if (N == 0) {
    const size_t vs = P->vdt == SHIRO_F64 ? 8 : 4;
    SHIRO_CUDA(cudaMemsetAsync(dA, 0, vs * (size_t)P->nnz, s));
    return SHIRO_OK;
  }
  if (P->vdt == SHIRO_F32 && dt == SHIRO_F32)
    return sddmm_typed<float>(P, dC, lddc, Bpack, ldp, B, ldb, N, dA, s);
  if (P->vdt == SHIRO_F32 && dt == SHIRO_BF16)
    return sddmm_typed<__nv_bfloat16>(P, dC, lddc, Bpack, ldp, B, ldb, N, dA, s);
  if (P->vdt == SHIRO_F64 && dt == SHIRO_F64)
    return sddmm_typed<double>(P, dC, lddc, Bpack, ldp, B, ldb, N, dA, s);
  SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "value/operand dtypes: F32 with F32 or BF16, or F64 with F64");
}

}  // namespace shiro

using namespace shiro;

extern "C" {

shiro_status shiro_sddmm(shiro_plan_t plan, const void* dC, int64_t lddc, const void* Bpack,
                         int64_t ldp, const void* B, int64_t ldb, int32_t N, shiro_dtype dt,
                         void* dA, void* stream) {
  if (!plan) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  return launch_sddmm(plan, dC, lddc, Bpack, ldp, B, ldb, N, dt, dA, (cudaStream_t)stream);
}

shiro_status shiro_spmm_backward(shiro_plan_t plan, shiro_plan_t planT, const void* dC,
                                 int64_t lddc, const void* Bpack, int64_t ldp, const void* B,
                                 int64_t ldb, int32_t N, shiro_dtype dt, void* dCpack,
                                 int64_t lddp, void* dB, int64_t lddb, void* dA, void* scratch,
                                 size_t scratch_bytes, void* stream) {
  if (!plan) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  cudaStream_t s = (cudaStream_t)stream;
  if (dB) {
    if (!planT || !(planT->flags & SHIRO_PLAN_TRANSPOSE))
      SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "dB needs the TRANSPOSE plan of the same matrix");
    if (planT->M != plan->K || planT->K != plan->M || planT->nnz != plan->nnz)
      SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "planT is not the transpose of plan");
    if (dA) {
      bool done = false;
      SHIRO_TRY(launch_backward_one(plan, planT, dC, lddc, B, ldb, N, dt, dCpack, lddp, dB, lddb,
                                    dA, scratch, scratch_bytes, s, &done));
      if (done) return SHIRO_OK;
    }
    SHIRO_TRY(launch_pack_spmm(planT, dC, lddc, N, dt, dCpack, lddp, dB, lddb, 0, scratch,
                               scratch_bytes, s));
  }
  if (dA) SHIRO_TRY(launch_sddmm(plan, dC, lddc, Bpack, ldp, B, ldb, N, dt, dA, s));
  return SHIRO_OK;
}

}  // extern "C"
