// pack.cu -- gather of the B rows named by Cols(A^(p,q)) into the packed buffer (Sec. 5.1
// stage 3): Bpack[r, :] = B[pack_src[r], :], bit-exact for any element type.
//
// A pure HBM copy (2 * packed_rows * N * sz bytes).  Each thread moves one 4-16 byte word of a
// row per step and four rows per loop iteration, so a CTA keeps 4 * 256 * 16 bytes in flight;
// consecutive threads touch consecutive words of a row, so every warp access is contiguous.
#include <algorithm>

#include "internal.cuh"

namespace shiro {

template <typename W>
__global__ void __launch_bounds__(256) k_pack_rows(const int32_t* __restrict__ src,
                                                   int64_t nrows, const char* __restrict__ B,
                                                   int64_t ldb_bytes, char* __restrict__ Bp,
                                                   int64_t ldp_bytes, int32_t wpr) {
  // Thread t of the block handles word t % wpr of row (t / wpr) of each group of rows.
  const int32_t rows_per_iter = blockDim.x / wpr;
  const int32_t sub = threadIdx.x / wpr;
  const int32_t w = threadIdx.x - sub * wpr;
  if (sub >= rows_per_iter) return;
  const int64_t stride = (int64_t)gridDim.x * rows_per_iter;
  constexpr int R = 4;
  for (int64_t r = (int64_t)blockIdx.x * rows_per_iter + sub; r < nrows; r += R * stride) {
    W v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int64_t rr = r + k * stride;
      if (rr < nrows) {
        const int64_t s = __ldg(src + rr);
        v[k] = __ldg(reinterpret_cast<const W*>(B + s * ldb_bytes) + w);
      }
    }
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int64_t rr = r + k * stride;
      if (rr < nrows) reinterpret_cast<W*>(Bp + rr * ldp_bytes)[w] = v[k];
    }
  }
}

// Rows wider than a CTA: one CTA per row at a time, threads stride over the words.
template <typename W>
__global__ void __launch_bounds__(256) k_pack_wide(const int32_t* __restrict__ src,
                                                   int64_t nrows, const char* __restrict__ B,
                                                   int64_t ldb_bytes, char* __restrict__ Bp,
                                                   int64_t ldp_bytes, int64_t wpr) {
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int64_t s = __ldg(src + r);
    const W* in = reinterpret_cast<const W*>(B + s * ldb_bytes);
    W* out = reinterpret_cast<W*>(Bp + r * ldp_bytes);
    for (int64_t w = threadIdx.x; w < wpr; w += blockDim.x) out[w] = __ldg(in + w);
  }
}

template <typename W>
static shiro_status launch_typed(const shiro_plan_s* P, const char* B, int64_t ldb_bytes,
                                 char* Bp, int64_t ldp_bytes, int64_t row_bytes, cudaStream_t s) {
  const int64_t wpr = row_bytes / (int64_t)sizeof(W);
  const int64_t nrows = P->packed_rows;
  const int64_t cap = (int64_t)P->sm_count * 8;
  if (wpr <= 256) {
    const int32_t rpi = 256 / (int32_t)wpr;
    const int64_t grid = std::min<int64_t>((nrows + rpi - 1) / rpi, cap);
    k_pack_rows<W><<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(
        P->d_pack_src, nrows, B, ldb_bytes, Bp, ldp_bytes, (int32_t)wpr);
  } else {
    const int64_t grid = std::min<int64_t>(nrows, cap);
    k_pack_wide<W><<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(
        P->d_pack_src, nrows, B, ldb_bytes, Bp, ldp_bytes, wpr);
  }
  SHIRO_CUDA(cudaGetLastError());
  return SHIRO_OK;
}

shiro_status launch_pack(const shiro_plan_s* P, const void* B, int64_t ldb, int32_t N,
                         shiro_dtype dt, void* Bpack, int64_t ldp, cudaStream_t s) {
  if (N < 0 || ldb < N || ldp < N) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "bad N or leading dimension");
  if (dt != SHIRO_F32 && dt != SHIRO_BF16 && dt != SHIRO_F64)
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "unknown dtype");
  if (N == 0 || P->packed_rows == 0) return SHIRO_OK;
  if (!B || !Bpack) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null B or Bpack");
  const int64_t esz = (int64_t)dtype_size(dt);
  const int64_t row_bytes = (int64_t)N * esz, ldb_b = ldb * esz, ldp_b = ldp * esz;
  const uintptr_t a = (uintptr_t)B | (uintptr_t)Bpack | (uintptr_t)row_bytes |
                      (uintptr_t)ldb_b | (uintptr_t)ldp_b;
  const char* b = (const char*)B;
  char* o = (char*)Bpack;
  if (a % 16 == 0) return launch_typed<uint4>(P, b, ldb_b, o, ldp_b, row_bytes, s);
  if (a % 8 == 0) return launch_typed<uint2>(P, b, ldb_b, o, ldp_b, row_bytes, s);
  if (a % 4 == 0) return launch_typed<uint32_t>(P, b, ldb_b, o, ldp_b, row_bytes, s);
  if (a % 2 == 0) return launch_typed<unsigned short>(P, b, ldb_b, o, ldp_b, row_bytes, s);
  SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "misaligned B or Bpack");
}

}  // namespace shiro

extern "C" shiro_status shiro_pack(shiro_plan_t plan, const void* B, int64_t ldb, int32_t N,
                                   shiro_dtype dt, void* Bpack, int64_t ldp, void* stream) {
  if (!plan) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  return shiro::launch_pack(plan, B, ldb, N, dt, Bpack, ldp, (cudaStream_t)stream);
}
