// internal.cuh -- shared definitions of libshiro's translation units (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "shiro.h"

namespace shiro {

void set_error(const char* fmt, ...);

#define SHIRO_CUDA(call)                                                                    \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      ::shiro::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                         __LINE__);                                                         \
      return SHIRO_ERR_CUDA;                                                                \
    }                                                                                       \
  } while (0)

#define SHIRO_FAIL(code, ...)        \
  do {                               \
    ::shiro::set_error(__VA_ARGS__); \
    return (code);                   \
  } while (0)

#define SHIRO_TRY(expr)                    \
  do {                                     \
    shiro_status s_ = (expr);              \
    if (s_ != SHIRO_OK) return s_;         \
  } while (0)

// Device status word bits (set by kernels, read back on the host).
enum : int {
  ST_BAD_ROWPTR = 1,
  ST_BAD_COL = 2,
  ST_OFF_DIAG = 4,
  ST_OVERFLOW = 8,
  ST_COUNTER = 16,
  ST_TIMEOUT = 32,  // a bounded device wait ran out (the kernel went on; results are not valid)
};

// One unit of SpMM/SDDMM work for one warp.
//   tag > 0 : rows [row, row + tag) (tag <= 32), nonzeros from e0 = rowptr[row];
//   tag <= 0: chunk of the long row `row`, partial-sum slot -tag - 1, nonzeros from e0.
struct alignas(16) Item {
  int32_t row;
  int32_t tag;
  int64_t e0;
};

struct alignas(16) LongRow {
  int32_t row;
  int32_t slot0;
  int32_t nchunks;
  int32_t pad;
};

// Tile geometry of the planned matrix, passed to kernels by value.
struct Geometry {
  int64_t M, K;
  int32_t Pr, Pc;
  int32_t diag_only;
  int32_t uniform_r, uniform_c;
  int64_t rstep, cstep;   // block sizes when uniform
  const int64_t* rb;      // device, Pr + 1
  const int64_t* cb;      // device, Pc + 1
};

__device__ __forceinline__ int32_t find_block(const int64_t* b, int32_t P, int64_t x) {
  // Last p with b[p] <= x (the non-empty block holding x when b[0] <= x < b[P]).
  int32_t lo = 0, hi = P;  // invariant: b[lo] <= x < b[hi]
  while (hi - lo > 1) {
    int32_t mid = (lo + hi) >> 1;
    if (b[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int32_t row_block(const Geometry& g, int64_t i) {
  return g.uniform_r ? (int32_t)(i / g.rstep) : find_block(g.rb, g.Pr, i);
}

__device__ __forceinline__ int32_t col_block(const Geometry& g, int64_t j) {
  return g.uniform_c ? (int32_t)(j / g.cstep) : find_block(g.cb, g.Pc, j);
}

}  // namespace shiro

struct shiro_plan_s {
  // The planned matrix (A, or A^T for a TRANSPOSE plan, or the block-diagonal batch).
  int64_t M = 0, K = 0, nnz = 0;
  shiro_dtype vdt = SHIRO_F32;
  uint32_t flags = 0;
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const void* val = nullptr;
  shiro::Geometry geo{};
  int32_t T = 0;

  // Device arrays carved from the workspace.
  int* d_status = nullptr;
  int64_t* d_rb = nullptr;
  int64_t* d_cb = nullptr;
  int64_t* d_woff = nullptr;             // T + 1 word offsets of the column bitmaps
  uint32_t* d_bitmap = nullptr;          // Wc words
  int64_t* d_wprefix = nullptr;          // Wc + 1 exclusive prefix of popcounts
  int64_t* d_rwoff = nullptr;            // T + 1 word offsets of the row bitmaps
  uint32_t* d_rbitmap = nullptr;         // Wr words
  unsigned long long* d_tile_nnz = nullptr;
  unsigned long long* d_tile_nrows = nullptr;
  int64_t* d_tile_cols_ptr = nullptr;    // T + 1
  int64_t* d_pack_ptr = nullptr;         // T + 1
  int32_t* d_cols_sorted = nullptr;      // cols_cap
  int32_t* d_pack_src = nullptr;         // == d_cols_sorted unless LOCAL_DIAG
  int32_t* d_remap = nullptr;            // nnz
  int64_t* d_scan_tmp = nullptr;         // block sums of the scans
  // Schedule.
  shiro::Item* d_items = nullptr;
  int32_t* d_slot_lr = nullptr;
  shiro::LongRow* d_lr = nullptr;
  int32_t* d_counters = nullptr;
  int64_t items_cap = 0, slots_cap = 0, lr_cap = 0;
  // Fused pack + SpMM: launch order (>= 0: item, < 0: pack chunk -code - 1), pack chunks
  // {first packed row, rows, row block, 0}, per-block chunk counts and completions.
  int32_t* d_fseq = nullptr;
  int4* d_pchunk = nullptr;
  int32_t* d_blk_need = nullptr;
  int32_t* d_blk_done = nullptr;
  int64_t fseq_cap = 0, pk_cap = 0, n_fseq = 0, n_pchunks = 0;
  // Transposed / batched copies of the planned matrix.
  int64_t* d_rowptr_own = nullptr;
  int32_t* d_col_own = nullptr;
  void* d_val_own = nullptr;
  int64_t* d_perm = nullptr;

  // Host copies.
  std::vector<int64_t> rb, cb, woff, rwoff;
  std::vector<int64_t> tile_nnz, tile_nrows, tile_ncols, tile_cols_ptr, pack_ptr;
  std::vector<int64_t> h_rowptr;
  int64_t Wc = 0, Wr = 0, cols_cap = 0;
  int64_t total_cols = 0, packed_rows = 0;
  int64_t n_items = 0, n_long = 0, n_slots = 0;
  int64_t max_row_nnz = 0;
  shiro_opts opts{};
  int sm_count = 0;
  int device = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0, ws_used = 0;
};

namespace shiro {

inline size_t dtype_size(shiro_dtype d) {
  return d == SHIRO_BF16 ? 2 : (d == SHIRO_F64 ? 8 : 4);
}

shiro_status resolve_opts(const shiro_opts* in, shiro_opts* out);
shiro_status build_schedule(shiro_plan_s* P, const shiro_opts& o, cudaStream_t s);
shiro_status read_status(shiro_plan_s* P, cudaStream_t s, const char* where);

// Launchers implemented in spmm.cu / sddmm.cu / pack.cu.
shiro_status launch_pack(const shiro_plan_s* P, const void* B, int64_t ldb, int32_t N,
                         shiro_dtype dt, void* Bpack, int64_t ldp, cudaStream_t s);
shiro_status launch_spmm(const shiro_plan_s* P, const void* Bpack, int64_t ldp, const void* B,
                         int64_t ldb, int32_t N, shiro_dtype dt, void* C, int64_t ldc,
                         uint32_t flags, void* scratch, size_t scratch_bytes, cudaStream_t s);
shiro_status launch_sddmm(const shiro_plan_s* P, const void* dC, int64_t lddc, const void* Bpack,
                          int64_t ldp, const void* B, int64_t ldb, int32_t N, shiro_dtype dt,
                          void* dA, cudaStream_t s);
size_t spmm_scratch_bytes(const shiro_plan_s* P, int32_t N, shiro_dtype dt);
// cudaOccupancyMaxActiveBlocksPerMultiprocessor, asked once per (device, kernel, block size,
// dynamic shared memory) and then answered from a table (the grid-sizing query otherwise costs
// host time on every launch).
cudaError_t occupancy_cached(int* per_sm, const void* kern, int threads, size_t smem);
template <typename K>
inline cudaError_t blocks_per_sm(int* per_sm, K kern, int threads, size_t smem) {
  return occupancy_cached(per_sm, reinterpret_cast<const void*>(kern), threads, smem);
}
// Pack + SpMM (one launch for FP32 rows of 512 bytes, and BF16 ones with pipeline 6; else pack
// then SpMM); same results as the two.
shiro_status launch_pack_spmm(const shiro_plan_s* P, const void* B, int64_t ldb, int32_t N,
                              shiro_dtype dt, void* Bpack, int64_t ldp, void* C, int64_t ldc,
                              uint32_t flags, void* scratch, size_t scratch_bytes, cudaStream_t s);
// dB (through the TRANSPOSE plan planT, as launch_pack_spmm) and dA of `plan` in one launch where
// the row shape and operands allow; *done = false (nothing launched) otherwise.
shiro_status launch_backward_one(const shiro_plan_s* plan, const shiro_plan_s* planT,
                                 const void* dC, int64_t lddc, const void* B, int64_t ldb,
                                 int32_t N, shiro_dtype dt, void* dCpack, int64_t lddp, void* dB,
                                 int64_t lddb, void* dA, void* scratch, size_t scratch_bytes,
                                 cudaStream_t s, bool* done);

}  // namespace shiro
