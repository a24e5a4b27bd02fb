// spmm.cu -- C entry points of the local SpMM over the packed B rows (Sec. 2.2 stages 3-4,
// Sec. 5.1 stage 5): argument checks and the dispatch to the per-storage-type instantiations of
// spmm_kernels.cuh, the schedule autotuner and the allocation-free variant.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace shiro {

namespace {
struct OccKey {
  int device;
  const void* kern;
  int threads;
  size_t smem;
  bool operator==(const OccKey& o) const {
    return device == o.device && kern == o.kern && threads == o.threads && smem == o.smem;
  }
};
std::mutex g_occ_mu;
std::vector<std::pair<OccKey, int>> g_occ;  // a few dozen kernel shapes at most
}  // namespace

cudaError_t occupancy_cached(int* per_sm, const void* kern, int threads, size_t smem) {
  OccKey k{0, kern, threads, smem};
  cudaError_t e = cudaGetDevice(&k.device);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    for (const auto& kv : g_occ)
      if (kv.first == k) {
        *per_sm = kv.second;
        return cudaSuccess;
      }
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_occ_mu);
  g_occ.emplace_back(k, *per_sm);
  return cudaSuccess;
}

// One translation unit per storage type (spmm_f32.cu, spmm_bf16.cu, spmm_f64.cu).
#define SHIRO_SPMM_TYPED(name)                                                                  \
  shiro_status name(const shiro_plan_s* P, const void* Bpack, int64_t ldp, const void* B,       \
                    int64_t ldb, int32_t N, shiro_dtype dt, void* C, int64_t ldc, uint32_t flags, \
                    void* scratch, cudaStream_t s);
SHIRO_SPMM_TYPED(spmm_f32)
SHIRO_SPMM_TYPED(spmm_bf16)
SHIRO_SPMM_TYPED(spmm_f64)
#undef SHIRO_SPMM_TYPED
#define SHIRO_FUSED_TYPED(name)                                                                  \
  shiro_status name(const shiro_plan_s* P, const void* B, int64_t ldb, int32_t N, shiro_dtype dt, \
                    void* Bpack, int64_t ldp, void* C, int64_t ldc, uint32_t flags,              \
                    void* scratch, cudaStream_t s, bool* fused);
SHIRO_FUSED_TYPED(spmm_fused_f32)
SHIRO_FUSED_TYPED(spmm_fused_bf16)
SHIRO_FUSED_TYPED(spmm_fused_f64)
#undef SHIRO_FUSED_TYPED
#define SHIRO_BWD_TYPED(name)                                                                    \
  shiro_status name(const shiro_plan_s* PT, const void* dC, int64_t lddc, int32_t N,             \
                    shiro_dtype dt, void* dCpack, int64_t lddp, void* dB, int64_t lddb,          \
                    const void* B, int64_t ldb, void* dA, void* scratch, cudaStream_t s,         \
                    bool* done);
SHIRO_BWD_TYPED(spmm_bwd_f32)
SHIRO_BWD_TYPED(spmm_bwd_bf16)
#undef SHIRO_BWD_TYPED

size_t spmm_scratch_bytes(const shiro_plan_s* P, int32_t N, shiro_dtype dt) {
  if (!P->n_slots) return 0;
  const size_t acc = dt == SHIRO_F64 ? 8 : 4;
  return (size_t)P->n_slots * (size_t)N * acc + 256;
}

shiro_status launch_spmm(const shiro_plan_s* P, const void* Bpack, int64_t ldp, const void* B,
                         int64_t ldb, int32_t N, shiro_dtype dt, void* C, int64_t ldc,
                         uint32_t flags, void* scratch, size_t scratch_bytes, cudaStream_t s) {
  if (N < 0 || ldp < N || ldc < N) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "bad N or leading dimension");
  // The gathers multiply a 32-bit row index by a 32-bit row stride.
  if (ldp > (int64_t)UINT32_MAX || ldb > (int64_t)UINT32_MAX)
    SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "leading dimensions of B / Bpack above 2^32 - 1 elements");
  if (!C && P->M > 0 && N > 0) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null C");
  if (!Bpack && P->packed_rows > 0 && N > 0) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null Bpack");
  if ((P->flags & SHIRO_PLAN_LOCAL_DIAG) && (!B || ldb < N))
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "LOCAL_DIAG plan needs B with ldb >= N");
  if (flags & ~SHIRO_SPMM_ACCUMULATE) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "unknown SpMM flags");
  const size_t need = spmm_scratch_bytes(P, N, dt);
  if (need && (!scratch || scratch_bytes < need))
    SHIRO_FAIL(SHIRO_ERR_INSUFFICIENT_WORKSPACE, "SpMM scratch of %zu bytes, need %zu",
               scratch_bytes, need);
  if (N == 0 || P->M == 0) return SHIRO_OK;
  if (P->vdt == SHIRO_F32 && dt == SHIRO_F32)
    return spmm_f32(P, Bpack, ldp, B, ldb, N, dt, C, ldc, flags, scratch, s);
  if (P->vdt == SHIRO_F32 && dt == SHIRO_BF16)
    return spmm_bf16(P, Bpack, ldp, B, ldb, N, dt, C, ldc, flags, scratch, s);
  if (P->vdt == SHIRO_F64 && dt == SHIRO_F64)
    return spmm_f64(P, Bpack, ldp, B, ldb, N, dt, C, ldc, flags, scratch, s);
  SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "value/operand dtypes: F32 with F32 or BF16, or F64 with F64");
}

shiro_status launch_pack_spmm(const shiro_plan_s* plan, const void* B, int64_t ldb, int32_t N,
                              shiro_dtype dt, void* Bpack, int64_t ldp, void* C, int64_t ldc,
                              uint32_t flags, void* scratch, size_t scratch_bytes,
                              cudaStream_t s) {
  // The checks of both halves first, so that nothing is launched on bad arguments.
  if (N < 0 || ldb < N || ldp < N || ldc < N)
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "bad N or leading dimension");
  if (dt != SHIRO_F32 && dt != SHIRO_BF16 && dt != SHIRO_F64)
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "unknown dtype");
  if (N == 0 || plan->M == 0) return SHIRO_OK;
  if (!B) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null B");
  if (ldp > (int64_t)UINT32_MAX || ldb > (int64_t)UINT32_MAX)
    SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "leading dimensions of B / Bpack above 2^32 - 1 elements");
  if (!C) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null C");
  if (!Bpack && plan->packed_rows > 0) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null Bpack");
  if (flags & ~SHIRO_SPMM_ACCUMULATE) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "unknown SpMM flags");
  const size_t need = spmm_scratch_bytes(plan, N, dt);
  if (need && (!scratch || scratch_bytes < need))
    SHIRO_FAIL(SHIRO_ERR_INSUFFICIENT_WORKSPACE, "SpMM scratch of %zu bytes, need %zu",
               scratch_bytes, need);
  bool fused = false;
  if (plan->vdt == SHIRO_F32 && dt == SHIRO_F32)
    SHIRO_TRY(spmm_fused_f32(plan, B, ldb, N, dt, Bpack, ldp, C, ldc, flags, scratch, s, &fused));
  else if (plan->vdt == SHIRO_F32 && dt == SHIRO_BF16)
    SHIRO_TRY(spmm_fused_bf16(plan, B, ldb, N, dt, Bpack, ldp, C, ldc, flags, scratch, s, &fused));
  else if (plan->vdt == SHIRO_F64 && dt == SHIRO_F64)
    SHIRO_TRY(spmm_fused_f64(plan, B, ldb, N, dt, Bpack, ldp, C, ldc, flags, scratch, s, &fused));
  if (fused) return SHIRO_OK;
  // Other row shapes and schedules: the two launches, same results.
  SHIRO_TRY(launch_pack(plan, B, ldb, N, dt, Bpack, ldp, s));
  return launch_spmm(plan, Bpack, ldp, B, ldb, N, dt, C, ldc, flags, scratch, scratch_bytes, s);
}

shiro_status launch_backward_one(const shiro_plan_s* plan, const shiro_plan_s* planT,
                                 const void* dC, int64_t lddc, const void* B, int64_t ldb,
                                 int32_t N, shiro_dtype dt, void* dCpack, int64_t lddp, void* dB,
                                 int64_t lddb, void* dA, void* scratch, size_t scratch_bytes,
                                 cudaStream_t s, bool* done) {
  *done = false;
  // Only well-formed calls with work to do; anything else goes the two-call way, which reports
  // the error or handles the empty case.
  if (!B || !dC || !dB || !dA || N <= 0 || plan->nnz == 0 || planT->M == 0) return SHIRO_OK;
  if (plan->vdt != SHIRO_F32 || planT->vdt != SHIRO_F32) return SHIRO_OK;
  if (dt != SHIRO_F32 && dt != SHIRO_BF16) return SHIRO_OK;
  if (lddc < N || lddp < N || lddb < N || ldb < N) return SHIRO_OK;
  if (lddp > (int64_t)UINT32_MAX || lddc > (int64_t)UINT32_MAX || ldb > (int64_t)UINT32_MAX)
    return SHIRO_OK;
  if (!dCpack && planT->packed_rows > 0) return SHIRO_OK;
  const size_t need = spmm_scratch_bytes(planT, N, dt);
  if (need && (!scratch || scratch_bytes < need)) return SHIRO_OK;
  if (dt == SHIRO_F32)
    return spmm_bwd_f32(planT, dC, lddc, N, dt, dCpack, lddp, dB, lddb, B, ldb, dA, scratch, s,
                        done);
  return spmm_bwd_bf16(planT, dC, lddc, N, dt, dCpack, lddp, dB, lddb, B, ldb, dA, scratch, s,
                       done);
}

}  // namespace shiro

using namespace shiro;

extern "C" {

shiro_status shiro_spmm_scratch(shiro_plan_t plan, int32_t N, shiro_dtype dt, size_t* bytes) {
  if (!plan || !bytes || N < 0) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "bad arguments");
  *bytes = spmm_scratch_bytes(plan, N, dt);
  return SHIRO_OK;
}

shiro_status shiro_spmm(shiro_plan_t plan, const void* Bpack, int64_t ldp, const void* B,
                        int64_t ldb, int32_t N, shiro_dtype dt, void* C, int64_t ldc,
                        uint32_t flags, void* scratch, size_t scratch_bytes, void* stream) {
  if (!plan) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  return launch_spmm(plan, Bpack, ldp, B, ldb, N, dt, C, ldc, flags, scratch, scratch_bytes,
                     (cudaStream_t)stream);
}

shiro_status shiro_pack_spmm(shiro_plan_t plan, const void* B, int64_t ldb, int32_t N,
                            shiro_dtype dt, void* Bpack, int64_t ldp, void* C, int64_t ldc,
                            uint32_t flags, void* scratch, size_t scratch_bytes, void* stream) {
  if (!plan) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  return launch_pack_spmm(plan, B, ldb, N, dt, Bpack, ldp, C, ldc, flags, scratch, scratch_bytes,
                          (cudaStream_t)stream);
}

shiro_status shiro_autotune(shiro_plan_t P, const void* Bpack, int64_t ldp, const void* B,
                            int64_t ldb, int32_t N, shiro_dtype dt, void* C, int64_t ldc,
                            void* scratch, size_t scratch_bytes, int32_t reps, void* stream,
                            shiro_opts* best) {
  if (!P) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  cudaStream_t s = (cudaStream_t)stream;
  if (reps < 1) reps = 3;
  const shiro_opts start = P->opts;
  // Candidate schedules from N and the degree profile: average nonzeros per row sets the group
  // size, the largest rows decide whether splitting matters at all.
  const double avg = P->M ? (double)P->nnz / (double)P->M : 0.0;
  std::vector<shiro_opts> cands;
  const int32_t groups[] = {0, 128, 256, 512, 1024};  // 0: automatic
  const int32_t chunks[] = {256, 512, 1024};
  const int32_t warps[] = {1, 2, 4};
  // Pipelines worth trying: register gathers (5), lane groups when rows are 128 or 256 bytes (3),
  // the per-lane copy ring for rows of 512 bytes to 2 KB (4), lean register gathers for rows of
  // 128 to 512 bytes (6; in persistent mode their counter form), the TMA gather4 ring for rows of
  // 512 bytes (7).
  const int64_t row_bytes = (int64_t)N * (int64_t)dtype_size(dt);
  const bool narrow = dt != SHIRO_F64 && (row_bytes == 128 || row_bytes == 256);
  const bool ringable = dt != SHIRO_F64 && (row_bytes == 512 || row_bytes == 1024 ||
                                            row_bytes == 2048);
  const bool leanable = dt != SHIRO_F64 &&
                        (row_bytes == 128 || row_bytes == 256 || row_bytes == 512);
  const bool g4able = dt != SHIRO_F64 && row_bytes == 512 && !(P->flags & SHIRO_PLAN_LOCAL_DIAG);
  const int32_t pipes[] = {5, 3, 4, 6, 7};
  for (int32_t gn : groups) {
    if (gn && gn < avg / 2) continue;
    for (int32_t ch : chunks) {
      if (P->max_row_nnz <= ch && ch != 512) continue;
      for (int32_t w : warps) {
        for (int32_t pipe : pipes) {
          if (pipe == 3 && !narrow) continue;
          if (pipe == 4 && !ringable) continue;
          if (pipe == 6 && (!leanable || w != 1)) continue;  // lean CTAs are always 2 warps
          if (pipe == 7 && (!g4able || w != 1)) continue;    // gather4 CTAs have a fixed shape
          shiro_opts o = start;
          o.group_nnz = gn;
          o.group_rows = 32;
          o.chunk_nnz = ch;
          o.long_row_nnz = 2 * ch;
          o.warps_per_cta = w;
          o.pipeline = pipe;  // persistent mode stays as the caller set it
          cands.push_back(o);
        }
      }
    }
  }
  cands.push_back(start);
  cudaEvent_t e0, e1;
  SHIRO_CUDA(cudaEventCreate(&e0));
  {
    const cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      SHIRO_FAIL(SHIRO_ERR_CUDA, "shiro_autotune: cudaEventCreate failed: %s",
                 cudaGetErrorString(e));
    }
  }
  float best_ms = 1e30f;
  shiro_opts best_o = start;
  shiro_status st = SHIRO_OK;
  for (const shiro_opts& o : cands) {
    st = build_schedule(P, o, s);
    if (st != SHIRO_OK) break;
    if (spmm_scratch_bytes(P, N, dt) > scratch_bytes) continue;
    st = launch_spmm(P, Bpack, ldp, B, ldb, N, dt, C, ldc, 0, scratch, scratch_bytes, s);
    if (st != SHIRO_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) {
      st = launch_spmm(P, Bpack, ldp, B, ldb, N, dt, C, ldc, 0, scratch, scratch_bytes, s);
      if (st != SHIRO_OK) break;
    }
    if (st != SHIRO_OK) break;
    cudaEventRecord(e1, s);
    {
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        st = SHIRO_ERR_CUDA;
        set_error("shiro_autotune: cudaEventSynchronize failed: %s", cudaGetErrorString(e));
        break;
      }
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best_o = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SHIRO_OK) {
    build_schedule(P, start, s);
    return st;
  }
  SHIRO_TRY(build_schedule(P, best_o, s));
  if (best) *best = best_o;
  return SHIRO_OK;
}

}  // extern "C"

// ---- allocation-free SpMM ----
//
// Scratch for callers that cannot allocate device memory: one array in the library's own module,
// created when the module is loaded on a device and kept until the process exits.  Its host-side
// name is not a device address; the address is looked up once per device below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SHIRO_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

extern "C" shiro_status shiro_spmm_noalloc(shiro_plan_t plan, const void* Bpack, int64_t ldp,
                                           const void* B, int64_t ldb, int32_t N,
                                           shiro_dtype dt, void* C, int64_t ldc, uint32_t flags,
                                           void* stream) {
  if (!plan) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "null plan");
  if (N < 0) SHIRO_FAIL(SHIRO_ERR_INVALID_ARG, "negative N");
  int dev = 0;
  SHIRO_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    SHIRO_FAIL(SHIRO_ERR_UNSUPPORTED, "device index %d beyond %d", dev, kMaxDevices);
  // The static array's address is per device: a plan of another device would get this device's.
  if (dev != plan->device)
    SHIRO_FAIL(SHIRO_ERR_INVALID_ARG,
               "shiro_spmm_noalloc: the plan belongs to device %d, the current device is %d",
               plan->device, dev);
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      SHIRO_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
      g_noalloc_ptr[dev] = ptr;
    }
    scratch = g_noalloc_ptr[dev];
  }
  const size_t need = spmm_scratch_bytes(plan, N, dt);
  if (need > (size_t)SHIRO_NOALLOC_SCRATCH_BYTES)
    SHIRO_FAIL(SHIRO_ERR_INSUFFICIENT_WORKSPACE,
               "shiro_spmm_noalloc: this plan's split rows need %zu bytes of scratch for N=%d, "
               "more than the %d-byte static scratch; use shiro_spmm with a caller buffer or a "
               "schedule with larger chunks",
               need, N, SHIRO_NOALLOC_SCRATCH_BYTES);
  // The static array needs no clearing: every chunk writes its partial-sum slot before the last
  // chunk of its row reads the slots back (the arrival counters live in the plan).
  return launch_spmm(plan, Bpack, ldp, B, ldb, N, dt, C, ldc, flags, scratch,
                     (size_t)SHIRO_NOALLOC_SCRATCH_BYTES, (cudaStream_t)stream);
}
