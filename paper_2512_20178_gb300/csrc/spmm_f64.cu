// spmm_f64.cu -- the SpMM kernels instantiated for double storage (double values).
#include "spmm_kernels.cuh"

namespace shiro {

shiro_status spmm_f64(const shiro_plan_s* P, const void* Bpack, int64_t ldp, const void* B,
                        int64_t ldb, int32_t N, shiro_dtype dt, void* C, int64_t ldc,
                        uint32_t flags, void* scratch, cudaStream_t s) {
  return spmm_typed<double, double>(P, Bpack, ldp, B, ldb, N, dt, C, ldc, flags, scratch, s);
}

shiro_status spmm_fused_f64(const shiro_plan_s* P, const void* B, int64_t ldb, int32_t N,
                              shiro_dtype dt, void* Bpack, int64_t ldp, void* C, int64_t ldc,
                              uint32_t flags, void* scratch, cudaStream_t s, bool* fused) {
  return spmm_fused_typed<double, double>(P, B, ldb, N, dt, Bpack, ldp, C, ldc, flags, scratch, s,
                                      fused);
}

}  // namespace shiro
