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

shiro_status spmm_bwd_f64(const shiro_plan_s* PT, const void* dC, int64_t lddc, int32_t N,
                          shiro_dtype dt, void* dCpack, int64_t lddp, void* dB, int64_t lddb,
                          const void* B, int64_t ldb, void* dA, void* scratch, cudaStream_t s,
                          bool* done) {
  return spmm_bwd_typed<double, double>(PT, dC, lddc, N, dt, dCpack, lddp, dB, lddb, B, ldb, dA,
                                    scratch, s, done);
}

}  // namespace shiro
