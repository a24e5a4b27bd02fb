// vec.cuh -- per-lane vector fragments of dense rows (FP32, BF16 storage, FP64).
//
// A warp covers a dense row in chunks of 32 * VEC elements; lane l owns elements
// [c * 32 * VEC + l * VEC, + VEC) of chunk c.  Loads are 4-16 bytes per lane, so one warp-wide
// load instruction moves 128-512 contiguous bytes of a row.  BF16 values are widened to FP32
// exactly (shift into the high half).
#pragma once

#include <type_traits>

#include "internal.cuh"

namespace shiro {

template <typename TB> struct AccOf { using T = float; };
template <> struct AccOf<double> { using T = double; };

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Load VEC consecutive elements at p (aligned to VEC * sizeof(TB)) into out[].
template <typename TB, int VEC, bool NC>
__device__ __forceinline__ void load_vec(const TB* p, typename AccOf<TB>::T (&out)[VEC]) {
  if constexpr (std::is_same<TB, float>::value) {
    if constexpr (VEC == 4) {
      float4 v = NC ? __ldg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
      out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    } else if constexpr (VEC == 2) {
      float2 v = NC ? __ldg(reinterpret_cast<const float2*>(p)) : *reinterpret_cast<const float2*>(p);
      out[0] = v.x; out[1] = v.y;
    } else {
      out[0] = NC ? __ldg(p) : *p;
    }
  } else if constexpr (std::is_same<TB, double>::value) {
    if constexpr (VEC == 2) {
      double2 v = NC ? __ldg(reinterpret_cast<const double2*>(p)) : *reinterpret_cast<const double2*>(p);
      out[0] = v.x; out[1] = v.y;
    } else {
      out[0] = NC ? __ldg(p) : *p;
    }
  } else {  // __nv_bfloat16 storage
    if constexpr (VEC == 8) {
      uint4 v = NC ? __ldg(reinterpret_cast<const uint4*>(p)) : *reinterpret_cast<const uint4*>(p);
      out[0] = bf16_lo(v.x); out[1] = bf16_hi(v.x); out[2] = bf16_lo(v.y); out[3] = bf16_hi(v.y);
      out[4] = bf16_lo(v.z); out[5] = bf16_hi(v.z); out[6] = bf16_lo(v.w); out[7] = bf16_hi(v.w);
    } else if constexpr (VEC == 4) {
      uint2 v = NC ? __ldg(reinterpret_cast<const uint2*>(p)) : *reinterpret_cast<const uint2*>(p);
      out[0] = bf16_lo(v.x); out[1] = bf16_hi(v.x); out[2] = bf16_lo(v.y); out[3] = bf16_hi(v.y);
    } else if constexpr (VEC == 2) {
      uint32_t v = NC ? __ldg(reinterpret_cast<const unsigned int*>(p)) : *reinterpret_cast<const uint32_t*>(p);
      out[0] = bf16_lo(v); out[1] = bf16_hi(v);
    } else {
      unsigned short v = NC ? __ldg(reinterpret_cast<const unsigned short*>(p)) : *reinterpret_cast<const unsigned short*>(p);
      out[0] = __uint_as_float(((uint32_t)v) << 16);
    }
  }
}

// Raw storage words of a VEC-element fragment, kept as loaded while the gather is in flight:
// the elements themselves for FP32 / FP64, packed BF16 pairs for BF16 (VEC / 2 words; one
// half-word in the low bits for VEC = 1), widened only where they are consumed, so a BF16 row
// in flight costs half the registers of its FP32 widening.
template <typename TB, int VEC> struct RawFrag {
  using T = TB;
  static constexpr int W = VEC;
};
template <int VEC> struct RawFrag<__nv_bfloat16, VEC> {
  using T = uint32_t;
  static constexpr int W = (VEC + 1) / 2;
};

template <typename TB, int VEC>
__device__ __forceinline__ void load_raw(const TB* p,
                                         typename RawFrag<TB, VEC>::T (&w)[RawFrag<TB, VEC>::W]) {
  if constexpr (!std::is_same<TB, __nv_bfloat16>::value) {
    load_vec<TB, VEC, true>(p, w);
  } else if constexpr (VEC == 8) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  } else if constexpr (VEC == 4) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    w[0] = v.x; w[1] = v.y;
  } else if constexpr (VEC == 2) {
    w[0] = __ldg(reinterpret_cast<const unsigned int*>(p));
  } else {
    w[0] = __ldg(reinterpret_cast<const unsigned short*>(p));
  }
}

// load_raw through L2 only (ld.global.cg): for rows that other warps of the same launch write
// (the fused pack + SpMM), which the non-coherent path must not read.
template <typename TB, int VEC>
__device__ __forceinline__ void load_raw_cg(const TB* p,
                                            typename RawFrag<TB, VEC>::T (&w)[RawFrag<TB, VEC>::W]) {
  if constexpr (std::is_same<TB, float>::value) {
    if constexpr (VEC == 4) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
      w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if constexpr (VEC == 2) {
      const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
      w[0] = v.x; w[1] = v.y;
    } else {
      w[0] = __ldcg(p);
    }
  } else if constexpr (std::is_same<TB, double>::value) {
    if constexpr (VEC == 2) {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
      w[0] = v.x; w[1] = v.y;
    } else {
      w[0] = __ldcg(p);
    }
  } else if constexpr (VEC == 8) {
    const uint4 v = __ldcg(reinterpret_cast<const uint4*>(p));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  } else if constexpr (VEC == 4) {
    const uint2 v = __ldcg(reinterpret_cast<const uint2*>(p));
    w[0] = v.x; w[1] = v.y;
  } else if constexpr (VEC == 2) {
    w[0] = __ldcg(reinterpret_cast<const unsigned int*>(p));
  } else {
    w[0] = __ldcg(reinterpret_cast<const unsigned short*>(p));
  }
}

// Store a raw fragment as loaded (a bit-exact row copy).
template <typename TB, int VEC>
__device__ __forceinline__ void store_raw(TB* p,
                                          const typename RawFrag<TB, VEC>::T (&w)[RawFrag<TB, VEC>::W]) {
  if constexpr (std::is_same<TB, float>::value) {
    if constexpr (VEC == 4) *reinterpret_cast<float4*>(p) = make_float4(w[0], w[1], w[2], w[3]);
    else if constexpr (VEC == 2) *reinterpret_cast<float2*>(p) = make_float2(w[0], w[1]);
    else *p = w[0];
  } else if constexpr (std::is_same<TB, double>::value) {
    if constexpr (VEC == 2) *reinterpret_cast<double2*>(p) = make_double2(w[0], w[1]);
    else *p = w[0];
  } else if constexpr (VEC == 8) {
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
  } else if constexpr (VEC == 4) {
    *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
  } else if constexpr (VEC == 2) {
    *reinterpret_cast<uint32_t*>(p) = w[0];
  } else {
    *reinterpret_cast<unsigned short*>(p) = (unsigned short)w[0];
  }
}

// acc[v] = fma(a, element v of the raw fragment, acc[v]) for v = 0 .. VEC-1, in that order (the
// BF16 widening is exact, so this equals widening first).
template <typename TB, int VEC, typename TV>
__device__ __forceinline__ void fma_raw(TV a, const typename RawFrag<TB, VEC>::T (&w)[RawFrag<TB, VEC>::W],
                                        typename AccOf<TB>::T (&acc)[VEC]) {
  using TA = typename AccOf<TB>::T;
#ifndef SHIRO_FFMA2
#define SHIRO_FFMA2 1
#endif
  // Pairs of FP32 accumulators by the paired FMA of sm_100 and later (fma.rn.f32x2): each element
  // is still one correctly rounded FMA, so the sums are bit-identical to the scalar form, in half
  // the multiply instructions.  BF16 fragments and FP32 fragments of 4 (R-MAT 2^20 SpMM, ms: BF16
  // N = 256 0.837 -> 0.821, BF16 N = 128 0.447 -> 0.441, FP32 N = 128 0.552 -> 0.549; R-MAT 2^22
  // BF16 N = 256 6.11 -> 5.98); FP32 fragments of 2 spilled with it (N = 64 0.368 -> 0.374).
  constexpr bool PAIRED = std::is_same<TB, __nv_bfloat16>::value ? VEC >= 2
                                                                  : (std::is_same<TB, float>::value && VEC >= 4);
  if constexpr (SHIRO_FFMA2 && PAIRED) {
    const float2 a2 = make_float2((float)a, (float)a);
#pragma unroll
    for (int k = 0; k < VEC / 2; ++k) {
      float2 b2;
      if constexpr (std::is_same<TB, __nv_bfloat16>::value)
        b2 = make_float2(bf16_lo(w[k]), bf16_hi(w[k]));
      else
        b2 = make_float2(w[2 * k], w[2 * k + 1]);
      const float2 r = __ffma2_rn(a2, b2, make_float2(acc[2 * k], acc[2 * k + 1]));
      acc[2 * k] = r.x;
      acc[2 * k + 1] = r.y;
    }
  } else if constexpr (!std::is_same<TB, __nv_bfloat16>::value) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = fma((TA)a, w[v], acc[v]);
  } else if constexpr (VEC == 1) {
    acc[0] = fma((TA)a, bf16_lo(w[0]), acc[0]);
  } else {
#pragma unroll
    for (int k = 0; k < VEC / 2; ++k) {
      acc[2 * k] = fma((TA)a, bf16_lo(w[k]), acc[2 * k]);
      acc[2 * k + 1] = fma((TA)a, bf16_hi(w[k]), acc[2 * k + 1]);
    }
  }
}

// Store VEC accumulator values (float or double) at p; STREAM uses an evict-first store.
template <typename TA, int VEC, bool STREAM>
__device__ __forceinline__ void store_vec(TA* p, const TA (&v)[VEC]) {
  if constexpr (std::is_same<TA, float>::value) {
    if constexpr (VEC == 8) {
      float4 a = make_float4(v[0], v[1], v[2], v[3]), b = make_float4(v[4], v[5], v[6], v[7]);
      if (STREAM) { __stcs(reinterpret_cast<float4*>(p), a); __stcs(reinterpret_cast<float4*>(p) + 1, b); }
      else { reinterpret_cast<float4*>(p)[0] = a; reinterpret_cast<float4*>(p)[1] = b; }
    } else if constexpr (VEC == 4) {
      float4 a = make_float4(v[0], v[1], v[2], v[3]);
      if (STREAM) __stcs(reinterpret_cast<float4*>(p), a); else *reinterpret_cast<float4*>(p) = a;
    } else if constexpr (VEC == 2) {
      float2 a = make_float2(v[0], v[1]);
      if (STREAM) __stcs(reinterpret_cast<float2*>(p), a); else *reinterpret_cast<float2*>(p) = a;
    } else {
      if (STREAM) __stcs(p, v[0]); else *p = v[0];
    }
  } else {
    if constexpr (VEC == 2) {
      double2 a = make_double2(v[0], v[1]);
      if (STREAM) __stcs(reinterpret_cast<double2*>(p), a); else *reinterpret_cast<double2*>(p) = a;
    } else {
      if (STREAM) __stcs(p, v[0]); else *p = v[0];
    }
  }
}

// Load VEC accumulator values from p, bypassing L1 (data written by other SMs in this launch).
template <typename TA, int VEC>
__device__ __forceinline__ void load_acc_cg(const TA* p, TA (&v)[VEC]) {
  if constexpr (std::is_same<TA, float>::value) {
    if constexpr (VEC == 8) {
      float4 a = __ldcg(reinterpret_cast<const float4*>(p)), b = __ldcg(reinterpret_cast<const float4*>(p) + 1);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else if constexpr (VEC == 4) {
      float4 a = __ldcg(reinterpret_cast<const float4*>(p));
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if constexpr (VEC == 2) {
      float2 a = __ldcg(reinterpret_cast<const float2*>(p));
      v[0] = a.x; v[1] = a.y;
    } else {
      v[0] = __ldcg(p);
    }
  } else {
    if constexpr (VEC == 2) {
      double2 a = __ldcg(reinterpret_cast<const double2*>(p));
      v[0] = a.x; v[1] = a.y;
    } else {
      v[0] = __ldcg(p);
    }
  }
}

// Store VEC accumulator values at p so that they stay in L2 (partials read back by another SM).
template <typename TA, int VEC>
__device__ __forceinline__ void store_acc_cg(TA* p, const TA (&v)[VEC]) {
  if constexpr (std::is_same<TA, float>::value) {
    if constexpr (VEC == 8) {
      __stcg(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
      __stcg(reinterpret_cast<float4*>(p) + 1, make_float4(v[4], v[5], v[6], v[7]));
    } else if constexpr (VEC == 4) {
      __stcg(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
    } else if constexpr (VEC == 2) {
      __stcg(reinterpret_cast<float2*>(p), make_float2(v[0], v[1]));
    } else {
      __stcg(p, v[0]);
    }
  } else {
    if constexpr (VEC == 2) __stcg(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
    else __stcg(p, v[0]);
  }
}

}  // namespace shiro
