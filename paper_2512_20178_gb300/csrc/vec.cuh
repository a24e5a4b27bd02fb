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
