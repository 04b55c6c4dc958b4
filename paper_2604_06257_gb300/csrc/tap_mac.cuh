// tap_mac.cuh -- load the two interpolation taps of a term for a lane's frames and
// accumulate c0 * x[i0] + c1 * x[i0 + 1] (complex), per IQ storage type.
//
// Storage types: float2 (complex64), __half2 (float16 pairs), __nv_bfloat162 (bfloat16
// pairs) hold one complex sample per element, frames contiguous within a sample row;
// C64Planar rows hold the F real parts, then the F imaginary parts (complex64 values),
// so that two frames' real (or imaginary) parts sit in adjacent registers and the
// complex multiply-accumulate runs as packed FP32x2 FMAs.
//
// Every storage type performs, per frame, exactly this FMA sequence in FP32:
//   re += c0r*x0.re; re += -c0i*x0.im; re += c1r*x1.re; re += -c1i*x1.im
//   im += c0r*x0.im; im += c0i*x0.re;  im += c1r*x1.im; im += c1i*x1.re
// so results do not depend on the storage layout.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <type_traits>

namespace mach {

struct C64Planar {};   // tag type: split complex64 rows (see above)

template <class IQ>
struct IqStore {       // element type in memory, elements per complex sample
  using E = IQ;
  static constexpr int eps = 1;
};
template <>
struct IqStore<C64Planar> {
  using E = float;
  static constexpr int eps = 2;
};

__device__ __forceinline__ float2 widen_bf16x2(uint32_t u) {   // exact
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

template <bool SMEM, class T>
__device__ __forceinline__ T ld(const T* p) {
  if constexpr (SMEM) return *p;
  else return __ldg(p);
}

// VEC consecutive complex samples (VEC = 1, 2 or 4) widened to float2.
template <class IQ, int VEC, bool SMEM>
__device__ __forceinline__ void load_vec(const IQ* p, float2 (&o)[VEC]) {
  if constexpr (std::is_same<IQ, float2>::value) {
    static_assert(VEC == 1 || VEC == 2 || VEC == 4, "1, 2 or 4 samples");
    if constexpr (VEC == 1) {
      o[0] = ld<SMEM>(p);
    } else {
#pragma unroll
      for (int h = 0; h < VEC / 2; ++h) {
        const float4 v = ld<SMEM>(reinterpret_cast<const float4*>(p) + h);
        o[2 * h] = make_float2(v.x, v.y);
        o[2 * h + 1] = make_float2(v.z, v.w);
      }
    }
  } else if constexpr (std::is_same<IQ, __half2>::value) {
    static_assert(VEC == 1 || VEC == 2 || VEC == 4, "1, 2 or 4 samples");
    if constexpr (VEC == 1) {
      o[0] = __half22float2(ld<SMEM>(p));
    } else if constexpr (VEC == 2) {
      const uint2 v = ld<SMEM>(reinterpret_cast<const uint2*>(p));
      o[0] = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
      o[1] = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
    } else {
      const uint4 v = ld<SMEM>(reinterpret_cast<const uint4*>(p));
      o[0] = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
      o[1] = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
      o[2] = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
      o[3] = __half22float2(*reinterpret_cast<const __half2*>(&v.w));
    }
  } else {
    static_assert(VEC == 1 || VEC == 2 || VEC == 4, "1, 2 or 4 samples");
    if constexpr (VEC == 1) {
      o[0] = widen_bf16x2(ld<SMEM>(reinterpret_cast<const unsigned int*>(p)));
    } else if constexpr (VEC == 2) {
      const uint2 v = ld<SMEM>(reinterpret_cast<const uint2*>(p));
      o[0] = widen_bf16x2(v.x);
      o[1] = widen_bf16x2(v.y);
    } else {
      const uint4 v = ld<SMEM>(reinterpret_cast<const uint4*>(p));
      o[0] = widen_bf16x2(v.x);
      o[1] = widen_bf16x2(v.y);
      o[2] = widen_bf16x2(v.z);
      o[3] = widen_bf16x2(v.w);
    }
  }
}

// Complex tap weights of a term record (a cos phi, a sin phi, w, .): c1 = w c and
// c0 = c - c1, each product and difference rounded on its own (never contracted into an
// FMA), so that every kernel derives the same bits from the same record.
__device__ __forceinline__ float4 tap_weights(const float4 r) {
  const float c1r = __fmul_rn(r.x, r.z), c1i = __fmul_rn(r.y, r.z);
  return make_float4(__fsub_rn(r.x, c1r), __fsub_rn(r.y, c1i), c1r, c1i);
}

__device__ __forceinline__ void mac1(float2& acc, float c0r, float c0i, float c1r, float c1i, float2 x0, float2 x1) {
  acc.x = fmaf(c0r, x0.x, acc.x);
  acc.x = fmaf(-c0i, x0.y, acc.x);
  acc.x = fmaf(c1r, x1.x, acc.x);
  acc.x = fmaf(-c1i, x1.y, acc.x);
  acc.y = fmaf(c0r, x0.y, acc.y);
  acc.y = fmaf(c0i, x0.x, acc.y);
  acc.y = fmaf(c1r, x1.y, acc.y);
  acc.y = fmaf(c1i, x1.x, acc.y);
}

// Packed FP32x2 fused multiply-add: d = a * b + c on both halves.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long A, B, Cc, D;
  asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(Cc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(D) : "l"(A), "l"(B), "l"(Cc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(D));
  return d;
}

// Accumulate one term into a lane's frames.  Interleaved types: acc[e] = (re, im) of
// frame e.  C64Planar (VEC = 4): acc[4m+2h] = (re of frames 2h, 2h+1) and
// acc[4m+2h+1] = (im of frames 2h, 2h+1) of vector m.
// r0: row i0 (the row i0 + 1 starts row_elems later); frames of vector m of lane jl:
// f_base + (jl + FL*m)*VEC .. + VEC - 1.
template <class IQ, int VEC, int NV, int FL, bool SMEM>
__device__ __forceinline__ void gather_mac(float2 (&acc)[VEC * NV], const typename IqStore<IQ>::E* r0, int row_elems,
                                           int F, int f_base, int jl, float c0r, float c0i, float c1r, float c1i) {
#pragma unroll
  for (int mm = 0; mm < NV; ++mm) {
    const int f = f_base + (jl + FL * mm) * VEC;
    if (f < F) {
      if constexpr (std::is_same<IQ, C64Planar>::value) {
        static_assert(VEC == 4, "split rows are read four frames at a time");
        const float4 ar = ld<SMEM>(reinterpret_cast<const float4*>(r0 + f));
        const float4 ai = ld<SMEM>(reinterpret_cast<const float4*>(r0 + F + f));
        const float4 br = ld<SMEM>(reinterpret_cast<const float4*>(r0 + row_elems + f));
        const float4 bi = ld<SMEM>(reinterpret_cast<const float4*>(r0 + row_elems + F + f));
        const float2 C0R = make_float2(c0r, c0r), C0N = make_float2(-c0i, -c0i), C0I = make_float2(c0i, c0i);
        const float2 C1R = make_float2(c1r, c1r), C1N = make_float2(-c1i, -c1i), C1I = make_float2(c1i, c1i);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float2 x0r = h ? make_float2(ar.z, ar.w) : make_float2(ar.x, ar.y);
          const float2 x0i = h ? make_float2(ai.z, ai.w) : make_float2(ai.x, ai.y);
          const float2 x1r = h ? make_float2(br.z, br.w) : make_float2(br.x, br.y);
          const float2 x1i = h ? make_float2(bi.z, bi.w) : make_float2(bi.x, bi.y);
          float2& re = acc[mm * 4 + 2 * h];
          float2& im = acc[mm * 4 + 2 * h + 1];
          re = ffma2(C0R, x0r, re);
          re = ffma2(C0N, x0i, re);
          re = ffma2(C1R, x1r, re);
          re = ffma2(C1N, x1i, re);
          im = ffma2(C0R, x0i, im);
          im = ffma2(C0I, x0r, im);
          im = ffma2(C1R, x1i, im);
          im = ffma2(C1I, x1r, im);
        }
      } else {
        float2 x0[VEC], x1[VEC];
        load_vec<IQ, VEC, SMEM>(r0 + f, x0);
        load_vec<IQ, VEC, SMEM>(r0 + row_elems + f, x1);
#pragma unroll
        for (int e = 0; e < VEC; ++e) mac1(acc[mm * VEC + e], c0r, c0i, c1r, c1i, x0[e], x1[e]);
      }
    }
  }
}

// Frame e (0 <= e < VEC) of vector mm of a lane's accumulators, as (re, im).
template <class IQ, int VEC>
__device__ __forceinline__ float2 acc_frame(const float2* acc_m, int e) {
  if constexpr (std::is_same<IQ, C64Planar>::value) {
    const float2 re = acc_m[2 * (e >> 1)], im = acc_m[2 * (e >> 1) + 1];
    return (e & 1) ? make_float2(re.y, im.y) : make_float2(re.x, im.x);
  } else {
    return acc_m[e];
  }
}

}  // namespace mach
