// Element types of the stored moments.
//
// FP64 and FP32 states store the shifted moments (d, j, A) as they are.  The
// 16-bit states (IEEE half, bfloat16) store them scaled by a power of two per
// field -- d * 2^6, j * 2^4, A * 2^10 -- so that the small values typical of
// a weakly compressible flow (d ~ 1e-4, off-diagonal A ~ 1e-6) stay in the
// normal range of FP16 (smallest normal 6.1e-5) instead of its subnormals.
// Arithmetic is FP32 in every case; the scaling is exact (powers of two).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

namespace llb {

template <class S>
struct IsNarrow : std::false_type {};
template <>
struct IsNarrow<__half> : std::true_type {};
template <>
struct IsNarrow<__nv_bfloat16> : std::true_type {};

// Scale of field f (one-component order d, jx, jy, jz, Axx..Ayz) in 16-bit storage.
__host__ __device__ constexpr float narrow_scale(int f) { return f == 0 ? 64.0f : (f < 4 ? 16.0f : 1024.0f); }

// Value of field f from its stored element.
template <class T, class S>
__device__ __forceinline__ T cv_field(S v, int f) {
    if constexpr (std::is_same<S, __half>::value)
        return T(__half2float(v)) * T(1.0f / narrow_scale(f));
    else if constexpr (std::is_same<S, __nv_bfloat16>::value)
        return T(__bfloat162float(v)) * T(1.0f / narrow_scale(f));
    else
        return T(v);
}

template <class T, class S>
__device__ __forceinline__ T ld_field(const S* p, int f) {
    return cv_field<T>(__ldg(p), f);
}

// Plain (non-__ldg) read, for buffers written earlier in the same kernel.
template <class S>
__device__ __forceinline__ double rd_field(const S& v, int f) {
    if constexpr (std::is_same<S, __half>::value)
        return (double)__half2float(v) / (double)narrow_scale(f);
    else if constexpr (std::is_same<S, __nv_bfloat16>::value)
        return (double)__bfloat162float(v) / (double)narrow_scale(f);
    else
        return (double)v;
}

template <class S, class T>
__device__ __forceinline__ S to_store(T v, int f) {
    if constexpr (std::is_same<S, __half>::value)
        return __float2half_rn(float(v) * narrow_scale(f));
    else if constexpr (std::is_same<S, __nv_bfloat16>::value)
        return __float2bfloat16_rn(float(v) * narrow_scale(f));
    else
        return S(v);
}

}  // namespace llb
