// Storage precision of the scalar fields (images, states, their gradients,
// adjoint levels, incremental fields): FP32, FP16 or BF16.  Arithmetic is
// always FP32; these helpers convert on load and store.  Internal header.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace claire {

enum class Storage : int { F32 = 0, F16 = 1, BF16 = 2 };

inline size_t storage_bytes(Storage s) { return s == Storage::F32 ? 4 : 2; }

template <class S>
__device__ __forceinline__ float to_f32(S v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class S>
__device__ __forceinline__ S from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// read-only cached load of one stored value, as FP32
template <class S>
__device__ __forceinline__ float ldf(const S* p) { return to_f32<S>(__ldg(p)); }

template <class S>
__device__ __forceinline__ void stf(S* p, float v) { *p = from_f32<S>(v); }

}  // namespace claire

// Dispatch a template body on the runtime storage type: defines the type
// alias SType inside the body.
#define CLAIRE_STORAGE_DISPATCH(storage, ...)            \
    do {                                                 \
        switch (storage) {                               \
        case ::claire::Storage::F16: {                   \
            using SType = __half;                        \
            __VA_ARGS__;                                 \
        } break;                                         \
        case ::claire::Storage::BF16: {                  \
            using SType = __nv_bfloat16;                 \
            __VA_ARGS__;                                 \
        } break;                                         \
        default: {                                       \
            using SType = float;                         \
            __VA_ARGS__;                                 \
        } break;                                         \
        }                                                \
    } while (0)
