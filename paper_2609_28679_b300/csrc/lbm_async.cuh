// Asynchronous 16-byte global-to-shared copies (cp.async) and the small
// helpers the staged kernels share: stored-to-float conversion and floor
// division for chunk-aligned staging origins.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace lbm {

__device__ __forceinline__ void cp_async16(const void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename S> __device__ __forceinline__ float stored_to_f(S v);
template <> __device__ __forceinline__ float stored_to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float stored_to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ float stored_to_f<__half>(__half v) { return __half2float(v); }

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

}  // namespace lbm
