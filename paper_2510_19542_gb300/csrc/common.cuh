// Device helpers shared by the frame kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace safr {

// The dynamic shared-memory limit of a kernel is a property of the kernel, shared
// by every plan that launches it.  Raise it once to everything the device allows
// next to the kernel's static shared memory (never lower it: a later plan with a
// smaller need must not break an earlier one), and report whether `need` fits:
// 1 it fits, 0 it is more than the device allows, -1 a CUDA call failed.
inline int smem_fit(const void *kernel, size_t need)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    const int avail = optin - (int)fa.sharedSizeBytes;
    if (need > (size_t)avail) return 0;
    if (fa.maxDynamicSharedSizeBytes < avail &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, avail) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return 1;
}

inline bool smem_limit_allows(const void *kernel, size_t need) { return smem_fit(kernel, need) == 1; }

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename T>
__device__ __forceinline__ float to_real(T v);
template <>
__device__ __forceinline__ float to_real<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_real<__half>(__half v) { return __half2float(v); }

template <typename R, typename T>
__device__ __forceinline__ R load_in(const T *p) { return (R)to_real<T>(*p); }
template <>
__device__ __forceinline__ double load_in<double, double>(const double *p) { return *p; }

// the same through L2 only (data another CTA of the same launch may have written)
template <typename R, typename T>
__device__ __forceinline__ R load_in_cg(const T *p) { return (R)to_real<T>(__ldcg(p)); }
template <>
__device__ __forceinline__ double load_in_cg<double, double>(const double *p) { return __ldcg(p); }

template <typename R>
__device__ __forceinline__ R block_sum(R v, R *red)
{
    // deterministic: fixed shuffle tree, then fixed order over warps
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    R t = 0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) t += red[i];
    return t;
}

template <typename TOUT>
__device__ __forceinline__ void store_out(TOUT *p, float v);
template <>
__device__ __forceinline__ void store_out<float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void store_out<__half>(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void store_out_d(double *p, double v) { *p = v; }

}  // namespace safr
