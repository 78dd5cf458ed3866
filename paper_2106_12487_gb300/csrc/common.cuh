// Shared device helpers: complex arithmetic on float2/double2 and type traits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };

template <typename T> using cplx_t = typename CplxOf<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) {
    return mk(a.x * s, a.y * s);
}
// multiply by -i (forward) or +i (inverse):  DIR = -1 -> -i, DIR = +1 -> +i
template <int DIR, typename C> __host__ __device__ __forceinline__ C cmul_i(C a) {
    return DIR < 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);
}

// Asynchronous global -> shared copy of one complex value (8 or 16 bytes);
// src_valid = false fills zeros without reading.
template <typename C>
__device__ __forceinline__ void cp_async_cplx(C* smem, const C* gmem, bool src_valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = src_valid ? (int)sizeof(C) : 0;
    if (sizeof(C) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Let launches of kernel k request the device's whole opt-in shared memory
// per block, less what k declares statically.
template <typename K>
inline cudaError_t allow_max_dyn_smem(K k) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes a;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
    return e;
}

#define BLOCH_CUDA_CHECK_RET(expr)                                  \
    do {                                                            \
        cudaError_t _e = (expr);                                    \
        if (_e != cudaSuccess) return set_cuda_error(_e, #expr);    \
    } while (0)
