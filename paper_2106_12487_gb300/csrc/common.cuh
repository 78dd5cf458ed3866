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

#define BLOCH_CUDA_CHECK_RET(expr)                                  \
    do {                                                            \
        cudaError_t _e = (expr);                                    \
        if (_e != cudaSuccess) return set_cuda_error(_e, #expr);    \
    } while (0)
