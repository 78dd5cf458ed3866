// Shared device helpers: complex arithmetic on float2/double2 and type traits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Float-float ("double-float") real: the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, a 48-bit significand evaluated on the FP32
// pipes.  Sum and product are formed from the error-free transformations --
// Knuth's two-sum (s + e = a + b exactly) and, for the product, the residual
// of a*b recovered with one fused multiply-add (Dekker's product) -- then
// renormalised.  The
// _rn intrinsics keep every step individually rounded (no contraction).
struct dfloat {
    float hi, lo;
    __host__ __device__ dfloat() : hi(0.f), lo(0.f) {}
    __host__ __device__ dfloat(float a) : hi(a), lo(0.f) {}
    __host__ __device__ dfloat(int a) : hi((float)a), lo(0.f) {}
    __host__ __device__ dfloat(double a) : hi((float)a), lo((float)(a - (double)(float)a)) {}
    __host__ __device__ dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ explicit operator float() const { return hi + lo; }
};

#ifdef __CUDACC__
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfloat(s, e);
}
__device__ __forceinline__ dfloat df_quick_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// The low parts are added without their own error term: the sum is then
// accurate to about 2^-48 of the larger operand (a normwise bound, the form
// FFT error analysis uses) rather than of the result.
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, b.hi);
    return df_quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_quick_two_sum(p, e);
}
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }
__device__ __forceinline__ bool operator==(dfloat a, dfloat b) { return a.hi == b.hi && a.lo == b.lo; }
#endif

struct dfloat2 {
    dfloat x, y;
};

#ifdef __CUDACC__
// read-only cached load of a real table entry of any of the field types
// Store of a streamed FP32 complex value that takes no L1 line.
__device__ __forceinline__ void st_stream(float2* p, float2 v) {
    asm volatile("st.global.L1::no_allocate.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ float ldg_t(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ldg_t(const double* p) { return __ldg(p); }
__device__ __forceinline__ dfloat ldg_t(const dfloat* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return dfloat(v.x, v.y);
}
#endif

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <> struct CplxOf<dfloat> { using type = dfloat2; };

template <typename T> using cplx_t = typename CplxOf<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ dfloat2 mk(dfloat a, dfloat b) { return dfloat2{a, b}; }

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
// Asynchronous 16-byte global -> shared copy that bypasses L1 (both
// addresses 16-byte aligned); src_valid = false fills zeros without reading.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool src_valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_valid ? 16 : 0));
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
