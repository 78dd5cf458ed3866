// FFT pass kernels of the Bloch stiffness and mass operators.
//
// Stiffness operator A_k (Eq. hatA, component form), Fourier basis in and out,
// five HBM passes with the pointwise work fused into the FFT passes:
//   pass 1  z: gamma_c = (q (x) U + U (x) q)_c in Voigt order (engineering
//            shear), inverse FFT along z                       3c in, 6c out
//   pass 2  y: inverse FFT along y, 6 components in place      6c in, 6c out
//   pass 3  x: inverse FFT along x, sigma = C_g(x) gamma / V,
//            forward FFT along x, in place                      6c + id in, 6c out
//   pass 4  y: forward FFT along y, in place                    6c in, 6c out
//   pass 5  z: forward FFT along z, divergence
//            out_i = sum_j q_j sigma_ij                         6c in, 3c out
// with q = xi + k.  The factor 1/V of F^-1 and the unit scaling are folded
// into the per-grain stiffness table.  Mass operator with non-uniform rho: the
// same chain on the three displacement components with rho_g(x)/V in pass 3.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace bloch {

// Division of n < 2^31 by an invariant divisor d >= 1 with one high multiply,
// an add and a shift (Granlund & Montgomery 1994, division by invariant
// integers): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(m, n) + n) >> l.
struct FastDiv {
    unsigned m = 1;
    int l = 0;
};
inline FastDiv make_fastdiv(unsigned d) {
    FastDiv f;
    int l = 0;
    while ((1ull << l) < (unsigned long long)d) ++l;
    f.l = l;
    f.m = (unsigned)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    return f;
}
__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) { return (__umulhi(f.m, n) + n) >> f.l; }

struct Geo {
    int Nx, Ny, Nz;
    long long V;
    AxisPlan ax[3];
    FastDiv dx, dy;   // division by Nx and by Ny
    // PCG convergence mask: system b is skipped when skip[b * skip_stride] == 0
    // (nullptr: every system runs); blockIdx.y / skip_ncomp is the system of a
    // per-component pass.
    const int* skip = nullptr;
    int skip_stride = 1;
    int skip_ncomp = 1;
    // plan error word: a pass whose staging wait runs out sets it (nullptr: none)
    int* err = nullptr;
};

__device__ __forceinline__ bool sys_idle(const Geo& g, int b) {
    return g.skip != nullptr && g.skip[(size_t)b * g.skip_stride] == 0;
}

__device__ __forceinline__ int pad_even(int n) { return (n + 1) & ~1; }

// ---------------------------------------------------------------- pass 1
template <typename T>
__global__ void __launch_bounds__(256, (sizeof(T) == 8) ? 2 : 1) k_pass_z_strain(const cplx_t<T>* __restrict__ U, cplx_t<T>* __restrict__ E,
                                                       const T* __restrict__ qtab, const cplx_t<T>* __restrict__ twz,
                                                       Geo g, int P) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int N = g.Nz;
    const int NP = N * P;
    C* tw = sm;
    C* sU = tw + pad_even(N);
    C* sA = sU + 3 * NP;
    C* sB = sA + NP;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int b = blockIdx.y;
    if (sys_idle(g, b)) return;
    const long long plane = (long long)g.Nx * g.Ny;
    const long long pi0 = (long long)blockIdx.x * P;
    const int np = (int)min((long long)P, plane - pi0);
    const C* Ub = U + (size_t)b * 3 * g.V;
    C* Eb = E + (size_t)b * 6 * g.V;
    const T* qx = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    const T* qy = qx + g.Nx;
    const T* qz = qy + g.Ny;
    const C zero = mk(T(0), T(0));

    for (int i = tid; i < N; i += nthr) tw[i] = twz[i];
    for (int e = tid; e < 3 * NP; e += nthr) {
        const int c = e / NP, r = e - c * NP, n = r / P, p = r - n * P;
        sU[e] = (p < np) ? Ub[(size_t)c * g.V + (size_t)n * plane + pi0 + p] : zero;
    }
    __syncthreads();
    for (int c = 0; c < 6; ++c) {
        for (int e = tid; e < NP; e += nthr) {
            const int n = e / P, p = e - n * P;
            const long long pi = pi0 + (p < np ? p : 0);
            const int x = (int)(pi % g.Nx), y = (int)(pi / g.Nx);
            const T ax = qx[x], ay = qy[y], az = qz[n];
            const C ux = sU[e], uy = sU[NP + e], uz = sU[2 * NP + e];
            C v;
            switch (c) {
                case 0: v = cscale(ux, ax); break;
                case 1: v = cscale(uy, ay); break;
                case 2: v = cscale(uz, az); break;
                case 3: v = cadd(cscale(uy, az), cscale(uz, ay)); break;
                case 4: v = cadd(cscale(ux, az), cscale(uz, ax)); break;
                default: v = cadd(cscale(ux, ay), cscale(uy, ax)); break;
            }
            sA[e] = v;
        }
        __syncthreads();
        C* res = fft_tile<+1, true>(sA, sB, g.ax[2], P, 0, tw, tid, nthr);
        for (int e = tid; e < NP; e += nthr) {
            const int n = e / P, p = e - n * P;
            if (p < np) Eb[(size_t)c * g.V + (size_t)n * plane + pi0 + p] = res[e];
        }
        __syncthreads();
    }
}

// ------------------------------------------------- plain FFT pass along y or z
// blockIdx.y enumerates (batch, component) pairs: offset blockIdx.y * V.
template <typename T, int DIR, int AXIS>
__global__ void __launch_bounds__(256) k_pass_axis(const cplx_t<T>* in, cplx_t<T>* out,
                                                   const cplx_t<T>* __restrict__ twa, Geo g, int P,
                                                   T out_scale) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int N = AXIS == 1 ? g.Ny : g.Nz;
    const int NP = N * P;
    C* tw = sm;
    C* sA = tw + pad_even(N);
    C* sB = sA + NP;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const long long npen = AXIS == 1 ? (long long)g.Nx * g.Nz : (long long)g.Nx * g.Ny;
    const long long pi0 = (long long)blockIdx.x * P;
    const int np = (int)min((long long)P, npen - pi0);
    if (sys_idle(g, (int)blockIdx.y / g.skip_ncomp)) return;
    const size_t off = (size_t)blockIdx.y * g.V;
    const C* src = in + off;
    C* dst = out + off;
    const long long plane = (long long)g.Nx * g.Ny;
    const C zero = mk(T(0), T(0));

    for (int i = tid; i < N; i += nthr) tw[i] = twa[i];
    for (int e = tid; e < NP; e += nthr) {
        const int n = e / P, p = e - n * P;
        C v = zero;
        if (p < np) {
            const long long pi = pi0 + p;
            size_t a;
            if (AXIS == 1) a = (size_t)(pi / g.Nx) * plane + (size_t)n * g.Nx + (size_t)(pi % g.Nx);
            else a = (size_t)n * plane + pi;
            v = src[a];
        }
        sA[e] = v;
    }
    __syncthreads();
    C* res = fft_tile<DIR, true>(sA, sB, g.ax[AXIS], P, 0, tw, tid, nthr);
    for (int e = tid; e < NP; e += nthr) {
        const int n = e / P, p = e - n * P;
        if (p < np) {
            const long long pi = pi0 + p;
            size_t a;
            if (AXIS == 1) a = (size_t)(pi / g.Nx) * plane + (size_t)n * g.Nx + (size_t)(pi % g.Nx);
            else a = (size_t)n * plane + pi;
            dst[a] = cscale(res[e], out_scale);
        }
    }
}

// ---------------------------------------------------------------- pass 3
// Rows along x; all six strain components of P rows in shared memory.
template <typename T>
__global__ void __launch_bounds__(256, (sizeof(T) == 8) ? 2 : 1) k_pass_x_stress(cplx_t<T>* E, const int32_t* __restrict__ ids,
                                                       const T* __restrict__ Ctab,
                                                       const cplx_t<T>* __restrict__ twx, Geo g, int P) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int N = g.Nx;
    const int NP = N * P;
    C* tw = sm;
    C* s0 = tw + pad_even(N);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int b = blockIdx.y;
    if (sys_idle(g, b)) return;
    const long long rows = (long long)g.Ny * g.Nz;
    const long long r0 = (long long)blockIdx.x * P;
    const int nr = (int)min((long long)P, rows - r0);
    C* Eb = E + (size_t)b * 6 * g.V;
    const C zero = mk(T(0), T(0));

    for (int i = tid; i < N; i += nthr) tw[i] = twx[i];
    for (int e = tid; e < 6 * NP; e += nthr) {
        const int c = e / NP, r = e - c * NP, p = r / N, n = r - p * N;
        s0[e] = (p < nr) ? Eb[(size_t)c * g.V + (size_t)(r0 + p) * N + n] : zero;
    }
    __syncthreads();
    C* buf[6];
    C* wk = s0 + 6 * NP;
#pragma unroll 1
    for (int c = 0; c < 6; ++c) {
        C* a = s0 + c * NP;
        C* res = fft_tile<+1, false>(a, wk, g.ax[0], P, N, tw, tid, nthr);
        if (res == wk) wk = a;
        buf[c] = res;
    }
    for (int e = tid; e < NP; e += nthr) {
        const int p = e / N, n = e - p * N;
        if (p < nr) {
            const int gid = ids[(size_t)(r0 + p) * N + n];
            const T* Cg = Ctab + (size_t)gid * 36;
            C gam[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) gam[c] = buf[c][e];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                T sr = 0, si = 0;
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    const T cij = ldg_t(Cg + i * 6 + j);
                    sr = fma(cij, gam[j].x, sr);
                    si = fma(cij, gam[j].y, si);
                }
                buf[i][e] = mk(sr, si);
            }
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < 6; ++c) {
        C* a = buf[c];
        C* res = fft_tile<-1, false>(a, wk, g.ax[0], P, N, tw, tid, nthr);
        if (res == wk) wk = a;
        buf[c] = res;
    }
    for (int e = tid; e < 6 * NP; e += nthr) {
        const int c = e / NP, r = e - c * NP, p = r / N, n = r - p * N;
        if (p < nr) Eb[(size_t)c * g.V + (size_t)(r0 + p) * N + n] = buf[c][r];
    }
}

// ---------------------------------------------------------------- pass 5
template <typename T>
__global__ void __launch_bounds__(256) k_pass_z_div(const cplx_t<T>* __restrict__ E, cplx_t<T>* __restrict__ out,
                                                    const T* __restrict__ qtab, const cplx_t<T>* __restrict__ twz,
                                                    Geo g, int P, T out_scale) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int N = g.Nz;
    const int NP = N * P;
    C* tw = sm;
    C* so = tw + pad_even(N);
    C* sA = so + 3 * NP;
    C* sB = sA + NP;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int b = blockIdx.y;
    if (sys_idle(g, b)) return;
    const long long plane = (long long)g.Nx * g.Ny;
    const long long pi0 = (long long)blockIdx.x * P;
    const int np = (int)min((long long)P, plane - pi0);
    const C* Eb = E + (size_t)b * 6 * g.V;
    C* ob = out + (size_t)b * 3 * g.V;
    const T* qx = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    const T* qy = qx + g.Nx;
    const T* qz = qy + g.Ny;
    const C zero = mk(T(0), T(0));

    for (int i = tid; i < N; i += nthr) tw[i] = twz[i];
    for (int e = tid; e < 3 * NP; e += nthr) so[e] = zero;
    for (int c = 0; c < 6; ++c) {
        for (int e = tid; e < NP; e += nthr) {
            const int n = e / P, p = e - n * P;
            sA[e] = (p < np) ? Eb[(size_t)c * g.V + (size_t)n * plane + pi0 + p] : zero;
        }
        __syncthreads();
        C* res = fft_tile<-1, true>(sA, sB, g.ax[2], P, 0, tw, tid, nthr);
        for (int e = tid; e < NP; e += nthr) {
            const int n = e / P, p = e - n * P;
            const long long pi = pi0 + (p < np ? p : 0);
            const int x = (int)(pi % g.Nx), y = (int)(pi / g.Nx);
            const T ax = qx[x], ay = qy[y], az = qz[n];
            const C s = res[e];
            C* ox = so + e;
            C* oy = so + NP + e;
            C* oz = so + 2 * NP + e;
            switch (c) {
                case 0: *ox = cadd(*ox, cscale(s, ax)); break;
                case 1: *oy = cadd(*oy, cscale(s, ay)); break;
                case 2: *oz = cadd(*oz, cscale(s, az)); break;
                case 3: *oy = cadd(*oy, cscale(s, az)); *oz = cadd(*oz, cscale(s, ay)); break;
                case 4: *ox = cadd(*ox, cscale(s, az)); *oz = cadd(*oz, cscale(s, ax)); break;
                default: *ox = cadd(*ox, cscale(s, ay)); *oy = cadd(*oy, cscale(s, ax)); break;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < 3 * NP; e += nthr) {
        const int c = e / NP, r = e - c * NP, n = r / P, p = r - n * P;
        if (p < np) ob[(size_t)c * g.V + (size_t)n * plane + pi0 + p] = cscale(so[e], out_scale);
    }
}

// ------------------------------------------- mass operator, non-uniform rho
template <typename T>
__global__ void __launch_bounds__(256) k_pass_x_rho(cplx_t<T>* W, const int32_t* __restrict__ ids,
                                                    const T* __restrict__ rtab,
                                                    const cplx_t<T>* __restrict__ twx, Geo g, int P) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int N = g.Nx;
    const int NP = N * P;
    C* tw = sm;
    C* s0 = tw + pad_even(N);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int b = blockIdx.y;
    if (sys_idle(g, b)) return;
    const long long rows = (long long)g.Ny * g.Nz;
    const long long r0 = (long long)blockIdx.x * P;
    const int nr = (int)min((long long)P, rows - r0);
    C* Wb = W + (size_t)b * 3 * g.V;
    const C zero = mk(T(0), T(0));

    for (int i = tid; i < N; i += nthr) tw[i] = twx[i];
    for (int e = tid; e < 3 * NP; e += nthr) {
        const int c = e / NP, r = e - c * NP, p = r / N, n = r - p * N;
        s0[e] = (p < nr) ? Wb[(size_t)c * g.V + (size_t)(r0 + p) * N + n] : zero;
    }
    __syncthreads();
    C* buf[3];
    C* wk = s0 + 3 * NP;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        C* a = s0 + c * NP;
        C* res = fft_tile<+1, false>(a, wk, g.ax[0], P, N, tw, tid, nthr);
        if (res == wk) wk = a;
        buf[c] = res;
    }
    for (int e = tid; e < NP; e += nthr) {
        const int p = e / N, n = e - p * N;
        if (p < nr) {
            const T r = ldg_t(rtab + ids[(size_t)(r0 + p) * N + n]);
#pragma unroll
            for (int c = 0; c < 3; ++c) buf[c][e] = cscale(buf[c][e], r);
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        C* a = buf[c];
        C* res = fft_tile<-1, false>(a, wk, g.ax[0], P, N, tw, tid, nthr);
        if (res == wk) wk = a;
        buf[c] = res;
    }
    for (int e = tid; e < 3 * NP; e += nthr) {
        const int c = e / NP, r = e - c * NP, p = r / N, n = r - p * N;
        if (p < nr) Wb[(size_t)c * g.V + (size_t)(r0 + p) * N + n] = buf[c][r];
    }
}

// ------------------------------------------- plain transform along x
// 1D FFT (DIR -1 forward, +1 inverse, unnormalised) of the three components
// of nb systems along x, in place, times out_scale; rows are contiguous, P
// rows per CTA, blockIdx.y = system.
template <typename T, int DIR>
__global__ void __launch_bounds__(256) k_pass_x(cplx_t<T>* W, const cplx_t<T>* __restrict__ twx, Geo g, int P,
                                                T out_scale) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int N = g.Nx;
    const int NP = N * P;
    C* tw = sm;
    C* s0 = tw + pad_even(N);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int b = blockIdx.y;
    const long long rows = (long long)g.Ny * g.Nz;
    const long long r0 = (long long)blockIdx.x * P;
    const int nr = (int)min((long long)P, rows - r0);
    C* Wb = W + (size_t)b * 3 * g.V;
    const C zero = mk(T(0), T(0));
    for (int i = tid; i < N; i += nthr) tw[i] = twx[i];
    for (int e = tid; e < 3 * NP; e += nthr) {
        const int c = e / NP, r = e - c * NP, p = r / N, n = r - p * N;
        s0[e] = (p < nr) ? Wb[(size_t)c * g.V + (size_t)(r0 + p) * N + n] : zero;
    }
    __syncthreads();
    C* buf[3];
    C* wk = s0 + 3 * NP;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        C* a = s0 + c * NP;
        C* res = fft_tile<DIR, false>(a, wk, g.ax[0], P, N, tw, tid, nthr);
        if (res == wk) wk = a;
        buf[c] = res;
    }
    __syncthreads();
    for (int e = tid; e < 3 * NP; e += nthr) {
        const int c = e / NP, r = e - c * NP, p = r / N, n = r - p * N;
        if (p < nr) Wb[(size_t)c * g.V + (size_t)(r0 + p) * N + n] = cscale(buf[c][r], out_scale);
    }
}

}  // namespace bloch
