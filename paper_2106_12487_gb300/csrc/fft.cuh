// Shared-memory Stockham FFT of a tile of pencils.
//
// A CTA holds P pencils of length N in shared memory and transforms all of
// them along their length with a mixed-radix Stockham autosort (out-of-place
// between two shared buffers, one barrier per stage).  Each thread owns one
// radix-R butterfly at a time: R values are read, multiplied by the stage
// twiddles, transformed in registers and written to their sorted position.
// The stage formulation is the Stockham autosort used for GPU FFTs by
// Govindaraju et al. (SC 2008): with Ns the product of the radices already
// applied, butterfly j reads x[j + r N/R] (r < R), twiddles by
// w_{Ns R}^{r (j mod Ns)}, and writes X[(j div Ns) Ns R + (j mod Ns) + r Ns].
//
// Radix kernels: powers of two (2..16) by unrolled radix-2 decimation in time
// with literal twiddles; 3, 5, 7 by a direct DFT (small test grids only).
// Direction: DIR = -1 forward (exp(-2 pi i ...)), DIR = +1 inverse; both
// unnormalised.
#pragma once

#include "common.cuh"

namespace bloch {

constexpr int kMaxStages = 12;

struct AxisPlan {
    int N;
    int nst;
    int radix[kMaxStages];
};

// cos(2 pi m / 16), m taken modulo 16
template <typename R>
__device__ __forceinline__ R cos16(int m) {
    switch (m & 15) {
        case 0: return R(1.0);
        case 1: case 15: return R(0.92387953251128675613);
        case 2: case 14: return R(0.70710678118654752440);
        case 3: case 13: return R(0.38268343236508977173);
        case 4: case 12: return R(0.0);
        case 5: case 11: return R(-0.38268343236508977173);
        case 6: case 10: return R(-0.70710678118654752440);
        case 7: case 9: return R(-0.92387953251128675613);
        default: return R(-1.0);
    }
}

// float-float values: hi = cos rounded to float, lo = the rounded remainder
template <>
__device__ __forceinline__ dfloat cos16<dfloat>(int m) {
    switch (m & 15) {
        case 0: return dfloat(1.0f, 0.0f);
        case 1: case 15: return dfloat(0.9238795042037964f, 2.830748968563057e-08f);
        case 2: case 14: return dfloat(0.7071067690849304f, 1.2101617485882343e-08f);
        case 3: case 13: return dfloat(0.3826834261417389f, 6.2233507236442165e-09f);
        case 4: case 12: return dfloat(0.0f, 0.0f);
        case 5: case 11: return dfloat(-0.3826834261417389f, -6.2233507236442165e-09f);
        case 6: case 10: return dfloat(-0.7071067690849304f, -1.2101617485882343e-08f);
        case 7: case 9: return dfloat(-0.9238795042037964f, -2.830748968563057e-08f);
        default: return dfloat(-1.0f, 0.0f);
    }
}

// x * exp(DIR * 2 pi i k / R) for power-of-two R <= 16 (k compile-time after unrolling)
template <int R, int DIR, typename C>
__device__ __forceinline__ C twiddle_pow2(C x, int k) {
    using T = decltype(x.x);
    if (k == 0) return x;
    if (4 * k == R) return cmul_i<DIR>(x);
    const int m = k * (16 / R);
    const T c = cos16<T>(m);
    const T s = T(DIR) * cos16<T>(m - 4);   // sin(2 pi m/16) = cos(2 pi (m-4)/16)
    return mk(x.x * c - x.y * s, x.x * s + x.y * c);
}

template <int R, int DIR, typename C>
struct RegDFT {
    __device__ __forceinline__ static void run(C* v) {
        if constexpr (R == 1) {
            return;
        } else if constexpr (R == 2) {
            C a = v[0], b = v[1];
            v[0] = cadd(a, b);
            v[1] = csub(a, b);
        } else if constexpr ((R & (R - 1)) == 0) {
            constexpr int H = R / 2;
            C e[H], o[H];
#pragma unroll
            for (int i = 0; i < H; ++i) {
                e[i] = v[2 * i];
                o[i] = v[2 * i + 1];
            }
            RegDFT<H, DIR, C>::run(e);
            RegDFT<H, DIR, C>::run(o);
#pragma unroll
            for (int k = 0; k < H; ++k) {
                C t = twiddle_pow2<R, DIR>(o[k], k);
                v[k] = cadd(e[k], t);
                v[k + H] = csub(e[k], t);
            }
        } else {
            // direct DFT for odd radices 3, 5, 7
            using T = decltype(v[0].x);
            C out[R];
#pragma unroll
            for (int k = 0; k < R; ++k) {
                C acc = v[0];
#pragma unroll
                for (int n = 1; n < R; ++n) {
                    double s, c;
                    sincospi(2.0 * double((n * k) % R) / double(R), &s, &c);
                    C w = mk(T(c), T(DIR) * T(s));
                    acc = cadd(acc, cmul(v[n], w));
                }
                out[k] = acc;
            }
#pragma unroll
            for (int k = 0; k < R; ++k) v[k] = out[k];
        }
    }
};

// Element (p, n) of a tile: pencil-fastest layout (PF) n*P + p, or
// length-fastest layout (LF) p*ld + n.
template <bool PF>
__device__ __forceinline__ int tile_idx(int p, int n, int P, int ld) {
    return PF ? n * P + p : p * ld + n;
}

// One Stockham stage of radix R over all P pencils of the tile.
// tw: table of exp(-2 pi i t / N), t < N (shared memory).
template <int R, int DIR, bool PF, typename C>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ src, C* __restrict__ dst, int N, int P,
                                               int ld, int Ns, const C* __restrict__ tw, int tid, int nthr) {
    const int NR = N / R;
    const int tasks = NR * P;
    const int twstep = N / (Ns * R);
    for (int t = tid; t < tasks; t += nthr) {
        int p, j;
        if (PF) {
            p = t % P;
            j = t / P;
        } else {
            j = t % NR;
            p = t / NR;
        }
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[tile_idx<PF>(p, j + r * NR, P, ld)];
        const int jm = j % Ns;
        if (Ns > 1) {
            const int base = jm * twstep;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = tw[r * base];
                if (DIR > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        RegDFT<R, DIR, C>::run(v);
        const int o = (j - jm) * R + jm;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[tile_idx<PF>(p, o + r * Ns, P, ld)] = v[r];
    }
}

// Odd radices only serve small test grids: keep them out of line so that
// their direct DFT does not raise the register allocation of the kernels.
template <int R, int DIR, bool PF, typename C>
__device__ __noinline__ void stockham_stage_odd(const C* __restrict__ src, C* __restrict__ dst, int N, int P, int ld,
                                                int Ns, const C* __restrict__ tw, int tid, int nthr) {
    stockham_stage<R, DIR, PF>(src, dst, N, P, ld, Ns, tw, tid, nthr);
}

// Transform every pencil of the tile held in `a`, using `b` as the second
// buffer.  Returns the buffer that holds the result (a or b).  Contains the
// barriers between stages; the caller must have synchronised after filling a.
template <int DIR, bool PF, typename C>
__device__ C* fft_tile(C* a, C* b, const AxisPlan& ap, int P, int ld, const C* tw, int tid, int nthr) {
    C* src = a;
    C* dst = b;
    int Ns = 1;
    for (int s = 0; s < ap.nst; ++s) {
        const int R = ap.radix[s];
        switch (R) {
            case 2: stockham_stage<2, DIR, PF>(src, dst, ap.N, P, ld, Ns, tw, tid, nthr); break;
            case 4: stockham_stage<4, DIR, PF>(src, dst, ap.N, P, ld, Ns, tw, tid, nthr); break;
            case 8: stockham_stage<8, DIR, PF>(src, dst, ap.N, P, ld, Ns, tw, tid, nthr); break;
            case 16: stockham_stage<16, DIR, PF>(src, dst, ap.N, P, ld, Ns, tw, tid, nthr); break;
            case 3: stockham_stage_odd<3, DIR, PF>(src, dst, ap.N, P, ld, Ns, tw, tid, nthr); break;
            case 5: stockham_stage_odd<5, DIR, PF>(src, dst, ap.N, P, ld, Ns, tw, tid, nthr); break;
            case 7: stockham_stage_odd<7, DIR, PF>(src, dst, ap.N, P, ld, Ns, tw, tid, nthr); break;
            default: break;
        }
        __syncthreads();
        C* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

}  // namespace bloch
