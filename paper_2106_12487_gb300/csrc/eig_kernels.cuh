// Block kernels of the eigensolvers: Gram projections, basis rotation,
// Rayleigh quotients and residuals of a block of vectors (Algorithm 1 steps
// K = conj(U^T) Kn, M = conj(U^T) Mn, U <- U Q, err2).
#pragma once

#include "common.cuh"
#include "vec.cuh"

namespace bloch {

constexpr int kGramChunk = 32;
constexpr int kQMax = 32;

// partial[slot][blk][i][j] = sum_e conj(A[slot][i][e]) B[slot][j][e], i, j < q.
// Vectors of one slot are contiguous: A + (slot*q + i)*n_per.
template <typename T>
__global__ void __launch_bounds__(256) k_gram(const cplx_t<T>* __restrict__ A, const cplx_t<T>* __restrict__ B, int q,
                                              long long n_per, double2* __restrict__ partial) {
    using C = cplx_t<T>;
    __shared__ C sA[kQMax][kGramChunk];
    __shared__ C sB[kQMax][kGramChunk];
    const int slot = blockIdx.y;
    const C* Ab = A + (size_t)slot * q * n_per;
    const C* Bb = B + (size_t)slot * q * n_per;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int npair = q * q;
    T acc[4][2];
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s][0] = acc[s][1] = T(0);
    const long long nchunk = (n_per + kGramChunk - 1) / kGramChunk;
    for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const long long e0 = ch * kGramChunk;
        for (int t = tid; t < q * kGramChunk; t += nthr) {
            const int i = t / kGramChunk, c = t - i * kGramChunk;
            const long long e = e0 + c;
            const C z = mk(T(0), T(0));
            sA[i][c] = e < n_per ? Ab[(size_t)i * n_per + e] : z;
            sB[i][c] = e < n_per ? Bb[(size_t)i * n_per + e] : z;
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int pr = tid + s * nthr;
            if (pr < npair) {
                const int i = pr / q, j = pr - i * q;
                T re = acc[s][0], im = acc[s][1];
#pragma unroll 8
                for (int c = 0; c < kGramChunk; ++c) {
                    const C a = sA[i][c], b = sB[j][c];
                    re = fma(a.x, b.x, fma(a.y, b.y, re));
                    im = fma(a.x, b.y, fma(-a.y, b.x, im));
                }
                acc[s][0] = re;
                acc[s][1] = im;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int pr = tid + s * nthr;
        if (pr < npair)
            partial[((size_t)slot * gridDim.x + blockIdx.x) * npair + pr] = make_double2(acc[s][0], acc[s][1]);
    }
}

// Register-tiled Gram: each thread owns a 4x4 tile of (i, j) pairs and one
// group of elements of every chunk; element groups are reduced through shared
// memory at the end.  partial layout as k_gram.
constexpr int kG2Chunk = 64;
template <typename T>
__global__ void __launch_bounds__(256) k_gram2(const cplx_t<T>* __restrict__ A, const cplx_t<T>* __restrict__ B, int q,
                                               long long n_per, double2* __restrict__ partial) {
    using C = cplx_t<T>;
    constexpr int QP = kQMax;   // padded rows
    __shared__ C sA[QP][kG2Chunk];
    __shared__ C sB[QP][kG2Chunk];
    const int slot = blockIdx.y;
    const C* Ab = A + (size_t)slot * q * n_per;
    const C* Bb = B + (size_t)slot * q * n_per;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int side = (q + 3) / 4;
    const int ntile = side * side;
    const int G = nthr / ntile;           // element groups
    const int tile = tid % ntile, grp = tid / ntile;
    const bool act = grp < G;
    const int i0 = (tile / side) * 4, j0 = (tile % side) * 4;
    T acc[4][4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c][0] = acc[a][c][1] = T(0);
    const long long nchunk = (n_per + kG2Chunk - 1) / kG2Chunk;
    const int rows = side * 4;
    for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const long long e0 = ch * kG2Chunk;
        for (int t = tid; t < rows * kG2Chunk; t += nthr) {
            const int i = t / kG2Chunk, c = t - i * kG2Chunk;
            const long long e = e0 + c;
            const bool ok = i < q && e < n_per;
            sA[i][c] = ok ? Ab[(size_t)i * n_per + e] : mk(T(0), T(0));
            sB[i][c] = ok ? Bb[(size_t)i * n_per + e] : mk(T(0), T(0));
        }
        __syncthreads();
        if (act) {
            for (int e = grp; e < kG2Chunk; e += G) {
                C a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a[u] = sA[i0 + u][e];
                    b[u] = sB[j0 + u][e];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        acc[u][v][0] = fma(a[u].x, b[v].x, fma(a[u].y, b[v].y, acc[u][v][0]));
                        acc[u][v][1] = fma(a[u].x, b[v].y, fma(-a[u].y, b[v].x, acc[u][v][1]));
                    }
            }
        }
        __syncthreads();
    }
    // reduce the element groups: reuse sA as a [ntile][16] complex scratch per group pass
    double2* out = partial + ((size_t)slot * gridDim.x + blockIdx.x) * q * q;
    C* red = &sA[0][0];   // QP*kG2Chunk >= ntile*16 entries (ntile <= 64)
    for (int gsum = 0; gsum < G; ++gsum) {
        if (act && grp == gsum) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    C& r = red[tile * 16 + u * 4 + v];
                    if (gsum == 0) r = mk(acc[u][v][0], acc[u][v][1]);
                    else r = mk(r.x + acc[u][v][0], r.y + acc[u][v][1]);
                }
        }
        __syncthreads();
    }
    for (int t = tid; t < q * q; t += nthr) {
        const int i = t / q, j = t - i * q;
        const int tl = (i / 4) * side + (j / 4);
        const C r = red[tl * 16 + (i % 4) * 4 + (j % 4)];
        out[t] = make_double2(r.x, r.y);
    }
}

static __global__ void k_gram_final(const double2* __restrict__ partial, int nblk, int npair, double2* __restrict__ out) {
    const int slot = blockIdx.y;
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= npair) return;
    double re = 0, im = 0;
    for (int b = 0; b < nblk; ++b) {
        const double2 v = partial[((size_t)slot * nblk + b) * npair + pr];
        re += v.x;
        im += v.y;
    }
    out[(size_t)slot * npair + pr] = make_double2(re, im);
}

// Out[slot][j][e] = sum_i In[slot][i][e] Q[slot][i][j]  (Q row-major q x q, double2)
template <typename T>
__global__ void __launch_bounds__(128) k_basis(const cplx_t<T>* __restrict__ In, cplx_t<T>* __restrict__ Out,
                                               const double2* __restrict__ Q, int q, long long n_per) {
    using C = cplx_t<T>;
    __shared__ C sQ[kQMax * kQMax];
    const int slot = blockIdx.y;
    for (int t = threadIdx.x; t < q * q; t += blockDim.x) {
        const double2 v = Q[(size_t)slot * q * q + t];
        sQ[t] = mk(T(v.x), T(v.y));
    }
    __syncthreads();
    const C* ib = In + (size_t)slot * q * n_per;
    C* ob = Out + (size_t)slot * q * n_per;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_per;
         e += (long long)gridDim.x * blockDim.x) {
        C v[kQMax];
#pragma unroll
        for (int i = 0; i < kQMax; ++i)
            if (i < q) v[i] = ib[(size_t)i * n_per + e];
        for (int j = 0; j < q; ++j) {
            T re = 0, im = 0;
#pragma unroll
            for (int i = 0; i < kQMax; ++i)
                if (i < q) {
                    const C w = sQ[i * q + j];
                    re = fma(v[i].x, w.x, fma(-v[i].y, w.y, re));
                    im = fma(v[i].x, w.y, fma(v[i].y, w.x, im));
                }
            ob[(size_t)j * n_per + e] = mk(re, im);
        }
    }
}

// Per vector v (blockIdx.y): partial sums of Re(u^H Ku), u^H (M u), |Ku|^2.
// M u = MU[v] if MU is given, else rho_s * u.
template <typename TK>
__global__ void k_rq_dots(const cplx_t<TK>* __restrict__ U, const cplx_t<TK>* __restrict__ KU,
                          const cplx_t<TK>* __restrict__ MU, double rho_s, long long n_per, double* partial) {
    using C = cplx_t<TK>;
    const int v = blockIdx.y;
    const C* u = U + (size_t)v * n_per;
    const C* ku = KU + (size_t)v * n_per;
    const C* mu = MU ? MU + (size_t)v * n_per : nullptr;
    TK acc[3] = {TK(0), TK(0), TK(0)};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_per;
         i += (long long)gridDim.x * blockDim.x) {
        const C a = u[i], b = ku[i];
        acc[0] += a.x * b.x + a.y * b.y;
        if (mu) {
            const C m = mu[i];
            acc[1] += a.x * m.x + a.y * m.y;
        } else {
            acc[1] += TK(rho_s) * (a.x * a.x + a.y * a.y);
        }
        acc[2] += b.x * b.x + b.y * b.y;
    }
    block_sum<TK, 3>(acc);
    if (threadIdx.x == 0) {
        double* o = partial + ((size_t)v * gridDim.x + blockIdx.x) * 3;
        o[0] = acc[0];
        o[1] = acc[1];
        o[2] = acc[2];
    }
}

// R[v] = M u - Ku / lambda_v  (computed in TK, stored in TR); partial |R|^2.
template <typename TK, typename TR>
__global__ void k_residual(const cplx_t<TK>* __restrict__ U, const cplx_t<TK>* __restrict__ KU,
                           const cplx_t<TK>* __restrict__ MU, double rho_s, const double* __restrict__ inv_lam,
                           cplx_t<TR>* __restrict__ R, long long n_per, double* partial) {
    using C = cplx_t<TK>;
    const int v = blockIdx.y;
    const C* u = U + (size_t)v * n_per;
    const C* ku = KU + (size_t)v * n_per;
    const C* mu = MU ? MU + (size_t)v * n_per : nullptr;
    cplx_t<TR>* r = R + (size_t)v * n_per;
    const TK il = TK(inv_lam[v]);
    TK acc[1] = {TK(0)};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_per;
         i += (long long)gridDim.x * blockDim.x) {
        const C a = u[i], b = ku[i];
        const C m = mu ? mu[i] : mk(TK(rho_s) * a.x, TK(rho_s) * a.y);
        const TK rx = m.x - b.x * il, ry = m.y - b.y * il;
        r[i] = mk(TR(rx), TR(ry));
        acc[0] += rx * rx + ry * ry;
    }
    block_sum<TK, 1>(acc);
    if (threadIdx.x == 0) partial[(size_t)v * gridDim.x + blockIdx.x] = acc[0];
}

// X[v] += U[v] * s_v
template <typename T>
__global__ void k_add_scaled(cplx_t<T>* X, const cplx_t<T>* __restrict__ U, const double* __restrict__ s,
                             long long n_per) {
    const int v = blockIdx.y;
    const T sv = T(s[v]);
    cplx_t<T>* x = X + (size_t)v * n_per;
    const cplx_t<T>* u = U + (size_t)v * n_per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_per;
         i += (long long)gridDim.x * blockDim.x) {
        const cplx_t<T> a = u[i], b = x[i];
        x[i] = mk(fma(a.x, sv, b.x), fma(a.y, sv, b.y));
    }
}

// Kn = (MU or rho_s U) - r
template <typename T>
__global__ void k_kn(const cplx_t<T>* __restrict__ U, const cplx_t<T>* __restrict__ MU, double rho_s,
                     const cplx_t<T>* __restrict__ r, cplx_t<T>* __restrict__ Kn, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const cplx_t<T> m = MU ? MU[i] : cscale(U[i], T(rho_s));
        Kn[i] = csub(m, r[i]);
    }
}

template <typename Ta, typename Tb>
__global__ void k_convert(const cplx_t<Ta>* __restrict__ a, cplx_t<Tb>* __restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = mk(Tb(a[i].x), Tb(a[i].y));
}

// U[idx[i]] = val[i]
template <typename T>
__global__ void k_scatter(cplx_t<T>* U, const long long* __restrict__ idx, const double2* __restrict__ val, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) U[idx[i]] = mk(T(val[i].x), T(val[i].y));
}

// out[v] = in[v] * s_v (vectors of n_per elements), possibly converting precision
template <typename Ta, typename Tb>
__global__ void k_scale_vecs(const cplx_t<Ta>* __restrict__ in, cplx_t<Tb>* __restrict__ out,
                             const double* __restrict__ s, long long n_per) {
    const int v = blockIdx.y;
    const Ta sv = Ta(s[v]);
    const cplx_t<Ta>* a = in + (size_t)v * n_per;
    cplx_t<Tb>* b = out + (size_t)v * n_per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_per;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = mk(Tb(a[i].x * sv), Tb(a[i].y * sv));
}

}  // namespace bloch

namespace bloch {

// ------------------------------------------------------- Lanczos block kernels
// partial[(slot*nblk + blk)*maxnv + i] = sum_e conj(V[slot][i][e]) W[slot][e], i < nv[slot]
template <typename T>
__global__ void k_vdots(const cplx_t<T>* __restrict__ V, long long vstride, const cplx_t<T>* __restrict__ W,
                        long long wstride, const int* __restrict__ nv, long long n, int maxnv,
                        double2* __restrict__ partial) {
    using C = cplx_t<T>;
    const int i = blockIdx.y, slot = blockIdx.z;
    T acc[2] = {T(0), T(0)};
    if (i < nv[slot]) {
        const C* v = V + (size_t)slot * vstride + (size_t)i * n;
        const C* w = W + (size_t)slot * wstride;
        for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
             e += (long long)gridDim.x * blockDim.x) {
            const C a = v[e], b = w[e];
            acc[0] += a.x * b.x + a.y * b.y;
            acc[1] += a.x * b.y - a.y * b.x;
        }
    }
    block_sum<T, 2>(acc);
    if (threadIdx.x == 0)
        partial[((size_t)slot * gridDim.x + blockIdx.x) * maxnv + i] = make_double2(acc[0], acc[1]);
}

// h[slot][i] = scale * sum_blk partial
static __global__ void k_vdots_final(const double2* __restrict__ partial, int nblk, int maxnv, double scale,
                                     double2* __restrict__ h) {
    const int slot = blockIdx.x;
    for (int i = threadIdx.x; i < maxnv; i += blockDim.x) {
        double re = 0, im = 0;
        for (int b = 0; b < nblk; ++b) {
            const double2 v = partial[((size_t)slot * nblk + b) * maxnv + i];
            re += v.x;
            im += v.y;
        }
        h[(size_t)slot * maxnv + i] = make_double2(scale * re, scale * im);
    }
}

// W[slot] -= sum_{i < nv[slot]} V[slot][i] h[slot][i]
template <typename T>
__global__ void k_vaxpy(const cplx_t<T>* __restrict__ V, long long vstride, cplx_t<T>* __restrict__ W,
                        long long wstride, const double2* __restrict__ h, const int* __restrict__ nv, long long n,
                        int maxnv) {
    using C = cplx_t<T>;
    __shared__ C sh[64];
    const int slot = blockIdx.y;
    const int m = nv[slot];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double2 v = h[(size_t)slot * maxnv + i];
        sh[i] = mk(T(v.x), T(v.y));
    }
    __syncthreads();
    const C* vb = V + (size_t)slot * vstride;
    C* w = W + (size_t)slot * wstride;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        C acc = w[e];
        for (int i = 0; i < m; ++i) {
            const C a = vb[(size_t)i * n + e], c = sh[i];
            acc.x -= a.x * c.x - a.y * c.y;
            acc.y -= a.x * c.y + a.y * c.x;
        }
        w[e] = acc;
    }
}

// dst[slot] (at per-slot element offsets) = src[slot] * s[slot]
template <typename T>
__global__ void k_copy_scaled(const cplx_t<T>* __restrict__ src, const long long* __restrict__ src_off,
                              cplx_t<T>* __restrict__ dst, const long long* __restrict__ dst_off,
                              const double* __restrict__ s, long long n) {
    const int slot = blockIdx.y;
    const T sv = T(s[slot]);
    const cplx_t<T>* a = src + src_off[slot];
    cplx_t<T>* b = dst + dst_off[slot];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        b[e] = cscale(a[e], sv);
}

// Deterministic start vector: counter-based hash -> uniform in [-1, 1) per
// real and imaginary part; the bin xi = 0 is left empty at k = 0.
__device__ __forceinline__ unsigned int hash_u32(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return (unsigned int)x;
}

template <typename T>
__global__ void k_start_random(cplx_t<T>* v, long long n, long long V, unsigned long long seed, int skip_bin0) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const T re = T(hash_u32(seed * 0x9E3779B97F4A7C15ULL + 2 * e) * (1.0 / 2147483648.0) - 1.0);
        const T im = T(hash_u32(seed * 0x9E3779B97F4A7C15ULL + 2 * e + 1) * (1.0 / 2147483648.0) - 1.0);
        v[e] = (skip_bin0 && (e % V) == 0) ? mk(T(0), T(0)) : mk(re, im);
    }
}

}  // namespace bloch
