// Block kernels of the eigensolvers: Gram projections, basis rotation,
// Rayleigh quotients and residuals of a block of vectors (Algorithm 1 steps
// K = conj(U^T) Kn, M = conj(U^T) Mn, U <- U Q, err2).
#pragma once

#include <algorithm>

#include "common.cuh"
#include "vec.cuh"

namespace bloch {

constexpr int kQMax = 32;

// Fused projections of Algorithm 1, one pass over the block:
//   K[slot][i][j] = sum_e conj(A[i][e]) Bk[i][e]                    (all i, j < q)
//   M[slot][i][j] = sum_e conj(A[i][e]) Bm[j][e]    Bm != nullptr   (all i, j)
//                 = sum_e conj(A[i][e]) A[j][e]     Bm == nullptr   (i <= j tiles, mirrored)
// partial[slot][blk][0..1][q][q] (K, then M); vectors of one slot are
// contiguous (A + (slot*q + i)*n_per).  Each thread owns a 4x4 tile of (i, j)
// and one group of elements of every chunk.  Chunks of kGKChunk elements are
// staged element-major (row length RS, odd, so consecutive elements fall in
// different banks and the tile rows a warp reads are spread) by cp.async, two
// chunks in flight; element groups are reduced through shared memory at the end.
constexpr int kGKChunk = 64;
constexpr int kGKThreads = 256;

__host__ __device__ constexpr int gk_rs(int q) { return ((q + 3) / 4) * 4 + 1; }
__host__ __device__ constexpr int gk_nmat(bool has_m) { return has_m ? 3 : 2; }
// dynamic shared memory of k_gram_km: two stages of nmat element-major tiles
template <typename T>
size_t gk_smem(int q, bool has_m) {
    const size_t stage = (size_t)gk_nmat(has_m) * kGKChunk * gk_rs(q) * sizeof(cplx_t<T>);
    const size_t red = (size_t)kGKThreads * 16 * sizeof(cplx_t<T>);
    return 2 * stage > red ? 2 * stage : red;
}

template <typename T>
__global__ void __launch_bounds__(kGKThreads) k_gram_km(const cplx_t<T>* __restrict__ A,
                                                        const cplx_t<T>* __restrict__ Bk,
                                                        const cplx_t<T>* __restrict__ Bm, int q, long long n_per,
                                                        double2* __restrict__ partial) {
    using C = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const bool has_m = Bm != nullptr;
    const int nmat = gk_nmat(has_m);
    const int RS = gk_rs(q);
    const int side = (q + 3) / 4;
    const int nk = side * side;
    const int nm = has_m ? side * side : side * (side + 1) / 2;
    const int ntile = nk + nm;
    const int G = kGKThreads / ntile;   // element groups (>= 2 for q <= 32)
    const int tid = threadIdx.x;
    const int tile = tid % ntile, grp = tid / ntile;
    const bool act = grp < G;
    // tile -> (matrix, i0, j0, operand pointers' matrix index)
    int which, i0, j0;
    if (tile < nk) {
        which = 0;
        i0 = (tile / side) * 4;
        j0 = (tile % side) * 4;
    } else if (has_m) {
        which = 1;
        i0 = ((tile - nk) / side) * 4;
        j0 = ((tile - nk) % side) * 4;
    } else {   // upper-triangular tile index t -> (ti <= tj)
        which = 1;
        int t = tile - nk, ti = 0;
        while (t >= side - ti) {
            t -= side - ti;
            ++ti;
        }
        i0 = ti * 4;
        j0 = (ti + t) * 4;
    }
    const int bmat = which == 0 ? 1 : (has_m ? 2 : 0);   // staged matrix of the right operand
    const int slot = blockIdx.y;
    const size_t sbase = (size_t)slot * q * n_per;
    const int stage_elems = nmat * kGKChunk * RS;
    auto stage_load = [&](long long ch, int buf) {
        C* dst = sm + (size_t)buf * stage_elems;
        const long long e0 = ch * kGKChunk;
        const int rows = side * 4;
        for (int t = tid; t < nmat * rows * kGKChunk; t += kGKThreads) {
            const int m = t / (rows * kGKChunk);
            const int r = t - m * rows * kGKChunk;
            const int i = r / kGKChunk, c = r - i * kGKChunk;
            const long long e = e0 + c;
            const bool ok = i < q && e < n_per;
            const C* src = (m == 0 ? A : (m == 1 ? Bk : Bm)) + sbase;
            cp_async_cplx(dst + ((size_t)m * kGKChunk + c) * RS + i, src + (ok ? (size_t)i * n_per + e : 0), ok);
        }
        cp_async_commit();
    };
    T acc[4][4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c][0] = acc[a][c][1] = T(0);
    const long long nchunk = (n_per + kGKChunk - 1) / kGKChunk;
    long long ch = blockIdx.x;
    if (ch < nchunk) stage_load(ch, 0);
    else cp_async_commit();
    if (ch + gridDim.x < nchunk) stage_load(ch + gridDim.x, 1);
    else cp_async_commit();
    int buf = 0;
    for (; ch < nchunk; ch += gridDim.x) {
        cp_async_wait<1>();
        __syncthreads();
        if (act) {
            const C* sa = sm + (size_t)buf * stage_elems;
            const C* sb = sa + (size_t)bmat * kGKChunk * RS;
            for (int e = grp; e < kGKChunk; e += G) {
                C a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a[u] = sa[e * RS + i0 + u];
                    b[u] = sb[e * RS + j0 + u];
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
        __syncthreads();   // every thread is done with this stage before it is refilled
        const long long nx = ch + 2 * (long long)gridDim.x;
        if (nx < nchunk) stage_load(nx, buf);
        else cp_async_commit();
        buf ^= 1;
    }
    cp_async_wait<0>();
    __syncthreads();
    // reduce the element groups through shared memory: red[tile][16]
    C* red = sm;
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
    const int npair = q * q;
    double2* out = partial + ((size_t)slot * gridDim.x + blockIdx.x) * 2 * npair;
    for (int t = tid; t < 2 * npair; t += kGKThreads) {
        const int w = t / npair, pr = t - w * npair;
        int i = pr / q, j = pr - i * q;
        bool conj_it = false;
        if (w == 1 && !has_m && i / 4 > j / 4) {   // lower tile of A^H A: mirror of (j, i)
            const int tmp = i;
            i = j;
            j = tmp;
            conj_it = true;
        }
        const int ti = i / 4, tj = j / 4;
        int tl;
        if (w == 0) tl = ti * side + tj;
        else if (has_m) tl = nk + ti * side + tj;
        else tl = nk + ti * side - ti * (ti - 1) / 2 + (tj - ti);
        const C r = red[tl * 16 + (i % 4) * 4 + (j % 4)];
        out[t] = make_double2(r.x, conj_it ? -r.y : r.y);
    }
}

// G[w][slot][pr] = sum over blocks of partial[slot][blk][w][pr]  (w = 0: K, 1: M)
static __global__ void k_gram_final(const double2* __restrict__ partial, int nblk, int npair, int nslot,
                                    double2* __restrict__ out) {
    const int slot = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * npair) return;
    const int w = t / npair, pr = t - w * npair;
    double re = 0, im = 0;
    for (int b = 0; b < nblk; ++b) {
        const double2 v = partial[((size_t)slot * nblk + b) * 2 * npair + t];
        re += v.x;
        im += v.y;
    }
    out[((size_t)w * nslot + slot) * npair + pr] = make_double2(re, im);
}

// Out[slot][j][e] = sum_i In[slot][i][e] Q[slot][i][j]  (Q row-major q x q, double2).
//
// k_basis_reg (q <= 32): each thread loads the q inputs of its element into
// registers at once (q loads in flight) and forms the outputs one by one from
// Q in shared memory (broadcast reads).
// k_basis_cols (q <= 63, Lanczos restarts with a large basis): output columns
// in chunks of 32 (blockIdx.y = slot * nchunk + chunk), the q x 32 slice of Q
// in dynamic shared memory, 32 accumulators per thread.
constexpr int kBasisQMax = 64;

template <typename T>
__global__ void __launch_bounds__(128) k_basis_reg(const cplx_t<T>* __restrict__ In, cplx_t<T>* __restrict__ Out,
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

constexpr int kBasisJC = 32;

template <typename T>
__global__ void __launch_bounds__(128) k_basis_cols(const cplx_t<T>* __restrict__ In, cplx_t<T>* __restrict__ Out,
                                                    const double2* __restrict__ Q, int q, long long n_per) {
    using C = cplx_t<T>;
    constexpr int JC = kBasisJC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sQ = reinterpret_cast<C*>(smem_raw);   // sQ[i * JC + jj] = Q[i][j0 + jj]
    const int nch = (q + JC - 1) / JC;
    const int slot = blockIdx.y / nch;
    const int j0 = (blockIdx.y - slot * nch) * JC;
    const int ncol = min(JC, q - j0);
    for (int t = threadIdx.x; t < q * JC; t += blockDim.x) {
        const int i = t / JC, jj = t - i * JC;
        const double2 v = jj < ncol ? Q[(size_t)slot * q * q + (size_t)i * q + j0 + jj] : make_double2(0.0, 0.0);
        sQ[t] = mk(T(v.x), T(v.y));
    }
    __syncthreads();
    const C* ib = In + (size_t)slot * q * n_per;
    C* ob = Out + (size_t)slot * q * n_per;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_per;
         e += (long long)gridDim.x * blockDim.x) {
        T re[JC], im[JC];
#pragma unroll
        for (int jj = 0; jj < JC; ++jj) re[jj] = im[jj] = T(0);
#pragma unroll 2
        for (int i = 0; i < q; ++i) {
            const C v = ib[(size_t)i * n_per + e];
#pragma unroll
            for (int jj = 0; jj < JC; ++jj) {
                const C w = sQ[i * JC + jj];
                re[jj] = fma(v.x, w.x, fma(-v.y, w.y, re[jj]));
                im[jj] = fma(v.x, w.y, fma(v.y, w.x, im[jj]));
            }
        }
#pragma unroll
        for (int jj = 0; jj < JC; ++jj)
            if (jj < ncol) ob[(size_t)(j0 + jj) * n_per + e] = mk(re[jj], im[jj]);
    }
}

// Basis rotation of nslot slots (q < kBasisQMax).
template <typename T>
void launch_basis(cudaStream_t st, int nslot, const cplx_t<T>* In, cplx_t<T>* Out, const double2* Q, int q,
                  long long n_per) {
    const unsigned gx = (unsigned)std::min<long long>((n_per + 127) / 128, 8192);
    if (q <= kQMax) {
        k_basis_reg<T><<<dim3(gx, nslot), 128, 0, st>>>(In, Out, Q, q, n_per);
    } else {
        const int nch = (q + kBasisJC - 1) / kBasisJC;
        k_basis_cols<T><<<dim3(gx, nslot * nch), 128, (size_t)q * kBasisJC * sizeof(cplx_t<T>), st>>>(In, Out, Q,
                                                                                                     q, n_per);
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

// Gamma point with a non-uniform density (rigid translations t_c = e_c at
// bin 0 span the null space of A_0; the spectrum is sought on their
// M-orthogonal complement).  alpha[v][c] = t_c^H M v / t_c^H M t_c for nv
// vectors whose M-images MV are given; t_c^H M v is MV's bin-0 entry of
// component c, and t_c^H M t_c = rhohat[0] with rhohat = (M t_0)_0.
template <typename T>
__global__ void k_gamma_alpha(const cplx_t<T>* __restrict__ MV, long long n3, long long V, int nv,
                              const cplx_t<T>* __restrict__ rhohat, double2* __restrict__ alpha) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * nv) return;
    const int v = t / 3, c = t - 3 * (t / 3);
    const cplx_t<T> m = MV[(size_t)v * n3 + (size_t)c * V];
    const double d = (double)rhohat[0].x;
    alpha[t] = make_double2((double)m.x / d, (double)m.y / d);
}

// v <- v - sum_c alpha_c t_c (bin 0 of each component) and, when MV is given,
// M v <- M v - sum_c alpha_c M t_c, with (M t_c)_c = rhohat and zero in the
// other components.  blockIdx.y = vector.
template <typename T>
__global__ void k_gamma_deflate(cplx_t<T>* __restrict__ Vv, cplx_t<T>* __restrict__ MV,
                                const cplx_t<T>* __restrict__ rhohat, long long n3, long long V,
                                const double2* __restrict__ alpha) {
    const int v = blockIdx.y;
    cplx_t<T> a[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) a[c] = mk(T(alpha[3 * v + c].x), T(alpha[3 * v + c].y));
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < V;
         e += (long long)gridDim.x * blockDim.x) {
        if (MV) {
            const cplx_t<T> r = rhohat[e];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cplx_t<T>& m = MV[(size_t)v * n3 + (size_t)c * V + e];
                m = csub(m, cmul(a[c], r));
            }
        }
        if (e == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cplx_t<T>& x = Vv[(size_t)v * n3 + (size_t)c * V];
                x = csub(x, a[c]);
            }
        }
    }
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

// h[slot][i] = scale * sum_blk partial; one block per (i, slot): blockIdx.x = i,
// blockIdx.y = slot (a strided sum per thread, then the block tree: fixed order)
static __global__ void k_vdots_final(const double2* __restrict__ partial, int nblk, int maxnv, double scale,
                                     double2* __restrict__ h) {
    const int i = blockIdx.x, slot = blockIdx.y;
    double acc[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        const double2 v = partial[((size_t)slot * nblk + b) * maxnv + i];
        acc[0] += v.x;
        acc[1] += v.y;
    }
    block_sum<double, 2>(acc);
    if (threadIdx.x == 0) h[(size_t)slot * maxnv + i] = make_double2(scale * acc[0], scale * acc[1]);
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
