// Block kernels of the eigensolvers: Gram projections, basis rotation,
// Rayleigh quotients and residuals of a block of vectors (Algorithm 1 steps
// K = conj(U^T) Kn, M = conj(U^T) Mn, U <- U Q, err2).
#pragma once

#include <algorithm>

#include "common.cuh"
#include "dense_eig.cuh"
#include "vec.cuh"

namespace bloch {

constexpr int kQMax = 32;

// Fused projections of Algorithm 1, one pass over the block:
//   K[slot][i][j] = sum_e conj(A[i][e]) Bk[i][e]                    (all i, j < q)
//   M[slot][i][j] = sum_e conj(A[i][e]) Bm[j][e]    Bm != nullptr   (all i, j)
//                 = sum_e conj(A[i][e]) A[j][e]     Bm == nullptr   (i <= j tiles, mirrored)
// partial[slot][blk][0..1][q][q] (K, then M).  Vector i of a slot lies at
// base + (i / seg) * segstride + (slot * seg + i % seg) * n_per: with seg = q
// the q vectors of a slot are contiguous; with seg < q the block is the
// concatenation of q / seg segments of seg vectors each, segment t starting
// t * segstride elements further (LOBPCG's [X, W, P]).  Each thread owns a 4x4 tile of (i, j)
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
                                                        double2* __restrict__ partial, int seg,
                                                        long long segstride) {
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
            const C* src = (m == 0 ? A : (m == 1 ? Bk : Bm));
            const size_t vo = ok ? (size_t)(i / seg) * segstride + ((size_t)slot * seg + i % seg) * n_per + e : 0;
            cp_async_cplx(dst + ((size_t)m * kGKChunk + c) * RS + i, src + vo, ok);
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

// Basis rotation Out[slot][j][e] = sum_{i < qi} In_slot,i[e] Q[slot][i][j], j < qo.
// Input vector i of a slot lies at In + slot * in_slot + (i / seg) * segstride
// + (i % seg) * n_per (seg = qi: contiguous; seg < qi: segmented block such as
// LOBPCG's [X, W, P]); Q[slot] at Q + slot * qstride with row stride ldq;
// outputs contiguous per slot at Out + slot * out_slot.
struct RotView {
    long long in_slot, segstride, out_slot, qstride;
    int qi, qo, seg, ldq;
};
__device__ __forceinline__ size_t rot_in(const RotView& r, int slot, int i, long long n_per) {
    return (size_t)slot * r.in_slot + (size_t)(i / r.seg) * r.segstride + (size_t)(i % r.seg) * n_per;
}

// k_basis_reg (qi <= QI <= 32, qo <= 32): each thread loads the qi inputs of
// its element into registers at once and forms the outputs one by one from Q
// in shared memory (broadcast reads).  The per-input offsets are computed once
// per CTA into shared memory, and every thread issues all QI loads before
// using them (indices past qi repeat the last input, an L1 hit, with zero
// rows of Q), so they are in flight together.
// k_basis_cols (any qi, qo): output columns in chunks of 32 (blockIdx.y =
// slot * nchunk + chunk), the qi x 32 slice of Q and the input offsets in
// dynamic shared memory, 32 accumulators per thread, inputs loaded 8 at a time.
constexpr int kBasisQMax = 64;

template <typename T, int QI>
__global__ void __launch_bounds__(128) k_basis_reg(const cplx_t<T>* __restrict__ In, cplx_t<T>* __restrict__ Out,
                                                   const double2* __restrict__ Q, RotView rv, long long n_per) {
    using C = cplx_t<T>;
    __shared__ C sQ[QI * kQMax];
    __shared__ long long soff[QI];
    const int slot = blockIdx.y;
    const int qi = rv.qi, qo = rv.qo;
    if (qi < 1) return;   // uniform over the grid
    for (int t = threadIdx.x; t < QI * qo; t += blockDim.x) {
        const int i = t / qo, j = t - i * qo;
        const double2 v = i < qi ? Q[(size_t)slot * rv.qstride + (size_t)i * rv.ldq + j] : make_double2(0.0, 0.0);
        sQ[t] = mk(T(v.x), T(v.y));
    }
    for (int i = threadIdx.x; i < QI; i += blockDim.x) soff[i] = (long long)rot_in(rv, slot, min(i, qi - 1), n_per);
    __syncthreads();
    C* ob = Out + (size_t)slot * rv.out_slot;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_per;
         e += (long long)gridDim.x * blockDim.x) {
        C v[QI];
#pragma unroll
        for (int i = 0; i < QI; ++i) v[i] = In[soff[i] + e];
        for (int j = 0; j < qo; ++j) {
            T re = 0, im = 0;
#pragma unroll
            for (int i = 0; i < QI; ++i) {
                const C w = sQ[i * qo + j];
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
                                                    const double2* __restrict__ Q, RotView rv, long long n_per) {
    using C = cplx_t<T>;
    constexpr int JC = kBasisJC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int IB = 8;   // inputs loaded together
    C* sQ = reinterpret_cast<C*>(smem_raw);   // sQ[i * JC + jj] = Q[i][j0 + jj], qi rounded up to IB rows
    const int qi = rv.qi, qo = rv.qo;
    if (qi < 1) return;   // uniform over the grid
    const int qr = (qi + IB - 1) / IB * IB;
    long long* soff = reinterpret_cast<long long*>(sQ + (size_t)qr * JC);   // input offsets
    const int nch = (qo + JC - 1) / JC;
    const int slot = blockIdx.y / nch;
    const int j0 = (blockIdx.y - slot * nch) * JC;
    const int ncol = min(JC, qo - j0);
    for (int t = threadIdx.x; t < qr * JC; t += blockDim.x) {
        const int i = t / JC, jj = t - i * JC;
        const double2 v = (jj < ncol && i < qi) ? Q[(size_t)slot * rv.qstride + (size_t)i * rv.ldq + j0 + jj]
                                                : make_double2(0.0, 0.0);
        sQ[t] = mk(T(v.x), T(v.y));
    }
    for (int i = threadIdx.x; i < qr; i += blockDim.x) soff[i] = (long long)rot_in(rv, slot, min(i, qi - 1), n_per);
    __syncthreads();
    C* ob = Out + (size_t)slot * rv.out_slot;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n_per;
         e += (long long)gridDim.x * blockDim.x) {
        T re[JC], im[JC];
#pragma unroll
        for (int jj = 0; jj < JC; ++jj) re[jj] = im[jj] = T(0);
        for (int i0 = 0; i0 < qr; i0 += IB) {   // rows past qi repeat the last input with zero Q rows
            C v[IB];
#pragma unroll
            for (int u = 0; u < IB; ++u) v[u] = In[soff[i0 + u] + e];
#pragma unroll
            for (int u = 0; u < IB; ++u)
#pragma unroll
                for (int jj = 0; jj < JC; ++jj) {
                    const C w = sQ[(i0 + u) * JC + jj];
                    re[jj] = fma(v[u].x, w.x, fma(-v[u].y, w.y, re[jj]));
                    im[jj] = fma(v[u].x, w.y, fma(v[u].y, w.x, im[jj]));
                }
        }
#pragma unroll
        for (int jj = 0; jj < JC; ++jj)
            if (jj < ncol) ob[(size_t)(j0 + jj) * n_per + e] = mk(re[jj], im[jj]);
    }
}

template <typename T>
void launch_rotate(cudaStream_t st, int nslot, const cplx_t<T>* In, cplx_t<T>* Out, const double2* Q,
                   const RotView& rv, long long n_per) {
    const unsigned gx = (unsigned)std::min<long long>((n_per + 127) / 128, 8192);
    if (rv.qi <= kQMax && rv.qo <= kQMax) {
        if (rv.qi <= 8) k_basis_reg<T, 8><<<dim3(gx, nslot), 128, 0, st>>>(In, Out, Q, rv, n_per);
        else if (rv.qi <= 16) k_basis_reg<T, 16><<<dim3(gx, nslot), 128, 0, st>>>(In, Out, Q, rv, n_per);
        else if (rv.qi <= 24) k_basis_reg<T, 24><<<dim3(gx, nslot), 128, 0, st>>>(In, Out, Q, rv, n_per);
        else k_basis_reg<T, kQMax><<<dim3(gx, nslot), 128, 0, st>>>(In, Out, Q, rv, n_per);
    } else {
        const int nch = (rv.qo + kBasisJC - 1) / kBasisJC;
        const size_t qr = (size_t)(rv.qi + 7) / 8 * 8;
        k_basis_cols<T><<<dim3(gx, nslot * nch), 128, qr * kBasisJC * sizeof(cplx_t<T>) + qr * sizeof(long long),
                          st>>>(In, Out, Q, rv, n_per);
    }
}

// Square rotation of nslot slots, Out[slot] = In[slot] Q[slot] (q x q row-major),
// In slot s at In + s * in_stride (in_stride <= 0: q * n_per).
template <typename T>
void launch_basis(cudaStream_t st, int nslot, const cplx_t<T>* In, cplx_t<T>* Out, const double2* Q, int q,
                  long long n_per, long long in_stride = 0) {
    RotView rv;
    rv.in_slot = in_stride > 0 ? in_stride : (long long)q * n_per;
    rv.segstride = 0;
    rv.out_slot = (long long)q * n_per;
    rv.qstride = (long long)q * q;
    rv.qi = rv.qo = rv.seg = rv.ldq = q;
    launch_rotate<T>(st, nslot, In, Out, Q, rv, n_per);
}

// First qo columns of the square rotation: Out[slot][j] = sum_i In[slot][i] Q[slot][i][j], j < qo
// (Q q x q row-major; outputs at the square layout's stride q * n_per).
template <typename T>
void launch_basis_first(cudaStream_t st, int nslot, const cplx_t<T>* In, cplx_t<T>* Out, const double2* Q, int q,
                        int qo, long long n_per, long long in_stride) {
    RotView rv;
    rv.in_slot = in_stride;
    rv.segstride = 0;
    rv.out_slot = (long long)q * n_per;
    rv.qstride = (long long)q * q;
    rv.qi = rv.seg = rv.ldq = q;
    rv.qo = qo;
    launch_rotate<T>(st, nslot, In, Out, Q, rv, n_per);
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

// Final sums of k_rq_dots for the nv vectors of one call (blockIdx.x = v):
// (Re u^H K u, u^H M u, |K u|^2) go to rq[d][0..2] with d = (first + v/nvs) q
// + vo + v % nvs, and 1/lambda (0 when lambda <= 0) to inv_call[v] and inv_slot[d].
static __global__ void k_rq_final(const double* __restrict__ partial, int dblk, int first, int nvs, int vo, int q,
                                  double* __restrict__ rq, double* __restrict__ inv_call,
                                  double* __restrict__ inv_slot) {
    const int v = blockIdx.x;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < dblk; j += blockDim.x) {
        const double* p = partial + ((size_t)v * dblk + j) * 3;
        acc[0] += p[0];
        acc[1] += p[1];
        acc[2] += p[2];
    }
    block_sum<double, 3>(acc);
    if (threadIdx.x == 0) {
        const size_t d = (size_t)(first + v / nvs) * q + vo + v % nvs;
        rq[d * 4 + 0] = acc[0];
        rq[d * 4 + 1] = acc[1];
        rq[d * 4 + 2] = acc[2];
        const double lam = acc[1] > 0.0 ? acc[0] / acc[1] : 0.0;
        const double il = lam > 0.0 ? 1.0 / lam : 0.0;
        inv_call[v] = il;
        inv_slot[d] = il;
    }
}

// Final sums of k_residual: |R|^2 to rq[d][3]
static __global__ void k_r2_final(const double* __restrict__ partial, int dblk, int first, int nvs, int vo, int q,
                                  double* __restrict__ rq) {
    const int v = blockIdx.x;
    double acc[1] = {0.0};
    for (int j = threadIdx.x; j < dblk; j += blockDim.x) acc[0] += partial[(size_t)v * dblk + j];
    block_sum<double, 1>(acc);
    if (threadIdx.x == 0) rq[((size_t)(first + v / nvs) * q + vo + v % nvs) * 4 + 3] = acc[0];
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

// the same conversion in place, for two types of equal size (float-float <-> FP64)
template <typename Ta, typename Tb>
__global__ void k_convert_inplace(void* p, size_t n) {
    static_assert(sizeof(cplx_t<Ta>) == sizeof(cplx_t<Tb>), "in-place conversion needs equal sizes");
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const cplx_t<Ta> a = reinterpret_cast<const cplx_t<Ta>*>(p)[i];
        reinterpret_cast<cplx_t<Tb>*>(p)[i] = mk(Tb(a.x), Tb(a.y));
    }
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
    if (m == 0) return;
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

// ---- two-pass classical Gram-Schmidt reading the basis three times (nv <= kGsMax)
// The first pass forms all nv inner products from one read of W; the second
// updates W and forms the inner products of the updated W in the same read
// of the basis; the last update also forms |W|^2.  Partials per (slot,
// block) as in k_vdots.  NV (8, 12, 16, 20, 24, 32) bounds nv at compile time so
// the accumulators stay in registers; every thread issues all NV loads of an
// element before using them (indices past nv repeat the last vector, an L1
// hit, with a zero coefficient or an unused product), so they are in flight
// together.
constexpr int kGsMax = 32;
constexpr int kGsKeep = 20;   // up to this NV the update keeps the basis elements in registers

__device__ __forceinline__ float2 ldca_c(const float2* p) { return __ldca(p); }
__device__ __forceinline__ double2 ldca_c(const double2* p) { return __ldca(p); }

template <int NV, typename T>
__device__ __forceinline__ void gs_write_partials(T (&acc)[2 * NV], int m, int maxnv, double2* __restrict__ partial) {
    block_sum<T, 2 * NV>(acc);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i)
            if (i < m)
                partial[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * maxnv + i] =
                    make_double2(acc[2 * i], acc[2 * i + 1]);
    }
}

// partial[(slot*gridDim.x + blk)*maxnv + i] = sum_e conj(V[slot][i][e]) W[slot][e], i < nv[slot]
template <typename T, int NV>
__global__ void __launch_bounds__(256, 2) k_vdots_all(const cplx_t<T>* __restrict__ V, long long vstride,
                                                   const cplx_t<T>* __restrict__ W, long long wstride,
                                                   const int* __restrict__ nv, long long n, int maxnv,
                                                   double2* __restrict__ partial) {
    using C = cplx_t<T>;
    const int slot = blockIdx.y;
    const int m = nv[slot];
    if (m <= 0) return;   // uniform over the block
    const C* vb = V + (size_t)slot * vstride;
    const C* w = W + (size_t)slot * wstride;
    T acc[2 * NV];
#pragma unroll
    for (int i = 0; i < 2 * NV; ++i) acc[i] = T(0);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const C b = w[e];
        C a[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) a[i] = vb[(size_t)min(i, m - 1) * n + e];   // all loads in flight
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            acc[2 * i] += a[i].x * b.x + a[i].y * b.y;
            acc[2 * i + 1] += a[i].x * b.y - a[i].y * b.x;
        }
    }
    gs_write_partials<NV>(acc, m, maxnv, partial);
}

// W[slot] -= sum_i V[slot][i] h[slot][i], then the inner products of the updated W
// with every V[slot][i] into partial (layout as k_vdots_all); the basis
// elements of the update are kept in registers for the products
template <typename T, int NV>
__global__ void __launch_bounds__(256, 2) k_vaxpy_dots(const cplx_t<T>* __restrict__ V, long long vstride,
                                                    cplx_t<T>* __restrict__ W, long long wstride,
                                                    const double2* __restrict__ h, const int* __restrict__ nv,
                                                    long long n, int maxnv, double2* __restrict__ partial) {
    using C = cplx_t<T>;
    __shared__ C sh[NV];
    const int slot = blockIdx.y;
    const int m = nv[slot];
    for (int i = threadIdx.x; i < NV; i += blockDim.x) {
        const double2 v = i < m ? h[(size_t)slot * maxnv + i] : make_double2(0.0, 0.0);
        sh[i] = mk(T(v.x), T(v.y));
    }
    __syncthreads();
    if (m <= 0) return;   // uniform over the block
    const C* vb = V + (size_t)slot * vstride;
    C* w = W + (size_t)slot * wstride;
    T acc[2 * NV];
#pragma unroll
    for (int i = 0; i < 2 * NV; ++i) acc[i] = T(0);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        C b = w[e];
        C a[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) a[i] = vb[(size_t)min(i, m - 1) * n + e];   // all loads in flight
#pragma unroll
        for (int i = 0; i < NV; ++i) {   // sh[i] = 0 for i >= m
            const C c = sh[i];
            b.x -= a[i].x * c.x - a[i].y * c.y;
            b.y -= a[i].x * c.y + a[i].y * c.x;
        }
        w[e] = b;
        if constexpr (NV > kGsKeep) {   // the basis elements again, from L1 (just fetched by this thread)
#pragma unroll
            for (int i = 0; i < NV; ++i) a[i] = ldca_c(vb + (size_t)min(i, m - 1) * n + e);
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            acc[2 * i] += a[i].x * b.x + a[i].y * b.y;
            acc[2 * i + 1] += a[i].x * b.y - a[i].y * b.x;
        }
    }
    gs_write_partials<NV>(acc, m, maxnv, partial);
}

// W[slot] -= sum_i V[slot][i] h[slot][i], and part[slot*gridDim.x + blk] = (sum |W|^2, 0)
template <typename T, int NV>
__global__ void __launch_bounds__(256, 2) k_vaxpy_norm(const cplx_t<T>* __restrict__ V, long long vstride,
                                                    cplx_t<T>* __restrict__ W, long long wstride,
                                                    const double2* __restrict__ h, const int* __restrict__ nv,
                                                    long long n, int maxnv, double2* __restrict__ part) {
    using C = cplx_t<T>;
    __shared__ C sh[NV];
    const int slot = blockIdx.y;
    const int m = nv[slot];
    for (int i = threadIdx.x; i < NV; i += blockDim.x) {
        const double2 v = i < m ? h[(size_t)slot * maxnv + i] : make_double2(0.0, 0.0);
        sh[i] = mk(T(v.x), T(v.y));
    }
    __syncthreads();
    if (m <= 0) return;   // uniform over the block
    const C* vb = V + (size_t)slot * vstride;
    C* w = W + (size_t)slot * wstride;
    T acc[2] = {T(0), T(0)};
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        C b = w[e];
        C a[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) a[i] = vb[(size_t)min(i, m - 1) * n + e];   // all loads in flight
#pragma unroll
        for (int i = 0; i < NV; ++i) {   // sh[i] = 0 for i >= m
            const C c = sh[i];
            b.x -= a[i].x * c.x - a[i].y * c.y;
            b.y -= a[i].x * c.y + a[i].y * c.x;
        }
        w[e] = b;
        acc[0] += b.x * b.x + b.y * b.y;
    }
    block_sum<T, 2>(acc);
    if (threadIdx.x == 0) part[(size_t)slot * gridDim.x + blockIdx.x] = make_double2(acc[0], 0.0);
}

// The three kernels above for the smallest NV >= nv.
template <typename T>
void launch_gs3(int which, dim3 grid, cudaStream_t st, const cplx_t<T>* V, long long vstride, cplx_t<T>* W,
                long long wstride, const double2* h, const int* d_nv, long long n, int nv, double2* out) {
#define BLOCH_GS3(NVC)                                                                                        \
    do {                                                                                                       \
        if (which == 0)                                                                                        \
            k_vdots_all<T, NVC><<<grid, 256, 0, st>>>(V, vstride, W, wstride, d_nv, n, nv, out);             \
        else if (which == 1)                                                                                   \
            k_vaxpy_dots<T, NVC><<<grid, 256, 0, st>>>(V, vstride, W, wstride, h, d_nv, n, nv, out);         \
        else                                                                                                   \
            k_vaxpy_norm<T, NVC><<<grid, 256, 0, st>>>(V, vstride, W, wstride, h, d_nv, n, nv, out);         \
    } while (0)
    if (nv <= 8) BLOCH_GS3(8);
    else if (nv <= 12) BLOCH_GS3(12);
    else if (nv <= 16) BLOCH_GS3(16);
    else if (nv <= 20) BLOCH_GS3(20);
    else if (nv <= 24) BLOCH_GS3(24);
    else BLOCH_GS3(32);
#undef BLOCH_GS3
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

// ------------------------------------------------ device-resident Lanczos
// All slots advance in lockstep (same step j), so the column of a step is a
// kernel argument and no per-step host synchronisation is needed.

// dst[s] = Vb[s][j] * (scale ? scale[s] : 1)   (blockIdx.y = slot)
template <typename T>
__global__ void k_get_col(const cplx_t<T>* __restrict__ Vb, long long slot_stride, int j, long long n3,
                          const double* __restrict__ scale, cplx_t<T>* __restrict__ dst) {
    const int sl = blockIdx.y;
    const T sv = scale ? T(scale[sl]) : T(1);
    const cplx_t<T>* a = Vb + (size_t)sl * slot_stride + (size_t)j * n3;
    cplx_t<T>* b = dst + (size_t)sl * n3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3;
         e += (long long)gridDim.x * blockDim.x)
        b[e] = cscale(a[e], sv);
}

// Vb[s][j] = src[s] * scale[s]
template <typename T>
__global__ void k_put_col(const cplx_t<T>* __restrict__ src, cplx_t<T>* __restrict__ Vb, long long slot_stride,
                          int j, long long n3, const double* __restrict__ scale) {
    const int sl = blockIdx.y;
    const T sv = T(scale[sl]);
    const cplx_t<T>* a = src + (size_t)sl * n3;
    cplx_t<T>* b = Vb + (size_t)sl * slot_stride + (size_t)j * n3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3;
         e += (long long)gridDim.x * blockDim.x)
        b[e] = cscale(a[e], sv);
}

// a[0..n) = v
static __global__ void k_fill_int(int* __restrict__ a, int n, int v) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = v;
}

// H[s][t][j] += h[s][t] for t < nv (Gram-Schmidt coefficients of step j;
// H row-major (m + 1) x m per slot)
static __global__ void k_h_accum(double2* __restrict__ H, const double2* __restrict__ h, int maxnv, int nv, int j,
                                 int m) {
    const int sl = blockIdx.x;
    double2* Hs = H + (size_t)sl * (m + 1) * m;
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        const double2 v = h[(size_t)sl * maxnv + t];
        Hs[(size_t)t * m + j].x += v.x;
        Hs[(size_t)t * m + j].y += v.y;
    }
}

// beta_s = sqrt(scale * Re dots[s]); H[s][j+1][j] = beta (j >= 0); inv[s] = 1/beta (0 if beta = 0)
static __global__ void k_lz_norm(const double2* __restrict__ dots, double scale, double2* __restrict__ H, int j,
                                 int m, int nact, double* __restrict__ inv) {
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= nact) return;
    const double beta = sqrt(fmax(scale * dots[sl].x, 0.0));
    if (j >= 0) H[(size_t)sl * (m + 1) * m + (size_t)(j + 1) * m + j] = make_double2(beta, 0.0);
    inv[sl] = beta > 0.0 ? 1.0 / beta : 0.0;
}

// Shared memory of k_lz_ritz for basis size m, in this order (16-byte aligned
// double2 first): two m x m double2 matrices, the rotation slots
// (jacobi_rot_slots(m) double2), m doubles, 2 * nthreads doubles of
// reductions, m ints.
__host__ __device__ constexpr size_t lz_ritz_smem(int m, int nthreads) {
    return (size_t)2 * m * m * sizeof(double2) + (size_t)jacobi_rot_slots(m) * sizeof(double2) +
           (size_t)m * sizeof(double) + (size_t)2 * nthreads * sizeof(double) + (size_t)m * sizeof(int);
}

// Thick-restart analysis of slot blockIdx.x (Section 3.3 shift-invert
// Lanczos, Ritz values theta of OP = A^-1 M, wanted: the largest): the
// Hermitian part of H[0:m][0:m] is diagonalised; theta[s][c] (descending)
// and the Ritz estimates est[s][c] = beta |y_{m-1,c}| (beta = |H[m][m-1]|)
// are written for every c < m; conv[s] = all neff[s] wanted estimates
// satisfy est <= tol |theta| with theta > 0.  Q[s] (m x m) receives the kc
// leading Ritz vectors in its columns (zero beyond), and H[s] is reset to the
// thick-restart matrix of kk leading Ritz pairs: diag(theta) and the row
// kk = beta y_{m-1, c}.
static __global__ void k_lz_ritz(int m, double2* __restrict__ H, const int* __restrict__ neff, double tol, int kc, int kk,
                          double2* __restrict__ Q, double* __restrict__ theta, double* __restrict__ est,
                          int* __restrict__ conv, int* __restrict__ jac_ok) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* A = reinterpret_cast<double2*>(smem_raw);
    double2* Y = A + m * m;
    double2* rot = Y + m * m;
    double* w = reinterpret_cast<double*>(rot + jacobi_rot_slots(m));
    double* red = w + m;
    int* perm = reinterpret_cast<int*>(red + 2 * blockDim.x);
    __shared__ double beta;
    const int sl = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    double2* Hs = H + (size_t)sl * (m + 1) * m;
    for (int e = tid; e < m * m; e += nt) {
        const int i = e / m, j = e % m;
        const double2 a = Hs[(size_t)i * m + j], b = Hs[(size_t)j * m + i];
        A[e] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    }
    if (tid == 0) beta = sqrt(zabs2(Hs[(size_t)m * m + (m - 1)]));
    __syncthreads();
    const bool ok = jacobi_herm(m, A, Y, w, red, rot);
    sort_ascending(m, w, perm);
    double* th = theta + (size_t)sl * m;
    double* es = est + (size_t)sl * m;
    for (int c = tid; c < m; c += nt) {
        const int ic = perm[m - 1 - c];
        th[c] = w[ic];
        es[c] = beta * sqrt(zabs2(Y[(m - 1) * m + ic]));
    }
    for (int e = tid; e < m * m; e += nt) {
        const int i = e / m, c = e % m;
        Q[(size_t)sl * m * m + e] = c < kc ? Y[i * m + perm[m - 1 - c]] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (tid == 0) {
        int cv = 1;
        for (int i = 0; i < neff[sl]; ++i) {
            const double t = th[i];
            if (!(t > 0.0) || es[i] > tol * fabs(t)) cv = 0;
        }
        conv[sl] = cv;
        jac_ok[sl] = ok ? 1 : 0;
    }
    for (int e = tid; e < (m + 1) * m; e += nt) Hs[e] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int c = tid; c < kk; c += nt) {
        const int ic = perm[m - 1 - c];
        Hs[(size_t)c * m + c] = make_double2(w[ic], 0.0);
        const double2 y = Y[(m - 1) * m + ic];
        Hs[(size_t)kk * m + c] = make_double2(beta * y.x, beta * y.y);
    }
}

// Restart copies of every slot: Vb[s][0..kk) = Tmp[s][0..kk), Vb[s][kk] = Vb[s][m]
template <typename T>
__global__ void k_lz_restart_copy(cplx_t<T>* __restrict__ Vb, const cplx_t<T>* __restrict__ Tmp, int m, int kk,
                                  long long n3) {
    const int sl = blockIdx.y;
    cplx_t<T>* vb = Vb + (size_t)sl * (m + 1) * n3;
    const cplx_t<T>* tb = Tmp + (size_t)sl * m * n3;
    const long long tot = (long long)(kk + 1) * n3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x)
        vb[e] = e < (long long)kk * n3 ? tb[e] : vb[(size_t)m * n3 + (e - (long long)kk * n3)];
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
