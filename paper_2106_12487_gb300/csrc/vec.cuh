// Pointwise and reduction kernels: wave-vector tables, Green-operator
// preconditioner (Eqs. matrixP, precond), dot products and the fused PCG
// updates of Algorithm 2.  Reductions: per-thread accumulation in the field
// precision, warp shuffle, one partial per block in FP64, and a one-block
// final sum per system (deterministic, no atomics).
#pragma once

#include "common.cuh"
#include "passes.cuh"

namespace bloch {

// P_ik = sum_m A[ik][m] mono_m(q), pairs ik in (xx, yy, zz, yz, xz, xy) and
// monomials (qx^2, qy^2, qz^2, qy qz, qx qz, qx qy), from the scaled C0.
struct PrecondCoef {
    double a[6][6];
    float af[6][6];   // the same coefficients rounded once to FP32 (FP32 kernels read these:
                      // no FP64 -> FP32 conversion per voxel)
};
template <typename T> __device__ __forceinline__ T pcoef(const PrecondCoef& pc, int i, int j);
template <> __device__ __forceinline__ float pcoef<float>(const PrecondCoef& pc, int i, int j) { return pc.af[i][j]; }
template <> __device__ __forceinline__ double pcoef<double>(const PrecondCoef& pc, int i, int j) { return pc.a[i][j]; }

// Per-system CG scalars (device resident).
struct CGSys {
    double rz;       // (r, z) of the current iterate
    double rz_new;
    double pAp;
    double rr;       // (r, r)
    double bb;       // (b, b) (scaled)
    double alpha;
    double beta;
    int active;
    int iters;
    int upd;         // took a step this iteration (x += alpha p is still to be applied)
};

// qtab[b][.] = ((xi + k_b) * qscale) for the x, y and z axes.
template <typename T>
__global__ void k_qtab(const double* __restrict__ kvec, const double* __restrict__ xi, int Nx, int Ny, int Nz,
                       int nb, double qscale, T* __restrict__ qtab) {
    const int S = Nx + Ny + Nz;
    const long long total = (long long)nb * S;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / S), j = (int)(i % S);
        const int ax = j < Nx ? 0 : (j < Nx + Ny ? 1 : 2);
        qtab[i] = T((xi[j] + kvec[3 * b + ax]) * qscale);
    }
}

template <typename T>
__global__ void k_scale(const cplx_t<T>* in, cplx_t<T>* out, T s, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = cscale(in[i], s);
}

// voxel index -> (x, y, z) in 32-bit unsigned arithmetic (V < 2^31 for every
// supported grid)
template <typename T>
__device__ __forceinline__ void voxel_q(const T* qb, const Geo& g, unsigned v, T& ax, T& ay, T& az) {
    const unsigned t = fdiv(v, g.dx);
    const int x = (int)(v - t * (unsigned)g.Nx);
    const unsigned z = fdiv(t, g.dy);
    const int y = (int)(t - z * (unsigned)g.Ny);
    ax = qb[x];
    ay = qb[g.Nx + y];
    az = qb[g.Nx + g.Ny + z];
}

// Correctly rounded reciprocal (the FP32 form uses the rounded reciprocal
// intrinsic instead of a full division).
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// z = P^-1(q) r for one voxel (three complex components); zero where q = 0.
template <typename T>
__device__ __forceinline__ void green_apply(const PrecondCoef& pc, T qx, T qy, T qz, const cplx_t<T> r[3],
                                            cplx_t<T> z[3]) {
    const T m[6] = {qx * qx, qy * qy, qz * qz, qy * qz, qx * qz, qx * qy};
    T P[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T s = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) s = fma(pcoef<T>(pc, i, j), m[j], s);
        P[i] = s;
    }
    const T a = P[0], bq = P[1], c = P[2], d = P[3], e = P[4], f = P[5];
    const T A = bq * c - d * d, B = a * c - e * e, Cc = a * bq - f * f;
    const T D = e * f - a * d, Ee = d * f - bq * e, F = d * e - c * f;
    const T det = a * A + f * F + e * Ee;
    if (m[0] + m[1] + m[2] == T(0) || det == T(0)) {
        z[0] = z[1] = z[2] = mk(T(0), T(0));
        return;
    }
    const T id = recip(det);
    z[0] = cscale(cadd(cadd(cscale(r[0], A), cscale(r[1], F)), cscale(r[2], Ee)), id);
    z[1] = cscale(cadd(cadd(cscale(r[0], F), cscale(r[1], B)), cscale(r[2], D)), id);
    z[2] = cscale(cadd(cadd(cscale(r[0], Ee), cscale(r[1], D)), cscale(r[2], Cc)), id);
}

// Preconditioner selection: the Green operator P^-1 computed per voxel, or a
// precomputed symmetric 3x3 table per voxel (the learned preconditioner), one
// table per group of `zgroup` consecutive systems.
struct PrecondSel {
    const float* ztab;   // nullptr: Green operator
    int zgroup;
};

template <typename T>
__device__ __forceinline__ void zsym_apply(const float* __restrict__ Z, const cplx_t<T> r[3], cplx_t<T> z[3]) {
    const T a = T(Z[0]), b = T(Z[1]), c = T(Z[2]), d = T(Z[3]), e = T(Z[4]), f = T(Z[5]);
    z[0] = cadd(cadd(cscale(r[0], a), cscale(r[1], f)), cscale(r[2], e));
    z[1] = cadd(cadd(cscale(r[0], f), cscale(r[1], b)), cscale(r[2], d));
    z[2] = cadd(cadd(cscale(r[0], e), cscale(r[1], d)), cscale(r[2], c));
}

template <typename T>
__device__ __forceinline__ void pre_apply(const PrecondSel& ps, const PrecondCoef& pc, int sys, unsigned v,
                                          long long V, T qx, T qy, T qz, const cplx_t<T> r[3], cplx_t<T> z[3]) {
    if (ps.ztab) zsym_apply<T>(ps.ztab + ((size_t)(sys / ps.zgroup) * V + v) * 6, r, z);
    else green_apply(pc, qx, qy, qz, r, z);
}

template <typename T>
__global__ void k_precond(const cplx_t<T>* r, cplx_t<T>* z, const T* __restrict__ qtab, Geo g, PrecondCoef pc,
                          PrecondSel ps, T out_scale) {
    using C = cplx_t<T>;
    const int b = blockIdx.y;
    const T* qb = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    const C* rb = r + (size_t)b * 3 * g.V;
    C* zb = z + (size_t)b * 3 * g.V;
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
        T ax, ay, az;
        voxel_q(qb, g, v, ax, ay, az);
        C rv[3] = {rb[v], rb[g.V + v], rb[2 * g.V + v]};
        C zv[3];
        pre_apply<T>(ps, pc, b, v, g.V, ax, ay, az, rv, zv);
#pragma unroll
        for (int c = 0; c < 3; ++c) zb[c * g.V + v] = cscale(zv[c], out_scale);
    }
}

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV values; result valid in thread 0.
template <typename T, int NV>
__device__ __forceinline__ void block_sum(T (&v)[NV]) {
    __shared__ T red[NV][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) red[i][w] = v[i];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            T s = lane < nw ? red[i][lane] : T(0);
            v[i] = warp_sum(s);
        }
    }
}

// partial[b][blk] = sum over the block's voxels of conj(a) b (complex)
template <typename T>
__global__ void k_dot_partial(const cplx_t<T>* a, const cplx_t<T>* bv, long long n_per, double2* partial) {
    using C = cplx_t<T>;
    const int b = blockIdx.y;
    const C* ab = a + (size_t)b * n_per;
    const C* bb = bv + (size_t)b * n_per;
    T acc[2] = {T(0), T(0)};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_per;
         i += (long long)gridDim.x * blockDim.x) {
        const C x = ab[i], y = bb[i];
        acc[0] += x.x * y.x + x.y * y.y;
        acc[1] += x.x * y.y - x.y * y.x;
    }
    block_sum<T, 2>(acc);
    if (threadIdx.x == 0) partial[(size_t)b * gridDim.x + blockIdx.x] = make_double2(acc[0], acc[1]);
}

static __global__ void k_dot_final(const double2* partial, int nblk, double2* out) {
    const int b = blockIdx.x;
    double acc[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        const double2 v = partial[(size_t)b * nblk + i];
        acc[0] += v.x;
        acc[1] += v.y;
    }
    block_sum<double, 2>(acc);
    if (threadIdx.x == 0) out[b] = make_double2(acc[0], acc[1]);
}

// --------------------------------------------------------------- PCG kernels
// r = s*b - Ax (Ax may be null -> r = s*b, x = 0), p = P^-1 r;
// partials (r,z), (r,r), (s b, s b).
template <typename T>
__global__ void k_cg_init(const cplx_t<T>* bvec, const cplx_t<T>* Ax, cplx_t<T>* x, cplx_t<T>* r, cplx_t<T>* p,
                          const T* __restrict__ qtab, Geo g, PrecondCoef pc, PrecondSel ps, T s, int zero_x,
                          double* partial) {
    using C = cplx_t<T>;
    const int b = blockIdx.y;
    const size_t off = (size_t)b * 3 * g.V;
    const T* qb = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    T acc[3] = {T(0), T(0), T(0)};
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
        C rv[3], zv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t i = off + c * g.V + v;
            const C bs = cscale(bvec[i], s);
            acc[2] += bs.x * bs.x + bs.y * bs.y;
            rv[c] = Ax ? csub(bs, Ax[i]) : bs;
            if (zero_x) x[i] = mk(T(0), T(0));
            r[i] = rv[c];
        }
        T ax, ay, az;
        voxel_q(qb, g, v, ax, ay, az);
        pre_apply<T>(ps, pc, b, v, g.V, ax, ay, az, rv, zv);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            p[off + c * g.V + v] = zv[c];
            acc[0] += rv[c].x * zv[c].x + rv[c].y * zv[c].y;
            acc[1] += rv[c].x * rv[c].x + rv[c].y * rv[c].y;
        }
    }
    block_sum<T, 3>(acc);
    if (threadIdx.x == 0) {
        double* o = partial + ((size_t)b * gridDim.x + blockIdx.x) * 3;
        o[0] = acc[0];
        o[1] = acc[1];
        o[2] = acc[2];
    }
}

// r -= alpha Ap; partials (r, P^-1 r), (r, r).  The matching x += alpha p is
// applied by k_cg_pupdate, which reads p anyway (one pass less over x here).
template <typename T>
__global__ void k_cg_update(cplx_t<T>* __restrict__ r, const cplx_t<T>* __restrict__ Ap,
                            const T* __restrict__ qtab, Geo g, PrecondCoef pc, PrecondSel ps, const CGSys* sys,
                            double* partial) {
    using C = cplx_t<T>;
    const int b = blockIdx.y;
    const size_t off = (size_t)b * 3 * g.V;
    const T* qb = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    const bool act = sys[b].active != 0;
    const T alpha = act ? T(sys[b].alpha) : T(0);
    T acc[2] = {T(0), T(0)};
    if (act) {
#pragma unroll 2
        for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
            C rv[3], zv[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t i = off + c * g.V + v;
                const C av = Ap[i];
                const C ro = r[i];
                rv[c] = mk(fma(-alpha, av.x, ro.x), fma(-alpha, av.y, ro.y));
                r[i] = rv[c];
            }
            T ax, ay, az;
            voxel_q(qb, g, v, ax, ay, az);
            pre_apply<T>(ps, pc, b, v, g.V, ax, ay, az, rv, zv);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[0] += rv[c].x * zv[c].x + rv[c].y * zv[c].y;
                acc[1] += rv[c].x * rv[c].x + rv[c].y * rv[c].y;
            }
        }
    }
    block_sum<T, 2>(acc);
    if (threadIdx.x == 0) {
        double* o = partial + ((size_t)b * gridDim.x + blockIdx.x) * 3;
        o[0] = acc[0];
        o[1] = acc[1];
        o[2] = 0.0;
    }
}

// For systems that took a step: x += alpha p (old p); then, if still active,
// p = P^-1 r + beta p.
template <typename T>
__global__ void k_cg_pupdate(const cplx_t<T>* __restrict__ r, cplx_t<T>* __restrict__ p, cplx_t<T>* __restrict__ x,
                             const T* __restrict__ qtab, Geo g, PrecondCoef pc, PrecondSel ps, const CGSys* sys) {
    using C = cplx_t<T>;
    const int b = blockIdx.y;
    if (!sys[b].upd) return;
    const bool act = sys[b].active != 0;
    const size_t off = (size_t)b * 3 * g.V;
    const T* qb = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    const T alpha = T(sys[b].alpha);
    const T beta = T(sys[b].beta);
#pragma unroll 2
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
        C pv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t i = off + c * g.V + v;
            pv[c] = p[i];
            const C xv = x[i];
            x[i] = mk(fma(alpha, pv[c].x, xv.x), fma(alpha, pv[c].y, xv.y));
        }
        if (act) {
            C rv[3], zv[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) rv[c] = r[off + c * g.V + v];
            T ax, ay, az;
            voxel_q(qb, g, v, ax, ay, az);
            pre_apply<T>(ps, pc, b, v, g.V, ax, ay, az, rv, zv);
#pragma unroll
            for (int c = 0; c < 3; ++c)
                p[off + c * g.V + v] = mk(fma(beta, pv[c].x, zv[c].x), fma(beta, pv[c].y, zv[c].y));
        }
    }
}

// Final sums of the 3-wide partials and the scalar recurrences of Algorithm 2.
// mode 0 (after init): rz, rr, bb; active = rr > tol^2 bb.
// mode 1 (after pAp dot, partial2 holds complex (p, Ap)): alpha = rz / pAp.
// mode 2 (after update): rz_new, rr; converge test; beta = rz_new/rz; rz = rz_new.
static __global__ void k_cg_scalars(const double* partial3, const double2* dots, int nblk, CGSys* sys, int mode,
                             double tol2, int* n_active) {
    const int b = blockIdx.x;
    double acc[3] = {0.0, 0.0, 0.0};
    if (mode != 1) {
        for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
            const double* v = partial3 + ((size_t)b * nblk + i) * 3;
            acc[0] += v[0];
            acc[1] += v[1];
            acc[2] += v[2];
        }
        block_sum<double, 3>(acc);
    }
    if (threadIdx.x != 0) return;
    CGSys& s = sys[b];
    if (mode == 0) {
        s.rz = acc[0];
        s.rr = acc[1];
        s.bb = acc[2];
        s.iters = 0;
        s.upd = 0;
        s.active = (s.rr > tol2 * s.bb) ? 1 : 0;
        if (s.active) atomicAdd(n_active, 1);
    } else if (mode == 1) {
        if (b == 0) *n_active = 0;   // recount in mode 2 (kernels of one stream are ordered)
        s.pAp = dots[b].x;
        s.alpha = (s.active && s.pAp > 0.0) ? s.rz / s.pAp : 0.0;
        s.upd = s.active;
    } else {
        if (!s.active) return;
        s.iters += 1;
        s.rz_new = acc[0];
        s.rr = acc[1];
        if (!(s.rr > tol2 * s.bb) || !(s.rz_new > 0.0)) {
            s.active = 0;
        } else {
            s.beta = s.rz_new / s.rz;
            s.rz = s.rz_new;
            atomicAdd(n_active, 1);
        }
    }
}

// Device tally of PCG runs enqueued without host synchronisation:
// tally[0] += sum of iterations, tally[1] += systems that missed tol,
// tally[2] += systems with a non-finite residual, tally[3] += loop
// iterations executed (*iter, the graph's iteration counter).
static __global__ void k_cg_tally(const CGSys* __restrict__ sys, int nb, double tol2, const int* __restrict__ iter,
                                  long long* __restrict__ tally) {
    long long it = 0, miss = 0, bad = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        it += sys[b].iters;
        const double rr = sys[b].rr, bb = sys[b].bb;
        if (!isfinite(rr) || !isfinite(bb)) ++bad;
        else if (rr > tol2 * bb) ++miss;
    }
    for (int o = 16; o > 0; o >>= 1) {
        it += __shfl_xor_sync(0xffffffffu, it, o);
        miss += __shfl_xor_sync(0xffffffffu, miss, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if (threadIdx.x == 0) {
        tally[0] += it;
        tally[1] += miss;
        tally[2] += bad;
        tally[3] += *iter;
    }
}

}  // namespace bloch
