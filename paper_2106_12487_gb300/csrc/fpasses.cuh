// Two-stage register FFT pass kernels for power-of-two axes N = RA * RB
// (N <= 256), the fast path of the stiffness operator.
//
// Each pencil is transformed in two Stockham stages: stage 1 (radix RA, no
// twiddles) loads its RA inputs straight from HBM into registers and writes
// to a shared-memory exchange buffer; stage 2 (radix RB, twiddles
// w_N^(r j)) reads the exchange buffer and either writes HBM directly or
// keeps its outputs in registers for the pointwise epilogue.  Only one
// shared-memory round trip and one barrier per component remain, and every
// global access is a coalesced row of consecutive pencils (y, z passes) or of
// consecutive elements of a row (x pass).
//
// Stage indexing (Stockham autosort, Ns = 1 then Ns = RA):
//   stage 1 task (p, j), j < RB: reads n = j + r RB, writes slot j RA + r
//   stage 2 task (p, j), j < RA: reads slot j + r RA, twiddle w_N^(r j),
//                                writes n = j + r RA
// The inverse x transform uses radices (RA, RB) and the forward one (RB, RA),
// so the elements a thread holds after the inverse are exactly the inputs of
// its forward stage 1: the stress is applied in registers.
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "passes.cuh"
#include "tma.cuh"

namespace bloch {

template <typename C>
__device__ __forceinline__ C twmul(C v, C w, int dir) {
    if (dir > 0) w.y = -w.y;
    return cmul(v, w);
}

// --------------------------------------------------- y pass (in place ok)
// blockIdx.y = batch*ncomp + comp (offset blockIdx.y * V).  PT pencils (PT
// consecutive x of the (x, z) plane) per CTA; one 32-bit division per task
// locates the pencil, elements step by Nx along it.
template <typename T, int DIR, int RA, int RB, int PT>
__global__ void __launch_bounds__(256) k_fpass_y(const cplx_t<T>* in, cplx_t<T>* out,
                                                 const cplx_t<T>* __restrict__ twa, Geo g) {
    using C = cplx_t<T>;
    constexpr int N = RA * RB;
    constexpr int NT = 256;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;
    const int tid = threadIdx.x;
    const unsigned nx = (unsigned)g.Nx;
    const unsigned npen = nx * (unsigned)g.Nz;
    const unsigned pi0 = blockIdx.x * PT;
    const unsigned plane = nx * (unsigned)g.Ny;
    if (sys_idle(g, (int)blockIdx.y / g.skip_ncomp)) return;
    const size_t off = (size_t)blockIdx.y * g.V;
    const C* src = in + off;
    C* dst = out + off;
    for (int i = tid; i < N; i += NT) tw[i] = twa[i];
#pragma unroll
    for (int t = tid; t < PT * RB; t += NT) {
        const int p = t % PT, j = t / PT;
        const unsigned pi = pi0 + p;
        C v[RA];
        if (pi < npen) {
            const unsigned z = pi / nx;
            const C* a = src + (z * plane + (pi - z * nx) + (unsigned)j * nx);
#pragma unroll
            for (int r = 0; r < RA; ++r) v[r] = a[(unsigned)(r * RB) * nx];
        } else {
#pragma unroll
            for (int r = 0; r < RA; ++r) v[r] = mk(T(0), T(0));
        }
        RegDFT<RA, DIR, C>::run(v);
#pragma unroll
        for (int r = 0; r < RA; ++r) buf[(j * RA + r) * PT + p] = v[r];
    }
    __syncthreads();
#pragma unroll
    for (int t = tid; t < PT * RA; t += NT) {
        const int p = t % PT, j = t / PT;
        C v[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) v[r] = buf[(j + r * RA) * PT + p];
#pragma unroll
        for (int r = 1; r < RB; ++r) v[r] = twmul(v[r], tw[r * j], DIR);
        RegDFT<RB, DIR, C>::run(v);
        const unsigned pi = pi0 + p;
        if (pi < npen) {
            const unsigned z = pi / nx;
            C* a = dst + (z * plane + (pi - z * nx) + (unsigned)j * nx);
#pragma unroll
            for (int r = 0; r < RB; ++r) a[(unsigned)(r * RA) * nx] = v[r];
        }
    }
}

// --------------------------------------------------- pass 1: strain + inverse z
// One thread per stage-2 task (blockDim.x == NT == P * RA, P = NT / RA).  The z
// transform of q_z U_k cannot be formed from that of U_k (q_z varies along
// the pencil), but q_x, q_y are constant on a z pencil, so with
// a_k = F_z^-1(U_k) and b_k = F_z^-1(q_z U_k) the six Voigt strains are
//   g_xx = q_x a_x, g_yy = q_y a_y, g_zz = b_z, g_yz = q_y a_z + b_y,
//   g_xz = q_x a_z + b_x, g_xy = q_y a_x + q_x a_y.
// Each displacement component is read once, in the order z, x, y (only a_z
// and a_x are carried between them); the next component's pencils stream
// into shared memory (cp.async, double buffered) while the current one is
// transformed.
// NT = 256 gives 16-32 neighbouring pencils per CTA, so each z row of the
// tile is 128-256 contiguous bytes in HBM.
// With use_tma the pencils are staged by the tensor memory accelerator: one
// tiled copy of P pencils x N points per component (tensor map over the field
// as [system * component][z][y * Nx + x] of 8-byte values), completed on an
// mbarrier; otherwise by cp.async.  A wait that runs out sets *g.err.
template <typename T, int RA, int RB, int NT = 128>
__global__ void __launch_bounds__(NT, 512 / NT) k_fpass_z_strain(const cplx_t<T>* __restrict__ U, cplx_t<T>* __restrict__ E,
                                                           const T* __restrict__ qtab,
                                                           const cplx_t<T>* __restrict__ twz, Geo g,
                                                           const __grid_constant__ CUtensorMap tmap, int use_tma) {
    using C = cplx_t<T>;
    constexpr int N = RA * RB;
    constexpr int P = NT / RA;
    constexpr int NP = N * P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t zbar[2];
    C* tw = reinterpret_cast<C*>(smem_raw + smem_pad128(smem_raw));   // 128-byte aligned (TMA destinations)
    C* stg = tw + N;          // 2 x NP staging
    C* bufA = stg + 2 * NP;   // NP
    C* bufB = bufA + NP;      // NP
    const int tid = threadIdx.x;
    const int b = blockIdx.y;
    if (sys_idle(g, b)) return;
    if (use_tma) {
        if (tid == 0) {
            mbar_init(smem_u32(&zbar[0]), 1);
            mbar_init(smem_u32(&zbar[1]), 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    const unsigned plane = (unsigned)g.Nx * (unsigned)g.Ny;
    const unsigned pi0 = blockIdx.x * P;
    const int np = (int)min((unsigned)P, plane - pi0);
    const C* Ub = U + (size_t)b * 3 * g.V;
    C* Eb = E + (size_t)b * 6 * g.V;
    const T* qxt = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    const T* qyt = qxt + g.Nx;
    const T* qzt = qyt + g.Ny;
    // FP32 with an even plane: two neighbouring pencils per 16-byte copy, past
    // L1 (P, pi0 and the plane even: 16-byte aligned pairs, each wholly inside
    // or outside the ragged tail); 8-byte copies otherwise
    const bool k16 = sizeof(C) == 8 && P % 2 == 0 && (plane & 1u) == 0;
    auto prefetch = [&](int k, C* dstb) {
        const C* src = Ub + (size_t)k * g.V;
        if (k16) {
#pragma unroll
            for (int e = 2 * tid; e < NP; e += 2 * NT) {
                const int n = e / P, p = e % P;
                const bool ok = p < np;
                cp_async16(dstb + e, src + (ok ? (size_t)n * plane + pi0 + p : 0), ok);
            }
        } else {
#pragma unroll
            for (int e = tid; e < NP; e += NT) {
                const int n = e / P, p = e % P;
                const bool ok = p < np;
                cp_async_cplx(dstb + e, src + (ok ? (size_t)n * plane + pi0 + p : 0), ok);
            }
        }
        cp_async_commit();
    };
    // component k into staging buffer bi
    auto stage_in = [&](int k, int bi) {
        if (use_tma) {
            if (tid == 0) {
                fence_async_smem();
                mbar_expect_tx(smem_u32(&zbar[bi]), (uint32_t)(NP * sizeof(C)));
                tma_load_3d(smem_u32(stg + bi * NP), &tmap, (int)pi0, 0, b * 3 + k, smem_u32(&zbar[bi]));
            }
        } else {
            prefetch(k, stg + bi * NP);
        }
    };
    stage_in(2, 0);
    stage_in(0, 1);
    for (int i = tid; i < N; i += NT) tw[i] = twz[i];
    const int p2 = tid % P, j2 = tid / P;
    const unsigned pi = pi0 + (p2 < np ? p2 : 0);
    const T qx = qxt[pi % (unsigned)g.Nx], qy = qyt[pi / (unsigned)g.Nx];
    // stage 1 has P * RB tasks per transform and two transforms per component
    // (plain and q_z-scaled): with P * RB == NT / 2 the first half of the CTA
    // runs the plain one and the second half the scaled one
    constexpr bool split = 2 * P * RB == NT;
    const int t1 = split ? tid % (P * RB) : tid;
    const int p1 = t1 % P, j1 = t1 / P;
    const bool st1 = split || tid < P * RB;
    const bool scaled = split && tid >= P * RB;
    C az[RB], ax[RB];
    auto store = [&](int c, int r, C v) {
        if (p2 < np) {
            C* d = Eb + (size_t)c * g.V + (size_t)(j2 + r * RA) * plane + pi0 + p2;
            if constexpr (sizeof(C) == 8) st_stream(d, v);
            else *d = v;
        }
    };
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        const int k = kk == 0 ? 2 : kk - 1;   // z, x, y
        if (use_tma) {
            if (!mbar_wait(smem_u32(&zbar[kk & 1]), (uint32_t)((kk >> 1) & 1)) && g.err) atomicExch(g.err, 1);
        } else if (kk < 2) {
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if constexpr (split) {
            const C* sb = stg + (kk & 1) * NP;
            C v[RA];
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                v[r] = sb[(j1 + r * RB) * P + p1];
                if (scaled) v[r] = cscale(v[r], qzt[j1 + r * RB]);
            }
            RegDFT<RA, +1, C>::run(v);
            C* dst = scaled ? bufB : bufA;
#pragma unroll
            for (int r = 0; r < RA; ++r) dst[(j1 * RA + r) * P + p1] = v[r];
        } else if (st1) {
            const C* sb = stg + (kk & 1) * NP;
            C u[RA], v[RA];
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                u[r] = sb[(j1 + r * RB) * P + p1];
                v[r] = u[r];
            }
            RegDFT<RA, +1, C>::run(v);
#pragma unroll
            for (int r = 0; r < RA; ++r) bufA[(j1 * RA + r) * P + p1] = v[r];
#pragma unroll
            for (int r = 0; r < RA; ++r) u[r] = cscale(u[r], qzt[j1 + r * RB]);
            RegDFT<RA, +1, C>::run(u);
#pragma unroll
            for (int r = 0; r < RA; ++r) bufB[(j1 * RA + r) * P + p1] = u[r];
        }
        __syncthreads();
        if (kk == 0) stage_in(1, 0);   // y into the buffer z has left
        C a[RB], bb[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            a[r] = bufA[(j2 + r * RA) * P + p2];
            bb[r] = bufB[(j2 + r * RA) * P + p2];
        }
#pragma unroll
        for (int r = 1; r < RB; ++r) {
            a[r] = twmul(a[r], tw[r * j2], +1);
            bb[r] = twmul(bb[r], tw[r * j2], +1);
        }
        RegDFT<RB, +1, C>::run(a);
        RegDFT<RB, +1, C>::run(bb);
        if (k == 2) {          // z: g_zz; keep a_z
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                store(2, r, bb[r]);
                az[r] = a[r];
            }
        } else if (k == 0) {   // x: g_xx, g_xz; keep a_x
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                store(0, r, cscale(a[r], qx));
                store(4, r, cadd(cscale(az[r], qx), bb[r]));
                ax[r] = a[r];
            }
        } else {               // y: g_yy, g_yz, g_xy
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                store(1, r, cscale(a[r], qy));
                store(3, r, cadd(cscale(az[r], qy), bb[r]));
                store(5, r, cadd(cscale(ax[r], qy), cscale(a[r], qx)));
            }
        }
    }
}

// --------------------------------------------------- pass 5: forward z + divergence
// One thread per stage-2 task (blockDim.x == NT == P * RA); the three output
// components of its RB elements are accumulated in registers:
//   out_x = q_x S11 + q_y S12 + q_z S13, out_y = q_x S12 + q_y S22 + q_z S23,
//   out_z = q_x S13 + q_y S23 + q_z S33   (S = forward z transform of sigma).
// Stress components stream into shared memory two ahead (cp.async).
// With dotp != nullptr the CTA also forms sum conj(dotp) * out over its
// pencils (the (p, A p) product of the PCG iteration, Algorithm 2) and writes
// it to dpart[b * gridDim.x + blockIdx.x].
template <typename T, int RA, int RB, int NT = 128>
__global__ void __launch_bounds__(NT, 512 / NT) k_fpass_z_div(const cplx_t<T>* __restrict__ E, cplx_t<T>* __restrict__ out,
                                                        const T* __restrict__ qtab, const cplx_t<T>* __restrict__ twz,
                                                        Geo g, T out_scale, const cplx_t<T>* __restrict__ dotp,
                                                        double2* __restrict__ dpart,
                                                        const __grid_constant__ CUtensorMap tmap, int use_tma) {
    using C = cplx_t<T>;
    constexpr int N = RA * RB;
    constexpr int P = NT / RA;
    constexpr int NP = N * P;
    // With 2 P RB == NT a component's radix-RA stage has tasks for half of the
    // CTA: the components then go in pairs (first half of the CTA on the
    // pair's first component, second half on its second), two pairs in
    // flight in four staging buffers and one exchange buffer per component.
    constexpr bool pair = 2 * P * RB == NT;
    constexpr int NSTG = pair ? 4 : 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t zbar[4];
    C* tw = reinterpret_cast<C*>(smem_raw + smem_pad128(smem_raw));   // 128-byte aligned (TMA destinations)
    C* stg = tw + N;             // NSTG x NP staging
    C* xb = stg + NSTG * NP;     // (pair ? 2 : 1) x NP exchange
    const int tid = threadIdx.x;
    const int b = blockIdx.y;
    if (sys_idle(g, b)) return;
    if (use_tma) {
        if (tid == 0) {
#pragma unroll
            for (int i = 0; i < NSTG; ++i) mbar_init(smem_u32(&zbar[i]), 1);
            fence_mbar_init();
        }
        __syncthreads();
    }
    const unsigned plane = (unsigned)g.Nx * (unsigned)g.Ny;
    const unsigned pi0 = blockIdx.x * P;
    const int np = (int)min((unsigned)P, plane - pi0);
    const C* Eb = E + (size_t)b * 6 * g.V;
    C* ob = out + (size_t)b * 3 * g.V;
    const T* qxt = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    const T* qyt = qxt + g.Nx;
    const T* qzt = qyt + g.Ny;
    const bool k16 = sizeof(C) == 8 && P % 2 == 0 && (plane & 1u) == 0;   // as in the z-strain pass
    auto prefetch = [&](int c, C* dstb) {
        const C* src = Eb + (size_t)c * g.V;
        if (k16) {
#pragma unroll
            for (int e = 2 * tid; e < NP; e += 2 * NT) {
                const int n = e / P, p = e % P;
                const bool ok = p < np;
                cp_async16(dstb + e, src + (ok ? (size_t)n * plane + pi0 + p : 0), ok);
            }
        } else {
#pragma unroll
            for (int e = tid; e < NP; e += NT) {
                const int n = e / P, p = e % P;
                const bool ok = p < np;
                cp_async_cplx(dstb + e, src + (ok ? (size_t)n * plane + pi0 + p : 0), ok);
            }
        }
        cp_async_commit();
    };
    // component c into staging buffer bi (TMA: one tiled copy, as in the z-strain pass)
    auto stage_in = [&](int c, int bi) {
        if (use_tma) {
            if (tid == 0) {
                fence_async_smem();
                mbar_expect_tx(smem_u32(&zbar[bi]), (uint32_t)(NP * sizeof(C)));
                tma_load_3d(smem_u32(stg + bi * NP), &tmap, (int)pi0, 0, b * 6 + c, smem_u32(&zbar[bi]));
            }
        } else {
            prefetch(c, stg + bi * NP);
        }
    };
    auto stage_wait = [&](int bi, int parity) {
        if (!mbar_wait(smem_u32(&zbar[bi]), (uint32_t)parity) && g.err) atomicExch(g.err, 1);
    };
#pragma unroll
    for (int c = 0; c < NSTG; ++c) stage_in(c, c);
    for (int i = tid; i < N; i += NT) tw[i] = twz[i];
    const int p2 = tid % P, j2 = tid / P;
    const unsigned pi = pi0 + (p2 < np ? p2 : 0);
    const T qv[2] = {qxt[pi % (unsigned)g.Nx], qyt[pi / (unsigned)g.Nx]};
    const int t1 = pair ? tid % (P * RB) : tid;
    const int p1 = t1 % P, j1 = t1 / P;
    const int half = pair ? tid / (P * RB) : 0;
    const bool st1 = pair || tid < P * RB;
    C acc[3][RB];
    // stage 2 of component c from exchange buffer xc, accumulated into out_a, out_b:
    // sigma_c contributes q_b sigma to out_a and q_a sigma to out_b
    auto stage2 = [&](const int c, const C* xc) {
        C v[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) v[r] = xc[(j2 + r * RA) * P + p2];
#pragma unroll
        for (int r = 1; r < RB; ++r) v[r] = twmul(v[r], tw[r * j2], -1);
        RegDFT<RB, -1, C>::run(v);
        const int ca = c < 3 ? c : (c == 3 ? 1 : 0);
        const int cb = c < 3 ? c : (c == 5 ? 1 : 2);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const T qz = qzt[j2 + r * RA];
            const T qa = ca == 2 ? qz : qv[ca];
            const T qb = cb == 2 ? qz : qv[cb];
            if (c < 3) {
                acc[ca][r] = cscale(v[r], qa);
            } else {
                acc[ca][r] = cadd(acc[ca][r], cscale(v[r], qb));
                acc[cb][r] = cadd(acc[cb][r], cscale(v[r], qa));
            }
        }
    };
    if constexpr (pair) {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            if (use_tma) {
                stage_wait((m & 1) * 2, m >> 1);
                stage_wait((m & 1) * 2 + 1, m >> 1);
            } else if (m < 2) {
                cp_async_wait<2>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();   // pair m landed; every thread is past the exchange reads of pair m - 1
            {
                const C* sb = stg + ((m & 1) * 2 + half) * NP;
                C v[RA];
#pragma unroll
                for (int r = 0; r < RA; ++r) v[r] = sb[(j1 + r * RB) * P + p1];
                RegDFT<RA, -1, C>::run(v);
                C* xh = xb + half * NP;
#pragma unroll
                for (int r = 0; r < RA; ++r) xh[(j1 * RA + r) * P + p1] = v[r];
            }
            __syncthreads();   // exchange written; the staging buffers of pair m are free
            if (m == 0) {
                stage_in(4, 0);
                stage_in(5, 1);
            }
            stage2(2 * m, xb);
            stage2(2 * m + 1, xb + NP);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (use_tma) stage_wait(c & 1, (c >> 1) & 1);
            else if (c < 5) cp_async_wait<1>();
            else cp_async_wait<0>();
            __syncthreads();
            if (st1) {
                const C* sb = stg + (c & 1) * NP;
                C v[RA];
#pragma unroll
                for (int r = 0; r < RA; ++r) v[r] = sb[(j1 + r * RB) * P + p1];
                RegDFT<RA, -1, C>::run(v);
#pragma unroll
                for (int r = 0; r < RA; ++r) xb[(j1 * RA + r) * P + p1] = v[r];
            }
            __syncthreads();
            if (c + 2 < 6) stage_in(c + 2, c & 1);
            else if (!use_tma) cp_async_commit();
            stage2(c, xb);
        }
    }
    T dre = T(0), dim = T(0);
    const C* pb = dotp ? dotp + (size_t)b * 3 * g.V : nullptr;
    if (p2 < np) {
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            const size_t a = (size_t)(j2 + r * RA) * plane + pi0 + p2;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const C o = cscale(acc[i][r], out_scale);
                if constexpr (sizeof(C) == 8) st_stream(ob + (size_t)i * g.V + a, o);
                else ob[(size_t)i * g.V + a] = o;
                if (pb) {
                    const C pv = pb[(size_t)i * g.V + a];
                    dre += pv.x * o.x + pv.y * o.y;
                    dim += pv.x * o.y - pv.y * o.x;
                }
            }
        }
    }
    if (dotp) {   // block reduction (NT / 32 warps); deterministic order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dre += __shfl_xor_sync(0xffffffffu, dre, o);
            dim += __shfl_xor_sync(0xffffffffu, dim, o);
        }
        __shared__ T red[2][NT / 32];
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = dre;
            red[1][tid >> 5] = dim;
        }
        __syncthreads();
        if (tid == 0) {
            double sr = 0.0, si = 0.0;
#pragma unroll
            for (int w = 0; w < NT / 32; ++w) {
                sr += (double)red[0][w];
                si += (double)red[1][w];
            }
            dpart[(size_t)b * gridDim.x + blockIdx.x] = make_double2(sr, si);
        }
    }
}

// --------------------------------------------------- pass 3: x rows, stress in registers
// One thread owns one stage-2 task (row p, j < RA) for all six components:
// blockDim.x == P * RA is required.  Shared rows are padded (one slot every 16)
// to spread the strided Stockham writes over the banks.
__device__ __forceinline__ int xpad(int n) { return n + (n >> 4); }

// Index of C_ij (any order) in the packed upper triangle of a symmetric 6x6.
__host__ __device__ constexpr int sym6(int i, int j) {
    return i <= j ? i * 6 - i * (i - 1) / 2 + (j - i) : j * 6 - j * (j - 1) / 2 + (i - j);
}

// sigma = C_g gamma at the element r of every component (packed symmetric
// table, 21 per grain), one row of C_g at a time so that few coefficients
// are live next to the six components held per element.
template <typename T, typename C, int R>
__device__ __forceinline__ void stress_at(C (&s)[6][R], int r, const T* __restrict__ Cg, T& energy) {
    C sig[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T sr = 0, si = 0;
#pragma unroll
        for (int jj = 0; jj < 6; ++jj) {
            const T cij = __ldg(Cg + sym6(i, jj));
            sr = fma(cij, s[jj][r].x, sr);
            si = fma(cij, s[jj][r].y, si);
        }
        sig[i] = mk(sr, si);
        energy = fma(s[i][r].x, sr, fma(s[i][r].y, si, energy));
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i][r] = sig[i];
}

// CTA sum in two steps around a barrier the caller already has: warp sums
// into red[] before it, thread 0 adds them (FP64) after it.
template <typename T>
__device__ __forceinline__ void warp_sum_to(T v, T* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
}
template <int NW, typename T>
__device__ __forceinline__ void red_to(const T* red, double2* dst) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) t += (double)red[w];
    *dst = make_double2(t, 0.0);
}

template <typename T, int RA, int RB>
__device__ __forceinline__ void x_stress_single(cplx_t<T>* E, const int32_t* __restrict__ ids,
                                                const T* __restrict__ Cpk, const cplx_t<T>* __restrict__ twx,
                                                const Geo& g, double2* __restrict__ dpart) {
    using C = cplx_t<T>;
    constexpr int N = RA * RB;
    constexpr int LD = N + N / 16;
    constexpr int P = 128 / RA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* stg = tw + N;          // 2 x P*LD staging (rows unpadded inside), reused by the forward exchange
    C* xb = stg + 2 * P * LD; // P*LD exchange of the inverse transform
    const int tid = threadIdx.x;
    const int b = blockIdx.y;
    const unsigned rows = (unsigned)g.Ny * (unsigned)g.Nz;
    const unsigned r0 = blockIdx.x * P;
    const int nr = (int)min((unsigned)P, rows - r0);
    C* Eb = E + (size_t)b * 6 * g.V;
    auto prefetch = [&](int c, C* dstb) {
        const C* src = Eb + (size_t)c * g.V + (size_t)r0 * N;
        if constexpr (LD % 2 == 0 && sizeof(C) == 8) {   // 16-byte rows: two values per copy, past L1
#pragma unroll
            for (int e = tid; e < P * N / 2; e += 128) {
                const int p = e / (N / 2), n = 2 * (e % (N / 2));
                const bool ok = p < nr;
                cp_async16(dstb + p * LD + n, src + (ok ? p * N + n : 0), ok);
            }
        } else {
#pragma unroll
            for (int e = tid; e < P * N; e += 128) {
                const int p = e / N, n = e % N;
                const bool ok = p < nr;
                cp_async_cplx(dstb + p * LD + n, src + (ok ? e : 0), ok);
            }
        }
        cp_async_commit();
    };
    prefetch(0, stg);
    prefetch(1, stg + P * LD);
    for (int i = tid; i < N; i += 128) tw[i] = twx[i];
    // stage-2 task of this thread
    const int j2 = tid % RA, p2 = tid / RA;
    const bool own = p2 < nr;
    C s[6][RB];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        if (c < 5) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();
        // inverse stage 1 (radix RA): tasks (p, j < RB), j fastest
        if (tid < P * RB) {
            const int j = tid % RB, p = tid / RB;
            const C* sb = stg + (c & 1) * P * LD + p * LD;
            C v[RA];
#pragma unroll
            for (int r = 0; r < RA; ++r) v[r] = sb[j + r * RB];
            RegDFT<RA, +1, C>::run(v);
#pragma unroll
            for (int r = 0; r < RA; ++r) xb[p * LD + xpad(j * RA + r)] = v[r];
        }
        __syncthreads();
        if (c + 2 < 6) prefetch(c + 2, stg + (c & 1) * P * LD);
        else cp_async_commit();
        // inverse stage 2 (radix RB), kept in registers
        C v[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) v[r] = xb[p2 * LD + xpad(j2 + r * RA)];
#pragma unroll
        for (int r = 1; r < RB; ++r) v[r] = twmul(v[r], tw[r * j2], +1);
        RegDFT<RB, +1, C>::run(v);
#pragma unroll
        for (int r = 0; r < RB; ++r) s[c][r] = v[r];
    }
    // stress sigma = C_g gamma at the RB owned elements (packed symmetric table, 21 per grain)
    __shared__ T red[4];
    {
        T energy = T(0);
        if (own) {
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                T e = T(0);
                stress_at<T>(s, r, Cpk + (size_t)ids[(size_t)(r0 + p2) * N + j2 + r * RA] * 21, e);
                energy += e;
            }
        }
        if (dpart) warp_sum_to(energy, red);
    }
    __syncthreads();   // the staging buffers become the forward exchange buffers; red[] complete
    if (dpart && tid == 0) red_to<4>(red, dpart + (size_t)b * gridDim.x + blockIdx.x);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        C* buf = stg + (c & 1) * P * LD;
        // forward stage 1 (radix RB, Ns = 1): the owned elements j2 + r RA are its inputs
        {
            C v[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) v[r] = s[c][r];
            RegDFT<RB, -1, C>::run(v);
#pragma unroll
            for (int r = 0; r < RB; ++r) buf[p2 * LD + xpad(j2 * RB + r)] = v[r];
        }
        __syncthreads();
        // forward stage 2 (radix RA, Ns = RB): tasks (p, j < RB)
        if (tid < P * RB) {
            const int j = tid % RB, p = tid / RB;
            C v[RA];
#pragma unroll
            for (int r = 0; r < RA; ++r) v[r] = buf[p * LD + xpad(j + r * RB)];
#pragma unroll
            for (int r = 1; r < RA; ++r) v[r] = twmul(v[r], tw[r * j], -1);
            RegDFT<RA, -1, C>::run(v);
            if (p < nr) {
#pragma unroll
                for (int r = 0; r < RA; ++r) Eb[(size_t)c * g.V + (size_t)(r0 + p) * N + j + r * RB] = v[r];
            }
        }
    }
}


// Balanced form for P * RB == 64 (N = 128 as 16 x 8, N = 32 as 8 x 4), where a
// component's radix-RA stage has tasks for only half of the 128 threads: the
// components are taken in pairs, threads 0-63 running the radix-RA stage of
// the pair's first component and threads 64-127 that of the second, so every
// warp works in every stage and one barrier serves two components.  The
// pairs' pencils stream in by cp.async, two pairs in flight (four staging
// buffers); the grain ids of the CTA's rows follow as a fifth group, so the
// stress step reads them from shared memory.  10 barriers per CTA.
template <int N>
constexpr int x_ids_ld() { return N + 16; }

template <typename T, int RA, int RB>
__device__ __forceinline__ void x_stress_paired(cplx_t<T>* E, const int32_t* __restrict__ ids,
                                                const T* __restrict__ Cpk, const cplx_t<T>* __restrict__ twx,
                                                const Geo& g, double2* __restrict__ dpart) {
    using C = cplx_t<T>;
    constexpr int N = RA * RB;
    constexpr int LD = N + N / 16;
    constexpr int P = 128 / RA;
    constexpr int LI = x_ids_ld<N>();
    static_assert(P * RB == 64, "paired x pass needs P * RB == 64");
    static_assert(P * LI * sizeof(int32_t) <= P * LD * sizeof(C), "grain-id tile must fit a staging buffer");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* stg = tw + N;          // 4 x P*LD: pair buffers (set 0: 0, 1; set 1: 2, 3)
    C* xb = stg + 4 * P * LD; // 2 x P*LD exchange of the inverse transform
    int32_t* sid = reinterpret_cast<int32_t*>(stg + 2 * P * LD);   // set 1, buffer 0, once free
    const int tid = threadIdx.x;
    const int b = blockIdx.y;
    const unsigned rows = (unsigned)g.Ny * (unsigned)g.Nz;
    const unsigned r0 = blockIdx.x * P;
    const int nr = (int)min((unsigned)P, rows - r0);
    C* Eb = E + (size_t)b * 6 * g.V;
    // two complex values per 16-byte copy, past L1 (which then keeps the stiffness table)
    static_assert(sizeof(C) == 8 && LD % 2 == 0, "paired x pass stages FP32 complex values in 16-byte rows");
    auto prefetch = [&](int c, C* dstb) {
        const C* src = Eb + (size_t)c * g.V + (size_t)r0 * N;
#pragma unroll
        for (int e = tid; e < P * N / 2; e += 128) {
            const int p = e / (N / 2), n = 2 * (e % (N / 2));
            const bool ok = p < nr;
            cp_async16(dstb + p * LD + n, src + (ok ? p * N + n : 0), ok);
        }
    };
    prefetch(0, stg);
    prefetch(1, stg + P * LD);
    cp_async_commit();
    prefetch(2, stg + 2 * P * LD);
    prefetch(3, stg + 3 * P * LD);
    cp_async_commit();
    for (int i = tid; i < N; i += 128) tw[i] = twx[i];
    const int half = tid >> 6;              // radix-RA stage: component 2m + half
    const int j1 = (tid & 63) % RB, p1 = (tid & 63) / RB;
    const int j2 = tid % RA, p2 = tid / RA; // radix-RB stage and the stress: one task per thread
    const bool own = p2 < nr;
    C s[6][RB];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        if (m < 2) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();   // pair m landed; every thread is past the exchange reads of pair m - 1
        {
            const C* sb = stg + ((m & 1) * 2 + half) * P * LD + p1 * LD;
            C v[RA];
#pragma unroll
            for (int r = 0; r < RA; ++r) v[r] = sb[j1 + r * RB];
            RegDFT<RA, +1, C>::run(v);
            C* xh = xb + half * P * LD + p1 * LD;
#pragma unroll
            for (int r = 0; r < RA; ++r) xh[xpad(j1 * RA + r)] = v[r];
        }
        __syncthreads();   // exchange written; the staging buffers of pair m are free
        if (m == 0) {      // pair 2 into set 0
            prefetch(4, stg);
            prefetch(5, stg + P * LD);
            cp_async_commit();
        } else if (m == 1) {   // the grain ids of the CTA's rows into set 1
            for (int e = tid; e < P * (N / 4); e += 128) {
                const int p = e / (N / 4), n4 = e % (N / 4);
                const bool ok = p < nr;
                cp_async16(sid + p * LI + 4 * n4, ids + (ok ? (size_t)(r0 + p) * N + 4 * n4 : 0), ok);
            }
            cp_async_commit();
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            C v[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) v[r] = xb[h * P * LD + p2 * LD + xpad(j2 + r * RA)];
#pragma unroll
            for (int r = 1; r < RB; ++r) v[r] = twmul(v[r], tw[r * j2], +1);
            RegDFT<RB, +1, C>::run(v);
#pragma unroll
            for (int r = 0; r < RB; ++r) s[2 * m + h][r] = v[r];
        }
    }
    cp_async_wait<0>();
    __syncthreads();   // grain ids visible; all staging buffers free for the forward exchange
    __shared__ T red[4];
    {
        T energy = T(0);
        if (own) {
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                T e = T(0);
                stress_at<T>(s, r, Cpk + (size_t)sid[p2 * LI + j2 + r * RA] * 21, e);
                energy += e;
            }
        }
        if (dpart) warp_sum_to(energy, red);
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        C* bufs = stg + (m & 1) * 2 * P * LD;
        // forward stage 1 (radix RB) of both components by every thread
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            C v[RB];
#pragma unroll
            for (int r = 0; r < RB; ++r) v[r] = s[2 * m + h][r];
            RegDFT<RB, -1, C>::run(v);
#pragma unroll
            for (int r = 0; r < RB; ++r) bufs[h * P * LD + p2 * LD + xpad(j2 * RB + r)] = v[r];
        }
        __syncthreads();   // a thread writing this buffer set again (pair m + 2) has passed the next barrier
        if (m == 0 && dpart && tid == 0) red_to<4>(red, dpart + (size_t)blockIdx.y * gridDim.x + blockIdx.x);
        // forward stage 2 (radix RA): component 2m + half
        {
            C v[RA];
            const C* bh = bufs + half * P * LD + p1 * LD;
#pragma unroll
            for (int r = 0; r < RA; ++r) v[r] = bh[xpad(j1 + r * RB)];
#pragma unroll
            for (int r = 1; r < RA; ++r) v[r] = twmul(v[r], tw[r * j1], -1);
            RegDFT<RA, -1, C>::run(v);
            if (p1 < nr) {
                C* dst = Eb + (size_t)(2 * m + half) * g.V + (size_t)(r0 + p1) * N + j1;
#pragma unroll
                for (int r = 0; r < RA; ++r) st_stream(dst + r * RB, v[r]);
            }
        }
    }
}

// Shared memory of k_fpass_z_strain<T, RA, RB, NT> and k_fpass_z_div<T, RA, RB, NT> (bytes).
template <typename T, int RA, int RB, int NT>
constexpr size_t fpass_z1_smem() {
    return (size_t)(RA * RB + 4 * RA * RB * (NT / RA)) * sizeof(cplx_t<T>) + kSmemAlignSlack;
}
template <typename T, int RA, int RB, int NT>
constexpr size_t fpass_z5_smem() {
    constexpr int P = NT / RA, NP = RA * RB * P;
    return (size_t)(RA * RB + (2 * P * RB == NT ? 6 : 3) * NP) * sizeof(cplx_t<T>) + kSmemAlignSlack;
}

// Shared memory of k_fpass_x_stress<T, RA, RB> (bytes).
template <typename T, int RA, int RB>
constexpr size_t fpass_x_smem() {
    constexpr int N = RA * RB, LD = N + N / 16, P = 128 / RA;
    return (size_t)(N + (P * RB == 64 ? 6 : 3) * P * LD) * sizeof(cplx_t<T>);
}

// With dpart != nullptr the CTA also forms the strain energy sum over its
// points of conj(gamma) . sigma, which by Parseval equals its share of
// (u, A_k u) for the apply's input u (the passes' transforms are unnormalised
// and the divergence is the transpose of the strain map), and writes it to
// dpart[b * gridDim.x + blockIdx.x]: the (p, A p) product of the PCG
// iteration (Algorithm 2) without a second read of p.
template <typename T, int RA, int RB>
__global__ void __launch_bounds__(128, 4) k_fpass_x_stress(cplx_t<T>* E, const int32_t* __restrict__ ids,
                                                           const T* __restrict__ Cpk,
                                                           const cplx_t<T>* __restrict__ twx, Geo g,
                                                           double2* __restrict__ dpart) {
    if (sys_idle(g, blockIdx.y)) return;
    if constexpr ((128 / RA) * RB == 64)
        x_stress_paired<T, RA, RB>(E, ids, Cpk, twx, g, dpart);
    else
        x_stress_single<T, RA, RB>(E, ids, Cpk, twx, g, dpart);
}

}  // namespace bloch
