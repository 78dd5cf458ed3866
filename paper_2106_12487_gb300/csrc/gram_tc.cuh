// Tensor-core (tcgen05) form of the Algorithm 1 projections for FP32 blocks:
//   K[i][j] = sum_e conj(A_i(e)) Bk_j(e),   M[i][j] = sum_e conj(A_i(e)) C_j(e)
// with C = Bm, or C = A for a uniform density.
//
// Real form.  A complex vector x of n elements is the real vector of its 2n
// interleaved (re, im) floats; rot(x) = (im, -re) element by element.  Then
//   Re conj(a).b = <a, b>,   Im conj(a).b = -<rot(a), b>.
// With the 2q "P" rows p_r = Bk_r (r < q), C_{r-q} (q <= r < 2q) and the 2q
// "Q" rows q_j = A_j (j < q), rot(A_{j-q}) (q <= j < 2q):
//   Re K[j][r] = <p_r, q_j>,     Im K[j][r] = -<p_r, q_{q+j}>,
//   Re M[j][r] = <p_{q+r}, q_j>, Im M[j][r] = -<p_{q+r}, q_{q+j}>.
// FP32 accuracy from TF32 inputs: x = hi + lo with hi = x rounded to TF32 and
// lo = x - hi (exact), <p, q> = <ph, qh> + <ph, ql> + <pl, qh> up to the
// dropped <pl, ql> (below 2^-22 of each product).  The split is stacked into
// the operands: the MMA's 128-row A operand holds ph (rows 0..2q-1) and pl
// (rows 2q..4q-1), its B operand qh (rows 0..2q-1) and ql (rows 2q..4q-1), so
// ONE MMA chain D = [ph; pl] [qh; ql]^T forms all four products at once, and
//   <p_r, q_j> = D[r][j] + D[r][2q + j] + D[2q + r][j].
//
// Data flow per CTA (one slot, a strided range of chunks of kTCElems complex
// elements): 256 threads load the chunk's rows from HBM (each warp 8 rows x 4
// elements: full 32-byte sectors), split them into hi/lo (and rot) and store
// them in the K-major, unswizzled core-matrix layout (8 rows x 16 bytes per
// 128-byte core matrix; core matrices adjacent in K 128 bytes apart, 8-row
// groups kTCSBO bytes apart) of one of two stages; one thread then issues the
// stage's MMAs (M = 128, N = Npad >= 4q, K = 8 floats each) into an FP32
// accumulator in tensor memory and commits them to the stage's mbarrier, which
// the threads wait on before they refill that stage.  Rows of A beyond 4q are
// never written: the 128-row operand reads whatever follows in shared memory
// there, which only reaches accumulator rows that are discarded.  At the end
// warps 0-3 copy the accumulator (warp w owns lanes 32w..32w+31 = rows of D)
// to shared memory, and all threads combine it into the CTA's partial K and M
// in FP64, in the layout k_gram_final sums.  Every wait is bounded: on a
// timeout the kernel raises *err and returns after releasing its tensor memory.
#pragma once

#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "tma.cuh"

namespace bloch {

constexpr int kTCThreads = 256;
constexpr int kQMaxTC = 32;                  // block size limit (4q rows fill M = 128)
constexpr int kTCElems = 32;                 // complex elements of a chunk
constexpr int kTCK = 2 * kTCElems;           // floats of a chunk (K extent of a stage)
constexpr int kTCSBO = (kTCK / 4) * 128;     // bytes between 8-row groups of a tile
constexpr int kTCLBO = 128;                  // bytes between core matrices adjacent in K

__host__ __device__ constexpr int tc_npad(int q) { return ((4 * q + 15) / 16) * 16; }
__host__ __device__ constexpr int tc_agroups(int q) { return (4 * q + 7) / 8; }
__host__ __device__ constexpr int tc_stage_bytes(int q) { return (tc_agroups(q) + tc_npad(q) / 8) * kTCSBO; }
__host__ __device__ constexpr int tc_tmem_cols(int q) { return tc_npad(q) <= 32 ? 32 : (tc_npad(q) <= 64 ? 64 : 128); }
// shared memory of k_gram_tc: two stages, room for the 128-row reads of the
// last stage's A tile, and the accumulator copy of the epilogue
inline size_t tc_smem_bytes(int q) {
    const size_t stage = (size_t)tc_stage_bytes(q);
    const size_t need_read = stage + 16 * (size_t)kTCSBO;
    const size_t dcopy = (size_t)128 * (tc_npad(q) + 1) * sizeof(float);
    return std::max(std::max(2 * stage, need_read), dcopy);
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// shared memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kTCLBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((kTCSBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// instruction descriptor: D f32, A and B tf32, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t tc_idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

// byte offset of element (row, k) of a K-major unswizzled tile
__device__ __forceinline__ uint32_t tc_off(int row, int k) {
    return (uint32_t)((row >> 3) * kTCSBO + (k >> 2) * kTCLBO + (row & 7) * 16 + (k & 3) * 4);
}

// hi part at row rh, lo part at row rh + lo_off of the same tile
__device__ __forceinline__ void tc_put(unsigned char* tile, int rh, int lo_off, int k, float x, float y) {
    const float hx = to_tf32(x), hy = to_tf32(y);
    *reinterpret_cast<float2*>(tile + tc_off(rh, k)) = make_float2(hx, hy);
    *reinterpret_cast<float2*>(tile + tc_off(rh + lo_off, k)) = make_float2(x - hx, y - hy);
}

__global__ void __launch_bounds__(kTCThreads) k_gram_tc(const float2* __restrict__ A, const float2* __restrict__ Bk,
                                                        const float2* __restrict__ Bm, int q, long long n_per,
                                                        double2* __restrict__ partial, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ __align__(8) unsigned long long bars[2];
    __shared__ uint32_t tmem_base;
    __shared__ int wait_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool has_m = Bm != nullptr;
    const int npad = tc_npad(q), ag = tc_agroups(q), ncols = tc_tmem_cols(q);
    const int stage = tc_stage_bytes(q);
    const int q2 = 2 * q;                     // rows of one split half
    const int nsrc = has_m ? 3 * q : 2 * q;   // source rows: Bk, A, (Bm)
    const int slot = blockIdx.y;
    const size_t sbase = (size_t)slot * q * n_per;
    const long long nchunk = (n_per + kTCElems - 1) / kTCElems;
    auto atile = [&](int s) -> unsigned char* { return sm + (size_t)s * stage; };
    auto btile = [&](int s) -> unsigned char* { return sm + (size_t)s * stage + (size_t)ag * kTCSBO; };
    // zero the padding rows once: A rows 4q .. 8ag, B rows 4q .. npad
    for (int s = 0; s < 2; ++s)
        for (int w = 0; w < 2; ++w) {
            const int r0 = 2 * q2, r1 = w == 0 ? 8 * ag : npad;
            unsigned char* t0 = w == 0 ? atile(s) : btile(s);
            for (int t = tid; t < (r1 - r0) * kTCK; t += kTCThreads)
                *reinterpret_cast<float*>(t0 + tc_off(r0 + t / kTCK, t % kTCK)) = 0.f;
        }
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t dtm = tmem_base;
    const uint32_t idesc = tc_idesc(npad);
    // warp task t: source rows 8 (t / 8) .. +7, elements 4 (t % 8) .. +3 of the chunk;
    // lane: row 8 (t / 8) + lane / 4, element 4 (t % 8) + lane % 4
    const int ntask = ((nsrc + 7) / 8) * (kTCElems / 4);
    constexpr int kMaxT = (3 * kQMaxTC / 8) * (kTCElems / 4) / (kTCThreads / 32);   // warp tasks per warp
    float2 cur[kMaxT], nxt[kMaxT];
    auto load = [&](long long ch, float2 (&v)[kMaxT]) {
#pragma unroll
        for (int i = 0; i < kMaxT; ++i) {
            const int t = warp + i * (kTCThreads / 32);
            v[i] = make_float2(0.f, 0.f);
            if (t < ntask && ch < nchunk) {
                const int s = 8 * (t / (kTCElems / 4)) + lane / 4;
                const long long e = ch * kTCElems + 4 * (t % (kTCElems / 4)) + (lane & 3);
                if (s < nsrc && e < n_per) {
                    const float2* src = s < q ? Bk + sbase + (size_t)s * n_per
                                              : (s < 2 * q ? A + sbase + (size_t)(s - q) * n_per
                                                           : Bm + sbase + (size_t)(s - 2 * q) * n_per);
                    v[i] = __ldg(src + e);
                }
            }
        }
    };
    bool ok = true;
    long long it = 0;
    long long ch = blockIdx.x;
    if (ch < nchunk) load(ch, cur);
    for (; ch < nchunk; ch += gridDim.x, ++it) {
        const int s = (int)(it & 1);
        load(ch + gridDim.x, nxt);   // next chunk in flight while this one is staged
        if (it >= 2) {   // the MMAs of iteration it - 2 have read this stage
            if (tid == 0) wait_ok = mbar_wait(smem_u32(&bars[s]), (uint32_t)(((it - 2) >> 1) & 1)) ? 1 : 0;
            __syncthreads();
            if (!wait_ok) {   // uniform across the block
                ok = false;
                break;
            }
        }
        unsigned char* at = atile(s);
        unsigned char* bt = btile(s);
#pragma unroll
        for (int i = 0; i < kMaxT; ++i) {
            const int t = warp + i * (kTCThreads / 32);
            if (t >= ntask) continue;
            const int src = 8 * (t / (kTCElems / 4)) + lane / 4;
            if (src >= nsrc) continue;
            const int k = 2 * (4 * (t % (kTCElems / 4)) + (lane & 3));
            const float2 v = cur[i];
            if (src < q) {
                tc_put(at, src, q2, k, v.x, v.y);                     // Bk_r -> p_r
            } else if (src < 2 * q) {
                const int j = src - q;
                tc_put(bt, j, q2, k, v.x, v.y);                       // A_j -> q_j
                tc_put(bt, q + j, q2, k, v.y, -v.x);                  // rot(A_j) -> q_{q+j}
                if (!has_m) tc_put(at, q + j, q2, k, v.x, v.y);       // C_j = A_j -> p_{q+j}
            } else {
                tc_put(at, q + (src - 2 * q), q2, k, v.x, v.y);       // C_j = Bm_j -> p_{q+j}
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t ba = smem_u32(at), bb = smem_u32(bt);
#pragma unroll
            for (int ks = 0; ks < kTCK / 8; ++ks) {
                const uint32_t o = (uint32_t)(ks * 2 * kTCLBO);
                tc_mma(dtm, tc_desc(ba + o), tc_desc(bb + o), idesc, (it > 0 || ks > 0) ? 1 : 0);
            }
            tc_commit(smem_u32(&bars[s]));
        }
#pragma unroll
        for (int i = 0; i < kMaxT; ++i) cur[i] = nxt[i];
    }
    // drain: the last one or two stages still in flight
    if (tid == 0) {
        bool d = ok;
        if (d && it >= 1) d = mbar_wait(smem_u32(&bars[(it - 1) & 1]), (uint32_t)(((it - 1) >> 1) & 1));
        if (d && it >= 2) d = mbar_wait(smem_u32(&bars[(it - 2) & 1]), (uint32_t)(((it - 2) >> 1) & 1));
        wait_ok = d ? 1 : 0;
        if (!d) atomicExch(err, 1);
    }
    __syncthreads();
    ok = wait_ok != 0;
    tc_fence_after();
    // accumulator -> shared memory (the stages are free now): dsm[row][col],
    // rows padded by one float so a warp's 32 rows fall in different banks
    float* dsm = reinterpret_cast<float*>(sm);
    const int ld = npad + 1;
    if (warp < 4) {
        const int r = 32 * warp + lane;
        for (int c0 = 0; c0 < npad; c0 += 16) {
            uint32_t v[16];
            if (it > 0 && ok) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(dtm + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0u;   // no chunk reached this CTA (or a timeout)
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) dsm[(size_t)r * ld + c0 + i] = __uint_as_float(v[i]);
        }
    }
    tc_fence_before();
    __syncthreads();
    // <p_r, q_j> = D[r][j] + D[r][2q + j] + D[2q + r][j]
    auto dot = [&](int r, int j) -> double {
        return (double)dsm[(size_t)r * ld + j] + (double)dsm[(size_t)r * ld + q2 + j] +
               (double)dsm[(size_t)(q2 + r) * ld + j];
    };
    const int npair = q * q;
    double2* out = partial + ((size_t)slot * gridDim.x + blockIdx.x) * 2 * npair;
    for (int t = tid; t < 2 * npair; t += kTCThreads) {
        const int w = t / npair, pr = t - w * npair;   // w 0: K, 1: M; entry X[j][r]
        const int j = pr / q, r = pr - j * q;
        const int pr_row = w * q + r;
        out[t] = make_double2(dot(pr_row, j), -dot(pr_row, q + j));
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(dtm), "r"(ncols) : "memory");
    }
}

}  // namespace bloch
