// Learned Fourier-space preconditioner: data collection from PCG runs,
// hand-written training (forward, backward, Adam) and the inference tables
// read by the CG kernels.  See learned.cuh for the model.
//
// Data: for each wave vector of a collection call, n_rhs seeded right-hand
// sides are solved to 1e-6 (x*); PCG is then rerun from zero and after each
// of its first n_iters iterations the per-Fourier-voxel moments of the
// residual r_j and error e_j = x* - x_j (both scaled by 1/||r_j||) are
// accumulated: A = Re r r^H, B = sym Re r e^H (six entries each), c = |e|^2.
// The loss of a parameter vector is sum_bins tr(Z Z A) - 2 tr(Z B) + c,
// normalised by the number of recorded iterates.
#include <cuda_runtime.h>

#include <atomic>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "eig_kernels.cuh"
#include "internal.h"
#include "learned.cuh"

namespace bloch {
constexpr int kLPH = 16;   // hidden width
constexpr int kLPN = lp_nparams(kLPH);
constexpr int kMom = 13;   // A (6), B (6), c
}  // namespace bloch

struct bloch_lp {
    float* d_prm = nullptr;     // kLPN parameters (device)
    float* d_m = nullptr;       // Adam moments
    float* d_v = nullptr;
    double* d_grad = nullptr;   // kLPN gradient + loss
    int adam_t = 0;
    unsigned long long version = 0;   // process-unique, renewed whenever the parameters change
    struct Block {
        int grid[3];
        long long V;
        float* d_mom;           // V x 13
        float* d_q;             // Nx+Ny+Nz scaled q table
        bloch::PrecondCoef pc;  // scaled C0 coefficients
        double C0V[36];         // scaled C0 (Voigt) for export
        float snorm;
        int samples;            // recorded iterates
    };
    std::vector<Block> blocks;
    long long total_samples = 0;
    double* d_w = nullptr;      // per-pair weights of the moment kernel
    int wcap = 0;
};

namespace bloch {

// Versions of learned-preconditioner parameters, unique within the process,
// so cached Z tables are never matched to another network's parameters.
static unsigned long long next_lp_version() {
    static std::atomic<unsigned long long> counter{0};
    return ++counter;
}

static unsigned long long lp_hash(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

// ---------------------------------------------------------------- kernels
// seeded right-hand sides, weighted toward long wavelengths:
// b(q) = (u + i v) / (1 + |q|^2 / 16) with u, v uniform in [-1, 1)
template <typename T>
__global__ void k_lp_rhs(cplx_t<T>* b, const T* __restrict__ qtab, Geo g, unsigned long long seed) {
    const int sys = blockIdx.y;
    const T* qb = qtab + (size_t)sys * (g.Nx + g.Ny + g.Nz);
    cplx_t<T>* bb = b + (size_t)sys * 3 * g.V;
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
        T qx, qy, qz;
        voxel_q(qb, g, v, qx, qy, qz);
        const T w = T(1) / (T(1) + (qx * qx + qy * qy + qz * qz) / T(16));
        const bool zero = qx == T(0) && qy == T(0) && qz == T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const unsigned long long idx = ((unsigned long long)sys * 3 + c) * (unsigned long long)g.V + v;
            const T re = T(hash_u32(seed * 0x9E3779B97F4A7C15ULL + 2 * idx) * (1.0 / 2147483648.0) - 1.0);
            const T im = T(hash_u32(seed * 0x9E3779B97F4A7C15ULL + 2 * idx + 1) * (1.0 / 2147483648.0) - 1.0);
            bb[(size_t)c * g.V + v] = zero ? mk(T(0), T(0)) : mk(re * w, im * w);
        }
    }
}

// Per-pair weights of the moments: 1/||r_j||^2, or 0 for a pair that is not
// recorded.  From the CG scalars: pairs are recorded while ||r_j|| > 1e-4 ||b||
// (below that the error e_j is dominated by the 1e-6 accuracy of x* itself).
__global__ void k_lp_weights_cg(const CGSys* __restrict__ sys, int nsys, double* __restrict__ w) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsys) w[s] = (sys[s].rr > 1e-8 * sys[s].bb) ? 1.0 / sys[s].rr : 0.0;
}

// From the inner products (r_j, r_j) of caller-supplied pairs (0 for r_j = 0).
__global__ void k_lp_weights_dot(const double2* __restrict__ rr, int n, double* __restrict__ w) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) w[s] = rr[s].x > 0.0 ? 1.0 / rr[s].x : 0.0;
}

// mom[v] += sum over pairs of w_j times the moments of (r_j, e_j) at voxel v:
// A = Re r r^H, B = sym Re r e^H (xx yy zz yz xz xy), c = |e|^2, where
// e_j = xs_j - x_j (CG iterates against the converged solution) or, with
// xs == nullptr, e_j = x_j (errors given directly).
__global__ void k_lp_moments(const float2* __restrict__ r, const float2* __restrict__ x,
                             const float2* __restrict__ xs, const double* __restrict__ w, int nsys, long long V,
                             float* __restrict__ mom) {
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)V; v += gridDim.x * blockDim.x) {
        float acc[kMom];
#pragma unroll
        for (int i = 0; i < kMom; ++i) acc[i] = 0.f;
        for (int s = 0; s < nsys; ++s) {
            const float sc = (float)w[s];
            if (sc == 0.f) continue;
            float2 rv[3], ev[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t i = ((size_t)s * 3 + c) * V + v;
                rv[c] = r[i];
                const float2 b = x[i];
                if (xs) {
                    const float2 a = xs[i];
                    ev[c] = make_float2(a.x - b.x, a.y - b.y);
                } else {
                    ev[c] = b;
                }
            }
            const int ii[6] = {0, 1, 2, 1, 0, 0}, jj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                const float2 a = rv[ii[t]], b = rv[jj[t]];
                acc[t] += sc * (a.x * b.x + a.y * b.y);
                // sym Re(r e^H): (Re r_i conj(e_j) + Re r_j conj(e_i)) / 2
                const float2 ei = ev[ii[t]], ej = ev[jj[t]];
                acc[6 + t] += sc * 0.5f * ((a.x * ej.x + a.y * ej.y) + (b.x * ei.x + b.y * ei.y));
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[12] += sc * (ev[c].x * ev[c].x + ev[c].y * ev[c].y);
        }
#pragma unroll
        for (int i = 0; i < kMom; ++i) mom[(size_t)v * kMom + i] += acc[i];
    }
}

// Loss and gradient over one data block.  Each thread evaluates one Fourier
// voxel (three branches) forward and backward to the pre-activations; the
// weight gradients are then formed from the per-sample vectors staged in
// shared memory, each thread owning a few parameters.
constexpr int kLPT = 128;          // threads (voxels) per tile
constexpr int kLPS = 3 * kLPT;     // samples per tile
__global__ void __launch_bounds__(kLPT) k_lp_grad(const float* __restrict__ prm_g, const float* __restrict__ mom,
                                                  const float* __restrict__ qt, Geo g, PrecondCoef pc, float snorm,
                                                  double wscale, double* __restrict__ grad) {
    constexpr int H = kLPH;
    extern __shared__ __align__(16) float lsm[];
    float* prm = lsm;                       // kLPN
    float* sf = prm + ((kLPN + 3) & ~3);    // kLPS x 5
    float* sh1 = sf + kLPS * kLPF;          // kLPS x H
    float* sh2 = sh1 + kLPS * H;
    float* sd1 = sh2 + kLPS * H;
    float* sd2 = sd1 + kLPS * H;
    float* sdo = sd2 + kLPS * H;            // kLPS
    const int tid = threadIdx.x;
    for (int i = tid; i < kLPN; i += kLPT) prm[i] = prm_g[i];
    constexpr int PER = (kLPN + kLPT - 1) / kLPT;
    double pacc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) pacc[k] = 0.0;
    double lacc = 0.0;
    const float* W2 = prm + H * kLPF + H;
    const float* w3 = W2 + H * H + H;
    __syncthreads();
    const long long ntiles = (g.V + kLPT - 1) / kLPT;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long v = tile * kLPT + tid;
        bool valid = v < g.V;
        float qx = 0, qy = 0, qz = 0;
        if (valid) {
            const unsigned nx = (unsigned)g.Nx, ny = (unsigned)g.Ny;
            const unsigned t = (unsigned)v / nx;
            const unsigned z = t / ny;
            qx = qt[(unsigned)v - t * nx];
            qy = qt[g.Nx + (t - z * ny)];
            qz = qt[g.Nx + g.Ny + z];
        }
        const float qn2 = qx * qx + qy * qy + qz * qz;
        if (qn2 == 0.f) valid = false;
        float P[3][3], mu[3], Vv[3][3];
        float o[3], gg[3];
        if (valid) {
            acoustic3<float>(pc, qx, qy, qz, P);
            sym3_eig<float>(P, mu, Vv);
            const float iq = 1.f / qn2;
            const float s = log1pf(sqrtf(qn2)) * snorm;
            // forward, one branch at a time (activations staged in shared memory)
#pragma unroll 1
            for (int a = 0; a < 3; ++a) {
        asm volatile("" ::: "memory");   // keep the weight loads inside the branch loop
                const int si = a * kLPT + tid;
                const float mua = a == 0 ? mu[0] : (a == 1 ? mu[1] : mu[2]);
                float f[kLPF] = {qx * qx * iq, qy * qy * iq, qz * qz * iq, mua * iq, s};
                float h1[H], h2[H];
                const float oa = lp_forward<H>(prm, f, h1, h2);
                if (a == 0) o[0] = oa; else if (a == 1) o[1] = oa; else o[2] = oa;
#pragma unroll
                for (int j = 0; j < kLPF; ++j) sf[si * kLPF + j] = f[j];
#pragma unroll
                for (int j = 0; j < H; ++j) {
                    sh1[si * H + j] = h1[j];
                    sh2[si * H + j] = h2[j];
                }
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) gg[a] = lp_softplus(o[a]);
            // Z, loss, dL/dZ = Z A + A Z - 2 B
            const float* m = mom + (size_t)v * kMom;
            float A[3][3], Bm[3][3], Z[3][3];
            const int ii[6] = {0, 1, 2, 1, 0, 0}, jj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                A[ii[t]][jj[t]] = A[jj[t]][ii[t]] = m[t];
                Bm[ii[t]][jj[t]] = Bm[jj[t]][ii[t]] = m[6 + t];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float z = 0.f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) z = fmaf(gg[a] / mu[a] * Vv[i][a], Vv[j][a], z);
                    Z[i][j] = z;
                }
            float ZA[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float s2 = 0.f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) s2 = fmaf(Z[i][k], A[k][j], s2);
                    ZA[i][j] = s2;
                }
            float L = m[12];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) L += ZA[i][j] * Z[j][i] - 2.f * Z[i][j] * Bm[j][i];
            lacc += (double)L;
            float dout[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float vGv = 0.f;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        vGv = fmaf(Vv[i][a] * (ZA[i][j] + ZA[j][i] - 2.f * Bm[i][j]), Vv[j][a], vGv);
                dout[a] = vGv / mu[a] * lp_sigmoid(o[a]);
            }
            // backward through the hidden layers, one branch at a time
#pragma unroll 1
            for (int a = 0; a < 3; ++a) {
                asm volatile("" ::: "memory");   // keep the weight loads inside the branch loop
                const int si = a * kLPT + tid;
                const float da = a == 0 ? dout[0] : (a == 1 ? dout[1] : dout[2]);
                sdo[si] = da;
                float d2[H];
#pragma unroll
                for (int i = 0; i < H; ++i) {
                    const float h = sh2[si * H + i];
                    d2[i] = da * w3[i] * (1.f - h * h);
                    sd2[si * H + i] = d2[i];
                }
#pragma unroll
                for (int j = 0; j < H; ++j) {
                    float s3 = 0.f;
#pragma unroll
                    for (int i = 0; i < H; ++i) s3 = fmaf(W2[i * H + j], d2[i], s3);
                    const float h = sh1[si * H + j];
                    sd1[si * H + j] = s3 * (1.f - h * h);
                }
            }
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int si = a * kLPT + tid;
                sdo[si] = 0.f;
#pragma unroll
                for (int j = 0; j < kLPF; ++j) sf[si * kLPF + j] = 0.f;
#pragma unroll
                for (int j = 0; j < H; ++j) sh1[si * H + j] = sh2[si * H + j] = sd1[si * H + j] = sd2[si * H + j] = 0.f;
            }
        }
        __syncthreads();
        // parameter gradients over the tile's samples
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int p = tid + k * kLPT;
            if (p >= kLPN) continue;
            float acc = 0.f;
            if (p < H * kLPF) {                                   // W1[i][j]
                const int i = p / kLPF, j = p % kLPF;
                for (int s2 = 0; s2 < kLPS; ++s2) acc = fmaf(sd1[s2 * H + i], sf[s2 * kLPF + j], acc);
            } else if (p < H * kLPF + H) {                        // b1[i]
                const int i = p - H * kLPF;
                for (int s2 = 0; s2 < kLPS; ++s2) acc += sd1[s2 * H + i];
            } else if (p < H * kLPF + H + H * H) {                // W2[i][j]
                const int q2 = p - H * kLPF - H, i = q2 / H, j = q2 % H;
                for (int s2 = 0; s2 < kLPS; ++s2) acc = fmaf(sd2[s2 * H + i], sh1[s2 * H + j], acc);
            } else if (p < H * kLPF + 2 * H + H * H) {            // b2[i]
                const int i = p - H * kLPF - H - H * H;
                for (int s2 = 0; s2 < kLPS; ++s2) acc += sd2[s2 * H + i];
            } else if (p < kLPN - 1) {                            // w3[j]
                const int j = p - (H * kLPF + 2 * H + H * H);
                for (int s2 = 0; s2 < kLPS; ++s2) acc = fmaf(sdo[s2], sh2[s2 * H + j], acc);
            } else {                                              // b3
                for (int s2 = 0; s2 < kLPS; ++s2) acc += sdo[s2];
            }
            pacc[k] += (double)acc;
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int p = tid + k * kLPT;
        if (p < kLPN) atomicAdd(&grad[p], pacc[k] * wscale);
    }
    double l1[1] = {lacc};
    block_sum<double, 1>(l1);
    if (tid == 0) atomicAdd(&grad[kLPN], l1[0] * wscale);
}

__global__ void k_lp_adam(float* prm, float* m, float* v, const double* __restrict__ grad, int n, float lr,
                          float b1c, float b2c) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float gr = (float)grad[i];
        m[i] = b1 * m[i] + (1.f - b1) * gr;
        v[i] = b2 * v[i] + (1.f - b2) * gr * gr;
        prm[i] -= lr * (m[i] / b1c) / (sqrtf(v[i] / b2c) + eps);
    }
}

// Z tables for ntab wave vectors: ztab[t][v][6]
template <typename TQ>
__global__ void k_lp_table(const float* __restrict__ prm_g, const TQ* __restrict__ qtab, int qstride_sys,
                           Geo g, PrecondCoef pc, float snorm, float* __restrict__ ztab) {
    __shared__ float prm[kLPN];
    for (int i = threadIdx.x; i < kLPN; i += blockDim.x) prm[i] = prm_g[i];
    __syncthreads();
    const int t = blockIdx.y;
    const TQ* qb = qtab + (size_t)t * qstride_sys * (g.Nx + g.Ny + g.Nz);
    float* zt = ztab + (size_t)t * g.V * 6;
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
        TQ qx, qy, qz;
        voxel_q(qb, g, v, qx, qy, qz);
        float Z[6];
        lp_Z<kLPH>(prm, pc, snorm, (float)qx, (float)qy, (float)qz, Z);
#pragma unroll
        for (int i = 0; i < 6; ++i) zt[(size_t)v * 6 + i] = Z[i];
    }
}

static float lp_snorm(const bloch_plan* pl) {
    const int Nmax = std::max(pl->Nx, std::max(pl->Ny, pl->Nz));
    return (float)(1.0 / std::log1p(Nmax / 2.0));
}

// Build the Z tables of ntab groups of systems whose q tables are set (the
// q table of group t is that of system t * qstride_sys) and activate them.
template <typename T>
bloch_status lp_activate(bloch_plan* pl, int ntab, int qstride_sys, int zgroup) {
    if (!pl->lp) {
        pl->psel = PrecondSel{nullptr, 1};
        return BLOCH_OK;
    }
    const size_t need = (size_t)ntab * pl->V * 6;
    if (need > pl->zcap) {
        pl->zkey.clear();
        cudaFree(pl->d_ztab);
        pl->d_ztab = nullptr;
        pl->zcap = 0;
        cudaError_t e = cudaMalloc((void**)&pl->d_ztab, need * sizeof(float));
        if (e != cudaSuccess) return set_cuda_error(e, "cudaMalloc (learned preconditioner tables)");
        pl->zcap = need;
    }
    // the tables depend on the network, the precision and the wave vector of
    // every qstride_sys-th system: rebuild only when one of them changed
    std::vector<double> key;
    key.reserve((size_t)3 * ntab + 4);
    key.push_back((double)sizeof(T));
    key.push_back((double)ntab);
    key.push_back((double)pl->lp->version);
    for (int t = 0; t < ntab; ++t)
        for (int a = 0; a < 3; ++a) key.push_back(pl->k_host[(size_t)t * qstride_sys * 3 + a]);
    if (key != pl->zkey) {
        dim3 gr((unsigned)std::min<long long>((pl->V + 255) / 256, 1024), ntab);
        ++pl->launches;
        k_lp_table<T><<<gr, 256, 0, pl->stream>>>(pl->lp->d_prm, ws_of<T>(pl).qtab, qstride_sys, geo_of<T>(pl),
                                                  pl->pc, lp_snorm(pl), pl->d_ztab);
        BLOCH_CUDA_CHECK_RET(cudaGetLastError());
        pl->zkey = key;
    }
    pl->psel = PrecondSel{pl->d_ztab, zgroup};
    return BLOCH_OK;
}

template bloch_status lp_activate<float>(bloch_plan*, int, int, int);
template bloch_status lp_activate<double>(bloch_plan*, int, int, int);

void lp_deactivate(bloch_plan* pl) { pl->psel = PrecondSel{nullptr, 1}; }

static bloch_status lp_weights_cap(bloch_lp* lp, int n) {
    if (n <= lp->wcap) return BLOCH_OK;
    cudaDeviceSynchronize();
    cudaFree(lp->d_w);
    lp->d_w = nullptr;
    lp->wcap = 0;
    cudaError_t e = cudaMalloc((void**)&lp->d_w, (size_t)n * sizeof(double));
    if (e != cudaSuccess) return set_cuda_error(e, "cudaMalloc (pair weights)");
    lp->wcap = n;
    return BLOCH_OK;
}

struct MomHook {
    bloch_plan* pl;
    const float2* x;
    const float2* xs;
    float* mom;
    double* w;
    int nsys;
    int n_iters;
    int recorded = 0;
};

static void mom_hook(void* ctx, int it) {
    MomHook* h = (MomHook*)ctx;
    if (it >= h->n_iters) return;
    h->pl->launches += 2;
    k_lp_weights_cg<<<(h->nsys + 127) / 128, 128, 0, h->pl->stream>>>(h->pl->ws_f.sys, h->nsys, h->w);
    k_lp_moments<<<(unsigned)std::min<long long>((h->pl->V + 255) / 256, 2048), 256, 0, h->pl->stream>>>(
        h->pl->ws_f.r, h->x, h->xs, h->w, h->nsys, h->pl->V, h->mom);
    h->recorded += h->nsys;
}

// New empty data block for the plan's grid whose q table is that of the
// plan's system 0 (set_k must have run).
static bloch_status lp_new_block(bloch_plan* pl, bloch_lp::Block& blk) {
    blk.grid[0] = pl->Nx;
    blk.grid[1] = pl->Ny;
    blk.grid[2] = pl->Nz;
    blk.V = pl->V;
    blk.pc = pl->pc;
    for (int i = 0; i < 36; ++i) blk.C0V[i] = pl->C0V[i] / pl->Cref;
    blk.snorm = lp_snorm(pl);
    blk.samples = 0;
    blk.d_mom = nullptr;
    blk.d_q = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc((void**)&blk.d_mom, (size_t)pl->V * kMom * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc((void**)&blk.d_q, (size_t)(pl->Nx + pl->Ny + pl->Nz) * sizeof(float))) != cudaSuccess) {
        cudaFree(blk.d_mom);
        return set_cuda_error(e, "cudaMalloc (data block)");
    }
    BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(blk.d_mom, 0, (size_t)pl->V * kMom * sizeof(float), pl->stream));
    BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(blk.d_q, pl->ws_f.qtab, (size_t)(pl->Nx + pl->Ny + pl->Nz) * sizeof(float),
                                         cudaMemcpyDeviceToDevice, pl->stream));
    return BLOCH_OK;
}

}  // namespace bloch

using namespace bloch;

extern "C" {

int32_t bloch_lp_num_params(void) { return kLPN; }

bloch_status bloch_lp_create(bloch_lp** out, uint64_t seed) {
    if (!out) return set_error(BLOCH_EINVAL, "out is NULL");
    *out = nullptr;
    bloch_lp* lp = new bloch_lp();
    lp->version = next_lp_version();
    std::vector<float> h(kLPN, 0.f);
    const int nh = kLPH * kLPF + kLPH + kLPH * kLPH + kLPH;
    for (int i = 0; i < nh; ++i) {
        unsigned long long x = (unsigned long long)i * 0x9E3779B97F4A7C15ULL + seed;
        x = lp_hash(x);
        const double u = (double)(x >> 40) / (double)(1ULL << 24);
        h[i] = (float)((2.0 * u - 1.0) * 0.5);
    }
    h[kLPN - 1] = (float)std::log(std::exp(1.0) - 1.0);   // softplus(b3) = 1
    cudaError_t e;
    if ((e = cudaMalloc((void**)&lp->d_prm, kLPN * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc((void**)&lp->d_m, kLPN * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc((void**)&lp->d_v, kLPN * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc((void**)&lp->d_grad, (kLPN + 1) * sizeof(double))) != cudaSuccess) {
        bloch_lp_destroy(lp);
        return set_cuda_error(e, "cudaMalloc (learned preconditioner)");
    }
    cudaMemcpy(lp->d_prm, h.data(), kLPN * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(lp->d_m, 0, kLPN * sizeof(float));
    cudaMemset(lp->d_v, 0, kLPN * sizeof(float));
    *out = lp;
    return BLOCH_OK;
}

void bloch_lp_destroy(bloch_lp* lp) {
    if (!lp) return;
    cudaDeviceSynchronize();
    cudaFree(lp->d_w);
    cudaFree(lp->d_prm);
    cudaFree(lp->d_m);
    cudaFree(lp->d_v);
    cudaFree(lp->d_grad);
    for (auto& b : lp->blocks) {
        cudaFree(b.d_mom);
        cudaFree(b.d_q);
    }
    delete lp;
}

bloch_status bloch_lp_params(bloch_lp* lp, double* get, const double* set) {
    if (!lp) return set_error(BLOCH_EINVAL, "lp is NULL");
    std::vector<float> h(kLPN);
    if (set) {
        for (int i = 0; i < kLPN; ++i) h[i] = (float)set[i];
        BLOCH_CUDA_CHECK_RET(cudaMemcpy(lp->d_prm, h.data(), kLPN * sizeof(float), cudaMemcpyHostToDevice));
        lp->version = bloch::next_lp_version();
    }
    if (get) {
        BLOCH_CUDA_CHECK_RET(cudaMemcpy(h.data(), lp->d_prm, kLPN * sizeof(float), cudaMemcpyDeviceToHost));
        for (int i = 0; i < kLPN; ++i) get[i] = h[i];
    }
    return BLOCH_OK;
}

bloch_status bloch_lp_collect(bloch_lp* lp, bloch_plan* pl, int32_t n_k, const double* k_list, int32_t n_rhs,
                              int32_t n_iters, uint64_t seed) {
    if (!lp || !pl || !k_list) return set_error(BLOCH_EINVAL, "NULL argument");
    if (n_k < 1 || n_rhs < 1 || n_iters < 1) return set_error(BLOCH_EINVAL, "n_k, n_rhs, n_iters must be >= 1");
    const bloch_lp* saved = pl->lp;
    pl->lp = nullptr;   // data come from the paper's Green preconditioner
    lp_deactivate(pl);
    bloch_status st = BLOCH_OK;
    float2 *b = nullptr, *xs = nullptr, *x = nullptr;
    const size_t n = (size_t)n_rhs * 3 * pl->V;
    cudaError_t e;
    if ((e = cudaMalloc((void**)&b, n * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc((void**)&xs, n * sizeof(float2))) != cudaSuccess ||
        (e = cudaMalloc((void**)&x, n * sizeof(float2))) != cudaSuccess) {
        cudaFree(b);
        cudaFree(xs);
        pl->lp = saved;
        return set_cuda_error(e, "cudaMalloc (collection buffers)");
    }
    for (int ik = 0; ik < n_k && st == BLOCH_OK; ++ik) {
        std::vector<double> kv((size_t)n_rhs * 3);
        for (int s = 0; s < n_rhs; ++s)
            for (int a = 0; a < 3; ++a) kv[(size_t)s * 3 + a] = k_list[3 * ik + a];
        if ((st = set_k<float>(pl, n_rhs, kv.data())) != BLOCH_OK) break;
        dim3 gr((unsigned)std::min<long long>((pl->V + 255) / 256, 1024), n_rhs);
        ++pl->launches;
        k_lp_rhs<float><<<gr, 256, 0, pl->stream>>>(b, pl->ws_f.qtab, pl->geo_f,
                                                    seed + 7919ULL * (unsigned long long)ik);
        st = pcg_run<float>(pl, n_rhs, b, xs, 1.0, 1e-6, 3000, false, nullptr, nullptr, nullptr);
        if (st == BLOCH_ENOTCONV_CG) st = BLOCH_OK;
        if (st != BLOCH_OK) break;
        bloch_lp::Block blk;
        if ((st = lp_new_block(pl, blk)) != BLOCH_OK) break;
        if ((st = lp_weights_cap(lp, n_rhs)) != BLOCH_OK) {
            cudaFree(blk.d_mom);
            cudaFree(blk.d_q);
            break;
        }
        MomHook h{pl, x, xs, blk.d_mom, lp->d_w, n_rhs, n_iters + 1};
        st = pcg_run<float>(pl, n_rhs, b, x, 1.0, 1e-30, n_iters, false, nullptr, nullptr, nullptr, mom_hook, &h);
        if (st == BLOCH_ENOTCONV_CG) st = BLOCH_OK;
        cudaStreamSynchronize(pl->stream);
        blk.samples = h.recorded;
        lp->total_samples += h.recorded;
        lp->blocks.push_back(blk);
    }
    cudaStreamSynchronize(pl->stream);
    cudaFree(b);
    cudaFree(xs);
    cudaFree(x);
    pl->lp = saved;
    return st;
}

bloch_status bloch_lp_add_pairs(bloch_lp* lp, bloch_plan* pl, const double* k, int32_t n_pairs, const void* r,
                                const void* e) {
    if (!lp || !pl || !k || !r || !e) return set_error(BLOCH_EINVAL, "NULL argument");
    if (n_pairs < 1 || n_pairs > 65535 / 6) return set_error(BLOCH_EINVAL, "n_pairs must be in [1, 10922]");
    bloch_status st;
    // grow the workspace first: growing reallocates the q tables set_k fills
    if ((st = ensure_cg<float>(pl, n_pairs)) != BLOCH_OK) return st;
    if ((st = set_k<float>(pl, 1, k)) != BLOCH_OK) return st;
    if ((st = lp_weights_cap(lp, n_pairs)) != BLOCH_OK) return st;
    const float2* rr = (const float2*)r;
    const float2* ee = (const float2*)e;
    launch_dot<float>(pl, n_pairs, rr, rr, 3 * pl->V, pl->ws_f.dots, pl->ws_f.part2);
    ++pl->launches;
    k_lp_weights_dot<<<(n_pairs + 127) / 128, 128, 0, pl->stream>>>(pl->ws_f.dots, n_pairs, lp->d_w);
    bloch_lp::Block blk;
    if ((st = lp_new_block(pl, blk)) != BLOCH_OK) return st;
    ++pl->launches;
    k_lp_moments<<<(unsigned)std::min<long long>((pl->V + 255) / 256, 2048), 256, 0, pl->stream>>>(
        rr, ee, nullptr, lp->d_w, n_pairs, pl->V, blk.d_mom);
    std::vector<double> w(n_pairs);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(w.data(), lp->d_w, sizeof(double) * n_pairs, cudaMemcpyDeviceToHost, pl->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(pl->stream);
    if (ce != cudaSuccess) {
        cudaFree(blk.d_mom);
        cudaFree(blk.d_q);
        return set_cuda_error(ce, "bloch_lp_add_pairs");
    }
    for (double wi : w) blk.samples += wi > 0.0 ? 1 : 0;
    lp->total_samples += blk.samples;
    lp->blocks.push_back(blk);
    return BLOCH_OK;
}

bloch_status bloch_lp_loss_grad(bloch_lp* lp, double* loss, double* grad) {
    if (!lp) return set_error(BLOCH_EINVAL, "lp is NULL");
    if (lp->blocks.empty()) return set_error(BLOCH_EINVAL, "no training data collected");
    BLOCH_CUDA_CHECK_RET(cudaMemset(lp->d_grad, 0, (kLPN + 1) * sizeof(double)));
    const double ws = 1.0 / (double)std::max<long long>(1, lp->total_samples);
    constexpr int H = kLPH;
    const size_t smem = (size_t)(((kLPN + 3) & ~3) + kLPS * kLPF + 4 * kLPS * H + kLPS) * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_lp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    for (auto& b : lp->blocks) {
        Geo g{};
        g.Nx = b.grid[0];
        g.Ny = b.grid[1];
        g.Nz = b.grid[2];
        g.V = b.V;
        g.dx = make_fastdiv((unsigned)g.Nx);
        g.dy = make_fastdiv((unsigned)g.Ny);
        const int nblk = (int)std::min<long long>((b.V + kLPT - 1) / kLPT, 608);
        k_lp_grad<<<nblk, kLPT, smem>>>(lp->d_prm, b.d_mom, b.d_q, g, b.pc, b.snorm, ws, lp->d_grad);
    }
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    std::vector<double> h(kLPN + 1);
    BLOCH_CUDA_CHECK_RET(cudaMemcpy(h.data(), lp->d_grad, (kLPN + 1) * sizeof(double), cudaMemcpyDeviceToHost));
    if (loss) *loss = h[kLPN];
    if (grad)
        for (int i = 0; i < kLPN; ++i) grad[i] = h[i];
    return BLOCH_OK;
}

bloch_status bloch_lp_train(bloch_lp* lp, int32_t steps, double lr, double* loss_out) {
    if (!lp) return set_error(BLOCH_EINVAL, "lp is NULL");
    if (steps < 0 || !(lr > 0)) return set_error(BLOCH_EINVAL, "steps >= 0 and lr > 0 required");
    for (int s = 0; s < steps; ++s) {
        double L = 0;
        bloch_status st = bloch_lp_loss_grad(lp, &L, nullptr);
        if (st != BLOCH_OK) return st;
        if (loss_out) loss_out[s] = L;
        lp->adam_t += 1;
        const float b1c = 1.f - std::pow(0.9f, (float)lp->adam_t);
        const float b2c = 1.f - std::pow(0.999f, (float)lp->adam_t);
        k_lp_adam<<<1, 512>>>(lp->d_prm, lp->d_m, lp->d_v, lp->d_grad, kLPN, (float)lr, b1c, b2c);
        BLOCH_CUDA_CHECK_RET(cudaGetLastError());
        lp->version = bloch::next_lp_version();
    }
    BLOCH_CUDA_CHECK_RET(cudaDeviceSynchronize());
    return BLOCH_OK;
}

int32_t bloch_lp_num_blocks(const bloch_lp* lp) { return lp ? (int32_t)lp->blocks.size() : 0; }

bloch_status bloch_lp_export_block(const bloch_lp* lp, int32_t block, int32_t grid[3], double* q, double* mom,
                                   double* C0V, int32_t* samples) {
    if (!lp || block < 0 || block >= (int)lp->blocks.size()) return set_error(BLOCH_EINVAL, "bad block index");
    const auto& b = lp->blocks[block];
    if (grid)
        for (int a = 0; a < 3; ++a) grid[a] = b.grid[a];
    if (C0V)
        for (int i = 0; i < 36; ++i) C0V[i] = b.C0V[i];
    if (samples) *samples = b.samples;
    if (q) {
        const int S = b.grid[0] + b.grid[1] + b.grid[2];
        std::vector<float> h(S);
        BLOCH_CUDA_CHECK_RET(cudaMemcpy(h.data(), b.d_q, S * sizeof(float), cudaMemcpyDeviceToHost));
        for (int i = 0; i < S; ++i) q[i] = h[i];
    }
    if (mom) {
        std::vector<float> h((size_t)b.V * kMom);
        BLOCH_CUDA_CHECK_RET(cudaMemcpy(h.data(), b.d_mom, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < h.size(); ++i) mom[i] = h[i];
    }
    return BLOCH_OK;
}

bloch_status bloch_plan_set_preconditioner(bloch_plan* pl, const bloch_lp* lp) {
    if (!pl) return set_error(BLOCH_EINVAL, "plan is NULL");
    pl->lp = lp;
    lp_deactivate(pl);
    return BLOCH_OK;
}

}  // extern "C"
