// Eigensolvers and the dispersion driver (Section 3.3, Algorithms 1 and 3).
//
// Subspace iteration (Algorithm 1) advances a batch of wave vectors ("slots")
// together, each slot holding its own block of q vectors [slot][q][3][V].
// One sweep, for every active slot:
//   KU = A_k U, lam_p = Rayleigh quotient of u_p, R = M U - KU diag(1/lam)
//   err1 (relative change of lam), err2 = max_p lam_p |R_p| / |KU_p|
//   delta = A_k^-1 R by PCG (Algorithm 2) on all slots x q systems at once
//   U_bar = U diag(1/lam) + delta          (= A_k^-1 M U, the paper's step)
//   Kn = M U - r_cg (= A_k U_bar exactly up to the recursive CG residual)
//   K = U_bar^H Kn, M = U_bar^H M U_bar, (K, M) -> (lam, Q), U <- U_bar Q
// Writing the paper's inverse step as a correction of U diag(1/lam) keeps the
// PCG right-hand side small, so the field precision (FP32 in the chosen form)
// only limits the correction, and the residual R can be formed in FP64 from
// an FP64 operator apply (the refinement phase) while every other step stays
// in FP32.  Converged slots are refilled from the queue of wave vectors.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "eig_kernels.cuh"
#include "gram_tc.cuh"
#include "internal.h"

namespace bloch {

using cd = std::complex<double>;

bloch_status plan_solver_buf(bloch_plan* pl, int pool, int idx, size_t bytes, void** out) {
    auto& v = pl->solver_bufs[pool];
    if ((int)v.size() <= idx) v.resize(idx + 1);
    bloch_plan::SolverBuf& b = v[idx];
    bytes = std::max<size_t>(bytes, 256);
    if (b.bytes < bytes) {
        cudaStreamSynchronize(pl->stream);   // an earlier solve may still use the old buffer
        if (b.p) {
            cudaFree(b.p);
            pl->device_bytes -= b.bytes;
        }
        b.p = nullptr;
        b.bytes = 0;
        cudaError_t e = cudaMalloc(&b.p, bytes);
        if (e != cudaSuccess) {
            b.p = nullptr;
            return set_cuda_error(e, "cudaMalloc (eigensolver block)");
        }
        b.bytes = bytes;
        pl->device_bytes += bytes;
    }
    *out = b.p;
    return BLOCH_OK;
}

size_t plan_solver_bytes(const bloch_plan* pl, int pool) {
    size_t t = 0;
    for (const auto& b : pl->solver_bufs[pool]) t += b.bytes;
    return t;
}

void plan_solver_release(bloch_plan* pl) {
    for (auto& v : pl->solver_bufs) {
        for (auto& b : v) cudaFree(b.p);
        v.clear();
    }
    for (int i = 0; i < 2; ++i) {
        cudaFree(pl->d_rhohat[i]);
        pl->d_rhohat[i] = nullptr;
    }
}

template <typename T>
bloch_status gamma_rhohat(bloch_plan* pl, const cplx_t<T>** out) {
    using C = cplx_t<T>;
    const int pi = std::is_same<T, float>::value ? 1 : 0;
    if (!pl->d_rhohat[pi]) {
        bloch_status st = ensure_ws<T>(pl, 1);
        if (st != BLOCH_OK) return st;
        const size_t n3 = (size_t)3 * pl->V;
        C* tmp = nullptr;
        if ((st = plan_solver_buf(pl, 2, 3, 2 * n3 * sizeof(C), (void**)&tmp)) != BLOCH_OK) return st;
        BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(tmp, 0, n3 * sizeof(C), pl->stream));
        const C one = mk(T(1), T(0));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(tmp, &one, sizeof(C), cudaMemcpyHostToDevice, pl->stream));
        launch_M<T>(pl, 1, tmp, tmp + n3, T(1));
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, (size_t)pl->V * sizeof(C));
        if (e != cudaSuccess) return set_cuda_error(e, "cudaMalloc (Gamma deflation table)");
        pl->device_bytes += (size_t)pl->V * sizeof(C);
        BLOCH_CUDA_CHECK_RET(
            cudaMemcpyAsync(p, tmp + n3, (size_t)pl->V * sizeof(C), cudaMemcpyDeviceToDevice, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));   // `one` leaves scope
        pl->d_rhohat[pi] = p;
    }
    *out = (const C*)pl->d_rhohat[pi];
    return BLOCH_OK;
}

template <typename T>
bloch_status gamma_deflate(bloch_plan* pl, int nv, cplx_t<T>* Vv, cplx_t<T>* MV, double2* d_alpha) {
    const cplx_t<T>* rh = nullptr;
    bloch_status st = gamma_rhohat<T>(pl, &rh);
    if (st != BLOCH_OK) return st;
    const long long n3 = 3 * pl->V;
    pl->launches += 2;
    k_gamma_alpha<T><<<(3 * nv + 127) / 128, 128, 0, pl->stream>>>(MV, n3, pl->V, nv, rh, d_alpha);
    const unsigned gx = (unsigned)std::min<long long>((pl->V + 255) / 256, 1024);
    k_gamma_deflate<T><<<dim3(gx, nv), 256, 0, pl->stream>>>(Vv, MV, rh, n3, pl->V, d_alpha);
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    return BLOCH_OK;
}

template bloch_status gamma_rhohat<float>(bloch_plan*, const float2**);
template bloch_status gamma_rhohat<double>(bloch_plan*, const double2**);
template bloch_status gamma_deflate<float>(bloch_plan*, int, float2*, float2*, double2*);
template bloch_status gamma_deflate<double>(bloch_plan*, int, double2*, double2*, double2*);

// ====================================================================
// Small dense Hermitian eigenproblems (host, FP64)
// ====================================================================

// Cyclic complex Jacobi.  A (n x n, row-major, Hermitian) is destroyed.
// w ascending; V row-major with eigenvectors in columns.
static bool herm_jacobi(int n, std::vector<cd>& A, std::vector<double>& w, std::vector<cd>& V) {
    V.assign((size_t)n * n, cd(0, 0));
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    bool ok = false;
    for (int sweep = 0; sweep < 200; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double a2 = std::norm(A[(size_t)i * n + j]);
                tot += a2;
                if (i != j) off += a2;
            }
        if (off <= 1e-32 * tot || tot == 0.0) {
            ok = true;
            break;
        }
        for (int p = 0; p < n - 1; ++p)
            for (int r = p + 1; r < n; ++r) {
                const cd apr = A[(size_t)p * n + r];
                const double mag = std::abs(apr);
                if (mag == 0.0) continue;
                const double app = A[(size_t)p * n + p].real(), arr = A[(size_t)r * n + r].real();
                if (mag < 1e-300 || mag <= 1e-18 * std::sqrt(std::fabs(app * arr)) * 1e-3) {
                    A[(size_t)p * n + r] = A[(size_t)r * n + p] = 0.0;
                    continue;
                }
                const cd e = apr / mag;  // exp(i phi)
                const double tau = (arr - app) / (2.0 * mag);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                const cd em = std::conj(e);
                // W: W_pp = c, W_pr = s, W_rp = -s e^{-i phi}, W_rr = c e^{-i phi}
                const cd Wpp = c, Wpr = s, Wrp = -s * em, Wrr = c * em;
                for (int i = 0; i < n; ++i) {  // A <- A W
                    const cd aip = A[(size_t)i * n + p], air = A[(size_t)i * n + r];
                    A[(size_t)i * n + p] = aip * Wpp + air * Wrp;
                    A[(size_t)i * n + r] = aip * Wpr + air * Wrr;
                }
                for (int j = 0; j < n; ++j) {  // A <- W^H A
                    const cd apj = A[(size_t)p * n + j], arj = A[(size_t)r * n + j];
                    A[(size_t)p * n + j] = std::conj(Wpp) * apj + std::conj(Wrp) * arj;
                    A[(size_t)r * n + j] = std::conj(Wpr) * apj + std::conj(Wrr) * arj;
                }
                for (int i = 0; i < n; ++i) {  // V <- V W
                    const cd vip = V[(size_t)i * n + p], vir = V[(size_t)i * n + r];
                    V[(size_t)i * n + p] = vip * Wpp + vir * Wrp;
                    V[(size_t)i * n + r] = vip * Wpr + vir * Wrr;
                }
                A[(size_t)p * n + r] = A[(size_t)r * n + p] = 0.0;
                A[(size_t)p * n + p] = A[(size_t)p * n + p].real();
                A[(size_t)r * n + r] = A[(size_t)r * n + r].real();
            }
    }
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](int a, int b) { return A[(size_t)a * n + a].real() < A[(size_t)b * n + b].real(); });
    std::vector<cd> Vs((size_t)n * n);
    w.resize(n);
    for (int j = 0; j < n; ++j) {
        w[j] = A[(size_t)ord[j] * n + ord[j]].real();
        for (int i = 0; i < n; ++i) Vs[(size_t)i * n + j] = V[(size_t)i * n + ord[j]];
    }
    V.swap(Vs);
    return ok;
}

// K Q = M Q diag(lam), Q^H M Q = I; K, M Hermitian (row-major), M positive definite.
// Returns 0 on success, 1 if M is not positive definite, 2 if Jacobi did not converge.
static int gen_herm_eig(int n, const cd* K, const cd* M, std::vector<double>& lam, std::vector<cd>& Q) {
    std::vector<cd> L((size_t)n * n, cd(0, 0));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            cd s = 0.5 * (M[(size_t)i * n + j] + std::conj(M[(size_t)j * n + i]));
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * std::conj(L[(size_t)j * n + k]);
            if (i == j) {
                if (!(s.real() > 0.0)) return 1;
                L[(size_t)i * n + i] = std::sqrt(s.real());
            } else {
                L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
            }
        }
    // X = L^-1 Kh (Kh = Hermitian part of K)
    std::vector<cd> X((size_t)n * n);
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) {
            cd s = 0.5 * (K[(size_t)i * n + c] + std::conj(K[(size_t)c * n + i]));
            for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * X[(size_t)k * n + c];
            X[(size_t)i * n + c] = s / L[(size_t)i * n + i];
        }
    // Cm = X L^-H = (L^-1 X^H)^H
    std::vector<cd> Y((size_t)n * n);
    for (int c = 0; c < n; ++c)
        for (int i = 0; i < n; ++i) {
            cd s = std::conj(X[(size_t)c * n + i]);
            for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * Y[(size_t)k * n + c];
            Y[(size_t)i * n + c] = s / L[(size_t)i * n + i];
        }
    std::vector<cd> Cm((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Cm[(size_t)i * n + j] = std::conj(Y[(size_t)j * n + i]);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) {
            const cd h = 0.5 * (Cm[(size_t)i * n + j] + std::conj(Cm[(size_t)j * n + i]));
            Cm[(size_t)i * n + j] = h;
            Cm[(size_t)j * n + i] = std::conj(h);
        }
    std::vector<cd> W;
    const bool ok = herm_jacobi(n, Cm, lam, W);
    // Q = L^-H W  (back substitution with L^H)
    Q.assign((size_t)n * n, cd(0, 0));
    for (int c = 0; c < n; ++c)
        for (int i = n - 1; i >= 0; --i) {
            cd s = W[(size_t)i * n + c];
            for (int k = i + 1; k < n; ++k) s -= std::conj(L[(size_t)k * n + i]) * Q[(size_t)k * n + c];
            Q[(size_t)i * n + c] = s / L[(size_t)i * n + i];
        }
    return ok ? 0 : 2;
}

// ====================================================================
// Start vectors (Section 3.3: "unit vectors corresponding to the lowest
// frequencies"): Fourier unit vectors at the bins of smallest |xi + k|,
// polarised along the eigenvectors of the reference acoustic tensor
// P0(xi + k), the q of lowest reference eigenvalue.
// ====================================================================
struct StartEntry {
    long long idx;  // element index comp*V + voxel
    double2 val;
};

static std::vector<StartEntry> start_vectors(const bloch_plan* pl, const double k[3], int q, bool gamma) {
    const int N[3] = {pl->Nx, pl->Ny, pl->Nz};
    int lo[3], hi[3];
    std::vector<int> mlist[3];
    for (int a = 0; a < 3; ++a) {
        const double kap = k[a] * pl->L[a] / (2.0 * M_PI);
        const int c = (int)std::lround(-kap);
        if (N[a] <= 13) {
            for (int m = 0; m < N[a]; ++m) mlist[a].push_back(m);
        } else {
            for (int d = -6; d <= 6; ++d) {
                const int mt = c + d;   // integer frequency
                const int half = (N[a] + 1) / 2;
                if (mt >= half || mt < half - N[a]) continue;
                mlist[a].push_back(mt >= 0 ? mt : mt + N[a]);
            }
        }
        (void)lo;
        (void)hi;
    }
    struct Cand {
        double q2;
        long long v;
        double qv[3];
    };
    std::vector<Cand> cands;
    const double* xi = pl->xi_host.data();
    for (int mz : mlist[2])
        for (int my : mlist[1])
            for (int mx : mlist[0]) {
                Cand c;
                c.qv[0] = xi[mx] + k[0];
                c.qv[1] = xi[pl->Nx + my] + k[1];
                c.qv[2] = xi[pl->Nx + pl->Ny + mz] + k[2];
                c.q2 = c.qv[0] * c.qv[0] + c.qv[1] * c.qv[1] + c.qv[2] * c.qv[2];
                c.v = ((long long)mz * pl->Ny + my) * pl->Nx + mx;
                if (gamma && c.q2 == 0.0) continue;
                cands.push_back(c);
            }
    std::sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) {
        return a.q2 < b.q2 || (a.q2 == b.q2 && a.v < b.v);
    });
    const size_t nc = std::min(cands.size(), (size_t)std::max(8 * q, 8));
    struct Item {
        double mu;
        long long v;
        int a;
        double w[3];
    };
    std::vector<Item> items;
    static const int vi[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    for (size_t c = 0; c < nc; ++c) {
        const double* qv = cands[c].qv;
        std::vector<cd> P(9);
        for (int i = 0; i < 3; ++i)
            for (int kk = 0; kk < 3; ++kk) {
                double s = 0;
                for (int j = 0; j < 3; ++j)
                    for (int l = 0; l < 3; ++l) s += pl->C0V[vi[i][j] * 6 + vi[kk][l]] * qv[j] * qv[l];
                P[i * 3 + kk] = s;
            }
        std::vector<double> w;
        std::vector<cd> Vv;
        herm_jacobi(3, P, w, Vv);
        for (int a = 0; a < 3; ++a) {
            Item it;
            it.mu = w[a];
            it.v = cands[c].v;
            it.a = a;
            for (int i = 0; i < 3; ++i) it.w[i] = Vv[i * 3 + a].real();
            items.push_back(it);
        }
    }
    std::sort(items.begin(), items.end(), [](const Item& x, const Item& y) {
        if (x.mu != y.mu) return x.mu < y.mu;
        if (x.v != y.v) return x.v < y.v;
        return x.a < y.a;
    });
    std::vector<StartEntry> out;
    const int nq = (int)std::min<size_t>(items.size(), (size_t)q);
    for (int p = 0; p < nq; ++p)
        for (int c = 0; c < 3; ++c) {
            StartEntry e;
            e.idx = (long long)p * 3 * pl->V + (long long)c * pl->V + items[p].v;
            e.val = make_double2(items[p].w[c], 0.0);
            out.push_back(e);
        }
    return out;
}

// ====================================================================
// Subspace iteration (Algorithm 1), batched over wave vectors
// ====================================================================
template <typename T>
struct Subspace {
    using C = cplx_t<T>;
    static constexpr int kEigThreads = 64;
    bloch_plan* pl;
    int n, q, B;
    long long n3;
    bool fp64res;     // FP32 fields with an FP64 residual refinement phase
    bool uniform;
    // LOBPCG (block method for a single wave vector; batched over wave
    // vectors like Algorithm 1): the block [X, W, P] is stored as three
    // segments of B*q vectors, X = U, W = T R (T = the Green operator), P the
    // previous search directions; A and M images alongside (KU, MU segments).
    bool lob = false;
    C *Wb = nullptr, *Pb = nullptr, *AWb = nullptr, *APb = nullptr, *MWb = nullptr, *MPb = nullptr;
    C *P2 = nullptr, *AP2 = nullptr, *MP2 = nullptr;
    double2* d_C3 = nullptr;
    double* d_lam3 = nullptr;
    size_t gsmem3 = 0;
    long long segs = 0;   // elements between the segments of the block
    double rho_s;
    double tol_eig, tol_lin;
    int max_outer, max_cg;
    const std::vector<std::array<double, 3>>* klist;
    double* omega_out;
    void* vecs_out;
    int n_bands;
    bloch_stats* st;
    bool any_unconverged = false;

    C *U = nullptr, *Ub = nullptr, *KU = nullptr, *R = nullptr, *MU = nullptr, *MUb = nullptr;
    double *d_part = nullptr, *d_scal = nullptr;
    double2 *d_gpart = nullptr, *d_G = nullptr, *d_Q = nullptr, *d_val = nullptr;
    long long* d_idx = nullptr;
    double2 *U64 = nullptr, *KU64 = nullptr, *MU64 = nullptr;
    double2* d_alpha = nullptr;   // Gamma-point deflation coefficients (non-uniform density)
    // per vector (slot * q + i): Rayleigh-quotient sums and |R|^2 (4 doubles),
    // 1/lambda, the projected problem's eigenvalues; per slot its status
    double *d_rq = nullptr, *d_invlam = nullptr, *d_lamq = nullptr;
    int* d_status = nullptr;
    long long* d_tally = nullptr;
    long long tally_host[4] = {0, 0, 0, 0};
    int eig_pending = 0;          // slots whose projected eigensolve status is read with the next residuals
    int gblk = 0, dblk = 0;
    size_t gsmem = 0;
    // tensor-core Gram (FP32 blocks, options.tensor_gram)
    bool use_tc = false;
    int gblk_tc = 0;
    size_t tcsmem = 0;
    int* d_gerr = nullptr;

    struct Slot {
        int kidx = -1;
        double k[3];
        bool gamma = false;
        int n_eff = 0;
        int sweeps = 0;
        int phase = 0;
        std::vector<double> lam, lam_prev, unorm2;
        double err1 = INFINITY, err2 = INFINITY, err2_prev = INFINITY;
        int stall = 0;
        double err2_best = INFINITY;   // LOBPCG: best FP32 residual so far
        bool has_prev = false;
    };
    std::vector<Slot> slots;
    int nact = 0;
    size_t next_k = 0;
    std::vector<int> order;   // k indices needing an iterative solve
    bool warm = false;        // warm start along segments of the k list
    // optional start blocks (q vectors per k = order[i] at init_blocks + i*q*n3)
    const C* init_blocks = nullptr;
    // segments: slot s walks order[seg_next[s] .. seg_end[s]) when warm starting
    std::vector<size_t> seg_next, seg_end;

    int nalloc = 0;   // buffers taken from the plan's pool 0
    template <typename X>
    bloch_status alloc(X** p, size_t n_el) {
        return plan_solver_buf(pl, 0, nalloc++, n_el * sizeof(X), (void**)p);
    }

    C* vec(C* base, int slot, int i = 0) const { return base + ((size_t)slot * q + i) * n3; }

    bloch_status setup() {
        bloch_status s;
        const size_t blk = (size_t)B * q * n3;
        segs = (long long)blk;
        const size_t ns = lob ? 3 : 1;   // X (and W, P) segments
        if ((s = alloc(&U, ns * blk)) || (s = alloc(&Ub, blk)) || (s = alloc(&KU, ns * blk)) || (s = alloc(&R, blk)))
            return s;
        if (!uniform) {
            if ((s = alloc(&MU, ns * blk)) || (s = alloc(&MUb, blk))) return s;
        }
        if (lob) {
            Wb = U + blk;
            Pb = U + 2 * blk;
            AWb = KU + blk;
            APb = KU + 2 * blk;
            if (!uniform) {
                MWb = MU + blk;
                MPb = MU + 2 * blk;
            }
            if ((s = alloc(&P2, blk)) || (s = alloc(&AP2, blk))) return s;
            if (!uniform && (s = alloc(&MP2, blk))) return s;
            if ((s = alloc(&d_C3, (size_t)B * 9 * q * q)) || (s = alloc(&d_lam3, (size_t)B * 3 * q))) return s;
            gsmem3 = gk_smem<T>(3 * q, !uniform);
            if (cudaFuncSetAttribute(k_svqb_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)gen_eig_smem(3 * q, kEigThreads)) != cudaSuccess)
                return set_error(BLOCH_ECUDA, "cudaFuncSetAttribute (LOBPCG Rayleigh-Ritz)");
        }
        dblk = (int)std::max(1LL, std::min<long long>((n3 + 255) / 256, std::max(1, 2048 / std::max(1, B * q))));
        gblk = (int)std::max(1LL, std::min<long long>((n3 + kGKChunk - 1) / kGKChunk, std::max(1, 608 / B)));
        gsmem = gk_smem<T>(q, !uniform);
        if (cudaFuncSetAttribute(k_gram_km<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max(gsmem, gsmem3)) != cudaSuccess)
            return set_error(BLOCH_ECUDA, "cudaFuncSetAttribute (Gram kernel)");
        if constexpr (std::is_same<T, float>::value) {
            use_tc = pl->opt.tensor_gram != 0 && q <= kQMaxTC;
            if (use_tc) {
                // about 16 CTAs per SM-slot of work, so each CTA's FP32 accumulator
                // sums a few thousand element pairs before the FP64 reduction
                gblk_tc = (int)std::max(1LL, std::min<long long>((n3 + kTCElems - 1) / kTCElems,
                                                                 std::max(1, 2432 / B)));
                tcsmem = tc_smem_bytes(q);
                if (allow_max_dyn_smem(k_gram_tc) != cudaSuccess)
                    return set_error(BLOCH_ECUDA, "cudaFuncSetAttribute (tensor-core Gram kernel)");
                if ((s = alloc(&d_gerr, 1))) return s;
                BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(d_gerr, 0, sizeof(int), pl->stream));
            }
        }
        const int gpart_blk = std::max(gblk, gblk_tc);
        if ((s = alloc(&d_part, (size_t)B * q * dblk * 3)) || (s = alloc(&d_scal, (size_t)B * q * 2)) ||
            (s = alloc(&d_gpart, (size_t)B * gpart_blk * 2 * q * q * (lob ? 9 : 1))) ||
            (s = alloc(&d_G, (size_t)2 * B * q * q * (lob ? 9 : 1))) ||
            (s = alloc(&d_Q, (size_t)B * q * q)) || (s = alloc(&d_idx, (size_t)3 * q)) ||
            (s = alloc(&d_val, (size_t)3 * q)))
            return s;
        if (!uniform && (s = alloc(&d_alpha, (size_t)3 * q))) return s;
        if ((s = alloc(&d_rq, (size_t)B * q * 4)) || (s = alloc(&d_invlam, (size_t)B * q)) ||
            (s = alloc(&d_lamq, (size_t)B * q)) || (s = alloc(&d_status, (size_t)B)) || (s = alloc(&d_tally, 4)))
            return s;
        BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(d_tally, 0, 4 * sizeof(long long), pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(d_rq, 0, (size_t)B * q * 4 * sizeof(double), pl->stream));
        if (cudaFuncSetAttribute(k_gen_herm_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gen_eig_smem(q, kEigThreads)) != cudaSuccess)
            return set_error(BLOCH_ECUDA, "cudaFuncSetAttribute (projected eigensolver)");
        if (fp64res) {
            if ((s = alloc(&U64, (size_t)q * n3)) || (s = alloc(&KU64, (size_t)q * n3))) return s;
            if (!uniform && (s = alloc(&MU64, (size_t)q * n3))) return s;
            if ((s = ensure_ws<double>(pl, q)) != BLOCH_OK) return s;
            if (pl->opt.refine_arith == 1 && (s = ensure_ws<dfloat>(pl, q)) != BLOCH_OK) return s;
        }
        if ((s = ensure_cg<T>(pl, B * q)) != BLOCH_OK) return s;
        slots.assign(B, Slot());
        return BLOCH_OK;
    }

    bloch_status set_k_range(int first, int count) {
        std::vector<double> kv((size_t)count * q * 3);
        for (int s = 0; s < count; ++s)
            for (int i = 0; i < q; ++i)
                for (int a = 0; a < 3; ++a) kv[((size_t)s * q + i) * 3 + a] = slots[first + s].k[a];
        return set_k<T>(pl, count * q, kv.data());
    }

    // LOBPCG: no search direction yet (a zero P is dropped by the rank-revealing Rayleigh-Ritz)
    bloch_status clear_directions(int s) {
        if (!lob) return BLOCH_OK;
        const size_t bytes = sizeof(C) * q * n3;
        BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(vec(Pb, s), 0, bytes, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(vec(APb, s), 0, bytes, pl->stream));
        if (!uniform) BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(vec(MPb, s), 0, bytes, pl->stream));
        return BLOCH_OK;
    }

    bloch_status init_slot(int s, int kidx) {
        TraceScope tr(pl, TR_SETUP);
        bloch_status cs = clear_directions(s);
        if (cs != BLOCH_OK) return cs;
        Slot& sl = slots[s];
        sl = Slot();
        sl.kidx = kidx;
        for (int a = 0; a < 3; ++a) sl.k[a] = (*klist)[kidx][a];
        sl.gamma = sl.k[0] == 0.0 && sl.k[1] == 0.0 && sl.k[2] == 0.0;
        sl.n_eff = sl.gamma ? n_bands - 3 : n_bands;
        sl.phase = 0;
        if (init_blocks) {
            size_t pos = 0;
            while (pos < order.size() && order[pos] != kidx) ++pos;
            BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(vec(U, s), init_blocks + pos * (size_t)q * n3,
                                                 sizeof(C) * q * n3, cudaMemcpyDeviceToDevice, pl->stream));
            return deflate_start(s);
        }
        std::vector<StartEntry> se = start_vectors(pl, sl.k, q, sl.gamma);
        BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(vec(U, s), 0, sizeof(C) * q * n3, pl->stream));
        std::vector<long long> idx(se.size());
        std::vector<double2> val(se.size());
        for (size_t i = 0; i < se.size(); ++i) {
            idx[i] = se[i].idx + (long long)s * q * n3;
            val[i] = se[i].val;
        }
        if (!se.empty()) {
            BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(d_idx, idx.data(), sizeof(long long) * idx.size(),
                                                 cudaMemcpyHostToDevice, pl->stream));
            BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(d_val, val.data(), sizeof(double2) * val.size(),
                                                 cudaMemcpyHostToDevice, pl->stream));
            ++pl->launches;
            // (the scatter buffers are rewritten by the next init in stream order)
            k_scatter<T><<<((int)se.size() + 127) / 128, 128, 0, pl->stream>>>(U, d_idx, d_val, (int)se.size());
        }
        return deflate_start(s);
    }

    // Gamma with a non-uniform density: the start block must be M-orthogonal
    // to the rigid translations (M couples bin 0 with the other bins)
    bloch_status deflate_start(int s) {
        if (uniform || !slots[s].gamma) return BLOCH_OK;
        launch_M<T>(pl, q, vec(U, s), vec(MU, s), T(1));
        return gamma_deflate<T>(pl, q, vec(U, s), vec(MU, s), d_alpha);
    }

    // Rayleigh quotients and residuals of vectors [vo, vo+nvs) of slots
    // [first, first+count) (nvs == q when count > 1): sums finished on the
    // device into d_rq, 1/lambda into d_invlam; residual_step reads them back
    // once and residual_finish turns them into the slots' lam, err1, err2.
    std::vector<double> stg_rq;
    template <typename TK>
    bloch_status residual_part(int first, int count, int vo, int nvs, const cplx_t<TK>* Uk, const cplx_t<TK>* KUk,
                               const cplx_t<TK>* MUk) {
        const int nv = count * nvs;
        if (nv == 0) return BLOCH_OK;
        dim3 gr(dblk, nv);
        pl->launches += 4;
        k_rq_dots<TK><<<gr, 256, 0, pl->stream>>>(Uk, KUk, MUk, rho_s, n3, d_part);
        k_rq_final<<<nv, 128, 0, pl->stream>>>(d_part, dblk, first, nvs, vo, q, d_rq, d_scal, d_invlam);
        k_residual<TK, T><<<gr, 256, 0, pl->stream>>>(Uk, KUk, MUk, rho_s, d_scal, vec(R, first, vo), n3, d_part);
        k_r2_final<<<nv, 128, 0, pl->stream>>>(d_part, dblk, first, nvs, vo, q, d_rq);
        return BLOCH_OK;
    }

    void residual_finish(int first, int count) {
        for (int s = 0; s < count; ++s) {
            Slot& sl = slots[first + s];
            sl.lam_prev = sl.lam;
            sl.lam.assign(q, 0.0);
            sl.unorm2.assign(q, 0.0);
            double e2 = 0;
            for (int i = 0; i < q; ++i) {
                const double* r = stg_rq.data() + ((size_t)s * q + i) * 4;   // (ukv, umu, kk, r2)
                const double lam = r[1] > 0 ? r[0] / r[1] : 0.0;
                sl.lam[i] = lam;
                sl.unorm2[i] = r[1];
                if (i < sl.n_eff && r[2] > 0) e2 = std::max(e2, lam * std::sqrt(r[3]) / std::sqrt(r[2]));
            }
            sl.err2_prev = sl.err2;
            sl.err2 = e2;
            if (sl.has_prev) {
                double num = 0, den = 0;
                for (int i = 0; i < sl.n_eff; ++i) {
                    num += (sl.lam[i] - sl.lam_prev[i]) * (sl.lam[i] - sl.lam_prev[i]);
                    den += sl.lam_prev[i] * sl.lam_prev[i];
                }
                sl.err1 = den > 0 ? std::sqrt(num / den) : 0.0;
            }
            sl.has_prev = true;
            st->k_applies += q;
        }
    }

    bloch_status residual_step(int first, int count) {
        bloch_status s;
        int i = first;
        while (i < first + count) {
            if (slots[i].phase == 0 || !fp64res) {
                int j = i;
                while (j < first + count && (slots[j].phase == 0 || !fp64res)) ++j;
                if ((s = set_k_range(i, j - i)) != BLOCH_OK) return s;
                TraceScope tr(pl, std::is_same<T, float>::value ? TR_RES32 : TR_RES64);
                launch_K<T>(pl, (j - i) * q, vec(U, i), vec(KU, i), T(1));
                if (!uniform) launch_M<T>(pl, (j - i) * q, vec(U, i), vec(MU, i), T(1));
                if ((s = residual_part<T>(i, j - i, 0, q, vec(U, i), vec(KU, i), uniform ? nullptr : vec(MU, i))) !=
                    BLOCH_OK)
                    return s;
                i = j;
            } else {
                // FP64 refinement: residuals and Rayleigh quotients of the wanted
                // vectors from an FP64 operator apply (once per eigenpair when the
                // check passes); the guard vectors of the block stay FP32
                TraceScope tr(pl, TR_RES64);
                const int nw = std::max(1, std::min(q, slots[i].n_eff));
                const size_t ne = (size_t)nw * n3;
                std::vector<double> kv((size_t)q * 3);
                for (int v = 0; v < q; ++v)
                    for (int a = 0; a < 3; ++a) kv[(size_t)v * 3 + a] = slots[i].k[a];
                if (pl->opt.refine_arith == 1) {
                    // operator applies in float-float (the U64 / KU64 / MU64 buffers hold
                    // float-float values first, FP64 ones after the in-place conversion)
                    pl->launches += 3 + (uniform ? 0 : 1);
                    k_convert<T, dfloat><<<1024, 256, 0, pl->stream>>>(vec(U, i), (dfloat2*)U64, ne);
                    if ((s = set_k<dfloat>(pl, nw, kv.data())) != BLOCH_OK) return s;
                    launch_K<dfloat>(pl, nw, (const dfloat2*)U64, (dfloat2*)KU64, dfloat(1.0f));
                    if (!uniform) launch_M<dfloat>(pl, nw, (const dfloat2*)U64, (dfloat2*)MU64, dfloat(1.0f));
                    k_convert_inplace<dfloat, double><<<1024, 256, 0, pl->stream>>>(KU64, ne);
                    if (!uniform) k_convert_inplace<dfloat, double><<<1024, 256, 0, pl->stream>>>(MU64, ne);
                    k_convert<T, double><<<1024, 256, 0, pl->stream>>>(vec(U, i), U64, ne);
                } else {
                    ++pl->launches;
                    k_convert<T, double><<<1024, 256, 0, pl->stream>>>(vec(U, i), U64, ne);
                    if ((s = set_k<double>(pl, nw, kv.data())) != BLOCH_OK) return s;
                    launch_K<double>(pl, nw, U64, KU64, 1.0);
                    if (!uniform) launch_M<double>(pl, nw, U64, MU64, 1.0);
                }
                if (lob) {
                    // LOBPCG's next Rayleigh-Ritz reads A X (and M X) of the block:
                    // the fresh FP64 images, rounded, replace the previous ones
                    ++pl->launches;
                    k_convert<double, T><<<1024, 256, 0, pl->stream>>>(KU64, vec(KU, i), ne);
                    if (!uniform) {
                        ++pl->launches;
                        k_convert<double, T><<<1024, 256, 0, pl->stream>>>(MU64, vec(MU, i), ne);
                    }
                }
                if ((s = residual_part<double>(i, 1, 0, nw, U64, KU64, uniform ? nullptr : MU64)) != BLOCH_OK) return s;
                if (nw < q) {
                    if ((s = set_k<T>(pl, q - nw, kv.data())) != BLOCH_OK) return s;
                    launch_K<T>(pl, q - nw, vec(U, i, nw), vec(KU, i, nw), T(1));
                    if (!uniform) launch_M<T>(pl, q - nw, vec(U, i, nw), vec(MU, i, nw), T(1));
                    if ((s = residual_part<T>(i, 1, nw, q - nw, vec(U, i, nw), vec(KU, i, nw),
                                              uniform ? nullptr : vec(MU, i, nw))) != BLOCH_OK)
                        return s;
                }
                ++i;
            }
        }
        BLOCH_CUDA_CHECK_RET(cudaGetLastError());
        // the one host synchronisation of a sweep: residual sums, the status of
        // the projected eigensolves that preceded them, PCG totals
        stg_rq.resize((size_t)count * q * 4);
        std::vector<int> stat(std::max(eig_pending, 1), 0);
        long long tl[4];
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(stg_rq.data(), d_rq + (size_t)first * q * 4,
                                             sizeof(double) * stg_rq.size(), cudaMemcpyDeviceToHost, pl->stream));
        if (eig_pending)
            BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(stat.data(), d_status, sizeof(int) * eig_pending,
                                                 cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(tl, d_tally, sizeof(tl), cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
        st->cg_iterations += tl[0] - tally_host[0];
        st->k_applies += tl[0] - tally_host[0];
        pl->launches += (unsigned long long)(tl[3] - tally_host[3]) * (unsigned long long)pl->pcg_launches_per_iter;
        const bool nonfinite = tl[2] > tally_host[2];
        for (int t = 0; t < 4; ++t) tally_host[t] = tl[t];
        if (nonfinite) return set_error(BLOCH_ENONFINITE, "PCG met a non-finite residual");
        for (int t = 0; t < eig_pending; ++t)
            if (stat[t] == 1) return set_error(BLOCH_ENOTCONV_EIG, "projected mass matrix lost definiteness");
        eig_pending = 0;
        residual_finish(first, count);
        return BLOCH_OK;
    }

    void finalize_slot(int s, bool converged) {
        TraceScope tr(pl, TR_SETUP);
        Slot& sl = slots[s];
        const double lam_scale = pl->Kscale / pl->rho_ref;
        double* om = omega_out + (size_t)sl.kidx * n_bands;
        int b = 0;
        if (sl.gamma)
            for (; b < std::min(3, n_bands); ++b) om[b] = 0.0;
        for (int i = 0; i < sl.n_eff; ++i) om[b + i] = std::sqrt(std::max(sl.lam[i], 0.0) * lam_scale);
        st->outer_iterations += sl.sweeps;
        st->max_rel_residual = std::max(st->max_rel_residual, sl.err2);
        if (!converged) {
            any_unconverged = true;
            st->k_unconverged += 1;
        }
        if (vecs_out) {
            C* out = (C*)vecs_out + (size_t)sl.kidx * n_bands * n3;
            if (sl.gamma) {
                cudaMemsetAsync(out, 0, sizeof(C) * std::min(3, n_bands) * n3, pl->stream);
                std::vector<long long> idx;
                std::vector<double2> val;
                const double nv = 1.0 / std::sqrt(pl->rho_ref * rho_s);
                for (int c = 0; c < std::min(3, n_bands); ++c) {
                    idx.push_back((long long)sl.kidx * n_bands * n3 + (long long)c * n3 + (long long)c * pl->V);
                    val.push_back(make_double2(nv, 0.0));
                }
                cudaMemcpyAsync(d_idx, idx.data(), sizeof(long long) * idx.size(), cudaMemcpyHostToDevice, pl->stream);
                cudaMemcpyAsync(d_val, val.data(), sizeof(double2) * val.size(), cudaMemcpyHostToDevice, pl->stream);
                ++pl->launches;
                k_scatter<T><<<1, 32, 0, pl->stream>>>((C*)vecs_out, d_idx, d_val, (int)idx.size());
                cudaStreamSynchronize(pl->stream);
            }
            if (sl.n_eff > 0) {
                std::vector<double> sc(sl.n_eff);
                for (int i = 0; i < sl.n_eff; ++i)
                    sc[i] = sl.unorm2[i] > 0 ? 1.0 / std::sqrt(pl->rho_ref * sl.unorm2[i]) : 0.0;
                cudaMemcpyAsync(d_scal, sc.data(), sizeof(double) * sl.n_eff, cudaMemcpyHostToDevice, pl->stream);
                dim3 gr(dblk, sl.n_eff);
                ++pl->launches;
                k_scale_vecs<T, T><<<gr, 256, 0, pl->stream>>>(vec(U, s), out + (size_t)b * n3, d_scal, n3);
                cudaStreamSynchronize(pl->stream);
            }
        }
    }

    // move slot `from` into slot `to` (device blocks U, R, MU and host state)
    bloch_status move_slot(int from, int to) {
        TraceScope tr(pl, TR_SETUP);
        const size_t bytes = sizeof(C) * q * n3;
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(vec(U, to), vec(U, from), bytes, cudaMemcpyDeviceToDevice, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(vec(R, to), vec(R, from), bytes, cudaMemcpyDeviceToDevice, pl->stream));
        if (!uniform)
            BLOCH_CUDA_CHECK_RET(
                cudaMemcpyAsync(vec(MU, to), vec(MU, from), bytes, cudaMemcpyDeviceToDevice, pl->stream));
        if (lob) {
            BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(vec(Pb, to), vec(Pb, from), bytes, cudaMemcpyDeviceToDevice, pl->stream));
            BLOCH_CUDA_CHECK_RET(
                cudaMemcpyAsync(vec(APb, to), vec(APb, from), bytes, cudaMemcpyDeviceToDevice, pl->stream));
            if (!uniform)
                BLOCH_CUDA_CHECK_RET(
                    cudaMemcpyAsync(vec(MPb, to), vec(MPb, from), bytes, cudaMemcpyDeviceToDevice, pl->stream));
        }
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(d_invlam + (size_t)to * q, d_invlam + (size_t)from * q,
                                             sizeof(double) * q, cudaMemcpyDeviceToDevice, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(d_rq + (size_t)to * q * 4, d_rq + (size_t)from * q * 4,
                                             sizeof(double) * q * 4, cudaMemcpyDeviceToDevice, pl->stream));
        slots[to] = slots[from];
        if (warm) {
            seg_next[to] = seg_next[from];
            seg_end[to] = seg_end[from];
        }
        return BLOCH_OK;
    }

    // Next wave vector of a slot's segment: start from the slot's converged
    // block (the paper's warm start) unless k or its predecessor is Gamma,
    // where the rigid-translation bin changes role (cold start instead).
    bloch_status continue_slot(int s, int kidx) {
        const Slot prev = slots[s];
        const double* kn = (*klist)[kidx].data();
        const bool gn = kn[0] == 0.0 && kn[1] == 0.0 && kn[2] == 0.0;
        if (prev.gamma || gn) return init_slot(s, kidx);
        bloch_status cs = clear_directions(s);
        if (cs != BLOCH_OK) return cs;
        Slot& sl = slots[s];
        sl = Slot();
        sl.kidx = kidx;
        for (int a = 0; a < 3; ++a) sl.k[a] = kn[a];
        sl.gamma = false;
        sl.n_eff = n_bands;
        sl.phase = 0;
        return BLOCH_OK;
    }

    // One LOBPCG iteration on every active slot (enqueued, no host wait):
    // W = T R with T = P^-1 (the Green operator, Eq. precond), A W and M W,
    // the Rayleigh-Ritz projection of (A, M) on [X, W, P] (3q vectors, one
    // Gram pass), its rank-revealing solve, X <- [X, W, P] C_q and
    // P <- [W, P] C_q (with A P, M P carried alongside).  The next residual
    // step applies A to the new X afresh.
    bloch_status lobpcg_step() {
        bloch_status s;
        const int q3 = 3 * q;
        if ((s = set_k_range(0, nact)) != BLOCH_OK) return s;
        if ((s = lp_activate<T>(pl, nact, q, q)) != BLOCH_OK) return s;
        TraceScope tr(pl, TR_PROJECT);
        launch_precond<T>(pl, nact * q, R, Wb, T(1));
        lp_deactivate(pl);
        {
            TraceScope trk(pl, std::is_same<T, float>::value ? TR_RES32 : TR_RES64);
            launch_K<T>(pl, nact * q, Wb, AWb, T(1));
            if (!uniform) launch_M<T>(pl, nact * q, Wb, MWb, T(1));
        }
        st->k_applies += (long long)nact * q;
        if (!uniform)
            for (int i = 0; i < nact; ++i)
                if (slots[i].gamma && (s = gamma_deflate<T>(pl, q, vec(Wb, i), vec(MWb, i), d_alpha)) != BLOCH_OK)
                    return s;
        const int np3 = q3 * q3;
        pl->launches += 3;
        k_gram_km<T><<<dim3(gblk, nact), kGKThreads, gsmem3, pl->stream>>>(U, KU, uniform ? nullptr : MU, q3, n3,
                                                                          d_gpart, q, segs);
        k_gram_final<<<dim3((2 * np3 + 127) / 128, nact), 128, 0, pl->stream>>>(d_gpart, gblk, np3, nact, d_G);
        // rank-revealing Rayleigh-Ritz: directions of [X, W, P] whose M-norm falls
        // below the field precision's resolution are dropped
        const double eps = std::is_same<T, float>::value ? 1e-6 : 1e-13;
        k_svqb_eig<<<nact, kEigThreads, gen_eig_smem(q3, kEigThreads), pl->stream>>>(
            q3, d_G, d_G + (size_t)nact * np3, uniform ? rho_s : 1.0, eps, d_lam3, d_C3, d_status);
        eig_pending = 0;
        RotView rx;
        rx.in_slot = (long long)q * n3;
        rx.segstride = segs;
        rx.out_slot = (long long)q * n3;
        rx.qstride = np3;
        rx.qi = q3;
        rx.qo = q;
        rx.seg = q;
        rx.ldq = q3;
        RotView rp = rx;
        rp.qi = 2 * q;   // [W, P] with the rows q..3q of C
        pl->launches += 3;
        launch_rotate<T>(pl->stream, nact, U, Ub, d_C3, rx, n3);
        launch_rotate<T>(pl->stream, nact, Wb, P2, d_C3 + q * q3, rp, n3);
        launch_rotate<T>(pl->stream, nact, AWb, AP2, d_C3 + q * q3, rp, n3);
        const size_t bytes = sizeof(C) * (size_t)nact * q * n3;
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(U, Ub, bytes, cudaMemcpyDeviceToDevice, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(Pb, P2, bytes, cudaMemcpyDeviceToDevice, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(APb, AP2, bytes, cudaMemcpyDeviceToDevice, pl->stream));
        // M P afresh (a carried M P drifts in FP32 and spoils the next projection's metric)
        if (!uniform) launch_M<T>(pl, nact * q, Pb, MPb, T(1));
        for (int i = 0; i < nact; ++i) slots[i].sweeps += 1;
        BLOCH_CUDA_CHECK_RET(cudaGetLastError());
        return BLOCH_OK;
    }

    bloch_status run() {
        bloch_status s;
        // fill the slots
        nact = 0;
        if (warm) {
            const int nseg = std::min<int>(B, (int)order.size());
            seg_next.assign(B, 0);
            seg_end.assign(B, 0);
            for (int g = 0; g < nseg; ++g) {
                seg_next[g] = order.size() * g / nseg;
                seg_end[g] = order.size() * (g + 1) / nseg;
            }
            for (int g = 0; g < nseg; ++g) {
                if ((s = init_slot(nact, order[seg_next[g]++])) != BLOCH_OK) return s;
                ++nact;
            }
        }
        while (!warm && nact < B && next_k < order.size()) {
            if ((s = init_slot(nact, order[next_k++])) != BLOCH_OK) return s;
            ++nact;
        }
        if (nact == 0) return BLOCH_OK;
        if ((s = residual_step(0, nact)) != BLOCH_OK) return s;
        const double tol = tol_eig;
        while (nact > 0) {
            // convergence / phase decisions on the residuals just computed
            std::vector<int> done;
            for (int i = 0; i < nact; ++i) {
                Slot& sl = slots[i];
                const bool test = sl.err1 <= tol && sl.err2 <= 10.0 * tol;
                if (fp64res && sl.phase == 0) {
                    // FP32 residuals drive the sweeps until the stop test passes in
                    // FP32 (or err2 stalls at the FP32 noise floor); the FP64
                    // residual then verifies, and drives further sweeps if needed.
                    // (LOBPCG's FP32 residual fluctuates at that floor rather than
                    // settling: it counts sweeps without a 10 % gain on its best)
                    int need = 2;
                    if (lob) {
                        if (sl.err2 < 0.9 * sl.err2_best) {
                            sl.err2_best = sl.err2;
                            sl.stall = 0;
                        } else {
                            sl.stall += 1;
                        }
                        need = 3;
                    } else if (sl.err2 > 0.9 * sl.err2_prev) {
                        sl.stall += 1;
                    } else {
                        sl.stall = 0;
                    }
                    if (test || (sl.sweeps >= 4 && sl.stall >= need)) sl.phase = 1;
                    if (sl.sweeps >= max_outer) done.push_back(i);
                } else if (test || sl.sweeps >= max_outer) {
                    done.push_back(i);
                }
            }
            if (!done.empty()) {
                std::vector<int> fresh;
                for (int i : done) finalize_slot(i, slots[i].err1 <= tol && slots[i].err2 <= 10.0 * tol);
                // refill from the queue, then compact
                std::vector<int> holes = done;
                std::vector<char> is_hole(nact, 0);
                for (int h : holes) is_hole[h] = 1;
                for (int h : holes) {
                    if (warm) {
                        if (seg_next[h] < seg_end[h]) {
                            const int kn = order[seg_next[h]++];
                            if ((s = continue_slot(h, kn)) != BLOCH_OK) return s;
                            is_hole[h] = 0;
                            fresh.push_back(h);
                        }
                    } else if (next_k < order.size()) {
                        if ((s = init_slot(h, order[next_k++])) != BLOCH_OK) return s;
                        is_hole[h] = 0;
                        fresh.push_back(h);
                    }
                }
                int last = nact - 1;
                for (int h = 0; h < nact; ++h) {
                    if (!is_hole[h]) continue;
                    while (last > h && is_hole[last]) --last;
                    if (last <= h) break;
                    // move last active into h
                    for (int& f : fresh)
                        if (f == last) f = h;
                    if ((s = move_slot(last, h)) != BLOCH_OK) return s;
                    is_hole[h] = 0;
                    is_hole[last] = 1;
                }
                int na = 0;
                for (int h = 0; h < nact; ++h)
                    if (!is_hole[h]) na = h + 1;
                nact = na;
                for (int f : fresh)
                    if ((s = residual_step(f, 1)) != BLOCH_OK) return s;
                if (nact == 0) break;
            }
            if (lob) {
                if ((s = lobpcg_step()) != BLOCH_OK) return s;
                if ((s = residual_step(0, nact)) != BLOCH_OK) return s;
                continue;
            }
            // inverse step on all active slots: delta = A^-1 R (enqueued; no host wait)
            if ((s = set_k_range(0, nact)) != BLOCH_OK) return s;
            if ((s = lp_activate<T>(pl, nact, q, q)) != BLOCH_OK) return s;
            s = pcg_enqueue<T>(pl, nact * q, R, Ub, 1.0, tol_lin, max_cg, d_tally);
            lp_deactivate(pl);
            if (s != BLOCH_OK) return s;
            st->linear_solves += (long long)nact * q;
            // U_bar = delta + U / lam (1/lam from the device)
            const int tr_proj = trace_begin(pl, TR_PROJECT);
            dim3 gv(dblk, nact * q);
            ++pl->launches;
            k_add_scaled<T><<<gv, 256, 0, pl->stream>>>(Ub, U, d_invlam, n3);
            // Kn = M U - r_cg (into KU), Mn = M U_bar
            const size_t ne = (size_t)nact * q * n3;
            ++pl->launches;
            k_kn<T><<<4096, 256, 0, pl->stream>>>(U, uniform ? nullptr : MU, rho_s, ws_of<T>(pl).r, KU, ne);
            if (!uniform) {
                launch_M<T>(pl, nact * q, Ub, MUb, T(1));
                // Gamma slots: keep U_bar M-orthogonal to the rigid translations
                // (A_0 x = R fixes x only up to them); A U_bar (Kn) is unchanged
                for (int i = 0; i < nact; ++i)
                    if (slots[i].gamma && (s = gamma_deflate<T>(pl, q, vec(Ub, i), vec(MUb, i), d_alpha)) != BLOCH_OK)
                        return s;
            }
            // projections K = Ub^H Kn, M = Ub^H Mn in one pass over the block
            dim3 gg(gblk, nact);
            const int npair = q * q;
            if constexpr (std::is_same<T, float>::value) {
                if (use_tc) {
                    ++pl->launches;
                    k_gram_tc<<<dim3(gblk_tc, nact), kTCThreads, tcsmem, pl->stream>>>(
                        Ub, KU, uniform ? nullptr : MUb, q, n3, d_gpart, d_gerr);
                    ++pl->launches;
                    k_gram_final<<<dim3((2 * npair + 127) / 128, nact), 128, 0, pl->stream>>>(d_gpart, gblk_tc,
                                                                                               npair, nact, d_G);
                }
            }
            if (!use_tc) {
                ++pl->launches;
                k_gram_km<T><<<gg, kGKThreads, gsmem, pl->stream>>>(Ub, KU, uniform ? nullptr : MUb, q, n3,
                                                                    d_gpart, q, 0LL);
                ++pl->launches;
                k_gram_final<<<dim3((2 * npair + 127) / 128, nact), 128, 0, pl->stream>>>(d_gpart, gblk, npair,
                                                                                           nact, d_G);
            }
            // EIG(K, M) of every slot on the device (FP64), then U = U_bar Q
            ++pl->launches;
            k_gen_herm_eig<<<nact, kEigThreads, gen_eig_smem(q, kEigThreads), pl->stream>>>(
                q, d_G, d_G + (size_t)nact * npair, uniform ? rho_s : 1.0, d_lamq, d_Q, d_status);
            eig_pending = nact;
            for (int i = 0; i < nact; ++i) slots[i].sweeps += 1;
            ++pl->launches;
            launch_basis<T>(pl->stream, nact, Ub, U, d_Q, q, n3);
            trace_end(pl, tr_proj);
            BLOCH_CUDA_CHECK_RET(cudaGetLastError());
            if (use_tc) {
                int gerr = 0;
                BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(&gerr, d_gerr, sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
                BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
                if (gerr) return set_error(BLOCH_ECUDA, "tensor-core Gram: a wait for the MMAs timed out");
            }
            if ((s = residual_step(0, nact)) != BLOCH_OK) return s;
        }
        return BLOCH_OK;
    }
};

template <typename T>
static bloch_status run_subspace(bloch_plan* pl, const std::vector<std::array<double, 3>>& ks, int n_bands,
                                 double* omega_out, void* vecs_out, bloch_stats* st, bool fp64res,
                                 const cplx_t<T>* init_blocks = nullptr) {
    Subspace<T> S;
    S.pl = pl;
    S.n3 = 3 * pl->V;
    S.n_bands = n_bands;
    S.n = n_bands;
    S.lob = pl->opt.method == BLOCH_LOBPCG && init_blocks == nullptr;
    const int qa = S.lob ? n_bands + 2 : std::min(2 * n_bands, n_bands + 8);
    S.q = pl->opt.block > 0 ? pl->opt.block : qa;
    S.q = std::max(S.q, n_bands + 1);
    if (S.q > kQMax) return set_error(BLOCH_EUNSUPPORTED, "block size above 32 vectors is not supported");
    if (S.lob) {
        // one Gram pass over [X, W, P]: 3q <= 44 (48 with a uniform density) tiles per CTA,
        // and its staging must fit the shared memory of a CTA
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const int qmax3 = pl->uniform_rho ? 48 : 44;
        if (3 * S.q > qmax3 || gk_smem<T>(3 * S.q, !pl->uniform_rho) > (size_t)optin)
            return set_error(BLOCH_EUNSUPPORTED, "LOBPCG block too large for one Gram pass (reduce the bands or the block)");
    }
    if ((long long)S.q > 3 * pl->V - 3) return set_error(BLOCH_EINVAL, "block larger than the problem");
    S.fp64res = fp64res;
    S.uniform = pl->uniform_rho;
    S.rho_s = pl->uniform_rho ? pl->rho_uniform_scaled : 1.0;
    S.tol_eig = pl->opt.tol_eig;
    S.tol_lin = pl->opt.tol_lin;
    if (std::is_same<T, float>::value) S.tol_lin = std::max(S.tol_lin, 3e-6);
    S.max_outer = pl->opt.max_outer;
    S.max_cg = pl->opt.max_cg;
    S.klist = &ks;
    S.omega_out = omega_out;
    S.vecs_out = vecs_out;
    S.st = st;
    S.warm = pl->opt.warm_start != 0 && init_blocks == nullptr;
    S.init_blocks = init_blocks;
    for (size_t i = 0; i < ks.size(); ++i) {
        const bool gamma = ks[i][0] == 0.0 && ks[i][1] == 0.0 && ks[i][2] == 0.0;
        if (gamma && n_bands <= 3) {
            for (int b = 0; b < n_bands; ++b) omega_out[i * n_bands + b] = 0.0;
            continue;
        }
        S.order.push_back((int)i);
    }
    // slots: from the options or from free memory
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    freeb += plan_solver_bytes(pl, 0);   // this solver's pool, held from earlier solves and reused
    const size_t blk = (size_t)S.q * S.n3 * sizeof(cplx_t<T>);
    const size_t per_slot = blk * (S.lob ? (S.uniform ? 15 : 20) : (S.uniform ? 9 : 11)) + 64 * 1024;
    long long Bmax = std::max<long long>(1, (long long)(0.6 * (double)freeb / (double)per_slot));
    Bmax = std::min<long long>(Bmax, 10922 / S.q);
    int B = pl->opt.k_batch > 0 ? pl->opt.k_batch : (int)Bmax;
    if (S.warm && pl->opt.k_batch <= 0)
        B = std::min<int>(B, std::max<int>(1, ((int)S.order.size() + 7) / 8));   // segments of ~8 wave vectors
    B = std::max(1, std::min<int>(B, (int)std::max<size_t>(1, S.order.size())));
    S.B = B;
    if (S.order.empty()) return BLOCH_OK;
    bloch_status s = S.setup();
    if (s != BLOCH_OK) return s;
    s = S.run();
    if (s != BLOCH_OK) return s;
    if (S.any_unconverged) return set_error(BLOCH_ENOTCONV_EIG, "eigensolver reached its sweep cap");
    return BLOCH_OK;
}

// ====================================================================
// Shift-invert Lanczos with thick restart (Section 3.3, Eqs. shift and
// def_invop): Lanczos on OP = A_k^-1 M in the M inner product; the n largest
// Ritz values theta of OP give lambda = 1/theta.  Restarting keeps the
// kk = n + (m - n)/2 leading Ritz vectors and the residual vector (thick
// restart, equivalent to implicit restart with exact shifts).
//
// Device resident: the slots (one wave vector each) advance in lockstep,
// one Lanczos step per slot per step, all slots sharing one batched PCG
// (Algorithm 2, graph-resident loop).  Every step -- the PCG, the two passes
// of classical Gram-Schmidt in the M inner product, the Lanczos coefficients
// and the normalisation -- runs on the device with no host synchronisation;
// the Ritz analysis of a restart (an FP64 Jacobi eigensolve per slot) runs on
// the device too, so the host synchronises once per restart cycle to read the
// convergence flags.  Converged slots are compacted out at a restart; a new
// batch of wave vectors starts when a batch is finished.
//
// A non-uniform density keeps the M-images of the basis vectors beside them
// (one mass-operator apply per step); at k = 0 the rigid translations are
// M-deflated from the start vector and from every new Lanczos vector.
// ====================================================================
template <typename T>
struct Lanczos {
    using C = cplx_t<T>;
    static constexpr int kThreadsRitz = 64;
    bloch_plan* pl;
    int n_bands, m, B;
    long long n3;
    bool uniform = true;
    double rho_s, tol_eig, tol_lin;
    int max_outer, max_cg;
    const std::vector<std::array<double, 3>>* klist;
    double* omega_out;
    void* vecs_out;
    bloch_stats* st;
    bool any_unconverged = false;
    std::vector<int> order;
    size_t next_k = 0;
    // optional hand-off to the refinement: the q_out leading Ritz vectors of
    // k = order[i] go to ritz_out + i * q_out * n3 (M-orthonormal)
    C* ritz_out = nullptr;
    int q_out = 0;

    C *Vb = nullptr, *MVb = nullptr, *Tmp = nullptr, *TmpM = nullptr, *Bc = nullptr, *Xc = nullptr, *MXc = nullptr;
    double2 *d_part = nullptr, *d_h = nullptr, *d_Q = nullptr, *d_H = nullptr, *d_alpha = nullptr;
    int *d_nv = nullptr, *d_neff = nullptr, *d_conv = nullptr, *d_jac = nullptr;
    double *d_s = nullptr, *d_theta = nullptr, *d_est = nullptr;
    long long* d_tally = nullptr;
    int nblk = 0;
    long long tally_host[4] = {0, 0, 0, 0};

    struct Slot {
        int kidx = -1;
        double k[3];
        bool gamma = false;
        int n_eff = 0;
    };
    std::vector<Slot> slots;
    int nact = 0;
    int restarts = 0;   // of the current batch (lockstep)

    int nalloc = 0;   // buffers taken from the plan's pool 1
    template <typename X>
    bloch_status alloc(X** p, size_t n_el) {
        return plan_solver_buf(pl, 1, nalloc++, n_el * sizeof(X), (void**)p);
    }
    long long stride() const { return (long long)(m + 1) * n3; }
    C* vb(int s, int i) const { return Vb + ((size_t)s * (m + 1) + i) * n3; }
    C* mvb(int s, int i) const { return MVb + ((size_t)s * (m + 1) + i) * n3; }
    int kk_restart() const { return std::min(m - 1, n_bands + (m - n_bands) / 2); }
    int kk_out() const { return ritz_out ? std::min(m, q_out) : n_bands; }
    unsigned gx() const { return (unsigned)std::max(1LL, std::min<long long>((n3 + 255) / 256, 2048 / std::max(1, B))); }

    bloch_status setup() {
        bloch_status s;
        nblk = (int)std::max(1LL, std::min<long long>((n3 + 255) / 256, std::max(1, 1024 / std::max(1, B))));
        if ((s = alloc(&Vb, (size_t)B * (m + 1) * n3)) || (s = alloc(&Tmp, (size_t)B * m * n3)) ||
            (s = alloc(&Bc, (size_t)B * n3)) || (s = alloc(&Xc, (size_t)B * n3)) ||
            (s = alloc(&d_part, (size_t)B * nblk * (m + 1))) || (s = alloc(&d_h, (size_t)B * (m + 1))) ||
            (s = alloc(&d_Q, (size_t)B * m * m)) || (s = alloc(&d_H, (size_t)B * (m + 1) * m)) ||
            (s = alloc(&d_nv, (size_t)B)) || (s = alloc(&d_neff, (size_t)B)) || (s = alloc(&d_conv, (size_t)B)) ||
            (s = alloc(&d_jac, (size_t)B)) || (s = alloc(&d_s, (size_t)B)) ||
            (s = alloc(&d_theta, (size_t)B * m)) || (s = alloc(&d_est, (size_t)B * m)) || (s = alloc(&d_tally, 4)))
            return s;
        if (!uniform) {
            if ((s = alloc(&MVb, (size_t)B * (m + 1) * n3)) || (s = alloc(&TmpM, (size_t)B * m * n3)) ||
                (s = alloc(&MXc, (size_t)B * n3)) || (s = alloc(&d_alpha, 3)))
                return s;
        }
        if ((s = ensure_cg<T>(pl, B)) != BLOCH_OK) return s;
        if (!uniform && (s = ensure_ws<T>(pl, B)) != BLOCH_OK) return s;
        BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(d_tally, 0, 4 * sizeof(long long), pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaFuncSetAttribute(k_lz_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)lz_ritz_smem(m, kThreadsRitz)));
        slots.assign(B, Slot());
        return BLOCH_OK;
    }

    // q tables, per-slot band counts and the learned tables for the current slot order
    bloch_status bind_slots() {
        std::vector<double> kv((size_t)nact * 3);
        std::vector<int> ne(nact);
        for (int i = 0; i < nact; ++i) {
            for (int a = 0; a < 3; ++a) kv[(size_t)i * 3 + a] = slots[i].k[a];
            ne[i] = slots[i].n_eff;
        }
        bloch_status s;
        if ((s = set_k<T>(pl, nact, kv.data())) != BLOCH_OK) return s;
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(d_neff, ne.data(), sizeof(int) * nact, cudaMemcpyHostToDevice, pl->stream));
        if ((s = lp_activate<T>(pl, nact, 1, 1)) != BLOCH_OK) return s;
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));   // host vectors above leave scope
        return BLOCH_OK;
    }

    // M-image of the nact vectors in Bc into MXc, and the Gamma deflation of both
    bloch_status m_image_and_deflate() {
        launch_M<T>(pl, nact, Bc, MXc, T(1));
        for (int i = 0; i < nact; ++i)
            if (slots[i].gamma) {
                bloch_status s = gamma_deflate<T>(pl, 1, Bc + (size_t)i * n3, MXc + (size_t)i * n3, d_alpha);
                if (s != BLOCH_OK) return s;
            }
        return BLOCH_OK;
    }

    // a new batch of wave vectors: random start vectors, M-normalised
    bloch_status start_batch() {
        TraceScope tr(pl, TR_SETUP);
        nact = 0;
        while (nact < B && next_k < order.size()) {
            Slot& sl = slots[nact];
            sl = Slot();
            sl.kidx = order[next_k++];
            for (int a = 0; a < 3; ++a) sl.k[a] = (*klist)[sl.kidx][a];
            sl.gamma = sl.k[0] == 0.0 && sl.k[1] == 0.0 && sl.k[2] == 0.0;
            sl.n_eff = sl.gamma ? n_bands - 3 : n_bands;
            ++pl->launches;
            k_start_random<T><<<1024, 256, 0, pl->stream>>>(Bc + (size_t)nact * n3, n3, pl->V, 12345ULL,
                                                            sl.gamma ? 1 : 0);
            ++nact;
        }
        restarts = 0;
        bloch_status s;
        if ((s = bind_slots()) != BLOCH_OK) return s;
        BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(d_H, 0, sizeof(double2) * (size_t)nact * (m + 1) * m, pl->stream));
        Workspace<T>& w = ws_of<T>(pl);
        if (uniform) {
            launch_dot<T>(pl, nact, Bc, Bc, n3, w.dots, w.part2);
        } else {
            if ((s = m_image_and_deflate()) != BLOCH_OK) return s;
            launch_dot<T>(pl, nact, Bc, MXc, n3, w.dots, w.part2);
        }
        pl->launches += 2;
        k_lz_norm<<<(nact + 63) / 64, 64, 0, pl->stream>>>(w.dots, uniform ? rho_s : 1.0, d_H, -1, m, nact, d_s);
        k_put_col<T><<<dim3(gx(), nact), 256, 0, pl->stream>>>(Bc, Vb, stride(), 0, n3, d_s);
        if (!uniform) {
            ++pl->launches;
            k_put_col<T><<<dim3(gx(), nact), 256, 0, pl->stream>>>(MXc, MVb, stride(), 0, n3, d_s);
        }
        BLOCH_CUDA_CHECK_RET(cudaGetLastError());
        return BLOCH_OK;
    }

    // one Lanczos step j -> j + 1 on every slot (no host synchronisation)
    bloch_status step(int j) {
        bloch_status s;
        Workspace<T>& w = ws_of<T>(pl);
        ++pl->launches;
        k_get_col<T><<<dim3(gx(), nact), 256, 0, pl->stream>>>(uniform ? Vb : MVb, stride(), j, n3, nullptr, Bc);
        pl->trace_pcg = TR_PCG_LZ;
        s = pcg_enqueue<T>(pl, nact, Bc, Xc, uniform ? rho_s : 1.0, tol_lin, max_cg, d_tally);
        pl->trace_pcg = TR_PCG_SUB;
        if (s != BLOCH_OK) return s;
        st->linear_solves += nact;
        const int tr_orth = trace_begin(pl, TR_ORTHO);
        if (!uniform) {
            launch_M<T>(pl, nact, Xc, MXc, T(1));
            for (int i = 0; i < nact; ++i)
                if (slots[i].gamma &&
                    (s = gamma_deflate<T>(pl, 1, Xc + (size_t)i * n3, MXc + (size_t)i * n3, d_alpha)) != BLOCH_OK)
                    return s;
        }
        const int nv = j + 1;
        ++pl->launches;
        k_fill_int<<<1, 64, 0, pl->stream>>>(d_nv, nact, nv);
        const C* Wm = uniform ? Xc : MXc;
        const double sc = uniform ? rho_s : 1.0;
        if (uniform && nv <= kGsMax && std::is_same<T, float>::value) {
            // the same two passes, reading the basis three times (dots; update + dots; update + norm)
            pl->launches += 9;
            const dim3 gg(nblk, nact);
            launch_gs3<T>(0, gg, pl->stream, Vb, stride(), Xc, n3, nullptr, d_nv, n3, nv, d_part);
            k_vdots_final<<<dim3(nv, nact), 256, 0, pl->stream>>>(d_part, nblk, nv, sc, d_h);
            k_h_accum<<<nact, 64, 0, pl->stream>>>(d_H, d_h, nv, nv, j, m);
            launch_gs3<T>(1, gg, pl->stream, Vb, stride(), Xc, n3, d_h, d_nv, n3, nv, d_part);
            k_vdots_final<<<dim3(nv, nact), 256, 0, pl->stream>>>(d_part, nblk, nv, sc, d_h);
            k_h_accum<<<nact, 64, 0, pl->stream>>>(d_H, d_h, nv, nv, j, m);
            launch_gs3<T>(2, gg, pl->stream, Vb, stride(), Xc, n3, d_h, d_nv, n3, nv, d_part);
            k_dot_final<<<nact, 256, 0, pl->stream>>>(d_part, nblk, w.dots);
            k_lz_norm<<<(nact + 63) / 64, 64, 0, pl->stream>>>(w.dots, sc, d_H, j, m, nact, d_s);
            ++pl->launches;
            k_put_col<T><<<dim3(gx(), nact), 256, 0, pl->stream>>>(Xc, Vb, stride(), j + 1, n3, d_s);
            trace_end(pl, tr_orth);
            BLOCH_CUDA_CHECK_RET(cudaGetLastError());
            return BLOCH_OK;
        }
        for (int pass = 0; pass < 2; ++pass) {
            pl->launches += 4;
            k_vdots<T><<<dim3(nblk, nv, nact), 256, 0, pl->stream>>>(Vb, stride(), Wm, n3, d_nv, n3, nv, d_part);
            k_vdots_final<<<dim3(nv, nact), 256, 0, pl->stream>>>(d_part, nblk, nv, sc, d_h);
            k_vaxpy<T><<<dim3(nblk, nact), 256, 0, pl->stream>>>(Vb, stride(), Xc, n3, d_h, d_nv, n3, nv);
            if (!uniform) {
                ++pl->launches;
                k_vaxpy<T><<<dim3(nblk, nact), 256, 0, pl->stream>>>(MVb, stride(), MXc, n3, d_h, d_nv, n3, nv);
            }
            k_h_accum<<<nact, 64, 0, pl->stream>>>(d_H, d_h, nv, nv, j, m);
        }
        launch_dot<T>(pl, nact, Xc, Wm, n3, w.dots, w.part2);
        pl->launches += 2;
        k_lz_norm<<<(nact + 63) / 64, 64, 0, pl->stream>>>(w.dots, sc, d_H, j, m, nact, d_s);
        k_put_col<T><<<dim3(gx(), nact), 256, 0, pl->stream>>>(Xc, Vb, stride(), j + 1, n3, d_s);
        if (!uniform) {
            ++pl->launches;
            k_put_col<T><<<dim3(gx(), nact), 256, 0, pl->stream>>>(MXc, MVb, stride(), j + 1, n3, d_s);
        }
        trace_end(pl, tr_orth);
        BLOCH_CUDA_CHECK_RET(cudaGetLastError());
        return BLOCH_OK;
    }

    // outputs of a slot whose Ritz vectors are in Tmp[s] (descending theta)
    void finish_slot(int s, const double* th, const double* es, bool conv) {
        Slot& sl = slots[s];
        const double lam_scale = pl->Kscale / pl->rho_ref;
        double* om = omega_out + (size_t)sl.kidx * n_bands;
        int b0 = 0;
        if (sl.gamma)
            for (; b0 < std::min(3, n_bands); ++b0) om[b0] = 0.0;
        double mx = 0.0;
        for (int i = 0; i < sl.n_eff; ++i) {
            om[b0 + i] = th[i] > 0 ? std::sqrt(lam_scale / th[i]) : 0.0;
            mx = std::max(mx, es[i] / std::max(std::fabs(th[i]), 1e-300));
        }
        st->outer_iterations += restarts;
        st->max_rel_residual = std::max(st->max_rel_residual, mx);
        if (!conv) {
            any_unconverged = true;
            if (!ritz_out) st->k_unconverged += 1;   // the hybrid's refinement decides for it
        }
        const C* ts = Tmp + (size_t)s * m * n3;
        if (ritz_out) {
            size_t pos = 0;
            while (pos < order.size() && order[pos] != sl.kidx) ++pos;
            C* dst = ritz_out + pos * (size_t)q_out * n3;
            const int kc = kk_out();
            cudaMemcpyAsync(dst, ts, sizeof(C) * (size_t)kc * n3, cudaMemcpyDeviceToDevice, pl->stream);
            if (kc < q_out)
                cudaMemsetAsync(dst + (size_t)kc * n3, 0, sizeof(C) * (size_t)(q_out - kc) * n3, pl->stream);
        }
        if (vecs_out) {
            C* out = (C*)vecs_out + (size_t)sl.kidx * n_bands * n3;
            if (sl.gamma) {
                cudaMemsetAsync(out, 0, sizeof(C) * std::min(3, n_bands) * n3, pl->stream);
                const C cv = mk(T(1.0 / std::sqrt(pl->rho_ref * rho_s)), T(0));
                for (int c = 0; c < std::min(3, n_bands); ++c)
                    cudaMemcpyAsync(out + (size_t)c * n3 + (size_t)c * pl->V, &cv, sizeof(C), cudaMemcpyHostToDevice,
                                    pl->stream);
                cudaStreamSynchronize(pl->stream);   // cv leaves scope
            }
            ++pl->launches;
            k_scale<T><<<1024, 256, 0, pl->stream>>>(ts, out + (size_t)b0 * n3, T(1.0 / std::sqrt(pl->rho_ref)),
                                                     (size_t)sl.n_eff * n3);
        }
    }

    // restart analysis of every slot (device), one host synchronisation;
    // converged slots are finished and compacted out
    bloch_status restart() {
        const int kr = kk_restart();
        const int kc = std::max(kr, kk_out());
        const int tr_rs = trace_begin(pl, TR_RESTART);
        pl->launches += 3;
        k_lz_ritz<<<nact, kThreadsRitz, lz_ritz_smem(m, kThreadsRitz), pl->stream>>>(
            m, d_H, d_neff, tol_eig, kc, kr, d_Q, d_theta, d_est, d_conv, d_jac);
        // only the kc kept or returned Ritz vectors are formed
        launch_basis_first<T>(pl->stream, nact, Vb, Tmp, d_Q, m, kc, n3, stride());
        k_lz_restart_copy<T><<<dim3(gx(), nact), 256, 0, pl->stream>>>(Vb, Tmp, m, kr, n3);
        if (!uniform) {
            pl->launches += 2;
            launch_basis_first<T>(pl->stream, nact, MVb, TmpM, d_Q, m, kc, n3, stride());
            k_lz_restart_copy<T><<<dim3(gx(), nact), 256, 0, pl->stream>>>(MVb, TmpM, m, kr, n3);
        }
        BLOCH_CUDA_CHECK_RET(cudaGetLastError());
        trace_end(pl, tr_rs);
        std::vector<double> th((size_t)nact * m), es((size_t)nact * m);
        std::vector<int> cv(nact), jo(nact);
        long long tl[4];
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(th.data(), d_theta, sizeof(double) * th.size(), cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(es.data(), d_est, sizeof(double) * es.size(), cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(cv.data(), d_conv, sizeof(int) * nact, cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(jo.data(), d_jac, sizeof(int) * nact, cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(tl, d_tally, sizeof(tl), cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
        // PCG totals since the previous restart
        st->cg_iterations += tl[0] - tally_host[0];
        st->k_applies += tl[0] - tally_host[0];
        pl->launches += (unsigned long long)(tl[3] - tally_host[3]) * (unsigned long long)pl->pcg_launches_per_iter;
        const bool nonfinite = tl[2] > tally_host[2];
        for (int i = 0; i < 4; ++i) tally_host[i] = tl[i];
        if (nonfinite) return set_error(BLOCH_ENONFINITE, "PCG met a non-finite residual in a Lanczos step");
        restarts += 1;
        TraceScope tr_out(pl, TR_RESTART);
        std::vector<char> done(nact, 0);
        for (int i = 0; i < nact; ++i) {
            const bool conv = cv[i] != 0 && jo[i] != 0;
            if (conv || restarts > max_outer) {
                finish_slot(i, th.data() + (size_t)i * m, es.data() + (size_t)i * m, conv);
                done[i] = 1;
            }
        }
        // compact: move the last active slot into each hole (basis kr + 1 vectors, H)
        int last = nact - 1;
        for (int h = 0; h < nact; ++h) {
            if (!done[h]) continue;
            while (last > h && done[last]) --last;
            if (last <= h) break;
            BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(vb(h, 0), vb(last, 0), sizeof(C) * (size_t)(kr + 1) * n3,
                                                 cudaMemcpyDeviceToDevice, pl->stream));
            if (!uniform)
                BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(mvb(h, 0), mvb(last, 0), sizeof(C) * (size_t)(kr + 1) * n3,
                                                     cudaMemcpyDeviceToDevice, pl->stream));
            BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(d_H + (size_t)h * (m + 1) * m, d_H + (size_t)last * (m + 1) * m,
                                                 sizeof(double2) * (size_t)(m + 1) * m, cudaMemcpyDeviceToDevice,
                                                 pl->stream));
            slots[h] = slots[last];
            done[h] = 0;
            done[last] = 1;
        }
        int na = 0;
        for (int h = 0; h < nact; ++h)
            if (!done[h]) na = h + 1;
        const bool changed = na != nact;
        nact = na;
        if (nact > 0 && changed) return bind_slots();
        return BLOCH_OK;
    }

    bloch_status run() {
        bloch_status s;
        while (next_k < order.size()) {
            if ((s = start_batch()) != BLOCH_OK) return s;
            int j = 0;
            while (nact > 0) {
                for (; j < m; ++j)
                    if ((s = step(j)) != BLOCH_OK) return s;
                if ((s = restart()) != BLOCH_OK) return s;
                j = kk_restart();
            }
        }
        lp_deactivate(pl);
        cudaStreamSynchronize(pl->stream);
        return BLOCH_OK;
    }
};

template <typename T>
static bloch_status run_lanczos(bloch_plan* pl, const std::vector<std::array<double, 3>>& ks, int n_bands,
                                double* omega_out, void* vecs_out, bloch_stats* st, cplx_t<T>* ritz_out = nullptr,
                                int q_out = 0, double tol_override = 0.0) {
    Lanczos<T> S;
    S.uniform = pl->uniform_rho;
    S.pl = pl;
    S.n3 = 3 * pl->V;
    S.n_bands = n_bands;
    S.m = pl->opt.ncv > 0 ? pl->opt.ncv : std::max(2 * n_bands + 1, 20);
    S.m = (int)std::min<long long>(S.m, 3 * pl->V - 4);
    if (S.m > kBasisQMax - 1)
        return set_error(BLOCH_EUNSUPPORTED, "Lanczos basis above 63 vectors is not supported");
    if (S.m < n_bands + 1) return set_error(BLOCH_EINVAL, "Lanczos basis too small for the requested bands");
    S.rho_s = pl->uniform_rho ? pl->rho_uniform_scaled : 1.0;
    S.tol_eig = tol_override > 0 ? tol_override : pl->opt.tol_eig;
    S.tol_lin = pl->opt.tol_lin;
    if (std::is_same<T, float>::value) S.tol_lin = std::max(S.tol_lin, 3e-6);
    S.ritz_out = ritz_out;
    S.q_out = q_out;
    if (q_out > S.m) S.m = std::min<int>(q_out + 4, 63);
    S.max_outer = pl->opt.max_outer;
    S.max_cg = pl->opt.max_cg;
    S.klist = &ks;
    S.omega_out = omega_out;
    S.vecs_out = vecs_out;
    S.st = st;
    for (size_t i = 0; i < ks.size(); ++i) {
        const bool gamma = ks[i][0] == 0.0 && ks[i][1] == 0.0 && ks[i][2] == 0.0;
        if (gamma && n_bands <= 3) {
            for (int b = 0; b < n_bands; ++b) omega_out[i * n_bands + b] = 0.0;
            continue;
        }
        S.order.push_back((int)i);
    }
    if (S.order.empty()) return BLOCH_OK;
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    freeb += plan_solver_bytes(pl, 1);   // this solver's pool, held from earlier solves and reused
    // basis, rotated basis, step vectors and CG workspace (twice the basis part
    // with a non-uniform density: the M-images are kept too)
    const size_t per_slot = (size_t)((2 * S.m + 1) * (S.uniform ? 1 : 2) + 2 + 6) * S.n3 * sizeof(cplx_t<T>);
    long long Bmax = std::max<long long>(1, (long long)(0.5 * (double)freeb / (double)per_slot));
    Bmax = std::min<long long>(Bmax, 64);
    int B = pl->opt.k_batch > 0 ? pl->opt.k_batch : (int)Bmax;
    S.B = std::max(1, std::min<int>(B, (int)S.order.size()));
    bloch_status s = S.setup();
    if (s != BLOCH_OK) return s;
    s = S.run();
    if (s != BLOCH_OK) return s;
    if (S.any_unconverged) return set_error(BLOCH_ENOTCONV_EIG, "Lanczos reached its restart cap");
    return BLOCH_OK;
}

// FP32 chosen form with method = Lanczos: FP32 shift-invert Lanczos (inner PCG
// at the FP32 tolerance) delivers the q leading Ritz vectors of every wave
// vector; Algorithm 1 sweeps then refine that block to the requested
// tolerance, with the FP64 residual check of the FP32 form.  Wave vectors go
// through in chunks so the hand-off buffer stays bounded.
static bloch_status run_hybrid(bloch_plan* pl, const std::vector<std::array<double, 3>>& ks, int n_bands,
                               double* omega_out, void* vecs_out, bloch_stats* st) {
    using C = float2;
    const int q = pl->opt.block > 0 ? pl->opt.block : std::min(2 * n_bands, n_bands + 8);
    const long long n3 = 3 * pl->V;
    const int chunk = std::max(1, std::min<int>((int)ks.size(), pl->opt.k_batch > 0 ? pl->opt.k_batch : 8));
    const size_t need = sizeof(C) * (size_t)chunk * q * n3;
    if (need > pl->handoff_bytes) {
        cudaStreamSynchronize(pl->stream);
        if (pl->d_handoff) pl->device_bytes -= pl->handoff_bytes;
        cudaFree(pl->d_handoff);
        pl->d_handoff = nullptr;
        pl->handoff_bytes = 0;
        cudaError_t e = cudaMalloc(&pl->d_handoff, need);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaMalloc (Lanczos hand-off)");
        pl->handoff_bytes = need;
        pl->device_bytes += need;
    }
    C* buf = (C*)pl->d_handoff;
    std::vector<double> om_tmp;
    bloch_status s = BLOCH_OK;
    bool unconverged = false;
    const double tol_l = pl->opt.hybrid_tol > 0 ? pl->opt.hybrid_tol : std::max(1e-5, 10.0 * pl->opt.tol_eig);
    for (size_t c0 = 0; c0 < ks.size() && s == BLOCH_OK; c0 += chunk) {
        std::vector<std::array<double, 3>> sub(ks.begin() + c0, ks.begin() + std::min(ks.size(), c0 + chunk));
        om_tmp.assign(sub.size() * n_bands, 0.0);
        s = run_lanczos<float>(pl, sub, n_bands, om_tmp.data(), nullptr, st, buf, q, tol_l);
        if (s == BLOCH_ENOTCONV_EIG) s = BLOCH_OK;   // the refinement decides convergence
        if (s != BLOCH_OK) break;
        void* vsub = vecs_out ? (void*)((C*)vecs_out + c0 * (size_t)n_bands * n3) : nullptr;
        // the refinement's inner solves only correct a small residual (reading of
        // Algorithm 1 in residual-correction form): 1e-3 relative is enough
        const double tol_lin_saved = pl->opt.tol_lin;
        pl->opt.tol_lin = std::max(tol_lin_saved, 1e-3);
        s = run_subspace<float>(pl, sub, n_bands, omega_out + c0 * n_bands, vsub, st, true, buf);
        pl->opt.tol_lin = tol_lin_saved;
        if (s == BLOCH_ENOTCONV_EIG) {
            unconverged = true;
            s = BLOCH_OK;
        }
    }
    cudaStreamSynchronize(pl->stream);
    if (s != BLOCH_OK) return s;
    if (unconverged) return set_error(BLOCH_ENOTCONV_EIG, "refinement reached its sweep cap");
    return BLOCH_OK;
}

}  // namespace bloch

using namespace bloch;

bloch_status bloch_solve_bands_impl(bloch_plan* pl, int n_k, const double* k_list, int n_bands, double* omega_out,
                                    void* vecs_out, bloch_stats* stats) {
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<std::array<double, 3>> ks(n_k);
    for (int i = 0; i < n_k; ++i)
        for (int a = 0; a < 3; ++a) {
            ks[i][a] = k_list[3 * i + a];
            if (!std::isfinite(ks[i][a])) return set_error(BLOCH_ENONFINITE, "k_list has a non-finite entry");
        }
    bloch_stats st;
    std::memset(&st, 0, sizeof(st));
    bloch_status s;
    const int tr_span = trace_begin(pl, TR_SPAN);
    if (pl->opt.autotune && !pl->tuned) {
        const int q = pl->opt.block > 0 ? pl->opt.block : std::min(2 * n_bands, n_bands + 8);
        s = bloch_plan_autotune(pl, pl->opt.precision, std::max(1, std::min(q, 10922)), nullptr);
        if (s != BLOCH_OK) return s;
    }
    if (pl->opt.method == BLOCH_SUBSPACE || pl->opt.method == BLOCH_LOBPCG) {
        if (pl->opt.precision == BLOCH_FP32)
            s = run_subspace<float>(pl, ks, n_bands, omega_out, vecs_out, &st, true);
        else
            s = run_subspace<double>(pl, ks, n_bands, omega_out, vecs_out, &st, false);
    } else {
        if (pl->opt.precision == BLOCH_FP32)
            s = run_hybrid(pl, ks, n_bands, omega_out, vecs_out, &st);
        else
            s = run_lanczos<double>(pl, ks, n_bands, omega_out, vecs_out, &st);
    }
    trace_end(pl, tr_span);
    cudaStreamSynchronize(pl->stream);
    st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    trace_add(pl, TR_WALL, 1e3 * st.seconds);
    trace_collect(pl);
    pl->last_stats = st;
    if (stats) *stats = st;
    return s;
}

extern "C" bloch_status bloch_host_gen_eig(int32_t n, const double* K, const double* M, double* lam, double* Q) {
    if (n < 1 || !K || !M || !lam || !Q) return set_error(BLOCH_EINVAL, "invalid arguments");
    std::vector<cd> Kc((size_t)n * n), Mc((size_t)n * n), Qc;
    for (size_t i = 0; i < (size_t)n * n; ++i) {
        Kc[i] = cd(K[2 * i], K[2 * i + 1]);
        Mc[i] = cd(M[2 * i], M[2 * i + 1]);
    }
    std::vector<double> w;
    const int rc = gen_herm_eig(n, Kc.data(), Mc.data(), w, Qc);
    if (rc == 1) return set_error(BLOCH_EINVAL, "M is not positive definite");
    for (int i = 0; i < n; ++i) lam[i] = w[i];
    for (size_t i = 0; i < (size_t)n * n; ++i) {
        Q[2 * i] = Qc[i].real();
        Q[2 * i + 1] = Qc[i].imag();
    }
    return rc == 0 ? BLOCH_OK : set_error(BLOCH_ENOTCONV_EIG, "Jacobi sweeps did not converge");
}
