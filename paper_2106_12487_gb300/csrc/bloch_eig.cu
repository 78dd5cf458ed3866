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

size_t plan_solver_bytes(const bloch_plan* pl) {
    size_t t = pl->handoff_bytes;
    for (const auto& v : pl->solver_bufs)
        for (const auto& b : v) t += b.bytes;
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
    bloch_plan* pl;
    int n, q, B;
    long long n3;
    bool fp64res;     // FP32 fields with an FP64 residual refinement phase
    bool uniform;
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
        if ((s = alloc(&U, blk)) || (s = alloc(&Ub, blk)) || (s = alloc(&KU, blk)) || (s = alloc(&R, blk))) return s;
        if (!uniform) {
            if ((s = alloc(&MU, blk)) || (s = alloc(&MUb, blk))) return s;
        }
        dblk = (int)std::max(1LL, std::min<long long>((n3 + 255) / 256, std::max(1, 2048 / std::max(1, B * q))));
        gblk = (int)std::max(1LL, std::min<long long>((n3 + kGKChunk - 1) / kGKChunk, std::max(1, 608 / B)));
        gsmem = gk_smem<T>(q, !uniform);
        if (cudaFuncSetAttribute(k_gram_km<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem) !=
            cudaSuccess)
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
            (s = alloc(&d_gpart, (size_t)B * gpart_blk * 2 * q * q)) || (s = alloc(&d_G, (size_t)2 * B * q * q)) ||
            (s = alloc(&d_Q, (size_t)B * q * q)) || (s = alloc(&d_idx, (size_t)3 * q)) ||
            (s = alloc(&d_val, (size_t)3 * q)))
            return s;
        if (!uniform && (s = alloc(&d_alpha, (size_t)3 * q))) return s;
        if (fp64res) {
            if ((s = alloc(&U64, (size_t)q * n3)) || (s = alloc(&KU64, (size_t)q * n3))) return s;
            if (!uniform && (s = alloc(&MU64, (size_t)q * n3))) return s;
            if ((s = ensure_ws<double>(pl, q)) != BLOCH_OK) return s;
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

    bloch_status init_slot(int s, int kidx) {
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
            k_scatter<T><<<((int)se.size() + 127) / 128, 128, 0, pl->stream>>>(U, d_idx, d_val, (int)se.size());
            // the scatter buffers are reused by the next init: wait for the copies
            BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
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
    // [first, first+count) (nvs == q when count > 1), staged per vector;
    // residual_finish turns the staged values into the slots' lam, err1, err2.
    std::vector<double> stg_ukv, stg_umu, stg_kk, stg_r2;
    template <typename TK>
    bloch_status residual_part(int first, int count, int vo, int nvs, const cplx_t<TK>* Uk, const cplx_t<TK>* KUk,
                               const cplx_t<TK>* MUk) {
        const int nv = count * nvs;
        if (nv == 0) return BLOCH_OK;
        const size_t need = (size_t)B * q;
        if (stg_ukv.size() < need) {
            stg_ukv.assign(need, 0.0);
            stg_umu.assign(need, 0.0);
            stg_kk.assign(need, 0.0);
            stg_r2.assign(need, 0.0);
        }
        dim3 gr(dblk, nv);
        ++pl->launches;
        k_rq_dots<TK><<<gr, 256, 0, pl->stream>>>(Uk, KUk, MUk, rho_s, n3, d_part);
        std::vector<double> part((size_t)nv * dblk * 3);
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(part.data(), d_part, sizeof(double) * part.size(),
                                             cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
        std::vector<double> inv(nv);
        for (int v = 0; v < nv; ++v) {
            double a = 0, b = 0, c = 0;
            for (int j = 0; j < dblk; ++j) {
                a += part[((size_t)v * dblk + j) * 3 + 0];
                b += part[((size_t)v * dblk + j) * 3 + 1];
                c += part[((size_t)v * dblk + j) * 3 + 2];
            }
            const size_t at = (size_t)(first + v / nvs) * q + vo + v % nvs;
            stg_ukv[at] = a;
            stg_umu[at] = b;
            stg_kk[at] = c;
            const double lam = (b > 0) ? a / b : 0.0;
            inv[v] = lam > 0 ? 1.0 / lam : 0.0;
        }
        BLOCH_CUDA_CHECK_RET(
            cudaMemcpyAsync(d_scal, inv.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, pl->stream));
        ++pl->launches;
        k_residual<TK, T><<<gr, 256, 0, pl->stream>>>(Uk, KUk, MUk, rho_s, d_scal, vec(R, first, vo), n3, d_part);
        std::vector<double> rp((size_t)nv * dblk);
        BLOCH_CUDA_CHECK_RET(
            cudaMemcpyAsync(rp.data(), d_part, sizeof(double) * rp.size(), cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
        for (int v = 0; v < nv; ++v) {
            double r2 = 0;
            for (int j = 0; j < dblk; ++j) r2 += rp[(size_t)v * dblk + j];
            stg_r2[(size_t)(first + v / nvs) * q + vo + v % nvs] = r2;
        }
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
                const size_t at = (size_t)(first + s) * q + i;
                const double lam = stg_umu[at] > 0 ? stg_ukv[at] / stg_umu[at] : 0.0;
                sl.lam[i] = lam;
                sl.unorm2[i] = stg_umu[at];
                if (i < sl.n_eff && stg_kk[at] > 0) e2 = std::max(e2, lam * std::sqrt(stg_r2[at]) / std::sqrt(stg_kk[at]));
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
                residual_finish(i, j - i);
                i = j;
            } else {
                // FP64 refinement: residuals and Rayleigh quotients of the wanted
                // vectors from an FP64 operator apply (once per eigenpair when the
                // check passes); the guard vectors of the block stay FP32
                TraceScope tr(pl, TR_RES64);
                const int nw = std::max(1, std::min(q, slots[i].n_eff));
                const size_t ne = (size_t)nw * n3;
                ++pl->launches;
                k_convert<T, double><<<1024, 256, 0, pl->stream>>>(vec(U, i), U64, ne);
                std::vector<double> kv((size_t)q * 3);
                for (int v = 0; v < q; ++v)
                    for (int a = 0; a < 3; ++a) kv[(size_t)v * 3 + a] = slots[i].k[a];
                if ((s = set_k<double>(pl, nw, kv.data())) != BLOCH_OK) return s;
                launch_K<double>(pl, nw, U64, KU64, 1.0);
                if (!uniform) launch_M<double>(pl, nw, U64, MU64, 1.0);
                if ((s = residual_part<double>(i, 1, 0, nw, U64, KU64, uniform ? nullptr : MU64)) != BLOCH_OK) return s;
                if (nw < q) {
                    if ((s = set_k<T>(pl, q - nw, kv.data())) != BLOCH_OK) return s;
                    launch_K<T>(pl, q - nw, vec(U, i, nw), vec(KU, i, nw), T(1));
                    if (!uniform) launch_M<T>(pl, q - nw, vec(U, i, nw), vec(MU, i, nw), T(1));
                    if ((s = residual_part<T>(i, 1, nw, q - nw, vec(U, i, nw), vec(KU, i, nw),
                                              uniform ? nullptr : vec(MU, i, nw))) != BLOCH_OK)
                        return s;
                }
                residual_finish(i, 1);
                ++i;
            }
        }
        BLOCH_CUDA_CHECK_RET(cudaGetLastError());
        return BLOCH_OK;
    }

    void finalize_slot(int s, bool converged) {
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
        const size_t bytes = sizeof(C) * q * n3;
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(vec(U, to), vec(U, from), bytes, cudaMemcpyDeviceToDevice, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(vec(R, to), vec(R, from), bytes, cudaMemcpyDeviceToDevice, pl->stream));
        if (!uniform)
            BLOCH_CUDA_CHECK_RET(
                cudaMemcpyAsync(vec(MU, to), vec(MU, from), bytes, cudaMemcpyDeviceToDevice, pl->stream));
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
        Slot& sl = slots[s];
        sl = Slot();
        sl.kidx = kidx;
        for (int a = 0; a < 3; ++a) sl.k[a] = kn[a];
        sl.gamma = false;
        sl.n_eff = n_bands;
        sl.phase = 0;
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
                    if (sl.err2 > 0.9 * sl.err2_prev) sl.stall += 1;
                    else sl.stall = 0;
                    if (test || (sl.sweeps >= 4 && sl.stall >= 2)) sl.phase = 1;
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
            // inverse step on all active slots: delta = A^-1 R
            if ((s = set_k_range(0, nact)) != BLOCH_OK) return s;
            if ((s = lp_activate<T>(pl, nact, q, q)) != BLOCH_OK) return s;
            long long cg_it = 0;
            s = pcg_run<T>(pl, nact * q, R, Ub, 1.0, tol_lin, max_cg, false, nullptr, nullptr, &cg_it);
            lp_deactivate(pl);
            st->cg_iterations += cg_it;
            st->k_applies += cg_it;
            st->linear_solves += (long long)nact * q;
            if (s != BLOCH_OK && s != BLOCH_ENOTCONV_CG) return s;
            // U_bar = delta + U / lam
            const int tr_proj = trace_begin(pl, TR_PROJECT);
            std::vector<double> inv((size_t)nact * q);
            for (int i = 0; i < nact; ++i)
                for (int j = 0; j < q; ++j) inv[(size_t)i * q + j] = slots[i].lam[j] > 0 ? 1.0 / slots[i].lam[j] : 0.0;
            BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(d_scal, inv.data(), sizeof(double) * inv.size(),
                                                 cudaMemcpyHostToDevice, pl->stream));
            dim3 gv(dblk, nact * q);
            ++pl->launches;
            k_add_scaled<T><<<gv, 256, 0, pl->stream>>>(Ub, U, d_scal, n3);
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
                                                                    d_gpart);
                ++pl->launches;
                k_gram_final<<<dim3((2 * npair + 127) / 128, nact), 128, 0, pl->stream>>>(d_gpart, gblk, npair,
                                                                                           nact, d_G);
            }
            trace_end(pl, tr_proj);
            std::vector<double2> G((size_t)2 * nact * npair);
            BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(G.data(), d_G, sizeof(double2) * G.size(), cudaMemcpyDeviceToHost,
                                                 pl->stream));
            int gerr = 0;
            if (use_tc)
                BLOCH_CUDA_CHECK_RET(
                    cudaMemcpyAsync(&gerr, d_gerr, sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
            BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
            if (gerr) return set_error(BLOCH_ECUDA, "tensor-core Gram: a wait for the MMAs timed out");
            std::vector<double2> Qh((size_t)nact * npair);
            for (int i = 0; i < nact; ++i) {
                std::vector<cd> Km(npair), Mm(npair), Qm;
                const double ms = uniform ? rho_s : 1.0;
                for (int t = 0; t < npair; ++t) {
                    const double2 a = G[(size_t)i * npair + t], b = G[(size_t)(nact + i) * npair + t];
                    Km[t] = cd(a.x, a.y);
                    Mm[t] = cd(b.x, b.y) * ms;
                }
                std::vector<double> lam;
                const int rc = gen_herm_eig(q, Km.data(), Mm.data(), lam, Qm);
                if (rc == 1) return set_error(BLOCH_ENOTCONV_EIG, "projected mass matrix lost definiteness");
                for (int t = 0; t < npair; ++t) Qh[(size_t)i * npair + t] = make_double2(Qm[t].real(), Qm[t].imag());
                slots[i].sweeps += 1;
            }
            BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(d_Q, Qh.data(), sizeof(double2) * Qh.size(), cudaMemcpyHostToDevice,
                                                 pl->stream));
            {
                TraceScope tr(pl, TR_PROJECT);
                ++pl->launches;
                launch_basis<T>(pl->stream, nact, Ub, U, d_Q, q, n3);
            }
            BLOCH_CUDA_CHECK_RET(cudaGetLastError());
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
    const int qa = std::min(2 * n_bands, n_bands + 8);
    S.q = pl->opt.block > 0 ? pl->opt.block : qa;
    S.q = std::max(S.q, n_bands + 1);
    if (S.q > kQMax) return set_error(BLOCH_EUNSUPPORTED, "block size above 32 vectors is not supported");
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
    freeb += plan_solver_bytes(pl);   // held by the plan from earlier solves, reused
    const size_t blk = (size_t)S.q * S.n3 * sizeof(cplx_t<T>);
    const size_t per_slot = blk * (S.uniform ? 9 : 11) + 64 * 1024;
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
// kk = n + (m - n)/2 wanted Ritz vectors and the residual vector (thick
// restart, equivalent to implicit restart with exact shifts).  Each slot (one
// wave vector) advances one Lanczos step per iteration; all slots share one
// batched PCG per step.  Orthogonalisation: classical Gram-Schmidt applied
// twice against the whole basis.
// ====================================================================
template <typename T>
struct Lanczos {
    using C = cplx_t<T>;
    bloch_plan* pl;
    int n_bands, m, B;
    long long n3;
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

    C *Vb = nullptr, *Tmp = nullptr, *Bc = nullptr, *Xc = nullptr;
    double2 *d_part = nullptr, *d_h = nullptr, *d_Q = nullptr;
    int* d_nv = nullptr;
    long long *d_src = nullptr, *d_dst = nullptr;
    double* d_s = nullptr;
    int nblk = 0;

    struct Slot {
        int kidx = -1;
        double k[3];
        bool gamma = false;
        int n_eff = 0;
        int j = 0;
        int restarts = 0;
        std::vector<cd> H;   // (m+1) x m
    };
    std::vector<Slot> slots;
    int nact = 0;
    int nalloc = 0;   // buffers taken from the plan's pool 1
    template <typename X>
    bloch_status alloc(X** p, size_t n_el) {
        return plan_solver_buf(pl, 1, nalloc++, n_el * sizeof(X), (void**)p);
    }
    C* vb(int s, int i) const { return Vb + ((size_t)s * (m + 1) + i) * n3; }

    bloch_status setup() {
        bloch_status s;
        nblk = (int)std::max(1LL, std::min<long long>((n3 + 255) / 256, std::max(1, 1024 / std::max(1, B))));
        if ((s = alloc(&Vb, (size_t)B * (m + 1) * n3)) || (s = alloc(&Tmp, (size_t)m * n3)) ||
            (s = alloc(&Bc, (size_t)B * n3)) || (s = alloc(&Xc, (size_t)B * n3)) ||
            (s = alloc(&d_part, (size_t)B * nblk * (m + 1))) || (s = alloc(&d_h, (size_t)B * (m + 1))) ||
            (s = alloc(&d_Q, (size_t)m * m)) || (s = alloc(&d_nv, (size_t)B)) || (s = alloc(&d_src, (size_t)B)) ||
            (s = alloc(&d_dst, (size_t)B)) || (s = alloc(&d_s, (size_t)B)))
            return s;
        if ((s = ensure_cg<T>(pl, B)) != BLOCH_OK) return s;
        slots.assign(B, Slot());
        return BLOCH_OK;
    }

    bloch_status upload_ll(long long* d, const std::vector<long long>& h) {
        BLOCH_CUDA_CHECK_RET(
            cudaMemcpyAsync(d, h.data(), sizeof(long long) * h.size(), cudaMemcpyHostToDevice, pl->stream));
        return BLOCH_OK;
    }

    // M-norms of Xc[0..nact) -> host
    bloch_status xnorms(std::vector<double>& nrm) {
        Workspace<T>& w = ws_of<T>(pl);
        launch_dot<T>(pl, nact, Xc, Xc, n3, w.dots, w.part2);
        std::vector<double2> d(nact);
        BLOCH_CUDA_CHECK_RET(
            cudaMemcpyAsync(d.data(), w.dots, sizeof(double2) * nact, cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
        nrm.resize(nact);
        for (int i = 0; i < nact; ++i) nrm[i] = std::sqrt(std::max(0.0, rho_s * d[i].x));
        return BLOCH_OK;
    }

    bloch_status init_slot(int s, int kidx) {
        Slot& sl = slots[s];
        sl = Slot();
        sl.kidx = kidx;
        for (int a = 0; a < 3; ++a) sl.k[a] = (*klist)[kidx][a];
        sl.gamma = sl.k[0] == 0.0 && sl.k[1] == 0.0 && sl.k[2] == 0.0;
        sl.n_eff = sl.gamma ? n_bands - 3 : n_bands;
        sl.j = 0;
        sl.H.assign((size_t)(m + 1) * m, cd(0, 0));
        ++pl->launches;
        k_start_random<T><<<1024, 256, 0, pl->stream>>>(vb(s, 0), n3, pl->V, 12345ULL, sl.gamma ? 1 : 0);
        // normalise in the M norm
        Workspace<T>& w = ws_of<T>(pl);
        launch_dot<T>(pl, 1, vb(s, 0), vb(s, 0), n3, w.dots, w.part2);
        double2 d;
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(&d, w.dots, sizeof(double2), cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
        const double sc = 1.0 / std::sqrt(rho_s * d.x);
        ++pl->launches;
        k_scale<T><<<1024, 256, 0, pl->stream>>>(vb(s, 0), vb(s, 0), T(sc), (size_t)n3);
        return BLOCH_OK;
    }

    // Ritz analysis of a slot whose basis is full: converge (output) or restart.
    // Returns true when the slot is finished.
    bool ritz(int s, bloch_status& err) {
        Slot& sl = slots[s];
        std::vector<cd> Hm((size_t)m * m);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j)
                Hm[(size_t)i * m + j] = 0.5 * (sl.H[(size_t)i * m + j] + std::conj(sl.H[(size_t)j * m + i]));
        std::vector<double> w;
        std::vector<cd> Y;
        herm_jacobi(m, Hm, w, Y);
        const double beta = std::abs(sl.H[(size_t)m * m + (m - 1)]);
        // wanted: largest theta (descending)
        std::vector<int> idx(m);
        for (int i = 0; i < m; ++i) idx[i] = m - 1 - i;
        bool conv = true;
        for (int i = 0; i < sl.n_eff; ++i) {
            const double th = w[idx[i]];
            const double res = beta * std::abs(Y[(size_t)(m - 1) * m + idx[i]]);
            if (!(th > 0.0) || res > tol_eig * std::fabs(th)) conv = false;
        }
        sl.restarts += 1;
        const bool done = conv || sl.restarts > max_outer;
        const int kk = done ? (ritz_out ? std::min(m, q_out) : sl.n_eff)
                            : std::min(m - 1, sl.n_eff + (m - sl.n_eff) / 2);
        // Q: m x m, columns = the kept Ritz vectors (descending theta), rest zero
        std::vector<double2> Qh((size_t)m * m, make_double2(0, 0));
        for (int c = 0; c < kk; ++c)
            for (int i = 0; i < m; ++i) {
                const cd y = Y[(size_t)i * m + idx[c]];
                Qh[(size_t)i * m + c] = make_double2(y.real(), y.imag());
            }
        cudaError_t e = cudaMemcpyAsync(d_Q, Qh.data(), sizeof(double2) * Qh.size(), cudaMemcpyHostToDevice,
                                        pl->stream);
        if (e != cudaSuccess) {
            err = set_cuda_error(e, "Lanczos restart upload");
            return true;
        }
        ++pl->launches;
        launch_basis<T>(pl->stream, 1, vb(s, 0), Tmp, d_Q, m, n3);
        if (done) {
            const double lam_scale = pl->Kscale / pl->rho_ref;
            double* om = omega_out + (size_t)sl.kidx * n_bands;
            int b0 = 0;
            if (sl.gamma)
                for (; b0 < std::min(3, n_bands); ++b0) om[b0] = 0.0;
            // ascending lambda = descending theta = order of the kept columns
            for (int i = 0; i < sl.n_eff; ++i) {
                const double th = w[idx[i]];
                om[b0 + i] = th > 0 ? std::sqrt(lam_scale / th) : 0.0;
            }
            st->outer_iterations += sl.restarts;
            double mx = 0;
            for (int i = 0; i < sl.n_eff; ++i) {
                const double th = w[idx[i]];
                mx = std::max(mx, beta * std::abs(Y[(size_t)(m - 1) * m + idx[i]]) / std::max(std::fabs(th), 1e-300));
            }
            st->max_rel_residual = std::max(st->max_rel_residual, mx);
            if (!conv) {
                any_unconverged = true;
                if (!ritz_out) st->k_unconverged += 1;   // the hybrid's refinement decides for it
            }
            if (ritz_out) {
                size_t pos = 0;
                while (pos < order.size() && order[pos] != sl.kidx) ++pos;
                C* dst = ritz_out + pos * (size_t)q_out * n3;
                cudaMemcpyAsync(dst, Tmp, sizeof(C) * (size_t)kk * n3, cudaMemcpyDeviceToDevice, pl->stream);
                if (kk < q_out)
                    cudaMemsetAsync(dst + (size_t)kk * n3, 0, sizeof(C) * (size_t)(q_out - kk) * n3, pl->stream);
            }
            if (vecs_out) {
                C* out = (C*)vecs_out + (size_t)sl.kidx * n_bands * n3;
                const double nv = 1.0 / std::sqrt(pl->rho_ref);
                if (sl.gamma) {
                    cudaMemsetAsync(out, 0, sizeof(C) * std::min(3, n_bands) * n3, pl->stream);
                    std::vector<double2> one(1, make_double2(1.0 / std::sqrt(pl->rho_ref * rho_s), 0.0));
                    for (int c = 0; c < std::min(3, n_bands); ++c) {
                        const C cv = mk(T(one[0].x), T(0));
                        cudaMemcpyAsync(out + (size_t)c * n3 + (size_t)c * pl->V, &cv, sizeof(C),
                                        cudaMemcpyHostToDevice, pl->stream);
                        cudaStreamSynchronize(pl->stream);
                    }
                }
                ++pl->launches;
                k_scale<T><<<1024, 256, 0, pl->stream>>>(Tmp, out + (size_t)b0 * n3, T(nv), (size_t)sl.n_eff * n3);
            }
            cudaStreamSynchronize(pl->stream);
            return true;
        }
        // restart: V[0..kk) = V Y_kk, V[kk] = v_{m}; H = [diag(theta); b^T]
        cudaMemcpyAsync(vb(s, 0), Tmp, sizeof(C) * kk * n3, cudaMemcpyDeviceToDevice, pl->stream);
        cudaMemcpyAsync(vb(s, kk), vb(s, m), sizeof(C) * n3, cudaMemcpyDeviceToDevice, pl->stream);
        std::fill(sl.H.begin(), sl.H.end(), cd(0, 0));
        const cd bm = sl.H.size() ? cd(beta, 0) : cd(0, 0);
        for (int c = 0; c < kk; ++c) {
            sl.H[(size_t)c * m + c] = w[idx[c]];
            sl.H[(size_t)kk * m + c] = bm * Y[(size_t)(m - 1) * m + idx[c]];
        }
        sl.j = kk;
        return false;
    }

    bloch_status run() {
        bloch_status s;
        nact = 0;
        while (nact < B && next_k < order.size()) {
            if ((s = init_slot(nact, order[next_k++])) != BLOCH_OK) return s;
            ++nact;
        }
        while (nact > 0) {
            // gather v_j of every slot
            std::vector<long long> src(nact), dst(nact);
            std::vector<double> one(nact, 1.0);
            std::vector<int> nv(nact);
            for (int i = 0; i < nact; ++i) {
                src[i] = ((long long)i * (m + 1) + slots[i].j) * n3;
                dst[i] = (long long)i * n3;
                nv[i] = slots[i].j + 1;
            }
            if ((s = upload_ll(d_src, src)) || (s = upload_ll(d_dst, dst))) return s;
            BLOCH_CUDA_CHECK_RET(
                cudaMemcpyAsync(d_s, one.data(), sizeof(double) * nact, cudaMemcpyHostToDevice, pl->stream));
            BLOCH_CUDA_CHECK_RET(
                cudaMemcpyAsync(d_nv, nv.data(), sizeof(int) * nact, cudaMemcpyHostToDevice, pl->stream));
            dim3 gc(nblk, nact);
            ++pl->launches;
            k_copy_scaled<T><<<gc, 256, 0, pl->stream>>>(Vb, d_src, Bc, d_dst, d_s, n3);
            // w = A^-1 (M v_j)
            std::vector<double> kv((size_t)nact * 3);
            for (int i = 0; i < nact; ++i)
                for (int a = 0; a < 3; ++a) kv[(size_t)i * 3 + a] = slots[i].k[a];
            if ((s = set_k<T>(pl, nact, kv.data())) != BLOCH_OK) return s;
            if ((s = lp_activate<T>(pl, nact, 1, 1)) != BLOCH_OK) return s;
            long long cg_it = 0;
            pl->trace_pcg = TR_PCG_LZ;
            s = pcg_run<T>(pl, nact, Bc, Xc, rho_s, tol_lin, max_cg, false, nullptr, nullptr, &cg_it);
            pl->trace_pcg = TR_PCG_SUB;
            lp_deactivate(pl);
            st->cg_iterations += cg_it;
            st->k_applies += cg_it;
            st->linear_solves += nact;
            if (s != BLOCH_OK && s != BLOCH_ENOTCONV_CG) return s;
            // two passes of classical Gram-Schmidt in the M inner product
            const int tr_orth = trace_begin(pl, TR_ORTHO);
            std::vector<cd> hsum((size_t)nact * (m + 1), cd(0, 0));
            int maxnv = 0;
            for (int i = 0; i < nact; ++i) maxnv = std::max(maxnv, nv[i]);
            for (int pass = 0; pass < 2; ++pass) {
                dim3 gd(nblk, maxnv, nact);
                ++pl->launches;
                k_vdots<T><<<gd, 256, 0, pl->stream>>>(Vb, (long long)(m + 1) * n3, Xc, n3, d_nv, n3, maxnv, d_part);
                ++pl->launches;
                k_vdots_final<<<dim3(maxnv, nact), 256, 0, pl->stream>>>(d_part, nblk, maxnv, rho_s, d_h);
                dim3 ga(nblk, nact);
                ++pl->launches;
                k_vaxpy<T><<<ga, 256, 0, pl->stream>>>(Vb, (long long)(m + 1) * n3, Xc, n3, d_h, d_nv, n3, maxnv);
                std::vector<double2> hh((size_t)nact * maxnv);
                BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(hh.data(), d_h, sizeof(double2) * hh.size(),
                                                     cudaMemcpyDeviceToHost, pl->stream));
                BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
                for (int i = 0; i < nact; ++i)
                    for (int t = 0; t < nv[i]; ++t)
                        hsum[(size_t)i * (m + 1) + t] += cd(hh[(size_t)i * maxnv + t].x, hh[(size_t)i * maxnv + t].y);
            }
            std::vector<double> nrm;
            if ((s = xnorms(nrm)) != BLOCH_OK) return s;
            std::vector<double> inv(nact);
            for (int i = 0; i < nact; ++i) {
                Slot& sl = slots[i];
                for (int t = 0; t <= sl.j; ++t) sl.H[(size_t)t * m + sl.j] = hsum[(size_t)i * (m + 1) + t];
                sl.H[(size_t)(sl.j + 1) * m + sl.j] = nrm[i];
                inv[i] = nrm[i] > 0 ? 1.0 / nrm[i] : 0.0;
                src[i] = (long long)i * n3;
                dst[i] = ((long long)i * (m + 1) + sl.j + 1) * n3;
            }
            if ((s = upload_ll(d_src, src)) || (s = upload_ll(d_dst, dst))) return s;
            BLOCH_CUDA_CHECK_RET(
                cudaMemcpyAsync(d_s, inv.data(), sizeof(double) * nact, cudaMemcpyHostToDevice, pl->stream));
            ++pl->launches;
            k_copy_scaled<T><<<gc, 256, 0, pl->stream>>>(Xc, d_src, Vb, d_dst, d_s, n3);
            trace_end(pl, tr_orth);
            BLOCH_CUDA_CHECK_RET(cudaGetLastError());
            // advance; analyse full bases
            std::vector<int> finished;
            for (int i = 0; i < nact; ++i) {
                slots[i].j += 1;
                if (slots[i].j == m) {
                    bloch_status err = BLOCH_OK;
                    if (ritz(i, err)) finished.push_back(i);
                    if (err != BLOCH_OK) return err;
                }
            }
            if (!finished.empty()) {
                cudaStreamSynchronize(pl->stream);
                std::vector<char> hole(nact, 0);
                for (int f : finished) hole[f] = 1;
                for (int f : finished)
                    if (next_k < order.size()) {
                        if ((s = init_slot(f, order[next_k++])) != BLOCH_OK) return s;
                        hole[f] = 0;
                    }
                int last = nact - 1;
                for (int h = 0; h < nact; ++h) {
                    if (!hole[h]) continue;
                    while (last > h && hole[last]) --last;
                    if (last <= h) break;
                    const int nvv = slots[last].j + 1;
                    BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(vb(h, 0), vb(last, 0), sizeof(C) * nvv * n3,
                                                         cudaMemcpyDeviceToDevice, pl->stream));
                    slots[h] = slots[last];
                    hole[h] = 0;
                    hole[last] = 1;
                }
                int na = 0;
                for (int h = 0; h < nact; ++h)
                    if (!hole[h]) na = h + 1;
                nact = na;
            }
        }
        return BLOCH_OK;
    }
};

template <typename T>
static bloch_status run_lanczos(bloch_plan* pl, const std::vector<std::array<double, 3>>& ks, int n_bands,
                                double* omega_out, void* vecs_out, bloch_stats* st, cplx_t<T>* ritz_out = nullptr,
                                int q_out = 0, double tol_override = 0.0) {
    if (!pl->uniform_rho)
        return set_error(BLOCH_EUNSUPPORTED, "the Lanczos solver needs a uniform density (use subspace iteration)");
    Lanczos<T> S;
    S.pl = pl;
    S.n3 = 3 * pl->V;
    S.n_bands = n_bands;
    S.m = pl->opt.ncv > 0 ? pl->opt.ncv : std::max(2 * n_bands + 1, 20);
    S.m = (int)std::min<long long>(S.m, 3 * pl->V - 4);
    if (S.m > kBasisQMax - 1)
        return set_error(BLOCH_EUNSUPPORTED, "Lanczos basis above 63 vectors is not supported");
    if (S.m < n_bands + 1) return set_error(BLOCH_EINVAL, "Lanczos basis too small for the requested bands");
    S.rho_s = pl->rho_uniform_scaled;
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
    freeb += plan_solver_bytes(pl);   // held by the plan from earlier solves, reused
    const size_t per_slot = (size_t)(S.m + 1 + 2 + 5) * S.n3 * sizeof(cplx_t<T>);
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
    if (pl->opt.method == BLOCH_SUBSPACE) {
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
