// Properties of computed bands: group velocity (Section 5.1, Eq. c_group)
// by the Hellmann-Feynman identity, and real-space eigenvector fields with
// their strain (Section 5.2, Eq. rotate_eigenvector).
//
// For an eigenpair A_k u = lambda M u (M independent of k):
//   d lambda / d k_m = u^H (dA_k/dk_m) u / u^H M u,
// and from the component form of Eq. (hatA), with q = xi + k, dq_j/dk_m = delta_jm,
// the stress field sigma = C(x) : F^-1(sym q (x) U) and S = F{sigma}:
//   u^H A_k u          = sum_xi conj(U_i) q_j S_ij,
//   u^H (dA_k/dk_m) u  = 2 Re sum_xi conj(U_i) S_im      (major symmetry of C).
// So one pass chain -- the K-apply's passes 1-4 and a forward z transform of
// the six stress components -- and one reduction give lambda (the Rayleigh
// quotient) and its gradient; d omega/d k = (d lambda/d k) / (2 omega).
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace bloch {

constexpr int kDkVals = 9;   // d_x (re, im), d_y, d_z, a (re, im), u^H M~ u

// Per system b = blockIdx.y, per block: partial sums over Fourier voxels of
//   d_m = sum_i conj(U_i) S_im,  a = sum_ij conj(U_i) q_j S_ij,  mu = Re sum conj(U) (M~ U)
// with M~ U = MU (non-uniform density) or rho_s U.  FP64 accumulation.
template <typename T>
__global__ void k_dk_partial(const cplx_t<T>* __restrict__ U, const cplx_t<T>* __restrict__ S,
                             const cplx_t<T>* __restrict__ MU, double rho_s, const T* __restrict__ qtab, Geo g,
                             double* __restrict__ partial) {
    using C = cplx_t<T>;
    const int b = blockIdx.y;
    const C* ub = U + (size_t)b * 3 * g.V;
    const C* sb = S + (size_t)b * 6 * g.V;
    const C* mb = MU ? MU + (size_t)b * 3 * g.V : nullptr;
    const T* qb = qtab + (size_t)b * (g.Nx + g.Ny + g.Nz);
    // Voigt index of S_im: rows i = x, y, z; columns m = x, y, z
    const int vo[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    double acc[kDkVals];
#pragma unroll
    for (int i = 0; i < kDkVals; ++i) acc[i] = 0.0;
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
        T qx, qy, qz;
        voxel_q(qb, g, v, qx, qy, qz);
        const double q[3] = {(double)qx, (double)qy, (double)qz};
        C u[3], s[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = ub[(size_t)c * g.V + v];
#pragma unroll
        for (int c = 0; c < 6; ++c) s[c] = sb[(size_t)c * g.V + v];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const double ur = (double)u[i].x, ui = (double)u[i].y;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const C sv = s[vo[i][m]];
                const double pr = ur * (double)sv.x + ui * (double)sv.y;   // Re conj(u) s
                const double pim = ur * (double)sv.y - ui * (double)sv.x;  // Im conj(u) s
                acc[2 * m] += pr;
                acc[2 * m + 1] += pim;
                acc[6] += q[m] * pr;
                acc[7] += q[m] * pim;
            }
            if (mb) {
                const C mv = mb[(size_t)i * g.V + v];
                acc[8] += ur * (double)mv.x + ui * (double)mv.y;
            } else {
                acc[8] += rho_s * (ur * ur + ui * ui);
            }
        }
    }
    block_sum<double, kDkVals>(acc);
    if (threadIdx.x == 0) {
        double* o = partial + ((size_t)b * gridDim.x + blockIdx.x) * kDkVals;
#pragma unroll
        for (int i = 0; i < kDkVals; ++i) o[i] = acc[i];
    }
}

template <typename T>
static bloch_status group_velocity_impl(bloch_plan* pl, int nb, const double* k, const cplx_t<T>* u,
                                        double* omega_out, double* c_out) {
    bloch_status st = ensure_cg<T>(pl, nb);
    if (st != BLOCH_OK) return st;
    if ((st = set_k<T>(pl, nb, k)) != BLOCH_OK) return st;
    Workspace<T>& w = ws_of<T>(pl);
    // M u first: the mass operator's passes use the same workspace E that
    // then holds the stress field
    const cplx_t<T>* MU = nullptr;
    if (!pl->uniform_rho) {
        launch_M<T>(pl, nb, u, w.Ap, T(1));
        MU = w.Ap;
    }
    launch_K_stress<T>(pl, nb, u);
    const int nblk = (int)std::max(1LL, std::min<long long>((pl->V + 255) / 256, 512));
    const size_t nval = (size_t)nb * nblk * kDkVals;
    double* d_part = nullptr;
    if ((st = plan_solver_buf(pl, 2, 0, nval * sizeof(double), (void**)&d_part)) != BLOCH_OK) return st;
    ++pl->launches;
    k_dk_partial<T><<<dim3(nblk, nb), 256, 0, pl->stream>>>(u, w.E, MU, pl->uniform_rho ? pl->rho_uniform_scaled : 1.0,
                                                            w.qtab, geo_of<T>(pl), d_part);
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    std::vector<double> h(nval);
    BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(h.data(), d_part, nval * sizeof(double), cudaMemcpyDeviceToHost, pl->stream));
    BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
    for (int b = 0; b < nb; ++b) {
        double s[kDkVals] = {0};
        for (int j = 0; j < nblk; ++j)
            for (int i = 0; i < kDkVals; ++i) s[i] += h[((size_t)b * nblk + j) * kDkVals + i];
        const double uMu = pl->rho_ref * s[8];   // u^H M u (SI)
        if (!(uMu > 0.0)) return set_error(BLOCH_EINVAL, "a vector is zero (u^H M u = 0)");
        const double lam = pl->Kscale * s[6] / uMu;
        const double om = lam > 0.0 ? std::sqrt(lam) : 0.0;
        if (omega_out) omega_out[b] = om;
        for (int m = 0; m < 3; ++m) {
            const double dlam = pl->Kscale * pl->qscale * 2.0 * s[2 * m] / uMu;
            c_out[(size_t)b * 3 + m] = om > 0.0 ? dlam / (2.0 * om) : 0.0;
        }
    }
    return BLOCH_OK;
}

// ------------------------------------------------ real-space eigenvectors
// Eq. (rotate_eigenvector): U(x) = e^{-i phi} F^-1(U^).  The paper takes phi
// as the one phase shared by every point of the field; phi = arg(s)/2 with
// s = sum_x sum_i U_i(x)^2 is that phase (mod pi) whenever the field has a
// single phase, and otherwise the single phase that maximises
// ||Re(e^{-i phi} U)|| (least squares).

// partial[b][blk] = sum over the block's elements of W^2 (complex square)
template <typename T>
__global__ void k_sq_partial(const cplx_t<T>* __restrict__ W, long long n_per, double2* __restrict__ partial) {
    const int b = blockIdx.y;
    const cplx_t<T>* w = W + (size_t)b * n_per;
    double acc[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_per;
         i += (long long)gridDim.x * blockDim.x) {
        const double a = (double)w[i].x, c = (double)w[i].y;
        acc[0] += a * a - c * c;
        acc[1] += 2.0 * a * c;
    }
    block_sum<double, 2>(acc);
    if (threadIdx.x == 0) partial[(size_t)b * gridDim.x + blockIdx.x] = make_double2(acc[0], acc[1]);
}

// W[b] *= ph[b] (complex)
template <typename T>
__global__ void k_phase(cplx_t<T>* W, long long n_per, const double2* __restrict__ ph) {
    const int b = blockIdx.y;
    const cplx_t<T> p = mk(T(ph[b].x), T(ph[b].y));
    cplx_t<T>* w = W + (size_t)b * n_per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_per;
         i += (long long)gridDim.x * blockDim.x)
        w[i] = cmul(w[i], p);
}

// Fourier-space strain of the periodic field, eps_ij = (d_j U_i + d_i U_j)/2 with
// d_j = i xi_j (the derivative of Section 5.2's epsilon_11 = dU_1/dx_1), times
// the phase ph[b]; Voigt-ordered tensor components (xx yy zz yz xz xy).
// xi from the q table of a zero wave vector (scaled by qscale; s = 1/qscale).
template <typename T>
__global__ void k_strain_hat(const cplx_t<T>* __restrict__ U, const T* __restrict__ xitab, Geo g,
                             const double2* __restrict__ ph, T s, cplx_t<T>* __restrict__ Eps) {
    using C = cplx_t<T>;
    const int b = blockIdx.y;
    const C p = mk(T(ph[b].x), T(ph[b].y));
    const C* ub = U + (size_t)b * 3 * g.V;
    C* eb = Eps + (size_t)b * 6 * g.V;
    for (unsigned v = blockIdx.x * blockDim.x + threadIdx.x; v < (unsigned)g.V; v += gridDim.x * blockDim.x) {
        T x0, x1, x2;
        voxel_q(xitab, g, v, x0, x1, x2);
        const T xi[3] = {x0 * s, x1 * s, x2 * s};
        C u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) u[c] = cmul(ub[(size_t)c * g.V + v], p);
        const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int i = pi[c], j = pj[c];
            // (i xi_j u_i + i xi_i u_j) / 2
            const C a = cadd(cscale(u[i], xi[j]), cscale(u[j], xi[i]));
            eb[(size_t)c * g.V + v] = cscale(cmul_i<+1>(a), T(0.5));
        }
    }
}

template <typename T>
static bloch_status eigvec_real_impl(bloch_plan* pl, int nb, const cplx_t<T>* uh, cplx_t<T>* ur, cplx_t<T>* eps,
                                     double* phi_out) {
    using C = cplx_t<T>;
    bloch_status st = ensure_ws<T>(pl, nb);
    if (st != BLOCH_OK) return st;
    const long long n3 = 3 * pl->V;
    BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(ur, uh, sizeof(C) * (size_t)nb * n3, cudaMemcpyDeviceToDevice, pl->stream));
    launch_fft3<T, +1>(pl, nb, ur, T(1.0 / (double)pl->V));       // F^-1 (numpy normalisation)
    const int nblk = (int)std::max(1LL, std::min<long long>((n3 + 255) / 256, 512));
    double2* d_part = nullptr;
    if ((st = plan_solver_buf(pl, 2, 1, sizeof(double2) * ((size_t)nb * nblk + nb), (void**)&d_part)) != BLOCH_OK)
        return st;
    double2* d_ph = d_part + (size_t)nb * nblk;
    ++pl->launches;
    k_sq_partial<T><<<dim3(nblk, nb), 256, 0, pl->stream>>>(ur, n3, d_part);
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    std::vector<double2> h((size_t)nb * nblk);
    BLOCH_CUDA_CHECK_RET(
        cudaMemcpyAsync(h.data(), d_part, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, pl->stream));
    BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
    std::vector<double2> ph(nb);
    for (int b = 0; b < nb; ++b) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < nblk; ++j) {
            re += h[(size_t)b * nblk + j].x;
            im += h[(size_t)b * nblk + j].y;
        }
        const double phi = 0.5 * std::atan2(im, re);
        if (phi_out) phi_out[b] = phi;
        ph[b] = make_double2(std::cos(phi), -std::sin(phi));   // e^{-i phi}
    }
    BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(d_ph, ph.data(), sizeof(double2) * nb, cudaMemcpyHostToDevice, pl->stream));
    const unsigned gx = (unsigned)std::min<long long>((n3 + 255) / 256, 2048);
    ++pl->launches;
    k_phase<T><<<dim3(gx, nb), 256, 0, pl->stream>>>(ur, n3, d_ph);
    if (eps) {
        std::vector<double> zero((size_t)nb * 3, 0.0);
        if ((st = set_k<T>(pl, nb, zero.data())) != BLOCH_OK) return st;
        const unsigned gv = (unsigned)std::min<long long>((pl->V + 255) / 256, 2048);
        ++pl->launches;
        k_strain_hat<T><<<dim3(gv, nb), 256, 0, pl->stream>>>(uh, ws_of<T>(pl).qtab, geo_of<T>(pl), d_ph,
                                                               T(1.0 / pl->qscale), eps);
        launch_fft3<T, +1>(pl, 2 * nb, eps, T(1.0 / (double)pl->V));   // six components = two 3-component fields
    }
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
    return BLOCH_OK;
}

}  // namespace bloch

using namespace bloch;

extern "C" bloch_status bloch_eigvec_real(bloch_plan* pl, int32_t nb, int32_t precision, const void* u_hat,
                                          void* u_real, void* strain, double* phi_out) {
    if (!pl) return set_error(BLOCH_EINVAL, "plan is NULL");
    if (nb < 1 || 2 * nb > 65535 / 3) return set_error(BLOCH_EINVAL, "nb must be in [1, 10922]");
    if (precision != BLOCH_FP32 && precision != BLOCH_FP64)
        return set_error(BLOCH_EINVAL, "precision must be BLOCH_FP32 or BLOCH_FP64");
    if (!u_hat || !u_real) return set_error(BLOCH_EINVAL, "NULL argument");
    if (u_hat == u_real || u_hat == strain) return set_error(BLOCH_EINVAL, "outputs may not alias u_hat");
    if (precision == BLOCH_FP32)
        return eigvec_real_impl<float>(pl, nb, (const float2*)u_hat, (float2*)u_real, (float2*)strain, phi_out);
    return eigvec_real_impl<double>(pl, nb, (const double2*)u_hat, (double2*)u_real, (double2*)strain, phi_out);
}

extern "C" bloch_status bloch_group_velocity(bloch_plan* pl, int32_t nb, const double* k, int32_t precision,
                                             const void* u, double* omega_out, double* c_out) {
    if (!pl) return set_error(BLOCH_EINVAL, "plan is NULL");
    if (nb < 1 || nb > 65535 / 6) return set_error(BLOCH_EINVAL, "nb must be in [1, 10922]");
    if (precision != BLOCH_FP32 && precision != BLOCH_FP64)
        return set_error(BLOCH_EINVAL, "precision must be BLOCH_FP32 or BLOCH_FP64");
    if (!k || !u || !c_out) return set_error(BLOCH_EINVAL, "NULL argument");
    bloch_status st;
    if (precision == BLOCH_FP32)
        st = group_velocity_impl<float>(pl, nb, k, (const float2*)u, omega_out, c_out);
    else
        st = group_velocity_impl<double>(pl, nb, k, (const double2*)u, omega_out, c_out);
    if (st != BLOCH_OK) return st;
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    return BLOCH_OK;
}
