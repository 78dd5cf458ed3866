// Learned Fourier-space preconditioner: device functions shared by the
// training kernels and the inference table.
//
//   Z(q) = sum_a g_a v_a v_a^T / mu_a,  P(q) = C0 : q q = sum_a mu_a v_a v_a^T,
//   g_a = softplus(MLP(f_a)),  f_a = (qh_x^2, qh_y^2, qh_z^2, mu_a/|q|^2, s),
//   s = log(1 + |q|) / log(1 + N/2)        (scaled units: q in 2 pi / L)
// Parameters (flat): W1 (H x 5), b1 (H), W2 (H x H), b2 (H), w3 (H), b3.
#pragma once

#include "common.cuh"
#include "vec.cuh"

namespace bloch {

constexpr int kLPF = 5;

__host__ __device__ constexpr int lp_nparams(int H) { return H * kLPF + H + H * H + H + H + 1; }

// Cyclic Jacobi on a symmetric 3x3 matrix (6 sweeps: converged to roundoff
// for 3x3).  Eigenvalues unsorted; columns of V are the eigenvectors.
template <typename T>
__device__ __forceinline__ void sym3_eig(T A[3][3], T mu[3], T V[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) V[i][j] = i == j ? T(1) : T(0);
#pragma unroll
    for (int sweep = 0; sweep < 6; ++sweep) {
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {
            const int p = pr == 2 ? 1 : 0;
            const int r = pr == 0 ? 1 : 2;
            const T apr = A[p][r];
            if (apr != T(0)) {
                const T th = (A[r][r] - A[p][p]) / (T(2) * apr);
                const T t = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
                const T c = T(1) / sqrt(t * t + T(1));
                const T s = t * c;
#pragma unroll
                for (int k = 0; k < 3; ++k) {   // A <- A J
                    const T akp = A[k][p], akr = A[k][r];
                    A[k][p] = c * akp - s * akr;
                    A[k][r] = s * akp + c * akr;
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {   // A <- J^T A
                    const T apk = A[p][k], ark = A[r][k];
                    A[p][k] = c * apk - s * ark;
                    A[r][k] = s * apk + c * ark;
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {   // V <- V J
                    const T vkp = V[k][p], vkr = V[k][r];
                    V[k][p] = c * vkp - s * vkr;
                    V[k][r] = s * vkp + c * vkr;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) mu[i] = A[i][i];
}

// P(q) from the scaled C0 monomial coefficients (same as the Green preconditioner)
template <typename T>
__device__ __forceinline__ void acoustic3(const PrecondCoef& pc, T qx, T qy, T qz, T P[3][3]) {
    const T m[6] = {qx * qx, qy * qy, qz * qz, qy * qz, qx * qz, qx * qy};
    T p6[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        T s = 0;
#pragma unroll
        for (int j = 0; j < 6; ++j) s = fma(pcoef<T>(pc, i, j), m[j], s);
        p6[i] = s;
    }
    P[0][0] = p6[0];
    P[1][1] = p6[1];
    P[2][2] = p6[2];
    P[1][2] = P[2][1] = p6[3];
    P[0][2] = P[2][0] = p6[4];
    P[0][1] = P[1][0] = p6[5];
}

__device__ __forceinline__ float lp_softplus(float o) { return o > 20.f ? o : log1pf(expf(o)); }
__device__ __forceinline__ float lp_sigmoid(float o) { return 1.f / (1.f + expf(-o)); }

// MLP forward for one feature vector; returns the output pre-activation and
// (optionally) the hidden activations.
template <int H>
__device__ __forceinline__ float lp_forward(const float* __restrict__ prm, const float f[kLPF], float h1[H],
                                            float h2[H]) {
    const float* W1 = prm;
    const float* b1 = W1 + H * kLPF;
    const float* W2 = b1 + H;
    const float* b2 = W2 + H * H;
    const float* w3 = b2 + H;
    const float b3 = w3[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        float z = b1[i];
#pragma unroll
        for (int j = 0; j < kLPF; ++j) z = fmaf(W1[i * kLPF + j], f[j], z);
        h1[i] = tanhf(z);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
        float z = b2[i];
#pragma unroll
        for (int j = 0; j < H; ++j) z = fmaf(W2[i * H + j], h1[j], z);
        h2[i] = tanhf(z);
    }
    float o = b3;
#pragma unroll
    for (int j = 0; j < H; ++j) o = fmaf(w3[j], h2[j], o);
    return o;
}

// Learned Z at one scaled wave vector (sym 6: xx, yy, zz, yz, xz, xy); zero at q = 0.
template <int H>
__device__ __forceinline__ void lp_Z(const float* __restrict__ prm, const PrecondCoef& pc, float snorm, float qx,
                                     float qy, float qz, float Z[6]) {
    const float qn2 = qx * qx + qy * qy + qz * qz;
    if (qn2 == 0.f) {
#pragma unroll
        for (int i = 0; i < 6; ++i) Z[i] = 0.f;
        return;
    }
    float P[3][3], mu[3], Vv[3][3];
    acoustic3<float>(pc, qx, qy, qz, P);
    sym3_eig<float>(P, mu, Vv);
    const float iq = 1.f / qn2;
    const float s = log1pf(sqrtf(qn2)) * snorm;
    float w[3];
#pragma unroll 1
    for (int a = 0; a < 3; ++a) {
        asm volatile("" ::: "memory");   // keep the weight loads inside the branch loop
        const float mua = a == 0 ? mu[0] : (a == 1 ? mu[1] : mu[2]);
        const float f[kLPF] = {qx * qx * iq, qy * qy * iq, qz * qz * iq, mua * iq, s};
        float h1[H], h2[H];
        const float wa = lp_softplus(lp_forward<H>(prm, f, h1, h2)) / mua;
        if (a == 0) w[0] = wa; else if (a == 1) w[1] = wa; else w[2] = wa;
    }
    const int ii[6] = {0, 1, 2, 1, 0, 0}, jj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        float z = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) z = fmaf(w[a] * Vv[ii[t]][a], Vv[jj[t]][a], z);
        Z[t] = z;
    }
}

}  // namespace bloch
