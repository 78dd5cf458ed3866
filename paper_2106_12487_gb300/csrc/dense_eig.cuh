// Small dense Hermitian eigenproblems on the device, FP64, one CTA per
// matrix (the projected problems of Algorithm 1, step EIG(K, M), and the
// Ritz problems of the Lanczos restarts), so the eigensolver loops need no
// host round trip.
//
// Standard problem: cyclic complex Jacobi.  Each rotation W (acting on rows
// and columns p < r) zeroes A[p][r]: with A[p][r] = |a| e^{i phi},
//   tau = (A_rr - A_pp) / (2 |a|),  t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
//   c = 1 / sqrt(1 + t^2),  s = t c,
//   W_pp = c, W_pr = s, W_rp = -s e^{-i phi}, W_rr = c e^{-i phi},
// A <- W^H A W, V <- V W.  One thread forms the rotation, the CTA's threads
// update the two columns and then the two rows in parallel.  Sweeps stop when
// the off-diagonal mass is below 1e-32 of the total (or after kJacMaxSweeps).
//
// Generalised problem K Q = M Q diag(lam), Q^H M Q = I: Cholesky M = L L^H,
// C = L^-1 K L^-H, Jacobi on C, Q = L^-H W.  Eigenvalues ascending.
#pragma once

#include "common.cuh"

namespace bloch {

constexpr int kJacMaxSweeps = 40;

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Jacobi on the n x n Hermitian A (shared memory, row-major, destroyed); V
// (shared, n x n) receives the eigenvectors in columns, w (shared, n) the
// eigenvalues, both unsorted.  Parallel ordering: each round applies n'/2
// disjoint rotations at once (n' = n rounded up to even; the pairs of a round
// come from the circle method -- index n'-1 fixed, the others rotating -- so
// n' - 1 rounds cover every pair once per sweep; pairs with the padding index
// are skipped).  Rotation parameters are formed from A at the start of the
// round, then all column updates (A W, V W), then all row updates (W^H A).
// red: shared scratch of 2 * blockDim.x doubles; rot: shared scratch of
// 5 * (n'/2) double2.  Returns true when converged.
__host__ __device__ constexpr int jacobi_rot_slots(int n) { return 5 * ((n + 1) / 2); }

static __device__ __forceinline__ void round_pair(int np, int rd, int i, int& p, int& r) {
    const int c = np - 1;   // the fixed index
    if (i == 0) {
        p = rd;
        r = c;
    } else {
        p = (rd + i) % c;
        r = (rd - i + c) % c;
    }
}

static __device__ bool jacobi_herm(int n, double2* A, double2* V, double* w, double* red, double2* rot) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int np = n + (n & 1);
    const int half = np / 2;
    for (int e = tid; e < n * n; e += nt) V[e] = make_double2((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    bool conv = n < 2;
    for (int sweep = 0; sweep < kJacMaxSweeps && !conv; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < n * n; e += nt) {
            const double a2 = zabs2(A[e]);
            tot += a2;
            if (e / n != e % n) off += a2;
        }
        red[tid] = off;
        red[nt + tid] = tot;
        __syncthreads();
        for (int s = nt / 2; s > 0; s >>= 1) {
            if (tid < s) {
                red[tid] += red[tid + s];
                red[nt + tid] += red[nt + tid + s];
            }
            __syncthreads();
        }
        const double offs = red[0], tots = red[nt];
        __syncthreads();
        if (offs <= 1e-32 * tots || tots == 0.0) {
            conv = true;
            break;
        }
        for (int rd = 0; rd < np - 1; ++rd) {
            // rotation parameters of the round's pairs (W_pp, W_pr, W_rp, W_rr, skip)
            for (int i = tid; i < half; i += nt) {
                int p, r;
                round_pair(np, rd, i, p, r);
                double2* R = rot + 5 * i;
                double skip = 1.0;
                if (p < n && r < n) {
                    const double2 apr = A[p * n + r];
                    const double mag = sqrt(zabs2(apr));
                    const double app = A[p * n + p].x, arr = A[r * n + r].x;
                    if (mag != 0.0 && (mag < 1e-300 || mag <= 1e-21 * sqrt(fabs(app * arr)))) {
                        A[p * n + r] = A[r * n + p] = make_double2(0.0, 0.0);   // negligible: drop it
                    } else if (mag != 0.0) {
                        skip = 0.0;
                        const double2 em = make_double2(apr.x / mag, -apr.y / mag);   // e^{-i phi}
                        const double tau = (arr - app) / (2.0 * mag);
                        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                        R[0] = make_double2(c, 0.0);
                        R[1] = make_double2(s, 0.0);
                        R[2] = make_double2(-s * em.x, -s * em.y);
                        R[3] = make_double2(c * em.x, c * em.y);
                    }
                }
                R[4] = make_double2(skip, 0.0);
            }
            __syncthreads();
            for (int e = tid; e < half * n; e += nt) {   // A <- A W, V <- V W (columns of every pair)
                const int i = e / n, row = e - i * n;
                const double2* R = rot + 5 * i;
                if (R[4].x != 0.0) continue;
                int p, r;
                round_pair(np, rd, i, p, r);
                const double2 aip = A[row * n + p], air = A[row * n + r];
                A[row * n + p] = zadd(zmul(aip, R[0]), zmul(air, R[2]));
                A[row * n + r] = zadd(zmul(aip, R[1]), zmul(air, R[3]));
                const double2 vip = V[row * n + p], vir = V[row * n + r];
                V[row * n + p] = zadd(zmul(vip, R[0]), zmul(vir, R[2]));
                V[row * n + r] = zadd(zmul(vip, R[1]), zmul(vir, R[3]));
            }
            __syncthreads();
            for (int e = tid; e < half * n; e += nt) {   // A <- W^H A (rows of every pair)
                const int i = e / n, col = e - i * n;
                const double2* R = rot + 5 * i;
                if (R[4].x != 0.0) continue;
                int p, r;
                round_pair(np, rd, i, p, r);
                const double2 apj = A[p * n + col], arj = A[r * n + col];
                A[p * n + col] = zadd(zmul(zconj(R[0]), apj), zmul(zconj(R[2]), arj));
                A[r * n + col] = zadd(zmul(zconj(R[1]), apj), zmul(zconj(R[3]), arj));
            }
            __syncthreads();
            for (int i = tid; i < half; i += nt) {   // a rotated pair is exactly decoupled
                if (rot[5 * i + 4].x != 0.0) continue;
                int p, r;
                round_pair(np, rd, i, p, r);
                A[p * n + r] = A[r * n + p] = make_double2(0.0, 0.0);
                A[p * n + p].y = 0.0;
                A[r * n + r].y = 0.0;
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < n; i += nt) w[i] = A[i * n + i].x;
    __syncthreads();
    return conv;
}

// perm[0..n) = indices of w in ascending order (stable), thread 0
static __device__ void sort_ascending(int n, const double* w, int* perm) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int i = 1; i < n; ++i) {
            const int pi = perm[i];
            int j = i - 1;
            while (j >= 0 && w[perm[j]] > w[pi]) {
                perm[j + 1] = perm[j];
                --j;
            }
            perm[j + 1] = pi;
        }
    }
    __syncthreads();
}

// Shared memory of k_gen_herm_eig for order n, in this order (16-byte
// aligned double2 first): four n x n double2 matrices, the rotation slots
// (jacobi_rot_slots(n) double2), n doubles, 2 * nthreads doubles of
// reductions, n ints.
__host__ __device__ constexpr size_t gen_eig_smem(int n, int nthreads) {
    return (size_t)4 * n * n * sizeof(double2) + (size_t)jacobi_rot_slots(n) * sizeof(double2) +
           (size_t)n * sizeof(double) + (size_t)2 * nthreads * sizeof(double) + (size_t)n * sizeof(int);
}

// Batched generalised problems, one per blockIdx.x: K, M (n x n row-major
// double2, Hermitised here) at K + b*n*n, M + b*n*n (M scaled by mscale);
// out: lam[b][n] ascending, Q[b] (n x n row-major, eigenvectors in columns,
// Q^H M Q = I); status[b] = 0 ok, 1 M not positive definite, 2 Jacobi did not
// converge.
static __global__ void k_gen_herm_eig(int n, const double2* __restrict__ K, const double2* __restrict__ M, double mscale,
                               double* __restrict__ lam, double2* __restrict__ Q, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* A = reinterpret_cast<double2*>(smem_raw);
    double2* L = A + n * n;
    double2* X = L + n * n;
    double2* W = X + n * n;
    double2* rot = W + n * n;
    double* w = reinterpret_cast<double*>(rot + jacobi_rot_slots(n));
    double* red = w + n;
    int* perm = reinterpret_cast<int*>(red + 2 * blockDim.x);
    __shared__ int bad;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int b = blockIdx.x;
    const double2* Kb = K + (size_t)b * n * n;
    const double2* Mb = M + (size_t)b * n * n;
    for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, j = e % n;
        const double2 k1 = Kb[i * n + j], k2 = Kb[j * n + i];
        A[e] = make_double2(0.5 * (k1.x + k2.x), 0.5 * (k1.y - k2.y));
        const double2 m1 = Mb[i * n + j], m2 = Mb[j * n + i];
        X[e] = make_double2(0.5 * mscale * (m1.x + m2.x), 0.5 * mscale * (m1.y - m2.y));   // Hermitian part of M
        L[e] = make_double2(0.0, 0.0);
    }
    if (tid == 0) bad = 0;
    __syncthreads();
    // Cholesky M = L L^H (lower), serial: n <= 32 in Algorithm 1
    if (tid == 0) {
        for (int i = 0; i < n && !bad; ++i)
            for (int j = 0; j <= i; ++j) {
                double2 s = X[i * n + j];
                for (int k = 0; k < j; ++k) s = zsub(s, zmul(L[i * n + k], zconj(L[j * n + k])));
                if (i == j) {
                    if (!(s.x > 0.0)) {
                        bad = 1;
                        break;
                    }
                    L[i * n + i] = make_double2(sqrt(s.x), 0.0);
                } else {
                    const double d = L[j * n + j].x;
                    L[i * n + j] = make_double2(s.x / d, s.y / d);
                }
            }
    }
    __syncthreads();
    if (bad) {
        if (tid == 0) status[b] = 1;
        return;
    }
    // X = L^-1 A (columns in parallel)
    for (int c = tid; c < n; c += nt)
        for (int i = 0; i < n; ++i) {
            double2 s = A[i * n + c];
            for (int k = 0; k < i; ++k) s = zsub(s, zmul(L[i * n + k], X[k * n + c]));
            const double d = L[i * n + i].x;
            X[i * n + c] = make_double2(s.x / d, s.y / d);
        }
    __syncthreads();
    // Y = L^-1 X^H into W; then C = Y^H into A (Hermitised)
    for (int c = tid; c < n; c += nt)
        for (int i = 0; i < n; ++i) {
            double2 s = zconj(X[c * n + i]);
            for (int k = 0; k < i; ++k) s = zsub(s, zmul(L[i * n + k], W[k * n + c]));
            const double d = L[i * n + i].x;
            W[i * n + c] = make_double2(s.x / d, s.y / d);
        }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, j = e % n;
        const double2 c1 = zconj(W[j * n + i]), c2 = zconj(W[i * n + j]);   // C_ij and conj(C_ji)
        A[e] = make_double2(0.5 * (c1.x + c2.x), 0.5 * (c1.y - c2.y));
    }
    __syncthreads();
    const bool conv = jacobi_herm(n, A, W, w, red, rot);
    // Q = L^-H W (columns in parallel) into X
    for (int c = tid; c < n; c += nt)
        for (int i = n - 1; i >= 0; --i) {
            double2 s = W[i * n + c];
            for (int k = i + 1; k < n; ++k) s = zsub(s, zmul(zconj(L[k * n + i]), X[k * n + c]));
            const double d = L[i * n + i].x;
            X[i * n + c] = make_double2(s.x / d, s.y / d);
        }
    __syncthreads();
    sort_ascending(n, w, perm);
    for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, j = e % n;
        Q[(size_t)b * n * n + e] = X[i * n + perm[j]];
    }
    for (int j = tid; j < n; j += nt) lam[(size_t)b * n + j] = w[perm[j]];
    if (tid == 0) status[b] = conv ? 0 : 2;
}

// Rank-revealing Rayleigh-Ritz of a pencil (K, M) whose M may be singular
// (SVQB, Stathopoulos & Wu 2002): the basis is first scaled to unit M-norm,
// s_i = M_ii^-1/2 (0 for a zero column), M' = S M S, K' = S K S; then
// M' = V D V^H (Jacobi), the directions with D > eps * max(D) are kept,
// Z = V_keep D_keep^-1/2 (M'-orthonormal), C = Z^H K' Z = Y diag(lam) Y^H
// (Jacobi) and the Ritz vectors in the original coordinates are Q = S Z Y.  One CTA per pencil (blockIdx.x); K, M, Q n x n
// row-major (double2) at b * n * n; M scaled by mscale.  Out: lam[b][0..r)
// ascending, Q[b] columns 0..r (the rest zero), rank[b] = r.  Shared memory:
// gen_eig_smem(n, blockDim.x).
static __global__ void k_svqb_eig(int n, const double2* __restrict__ K, const double2* __restrict__ M, double mscale,
                                  double eps, double* __restrict__ lam, double2* __restrict__ Q,
                                  int* __restrict__ rank) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* A = reinterpret_cast<double2*>(smem_raw);   // M, then C
    double2* Vm = A + n * n;                            // eigenvectors of M, then Z
    double2* Kh = Vm + n * n;
    double2* Y = Kh + n * n;
    double2* rot = Y + n * n;
    double* w = reinterpret_cast<double*>(rot + jacobi_rot_slots(n));
    double* red = w + n;
    int* perm = reinterpret_cast<int*>(red + 2 * blockDim.x);
    __shared__ int r_sh;
    __shared__ double dmax_sh;
    __shared__ double sc[64];   // s_i (n <= 64)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int b = blockIdx.x;
    const double2* Kb = K + (size_t)b * n * n;
    const double2* Mb = M + (size_t)b * n * n;
    for (int i = tid; i < n; i += nt) {
        const double d = mscale * Mb[i * n + i].x;
        sc[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, j = e % n;
        const double sij = sc[i] * sc[j];
        const double2 m1 = Mb[i * n + j], m2 = Mb[j * n + i];
        A[e] = make_double2(0.5 * sij * mscale * (m1.x + m2.x), 0.5 * sij * mscale * (m1.y - m2.y));
        const double2 k1 = Kb[i * n + j], k2 = Kb[j * n + i];
        Kh[e] = make_double2(0.5 * sij * (k1.x + k2.x), 0.5 * sij * (k1.y - k2.y));
    }
    __syncthreads();
    jacobi_herm(n, A, Vm, w, red, rot);
    if (tid == 0) {
        double dm = 0.0;
        for (int i = 0; i < n; ++i) dm = fmax(dm, w[i]);
        dmax_sh = dm;
        int r = 0;   // kept directions, compacted to the front in original order
        for (int i = 0; i < n; ++i)
            if (w[i] > eps * dm && dm > 0.0) perm[r++] = i;
        r_sh = r;
    }
    __syncthreads();
    const int r = r_sh;
    // Z[:, c] = Vm[:, perm[c]] / sqrt(w[perm[c]]) into Y (n x r, row-major n x n storage)
    for (int e = tid; e < n * r; e += nt) {
        const int i = e / r, c = e % r;
        const double s = 1.0 / sqrt(w[perm[c]]);
        const double2 v = Vm[i * n + perm[c]];
        Y[i * n + c] = make_double2(v.x * s, v.y * s);
    }
    __syncthreads();
    // T = Kh Z (n x r) into Vm
    for (int e = tid; e < n * r; e += nt) {
        const int i = e / r, c = e % r;
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < n; ++k) acc = zadd(acc, zmul(Kh[i * n + k], Y[k * n + c]));
        Vm[i * n + c] = acc;
    }
    __syncthreads();
    // C = Z^H T (r x r, stored r x r row-major) into A
    for (int e = tid; e < r * r; e += nt) {
        const int i = e / r, j = e % r;
        double2 acc = make_double2(0.0, 0.0);
        for (int k = 0; k < n; ++k) acc = zadd(acc, zmul(zconj(Y[k * n + i]), Vm[k * n + j]));
        A[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < r * r; e += nt) {   // Hermitian part (in Kh, r x r)
        const int i = e / r, j = e % r;
        const double2 a = A[i * r + j], c = A[j * r + i];
        Kh[e] = make_double2(0.5 * (a.x + c.x), 0.5 * (a.y - c.y));
    }
    __syncthreads();
    jacobi_herm(r, Kh, Vm, w, red, rot);   // eigenvectors (r x r) in Vm
    sort_ascending(r, w, perm);
    // Q = Z Y_sorted (n x r), zero beyond r
    double2* Qb = Q + (size_t)b * n * n;
    for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, c = e % n;
        double2 acc = make_double2(0.0, 0.0);
        if (c < r)
            for (int k = 0; k < r; ++k) acc = zadd(acc, zmul(Y[i * n + k], Vm[k * r + perm[c]]));
        Qb[e] = make_double2(sc[i] * acc.x, sc[i] * acc.y);
    }
    for (int c = tid; c < n; c += nt) lam[(size_t)b * n + c] = c < r ? w[perm[c]] : 0.0;
    if (tid == 0) rank[b] = r;
}

}  // namespace bloch
