// Autotuner of the batched stiffness operator: picks the FFT pass variant and
// the pencils-per-CTA cap of the shared-memory passes by timing one A_k apply
// of the requested batch for every candidate, then reports the batch size at
// which the time per system stops falling.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

using namespace bloch;

namespace {

// Deterministic pseudo-random complex field in [-1, 1)^2 (splitmix64 finaliser).
template <typename C>
__global__ void k_tune_fill(C* v, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        unsigned long long x = 0x9E3779B97F4A7C15ULL * (unsigned long long)(e + 1);
        x ^= x >> 30;
        x *= 0xBF58476D1CE4E5B9ULL;
        x ^= x >> 27;
        x *= 0x94D049BB133111EBULL;
        x ^= x >> 31;
        const double re = (double)(x & 0xffffffffULL) * (1.0 / 2147483648.0) - 1.0;
        const double im = (double)(x >> 32) * (1.0 / 2147483648.0) - 1.0;
        v[e] = mk((decltype(v[0].x))re, (decltype(v[0].x))im);
    }
}

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Mean time (ms) of `reps` applies after one untimed apply; < 0 on failure.
template <typename T>
double time_apply(bloch_plan* pl, int nb, const cplx_t<T>* u, cplx_t<T>* out, Timer& t, int reps) {
    pl->pending = BLOCH_OK;
    launch_K<T>(pl, nb, u, out, T(1));
    if (cudaEventRecord(t.a, pl->stream) != cudaSuccess) return -1.0;
    for (int i = 0; i < reps; ++i) launch_K<T>(pl, nb, u, out, T(1));
    if (cudaEventRecord(t.b, pl->stream) != cudaSuccess) return -1.0;
    if (cudaEventSynchronize(t.b) != cudaSuccess || cudaGetLastError() != cudaSuccess) return -1.0;
    if (pl->pending != BLOCH_OK) return -1.0;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) return -1.0;
    return (double)ms / reps;
}

template <typename T>
bloch_status tune(bloch_plan* pl, int systems, bloch_tune_report* rep) {
    using C = cplx_t<T>;
    const int precision = std::is_same<T, float>::value ? BLOCH_FP32 : BLOCH_FP64;
    const long long n = (long long)systems * 3 * pl->V;
    C* buf = nullptr;
    cudaError_t e = cudaMalloc((void**)&buf, sizeof(C) * (size_t)(2 * n));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(BLOCH_ENOMEM, "autotune: cannot allocate the trial fields");
    }
    C* u = buf;
    C* out = buf + n;
    std::vector<double> k((size_t)3 * systems);
    for (int s = 0; s < systems; ++s) {   // one wave vector inside the first Brillouin zone
        k[3 * s + 0] = 0.50 * M_PI / pl->L[0];
        k[3 * s + 1] = 0.25 * M_PI / pl->L[1];
        k[3 * s + 2] = 0.125 * M_PI / pl->L[2];
    }
    bloch_status st = set_k<T>(pl, systems, k.data());
    Timer t;
    if (st == BLOCH_OK && (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess))
        st = set_error(BLOCH_ECUDA, "autotune: cudaEventCreate failed");
    if (st == BLOCH_OK) {
        ++pl->launches;
        k_tune_fill<C><<<1024, 256, 0, pl->stream>>>(u, n);
        if (cudaGetLastError() != cudaSuccess) st = set_error(BLOCH_ECUDA, "autotune: fill launch failed");
    }
    const int old_variant = pl->variant, old_pmax = pl->tile_f.pmax;
    double best = -1.0;
    int best_v = old_variant, best_p = old_pmax, cand = 0;
    double per_var[3] = {-1.0, -1.0, -1.0};
    const int pmaxes[4] = {4, 8, 16, 32};
    const int reps = 3;
    for (int v = 0; v < 3 && st == BLOCH_OK; ++v) {
        if (v == 0 && !has_fast_pass(pl, precision)) continue;
        const bool sweep = v != 2 && (v == 1 || has_generic_pass(pl, precision));
        for (int ip = 0; ip < (sweep ? 4 : 1) && st == BLOCH_OK; ++ip) {
            const int pm = sweep ? pmaxes[ip] : kDefaultPmax;
            configure_passes(pl, v, pm);
            const double ms = time_apply<T>(pl, systems, u, out, t, reps);
            if (ms < 0) {
                if (v == 2) {   // cuFFT may lack memory for its plan: not a failure of the tuner
                    cudaGetLastError();
                    pl->pending = BLOCH_OK;
                    continue;
                }
                st = set_error(BLOCH_ECUDA, "autotune: a trial apply failed");
                break;
            }
            ++cand;
            const double per = ms / systems;
            if (per_var[v] < 0 || per < per_var[v]) per_var[v] = per;
            if (best < 0 || per < best) {
                best = per;
                best_v = v;
                best_p = pm;
            }
        }
    }
    cudaFree(buf);
    configure_passes(pl, st == BLOCH_OK ? best_v : old_variant, st == BLOCH_OK ? best_p : old_pmax);
    if (st != BLOCH_OK) return st;
    // batch sweep with the chosen configuration
    int sat = systems;
    std::vector<std::pair<int, double>> curve{{systems, best}};
    for (int mult = 2; mult <= 8; mult *= 2) {
        const int nb = systems * mult;
        if (nb > 10922) break;
        const long long nn = (long long)nb * 3 * pl->V;
        size_t freeb = 0, totb = 0;
        cudaMemGetInfo(&freeb, &totb);
        // trial fields (2 x 3 V) plus the operator workspace the batch grows (6 V) per system
        const size_t need = sizeof(C) * (size_t)(nn / 3) * 12;
        if (need > freeb / 4) break;
        C* b2 = nullptr;
        if (cudaMalloc((void**)&b2, sizeof(C) * (size_t)(2 * nn)) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        std::vector<double> kk((size_t)3 * nb);
        for (int s = 0; s < nb; ++s) std::memcpy(&kk[3 * s], &k[0], 3 * sizeof(double));
        bloch_status s2 = set_k<T>(pl, nb, kk.data());
        double ms = -1.0;
        if (s2 == BLOCH_OK) {
            ++pl->launches;
            k_tune_fill<C><<<1024, 256, 0, pl->stream>>>(b2, nn);
            ms = time_apply<T>(pl, nb, b2, b2 + nn, t, reps);
        }
        cudaFree(b2);
        if (s2 != BLOCH_OK || ms < 0) {
            cudaGetLastError();
            pl->pending = BLOCH_OK;
            break;
        }
        curve.push_back({nb, ms / nb});
    }
    double floor_t = best;
    for (auto& c : curve) floor_t = std::min(floor_t, c.second);
    for (auto& c : curve)
        if (c.second <= 1.05 * floor_t) {
            sat = c.first;
            break;
        }
    pl->tuned = true;
    if (rep) {
        rep->fft_variant = best_v;
        rep->tile_pmax = best_p;
        rep->saturating_systems = sat;
        rep->candidates = cand;
        for (int v = 0; v < 3; ++v) rep->ms_per_system[v] = per_var[v];
    }
    return BLOCH_OK;
}

}  // namespace

extern "C" bloch_status bloch_plan_autotune(bloch_plan* pl, int32_t precision, int32_t systems,
                                            bloch_tune_report* report) {
    if (!pl) return set_error(BLOCH_EINVAL, "plan is NULL");
    if (systems < 1 || systems > 10922) return set_error(BLOCH_EINVAL, "systems must be in [1, 10922]");
    if (precision == BLOCH_FP32) return tune<float>(pl, systems, report);
    if (precision == BLOCH_FP64) return tune<double>(pl, systems, report);
    return set_error(BLOCH_EINVAL, "precision must be BLOCH_FP32 or BLOCH_FP64");
}

namespace {

// Independent FMA chains: 8 accumulators per thread, 16 x 8 FMAs per loop trip.
template <typename T>
__global__ void k_fma_chain(T* out, int trips) {
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = T(threadIdx.x) * T(1e-6) + T(i);
    const T m = T(1.0000001), c = T(1e-12);
    for (int it = 0; it < trips; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fma(a[i], m, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <typename T>
bloch_status fma_rate(int blocks, int trips, double* gflops) {
    const int threads = 256;
    T* d = nullptr;
    if (cudaMalloc(&d, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) {
        cudaGetLastError();
        return set_error(BLOCH_ENOMEM, "FMA probe: device allocation failed");
    }
    Timer t;
    bloch_status st = BLOCH_OK;
    if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) st = BLOCH_ECUDA;
    if (st == BLOCH_OK) {
        for (int w = 0; w < 3; ++w) k_fma_chain<T><<<blocks, threads>>>(d, trips);
        cudaEventRecord(t.a);
        k_fma_chain<T><<<blocks, threads>>>(d, trips);
        cudaEventRecord(t.b);
        float ms = 0.f;
        if (cudaEventSynchronize(t.b) != cudaSuccess || cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess || ms <= 0.f)
            st = BLOCH_ECUDA;
        else
            *gflops = 2.0 * blocks * threads * (double)trips * 16 * 8 / ms / 1e6;
    }
    cudaFree(d);
    return st == BLOCH_OK ? st : set_error(st, "FMA probe: CUDA error");
}

}  // namespace

extern "C" bloch_status bloch_fma_peaks(double* fp64_gflops, double* fp32_gflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return set_error(BLOCH_ECUDA, "FMA probe: no device");
    double g64 = 0.0, g32 = 0.0;
    bloch_status st = fma_rate<double>(sms * 8, 2000, &g64);
    if (st == BLOCH_OK) st = fma_rate<float>(sms * 8, 16000, &g32);
    if (st != BLOCH_OK) return st;
    if (fp64_gflops) *fp64_gflops = g64;
    if (fp32_gflops) *fp32_gflops = g32;
    return BLOCH_OK;
}
