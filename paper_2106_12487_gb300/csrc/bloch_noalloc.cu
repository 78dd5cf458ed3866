// Allocation-free variant of the stiffness operator apply.
//
// bloch_apply_K runs its FFT passes through a plan-owned scratch buffer that
// grows with cudaMalloc the first time a larger batch is seen.  Callers that
// may not allocate device memory at the point of the call (services with a
// fixed device-memory budget, code embedded in a framework that owns the
// allocator, real-time loops in which an allocator call may stall the
// device) use bloch_apply_K_noalloc
// instead: its scratch is one file-scope device array of fixed size.  The
// array is placed on a device when this file's module is loaded there --
// with CUDA's lazy module loading, at the first call of the entry point on
// that device -- and held until the process exits.  The operator, its kernels
// (the same pass kernels and launch shapes) and its results are those of
// bloch_apply_K in FP32.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "internal.h"

namespace bloch {

// Scratch layout inside the one static array: the six-component FFT-pass
// intermediates (6 x V x nb float2) first, then the per-system q tables
// ((Nx+Ny+Nz) x nb float) and the wave vectors (3 x nb double).
constexpr size_t kNoAllocPassBytes = (size_t)96 << 20;   // 96 MiB: nb*V <= 2^21 (one 128^3 system)
constexpr size_t kNoAllocTableBytes = (size_t)1 << 20;   // 1 MiB for q tables and wave vectors
constexpr size_t kNoAllocBytes = kNoAllocPassBytes + kNoAllocTableBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Shared-memory attributes of this file's kernel instances (each translation
// unit holds its own copies of the template kernels).
template <typename K>
static cudaError_t smem_attr(K k) {
    cudaError_t e = allow_max_dyn_smem(k);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

template <int RA, int RB>
static cudaError_t attrs_n() {
    cudaError_t e;
    constexpr int PT = (RA * RB * 32 * sizeof(float2) <= 64 * 1024) ? 32 : 16;
    if ((e = smem_attr(k_fpass_y<float, +1, RA, RB, PT>)) != cudaSuccess) return e;
    if ((e = smem_attr(k_fpass_y<float, -1, RA, RB, PT>)) != cudaSuccess) return e;
    if constexpr (RB <= 8) {
        if ((e = smem_attr(k_fpass_z_strain<float, RA, RB, kFastZThreads>)) != cudaSuccess) return e;
        if ((e = smem_attr(k_fpass_z_div<float, RA, RB, kFastZThreads>)) != cudaSuccess) return e;
        if ((e = smem_attr(k_fpass_x_stress<float, RA, RB>)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t set_attrs() {
    cudaError_t e;
    if ((e = smem_attr(k_pass_z_strain<float>)) != cudaSuccess) return e;
    if ((e = smem_attr(k_pass_axis<float, +1, 1>)) != cudaSuccess) return e;
    if ((e = smem_attr(k_pass_axis<float, -1, 1>)) != cudaSuccess) return e;
    if ((e = smem_attr(k_pass_x_stress<float>)) != cudaSuccess) return e;
    if ((e = smem_attr(k_pass_z_div<float>)) != cudaSuccess) return e;
    if ((e = attrs_n<4, 4>()) != cudaSuccess) return e;
    if ((e = attrs_n<8, 4>()) != cudaSuccess) return e;
    if ((e = attrs_n<8, 8>()) != cudaSuccess) return e;
    if ((e = attrs_n<16, 8>()) != cudaSuccess) return e;
    return attrs_n<16, 16>();
}

// Set-up, once per device (with that device current): the device address of
// the scratch array and the kernel attributes.
constexpr int kMaxDevices = 64;
static void* g_noalloc_ptr[kMaxDevices] = {nullptr};
static std::mutex g_noalloc_mu;

static bloch_status noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(BLOCH_EUNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        e = set_attrs();
        if (e != cudaSuccess) return set_cuda_error(e, "cudaFuncSetAttribute (allocation-free passes)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return BLOCH_OK;
}

static bool fast_len(int N) { return N == 16 || N == 32 || N == 64 || N == 128; }

template <int RA, int RB>
static void y_pass(bloch_plan* pl, int DIR, int nb, float2* E) {
    constexpr int N = RA * RB;
    constexpr int PT = (N * 32 * sizeof(float2) <= 64 * 1024) ? 32 : 16;
    const long long npen = (long long)pl->Nx * pl->Nz;
    const size_t smem = (size_t)(N + N * PT) * sizeof(float2);
    dim3 gr((unsigned)((npen + PT - 1) / PT), nb * 6);
    if (DIR > 0)
        k_fpass_y<float, +1, RA, RB, PT><<<gr, 256, smem, pl->stream>>>(E, E, pl->d_twf[1], pl->geo_f);
    else
        k_fpass_y<float, -1, RA, RB, PT><<<gr, 256, smem, pl->stream>>>(E, E, pl->d_twf[1], pl->geo_f);
}

// z passes: kFastZThreads threads per CTA over P = kFastZThreads / RA
// neighbouring pencils, the launch shape of bloch_apply_K
template <int RA, int RB>
static void z_strain(bloch_plan* pl, int nb, const float2* u, float2* E, const float* qtab) {
    constexpr int NT = kFastZThreads;
    constexpr int P = NT / RA;
    const long long npen = (long long)pl->Nx * pl->Ny;
    dim3 gr((unsigned)((npen + P - 1) / P), nb);
    CUtensorMap map;   // encoded on the host: no device memory
    const int tma = encode_zmap(&map, u, pl, 3LL * nb, P) ? 1 : 0;
    k_fpass_z_strain<float, RA, RB, NT><<<gr, NT, fpass_z1_smem<float, RA, RB, NT>(), pl->stream>>>(
        u, E, qtab, pl->d_twf[2], pl->geo_f, map, tma);
}

template <int RA, int RB>
static void x_stress(bloch_plan* pl, int nb, float2* E) {
    constexpr int P = 128 / RA;
    const long long rows = (long long)pl->Ny * pl->Nz;
    dim3 gr((unsigned)((rows + P - 1) / P), nb);
    k_fpass_x_stress<float, RA, RB><<<gr, 128, fpass_x_smem<float, RA, RB>(), pl->stream>>>(
        E, pl->d_ids, pl->d_Cpf, pl->d_twf[0], pl->geo_f, nullptr);
}

template <int RA, int RB>
static void z_div(bloch_plan* pl, int nb, const float2* E, float2* out, const float* qtab) {
    constexpr int NT = kFastZThreads;
    constexpr int P = NT / RA;
    const long long npen = (long long)pl->Nx * pl->Ny;
    dim3 gr((unsigned)((npen + P - 1) / P), nb);
    CUtensorMap map;
    const int tma = encode_zmap(&map, E, pl, 6LL * nb, P) ? 1 : 0;
    k_fpass_z_div<float, RA, RB, NT><<<gr, NT, fpass_z5_smem<float, RA, RB, NT>(), pl->stream>>>(
        E, out, qtab, pl->d_twf[2], pl->geo_f, (float)pl->Kscale, nullptr, nullptr, map, tma);
}

#define NOALLOC_SWITCH(N, FN, ...)                \
    switch (N) {                                  \
        case 16: FN<4, 4>(__VA_ARGS__); break;    \
        case 32: FN<8, 4>(__VA_ARGS__); break;    \
        case 64: FN<8, 8>(__VA_ARGS__); break;    \
        default: FN<16, 8>(__VA_ARGS__); break;   \
    }

}  // namespace bloch

using namespace bloch;

extern "C" bloch_status bloch_apply_K_noalloc(bloch_plan* pl, int32_t nb, const double* k, const void* u, void* Ku) {
    if (!pl) return set_error(BLOCH_EINVAL, "plan is NULL");
    if (!k || !u || !Ku) return set_error(BLOCH_EINVAL, "NULL argument");
    if (u == Ku) return set_error(BLOCH_EINVAL, "Ku may not alias u");
    // the y passes launch 6 * nb CTA rows (gridDim.y <= 65535), as in bloch_apply_K
    if (nb < 1 || nb > 65535 / 6) return set_error(BLOCH_EINVAL, "nb must be in [1, 10922]");
    if (!pl->fast) return set_error(BLOCH_EUNSUPPORTED, "bloch_apply_K_noalloc runs the default FFT variant only");
    const size_t pass_bytes = (size_t)6 * (size_t)pl->V * (size_t)nb * sizeof(float2);
    if (pass_bytes > kNoAllocPassBytes)
        return set_error(BLOCH_EINVAL, "bloch_apply_K_noalloc: nb * V = " + std::to_string((long long)nb * pl->V) +
                                           " exceeds its fixed scratch (nb * V <= 2097152)");
    const int S = pl->Nx + pl->Ny + pl->Nz;
    const size_t q_bytes = ((size_t)S * nb * sizeof(float) + 255) / 256 * 256;
    const size_t k_bytes = (size_t)3 * nb * sizeof(double);
    if (q_bytes + k_bytes > kNoAllocTableBytes)
        return set_error(BLOCH_EINVAL, "bloch_apply_K_noalloc: (Nx+Ny+Nz+6) * nb exceeds its 1 MiB table scratch");
    for (int i = 0; i < 3 * nb; ++i)
        if (!std::isfinite(k[i])) return set_error(BLOCH_ENONFINITE, "wave vector has a non-finite component");

    void* base = nullptr;
    bloch_status st = noalloc_scratch(&base);
    if (st != BLOCH_OK) return st;
    unsigned char* b = (unsigned char*)base;
    float2* E = (float2*)b;
    float* qtab = (float*)(b + kNoAllocPassBytes);
    double* kvec = (double*)(b + kNoAllocPassBytes + q_bytes);

    cudaError_t e = cudaMemcpyAsync(kvec, k, k_bytes, cudaMemcpyHostToDevice, pl->stream);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaMemcpyAsync (wave vectors)");
    const int qblocks = (int)std::min<long long>(1024, ((long long)nb * S + 255) / 256);
    k_qtab<float><<<qblocks, 256, 0, pl->stream>>>(kvec, pl->d_xi, pl->Nx, pl->Ny, pl->Nz, nb, pl->qscale, qtab);

    // the five passes of the K-apply, the kernels of bloch_apply_K (two-stage
    // register passes on axes of 16..128, shared-memory Stockham passes otherwise)
    const Geo& g = pl->geo_f;
    const TileCfg& t = pl->tile_f;
    const long long pxy = (long long)pl->Nx * pl->Ny, pxz = (long long)pl->Nx * pl->Nz,
                    pyz = (long long)pl->Ny * pl->Nz;
    dim3 g1((unsigned)((pxy + t.Pz5 - 1) / t.Pz5), nb);
    dim3 g2((unsigned)((pxz + t.Py2 - 1) / t.Py2), nb * 6);
    dim3 g3((unsigned)((pyz + t.Px7 - 1) / t.Px7), nb);
    const float2* uu = (const float2*)u;
    float2* out = (float2*)Ku;
    const bool fz = fast_len(pl->Nz), fy = fast_len(pl->Ny) || pl->Ny == 256, fx = fast_len(pl->Nx);
    if (fz) {
        NOALLOC_SWITCH(pl->Nz, z_strain, pl, nb, uu, E, qtab);
    } else {
        k_pass_z_strain<float><<<g1, 256, t.smem_z5, pl->stream>>>(uu, E, qtab, pl->d_twf[2], g, t.Pz5);
    }
    if (fy) {
        if (pl->Ny == 256) y_pass<16, 16>(pl, +1, nb, E);
        else NOALLOC_SWITCH(pl->Ny, y_pass, pl, +1, nb, E);
    } else {
        k_pass_axis<float, +1, 1><<<g2, 256, t.smem_y2, pl->stream>>>(E, E, pl->d_twf[1], g, t.Py2, 1.0f);
    }
    if (fx) {
        NOALLOC_SWITCH(pl->Nx, x_stress, pl, nb, E);
    } else {
        k_pass_x_stress<float><<<g3, 256, t.smem_x7, pl->stream>>>(E, pl->d_ids, pl->d_Cf, pl->d_twf[0], g, t.Px7);
    }
    if (fy) {
        if (pl->Ny == 256) y_pass<16, 16>(pl, -1, nb, E);
        else NOALLOC_SWITCH(pl->Ny, y_pass, pl, -1, nb, E);
    } else {
        k_pass_axis<float, -1, 1><<<g2, 256, t.smem_y2, pl->stream>>>(E, E, pl->d_twf[1], g, t.Py2, 1.0f);
    }
    if (fz) {
        NOALLOC_SWITCH(pl->Nz, z_div, pl, nb, E, out, qtab);
    } else {
        k_pass_z_div<float><<<g1, 256, t.smem_z5, pl->stream>>>(E, out, qtab, pl->d_twf[2], g, t.Pz5,
                                                                (float)pl->Kscale);
    }
    pl->launches += 6;
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error(e, "bloch_apply_K_noalloc launch");
    return BLOCH_OK;
}
