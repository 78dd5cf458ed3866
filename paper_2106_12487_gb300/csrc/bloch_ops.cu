// Plan creation, operator launchers, batched PCG and the C ABI entry points
// for the operators (Section 3.2 Eqs. hatA/hatM, Section 3.3 Algorithm 2).
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <string>
#include <vector>

#include "eig_kernels.cuh"
#include "internal.h"

namespace bloch {

static thread_local std::string g_last_error;

bloch_status set_error(bloch_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

bloch_status set_cuda_error(cudaError_t e, const char* what) {
    g_last_error = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? BLOCH_ENOMEM : BLOCH_ECUDA;
}

template <> Workspace<float>& ws_of<float>(bloch_plan* pl) { return pl->ws_f; }
template <> Workspace<double>& ws_of<double>(bloch_plan* pl) { return pl->ws_d; }
template <> Workspace<dfloat>& ws_of<dfloat>(bloch_plan* pl) { return pl->ws_x; }
// float-float runs the FP64 radix schedule and tiles (same 16-byte complex)
template <> const Geo& geo_of<dfloat>(const bloch_plan* pl) { return pl->geo_d; }
template <> const Geo& geo_of<float>(const bloch_plan* pl) { return pl->geo_f; }
template <> const Geo& geo_of<double>(const bloch_plan* pl) { return pl->geo_d; }
template <typename T> static const TileCfg& tile_of(const bloch_plan* pl);
template <> const TileCfg& tile_of<float>(const bloch_plan* pl) { return pl->tile_f; }
template <> const TileCfg& tile_of<double>(const bloch_plan* pl) { return pl->tile_d; }
template <> const TileCfg& tile_of<dfloat>(const bloch_plan* pl) { return pl->tile_d; }
template <typename T> static const cplx_t<T>* tw_of(const bloch_plan* pl, int axis);
template <> const float2* tw_of<float>(const bloch_plan* pl, int axis) { return pl->d_twf[axis]; }
template <> const double2* tw_of<double>(const bloch_plan* pl, int axis) { return pl->d_twd[axis]; }
template <> const dfloat2* tw_of<dfloat>(const bloch_plan* pl, int axis) { return pl->d_twx[axis]; }
template <typename T> static const T* ctab_of(const bloch_plan* pl);
template <> const float* ctab_of<float>(const bloch_plan* pl) { return pl->d_Cf; }
template <> const double* ctab_of<double>(const bloch_plan* pl) { return pl->d_Cd; }
template <> const dfloat* ctab_of<dfloat>(const bloch_plan* pl) { return pl->d_Cx; }
template <typename T> static const T* cpk_of(const bloch_plan* pl);
template <> const float* cpk_of<float>(const bloch_plan* pl) { return pl->d_Cpf; }
template <> const double* cpk_of<double>(const bloch_plan* pl) { return pl->d_Cpd; }
template <typename T> static const T* rtab_of(const bloch_plan* pl);
template <> const float* rtab_of<float>(const bloch_plan* pl) { return pl->d_rf; }
template <> const double* rtab_of<double>(const bloch_plan* pl) { return pl->d_rd; }
template <> const dfloat* rtab_of<dfloat>(const bloch_plan* pl) { return pl->d_rx; }

// ------------------------------------------------------------ host helpers
static bool fast_axis(int N);
static bool fast_x(int N);

static bool factor_ok(int n) {
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

// Radix schedule: power-of-two part in as few stages as possible (each at most
// max_r), then the odd factors 3, 5, 7.
static AxisPlan make_axis(int N, int max_log2) {
    AxisPlan ap{};
    ap.N = N;
    int n = N, l2 = 0;
    while (n % 2 == 0) {
        n /= 2;
        ++l2;
    }
    int nst2 = (l2 + max_log2 - 1) / max_log2;
    for (int s = 0; s < nst2; ++s) {
        const int bits = l2 / (nst2 - s);
        ap.radix[ap.nst++] = 1 << bits;
        l2 -= bits;
    }
    for (int p : {3, 5, 7})
        while (n % p == 0) {
            ap.radix[ap.nst++] = p;
            n /= p;
        }
    return ap;
}

static int choose_P(int N, int bufs, size_t elem, size_t budget, long long npen, int pmax) {
    int P = pmax;
    while (P > 1 && (size_t)bufs * N * P * elem + (size_t)(N + 1) * elem > budget) P >>= 1;
    while (P > 1 && (long long)(P / 2) >= npen) P >>= 1;
    return P;
}

// Pencils per CTA of the shared-memory passes: at most pmax (z, y) or pmax / 2
// (x), reduced until the tile fits the shared-memory budget of its pass.
template <typename T>
static TileCfg make_tiles(int Nx, int Ny, int Nz, int pmax) {
    TileCfg t{};
    const size_t el = sizeof(cplx_t<T>);
    auto pad = [&](int N) { return (size_t)((N + 1) & ~1) * el; };
    const int px = std::max(1, pmax / 2);
    t.pmax = pmax;
    t.Pz5 = choose_P(Nz, 5, el, 96 * 1024, (long long)Nx * Ny, pmax);
    t.Py2 = choose_P(Ny, 2, el, 64 * 1024, (long long)Nx * Nz, pmax);
    t.Pz2 = choose_P(Nz, 2, el, 64 * 1024, (long long)Nx * Ny, pmax);
    t.Px7 = choose_P(Nx, 7, el, 96 * 1024, (long long)Ny * Nz, px);
    t.Px4 = choose_P(Nx, 4, el, 64 * 1024, (long long)Ny * Nz, px);
    t.smem_z5 = pad(Nz) + (size_t)5 * Nz * t.Pz5 * el;
    t.smem_y2 = pad(Ny) + (size_t)2 * Ny * t.Py2 * el;
    t.smem_z2 = pad(Nz) + (size_t)2 * Nz * t.Pz2 * el;
    t.smem_x7 = pad(Nx) + (size_t)7 * Nx * t.Px7 * el;
    t.smem_x4 = pad(Nx) + (size_t)4 * Nx * t.Px4 * el;
    return t;
}

template <typename T>
static cudaError_t set_smem_attrs() {
    cudaError_t e;
#define SETA(f)                   \
    e = allow_max_dyn_smem(f);    \
    if (e != cudaSuccess) return e;
    SETA(k_pass_z_strain<T>);
    SETA((k_pass_axis<T, +1, 1>));
    SETA((k_pass_axis<T, -1, 1>));
    SETA((k_pass_axis<T, +1, 2>));
    SETA((k_pass_axis<T, -1, 2>));
    SETA(k_pass_x_stress<T>);
    SETA(k_pass_z_div<T>);
    SETA(k_pass_x_rho<T>);
    SETA((k_pass_x<T, +1>));
    SETA((k_pass_x<T, -1>));
#undef SETA
    return cudaSuccess;
}

int vec_blocks(const bloch_plan* pl, int nb) {
    long long b = (pl->V + 255) / 256;
    long long cap = std::max(1, 4096 / std::max(nb, 1));
    return (int)std::max(1LL, std::min(b, cap));
}

template <typename T>
static cudaError_t dmalloc(T** p, size_t n, size_t* acc) {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e == cudaSuccess && acc) *acc += n * sizeof(T);
    return e;
}

// ------------------------------------------------------------ workspaces
template <typename T>
bloch_status ensure_ws(bloch_plan* pl, int nb) {
    Workspace<T>& w = ws_of<T>(pl);
    if (nb <= w.cap) return BLOCH_OK;
    cudaStreamSynchronize(pl->stream);
    const int S = pl->Nx + pl->Ny + pl->Nz;
    if (w.E) pl->device_bytes -= (size_t)w.cap * (6 * pl->V * sizeof(cplx_t<T>) + S * sizeof(T) + 3 * sizeof(double));
    cudaFree(w.E);
    cudaFree(w.qtab);
    cudaFree(w.kvec);
    w.E = nullptr;
    w.qtab = nullptr;
    w.kvec = nullptr;
    w.cap = 0;
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.E, (size_t)6 * pl->V * nb, &pl->device_bytes));
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.qtab, (size_t)S * nb, &pl->device_bytes));
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.kvec, (size_t)3 * nb, &pl->device_bytes));
    w.cap = nb;
    return BLOCH_OK;
}

template <typename T>
bloch_status ensure_cg(bloch_plan* pl, int nb) {
    bloch_status st = ensure_ws<T>(pl, nb);
    if (st != BLOCH_OK) return st;
    Workspace<T>& w = ws_of<T>(pl);
    if (nb <= w.cg_cap) return BLOCH_OK;
    cudaStreamSynchronize(pl->stream);
    const size_t vec = (size_t)3 * pl->V * sizeof(cplx_t<T>);
    if (w.r) pl->device_bytes -= (size_t)w.cg_cap * (3 * vec + pl->nblk_max * (3 * sizeof(double) + sizeof(double2)) +
                                                     sizeof(double2) + sizeof(CGSys) + w.zblk * sizeof(double2));
    cudaFree(w.partz);
    w.partz = nullptr;
    cudaFree(w.r);
    cudaFree(w.p);
    cudaFree(w.Ap);
    cudaFree(w.part3);
    cudaFree(w.part2);
    cudaFree(w.dots);
    cudaFree(w.sys);
    w.r = w.p = w.Ap = nullptr;
    w.part3 = nullptr;
    w.part2 = w.dots = nullptr;
    w.sys = nullptr;
    w.cg_cap = 0;
    const size_t n = (size_t)3 * pl->V * nb;
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.r, n, &pl->device_bytes));
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.p, n, &pl->device_bytes));
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.Ap, n, &pl->device_bytes));
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.part3, (size_t)nb * pl->nblk_max * 3, &pl->device_bytes));
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.part2, (size_t)nb * pl->nblk_max, &pl->device_bytes));
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.dots, (size_t)nb, &pl->device_bytes));
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.sys, (size_t)nb, &pl->device_bytes));
    // the fused (p, Ap) partials need one slot per CTA of the fast x or z pass that forms them,
    // for any fast variant later chosen (>= CTAs per system for every P >= 2)
    w.zblk = std::is_same<T, float>::value && (fast_x(pl->Nz) || fast_x(pl->Nx))
                 ? (int)((std::max((long long)pl->Nx * pl->Ny, (long long)pl->Ny * pl->Nz) + 1) / 2)
                 : 0;
    if (w.zblk) BLOCH_CUDA_CHECK_RET(dmalloc(&w.partz, (size_t)nb * w.zblk, &pl->device_bytes));
    w.cg_cap = nb;
    return BLOCH_OK;
}

template <typename T>
bloch_status set_k(bloch_plan* pl, int nb, const double* k_host) {
    bloch_status st = ensure_ws<T>(pl, nb);
    if (st != BLOCH_OK) return st;
    for (int i = 0; i < 3 * nb; ++i)
        if (!std::isfinite(k_host[i])) return set_error(BLOCH_ENONFINITE, "wave vector has a non-finite component");
    Workspace<T>& w = ws_of<T>(pl);
    pl->k_host.assign(k_host, k_host + 3 * (size_t)nb);
    BLOCH_CUDA_CHECK_RET(
        cudaMemcpyAsync(w.kvec, k_host, sizeof(double) * 3 * nb, cudaMemcpyHostToDevice, pl->stream));
    const int S = pl->Nx + pl->Ny + pl->Nz;
    const int blocks = (int)std::min<long long>(1024, ((long long)nb * S + 255) / 256);
    ++pl->launches;
    k_qtab<T><<<blocks, 256, 0, pl->stream>>>(w.kvec, pl->d_xi, pl->Nx, pl->Ny, pl->Nz, nb, pl->qscale, w.qtab);
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    return BLOCH_OK;
}

// ------------------------------------------------------------ operators
template <typename T>
void launch_K_generic(bloch_plan* pl, int nb, const cplx_t<T>* u, cplx_t<T>* out, T out_scale);

// ------------------------------------------------ fast two-stage passes
static bool fast_axis(int N) { return N == 16 || N == 32 || N == 64 || N == 128 || N == 256; }
static bool fast_x(int N) { return N == 16 || N == 32 || N == 64 || N == 128; }

void drop_pcg_graphs(bloch_plan* pl) {
    for (auto& e : pl->pcg_graphs) {
        cudaGraphExecDestroy(e.exec);
        cudaGraphDestroy(e.graph);
    }
    pl->pcg_graphs.clear();
}

void configure_passes(bloch_plan* pl, int variant, int pmax) {
    drop_pcg_graphs(pl);   // instantiated graphs hold the previous launch configuration
    pl->variant = variant;
    pl->fast = variant == 0;
    pl->tile_f = make_tiles<float>(pl->Nx, pl->Ny, pl->Nz, pmax);
    pl->tile_d = make_tiles<double>(pl->Nx, pl->Ny, pl->Nz, pmax);
}

// CTAs per system of the fast z passes (P = 128 / RA pencils each), 0 when
// the fast z passes do not serve this plan in FP32
int fast_z_blocks(const bloch_plan* pl) {
    if (!pl->fast || !fast_x(pl->Nz)) return 0;
    const int RA = pl->Nz == 16 ? 4 : (pl->Nz == 128 ? 16 : 8);
    const int P = kFastZThreads / RA;
    const long long npen = (long long)pl->Nx * pl->Ny;
    return (int)((npen + P - 1) / P);
}

bool has_fast_pass(const bloch_plan* pl, int precision) {
    if (fast_axis(pl->Ny)) return true;
    return precision == BLOCH_FP32 && (fast_x(pl->Nz) || fast_x(pl->Nx));
}

bool has_generic_pass(const bloch_plan* pl, int precision) {
    if (!fast_axis(pl->Ny)) return true;
    return precision != BLOCH_FP32 || !fast_x(pl->Nz) || !fast_x(pl->Nx);
}


template <typename K>
static void fast_attr(K k) {
    allow_max_dyn_smem(k);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

template <typename T, int RA, int RB, bool Z>
static void set_fast_attrs_n() {
    constexpr int PT = (RA * RB * 32 * sizeof(cplx_t<T>) <= 64 * 1024) ? 32 : 16;
    fast_attr(k_fpass_y<T, +1, RA, RB, PT>);
    fast_attr(k_fpass_y<T, -1, RA, RB, PT>);
    if constexpr (Z) {
        fast_attr(k_fpass_z_strain<T, RA, RB, kFastZThreads>);
        fast_attr(k_fpass_z_div<T, RA, RB, kFastZThreads>);
        if constexpr (RB <= 8) fast_attr(k_fpass_x_stress<T, RA, RB>);
    }
}

// the z and x fast passes exist in FP32 only (their register budget); the
// y passes serve FP32, FP64 and float-float
template <typename T>
static void set_fast_attrs() {
    constexpr bool Z = std::is_same<T, float>::value;
    set_fast_attrs_n<T, 4, 4, Z>();
    set_fast_attrs_n<T, 8, 4, Z>();
    set_fast_attrs_n<T, 8, 8, Z>();
    set_fast_attrs_n<T, 16, 8, Z>();
    set_fast_attrs_n<T, 16, 16, false>();
}

template <typename T, int RA, int RB>
static void fast_y(bloch_plan* pl, int DIR, int nb, cplx_t<T>* E) {
    const Geo& g = geo_of<T>(pl);
    constexpr int N = RA * RB;
    constexpr int PT = (N * 32 * sizeof(cplx_t<T>) <= 64 * 1024) ? 32 : 16;
    const long long npen = (long long)pl->Nx * pl->Nz;
    const size_t smem = (size_t)(N + N * PT) * sizeof(cplx_t<T>);
    dim3 gr((unsigned)((npen + PT - 1) / PT), nb * 6);
    ++pl->launches;
    if (DIR > 0)
        k_fpass_y<T, +1, RA, RB, PT><<<gr, 256, smem, pl->stream>>>(E, E, tw_of<T>(pl, 1), g);
    else
        k_fpass_y<T, -1, RA, RB, PT><<<gr, 256, smem, pl->stream>>>(E, E, tw_of<T>(pl, 1), g);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

bool encode_zmap(CUtensorMap* map, const void* base, const bloch_plan* pl, long long nsc, int P) {
    std::memset(map, 0, sizeof(*map));
    const unsigned long long plane = (unsigned long long)pl->Nx * pl->Ny;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
    if (!enc || base == nullptr || ((uintptr_t)base & 15) || (plane * 8) % 16 || plane < (unsigned long long)P ||
        pl->Nz > 256 || nsc < 1)
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)plane, (cuuint64_t)pl->Nz, (cuuint64_t)nsc};
    const cuuint64_t strides[2] = {(cuuint64_t)(plane * 8), (cuuint64_t)(plane * 8 * (unsigned long long)pl->Nz)};
    const cuuint32_t box[3] = {(cuuint32_t)P, (cuuint32_t)pl->Nz, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        std::memset(map, 0, sizeof(*map));
        return false;
    }
    return true;
}

bloch_status check_pass_err(bloch_plan* pl) {
    int e = 0;
    BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(&e, pl->d_perr, sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
    BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
    if (e) {
        cudaMemsetAsync(pl->d_perr, 0, sizeof(int), pl->stream);
        return set_error(BLOCH_ECUDA, "a pass's staging copy did not complete within its wait bound");
    }
    return BLOCH_OK;
}

template <typename T, int RA, int RB>
static void fast_z1(bloch_plan* pl, int nb, const cplx_t<T>* u) {
    const Geo& g = geo_of<T>(pl);
    constexpr int NT = kFastZThreads;
    constexpr int P = NT / RA;
    const long long npen = (long long)pl->Nx * pl->Ny;
    const size_t smem = fpass_z1_smem<T, RA, RB, NT>();
    dim3 gr((unsigned)((npen + P - 1) / P), nb);
    ++pl->launches;
    CUtensorMap map;
    const int tma = encode_zmap(&map, u, pl, 3LL * nb, P) ? 1 : 0;
    k_fpass_z_strain<T, RA, RB, NT><<<gr, NT, smem, pl->stream>>>(u, ws_of<T>(pl).E, ws_of<T>(pl).qtab,
                                                                   tw_of<T>(pl, 2), g, map, tma);
}

template <typename T, int RA, int RB>
static void fast_z5(bloch_plan* pl, int nb, cplx_t<T>* out, T out_scale, const cplx_t<T>* dotp, double2* dpart) {
    const Geo& g = geo_of<T>(pl);
    constexpr int NT = kFastZThreads;
    constexpr int P = NT / RA;
    const long long npen = (long long)pl->Nx * pl->Ny;
    const size_t smem = fpass_z5_smem<T, RA, RB, NT>();
    dim3 gr((unsigned)((npen + P - 1) / P), nb);
    ++pl->launches;
    CUtensorMap map;
    const int tma = encode_zmap(&map, ws_of<T>(pl).E, pl, 6LL * nb, P) ? 1 : 0;
    k_fpass_z_div<T, RA, RB, NT><<<gr, NT, smem, pl->stream>>>(ws_of<T>(pl).E, out, ws_of<T>(pl).qtab,
                                                                tw_of<T>(pl, 2), g, out_scale, dotp, dpart, map,
                                                                tma);
}

// returns the CTAs per system (the number of (p, A p) partials written when dpart != nullptr)
template <typename T, int RA, int RB>
static int fast_x3(bloch_plan* pl, int nb, double2* dpart) {
    const Geo& g = geo_of<T>(pl);
    constexpr int P = 128 / RA;
    const size_t smem = fpass_x_smem<T, RA, RB>();
    const long long rows = (long long)pl->Ny * pl->Nz;
    dim3 gr((unsigned)((rows + P - 1) / P), nb);
    ++pl->launches;
    k_fpass_x_stress<T, RA, RB><<<gr, 128, smem, pl->stream>>>(ws_of<T>(pl).E, pl->d_ids, cpk_of<T>(pl),
                                                                 tw_of<T>(pl, 0), g, dpart);
    return (int)gr.x;
}

#define BLOCH_FAST_SWITCH(N, FN, ...)              \
    switch (N) {                                    \
        case 16: FN<T, 4, 4>(__VA_ARGS__); break;   \
        case 32: FN<T, 8, 4>(__VA_ARGS__); break;   \
        case 64: FN<T, 8, 8>(__VA_ARGS__); break;   \
        case 128: FN<T, 16, 8>(__VA_ARGS__); break; \
        default: FN<T, 16, 16>(__VA_ARGS__); break; \
    }
#define BLOCH_FAST_SWITCH_Z(N, FN, ...)             \
    switch (N) {                                    \
        case 16: FN<T, 4, 4>(__VA_ARGS__); break;   \
        case 32: FN<T, 8, 4>(__VA_ARGS__); break;   \
        case 64: FN<T, 8, 8>(__VA_ARGS__); break;   \
        default: FN<T, 16, 8>(__VA_ARGS__); break;  \
    }

template <typename T>
int launch_K(bloch_plan* pl, int nb, const cplx_t<T>* u, cplx_t<T>* out, T out_scale, const cplx_t<T>* dotp,
             double2* dpart) {
    if (pl->variant == 2) {
        Workspace<T>& w = ws_of<T>(pl);
        if (!cufft_launch_K<T>(pl, nb, u, out, out_scale, w.E, w.qtab, ctab_of<T>(pl), geo_of<T>(pl)))
            pl->pending = set_error(BLOCH_ECUDA, "cuFFT plan or execution failed");
        return 0;
    }
    int fused = 0;
    if (pl->fast) {
        Workspace<T>& w = ws_of<T>(pl);
        const Geo& g = geo_of<T>(pl);
        const TileCfg& t = tile_of<T>(pl);
        const long long pxy = (long long)pl->Nx * pl->Ny, pxz = (long long)pl->Nx * pl->Nz,
                        pyz = (long long)pl->Ny * pl->Nz;
        const bool fz = fast_x(pl->Nz) && std::is_same<T, float>::value;
        const bool fy = fast_axis(pl->Ny);
        const bool fx = fast_x(pl->Nx) && std::is_same<T, float>::value;
        dim3 g1((unsigned)((pxy + t.Pz5 - 1) / t.Pz5), nb);
        dim3 g2((unsigned)((pxz + t.Py2 - 1) / t.Py2), nb * 6);
        dim3 g3((unsigned)((pyz + t.Px7 - 1) / t.Px7), nb);
        bool done1 = false;
        if constexpr (std::is_same<T, float>::value) {
            if (fz) {
                BLOCH_FAST_SWITCH_Z(pl->Nz, fast_z1, pl, nb, u);
                done1 = true;
            }
        }
        if (!done1) {
            ++pl->launches;
            k_pass_z_strain<T><<<g1, 256, t.smem_z5, pl->stream>>>(u, w.E, w.qtab, tw_of<T>(pl, 2), g, t.Pz5);
        }
        if (fy) {
            BLOCH_FAST_SWITCH(pl->Ny, fast_y, pl, +1, nb, w.E);
        } else {
            ++pl->launches;
            k_pass_axis<T, +1, 1><<<g2, 256, t.smem_y2, pl->stream>>>(w.E, w.E, tw_of<T>(pl, 1), g, t.Py2, T(1));
        }
        // (p, A p) partials: from the strain energy in the fast x pass where it runs,
        // else from the fast z-divergence pass (which then reads p once more)
        bool done3 = false;
        const bool xdot = fx && dpart && dotp;
        if constexpr (std::is_same<T, float>::value) {
            if (fx) {
                double2* xd = xdot ? dpart : nullptr;
                int xb = 0;
                switch (pl->Nx) {
                    case 16: xb = fast_x3<T, 4, 4>(pl, nb, xd); break;
                    case 32: xb = fast_x3<T, 8, 4>(pl, nb, xd); break;
                    case 64: xb = fast_x3<T, 8, 8>(pl, nb, xd); break;
                    default: xb = fast_x3<T, 16, 8>(pl, nb, xd); break;
                }
                if (xdot) fused = xb;
                done3 = true;
            }
        }
        if (!done3) {
            ++pl->launches;
            k_pass_x_stress<T><<<g3, 256, t.smem_x7, pl->stream>>>(w.E, pl->d_ids, ctab_of<T>(pl), tw_of<T>(pl, 0),
                                                                    g, t.Px7);
        }
        if (fy) {
            BLOCH_FAST_SWITCH(pl->Ny, fast_y, pl, -1, nb, w.E);
        } else {
            ++pl->launches;
            k_pass_axis<T, -1, 1><<<g2, 256, t.smem_y2, pl->stream>>>(w.E, w.E, tw_of<T>(pl, 1), g, t.Py2, T(1));
        }
        bool done5 = false;
        if constexpr (std::is_same<T, float>::value) {
            if (fz) {
                const bool zdot = !xdot && dpart && dotp;
                BLOCH_FAST_SWITCH_Z(pl->Nz, fast_z5, pl, nb, out, out_scale, zdot ? dotp : nullptr,
                                    zdot ? dpart : nullptr);
                done5 = true;
                if (zdot) fused = fast_z_blocks(pl);
            }
        }
        if (!done5) {
            ++pl->launches;
            k_pass_z_div<T><<<g1, 256, t.smem_z5, pl->stream>>>(w.E, out, w.qtab, tw_of<T>(pl, 2), g, t.Pz5,
                                                                out_scale);
        }
        return fused;
    }
    launch_K_generic<T>(pl, nb, u, out, out_scale);
    return 0;
}

template <typename T>
void launch_K_generic(bloch_plan* pl, int nb, const cplx_t<T>* u, cplx_t<T>* out, T out_scale) {
    Workspace<T>& w = ws_of<T>(pl);
    const Geo& g = geo_of<T>(pl);
    const TileCfg& t = tile_of<T>(pl);
    const long long pxy = (long long)pl->Nx * pl->Ny, pxz = (long long)pl->Nx * pl->Nz,
                    pyz = (long long)pl->Ny * pl->Nz;
    dim3 g1((unsigned)((pxy + t.Pz5 - 1) / t.Pz5), nb);
    ++pl->launches;
    k_pass_z_strain<T><<<g1, 256, t.smem_z5, pl->stream>>>(u, w.E, w.qtab, tw_of<T>(pl, 2), g, t.Pz5);
    dim3 g2((unsigned)((pxz + t.Py2 - 1) / t.Py2), nb * 6);
    ++pl->launches;
    k_pass_axis<T, +1, 1><<<g2, 256, t.smem_y2, pl->stream>>>(w.E, w.E, tw_of<T>(pl, 1), g, t.Py2, T(1));
    dim3 g3((unsigned)((pyz + t.Px7 - 1) / t.Px7), nb);
    ++pl->launches;
    k_pass_x_stress<T><<<g3, 256, t.smem_x7, pl->stream>>>(w.E, pl->d_ids, ctab_of<T>(pl), tw_of<T>(pl, 0), g, t.Px7);
    ++pl->launches;
    k_pass_axis<T, -1, 1><<<g2, 256, t.smem_y2, pl->stream>>>(w.E, w.E, tw_of<T>(pl, 1), g, t.Py2, T(1));
    ++pl->launches;
    k_pass_z_div<T><<<g1, 256, t.smem_z5, pl->stream>>>(w.E, out, w.qtab, tw_of<T>(pl, 2), g, t.Pz5, out_scale);
}

// Float-float operator: the shared-memory z and x passes; the two-stage
// register y passes where the y axis has one (fft_variant 0)
template <>
int launch_K<dfloat>(bloch_plan* pl, int nb, const dfloat2* u, dfloat2* out, dfloat out_scale, const dfloat2*,
                     double2*) {
    using T = dfloat;
    if (!pl->fast || !fast_axis(pl->Ny)) {
        launch_K_generic<T>(pl, nb, u, out, out_scale);
        return 0;
    }
    Workspace<T>& w = ws_of<T>(pl);
    const Geo& g = geo_of<T>(pl);
    const TileCfg& t = tile_of<T>(pl);
    const long long pxy = (long long)pl->Nx * pl->Ny, pyz = (long long)pl->Ny * pl->Nz;
    dim3 g1((unsigned)((pxy + t.Pz5 - 1) / t.Pz5), nb);
    dim3 g3((unsigned)((pyz + t.Px7 - 1) / t.Px7), nb);
    ++pl->launches;
    k_pass_z_strain<T><<<g1, 256, t.smem_z5, pl->stream>>>(u, w.E, w.qtab, tw_of<T>(pl, 2), g, t.Pz5);
    BLOCH_FAST_SWITCH(pl->Ny, fast_y, pl, +1, nb, w.E);
    ++pl->launches;
    k_pass_x_stress<T><<<g3, 256, t.smem_x7, pl->stream>>>(w.E, pl->d_ids, ctab_of<T>(pl), tw_of<T>(pl, 0), g, t.Px7);
    BLOCH_FAST_SWITCH(pl->Ny, fast_y, pl, -1, nb, w.E);
    ++pl->launches;
    k_pass_z_div<T><<<g1, 256, t.smem_z5, pl->stream>>>(w.E, out, w.qtab, tw_of<T>(pl, 2), g, t.Pz5, out_scale);
    return 0;
}

// Fourier-space stress of nb systems whose q tables are set, into the
// operator workspace E (6 components per system, Voigt order xx yy zz yz xz
// xy): S = F{ C~(x) : F^-1(sym q (x) u) }, i.e. the K-apply's passes 1-4 and a
// forward z transform of the six stress components in place of its
// divergence.  Shared-memory passes (any grid, both precisions).
template <typename T>
void launch_K_stress(bloch_plan* pl, int nb, const cplx_t<T>* u) {
    Workspace<T>& w = ws_of<T>(pl);
    const Geo& g = geo_of<T>(pl);
    const TileCfg& t = tile_of<T>(pl);
    const long long pxy = (long long)pl->Nx * pl->Ny, pxz = (long long)pl->Nx * pl->Nz,
                    pyz = (long long)pl->Ny * pl->Nz;
    dim3 g1((unsigned)((pxy + t.Pz5 - 1) / t.Pz5), nb);
    dim3 g2((unsigned)((pxz + t.Py2 - 1) / t.Py2), nb * 6);
    dim3 g3((unsigned)((pyz + t.Px7 - 1) / t.Px7), nb);
    dim3 gz((unsigned)((pxy + t.Pz2 - 1) / t.Pz2), nb * 6);
    pl->launches += 5;
    k_pass_z_strain<T><<<g1, 256, t.smem_z5, pl->stream>>>(u, w.E, w.qtab, tw_of<T>(pl, 2), g, t.Pz5);
    k_pass_axis<T, +1, 1><<<g2, 256, t.smem_y2, pl->stream>>>(w.E, w.E, tw_of<T>(pl, 1), g, t.Py2, T(1));
    k_pass_x_stress<T><<<g3, 256, t.smem_x7, pl->stream>>>(w.E, pl->d_ids, ctab_of<T>(pl), tw_of<T>(pl, 0), g, t.Px7);
    k_pass_axis<T, -1, 1><<<g2, 256, t.smem_y2, pl->stream>>>(w.E, w.E, tw_of<T>(pl, 1), g, t.Py2, T(1));
    k_pass_axis<T, -1, 2><<<gz, 256, t.smem_z2, pl->stream>>>(w.E, w.E, tw_of<T>(pl, 2), g, t.Pz2, T(1));
}

// In-place 3D FFT of nb three-component fields (DIR -1 forward, +1 inverse;
// unnormalised), times out_scale: shared-memory passes along z, y and x.
template <typename T, int DIR>
void launch_fft3(bloch_plan* pl, int nb, cplx_t<T>* W, T out_scale) {
    const Geo& g = geo_of<T>(pl);
    const TileCfg& t = tile_of<T>(pl);
    const long long pxy = (long long)pl->Nx * pl->Ny, pxz = (long long)pl->Nx * pl->Nz,
                    pyz = (long long)pl->Ny * pl->Nz;
    dim3 gz((unsigned)((pxy + t.Pz2 - 1) / t.Pz2), nb * 3);
    dim3 gy((unsigned)((pxz + t.Py2 - 1) / t.Py2), nb * 3);
    dim3 gx((unsigned)((pyz + t.Px4 - 1) / t.Px4), nb);
    pl->launches += 3;
    k_pass_axis<T, DIR, 2><<<gz, 256, t.smem_z2, pl->stream>>>(W, W, tw_of<T>(pl, 2), g, t.Pz2, T(1));
    k_pass_axis<T, DIR, 1><<<gy, 256, t.smem_y2, pl->stream>>>(W, W, tw_of<T>(pl, 1), g, t.Py2, T(1));
    k_pass_x<T, DIR><<<gx, 256, t.smem_x4, pl->stream>>>(W, tw_of<T>(pl, 0), g, t.Px4, out_scale);
}

template <typename T>
void launch_M(bloch_plan* pl, int nb, const cplx_t<T>* u, cplx_t<T>* out, T out_scale) {
    const long long n = (long long)nb * 3 * pl->V;
    if (pl->uniform_rho) {
        const int blocks = (int)std::min<long long>(4096, (n + 255) / 256);
        ++pl->launches;
        k_scale<T><<<blocks, 256, 0, pl->stream>>>(
            u, out, T(pl->rho_uniform_scaled * static_cast<double>(out_scale)), (size_t)n);
        return;
    }
    Workspace<T>& w = ws_of<T>(pl);
    const Geo& g = geo_of<T>(pl);
    const TileCfg& t = tile_of<T>(pl);
    const long long pxy = (long long)pl->Nx * pl->Ny, pxz = (long long)pl->Nx * pl->Nz,
                    pyz = (long long)pl->Ny * pl->Nz;
    dim3 gz((unsigned)((pxy + t.Pz2 - 1) / t.Pz2), nb * 3);
    dim3 gy((unsigned)((pxz + t.Py2 - 1) / t.Py2), nb * 3);
    dim3 gx((unsigned)((pyz + t.Px4 - 1) / t.Px4), nb);
    ++pl->launches;
    k_pass_axis<T, +1, 2><<<gz, 256, t.smem_z2, pl->stream>>>(u, w.E, tw_of<T>(pl, 2), g, t.Pz2, T(1));
    ++pl->launches;
    k_pass_axis<T, +1, 1><<<gy, 256, t.smem_y2, pl->stream>>>(w.E, w.E, tw_of<T>(pl, 1), g, t.Py2, T(1));
    ++pl->launches;
    k_pass_x_rho<T><<<gx, 256, t.smem_x4, pl->stream>>>(w.E, pl->d_ids, rtab_of<T>(pl), tw_of<T>(pl, 0), g, t.Px4);
    ++pl->launches;
    k_pass_axis<T, -1, 1><<<gy, 256, t.smem_y2, pl->stream>>>(w.E, w.E, tw_of<T>(pl, 1), g, t.Py2, T(1));
    ++pl->launches;
    k_pass_axis<T, -1, 2><<<gz, 256, t.smem_z2, pl->stream>>>(w.E, out, tw_of<T>(pl, 2), g, t.Pz2, out_scale);
}

template <typename T>
void launch_precond(bloch_plan* pl, int nb, const cplx_t<T>* r, cplx_t<T>* z, T out_scale) {
    dim3 gr(vec_blocks(pl, nb), nb);
    ++pl->launches;
    k_precond<T><<<gr, 256, 0, pl->stream>>>(r, z, ws_of<T>(pl).qtab, geo_of<T>(pl), pl->pc, pl->psel, out_scale);
}

template <typename T>
void launch_dot(bloch_plan* pl, int nb, const cplx_t<T>* a, const cplx_t<T>* c, long long n_per, double2* out,
                double2* partial) {
    const int nblk = vec_blocks(pl, nb);
    dim3 gr(nblk, nb);
    ++pl->launches;
    k_dot_partial<T><<<gr, 256, 0, pl->stream>>>(a, c, n_per, partial);
    ++pl->launches;
    k_dot_final<<<nb, 256, 0, pl->stream>>>(partial, nblk, out);
}

// ------------------------------------------------------------ PCG (Algorithm 2)
// Loop condition of the graph-resident PCG: continue while a system is active
// and the iteration cap is not reached (the cap bounds every launch).
static __global__ void k_cg_cond(cudaGraphConditionalHandle h, const int* __restrict__ n_active, int* iter,
                                 int max_iter) {
    const int i = ++(*iter);
    cudaGraphSetConditional(h, (*n_active > 0 && i < max_iter) ? 1u : 0u);
}

// One PCG iteration (operator, (p, Ap), alpha, updates, beta, p-update, loop
// condition) enqueued on the plan's stream; captured into the WHILE body.
template <typename T>
static void pcg_iteration(bloch_plan* pl, int nb, cplx_t<T>* x, double tol2, int nblk,
                          cudaGraphConditionalHandle* h, int max_iter) {
    Workspace<T>& w = ws_of<T>(pl);
    const Geo& g = geo_of<T>(pl);
    dim3 gr(nblk, nb);
    // A p for the systems still active (the passes skip converged ones), with
    // the (p, A p) partials fused into the last pass where it can
    static_assert(sizeof(CGSys) % sizeof(int) == 0, "CGSys must be a whole number of ints");
    Geo& gk = std::is_same<T, float>::value ? pl->geo_f : pl->geo_d;
    gk.skip = &w.sys[0].active;
    gk.skip_stride = (int)(sizeof(CGSys) / sizeof(int));
    gk.skip_ncomp = 6;
    const int zb = launch_K<T>(pl, nb, w.p, w.Ap, T(1), w.p, w.partz);
    gk.skip = nullptr;
    gk.skip_stride = 1;
    gk.skip_ncomp = 1;
    if (zb > 0) {
        ++pl->launches;
        k_dot_final<<<nb, 256, 0, pl->stream>>>(w.partz, zb, w.dots);
    } else {
        launch_dot<T>(pl, nb, w.p, w.Ap, 3 * pl->V, w.dots, w.part2);
    }
    ++pl->launches;
    k_cg_scalars<<<nb, 32, 0, pl->stream>>>(w.part3, w.dots, nblk, w.sys, 1, tol2, pl->d_nactive);
    ++pl->launches;
    k_cg_update<T><<<gr, 256, 0, pl->stream>>>(w.r, w.Ap, w.qtab, g, pl->pc, pl->psel, w.sys, w.part3);
    // (mode 1 above zeroed the active count that mode 2 accumulates)
    ++pl->launches;
    k_cg_scalars<<<nb, 256, 0, pl->stream>>>(w.part3, w.dots, nblk, w.sys, 2, tol2, pl->d_nactive);
    ++pl->launches;
    k_cg_pupdate<T><<<gr, 256, 0, pl->stream>>>(w.r, w.p, x, w.qtab, g, pl->pc, pl->psel, w.sys);
    if (h) {
        ++pl->launches;
        k_cg_cond<<<1, 1, 0, pl->stream>>>(*h, pl->d_nactive, pl->d_iter, max_iter);
    }
}

template <typename T>
static bloch_status pcg_graph(bloch_plan* pl, int nb, const cplx_t<T>* b, cplx_t<T>* x, double tol2, int nblk,
                              int max_iter, cudaGraphExec_t* out, int* launches_per_iter) {
    Workspace<T>& w = ws_of<T>(pl);
    const int prec = std::is_same<T, float>::value ? 1 : 0;
    for (auto& e : pl->pcg_graphs)
        if (e.prec == prec && e.nb == nb && e.max_iter == max_iter && e.tol2 == tol2 && e.b == b && e.x == x &&
            e.E == w.E && e.r == w.r && e.ztab == pl->psel.ztab && e.zgroup == pl->psel.zgroup) {
            *out = e.exec;
            *launches_per_iter = e.launches_per_iter;
            return BLOCH_OK;
        }
    if (pl->pcg_graphs.size() >= 16) {
        cudaGraphExecDestroy(pl->pcg_graphs.front().exec);
        cudaGraphDestroy(pl->pcg_graphs.front().graph);
        pl->pcg_graphs.erase(pl->pcg_graphs.begin());
    }
    cudaGraph_t graph;
    BLOCH_CUDA_CHECK_RET(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_cuda_error(e, "cudaGraphConditionalHandleCreate");
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_cuda_error(e, "cudaGraphAddNode (conditional)");
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // capture on the plan's private stream (the caller's stream may be the
    // legacy default stream, which cannot be captured); capturing runs nothing
    e = cudaStreamBeginCaptureToGraph(pl->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_cuda_error(e, "cudaStreamBeginCaptureToGraph");
    }
    const unsigned long long l0 = pl->launches;
    cudaStream_t user = pl->stream;
    pl->stream = pl->cap_stream;
    pcg_iteration<T>(pl, nb, x, tol2, nblk, &h, max_iter);
    pl->stream = user;
    const int per_iter = (int)(pl->launches - l0);
    pl->launches = l0;   // counted per executed iteration, not at capture
    cudaGraph_t captured;
    e = cudaStreamEndCapture(pl->cap_stream, &captured);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_cuda_error(e, "cudaStreamEndCapture");
    }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return set_cuda_error(e, "cudaGraphInstantiate");
    }
    bloch_plan::PcgGraph pg{prec, nb, max_iter, per_iter, tol2, b, x, w.E, w.r, pl->psel.ztab, pl->psel.zgroup,
                            graph, exec};
    pl->pcg_graphs.push_back(pg);
    *out = exec;
    *launches_per_iter = per_iter;
    return BLOCH_OK;
}

template <typename T>
bloch_status pcg_run(bloch_plan* pl, int nb, const cplx_t<T>* b, cplx_t<T>* x, double rhs_scale, double tol,
                     int max_iter, bool use_x0, int* iters, double* relres, long long* total_iters,
                     void (*hook)(void*, int), void* hook_ctx) {
    bloch_status st = ensure_cg<T>(pl, nb);
    if (st != BLOCH_OK) return st;
    TraceScope trace_pcg(pl, pl->trace_pcg);
    Workspace<T>& w = ws_of<T>(pl);
    const Geo& g = geo_of<T>(pl);
    const int nblk = vec_blocks(pl, nb);
    dim3 gr(nblk, nb);
    const double tol2 = tol * tol;
    if (use_x0) launch_K<T>(pl, nb, x, w.Ap, T(1));
    ++pl->launches;
    k_cg_init<T><<<gr, 256, 0, pl->stream>>>(b, use_x0 ? w.Ap : nullptr, x, w.r, w.p, w.qtab, g, pl->pc, pl->psel,
                                              T(rhs_scale), use_x0 ? 0 : 1, w.part3);
    BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(pl->d_nactive, 0, sizeof(int), pl->stream));
    ++pl->launches;
    k_cg_scalars<<<nb, 256, 0, pl->stream>>>(w.part3, w.dots, nblk, w.sys, 0, tol2, pl->d_nactive);
    BLOCH_CUDA_CHECK_RET(
        cudaMemcpyAsync(pl->h_nactive, pl->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
    BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
    if (hook) hook(hook_ctx, 0);
    int it = 0;
    long long tot = 0;
    // graph-resident loop (not with a per-iteration host hook, nor with the
    // cuFFT baseline, whose plans are created on first use)
    const bool use_graph = pl->opt.cuda_graph != 0 && hook == nullptr && pl->variant != 2;
    if (use_graph && *pl->h_nactive > 0 && max_iter > 0) {
        cudaGraphExec_t exec;
        int per_iter = 0;
        bloch_status gs = pcg_graph<T>(pl, nb, b, x, tol2, nblk, max_iter, &exec, &per_iter);
        if (gs != BLOCH_OK) return gs;
        BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(pl->d_iter, 0, sizeof(int), pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaGraphLaunch(exec, pl->stream));
        int iters_done = 0;
        BLOCH_CUDA_CHECK_RET(
            cudaMemcpyAsync(&iters_done, pl->d_iter, sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
        pl->launches += (unsigned long long)iters_done * per_iter;
        it = iters_done;
    }
    while (!use_graph && *pl->h_nactive > 0 && it < max_iter) {
        tot += *pl->h_nactive;
        pcg_iteration<T>(pl, nb, x, tol2, nblk, nullptr, max_iter);
        BLOCH_CUDA_CHECK_RET(
            cudaMemcpyAsync(pl->h_nactive, pl->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
        ++it;
        if (hook) hook(hook_ctx, it);
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
    }
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    if (pl->pending != BLOCH_OK) {
        const bloch_status p = pl->pending;
        pl->pending = BLOCH_OK;
        return p;
    }
    std::vector<CGSys> hs(nb);
    BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(hs.data(), w.sys, sizeof(CGSys) * nb, cudaMemcpyDeviceToHost, pl->stream));
    BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
    bool all = true, finite = true;
    for (int i = 0; i < nb; ++i) {
        const double rel = hs[i].bb > 0 ? std::sqrt(std::max(hs[i].rr, 0.0) / hs[i].bb) : 0.0;
        if (!std::isfinite(hs[i].rr) || !std::isfinite(hs[i].bb)) finite = false;
        if (iters) iters[i] = hs[i].iters;
        if (relres) relres[i] = rel;
        if (!(rel <= tol)) all = false;
    }
    if (use_graph) {
        tot = 0;
        for (int i = 0; i < nb; ++i) tot += hs[i].iters;
    }
    if (total_iters) *total_iters += tot;
    if (!finite) return set_error(BLOCH_ENONFINITE, "PCG met a non-finite residual");
    if (!all) return set_error(BLOCH_ENOTCONV_CG, "PCG reached its iteration cap before the tolerance");
    return BLOCH_OK;
}

template <typename T>
bloch_status pcg_enqueue(bloch_plan* pl, int nb, const cplx_t<T>* b, cplx_t<T>* x, double rhs_scale, double tol,
                         int max_iter, long long* tally) {
    const double tol2 = tol * tol;
    if (pl->opt.cuda_graph == 0 || pl->variant == 2 || max_iter <= 0) {
        // host-driven loop: synchronises per iteration; the tally is added on the host
        long long it = 0;
        bloch_status st = pcg_run<T>(pl, nb, b, x, rhs_scale, tol, max_iter, false, nullptr, nullptr, &it);
        if (st != BLOCH_OK && st != BLOCH_ENOTCONV_CG) return st;
        long long add[4] = {it, st == BLOCH_ENOTCONV_CG ? 1 : 0, 0, 0};
        long long cur[4];
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(cur, tally, sizeof(cur), cudaMemcpyDeviceToHost, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
        for (int i = 0; i < 4; ++i) cur[i] += add[i];
        BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(tally, cur, sizeof(cur), cudaMemcpyHostToDevice, pl->stream));
        BLOCH_CUDA_CHECK_RET(cudaStreamSynchronize(pl->stream));
        return BLOCH_OK;
    }
    bloch_status st = ensure_cg<T>(pl, nb);
    if (st != BLOCH_OK) return st;
    TraceScope trace_pcg(pl, pl->trace_pcg);
    Workspace<T>& w = ws_of<T>(pl);
    const Geo& g = geo_of<T>(pl);
    const int nblk = vec_blocks(pl, nb);
    dim3 gr(nblk, nb);
    ++pl->launches;
    k_cg_init<T><<<gr, 256, 0, pl->stream>>>(b, nullptr, x, w.r, w.p, w.qtab, g, pl->pc, pl->psel, T(rhs_scale), 1,
                                              w.part3);
    BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(pl->d_nactive, 0, sizeof(int), pl->stream));
    ++pl->launches;
    k_cg_scalars<<<nb, 256, 0, pl->stream>>>(w.part3, w.dots, nblk, w.sys, 0, tol2, pl->d_nactive);
    cudaGraphExec_t exec;
    int per_iter = 0;
    if ((st = pcg_graph<T>(pl, nb, b, x, tol2, nblk, max_iter, &exec, &per_iter)) != BLOCH_OK) return st;
    BLOCH_CUDA_CHECK_RET(cudaMemsetAsync(pl->d_iter, 0, sizeof(int), pl->stream));
    BLOCH_CUDA_CHECK_RET(cudaGraphLaunch(exec, pl->stream));
    // launches are counted per executed iteration by the caller's tally
    pl->launches += 1;
    k_cg_tally<<<1, 32, 0, pl->stream>>>(w.sys, nb, tol2, pl->d_iter, tally);
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    pl->pcg_launches_per_iter = per_iter;
    return BLOCH_OK;
}

#define INST(T)                                                                                          \
    template bloch_status ensure_ws<T>(bloch_plan*, int);                                                \
    template bloch_status ensure_cg<T>(bloch_plan*, int);                                                \
    template bloch_status set_k<T>(bloch_plan*, int, const double*);                                     \
    template int launch_K<T>(bloch_plan*, int, const cplx_t<T>*, cplx_t<T>*, T, const cplx_t<T>*, double2*); \
    template void launch_M<T>(bloch_plan*, int, const cplx_t<T>*, cplx_t<T>*, T);                        \
    template void launch_K_stress<T>(bloch_plan*, int, const cplx_t<T>*);                                 \
    template void launch_fft3<T, -1>(bloch_plan*, int, cplx_t<T>*, T);                                   \
    template void launch_fft3<T, +1>(bloch_plan*, int, cplx_t<T>*, T);                                   \
    template void launch_precond<T>(bloch_plan*, int, const cplx_t<T>*, cplx_t<T>*, T);                  \
    template void launch_dot<T>(bloch_plan*, int, const cplx_t<T>*, const cplx_t<T>*, long long,         \
                                double2*, double2*);                                                     \
    template bloch_status pcg_run<T>(bloch_plan*, int, const cplx_t<T>*, cplx_t<T>*, double, double, int, \
                                     bool, int*, double*, long long*, void (*)(void*, int), void*);       \
    template bloch_status pcg_enqueue<T>(bloch_plan*, int, const cplx_t<T>*, cplx_t<T>*, double, double, int, \
                                         long long*);
INST(float)
INST(double)
#undef INST
template bloch_status ensure_ws<dfloat>(bloch_plan*, int);
template bloch_status set_k<dfloat>(bloch_plan*, int, const double*);
template void launch_M<dfloat>(bloch_plan*, int, const dfloat2*, dfloat2*, dfloat);

}  // namespace bloch

using namespace bloch;

// ============================================================== C ABI
template <typename T>
static bloch_status apply_K_real_impl(bloch_plan* pl, int nb, const double* k, const cplx_t<T>* u, cplx_t<T>* Ku) {
    bloch_status st = ensure_cg<T>(pl, nb);
    if (st != BLOCH_OK) return st;
    if ((st = set_k<T>(pl, nb, k)) != BLOCH_OK) return st;
    Workspace<T>& w = ws_of<T>(pl);
    BLOCH_CUDA_CHECK_RET(cudaMemcpyAsync(w.Ap, u, sizeof(cplx_t<T>) * (size_t)nb * 3 * pl->V,
                                         cudaMemcpyDeviceToDevice, pl->stream));
    launch_fft3<T, -1>(pl, nb, w.Ap, T(1));                       // u^ = F u
    launch_K<T>(pl, nb, w.Ap, Ku, T(pl->Kscale));                 // A_k u^
    launch_fft3<T, +1>(pl, nb, Ku, T(1.0 / (double)pl->V));       // F^-1
    return BLOCH_OK;
}

extern "C" {

void bloch_default_options(bloch_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = BLOCH_FP64;
    opt->method = BLOCH_SUBSPACE;
    opt->tol_lin = 1e-10;
    opt->tol_eig = 1e-10;
    opt->max_cg = 2000;
    opt->max_outer = 500;
    opt->block = 0;
    opt->k_batch = 0;
    opt->ncv = 0;
    opt->warm_start = 1;
    opt->cuda_graph = 1;
    opt->fft_variant = 0;
}

const char* bloch_last_error(void) { return g_last_error.c_str(); }

size_t bloch_plan_device_bytes(const bloch_plan* plan) { return plan ? plan->device_bytes : 0; }

uint64_t bloch_plan_kernel_launches(const bloch_plan* plan) { return plan ? plan->launches : 0; }

static void free_ws_all(bloch_plan* pl) {
    auto fr = [](auto& w) {
        cudaFree(w.E);
        cudaFree(w.qtab);
        cudaFree(w.kvec);
        cudaFree(w.r);
        cudaFree(w.p);
        cudaFree(w.Ap);
        cudaFree(w.part3);
        cudaFree(w.part2);
        cudaFree(w.dots);
        cudaFree(w.sys);
    };
    fr(pl->ws_f);
    fr(pl->ws_d);
    fr(pl->ws_x);
}

void bloch_plan_destroy(bloch_plan* pl) {
    if (!pl) return;
    cudaStreamSynchronize(pl->stream);
    cufft_release(pl);
    drop_pcg_graphs(pl);
    trace_release(pl);
    cudaFree(pl->d_iter);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    free_ws_all(pl);
    cudaFree(pl->d_xi);
    cudaFree(pl->d_ids);
    cudaFree(pl->d_Cf);
    cudaFree(pl->d_Cd);
    cudaFree(pl->d_Cpf);
    cudaFree(pl->d_Cpd);
    cudaFree(pl->d_rf);
    cudaFree(pl->d_rd);
    for (int a = 0; a < 3; ++a) {
        cudaFree(pl->d_twf[a]);
        cudaFree(pl->d_twd[a]);
        cudaFree(pl->d_twx[a]);
    }
    cudaFree(pl->d_Cx);
    cudaFree(pl->d_rx);
    cudaFree(pl->d_nactive);
    cudaFree(pl->d_perr);
    cudaFreeHost(pl->h_nactive);
    cudaFree(pl->d_ztab);
    cudaFree(pl->d_handoff);
    plan_solver_release(pl);
    delete pl;
}

static bool cholesky_pd(const double* A6) {
    double L[36] = {0};
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A6[i * 6 + j];
            for (int k = 0; k < j; ++k) s -= L[i * 6 + k] * L[j * 6 + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i * 6 + i] = std::sqrt(s);
            } else {
                L[i * 6 + j] = s / L[j * 6 + j];
            }
        }
    return true;
}

bloch_status bloch_plan_create(bloch_plan** out, const int32_t grid[3], const double L[3], const int32_t* grain_ids,
                               int32_t G, const double* C_per_grain, const double* rho, const bloch_options* opt,
                               void* cuda_stream) {
    if (!out) return set_error(BLOCH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !L || !grain_ids || !C_per_grain || !rho) return set_error(BLOCH_EINVAL, "NULL argument");
    for (int a = 0; a < 3; ++a) {
        if (grid[a] < 1) return set_error(BLOCH_EINVAL, "grid sizes must be >= 1");
        if (grid[a] > 512 || !factor_ok(grid[a]))
            return set_error(BLOCH_EUNSUPPORTED, "grid sizes must be <= 512 with prime factors in {2,3,5,7}");
        if (!(L[a] > 0.0) || !std::isfinite(L[a])) return set_error(BLOCH_EINVAL, "cell lengths must be > 0");
    }
    if (G < 1) return set_error(BLOCH_EINVAL, "G must be >= 1");
    const long long V = (long long)grid[0] * grid[1] * grid[2];
    for (int g = 0; g < G; ++g) {
        const double* C = C_per_grain + (size_t)g * 36;
        double mx = 0;
        for (int i = 0; i < 36; ++i) {
            if (!std::isfinite(C[i])) return set_error(BLOCH_ENONFINITE, "stiffness has a non-finite entry");
            mx = std::max(mx, std::fabs(C[i]));
        }
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < i; ++j)
                if (std::fabs(C[i * 6 + j] - C[j * 6 + i]) > 1e-10 * mx)
                    return set_error(BLOCH_EINVAL, "stiffness of grain " + std::to_string(g) + " is not symmetric");
        if (!cholesky_pd(C))
            return set_error(BLOCH_EINVAL, "stiffness of grain " + std::to_string(g) + " is not positive definite");
        if (!(rho[g] > 0.0) || !std::isfinite(rho[g]))
            return set_error(BLOCH_EINVAL, "density of grain " + std::to_string(g) + " must be > 0");
    }
    std::vector<long long> counts(G, 0);
    for (long long v = 0; v < V; ++v) {
        const int id = grain_ids[v];
        if (id < 0 || id >= G) return set_error(BLOCH_EINVAL, "grain id out of range at voxel " + std::to_string(v));
        counts[id]++;
    }

    bloch_plan* pl = new bloch_plan();
    pl->Nx = grid[0];
    pl->Ny = grid[1];
    pl->Nz = grid[2];
    pl->V = V;
    for (int a = 0; a < 3; ++a) pl->L[a] = L[a];
    pl->G = G;
    if (opt) pl->opt = *opt;
    else bloch_default_options(&pl->opt);
    if (pl->opt.tile_pmax != 0 && pl->opt.tile_pmax != 4 && pl->opt.tile_pmax != 8 && pl->opt.tile_pmax != 16 &&
        pl->opt.tile_pmax != 32) {
        delete pl;
        return set_error(BLOCH_EINVAL, "tile_pmax must be 0, 4, 8, 16 or 32");
    }
    if (!(pl->opt.hybrid_tol >= 0.0) || !(pl->opt.hybrid_tol < 1.0)) {
        delete pl;
        return set_error(BLOCH_EINVAL, "hybrid_tol must be in [0, 1)");
    }
    if (pl->opt.tensor_gram != 0 && pl->opt.tensor_gram != 1) {
        delete pl;
        return set_error(BLOCH_EINVAL, "tensor_gram must be 0 or 1");
    }
    if (pl->opt.fft_variant < 0 || pl->opt.fft_variant > 2) {
        delete pl;
        return set_error(BLOCH_EINVAL, "fft_variant must be 0, 1 or 2");
    }
    if (pl->opt.refine_arith != 0 && pl->opt.refine_arith != 1) {
        delete pl;
        return set_error(BLOCH_EINVAL, "refine_arith must be 0 or 1");
    }
    pl->stream = (cudaStream_t)cuda_stream;
    std::memset(&pl->last_stats, 0, sizeof(pl->last_stats));
    pl->ids_host.assign(grain_ids, grain_ids + V);
    pl->C_host.assign(C_per_grain, C_per_grain + (size_t)G * 36);
    pl->rho_host.assign(rho, rho + G);

    // volume averages (Section 3.3: C0 is the volume-averaged stiffness)
    double rbar = 0;
    for (int i = 0; i < 36; ++i) pl->C0V[i] = 0;
    for (int g = 0; g < G; ++g) {
        const double w = (double)counts[g] / (double)V;
        for (int i = 0; i < 36; ++i) pl->C0V[i] += w * C_per_grain[(size_t)g * 36 + i];
        rbar += w * rho[g];
    }
    pl->uniform_rho = true;
    for (int g = 0; g < G; ++g)
        if (counts[g] > 0 && rho[g] != rho[grain_ids[0]]) pl->uniform_rho = false;
    pl->rho_ref = rbar;
    pl->rho_uniform_scaled = rho[grain_ids[0]] / rbar;
    pl->qscale = std::max(L[0], std::max(L[1], L[2])) / (2.0 * M_PI);
    pl->Cref = std::max(pl->C0V[0], std::max(pl->C0V[7], pl->C0V[14]));
    pl->Kscale = pl->Cref / (pl->qscale * pl->qscale);

    // preconditioner coefficients from the scaled C0 tensor
    {
        static const int vi[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
        static const int pr[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
        for (int a = 0; a < 6; ++a) {
            const int i = pr[a][0], k = pr[a][1];
            for (int m = 0; m < 6; ++m) {
                const int j = pr[m][0], l = pr[m][1];
                double c = pl->C0V[vi[i][j] * 6 + vi[k][l]];
                if (j != l) c += pl->C0V[vi[i][l] * 6 + vi[k][j]];
                pl->pc.a[a][m] = c / pl->Cref;
                pl->pc.af[a][m] = (float)pl->pc.a[a][m];
            }
        }
    }

    // frequencies (Eq. frequencies, FFT bin order)
    pl->xi_host.resize(pl->Nx + pl->Ny + pl->Nz);
    {
        int o = 0;
        for (int a = 0; a < 3; ++a) {
            const int N = grid[a];
            for (int m = 0; m < N; ++m) {
                const int mt = m < (N + 1) / 2 ? m : m - N;
                pl->xi_host[o++] = 2.0 * M_PI / L[a] * mt;
            }
        }
    }

    auto fail = [&](bloch_status st) {
        bloch_plan_destroy(pl);
        return st;
    };
    cudaError_t e;
#define CK(expr)                                                       \
    if ((e = (expr)) != cudaSuccess) return fail(set_cuda_error(e, #expr));
    size_t* acc = &pl->device_bytes;
    CK(dmalloc(&pl->d_xi, pl->xi_host.size(), acc));
    CK(cudaMemcpy(pl->d_xi, pl->xi_host.data(), sizeof(double) * pl->xi_host.size(), cudaMemcpyHostToDevice));
    CK(dmalloc(&pl->d_ids, (size_t)V, acc));
    CK(cudaMemcpy(pl->d_ids, grain_ids, sizeof(int32_t) * V, cudaMemcpyHostToDevice));
    {
        std::vector<double> cd((size_t)G * 36);
        std::vector<float> cf((size_t)G * 36);
        std::vector<double> rd(G);
        std::vector<float> rf(G);
        for (size_t i = 0; i < cd.size(); ++i) {
            cd[i] = C_per_grain[i] / (pl->Cref * (double)V);
            cf[i] = (float)cd[i];
        }
        for (int g = 0; g < G; ++g) {
            rd[g] = rho[g] / (pl->rho_ref * (double)V);
            rf[g] = (float)rd[g];
        }
        std::vector<double> pd((size_t)G * 21);
        std::vector<float> pf((size_t)G * 21);
        for (int g = 0; g < G; ++g) {
            int k = 0;
            for (int i = 0; i < 6; ++i)
                for (int j = i; j < 6; ++j, ++k) {
                    pd[(size_t)g * 21 + k] = cd[(size_t)g * 36 + i * 6 + j];
                    pf[(size_t)g * 21 + k] = (float)pd[(size_t)g * 21 + k];
                }
        }
        CK(dmalloc(&pl->d_Cpd, pd.size(), acc));
        CK(dmalloc(&pl->d_Cpf, pf.size(), acc));
        CK(cudaMemcpy(pl->d_Cpd, pd.data(), sizeof(double) * pd.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(pl->d_Cpf, pf.data(), sizeof(float) * pf.size(), cudaMemcpyHostToDevice));
        CK(dmalloc(&pl->d_Cd, cd.size(), acc));
        CK(dmalloc(&pl->d_Cf, cf.size(), acc));
        CK(dmalloc(&pl->d_rd, rd.size(), acc));
        CK(dmalloc(&pl->d_rf, rf.size(), acc));
        CK(cudaMemcpy(pl->d_Cd, cd.data(), sizeof(double) * cd.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(pl->d_Cf, cf.data(), sizeof(float) * cf.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(pl->d_rd, rd.data(), sizeof(double) * rd.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(pl->d_rf, rf.data(), sizeof(float) * rf.size(), cudaMemcpyHostToDevice));
        std::vector<dfloat> cx(cd.size()), rx(rd.size());
        for (size_t i = 0; i < cd.size(); ++i) cx[i] = dfloat(cd[i]);
        for (size_t i = 0; i < rd.size(); ++i) rx[i] = dfloat(rd[i]);
        CK(dmalloc(&pl->d_Cx, cx.size(), acc));
        CK(dmalloc(&pl->d_rx, rx.size(), acc));
        CK(cudaMemcpy(pl->d_Cx, cx.data(), sizeof(dfloat) * cx.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(pl->d_rx, rx.data(), sizeof(dfloat) * rx.size(), cudaMemcpyHostToDevice));
    }
    for (int a = 0; a < 3; ++a) {
        const int N = grid[a];
        std::vector<double2> td(N);
        std::vector<float2> tf(N);
        for (int t = 0; t < N; ++t) {
            const long double ang = -2.0L * 3.141592653589793238462643383279502884L * t / N;
            td[t] = make_double2((double)std::cos(ang), (double)std::sin(ang));
            tf[t] = make_float2((float)td[t].x, (float)td[t].y);
        }
        CK(dmalloc(&pl->d_twd[a], (size_t)N, acc));
        CK(dmalloc(&pl->d_twf[a], (size_t)N, acc));
        CK(cudaMemcpy(pl->d_twd[a], td.data(), sizeof(double2) * N, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(pl->d_twf[a], tf.data(), sizeof(float2) * N, cudaMemcpyHostToDevice));
        std::vector<dfloat2> tx(N);
        for (int t = 0; t < N; ++t) {   // hi/lo split of the twiddle, from the extended-precision angle
            const long double ang = -2.0L * 3.141592653589793238462643383279502884L * t / N;
            const long double c = std::cos(ang), sn = std::sin(ang);
            const float ch = (float)c, sh = (float)sn;
            tx[t] = dfloat2{dfloat(ch, (float)(c - (long double)ch)), dfloat(sh, (float)(sn - (long double)sh))};
        }
        CK(dmalloc(&pl->d_twx[a], (size_t)N, acc));
        CK(cudaMemcpy(pl->d_twx[a], tx.data(), sizeof(dfloat2) * N, cudaMemcpyHostToDevice));
    }
    CK(dmalloc(&pl->d_nactive, 1, acc));
    CK(dmalloc(&pl->d_perr, 1, acc));
    CK(cudaMemset(pl->d_perr, 0, sizeof(int)));
    CK(dmalloc(&pl->d_iter, 1, acc));
    CK(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
    CK(cudaMallocHost((void**)&pl->h_nactive, sizeof(int)));
    CK(set_smem_attrs<float>());
    CK(set_smem_attrs<double>());
    CK(set_smem_attrs<dfloat>());
    set_fast_attrs<float>();
    set_fast_attrs<double>();
    set_fast_attrs<dfloat>();
    pl->fast = pl->opt.fft_variant == 0;
    pl->variant = pl->opt.fft_variant;
#undef CK
    for (Geo* gp : {&pl->geo_f, &pl->geo_d}) {
        gp->Nx = pl->Nx;
        gp->Ny = pl->Ny;
        gp->Nz = pl->Nz;
        gp->V = V;
        gp->dx = make_fastdiv((unsigned)pl->Nx);
        gp->dy = make_fastdiv((unsigned)pl->Ny);
        gp->err = pl->d_perr;
    }
    for (int a = 0; a < 3; ++a) {
        pl->geo_f.ax[a] = make_axis(grid[a], 4);   // radices up to 16 in FP32
        pl->geo_d.ax[a] = make_axis(grid[a], 3);   // up to 8 in FP64 (register budget)
    }
    const int pmax = pl->opt.tile_pmax > 0 ? pl->opt.tile_pmax : kDefaultPmax;
    pl->tile_f = make_tiles<float>(pl->Nx, pl->Ny, pl->Nz, pmax);
    pl->tile_d = make_tiles<double>(pl->Nx, pl->Ny, pl->Nz, pmax);
    pl->nblk_max = vec_blocks(pl, 1);
    *out = pl;
    return BLOCH_OK;
}

static bloch_status check_common(bloch_plan* pl, int nb, int precision, bool ff_ok = false) {
    if (!pl) return set_error(BLOCH_EINVAL, "plan is NULL");
    if (nb < 1 || nb > 65535 / 6) return set_error(BLOCH_EINVAL, "nb must be in [1, 10922]");
    if (precision != BLOCH_FP32 && precision != BLOCH_FP64 && !(ff_ok && precision == BLOCH_FF))
        return set_error(BLOCH_EINVAL, ff_ok ? "precision must be BLOCH_FP32, BLOCH_FP64 or BLOCH_FF"
                                             : "precision must be BLOCH_FP32 or BLOCH_FP64");
    return BLOCH_OK;
}

// scratch of nb float-float three-component vectors (the rounded input of a BLOCH_FF apply)
static bloch_status ensure_cg_ff(bloch_plan* pl, int nb) {
    Workspace<dfloat>& w = pl->ws_x;
    bloch_status st = ensure_ws<dfloat>(pl, nb);
    if (st != BLOCH_OK) return st;
    if (nb <= w.cg_cap) return BLOCH_OK;
    cudaStreamSynchronize(pl->stream);
    if (w.r) pl->device_bytes -= (size_t)w.cg_cap * 3 * pl->V * sizeof(dfloat2);
    cudaFree(w.r);
    w.r = nullptr;
    w.cg_cap = 0;
    BLOCH_CUDA_CHECK_RET(dmalloc(&w.r, (size_t)3 * pl->V * nb, &pl->device_bytes));
    w.cg_cap = nb;
    return BLOCH_OK;
}

bloch_status bloch_apply_K(bloch_plan* pl, int32_t nb, const double* k, int32_t precision, const void* u,
                           void* Ku) {
    bloch_status st = check_common(pl, nb, precision, true);
    if (st != BLOCH_OK) return st;
    if (!k || !u || !Ku) return set_error(BLOCH_EINVAL, "NULL argument");
    if (u == Ku) return set_error(BLOCH_EINVAL, "Ku may not alias u");
    if (precision == BLOCH_FP32) {
        if ((st = set_k<float>(pl, nb, k)) != BLOCH_OK) return st;
        launch_K<float>(pl, nb, (const float2*)u, (float2*)Ku, (float)pl->Kscale);
    } else if (precision == BLOCH_FF) {
        // double2 in, float-float passes (input rounded into a float-float copy), double2 out
        Workspace<dfloat>& w = ws_of<dfloat>(pl);
        if ((st = ensure_cg_ff(pl, nb)) != BLOCH_OK) return st;
        if ((st = set_k<dfloat>(pl, nb, k)) != BLOCH_OK) return st;
        const size_t n = (size_t)nb * 3 * pl->V;
        pl->launches += 2;
        k_convert<double, dfloat><<<2048, 256, 0, pl->stream>>>((const double2*)u, w.r, n);
        launch_K<dfloat>(pl, nb, w.r, (dfloat2*)Ku, dfloat(pl->Kscale));
        k_convert_inplace<dfloat, double><<<2048, 256, 0, pl->stream>>>(Ku, n);
    } else {
        if ((st = set_k<double>(pl, nb, k)) != BLOCH_OK) return st;
        launch_K<double>(pl, nb, (const double2*)u, (double2*)Ku, pl->Kscale);
    }
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    if (pl->pending != BLOCH_OK) {
        const bloch_status p = pl->pending;
        pl->pending = BLOCH_OK;
        return p;
    }
    return BLOCH_OK;
}

bloch_status bloch_apply_K_real(bloch_plan* pl, int32_t nb, const double* k, int32_t precision, const void* u,
                                void* Ku) {
    bloch_status st = check_common(pl, nb, precision);
    if (st != BLOCH_OK) return st;
    if (!k || !u || !Ku) return set_error(BLOCH_EINVAL, "NULL argument");
    if (u == Ku) return set_error(BLOCH_EINVAL, "Ku may not alias u");
    if (precision == BLOCH_FP32)
        st = apply_K_real_impl<float>(pl, nb, k, (const float2*)u, (float2*)Ku);
    else
        st = apply_K_real_impl<double>(pl, nb, k, (const double2*)u, (double2*)Ku);
    if (st != BLOCH_OK) return st;
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    if (pl->pending != BLOCH_OK) {
        const bloch_status p = pl->pending;
        pl->pending = BLOCH_OK;
        return p;
    }
    return BLOCH_OK;
}

bloch_status bloch_apply_M(bloch_plan* pl, int32_t nb, int32_t precision, const void* u, void* Mu) {
    bloch_status st = check_common(pl, nb, precision);
    if (st != BLOCH_OK) return st;
    if (!u || !Mu) return set_error(BLOCH_EINVAL, "NULL argument");
    if (precision == BLOCH_FP32) {
        if ((st = ensure_ws<float>(pl, nb)) != BLOCH_OK) return st;
        launch_M<float>(pl, nb, (const float2*)u, (float2*)Mu, (float)pl->rho_ref);
    } else {
        if ((st = ensure_ws<double>(pl, nb)) != BLOCH_OK) return st;
        launch_M<double>(pl, nb, (const double2*)u, (double2*)Mu, pl->rho_ref);
    }
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    return BLOCH_OK;
}

bloch_status bloch_apply_precond(bloch_plan* pl, int32_t nb, const double* k, int32_t precision, const void* r,
                                 void* z) {
    bloch_status st = check_common(pl, nb, precision);
    if (st != BLOCH_OK) return st;
    if (!k || !r || !z) return set_error(BLOCH_EINVAL, "NULL argument");
    if (precision == BLOCH_FP32) {
        if ((st = set_k<float>(pl, nb, k)) != BLOCH_OK) return st;
        if ((st = lp_activate<float>(pl, nb, 1, 1)) != BLOCH_OK) return st;
        launch_precond<float>(pl, nb, (const float2*)r, (float2*)z, (float)(1.0 / pl->Kscale));
    } else {
        if ((st = set_k<double>(pl, nb, k)) != BLOCH_OK) return st;
        if ((st = lp_activate<double>(pl, nb, 1, 1)) != BLOCH_OK) return st;
        launch_precond<double>(pl, nb, (const double2*)r, (double2*)z, 1.0 / pl->Kscale);
    }
    lp_deactivate(pl);
    BLOCH_CUDA_CHECK_RET(cudaGetLastError());
    return BLOCH_OK;
}

bloch_status bloch_pcg(bloch_plan* pl, int32_t nb, const double* k, int32_t precision, const void* b, void* x,
                       double tol, int32_t max_iter, int32_t use_x0, int32_t* iters, double* rel_res) {
    bloch_status st = check_common(pl, nb, precision);
    if (st != BLOCH_OK) return st;
    if (!k || !b || !x) return set_error(BLOCH_EINVAL, "NULL argument");
    if (!(tol > 0.0) || max_iter < 0) return set_error(BLOCH_EINVAL, "tol must be > 0 and max_iter >= 0");
    if (precision == BLOCH_FP32) {
        if ((st = set_k<float>(pl, nb, k)) != BLOCH_OK) return st;
        if ((st = lp_activate<float>(pl, nb, 1, 1)) != BLOCH_OK) return st;
        st = pcg_run<float>(pl, nb, (const float2*)b, (float2*)x, 1.0 / pl->Kscale, tol, max_iter, use_x0 != 0, iters,
                            rel_res, nullptr);
    } else {
        if ((st = set_k<double>(pl, nb, k)) != BLOCH_OK) return st;
        if ((st = lp_activate<double>(pl, nb, 1, 1)) != BLOCH_OK) return st;
        st = pcg_run<double>(pl, nb, (const double2*)b, (double2*)x, 1.0 / pl->Kscale, tol, max_iter, use_x0 != 0,
                             iters, rel_res, nullptr);
    }
    lp_deactivate(pl);
    if (st == BLOCH_OK || st == BLOCH_ENOTCONV_CG) {
        const bloch_status e = check_pass_err(pl);
        if (e != BLOCH_OK) return e;
    }
    return st;
}

bloch_status bloch_solve_bands(bloch_plan* pl, int32_t n_k, const double* k_list, int32_t n_bands,
                               double* omega_out, void* vecs_out, bloch_stats* stats) {
    if (!pl) return set_error(BLOCH_EINVAL, "plan is NULL");
    if (n_k < 1 || !k_list || !omega_out) return set_error(BLOCH_EINVAL, "n_k >= 1, k_list and omega_out required");
    if (n_bands < 1 || (long long)n_bands >= 3 * pl->V) return set_error(BLOCH_EINVAL, "n_bands must be in [1, 3V)");
    const bloch_status st = bloch_solve_bands_impl(pl, n_k, k_list, n_bands, omega_out, vecs_out, stats);
    if (st == BLOCH_OK || st == BLOCH_ENOTCONV_EIG) {
        const bloch_status e = check_pass_err(pl);
        if (e != BLOCH_OK) return e;
    }
    return st;
}

}  // extern "C"
