// Internal plan structure and operator launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/bloch.h"
#include "fft.cuh"
#include "passes.cuh"
#include "vec.cuh"
#include "fpasses.cuh"

namespace bloch {

bloch_status set_error(bloch_status st, const std::string& msg);
bloch_status set_cuda_error(cudaError_t e, const char* what);

// Per-precision device workspace, grown on demand (capacity in systems).
template <typename T>
struct Workspace {
    using C = cplx_t<T>;
    int cap = 0;            // systems the buffers hold
    C* E = nullptr;         // 6 x V x cap  (FFT-pass intermediates)
    T* qtab = nullptr;      // (Nx+Ny+Nz) x cap
    double* kvec = nullptr; // 3 x cap
    int cg_cap = 0;
    C* r = nullptr;         // 3 x V x cg_cap
    C* p = nullptr;
    C* Ap = nullptr;
    double* part3 = nullptr;  // cg_cap x nblk_max x 3
    double2* part2 = nullptr; // cg_cap x nblk_max
    double2* dots = nullptr;  // cg_cap
    CGSys* sys = nullptr;     // cg_cap
    double2* partz = nullptr; // cg_cap x zblk: (p, Ap) partials of the fused x-stress or z-divergence pass
    int zblk = 0;
};

constexpr int kDefaultPmax = 32;
// threads per CTA of the fast z passes (P = kFastZThreads / RA neighbouring pencils)
constexpr int kFastZThreads = 256;

// Phases of a band solve timed by the tracer (bloch_plan_trace).
enum TracePhase {
    TR_PCG_SUB = 0, TR_PCG_LZ, TR_RES32, TR_RES64, TR_ORTHO, TR_PROJECT, TR_RESTART, TR_SETUP, TR_SPAN, TR_WALL,
    TR_NPHASE
};

// Event-pair timing of solver phases on the plan's stream; pairs are read
// back after the solve's final synchronisation.
struct Tracer {
    bool on = false;
    struct Pair {
        int phase;
        cudaEvent_t a, b;
        bool ended;
    };
    std::vector<Pair> open;
    std::vector<cudaEvent_t> pool;
    double ms[TR_NPHASE] = {};
    long long count[TR_NPHASE] = {};
};

struct TileCfg {
    int pmax;   // cap on pencils per CTA the tiles were made with
    int Pz5;    // pencils per CTA, z passes with 5 buffers (strain / divergence)
    int Py2;    // y pass, 2 buffers
    int Pz2;    // z pass, 2 buffers (mass operator)
    int Px7;    // x stress pass, 7 buffers
    int Px4;    // x rho pass, 4 buffers
    size_t smem_z5, smem_y2, smem_z2, smem_x7, smem_x4;
};

}  // namespace bloch

struct bloch_plan {
    int Nx, Ny, Nz;
    long long V;
    double L[3];
    int G;
    bloch_options opt;
    cudaStream_t stream;

    // unit scaling: q~ = q*qscale, C~ = C/Cref, rho~ = rho/rho_ref
    double qscale, Cref, rho_ref, Kscale;
    bool uniform_rho;
    double rho_uniform_scaled;     // rho/rho_ref when uniform
    double C0V[36];                // volume-averaged Voigt stiffness (Pa)
    bloch::PrecondCoef pc;         // scaled

    std::vector<double> xi_host;   // Nx + Ny + Nz (rad/m, FFT order)
    std::vector<int32_t> ids_host;
    std::vector<double> C_host;    // G x 36 (Pa)
    std::vector<double> rho_host;  // G

    double* d_xi = nullptr;
    int32_t* d_ids = nullptr;
    float* d_Cf = nullptr;
    double* d_Cd = nullptr;
    float* d_Cpf = nullptr;        // G x 21 packed upper triangle (fast x pass)
    double* d_Cpd = nullptr;
    float* d_rf = nullptr;
    double* d_rd = nullptr;
    float2* d_twf[3] = {nullptr, nullptr, nullptr};
    double2* d_twd[3] = {nullptr, nullptr, nullptr};
    // float-float copies (the FP64-class check of the FP32 form on the FP32 pipes)
    dfloat2* d_twx[3] = {nullptr, nullptr, nullptr};
    dfloat* d_Cx = nullptr;
    dfloat* d_rx = nullptr;
    int* d_nactive = nullptr;
    int* d_perr = nullptr;    // pass error word (a staging wait ran out), Geo::err
    int* h_nactive = nullptr;     // pinned

    bloch::Geo geo_f, geo_d;
    bloch::TileCfg tile_f, tile_d;
    int nblk_max;
    bool fast = true;              // use the two-stage register FFT passes where the axis allows
    int variant = 0;               // options.fft_variant, or the autotuner's choice
    bool tuned = false;            // bloch_plan_autotune has configured the passes
    bloch::Tracer trace;           // phase timing (bloch_plan_trace)
    int trace_pcg = 0;             // phase PCG solves are traced under (TR_PCG_SUB or TR_PCG_LZ)
    bloch_status pending = BLOCH_OK;   // failure inside a launcher, reported by the entry point
    // learned preconditioner (bloch_plan_set_preconditioner): parameters and
    // the per-wave-vector Z tables the CG kernels read while it is active
    const struct bloch_lp* lp = nullptr;
    bloch::PrecondSel psel{nullptr, 1};
    float* d_ztab = nullptr;
    size_t zcap = 0;
    std::vector<double> zkey;      // what the current tables were built for (lp_activate)
    std::vector<double> k_host;    // wave vectors (rad/m) of the systems of the last set_k
    // instantiated PCG-loop graphs (conditional WHILE node), keyed by their bound pointers
    struct PcgGraph {
        int prec, nb, max_iter, launches_per_iter;
        double tol2;
        const void *b, *x, *E, *r, *ztab;
        int zgroup;
        cudaGraph_t graph;
        cudaGraphExec_t exec;
    };
    std::vector<PcgGraph> pcg_graphs;
    int* d_iter = nullptr;
    int pcg_launches_per_iter = 0;     // kernels per PCG iteration of the last enqueued graph
    cudaStream_t cap_stream = nullptr;   // private stream used only to capture graphs

    // hand-off block of the FP32 Lanczos -> Algorithm 1 form (chunk x q x 3V float2),
    // kept by the plan and grown on demand
    void* d_handoff = nullptr;
    size_t handoff_bytes = 0;
    // block buffers of the eigensolvers (pool 0: subspace iteration, 1: Lanczos,
    // 2: band properties),
    // kept between bloch_solve_bands calls and grown on demand, so a solve
    // allocates (and synchronises on a free) only when it needs more than before
    struct SolverBuf {
        void* p = nullptr;
        size_t bytes = 0;
    };
    std::vector<SolverBuf> solver_bufs[3];   // pool 2: band properties (bloch_props.cu)
    // (M~ t_0)_0 of the rigid translation t_0 = e_x at bin 0 (V complex, FP64 and
    // FP32), for Gamma with a non-uniform density; built on first use
    void* d_rhohat[2] = {nullptr, nullptr};

    bloch::Workspace<float> ws_f;
    bloch::Workspace<double> ws_d;
    bloch::Workspace<dfloat> ws_x;
    size_t device_bytes = 0;
    unsigned long long launches = 0;   // kernels launched by this plan
    bloch_stats last_stats;
};

namespace bloch {

template <typename T> Workspace<T>& ws_of(bloch_plan* pl);
template <typename T> const Geo& geo_of(const bloch_plan* pl);

// Grow the operator workspace to hold nb systems.
template <typename T> bloch_status ensure_ws(bloch_plan* pl, int nb);
// Grow the PCG workspace to hold nb systems.
template <typename T> bloch_status ensure_cg(bloch_plan* pl, int nb);
// Upload nb wave vectors (host, rad/m) and build the scaled q tables.
template <typename T> bloch_status set_k(bloch_plan* pl, int nb, const double* k_host);
// Scaled stiffness operator on nb systems whose q tables are set: out = out_scale * A~ u.
// With dotp / dpart, a pass that can also forms per-CTA partials of
// sum conj(dotp) * out per system in dpart and the call returns the number of
// partials per system; it returns 0 when no pass did (the caller forms the dot).
template <typename T>
int launch_K(bloch_plan* pl, int nb, const cplx_t<T>* u, cplx_t<T>* out, T out_scale,
             const cplx_t<T>* dotp = nullptr, double2* dpart = nullptr);
// Fourier-space stress S = F{C~ : F^-1(sym q (x) u)} of nb systems (q tables
// set) into the operator workspace E, 6 Voigt components per system.
template <typename T> void launch_K_stress(bloch_plan* pl, int nb, const cplx_t<T>* u);
// In-place 3D FFT of nb three-component fields (DIR -1 forward, +1 inverse,
// unnormalised), times out_scale; shared-memory passes.
template <typename T, int DIR> void launch_fft3(bloch_plan* pl, int nb, cplx_t<T>* W, T out_scale);
// Scaled mass operator: out = out_scale * M~ u (M~ = M / rho_ref).  out may alias u.
template <typename T> void launch_M(bloch_plan* pl, int nb, const cplx_t<T>* u, cplx_t<T>* out, T out_scale);
// Scaled preconditioner on nb systems: z = out_scale * P~^-1 r.
template <typename T> void launch_precond(bloch_plan* pl, int nb, const cplx_t<T>* r, cplx_t<T>* z, T out_scale);
// Batched PCG on the scaled operator: A~ x = rhs_scale * b.
template <typename T>
bloch_status pcg_run(bloch_plan* pl, int nb, const cplx_t<T>* b, cplx_t<T>* x, double rhs_scale, double tol,
                     int max_iter, bool use_x0, int* iters, double* relres, long long* total_iters,
                     void (*hook)(void*, int) = nullptr, void* hook_ctx = nullptr);
// Batched PCG enqueued on the plan's stream with no host synchronisation
// (the loop is the graph's device-side WHILE node; falls back to pcg_run where
// graphs are off).  Adds iterations, missed tolerances, non-finite residuals
// and loop iterations to tally[0..3] (device, long long; the host-loop
// fallback counts its launches itself and adds 0 loop iterations).
template <typename T>
bloch_status pcg_enqueue(bloch_plan* pl, int nb, const cplx_t<T>* b, cplx_t<T>* x, double rhs_scale, double tol,
                         int max_iter, long long* tally);
// dots[b] = sum conj(a_b) c_b over n_per elements per system (device result).
template <typename T>
void launch_dot(bloch_plan* pl, int nb, const cplx_t<T>* a, const cplx_t<T>* c, long long n_per, double2* out,
                double2* partial);

int vec_blocks(const bloch_plan* pl, int nb);

// Tracer: start / end a phase interval on the plan's stream (no-ops when off),
// add host milliseconds to a phase, and read back completed pairs (the stream
// must have been synchronised).  TraceScope brackets a C++ scope.
int trace_begin(bloch_plan* pl, int phase);
void trace_end(bloch_plan* pl, int idx);
void trace_add(bloch_plan* pl, int phase, double ms);
void trace_collect(bloch_plan* pl);
void trace_release(bloch_plan* pl);
struct TraceScope {
    bloch_plan* pl;
    int idx;
    TraceScope(bloch_plan* p, int phase) : pl(p), idx(trace_begin(p, phase)) {}
    ~TraceScope() { trace_end(pl, idx); }
};

// Destroy the instantiated PCG-loop graphs of the plan.
void drop_pcg_graphs(bloch_plan* pl);
// Select the FFT pass variant (0, 1, 2) and the pencils-per-CTA cap of the
// shared-memory passes for both precisions; drops cached graphs.
void configure_passes(bloch_plan* pl, int variant, int pmax);
// Whether the fast (two-stage register) passes serve at least one pass of the
// chain in this precision, and whether a shared-memory pass remains in it.
bool has_fast_pass(const bloch_plan* pl, int precision);
// CTAs per system of the fast FP32 z passes (0 when they do not serve the plan).
int fast_z_blocks(const bloch_plan* pl);
bool has_generic_pass(const bloch_plan* pl, int precision);

// plain-form baseline (bloch_cufft.cu): Eq. (hatA) with cuFFT 3D transforms
template <typename T>
bool cufft_launch_K(bloch_plan* pl, int nb, const cplx_t<T>* u, cplx_t<T>* out, T out_scale, cplx_t<T>* E,
                    const T* qtab, const T* Ctab, const Geo& g);
void cufft_release(const bloch_plan* pl);

// learned preconditioner (learned.cu): build the Z tables of ntab system
// groups (group t uses the q table of system t * qstride_sys, T-typed q
// tables) and make the CG kernels use them; no-op when no network is set.
template <typename T>
bloch_status lp_activate(bloch_plan* pl, int ntab, int qstride_sys, int zgroup);
void lp_deactivate(bloch_plan* pl);

}  // namespace bloch

namespace bloch {
// eigensolver buffers kept by the plan (bloch_eig.cu): buffer idx of pool, at least bytes
bloch_status plan_solver_buf(bloch_plan* pl, int pool, int idx, size_t bytes, void** out);
size_t plan_solver_bytes(const bloch_plan* pl, int pool);
// Tensor map for the TMA staging of the fast z passes: a complex FP32 field of
// nsc [Nz][Ny * Nx] blocks at base, box P pencils x Nz; false where TMA cannot
// serve (no driver entry point, base or strides not 16-byte multiples, fewer
// than P pencils in a plane), *map then zeroed.
bool encode_zmap(CUtensorMap* map, const void* base, const bloch_plan* pl, long long nsc, int P);
// reads and clears the plan's pass error word (synchronises the plan's stream)
bloch_status check_pass_err(bloch_plan* pl);
void plan_solver_release(bloch_plan* pl);
// (M~ t_0)_0 for the Gamma-point deflation (non-uniform density), built once per precision
template <typename T> bloch_status gamma_rhohat(bloch_plan* pl, const cplx_t<T>** out);
// M-deflate the rigid translations out of nv vectors V (and their M-images MV,
// which must be current; MV is updated too)
template <typename T>
bloch_status gamma_deflate(bloch_plan* pl, int nv, cplx_t<T>* V, cplx_t<T>* MV, double2* d_alpha);
}  // namespace bloch

// eigensolver entry (bloch_eig.cu)
bloch_status bloch_solve_bands_impl(bloch_plan* pl, int n_k, const double* k_list, int n_bands, double* omega_out,
                                    void* vecs_out, bloch_stats* stats);
