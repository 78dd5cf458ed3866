/*
 * bloch.h -- C ABI of the GB300 (sm_103a) FFT-based Bloch-wave dispersion library.
 *
 * The library applies, inverts and diagonalises the Fourier-space Bloch-wave
 * operators of Segurado & Lebensohn, "An FFT-based approach for Bloch wave
 * analysis: application to polycrystals" (arXiv 2106.12487):
 *
 *   stiffness  A_k{U}_i = (xi_j + k_j) F{ C_ijkl(x) F^-1((xi_l + k_l) U_k) }   Section 3.2, Eq. (hatA)
 *   mass       M{U}     = F{ rho(x) F^-1(U) }                                  Section 3.2, Eq. (hatM)
 *   inverse    A_k^-1 by conjugate gradient with the Green-operator
 *              preconditioner P_ik = C0_ijkl (xi+k)_j (xi+k)_l                  Section 3.3, Algorithm 2,
 *                                                                             Eqs. (matrixP), (precond)
 *   bands      the n lowest omega = sqrt(lambda) of A_k U = lambda M U for a
 *              list of wave vectors, by shift-invert Lanczos or subspace
 *              iteration                                                      Section 3.3, Algorithms 1 and 3
 *
 * Conventions shared by every entry point
 *   - grid = {Nx, Ny, Nz}; every field is stored [batch][component][z][y][x]
 *     (x fastest), components (x, y, z); a "vector" is 3*V complex values with
 *     V = Nx*Ny*Nz.  Fourier fields use the standard FFT bin order along each
 *     axis: bin m carries xi = 2*pi/L*(m if m < ceil(N/2) else m - N), which is
 *     the set of Eq. (frequencies).
 *   - Complex values are interleaved (re, im): float2 for BLOCH_FP32 buffers,
 *     double2 for BLOCH_FP64 buffers.  Device pointers must be 16-byte aligned.
 *   - SI units throughout: Pa, kg/m^3, m, rad/m, rad/s.
 *   - Stiffness tables are 6x6 Voigt matrices in the order (11,22,33,23,13,12)
 *     with engineering shear strain (sigma_V = C_V eps_V, eps_V = (e11, e22,
 *     e33, 2e23, 2e13, 2e12)), row-major, symmetric positive definite.
 *   - Ownership: the caller owns every buffer it passes; the plan copies what
 *     it keeps during bloch_plan_create.  Device work is enqueued on the
 *     plan's CUDA stream; entry points that return host results synchronise
 *     that stream before returning.
 *   - Errors: every entry point returns a bloch_status; no exception crosses
 *     the ABI.  bloch_last_error() returns a thread-local message describing
 *     the most recent failure on the calling thread.
 */
#ifndef BLOCH_H
#define BLOCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BLOCH_OK = 0,
    BLOCH_EINVAL = 1,        /* an argument is out of range or inconsistent      */
    BLOCH_ENOMEM = 2,        /* device or host allocation failed                 */
    BLOCH_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed      */
    BLOCH_ENOTCONV_CG = 4,   /* PCG hit its iteration cap before the tolerance   */
    BLOCH_ENOTCONV_EIG = 5,  /* the eigensolver hit its sweep/restart cap        */
    BLOCH_ENONFINITE = 6,    /* NaN or Inf met in inputs or iterates             */
    BLOCH_EUNSUPPORTED = 7   /* grid size with a prime factor > 7 or too large;
                                a block or basis above the solver's limits      */
} bloch_status;

/* BLOCH_FF: double2 buffers, arithmetic in float-float (pairs hi + lo of floats,
   a 48-bit significand, about 4e-15 relative per operation) on the FP32 pipes;
   accepted by bloch_apply_K. */
typedef enum { BLOCH_FP64 = 0, BLOCH_FP32 = 1, BLOCH_FF = 2 } bloch_precision;
typedef enum { BLOCH_LANCZOS = 0, BLOCH_SUBSPACE = 1, BLOCH_LOBPCG = 2 } bloch_method;

typedef struct bloch_plan bloch_plan;   /* opaque; owned by the library */

/* Solver options.  bloch_default_options() fills the defaults listed here. */
typedef struct {
    int32_t precision;   /* BLOCH_FP64: fields and CG in FP64 (the paper's plain form).
                            BLOCH_FP32: fields and CG in FP32 complex with FP32
                            accumulation, then an FP64 Rayleigh-Ritz refinement of the
                            converged block.  Default BLOCH_FP64.                       */
    int32_t method;      /* BLOCH_LANCZOS (shift-invert Lanczos with thick restart, Section
                            3.3), BLOCH_SUBSPACE (Algorithm 1) or BLOCH_LOBPCG (locally
                            optimal block preconditioned CG on the pencil (A_k, M), block
                            [X, W = T R, P] with T the Green preconditioner of Eq.
                            (precond) and a rank-revealing Rayleigh-Ritz; no inner PCG;
                            block q = n + 2 unless set, 3q <= 44, 48 with a uniform
                            density).  Every method handles any density and k = 0.
                            Default BLOCH_SUBSPACE.                                     */
    double tol_lin;      /* PCG stop: ||Y - A U||_2 <= tol_lin ||Y||_2.  Default 1e-10.  */
    double tol_eig;      /* eigensolver stop (see bloch_solve_bands).  Default 1e-10.    */
    int32_t max_cg;      /* PCG iteration cap per solve.  Default 2000.                  */
    int32_t max_outer;   /* sweep cap (subspace) or restart cap (Lanczos).  Default 500. */
    int32_t block;       /* subspace block size q; 0 = min(2n, n+8) (Algorithm 1).      */
    int32_t k_batch;     /* wave vectors advanced together; 0 = choose from free memory. */
    int32_t ncv;         /* Lanczos basis size; 0 = max(2n+1, 20).                       */
    int32_t warm_start;  /* subspace iteration: 1 = the k list is split into k_batch
                            contiguous segments solved in parallel, and within a segment
                            each k starts from the converged block of the previous k
                            (Section 3.3); 0 = every k starts from the plane-wave start
                            vectors.  Default 1.                                        */
    int32_t cuda_graph;  /* 1 = each PCG loop runs as one CUDA graph launch: a conditional
                            WHILE node whose body is one iteration and whose condition is
                            set on the device (systems still active, iteration cap not
                            reached), so no host synchronisation happens per iteration;
                            0 = host-driven loop with one synchronisation per iteration.
                            Default 1.                                                  */
    int32_t fft_variant; /* 0 = two-stage register FFT passes where the axis length is a
                            power of two in [16, 256], shared-memory Stockham passes
                            elsewhere; 1 = shared-memory Stockham passes everywhere;
                            2 = plain-form baseline: cuFFT 3D transforms with unfused
                            pointwise kernels.  All compute the same operator.
                            Default 0.                                                  */
    int32_t autotune;    /* 1 = the first bloch_solve_bands call on the plan runs
                            bloch_plan_autotune (precision of these options, systems =
                            the eigensolver's block size) and keeps its choice of FFT
                            pass variant and tile sizes, overriding fft_variant;
                            0 = use fft_variant as given.  Default 0.                   */
    int32_t tile_pmax;   /* cap on pencils per CTA of the shared-memory passes (z and y
                            passes; x passes use half of it), one of 4, 8, 16, 32; each
                            pass lowers it further to fit its shared-memory budget.
                            0 = 32.  Default 0.                                         */
    int32_t tensor_gram; /* Algorithm 1 projections of FP32 blocks: 1 = on the tensor cores
                            (tcgen05, TF32 inputs split hi + lo so products keep FP32
                            accuracy, FP32 accumulation per CTA, FP64 across CTAs);
                            0 = on the CUDA cores.  FP64 blocks always use the CUDA
                            cores.  Default 0.                                          */
    double hybrid_tol;   /* FP32 with BLOCH_LANCZOS: the Lanczos stage stops once its Ritz
                            estimates reach this relative accuracy and hands its block to
                            the Algorithm 1 refinement, which alone decides convergence
                            (tol_eig).  0 = max(1e-5, 10 tol_eig).  Default 0.          */
    int32_t refine_arith; /* arithmetic of the FP64 check of the FP32 form (the operator
                            applies to the wanted vectors): 0 = IEEE FP64; 1 = float-float
                            operator applies (BLOCH_FF) whose results are summed in FP64
                            into the Rayleigh quotients and residuals.  GB300 runs FP64 at
                            1/74 of its FP32 rate, so 1 makes the check several times
                            cheaper at ~4e-15 relative accuracy.  Default 0.            */
} bloch_options;

/* Outcome of bloch_plan_autotune. */
typedef struct {
    int32_t fft_variant;         /* chosen pass variant (meaning as in bloch_options)       */
    int32_t tile_pmax;           /* chosen cap on pencils per CTA of the shared-memory
                                    passes (z and y passes; x passes use half of it)       */
    int32_t saturating_systems;  /* smallest number of systems per launch whose time per
                                    system is within 5 % of the best measured with the
                                    chosen configuration (batches of systems, 2 systems,
                                    4 systems ... up to 8 x systems, as memory allows)   */
    int32_t candidates;          /* configurations timed                                    */
    double ms_per_system[3];     /* best time of one A_k apply per system for variants 0,
                                    1, 2 (milliseconds); -1 where the variant was not timed
                                    (variant 0 when no axis has a fast pass)             */
} bloch_tune_report;

/* Statistics of the last bloch_solve_bands call (all counts summed over k). */
typedef struct {
    int64_t cg_iterations;     /* PCG iterations (each = one A_k apply per system)   */
    int64_t linear_solves;     /* PCG solves                                         */
    int64_t k_applies;         /* all A_k applies, incl. residual checks/refinement  */
    int64_t outer_iterations;  /* subspace sweeps or Lanczos restarts                */
    double max_rel_residual;   /* max over bands of ||A u - lam M u|| / ||A u|| (FP64) */
    double seconds;            /* wall time of the call                              */
    int64_t k_unconverged;     /* wave vectors that reached the sweep/restart cap
                                  before the tolerance (their omega are the last
                                  estimates; the call returns BLOCH_ENOTCONV_EIG) */
} bloch_stats;

/* Fill *opt with the defaults above. */
void bloch_default_options(bloch_options* opt);

/*
 * Create a plan for one voxelised periodic cell (Section 3.2 discretisation,
 * Algorithm 3 step (a)).
 *   grid          {Nx, Ny, Nz}, each >= 1 with prime factors in {2,3,5,7} and <= 512
 *   L             cell edge lengths (m), > 0
 *   grain_ids     host, V int32 values in [0, G), layout [z][y][x]
 *   G             number of grains (>= 1)
 *   C_per_grain   host, G x 6 x 6 Voigt stiffness (Pa), symmetric positive definite
 *   rho           host, G densities (kg/m^3), > 0
 *   opt           solver options (may be NULL for defaults); copied
 *   cuda_stream   cudaStream_t to enqueue on (NULL = legacy default stream)
 * The plan stores grain ids (int32) and per-grain tables on the device, the
 * volume-averaged stiffness C0 used by the preconditioner, the frequency and
 * twiddle tables.  Returns BLOCH_EINVAL on invalid arguments (message in
 * bloch_last_error), BLOCH_EUNSUPPORTED for grid sizes outside the limits,
 * BLOCH_ENOMEM / BLOCH_ECUDA on device failures.  On failure *out is NULL.
 */
bloch_status bloch_plan_create(bloch_plan** out, const int32_t grid[3], const double L[3],
                               const int32_t* grain_ids, int32_t G, const double* C_per_grain,
                               const double* rho, const bloch_options* opt, void* cuda_stream);

/* Release every device and host resource of the plan (NULL is ignored). */
void bloch_plan_destroy(bloch_plan* plan);

/*
 * Stiffness operator, Eq. (hatA), on nb Fourier-space vectors at once.
 *   k          host, nb x 3 wave vectors (rad/m), one per vector
 *   precision  BLOCH_FP32 (u, Ku are float2), BLOCH_FP64 (double2) or BLOCH_FF
 *              (double2 buffers, float-float arithmetic; u is rounded to
 *              float-float on entry)
 *   u          device, nb x 3 x V complex, Fourier basis; not modified
 *   Ku         device, nb x 3 x V complex; may not alias u
 * Enqueued on the plan's stream (asynchronous).  Scratch: 6 x V complex per
 * vector, held by the plan and grown on demand.  The FP32 fast z passes stage
 * their pencils with TMA tiles when u is 16-byte aligned and Nx * Ny is even
 * (cp.async otherwise); a staging wait that runs out sets the plan's pass
 * error word, reported by the next bloch_pcg or bloch_solve_bands.
 */
bloch_status bloch_apply_K(bloch_plan* plan, int32_t nb, const double* k, int32_t precision,
                           const void* u, void* Ku);

/*
 * Stiffness operator in the real-space basis: Ku = F^-1 A_k F u, the
 * sequence of Section 3.2 spelled out on grid values of the periodic part of
 * the Bloch displacement -- forward 3D FFT of the three components, Eq.
 * (hatA) in Fourier space, inverse 3D FFT.  F is the unnormalised DFT
 * (exp(-i xi.x) over the voxel centres' grid) and F^-1 carries 1/V, so
 * bloch_apply_K(F u) = F bloch_apply_K_real(u).
 *   k, precision  as bloch_apply_K
 *   u             device, nb x 3 x V complex, real-space grid values; not modified
 *   Ku            device, nb x 3 x V complex; may not alias u
 * Enqueued on the plan's stream.  Scratch: the operator workspace of
 * bloch_apply_K plus 9 x V complex per vector of solver workspace, held by
 * the plan and grown on demand.  Errors as bloch_apply_K.
 */
bloch_status bloch_apply_K_real(bloch_plan* plan, int32_t nb, const double* k, int32_t precision,
                                const void* u, void* Ku);

/*
 * Mass operator, Eq. (hatM): Mu = F{rho(x) F^-1 u} on nb Fourier-space vectors.
 * With a uniform density this is exactly rho*u (F F^-1 = I) and costs one
 * scaling; otherwise three inverse and three forward 3D FFTs per vector.
 * Same buffer conventions as bloch_apply_K; Mu may alias u.
 */
bloch_status bloch_apply_M(bloch_plan* plan, int32_t nb, int32_t precision, const void* u, void* Mu);

/*
 * Green-operator preconditioner, Eqs. (matrixP) and (precond):
 * z(xi) = P^-1(xi + k) r(xi), P_ik = C0_ijkl (xi+k)_j (xi+k)_l, with C0 the
 * volume average of C(x); bins where xi + k = 0 give z = 0.
 * Same buffer conventions as bloch_apply_K; z may alias r.
 */
bloch_status bloch_apply_precond(bloch_plan* plan, int32_t nb, const double* k, int32_t precision,
                                 const void* r, void* z);

/*
 * Inverse operator of Eq. (def_invop) by preconditioned CG (Algorithm 2),
 * nb independent systems A_{k_b} x_b = b_b advanced together.
 *   b          device, nb x 3 x V complex right-hand sides (bin 0 must be zero when k = 0)
 *   x          device, nb x 3 x V complex; on entry the start vector if use_x0 != 0,
 *              else ignored (x0 = 0); on exit the solutions
 *   tol        stop when ||b - A x||_2 <= tol ||b||_2 (recursive residual)
 *   max_iter   iteration cap
 *   iters      host, nb (may be NULL): iterations taken per system
 *   rel_res    host, nb (may be NULL): final recursive relative residual per system
 * Synchronises the stream.  Returns BLOCH_ENOTCONV_CG if any system missed tol,
 * and BLOCH_ECUDA if a pass kernel since the previous synchronising call gave
 * up waiting for its staging copies (the plan's pass error word; then cleared).
 */
bloch_status bloch_pcg(bloch_plan* plan, int32_t nb, const double* k, int32_t precision,
                       const void* b, void* x, double tol, int32_t max_iter, int32_t use_x0,
                       int32_t* iters, double* rel_res);

/*
 * Dispersion bands, Algorithm 3: for each wave vector k_r the n_bands lowest
 * eigenvalues lambda of A_k U = lambda M U, reported as omega = sqrt(lambda)
 * (rad/s), ascending.  At k = 0 the three rigid translations are reported as
 * omega = 0 and the rest is sought on their M-orthogonal complement.
 *   n_k, k_list   host, n_k x 3 (rad/m)
 *   n_bands       >= 1 and < 3V
 *   omega_out     host, n_k x n_bands
 *   vecs_out      optional device buffer n_k x n_bands x 3 x V complex in the
 *                 precision of the options (NULL = not returned), M-normalised
 *   stats         optional host struct (NULL = not returned)
 * Stop test (options.method = BLOCH_SUBSPACE, Algorithm 1): err1 <= tol_eig
 * and err2 <= 10 tol_eig (relative eigenvalue change, max relative residual).
 * With BLOCH_FP32 the FP32 iteration stops at the FP32 noise floor and the
 * block is refined by an FP64 Rayleigh-Ritz projection.  Synchronises; returns
 * BLOCH_ECUDA when the plan's pass error word is set (as bloch_pcg).
 */
bloch_status bloch_solve_bands(bloch_plan* plan, int32_t n_k, const double* k_list, int32_t n_bands,
                               double* omega_out, void* vecs_out, bloch_stats* stats);

/*
 * Group velocity of eigenvectors, Section 5.1 Eq. (c_group): c = d omega / d k
 * for each given vector u of A_k u = lambda M u, by the Hellmann-Feynman
 * identity d lambda/d k_m = u^H (dA_k/dk_m) u / u^H M u (M does not depend on
 * k), with u^H (dA_k/dk_m) u = 2 Re sum_xi conj(U_i) F{sigma_im} from the
 * component form of Eq. (hatA), sigma = C(x) : F^-1(sym (xi+k) (x) U) the
 * mode's stress, and d omega/d k = (d lambda/d k) / (2 omega).  lambda is the
 * Rayleigh quotient of u, so u should be an eigenvector (as returned by
 * bloch_solve_bands; any normalisation) of a simple eigenvalue -- within a
 * degenerate eigenspace the result depends on the vector chosen.  The wave
 * speeds of Section 5.2 are |c| of the acoustic branches at small k.
 *   nb         vectors (1..10922)
 *   k          host, nb x 3 (rad/m), the wave vector of each vector
 *   precision  BLOCH_FP32 or BLOCH_FP64 (u's type; arithmetic in that type,
 *              sums in FP64)
 *   u          device, nb x 3 x V complex, Fourier basis
 *   omega_out  host, nb (may be NULL): sqrt of the Rayleigh quotient (rad/s)
 *   c_out      host, nb x 3 (m/s); 0 where omega = 0 (rigid translations at k = 0)
 * Synchronises the plan's stream.  Errors: BLOCH_EINVAL (arguments, a zero
 * vector), BLOCH_ENONFINITE (k), BLOCH_ENOMEM, BLOCH_ECUDA.
 */
bloch_status bloch_group_velocity(bloch_plan* plan, int32_t nb, const double* k, int32_t precision, const void* u,
                                  double* omega_out, double* c_out);

/*
 * Real-space eigenvector fields, Section 5.2 Eq. (rotate_eigenvector):
 * U(x) = e^{-i phi} F^-1(U^) with F^-1 normalised by 1/V.  The paper takes phi
 * as the single phase of the field; here phi = arg(sum_x sum_i U_i(x)^2) / 2,
 * which is that phase (mod pi) whenever the field has one, and otherwise the
 * single phase maximising ||Re(e^{-i phi} F^-1(U^))||.  Optionally the strain
 * of the same field, eps_ij = (dU_i/dx_j + dU_j/dx_i)/2 computed spectrally
 * with d/dx_j = i xi_j (Section 5.2's epsilon_11 = dU_1/dx_1 is eps_xx).
 *   nb         fields (1..10922)
 *   precision  BLOCH_FP32 or BLOCH_FP64
 *   u_hat      device, nb x 3 x V complex, Fourier basis (not modified)
 *   u_real     device, nb x 3 x V complex: the phase-rotated real-space fields
 *   strain     device, nb x 6 x V complex, tensor components (xx yy zz yz xz
 *              xy), or NULL
 *   phi_out    host, nb (may be NULL): phi (rad)
 * Outputs may not alias u_hat.  Synchronises the plan's stream.
 */
bloch_status bloch_eigvec_real(bloch_plan* plan, int32_t nb, int32_t precision, const void* u_hat, void* u_real,
                               void* strain, double* phi_out);

/*
 * Host utility (no GPU): the dense generalised Hermitian eigenproblem
 * K Q = M Q diag(lam) solved for the projected matrices of Algorithm 1
 * (step EIG(K, M)), by Cholesky of M and cyclic complex Jacobi, in FP64.
 *   n      matrix order
 *   K, M   n x n row-major complex (interleaved re, im), Hermitian; M positive definite
 *   lam    out, n eigenvalues ascending
 *   Q      out, n x n row-major complex, eigenvectors in columns, Q^H M Q = I
 * Returns BLOCH_EINVAL if M is not positive definite.
 */
bloch_status bloch_host_gen_eig(int32_t n, const double* K, const double* M, double* lam, double* Q);

/*
 * Allocation-free stiffness apply (no counterpart in the paper; same operator,
 * same FP32 pass kernels and launch shapes as bloch_apply_K with precision
 * BLOCH_FP32 and fft_variant 0).
 *
 * For callers that must not allocate device memory at the point of the call:
 * services whose device memory is carved up in advance (a fixed budget or a
 * pool that must not grow), code embedded in a host framework that owns the
 * allocator, and latency-critical loops in which a cudaMalloc or cudaFree
 * (which can synchronise the device) is not acceptable.  bloch_apply_K grows
 * a plan-owned scratch buffer with cudaMalloc when it first meets a larger
 * batch; this entry point calls no cudaMalloc, cudaFree or allocating library
 * routine.  Its FFT-pass scratch is one fixed file-scope device array of
 * 97 MiB.  The array is placed on a GPU when the library's module holding it
 * is loaded there: with CUDA's default lazy module loading that happens at
 * the first call of this entry point on the device, so that first call does
 * take the 97 MiB (and can fail with BLOCH_ENOMEM / BLOCH_ECUDA if the device
 * is full).  Make one warm-up call per device before fixing the process's
 * device-memory budget; from then on the array stays until the process exits.
 *   plan   an existing plan (created beforehand; creation itself allocates)
 *   nb     systems, 1 <= nb <= 10922, with nb * Nx*Ny*Nz <= 2097152 (one
 *          128^3 system, eight 64^3 systems) and (Nx+Ny+Nz+6) * nb <= 262144;
 *          larger requests return BLOCH_EINVAL with the limit in
 *          bloch_last_error() and enqueue nothing
 *   The plan must use fft_variant 0 (else BLOCH_EUNSUPPORTED, nothing enqueued).
 *   k      host, nb x 3 wave vectors (rad/m)
 *   u, Ku  device, nb x 3 x V float2 each, as in bloch_apply_K (Ku may not alias u)
 * The first call on a device does a one-time set-up on that device (looks up
 * the array's device address and sets kernel attributes); make that first
 * call before any stream capture.  Every call uses the same array, so calls
 * that overlap on the GPU (on different streams, or from different threads)
 * race on the scratch; serialise them.  The array keeps the previous call's
 * intermediates; each call overwrites everything it reads.
 */
bloch_status bloch_apply_K_noalloc(bloch_plan* plan, int32_t nb, const double* k, const void* u, void* Ku);

/*
 * Learned Fourier-space preconditioner.  A small network rescales the branches
 * of the Green preconditioner per Fourier voxel:
 *   Z(q) = sum_a g_a v_a v_a^T / mu_a,  (mu_a, v_a) the eigenpairs of
 *   P(q) = C0 : q q (Eq. matrixP), g_a = softplus(MLP(f_a)) > 0,
 *   f_a = (qh_x^2, qh_y^2, qh_z^2, mu_a / |q|^2, log(1+|q|)/log(1+N/2)),
 * with q in units of 2 pi / L and C0 in units of its largest diagonal entry;
 * MLP 5 -> 16 -> 16 -> 1 with tanh.  Z is symmetric positive definite, so
 * plain CG stays valid, and a fresh network gives g = 1, i.e. exactly the
 * paper's preconditioner P^-1 (Eq. precond).  The paper has no learned part.
 * Training data are per-Fourier-voxel moments of CG residuals r_j and errors
 * e_j = x* - x_j (each pair scaled by 1/||r_j||); the loss is the mean of
 * ||Z r_j - e_j||^2.  Parameters, data and optimiser state live on the
 * device; the collection runs on the plan's stream, training on the default
 * stream.
 */
typedef struct bloch_lp bloch_lp;

/* Number of network parameters (flat order W1 (16x5), b1, W2 (16x16), b2, w3, b3). */
int32_t bloch_lp_num_params(void);

/* New network with deterministic seeded hidden weights and g = 1. */
bloch_status bloch_lp_create(bloch_lp** out, uint64_t seed);

/* Release the network and its data (NULL is ignored). */
void bloch_lp_destroy(bloch_lp* lp);

/* Copy parameters out (get != NULL) and/or in (set != NULL); host, bloch_lp_num_params() values. */
bloch_status bloch_lp_params(bloch_lp* lp, double* get, const double* set);

/*
 * Record training data on a plan: for each of n_k wave vectors (host, n_k x 3),
 * n_rhs seeded right-hand sides (weight 1/(1+|q|^2/16) in scaled units) are
 * solved to 1e-6 in FP32 with the Green preconditioner, then PCG is rerun from
 * zero and the moments of iterates 0..n_iters are added to a new data block.
 */
bloch_status bloch_lp_collect(bloch_lp* lp, bloch_plan* plan, int32_t n_k, const double* k_list, int32_t n_rhs,
                              int32_t n_iters, uint64_t seed);

/*
 * Add one data block from caller-supplied pairs (the caller's own CG runs, or
 * any residual/error pairs of the plan's operator): for each pair j the
 * per-Fourier-voxel moments A = Re r_j r_j^H, B = sym Re r_j e_j^H (six
 * entries each, order xx yy zz yz xz xy) and c = |e_j|^2, each weighted by
 * 1/||r_j||_2^2 (pairs with r_j = 0 are skipped), are summed into a new block.
 * The block's wave vector (the network's q features) is k.
 *   k        host, 3 (rad/m)
 *   n_pairs  1 <= n_pairs <= 10922
 *   r, e     device, n_pairs x 3 x V float2 each, Fourier basis of the plan's grid
 * Runs on the plan's stream and synchronises it; grows the plan's PCG
 * workspace to n_pairs systems.  Errors: BLOCH_EINVAL, BLOCH_ENONFINITE (k),
 * BLOCH_ENOMEM, BLOCH_ECUDA.
 */
bloch_status bloch_lp_add_pairs(bloch_lp* lp, bloch_plan* plan, const double* k, int32_t n_pairs, const void* r,
                                const void* e);

/* Loss (mean over recorded iterates) and its gradient (host, bloch_lp_num_params() values; may be NULL). */
bloch_status bloch_lp_loss_grad(bloch_lp* lp, double* loss, double* grad);

/* `steps` full-batch Adam steps (beta 0.9/0.999) with learning rate lr; loss_out (host, steps) may be NULL. */
bloch_status bloch_lp_train(bloch_lp* lp, int32_t steps, double lr, double* loss_out);

/* Number of data blocks recorded so far. */
int32_t bloch_lp_num_blocks(const bloch_lp* lp);

/*
 * Copy one data block to the host (any pointer may be NULL): grid {Nx,Ny,Nz};
 * q = scaled xi + k tables (Nx+Ny+Nz values); mom = V x 13 moments
 * (A: xx yy zz yz xz xy, B: same order, c); C0V = scaled 6x6 Voigt C0;
 * samples = recorded iterates.
 */
bloch_status bloch_lp_export_block(const bloch_lp* lp, int32_t block, int32_t grid[3], double* q, double* mom,
                                   double* C0V, int32_t* samples);

/*
 * Use a trained network in every PCG of this plan (NULL: back to the Green
 * preconditioner).  The network must outlive its use by the plan.
 */
bloch_status bloch_plan_set_preconditioner(bloch_plan* plan, const bloch_lp* lp);

/*
 * Autotuner of the batched operator (no counterpart in the paper; it serves
 * the Algorithm 3 loop, which applies A_k to many systems at once).  Times,
 * with CUDA events on the plan's stream, one A_k apply of `systems` systems
 * (deterministic pseudo-random Fourier fields, one nonzero wave vector) for
 * each candidate configuration: fft_variant 0 (when an axis has a fast pass)
 * and 1, each with pencils-per-CTA caps {4, 8, 16, 32} for the shared-memory
 * passes it uses, and 2 (cuFFT).  The fastest configuration is kept by the
 * plan for both precisions (all compute the same operator) and reported in
 * *report (may be NULL).  Then times batches of 2x, 4x, 8x systems with it
 * to report the saturating batch size.
 *   precision  BLOCH_FP32 or BLOCH_FP64: the field type timed
 *   systems    systems per launch to tune for, in [1, 10922]
 * Allocates 2 x systems x 3 x V complex of scratch for the call (more for the
 * batch sweep, skipped where memory is short) and grows the plan's operator
 * workspace.  Must not run concurrently with other calls on the same plan.
 * Errors: BLOCH_EINVAL (arguments), BLOCH_ENOMEM, BLOCH_ECUDA.
 */
bloch_status bloch_plan_autotune(bloch_plan* plan, int32_t precision, int32_t systems, bloch_tune_report* report);

/*
 * Phase tracer of bloch_solve_bands (no counterpart in the paper).  While
 * enabled, every solve records CUDA-event pairs on the plan's stream around
 * its phases and adds their durations (milliseconds) to the slots:
 *   0 PCG solves of the Algorithm 1 inverse step (and bloch_pcg calls)
 *   1 PCG solves of the Lanczos steps
 *   2 FP32 residual applies (A_k u, M u, Rayleigh quotients, residual norms)
 *   3 FP64 residual applies (the FP64 check of the FP32 form, incl. conversion)
 *   4 Lanczos orthogonalisation (inner products, updates, normalisation)
 *   5 Algorithm 1 projections (correction, Gram matrices, the projected
 *     eigensolve, basis rotation)
 *   6 Lanczos restarts (Ritz analysis, basis rotation, restart copies,
 *     compaction of converged wave vectors)
 *   7 slot set-up and output (start vectors, wave-vector tables, hand-off
 *     between the solvers, eigenvector output)
 *   8 GPU span of the solve (first to last event; 8 minus the sum of 0-7 is
 *     the time the stream had no traced work: idle gaps and small kernels)
 *   9 host wall time of the solve
 * count[i] = intervals recorded.  bloch_plan_trace synchronises the plan's
 * stream, writes the totals since the previous call to *out (may be NULL),
 * resets them, and then turns tracing on (enable = 1) or off (0).  Tracing
 * costs two event records per phase interval (none per PCG iteration).
 * Errors: BLOCH_EINVAL, BLOCH_ECUDA.
 */
typedef struct {
    double ms[10];
    int64_t count[10];
} bloch_trace;

bloch_status bloch_plan_trace(bloch_plan* plan, int32_t enable, bloch_trace* out);

/*
 * FMA throughput of the current device (no counterpart in the paper): the
 * denominators of the ALU-bound chains' rooflines (the FP64 operator is
 * bound by GB300's FP64 units, not by HBM).  Times, with CUDA events after
 * three warm-up launches, one launch of 8 CTAs of 256 threads per SM in
 * which every thread runs independent chains of fused multiply-adds on 8
 * accumulators (no memory traffic but one store per thread), once in FP64
 * and once in FP32; an FMA counts as 2 flops.
 *   fp64_gflops, fp32_gflops  (out, host) GFLOP/s; either may be NULL
 * Allocates 2.4 MB of device scratch for the call.
 * Errors: BLOCH_ENOMEM, BLOCH_ECUDA.
 */
bloch_status bloch_fma_peaks(double* fp64_gflops, double* fp32_gflops);

/* Message describing the last failure on the calling thread ("" if none). */
const char* bloch_last_error(void);

/* Bytes of device memory held by the plan right now (tables + scratch). */
size_t bloch_plan_device_bytes(const bloch_plan* plan);

/* Number of CUDA kernels the plan has launched since it was created. */
uint64_t bloch_plan_kernel_launches(const bloch_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* BLOCH_H */
