/*
 * mgglam.h -- C ABI of the GB300 (sm_103a) MG-GLAM scalar-field library.
 *
 * The library solves, on a periodic N^3 particle mesh in GLAM code units
 * (Sec. 3.1.1; cell size h = 1 on the finest level), the quasi-static scalar
 * field equation of three modified-gravity models and provides the particle
 * steps around it:
 *   f(R) Hu-Sawicki, n = 0, 1, 2   Eq. fR_eom_codeunit2 (unknown u = (-f_R)^{1/(n+1)})
 *   symmetron                      Eq. sym_eom_code_unit (unknown u = phi/phi_*)
 *   coupled quintessence (CQ)      Eq. csf_eom_code (unknown phi~ = c~^2 delta phi)
 * by FAS multigrid with red-black nonlinear Gauss-Seidel smoothing (Sec. 3.2.1,
 * closed-form local roots of Secs. 3.2.4-3.2.5; Newton-Gauss-Seidel for CQ,
 * Sec. 3.2.3), 8-child-mean restriction and 27/9/3/1 trilinear prolongation.
 *
 * Conventions shared by every entry point:
 *  - Mesh arrays are contiguous, row-major [i][j][k] with k fastest
 *    (index (i*N + j)*N + k); cell c spans [c, c+1) with its centre at c + 1/2.
 *  - Pointers documented "device" must be CUDA device (or managed) memory on the
 *    current device; "host" pointers are ordinary host memory.  The caller owns
 *    every buffer it passes; the library never frees them.
 *  - 'stream' is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; calls return after enqueueing unless
 *    documented otherwise (the solvers read the residual back to decide
 *    convergence and therefore synchronise 'stream' at those points).
 *  - The library keeps scratch memory (the multigrid level pyramid, reduction
 *    partials) in a cache keyed by (device, N, precision), allocated on first
 *    use and reused afterwards; mgglam_release() frees it.  Calls that share a
 *    cache entry must be ordered on the GPU (same stream, or synchronised).
 *  - Every entry point returns an mgglam_status; nothing aborts or throws.
 *    Invalid arguments are rejected before any work is enqueued.
 */
#ifndef MGGLAM_H
#define MGGLAM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MGGLAM_OK = 0,
  MGGLAM_ERR_ARG = -1,           /* null pointer, bad model/parameter value */
  MGGLAM_ERR_SHAPE = -2,         /* mesh size not supported (see each call) */
  MGGLAM_ERR_CUDA = -3,          /* a CUDA runtime call failed */
  MGGLAM_ERR_NOT_CONVERGED = -4, /* max_cycles reached above tol (results still written) */
  MGGLAM_ERR_NONFINITE = -5,     /* residual became NaN/Inf */
  MGGLAM_ERR_TIMEOUT = -6,       /* a bounded device-side wait expired */
  MGGLAM_ERR_OOM = -7            /* scratch allocation failed */
} mgglam_status;

typedef enum { MGGLAM_FR = 0, MGGLAM_SYMMETRON = 1, MGGLAM_CQ = 2 } mgglam_model;

typedef enum {
  MGGLAM_FP64 = 0, /* every level and sweep in FP64 */
  MGGLAM_MIXED = 1 /* FP64 fine residual + defect correction around FP32 FAS cycles */
} mgglam_precision;

/* Model and solver parameters.  All physical values in GLAM code units;
 * box in Mpc/h.  mgglam_default_params() fills the defaults noted here. */
typedef struct {
  int model;          /* mgglam_model */
  int n;              /* f(R): Hu-Sawicki index 0, 1 or 2 (Eq. fR_HS) */
  int keep_exp;       /* CQ: keep exp(beta phi~/c~^2) before (1+delta) (Sec. 3.2.3 drops it; default 0) */
  int precision;      /* mgglam_precision (default MGGLAM_MIXED) */
  double fR0_abs;     /* f(R): |f_R0| */
  double omega_m;     /* matter density parameter today (default 0.3) */
  double omega_l;     /* 1 - omega_m (default 0.7) */
  double box;         /* box side L in Mpc/h; c~ = (N/L) c/H0 */
  double a_star;      /* symmetron: symmetry-breaking scale factor a_* */
  double xi;          /* symmetron: xi = H0/m_* (range * H0/c) */
  double beta_star;   /* symmetron: coupling beta_* (forces only) */
  double alpha;       /* CQ: potential slope alpha > 0 (Eq. csf_potential) */
  double beta;        /* CQ: coupling beta < 0 (Eq. csf_coupling_function) */
  double lambda;      /* CQ: lambda of Eq. csf_param_lambda (from the background solver) */
  double phibar;      /* CQ: background field phibar(a) > 0 */
  int levels;         /* multigrid levels; 0 = halve while the mesh stays even and >= 4 (default 0) */
  int nu1, nu2;       /* pre-/post-smoothing red-black sweeps per level (default 2, 2) */
  int coarse_sweeps;  /* red-black sweeps on the coarsest level (default 16) */
  int max_cycles;     /* cap on multigrid cycles (default 50) */
  int inner_cycles;   /* MIXED: FP32 V-cycles per FP64 defect-correction step; 0 (default) =
                         adaptive: enough to reach tol at the observed contraction, capped
                         where single precision stops gaining within one step */
  int check_every;    /* FP64: test convergence every k cycles (default 1) */
  int sweep_chunk;    /* MIXED: <= 0 (default): one smoothing kernel per colour on every
                         level; > 0: the fused two-colour sweep kernel, with this many
                         planes per CTA, on every level whose tile divides the mesh */
  int sweep_slab;     /* MIXED, per-colour kernels on levels of side >= 256: planes per slab
                         of the L2-blocked sweep (first colour on a slab, then the second
                         colour one plane behind it, while the slab is still in L2; the
                         result equals the unblocked sweep bit for bit).  <= 0 (default):
                         one pass per colour (measured faster at 256^3: the kernel is bound
                         by instruction issue, and the extra launches cost more than the
                         DRAM traffic they save) */
  int tail_cells;     /* MIXED: the coarsest levels, from the first level (below the finest)
                         with at most this many cells, run as one thread block with the
                         levels in shared memory (same arithmetic, fewer launches).
                         0 (default) = 512; < 0 = off; at most 4096 */
  int cycle;          /* multigrid cycle: 0 (default) V, 1 F, 2 W (Sec. 3.2.1; each level
                         recurses once (V), twice (W), or F then V (F)) */
  int fmg;            /* 1: full-multigrid start (f(R), symmetron): the first cycle solves
                         the coarse problems first and starts each level from the prolonged
                         coarser solution, with one cycle per level (FP64: the whole
                         problem from the background; MIXED: the first outer step's
                         correction problem); 0 (default): cycles from the initial guess.
                         CQ ignores it: its equation is Poisson-like with a mass far below
                         the mesh scales, so the coarse solutions leave the field's mean
                         undetermined and the start gains nothing */
} mgglam_params;

/* Per-solve statistics.  resid values are the relative global residual:
 * RMS of the fine-level local residual divided by the RMS of the model's
 * linear source term (f(R): Om delta/a; symmetron: a^2/(2xi^2)(a_star/a)^3 ubar delta;
 * CQ: 3 beta Om e^{beta phibar} delta / a), or by 1 when that is zero (below
 * 1e-12 of the term's coefficient: a uniform density, up to rounding). */
typedef struct {
  int cycles;               /* multigrid cycles run (MIXED: inner FP32 V-cycles) */
  int outer;                /* MIXED: FP64 defect-correction steps */
  int converged;            /* 1 if resid <= tol */
  int pad;
  long long guarded;        /* f(R): cells where the coarse-grid correction would have left the
                               field not positive and the positivity guard replaced it (reading
                               of Sec. 3.2.1's correction step: the value is set to half its
                               value before the correction), summed over all levels and cycles
                               (MIXED: over the inner FP32 cycles) */
  double resid0;            /* before the first cycle */
  double resid;             /* at return */
  double seconds;           /* host wall time of the call */
  double resid_hist[64];    /* resid before cycle 0, after each checked cycle (first 64) */
} mgglam_stats;

/* Library version string (static storage). */
const char* mgglam_version(void);

/* Human-readable name of a status code (static storage). */
const char* mgglam_status_string(int status);

/* Fill *prm with the defaults listed in mgglam_params.  MGGLAM_ERR_ARG if prm is NULL. */
int mgglam_default_params(mgglam_params* prm);

/*
 * Cloud-in-cell density assignment (Sec. 3.1): each particle adds mass N^3/np
 * shared between the 8 nearest cell centres with weights
 * prod_d (1 - |x_d - (c_d + 1/2)|), periodic, so that the mean density is 1.
 *   pos    [np][3] float32 positions in cell units; any real value is wrapped
 *          periodically into [0, N).  Device memory, or page-locked host memory
 *          (cudaHostAlloc / pinned), which the kernel reads in place over the
 *          host link (no separate copy).
 *   np     number of particles (>= 1).
 *   N      mesh side, 2 <= N <= 2048.
 *   rho    device, N^3 float32 output (overwritten).
 * Accumulation is in 64-bit fixed point (2^-32 of a particle's weight), so the
 * result is bitwise reproducible and independent of particle order.
 * Errors: MGGLAM_ERR_ARG (null pointer, np < 1), MGGLAM_ERR_SHAPE (N),
 * MGGLAM_ERR_OOM, MGGLAM_ERR_CUDA.
 */
int mgglam_deposit_cic(const float* pos, long long np, int N, float* rho, void* stream);

/*
 * The same deposit (identical result) for particles in page-locked host memory,
 * with the host-to-device copy overlapped with the deposit: the positions are
 * copied in 'chunks' pieces on the library's copy stream into pos_dev, and
 * each piece is deposited (on 'stream') as soon as it has arrived.
 *   pos_host  page-locked host, [np][3] float32 (read; unchanged).
 *   pos_dev   device, [np][3] float32 staging buffer; holds a copy of pos_host
 *             on return (the gather can use it).  Not touched before earlier
 *             work on 'stream' completes.
 *   chunks    1..32, 0 = 8.
 * Errors as mgglam_deposit_cic; MGGLAM_ERR_ARG for chunks outside 0..32.
 */
int mgglam_deposit_cic_host(const float* pos_host, float* pos_dev, long long np, int N, float* rho, int chunks,
                            void* stream);

/*
 * The same CIC density assignment as mgglam_deposit_cic (identical result, bit
 * for bit), for callers that must not trigger a device allocation.
 * mgglam_deposit_cic takes its accumulator from the library's scratch cache
 * and calls cudaMalloc the first time it sees a mesh size.  Some callers
 * cannot allow that: applications that hand all device memory to their own
 * pool allocator and run inside a fixed budget (a foreign cudaMalloc can fail
 * or push them over it), and time-stepping loops that cannot absorb the
 * implicit device-wide synchronisation of cudaMalloc in the middle of a step.
 * This entry point allocates nothing.  Its accumulator is a fixed device array
 * compiled into the library, sized for meshes up to N = 128 (128^3 64-bit
 * integers = 16 MiB); every GPU on which the library is loaded holds that
 * array until the process exits.
 *   Arguments and layout as for mgglam_deposit_cic.
 *   N must satisfy 2 <= N <= 128; larger meshes return MGGLAM_ERR_SHAPE before
 *   any work is enqueued (use mgglam_deposit_cic for them).
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before starting
 * any stream capture.  mgglam_release() drops the cached address of the
 * current device, so the next call looks it up again.  Each call clears the
 * part of the array it uses before accumulating, but all calls share the one
 * array: calls that may run at the same time on the GPU (different streams
 * without ordering, or several host threads) race and corrupt each other's
 * results.
 * The paper has no counterpart to this entry point: it exists for callers
 * that cannot allocate device memory.
 * Errors: MGGLAM_ERR_ARG (null pointer, np < 1), MGGLAM_ERR_SHAPE (N),
 * MGGLAM_ERR_CUDA.
 */
int mgglam_deposit_cic_static(const float* pos, long long np, int N, float* rho, void* stream);

/*
 * Solve the model's discrete scalar-field equation N_h(u; rho) = 0 (the
 * fine-level local residual of Eq. residual_d set to zero) by multigrid cycles
 * until the relative global residual (see mgglam_stats) is <= tol or
 * prm->max_cycles cycles have run.
 *   prm    host, model + solver parameters (prm->precision selects FP64 or MIXED).
 *   a      scale factor (> 0).
 *   rho    device, N^3 float32 density (any positive mean: it is rescaled to
 *          mean 1 in FP64, Eq. code_units2's mean-1 convention).
 *   N      mesh side; even, 4 <= N <= 2048.
 *   field  device, N^3 float64, in/out: on input the initial guess, or if its
 *          first element is NaN the background value (f(R), symmetron ubar; CQ 0);
 *          on output the solution (f(R): u = (-f_R)^{1/(n+1)}; symmetron: u;
 *          CQ: phi~).
 *   tol    target relative residual (>= 0).
 *   stats  host, may be NULL.
 * Returns MGGLAM_OK when converged, MGGLAM_ERR_NOT_CONVERGED if max_cycles was
 * reached first (field holds the last iterate), MGGLAM_ERR_NONFINITE if the
 * residual became NaN/Inf, or an argument/CUDA/allocation error (after which
 * the field's contents are unspecified).  Synchronises 'stream' once per
 * convergence check.
 */
int mgglam_solve_scalar(const mgglam_params* prm, double a, const float* rho, int N,
                        double* field, double tol, mgglam_stats* stats, void* stream);

/*
 * Fifth force on particles (Sec. 3.1: three-point central differences at cell
 * centres, CIC-interpolated to the particle with the deposit's weights):
 *   f(R):      F = prefactor * (c~^2/2) grad f_R,  f_R = -u^{n+1}   (Eq. F5_fR_codeunit)
 *   symmetron: F = prefactor * (-3 xi^2 Om beta_*^2 c~^2 a_*^-3) grad(u^2)  (Eq. F_5_codeunit)
 *   CQ:        F = prefactor * (-beta) grad phi~   (the fifth-force part of Eq. csf_particle_geodesic_code2)
 * prefactor is the caller's time factor (e.g. H0/adot).
 *   field  device, N^3 float64 solution from mgglam_solve_scalar.
 *   pos    [np][3] float32 positions (cell units, wrapped periodically); device
 *          or page-locked host memory (read in place).
 *   force  [np][3] float32 output (overwritten); device or page-locked host
 *          memory (written in place).
 * Errors: MGGLAM_ERR_ARG, MGGLAM_ERR_SHAPE (N even, 4..2048), MGGLAM_ERR_OOM, MGGLAM_ERR_CUDA.
 */
int mgglam_gather_force(const mgglam_params* prm, double a, const double* field, int N,
                        const float* pos, long long np, float* force, double prefactor,
                        void* stream);

/*
 * The same gather with the forces delivered to page-locked host memory, the
 * device-to-host copy overlapped with the gather: the particles are gathered
 * in 'chunks' pieces into force_dev and each piece is copied to force_host on
 * the library's copy stream while the next is computed.  Work later enqueued
 * on 'stream' (and a synchronisation of it) waits for the last copy.
 *   pos_dev     device, [np][3] float32 positions.
 *   force_dev   device, [np][3] float32 staging buffer (overwritten).
 *   force_host  page-locked host, [np][3] float32 output.
 *   chunks      1..32, 0 = 8.
 * Errors as mgglam_gather_force; MGGLAM_ERR_ARG for chunks outside 0..32.
 */
int mgglam_gather_force_host(const mgglam_params* prm, double a, const double* field, int N, const float* pos_dev,
                             long long np, float* force_dev, float* force_host, double prefactor, int chunks,
                             void* stream);

/*
 * Adjoint of the solve: gradients of a scalar loss l(u*) with respect to the
 * density and (f(R)) ln|f_R0|, given g = dl/du* at the solution u* of
 * mgglam_solve_scalar (f(R) any n, or the symmetron).  With J = dN/du at u*
 * (N the discrete operator of Eq. fR_eom_codeunit2 / Eq. sym_eom_code_unit),
 * the adjoint field lambda solves J^T lambda = g, written as the symmetric
 * screened-Poisson problem -c~^2 Delta_h lambda + m lambda = sigma g
 * (f(R): m = K/((n+1)u^{n+2}), sigma = 1/((n+1)u^n); symmetron:
 * m = a^2/(2xi^2)(rho a*^3/a^3 - 1 + 3u^2), sigma = -1), and is found by
 * multigrid (FP64 residual, FP32 correction V-cycles with the forward solve's
 * transfers; the coarse-level coefficients are rebuilt from u* on each call, no
 * forward iterate is stored).  Then
 *   grad_rho[i] = dl/d delta_i = -(dN_i/d delta_i) lambda_i   (delta = rho/mean - 1)
 *   grad_rho_raw[j] = dl/d rho_j for the rho passed in, through the solver's
 *                mean-1 normalisation (Eq. code_units2's convention):
 *                (grad_rho[j] - sum_i grad_rho[i] rho_i / sum_i rho_i) / mean(rho)
 *   *grad_logfR0 = dl/d ln|f_R0| = sum_i lambda_i K/((n+1) u_i)   (f(R); 0 otherwise)
 *   prm, a, rho, N   as passed to mgglam_solve_scalar (rho device float32)
 *   field            device, N^3 float64, the converged u*
 *   grad_field       device, N^3 float64, g = dl/du*
 *   grad_rho         device, N^3 float64 output
 *   grad_rho_raw     device, N^3 float64 output, or NULL (not formed); must
 *                    not alias grad_rho
 *   grad_logfR0      host, may be NULL
 *   tol              relative residual of the adjoint equation
 * Returns as mgglam_solve_scalar; MGGLAM_ERR_ARG for the CQ model (not supported).
 * The paper differentiates nothing; this serves gradient-based inference
 * through the solver (the paper's emulator motivation, Sec. 6).
 */
int mgglam_solve_adjoint(const mgglam_params* prm, double a, const double* field, const float* rho, int N,
                         const double* grad_field, double* grad_rho, double* grad_rho_raw, double* grad_logfR0,
                         double tol, mgglam_stats* stats, void* stream);

/*
 * Many independent solves at once (an emulator's parameter grid, several
 * realisations): each solve s has its own parameters prm[s] (model, f(R) n,
 * |f_R0|, symmetron parameters, box), scale factor a[s], density rho[s] and mesh
 * N[s]; every solve is the mixed-precision solve of mgglam_solve_scalar
 * (prm[s].precision is ignored), carried to tol.  The solves advance in lock
 * step: each multigrid phase is one kernel launch over the blocks of all solves
 * that take part in it, one V-cycle of the batch is replayed as a CUDA graph,
 * and converged solves drop out (their blocks exit at once).
 *   count   number of solves (>= 1)
 *   prm     host array [count]; nu1, nu2, coarse_sweeps must agree across solves;
 *           inner_cycles and max_cycles are taken from prm[0]; cycle must be 0
 *           (V-cycles)
 *   a       host array [count]
 *   rho     host array [count] of device float32 N[s]^3 pointers
 *   N       host array [count]; each a multiple of 32, 32..2048
 *   field   host array [count] of device float64 N[s]^3 pointers (in/out as for
 *           mgglam_solve_scalar)
 *   stats   host array [count] or NULL (seconds = the whole batch's time)
 * Scratch for a batch is cached by its list of mesh sizes and levels.  Returns
 * MGGLAM_OK when every solve converged, else MGGLAM_ERR_NOT_CONVERGED /
 * MGGLAM_ERR_NONFINITE (per-solve outcome in stats), or an argument error.
 * Not in the paper (it runs independent realisations with MPI, Sec. 3.1).
 */
int mgglam_solve_batch(int count, const mgglam_params* prm, const double* a, const float* const* rho, const int* N,
                       double* const* field, double tol, mgglam_stats* stats, void* stream);

/* ---- single-step entry points (one multigrid operation on one level, FP64) ----
 * These expose each step of the path for testing and for callers composing
 * their own cycles.  'n' is the level's mesh side, 'h' its cell size (the finest
 * level has h = 1 and c~ is fixed by the finest mesh side Nfine = n*h); 'rho'
 * is the level's float64 density with mean 1 on the finest level; 'S' is the
 * level's FAS source (may be NULL on the finest level, meaning S = 0).  All
 * arrays are device float64 n^3 unless noted. */

/* Red-black sweeps (black = (i+j+k) even first, then red; Sec. 3.2.1), in place on u. */
int mgglam_smooth(const mgglam_params* prm, double a, int n, double h, double* u,
                  const double* rho, const double* S, int sweeps, void* stream);

/* Local residual d = N_h(u) - S (Eq. residual_d); d may be NULL.  *sumsq (host)
 * receives sum d^2 (synchronises 'stream'); sumsq may be NULL. */
int mgglam_residual(const mgglam_params* prm, double a, int n, double h, const double* u,
                    const double* rho, const double* S, double* d, double* sumsq, void* stream);

/* Restriction: coarse[(n/2)^3] = mean of the 8 children of each coarse cell (Sec. 3.2.1). */
int mgglam_restrict(int n, const double* fine, double* coarse, void* stream);

/* Coarse-grid correction, Eq. solution_correction: u_fine += P(uH - RuH) with
 * the 27/9/3/1 (/64) prolongation; uH, RuH are (n/2)^3 for fine side n.  For
 * f(R), a fine value that is not positive afterwards is set to half its value
 * before the correction. */
int mgglam_prolong_correct(const mgglam_params* prm, int n, const double* uH, const double* RuH,
                           double* u_fine, void* stream);

/* Free every cached scratch allocation on the current device (and forget the
 * cached address of mgglam_deposit_cic_static's array there). */
int mgglam_release(void);

/* ---- Coupled-quintessence background (host code, once per parameter set) --
 *
 * Sec. 3.2.3 ("background cosmology solver"), Eqs. csf_background_eom,
 * csf_background_Friedmann, csf_background_Raychaudhuri and their code-unit
 * form Eq. csf_background_eom_codeunit, for A(phi) = exp(beta phi) and
 * V = Lambda^4/phi^alpha (Eqs. csf_coupling_function, csf_potential) with
 * Lambda^4/M_Pl^2 = H0^2 lambda^2 (Eq. csf_param_lambda).  Flat universe,
 * radiation = CMB photons at 2.7255 K plus 3.046 massless neutrino species.
 * lambda is not free: it is found, as in the paper, by shooting until the
 * H(a=1) of the integration from z = 1e5 equals H0.
 *
 * alpha > 0, beta, omega_m in (0,1), h = H0/(100 km/s/Mpc) > 0, a in (0, 1].
 * Outputs (host scalars): lambda; phibar(a); dphibar/dln a at a; E = H(a)/H0.
 * phibar and lambda are what mgglam_params.phibar and .lambda take for the CQ
 * solve; dphibar/dln a and E enter the particle update (Eq.
 * csf_particle_geodesic_code2).  Returns MGGLAM_ERR_ARG for invalid inputs,
 * MGGLAM_ERR_NONFINITE if an integration fails, MGGLAM_ERR_NOT_CONVERGED if
 * no lambda in [2^-60, 2^60] matches H0.  Touches no GPU state. */
int mgglam_cq_background(double alpha, double beta, double omega_m, double h, double a, double* lambda,
                         double* phibar, double* dphibar_dlna, double* E);

/* Present-day radiation density parameter Omega_r for H0 = 100 h km/s/Mpc
 * (photons at 2.7255 K, 3.046 massless neutrinos; Sec. 3.2.3). */
double mgglam_radiation_density(double h);

/* ---- Particle-mesh time step (Sec. 3.1 and the particle equations of
 * Secs. 3.2.3-3.2.5) ------------------------------------------------------ */

/*
 * Periodic Poisson equation by FFT, the PM gravity solver of Sec. 3.1 (Eq.
 * GR_poisson_codeunit with the discrete Green's function of the 7-point
 * Laplacian): phi solves grad_h^2 phi = coef (rho/mean(rho) - 1) on the N^3
 * mesh (h = 1), with mean(phi) = 0.  Single-precision FFTs of power-of-two
 * length, twiddles from double precision: phi carries ~1e-6 relative error.
 *   rho  device, N^3 float32 density (row-major [x][y][z]); any positive mean.
 *   N    power of two, 8 <= N <= 1024.
 *   coef for the Newtonian potential (3/2) Om / a.
 *   phi  device, N^3 float32 output (may not alias rho).
 * The library keeps an N^3 complex work array per (device, N), freed by
 * mgglam_release.  Errors: MGGLAM_ERR_ARG, MGGLAM_ERR_SHAPE, MGGLAM_ERR_OOM,
 * MGGLAM_ERR_CUDA.
 */
int mgglam_poisson_fft(const float* rho, int N, double coef, float* phi, void* stream);

/* Scalars of one PM step from a to a + da. */
typedef struct {
  double a;           /* scale factor of the positions (the force time a_n) */
  double da;          /* step in a (> 0) */
  double E_a;         /* H(a)/H0 */
  double E_half;      /* H(a + da/2)/H0 */
  double dphibar_da;  /* CQ: d phibar / da at a (the momentum drag); unused otherwise */
  int scalar;         /* 1: the model's scalar field and fifth force; 0: LCDM (Newtonian only) */
} mgglam_pm_step_desc;

/*
 * One leapfrog step of the PM N-body code, positions at a, momenta at
 * a - da/2 (code units of Eq. code_units: x in cells, p~):
 *   rho = CIC deposit of pos; grad^2 Phi_N = (3/2) Om/a delta (FFT);
 *   scalar: the model's field solved at a from 'field' (the previous step's
 *           solution, or NaN in its first element for the background), as
 *           mgglam_solve_scalar;
 *   p += da (H0/adot) grad Psi - gamma p da (drag at the midpoint),
 *     Psi = -sN Phi_N + (the fifth-force potential of mgglam_gather_force),
 *     sN = e^{beta phibar} for CQ (Sec. 3.2.3), else 1; H0/adot = 1/(a E_a);
 *     gamma = beta dphibar/da (CQ, Eq. csf_particle_geodesic_code2),
 *     9 Om beta*^2 xi^2 sqrt(1 - (a_star/a)^3) a^-4 u(x) (symmetron, a > a_star,
 *     Eq. F_x_codeunit), 0 otherwise;
 *   pos += da p / ((a + da/2)^3 E_half), wrapped into [0, N).
 *   pos, mom  device, [np][3] float32, updated in place.
 *   field     device, N^3 float64 (desc->scalar), in/out; else may be NULL.
 *   rho_work, psi_work  device, N^3 float32 scratch each (rho_work holds the
 *             density on return, psi_work the total potential Psi).
 *   N         power of two, 8 <= N <= 1024.
 * Returns the scalar solve's status (MGGLAM_ERR_NOT_CONVERGED still moves the
 * particles with the last iterate), or an argument/CUDA/allocation error
 * before anything moves.
 */
int mgglam_pm_step(const mgglam_params* prm, const mgglam_pm_step_desc* desc, int N, float* pos, float* mom,
                   long long np, double* field, double tol, float* rho_work, float* psi_work, mgglam_stats* stats,
                   void* stream);

/* ---- tracing (not part of the paper's method: measurement support) ---- */

/* Accumulated CUDA-event timing of one class of kernel launches. */
typedef struct {
  char name[40];        /* kernel class, e.g. "smooth32_fine" */
  long long launches;   /* timed launches */
  double ms;            /* summed event-to-event time on the launching stream */
  double bytes;         /* summed algorithmic bytes of those launches (the data
                           the operation must read and write once) */
} mgglam_kernel_profile;

/* Start timing: every later fine-level kernel launch (and the deposit and
 * gather kernels) is bracketed by a pair of CUDA events recorded on its
 * stream; the coarse levels of a multigrid cycle are timed as one class.
 * Clears earlier records. */
int mgglam_profile_start(void);

/* Stop timing, synchronise the device, and write up to max_entries per-class
 * totals to out (host array); *n_entries (host) receives the number of classes
 * that had launches.  out may be NULL to query the count.  MGGLAM_ERR_CUDA if
 * the device synchronisation fails. */
int mgglam_profile_stop(mgglam_kernel_profile* out, int max_entries, int* n_entries);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all streams), counted at enqueue time. */
long long mgglam_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* MGGLAM_H */
