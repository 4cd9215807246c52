// mg_internal.h -- host-side interfaces between the C-ABI layer and the
// kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/mgglam.h"
#include "mg_model.cuh"

namespace mg {

constexpr int kMaxLevels = 16;

// Inner-cycle schedule of the mixed-precision solvers (host side).
// Residual reduction one FP32 inner solve can deliver before its own rounding
// limits it (measured: a step stalls at a few 1e-7 of its starting residual).
// The inner-cycle count of an outer step is capped at what reaches it: more
// cycles gain nothing until the next float-float/FP64 residual.
constexpr double kFp32StepGain = 1e-5;

// Per-cycle residual contraction assumed before one has been measured.  A
// V(2,1) cycle contracts the f(R) residual by ~0.08 on the 256^3 workload; the
// estimate errs on the slow side, because planning too few cycles costs a
// whole extra outer step (a float-float residual and a host synchronisation),
// while planning one too many costs one cycle.  Convergence is always decided
// on the outer residual, and a measured contraction replaces this estimate as
// soon as an outer step is not limited by single precision.
constexpr double kInitialContraction = 0.1;

// Residual reduction assumed for the full-multigrid start when an outer step is
// planned (mgglam_params.fmg); like kInitialContraction it errs on the slow side.
constexpr double kFmgGain = 0.05;

// One multigrid level.  FP64 arrays serve the FP64 path (and the FP64 fine
// level of the mixed path); FP32 arrays serve the mixed path's inner cycles.
struct Level {
  int n = 0;
  double h = 1.0;
  size_t n3 = 0;
  // FP64 path
  double* u = nullptr;    // solution (level 0: the caller's field)
  double* rho = nullptr;  // density, mean 1 on level 0
  double* S = nullptr;    // FAS source (level 0: none)
  double* Ru = nullptr;   // restricted fine solution R u^{l-1}
  // mixed path (FP32, correction form)
  float* e = nullptr;     // correction e on this level (level 0: two buffers, ping-pong)
  float* e_alt = nullptr;
  float* ub = nullptr;    // base field the correction is added to
  float* S32 = nullptr;   // source (level 0: tau = -r64)
  float* Re = nullptr;    // restricted correction R e^{l-1}
  float* rho32 = nullptr; // density, mean 1
};

struct Workspace {
  int device = -1;
  int N = 0;
  int precision = 0;
  int nlev = 0;
  int levels_req = 0;
  Level lev[kMaxLevels];
  void* base = nullptr;
  size_t bytes = 0;
  double* src64 = nullptr;      // mixed path: FP64 u-independent source term on the fine level
  double* partials = nullptr;   // kMaxReduceBlocks doubles
  double* scalars = nullptr;    // device scalars, see Scalar
  double* h_scalars = nullptr;  // pinned host mirror
  int64_t* cic_acc = nullptr;   // fixed-point deposit accumulator (allocated on demand)
  size_t cic_bytes = 0;
  // CUDA graph of the coarse part of a V-cycle (levels >= 1), captured on
  // cap_stream for the parameter signature coarse_sig and replayed on the
  // caller's stream; coarse_launches = kernels in the graph.
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t coarse_exec = nullptr;
  unsigned long long coarse_sig = 0;
  long long coarse_launches = 0;
};

// Slots of Workspace::scalars.
// SC_FFC: start of the float-float residual constants (48 bytes, mixed path).
// SC_GUARD holds a 64-bit integer: the positivity-guard replacements of the running solve.
enum Scalar { SC_MEAN = 0, SC_SUMSQ = 1, SC_SRC = 2, SC_FLAG = 3, SC_GUARD = 4, SC_FFC = 8, SC_COUNT = 16 };
inline unsigned long long* guard_of(Workspace* ws) {
  return reinterpret_cast<unsigned long long*>(ws->scalars + SC_GUARD);
}

int count_levels(int N, int levels);

// Planes per CTA of a z-marching kernel 'kern' (threads per CTA) over 'tiles'
// (j,k) tiles of a level of side n, sized to whole waves of resident CTAs.
int march_chunk(int n, long long tiles, const void* kern, int threads);

// Normaliser of the relative residual: the RMS of the model's linear source
// term (coefficient x RMS(delta)), or 1 where the density is uniform.  A
// source below 1e-12 of its coefficient counts as uniform: that is rounding in
// delta = rho/mean - 1, not structure.
double source_norm(const ModelDev& m, double src_rms);

// Build the device model constants for level-independent use (c~ from N_fine).
int make_model(const mgglam_params* prm, double a, int Nfine, ModelDev* m);

// Workspace cache (one per (device, N, precision, levels)).
int get_workspace(int N, int precision, int levels, Workspace** ws);
void release_workspaces();

// ---- FP64 kernels (solve64.cu) ----
int launch_smooth64(const ModelDev& m, int n, double h, double* u, const double* rho,
                    const double* S, int sweeps, cudaStream_t st);
int launch_residual64(const ModelDev& m, int n, double h, const double* u, const double* rho,
                      const double* S, double* d, double* partials, double* out_sum,
                      cudaStream_t st);
int launch_restrict64(int nf, const double* fine, double* coarse, cudaStream_t st);
int launch_prolong_correct64(const ModelDev& m, int nc, const double* uH, const double* RuH, unsigned long long* guard,
                             double* uf, cudaStream_t st);
int launch_coarse64(const ModelDev& m, int n, double h, double* u, const double* rho,
                    const double* S, int sweeps, cudaStream_t st);
int launch_residual_restrict64(const ModelDev& m, int nf, double hf, const double* u,
                               const double* rho, const double* S, double* Ru, double* uH,
                               double* Rd, cudaStream_t st);
int launch_fas_source64(const ModelDev& m, int nc, double hc, const double* Ru,
                        const double* rho, double* S, cudaStream_t st);
int launch_density_mean(const float* rho32, size_t n3, double* partials, double* out_sum,
                        cudaStream_t st);
int launch_density_to64(const float* rho32, size_t n3, const double* sum, double* rho64,
                        cudaStream_t st);
int launch_src_sumsq(const ModelDev& m, const double* rho64, size_t n3, double* partials,
                     double* out, cudaStream_t st);
int launch_init_background(const ModelDev& m, double* field, size_t n3, cudaStream_t st);

// ---- tracing (profile.cu) ----
enum ProfClass {
  PC_SMOOTH32_FINE = 0, PC_RESTRICT32_FINE, PC_PROLONG32_FINE, PC_OUTER_RESID, PC_APPLY_CORR,
  PC_SMOOTH64_FINE, PC_RESTRICT64_FINE, PC_PROLONG64_FINE, PC_RESID64_FINE, PC_COARSE_LEVELS,
  PC_DEPOSIT, PC_DEPOSIT_FINISH, PC_TRANSFORM, PC_GATHER, PC_POISSON_FFT, PC_PM_POTENTIAL, PC_PM_KICK_DRIFT,
  PC_COUNT
};
void note_launch(int n);
long long launch_count();
void prof_begin(int cls, cudaStream_t st, double alg_bytes);
void prof_end(cudaStream_t st);

// ---- solvers ----
int solve_fp64(const mgglam_params* prm, double a, const float* rho, int N, double* field,
               double tol, mgglam_stats* stats, cudaStream_t st);
int solve_mixed(const mgglam_params* prm, double a, const float* rho, int N, double* field,
                double tol, mgglam_stats* stats, cudaStream_t st);

// ---- PM step (fft.cu, pm.cu) ----
int poisson_fft(const float* rho, int N, double coef, float* phi, cudaStream_t st);
void release_fft_plans();
int pm_step(const mgglam_params* prm, const mgglam_pm_step_desc* d, int N, float* pos, float* mom, long long np,
            double* field, double tol, float* rho_work, float* psi_work, mgglam_stats* stats, cudaStream_t st);

// ---- adjoint (adjoint.cu), batch (batch.cu) ----
void release_adjoint_work();
void release_batches();

// ---- particles (particles.cu) ----
int deposit_cic(const float* pos, long long np, int N, float* rho, cudaStream_t st);
void forget_static_deposit_address();
int gather_force(const ModelDev& m, int kind, int n_fr, const mgglam_params* prm,
                 const double* field, int N, const float* pos, long long np, float* force,
                 double prefactor, cudaStream_t st);
int gather_chunk(const ModelDev& m, int kind, const mgglam_params* prm, int N, const float* pos, long long np,
                 float* force, double prefactor, cudaStream_t st);
int deposit_cic_host(const float* pos_host, float* pos_dev, long long np, int N, float* rho, int chunks,
                     cudaStream_t st);
int gather_force_host(const ModelDev& m, int kind, const mgglam_params* prm, const double* field, int N,
                      const float* pos_dev, long long np, float* force_dev, float* force_host, double prefactor,
                      int chunks, cudaStream_t st);

}  // namespace mg

#define MG_CUDA_TRY(call)                                  \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return MGGLAM_ERR_CUDA;         \
  } while (0)
