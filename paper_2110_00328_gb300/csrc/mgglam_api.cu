// mgglam_api.cu -- the extern "C" entry points of include/mgglam.h: argument
// checks, host-side background scalars (GLAM code units), the scratch cache,
// and dispatch to the kernel translation units.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

// c / H0 in Mpc/h: the speed of light over 100 km/s/Mpc.
static const double kCOverH0 = 299792.458 / 100.0;

// Planes per CTA of a z-marching kernel over 'tiles' (j,k) tiles of a level of
// side n.  Each CTA marches its whole chunk, so a last wave holding a few CTAs
// costs as much as a full one: the chunk minimises waves x (chunk + 4: the two
// prologue planes and about as much again for the CTA's start and reduction),
// with the resident CTAs per SM from the occupancy calculator, at least 8
// planes (halo re-reads <= 25%), and the CTA count within the partial-sum array.
int march_chunk(int n, long long tiles, const void* kern, int threads) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const long long R = (long long)(sms > 0 ? sms : 1) * per_sm;
  int best = n;
  long long best_cost = -1;
  for (int c = n < 8 ? n : 8; c <= n; ++c) {
    const long long ctas = tiles * ((n + c - 1) / c);
    if (ctas > kMaxReduceBlocks) continue;
    const long long cost = ((ctas + R - 1) / R) * (c + 4);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  return best;
}

double source_norm(const ModelDev& m, double src_rms) {
  double coef;
  if (is_fr(m.kind)) coef = m.om_a;
  else if (m.kind == KSYM) coef = m.msym * m.rat3 * m.ubar;
  else coef = m.cq_src;
  coef = fabs(coef);
  return src_rms > 1e-12 * coef && src_rms > 0.0 ? src_rms : 1.0;
}

int count_levels(int N, int levels) {
  int nl = 1, n = N;
  if (levels > 0) {
    for (int l = 1; l < levels && l < kMaxLevels; ++l) {
      if (n % 2 != 0 || n / 2 < 2) break;
      n /= 2;
      ++nl;
    }
    return nl;
  }
  while (nl < kMaxLevels && n % 2 == 0 && n / 2 >= 4 && (n / 2) % 2 == 0) {
    n /= 2;
    ++nl;
  }
  return nl;
}

// Background scalars at scale factor a (a0 of the path):
//  c~ = (N/L) c/H0 (Sec. 3.1.1); f(R): Rbar(a) = 3 (Om a^-3 + 4 OL) (Sec. 3.2.5),
//  fbar_R(a) = -|fR0| (Rbar(1)/Rbar(a))^{n+1} (Eq. fR_HS), ubar = (-fbar_R)^{1/(n+1)};
//  symmetron: ubar = sqrt(1 - (a_star/a)^3) (Eq. varphi_min_symm);
//  CQ: source 3 beta Om e^{beta phibar}/a and potential alpha lambda^2 a^2 (Eq. csf_eom_code).
int make_model(const mgglam_params* prm, double a, int Nfine, ModelDev* m) {
  memset(m, 0, sizeof(*m));
  if (!(a > 0.0) || !(prm->box > 0.0)) return MGGLAM_ERR_ARG;
  const double ct = ((double)Nfine / prm->box) * kCOverH0;
  m->c2 = ct * ct;
  m->om_a = prm->omega_m / a;
  switch (prm->model) {
    case MGGLAM_FR: {
      if (prm->n < 0 || prm->n > 2 || !(prm->fR0_abs > 0.0)) return MGGLAM_ERR_ARG;
      const double Rb_a = 3.0 * (prm->omega_m / (a * a * a) + 4.0 * prm->omega_l);
      const double Rb_1 = 3.0 * (prm->omega_m + 4.0 * prm->omega_l);
      const double fRbar = -prm->fR0_abs * pow(Rb_1 / Rb_a, (double)(prm->n + 1));
      m->ubar = pow(-fRbar, 1.0 / (double)(prm->n + 1));
      m->K0 = Rb_a * a * a / 3.0;
      m->K = m->K0 * m->ubar;
      m->kind = prm->n;  // KFR0, KFR1, KFR2
      break;
    }
    case MGGLAM_SYMMETRON: {
      if (!(prm->xi > 0.0) || !(prm->a_star > 0.0)) return MGGLAM_ERR_ARG;
      const double r = prm->a_star / a;
      const double s = 1.0 - r * r * r;
      m->ubar = s > 0.0 ? sqrt(s) : 0.0;
      m->msym = a * a / (2.0 * prm->xi * prm->xi);
      m->rat3 = r * r * r;
      m->xi2_a2 = prm->xi * prm->xi / (a * a);
      m->kind = KSYM;
      break;
    }
    case MGGLAM_CQ: {
      if (!(prm->phibar > 0.0) || !(prm->alpha > 0.0)) return MGGLAM_ERR_ARG;
      m->ubar = 0.0;
      m->cq_src = 3.0 * prm->beta * prm->omega_m * exp(prm->beta * prm->phibar) / a;
      m->cq_pot = prm->alpha * prm->lambda * prm->lambda * a * a;
      m->alpha = prm->alpha;
      m->phibar = prm->phibar;
      m->beta = prm->beta;
      m->pot0 = pow(prm->phibar, -1.0 - prm->alpha);
      m->keep_exp = prm->keep_exp ? 1 : 0;
      m->kind = KCQ;
      break;
    }
    default:
      return MGGLAM_ERR_ARG;
  }
  return MGGLAM_OK;
}

// ---------------------------------------------------------------------------
// Scratch cache
// ---------------------------------------------------------------------------

static std::mutex g_mu;
static Workspace* g_ws[64];
static int g_nws = 0;

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

int get_workspace(int N, int precision, int levels, Workspace** out) {
  int dev = 0;
  MG_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < g_nws; ++i) {
    Workspace* w = g_ws[i];
    if (w->device == dev && w->N == N && w->precision == precision && w->levels_req == levels) {
      *out = w;
      return MGGLAM_OK;
    }
  }
  if (g_nws >= 64) return MGGLAM_ERR_OOM;
  Workspace* w = new Workspace();
  w->device = dev;
  w->N = N;
  w->precision = precision;
  w->levels_req = levels;
  w->nlev = count_levels(N, levels);
  // layout pass (sizes), then one allocation
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
  size_t o_partials = take(kMaxReduceBlocks * sizeof(double));
  size_t o_scalars = take(SC_COUNT * sizeof(double));
  size_t o_src64 = precision == MGGLAM_MIXED ? take((size_t)N * N * N * sizeof(double)) : 0;
  struct Offs { size_t u, rho, S, Ru, e, e_alt, ub, S32, Re, rho32; } offs[kMaxLevels];
  for (int l = 0, n = N; l < w->nlev; ++l, n /= 2) {
    Level& L = w->lev[l];
    L.n = n;
    L.h = (double)(1 << l);
    L.n3 = (size_t)n * n * n;
    Offs& o = offs[l];
    memset(&o, 0xff, sizeof(o));
    o.rho = take(L.n3 * 8);
    if (precision == MGGLAM_FP64 || l == 0) {
      if (l > 0) {
        o.u = take(L.n3 * 8);
        o.S = take(L.n3 * 8);
        o.Ru = take(L.n3 * 8);
      }
    }
    if (precision == MGGLAM_MIXED) {
      o.e = take(L.n3 * 4);
      o.e_alt = take(L.n3 * 4);
      o.ub = take(L.n3 * 4);
      o.S32 = take(L.n3 * 4);
      if (l > 0) o.Re = take(L.n3 * 4);
      o.rho32 = take(L.n3 * 4);
    }
  }
  if (cudaMalloc(&w->base, off) != cudaSuccess) {
    cudaGetLastError();
    delete w;
    return MGGLAM_ERR_OOM;
  }
  if (cudaMallocHost((void**)&w->h_scalars, SC_COUNT * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(w->base);
    delete w;
    return MGGLAM_ERR_OOM;
  }
  w->bytes = off;
  char* b = (char*)w->base;
  w->partials = (double*)(b + o_partials);
  w->scalars = (double*)(b + o_scalars);
  if (precision == MGGLAM_MIXED) w->src64 = (double*)(b + o_src64);
  const size_t NONE = ~(size_t)0;
  for (int l = 0; l < w->nlev; ++l) {
    Level& L = w->lev[l];
    Offs& o = offs[l];
    L.rho = (double*)(b + o.rho);
    if (o.u != NONE) L.u = (double*)(b + o.u);
    if (o.S != NONE) L.S = (double*)(b + o.S);
    if (o.Ru != NONE) L.Ru = (double*)(b + o.Ru);
    if (o.e != NONE) L.e = (float*)(b + o.e);
    if (o.e_alt != NONE) L.e_alt = (float*)(b + o.e_alt);
    if (o.ub != NONE) L.ub = (float*)(b + o.ub);
    if (o.S32 != NONE) L.S32 = (float*)(b + o.S32);
    if (o.Re != NONE) L.Re = (float*)(b + o.Re);
    if (o.rho32 != NONE) L.rho32 = (float*)(b + o.rho32);
  }
  g_ws[g_nws++] = w;
  *out = w;
  return MGGLAM_OK;
}

void release_workspaces() {
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  int keep = 0;
  for (int i = 0; i < g_nws; ++i) {
    Workspace* w = g_ws[i];
    if (w->device == dev) {
      if (w->coarse_exec) cudaGraphExecDestroy(w->coarse_exec);
      if (w->cap_stream) cudaStreamDestroy(w->cap_stream);
      cudaFree(w->base);
      cudaFreeHost(w->h_scalars);
      if (w->cic_acc) cudaFree(w->cic_acc);
      delete w;
    } else {
      g_ws[keep++] = w;
    }
  }
  g_nws = keep;
}

static int check_mesh(int N) { return (N >= 4 && N <= 2048 && N % 2 == 0) ? MGGLAM_OK : MGGLAM_ERR_SHAPE; }

}  // namespace mg

using namespace mg;

extern "C" {

const char* mgglam_version(void) { return "mgglam-gb300 0.1 (sm_103a)"; }

const char* mgglam_status_string(int s) {
  switch (s) {
    case MGGLAM_OK: return "ok";
    case MGGLAM_ERR_ARG: return "invalid argument";
    case MGGLAM_ERR_SHAPE: return "unsupported mesh size";
    case MGGLAM_ERR_CUDA: return "CUDA error";
    case MGGLAM_ERR_NOT_CONVERGED: return "not converged";
    case MGGLAM_ERR_NONFINITE: return "non-finite residual";
    case MGGLAM_ERR_TIMEOUT: return "device wait timed out";
    case MGGLAM_ERR_OOM: return "out of device memory";
    default: return "unknown status";
  }
}

int mgglam_default_params(mgglam_params* p) {
  if (!p) return MGGLAM_ERR_ARG;
  memset(p, 0, sizeof(*p));
  p->model = MGGLAM_FR;
  p->n = 1;
  p->precision = MGGLAM_MIXED;
  p->fR0_abs = 1e-5;
  p->omega_m = 0.3;
  p->omega_l = 0.7;
  p->box = 256.0;
  p->a_star = 0.5;
  p->xi = 100.0 / 299792.458;
  p->beta_star = 1.0;
  p->alpha = 0.1;
  p->beta = -0.05;
  p->lambda = 1.0;
  p->phibar = 1.0;
  p->levels = 0;
  p->nu1 = 2;
  p->nu2 = 2;
  p->coarse_sweeps = 16;
  p->max_cycles = 50;
  p->inner_cycles = 0;
  p->check_every = 1;
  return MGGLAM_OK;
}

static int check_params(const mgglam_params* prm) {
  if (!prm) return MGGLAM_ERR_ARG;
  if (prm->nu1 < 0 || prm->nu2 < 0 || prm->coarse_sweeps < 0 || prm->max_cycles < 0) return MGGLAM_ERR_ARG;
  if (prm->precision != MGGLAM_FP64 && prm->precision != MGGLAM_MIXED) return MGGLAM_ERR_ARG;
  if (prm->cycle < 0 || prm->cycle > 2) return MGGLAM_ERR_ARG;
  if (prm->fmg != 0 && prm->fmg != 1) return MGGLAM_ERR_ARG;
  return MGGLAM_OK;
}

int mgglam_solve_scalar(const mgglam_params* prm, double a, const float* rho, int N, double* field,
                        double tol, mgglam_stats* stats, void* stream) {
  int rc = check_params(prm);
  if (rc) return rc;
  if (!rho || !field || !(tol >= 0.0)) return MGGLAM_ERR_ARG;
  if ((rc = check_mesh(N))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (prm->precision == MGGLAM_FP64) return solve_fp64(prm, a, rho, N, field, tol, stats, st);
  return solve_mixed(prm, a, rho, N, field, tol, stats, st);
}

int mgglam_deposit_cic(const float* pos, long long np, int N, float* rho, void* stream) {
  if (!pos || !rho || np < 1) return MGGLAM_ERR_ARG;
  if (N < 2 || N > 2048) return MGGLAM_ERR_SHAPE;
  return deposit_cic(pos, np, N, rho, (cudaStream_t)stream);
}

int mgglam_gather_force(const mgglam_params* prm, double a, const double* field, int N, const float* pos,
                        long long np, float* force, double prefactor, void* stream) {
  if (!prm || !field || !pos || !force || np < 1) return MGGLAM_ERR_ARG;
  int rc = check_mesh(N);
  if (rc) return rc;
  ModelDev m;
  if ((rc = make_model(prm, a, N, &m))) return rc;
  return gather_force(m, m.kind, prm->n, prm, field, N, pos, np, force, prefactor, (cudaStream_t)stream);
}

int mgglam_deposit_cic_host(const float* pos_host, float* pos_dev, long long np, int N, float* rho, int chunks,
                            void* stream) {
  if (!pos_host || !pos_dev || !rho || np < 1 || chunks < 0 || chunks > 32) return MGGLAM_ERR_ARG;
  if (N < 2 || N > 2048) return MGGLAM_ERR_SHAPE;
  return deposit_cic_host(pos_host, pos_dev, np, N, rho, chunks ? chunks : 8, (cudaStream_t)stream);
}

int mgglam_gather_force_host(const mgglam_params* prm, double a, const double* field, int N, const float* pos_dev,
                             long long np, float* force_dev, float* force_host, double prefactor, int chunks,
                             void* stream) {
  if (!prm || !field || !pos_dev || !force_dev || !force_host || np < 1 || chunks < 0 || chunks > 32)
    return MGGLAM_ERR_ARG;
  int rc = check_mesh(N);
  if (rc) return rc;
  ModelDev m;
  if ((rc = make_model(prm, a, N, &m))) return rc;
  return gather_force_host(m, m.kind, prm, field, N, pos_dev, np, force_dev, force_host, prefactor,
                           chunks ? chunks : 8, (cudaStream_t)stream);
}

int mgglam_smooth(const mgglam_params* prm, double a, int n, double h, double* u, const double* rho,
                  const double* S, int sweeps, void* stream) {
  if (!prm || !u || !rho || sweeps < 0 || !(h >= 1.0)) return MGGLAM_ERR_ARG;
  if (n < 2 || n % 2) return MGGLAM_ERR_SHAPE;
  ModelDev m;
  int rc = make_model(prm, a, (int)llround(n * h), &m);
  if (rc) return rc;
  return launch_smooth64(m, n, h, u, rho, S, sweeps, (cudaStream_t)stream);
}

int mgglam_residual(const mgglam_params* prm, double a, int n, double h, const double* u, const double* rho,
                    const double* S, double* d, double* sumsq, void* stream) {
  if (!prm || !u || !rho || !(h >= 1.0)) return MGGLAM_ERR_ARG;
  if (n < 2) return MGGLAM_ERR_SHAPE;
  ModelDev m;
  int rc = make_model(prm, a, (int)llround(n * h), &m);
  if (rc) return rc;
  Workspace* ws = nullptr;
  // a small cache entry provides the partial-sum scratch
  if ((rc = get_workspace(4, MGGLAM_FP64, 1, &ws))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = launch_residual64(m, n, h, u, rho, S, d, ws->partials, ws->scalars + SC_SUMSQ, st))) return rc;
  if (sumsq) {
    MG_CUDA_TRY(cudaMemcpyAsync(ws->h_scalars + SC_SUMSQ, ws->scalars + SC_SUMSQ, sizeof(double),
                                cudaMemcpyDeviceToHost, st));
    MG_CUDA_TRY(cudaStreamSynchronize(st));
    *sumsq = ws->h_scalars[SC_SUMSQ];
  }
  return MGGLAM_OK;
}

int mgglam_restrict(int n, const double* fine, double* coarse, void* stream) {
  if (!fine || !coarse) return MGGLAM_ERR_ARG;
  if (n < 2 || n % 2) return MGGLAM_ERR_SHAPE;
  return launch_restrict64(n, fine, coarse, (cudaStream_t)stream);
}

int mgglam_prolong_correct(const mgglam_params* prm, int n, const double* uH, const double* RuH, double* u_fine,
                           void* stream) {
  if (!prm || !uH || !RuH || !u_fine) return MGGLAM_ERR_ARG;
  if (n < 2 || n % 2) return MGGLAM_ERR_SHAPE;
  ModelDev m;
  memset(&m, 0, sizeof(m));
  m.kind = prm->model == MGGLAM_FR ? KFR1 : (prm->model == MGGLAM_SYMMETRON ? KSYM : KCQ);
  return launch_prolong_correct64(m, n / 2, uH, RuH, nullptr, u_fine, (cudaStream_t)stream);
}

int mgglam_poisson_fft(const float* rho, int N, double coef, float* phi, void* stream) {
  if (!rho || !phi || rho == phi || !(coef == coef)) return MGGLAM_ERR_ARG;
  return poisson_fft(rho, N, coef, phi, (cudaStream_t)stream);
}

int mgglam_pm_step(const mgglam_params* prm, const mgglam_pm_step_desc* d, int N, float* pos, float* mom,
                   long long np, double* field, double tol, float* rho_work, float* psi_work, mgglam_stats* stats,
                   void* stream) {
  int rc = check_params(prm);
  if (rc) return rc;
  if (!d || !pos || !mom || np < 1 || !rho_work || !psi_work || rho_work == psi_work) return MGGLAM_ERR_ARG;
  if (d->scalar && (!field || !(tol >= 0.0))) return MGGLAM_ERR_ARG;
  if (!(d->a > 0.0) || !(d->da > 0.0) || !(d->E_a > 0.0) || !(d->E_half > 0.0) || !(d->dphibar_da == d->dphibar_da))
    return MGGLAM_ERR_ARG;
  if (N < 8 || N > 1024 || (N & (N - 1))) return MGGLAM_ERR_SHAPE;
  return pm_step(prm, d, N, pos, mom, np, field, tol, rho_work, psi_work, stats, (cudaStream_t)stream);
}

int mgglam_release(void) {
  cudaError_t e = cudaDeviceSynchronize();
  release_workspaces();
  release_fft_plans();
  release_adjoint_work();
  release_batches();
  forget_static_deposit_address();
  return e == cudaSuccess ? MGGLAM_OK : MGGLAM_ERR_CUDA;
}

}  // extern "C"
