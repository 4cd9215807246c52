// pm.cu -- one particle-mesh time step of the N-body code (Sec. 3.1, with the
// modified-gravity forces of Secs. 3.2.3-3.2.5).
//
// Step from a_n to a_n + da, positions x at a_n, momenta p at a_n - da/2:
//   1. rho      = CIC deposit of x                                  (mgglam_deposit_cic)
//   2. Phi_N    : grad^2 Phi_N = (3/2) Om / a_n delta                (Eq. GR_poisson_codeunit; FFT)
//   3. scalar   : the model's field equation at a_n, from the field of the previous step
//   4. Psi      = s5 T(field) - sN Phi_N; the force is (H0/adot) grad Psi with
//        sN = e^{beta phibar} (CQ: the Newtonian force carries the background coupling), 1 otherwise;
//        s5 T the fifth-force potential of mgglam_gather_force (f(R): (c~^2/2) f_R;
//        symmetron: -3 xi^2 Om beta*^2 c~^2 a*^-3 u^2; CQ: -beta phi~)
//   5. kick     : dp/da = (H0/adot) grad Psi - gamma p   (Eqs. csf_particle_geodesic_code2, F_x_codeunit)
//        gamma = beta dphibar/da (CQ); 9 Om beta*^2 xi^2 sqrt(1 - (a*/a)^3) a^-4 u(x) (symmetron, a > a*);
//        0 otherwise.  Leapfrog with the drag taken at the midpoint:
//        p' = [p (1 - gamma da/2) + da (H0/adot) grad Psi] / (1 + gamma da/2)
//   6. drift    : dx/da = H0 / (a^2 adot) p, evaluated at a_n + da/2; x wrapped into [0, N).
// With H0/adot = 1 / (a E(a)), E = H/H0 given by the caller at a_n and a_n + da/2.
#include <math.h>

#include "cic.cuh"
#include "ff.cuh"
#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

// Psi = s5 (T - Tbar) - sN Phi_N in place over phi (FP64 field, FP32 Psi); the
// transform T as in the gather (k_transform: float-float for f(R) and the
// symmetron, FP64 for CQ).
template <int K, bool SCALAR>
__global__ void k_pm_potential(const double* __restrict__ u, float* __restrict__ phi, long long n3, double ubar,
                               double beta, float s5, float sN) {
  const ff ub = ff_from_double(ubar);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    float v = -sN * phi[t];
    if constexpr (SCALAR) {
      float d;
      if constexpr (K == KCQ) {
        d = (float)(beta * u[t]);
      } else {
        const ff w = ff_from_double(u[t]);
        const ff dw_ = ff_sub(w, ub);
        ff T;
        if constexpr (K == KFR0) T = ff_neg(dw_);
        else if constexpr (K == KFR1) T = ff_neg(ff_mul(dw_, ff_add(w, ub)));
        else if constexpr (K == KFR2) T = ff_neg(ff_mul(dw_, ff_add(ff_add(ff_sqr(w), ff_mul(w, ub)), ff_sqr(ub))));
        else T = ff_mul(dw_, ff_add(w, ub));
        d = ff_to_float(T);
      }
      v = fmaf(s5, d, v);
    }
    phi[t] = v;
  }
}

// CIC interpolation of an FP64 mesh at (x, y, z), in single precision.
__device__ __forceinline__ float cic_interp64(const double* __restrict__ u, int N, float x, float y, float z) {
  int i0, i1, j0, j1, k0, k1;
  float wx[2], wy[2], wz[2];
  cic_axis_f(x, N, i0, i1, wx[0], wx[1]);
  cic_axis_f(y, N, j0, j1, wy[0], wy[1]);
  cic_axis_f(z, N, k0, k1, wz[0], wz[1]);
  const int ii[2] = {i0, i1}, jj[2] = {j0, j1}, kk[2] = {k0, k1};
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 2; ++c)
        s += wx[a] * wy[b] * wz[c] * (float)u[((long long)ii[a] * N + jj[b]) * N + kk[c]];
  return s;
}

// Kick and drift of every particle.  kick = da H0/adot(a_n); drift = da H0/(a^2 adot) at
// a_n + da/2; gdrag = gamma da for a uniform drag (CQ); sym_drag = the symmetron's
// gamma da per unit u (0 when absent), u interpolated from the field.
__global__ void __launch_bounds__(kThreads) k_pm_kick_drift(const float* __restrict__ psi, int N,
                                                            float* __restrict__ pos, float* __restrict__ mom,
                                                            long long np, float kick, float drift, float gdrag,
                                                            float sym_drag, const double* __restrict__ field) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < np;
       q += (long long)gridDim.x * blockDim.x) {
    const float x = pos[3 * q + 0], y = pos[3 * q + 1], z = pos[3 * q + 2];
    const float3 g = cic_grad(psi, N, x, y, z);
    float gd = gdrag;
    if (sym_drag != 0.f) gd += sym_drag * cic_interp64(field, N, x, y, z);
    const float c0 = 1.f - 0.5f * gd, ci = 1.f / (1.f + 0.5f * gd);
    const float px = (mom[3 * q + 0] * c0 + kick * g.x) * ci;
    const float py = (mom[3 * q + 1] * c0 + kick * g.y) * ci;
    const float pz = (mom[3 * q + 2] * c0 + kick * g.z) * ci;
    mom[3 * q + 0] = px;
    mom[3 * q + 1] = py;
    mom[3 * q + 2] = pz;
    pos[3 * q + 0] = wrap_pos(x + drift * px, N);
    pos[3 * q + 1] = wrap_pos(y + drift * py, N);
    pos[3 * q + 2] = wrap_pos(z + drift * pz, N);
  }
}

// Fifth-force potential factor s5 (the gather's force_scale).
static double pm_s5(const ModelDev& m, const mgglam_params* prm) {
  if (is_fr(m.kind)) return 0.5 * m.c2;
  if (m.kind == KSYM)
    return -3.0 * prm->xi * prm->xi * prm->omega_m * prm->beta_star * prm->beta_star * m.c2 /
           (prm->a_star * prm->a_star * prm->a_star);
  return -1.0;
}

int pm_step(const mgglam_params* prm, const mgglam_pm_step_desc* d, int N, float* pos, float* mom, long long np,
            double* field, double tol, float* rho_work, float* psi_work, mgglam_stats* stats, cudaStream_t st) {
  const double a = d->a, da = d->da;
  int rc;
  ModelDev m;
  if ((rc = make_model(prm, a, N, &m))) return rc;
  const long long n3 = (long long)N * N * N;
  // 1-2: density and Newtonian potential
  if ((rc = deposit_cic(pos, np, N, rho_work, st))) return rc;
  if ((rc = poisson_fft(rho_work, N, 1.5 * prm->omega_m / a, psi_work, st))) return rc;
  // 3: the scalar field (warm start from the caller's field)
  int solve_rc = MGGLAM_OK;
  if (d->scalar) {
    solve_rc = prm->precision == MGGLAM_FP64 ? solve_fp64(prm, a, rho_work, N, field, tol, stats, st)
                                             : solve_mixed(prm, a, rho_work, N, field, tol, stats, st);
    if (solve_rc != MGGLAM_OK && solve_rc != MGGLAM_ERR_NOT_CONVERGED) return solve_rc;
  }
  // 4: total potential
  const float sN = (float)(d->scalar && m.kind == KCQ ? exp(prm->beta * prm->phibar) : 1.0);
  const float s5 = (float)pm_s5(m, prm);
  const int g = stream_grid(n3);
  prof_begin(PC_PM_POTENTIAL, st, (d->scalar ? 16.0 : 8.0) * n3);
  if (!d->scalar) {
    k_pm_potential<KFR1, false><<<g, kThreads, 0, st>>>(nullptr, psi_work, n3, 0.0, 0.0, 0.f, sN);
  } else {
    switch (m.kind) {
      case KFR0: k_pm_potential<KFR0, true><<<g, kThreads, 0, st>>>(field, psi_work, n3, m.ubar, 0.0, s5, sN); break;
      case KFR1: k_pm_potential<KFR1, true><<<g, kThreads, 0, st>>>(field, psi_work, n3, m.ubar, 0.0, s5, sN); break;
      case KFR2: k_pm_potential<KFR2, true><<<g, kThreads, 0, st>>>(field, psi_work, n3, m.ubar, 0.0, s5, sN); break;
      case KSYM: k_pm_potential<KSYM, true><<<g, kThreads, 0, st>>>(field, psi_work, n3, m.ubar, 0.0, s5, sN); break;
      default: k_pm_potential<KCQ, true><<<g, kThreads, 0, st>>>(field, psi_work, n3, 0.0, prm->beta, s5, sN); break;
    }
  }
  prof_end(st);
  note_launch(1);
  // 5-6: kick and drift
  const double ah = a + 0.5 * da;
  const float kick = (float)(da / (a * d->E_a));
  const float drift = (float)(da / (ah * ah * ah * d->E_half));
  float gdrag = 0.f, sym_drag = 0.f;
  if (d->scalar && m.kind == KCQ) gdrag = (float)(prm->beta * d->dphibar_da * da);
  if (d->scalar && m.kind == KSYM && prm->a_star < a) {
    const double r = prm->a_star / a;
    sym_drag = (float)(9.0 * prm->omega_m * prm->beta_star * prm->beta_star * prm->xi * prm->xi *
                       sqrt(1.0 - r * r * r) / (a * a * a * a) * da);
  }
  prof_begin(PC_PM_KICK_DRIFT, st, 48.0 * np + 4.0 * n3);
  k_pm_kick_drift<<<grid_for(np, kThreads, 1 << 20), kThreads, 0, st>>>(psi_work, N, pos, mom, np, kick, drift,
                                                                         gdrag, sym_drag, field);
  prof_end(st);
  note_launch(1);
  MG_CUDA_TRY(cudaGetLastError());
  return solve_rc;
}

}  // namespace mg
