// solve64.cu -- FP64 multigrid kernels and the plain-FP64 FAS solver.
//
// FAS V-cycle (Sec. 3.2.1): on each level nu1 red-black sweeps, restriction of
// u and of the local residual d (8-child mean), coarse source
// S^H = N^H(R u) - R d (Eq. general_pde_numerical_coarse), coarse initial guess
// R u, recursion, correction u += P(u^H - R u) (Eq. solution_correction, 27/9/3/1
// weights), nu2 sweeps.  The coarsest level is relaxed with a fixed number of
// sweeps by a single CTA.
#include <math.h>
#include <stdio.h>

#include <chrono>

#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

// ---------------------------------------------------------------------------
// Device arithmetic of one cell
// ---------------------------------------------------------------------------

// Sum over the six face neighbours of the field that enters the Laplacian
// (f(R): w = u^{n+1}; symmetron, CQ: u itself).
template <int K>
__device__ __forceinline__ double nb_sum64(const double* __restrict__ u, int n, int i, int j, int k) {
  const int ip = wrapi(i + 1, n), im = wrapi(i - 1, n);
  const int jp = wrapi(j + 1, n), jm = wrapi(j - 1, n);
  const int kp = wrapi(k + 1, n), km = wrapi(k - 1, n);
  return fr_or_id<K>(u[cidx(n, ip, j, k)]) + fr_or_id<K>(u[cidx(n, im, j, k)]) +
         fr_or_id<K>(u[cidx(n, i, jp, k)]) + fr_or_id<K>(u[cidx(n, i, jm, k)]) +
         fr_or_id<K>(u[cidx(n, i, j, kp)]) + fr_or_id<K>(u[cidx(n, i, j, km)]);
}

// N_h(u) at one cell (see mg_model.cuh for the three operators).
template <int K>
__device__ __forceinline__ double local_N64(const ModelDev& m, double h, double uc, double rhoc,
                                            double Lnb) {
  const double ih2 = 1.0 / (h * h);
  if constexpr (is_fr(K)) {
    const double w = fr_w<K>(uc);
    return -m.c2 * (Lnb - 6.0 * w) * ih2 + m.om_a * (rhoc - 1.0) + m.K0 - m.K / uc;
  } else if constexpr (K == KSYM) {
    return m.c2 * (Lnb - 6.0 * uc) * ih2 - m.msym * ((rhoc * m.rat3 - 1.0) * uc + uc * uc * uc);
  } else {
    const double E = m.keep_exp ? exp(m.beta * uc / m.c2) : 1.0;
    const double x = m.phibar + uc / m.c2;
    return (Lnb - 6.0 * uc) * ih2 - m.cq_src * (E * rhoc - 1.0) +
           m.cq_pot * (pow(x, -1.0 - m.alpha) - m.pot0);
  }
}

// Gauss-Seidel update of one cell: the exact local root for f(R) and the
// symmetron (nonlinear GS, Secs. 3.2.4-3.2.5), one Newton step for CQ
// (Eq. relaxation_iteration, Sec. 3.2.3).  The FAS source S enters p (f(R))
// or q (symmetron) of the local polynomial.
template <int K>
__device__ __forceinline__ double local_update64(const ModelDev& m, double h, double uc,
                                                 double rhoc, double s, double Lnb) {
  if constexpr (is_fr(K)) {
    const double al = h * h / (6.0 * m.c2);
    const double p = al * (m.om_a * (rhoc - 1.0) + m.K0 - s) - Lnb * (1.0 / 6.0);
    const double q = -al * m.K;
    return fr_root<K>(p, q);
  } else if constexpr (K == KSYM) {
    const double g = m.c2 * m.xi2_a2 / (h * h);
    const double p = rhoc * m.rat3 - 1.0 + 12.0 * g;
    const double q = -2.0 * g * Lnb + 2.0 * m.xi2_a2 * s;
    return sym_root(p, q, uc);
  } else {
    const double ih2 = 1.0 / (h * h);
    const double x = m.phibar + uc / m.c2;
    const double E = m.keep_exp ? exp(m.beta * uc / m.c2) : 1.0;
    const double dE = m.keep_exp ? (m.beta / m.c2) * E : 0.0;
    const double px = pow(x, -1.0 - m.alpha);
    const double r = (Lnb - 6.0 * uc) * ih2 - m.cq_src * (E * rhoc - 1.0) + m.cq_pot * (px - m.pot0) - s;
    const double dr = -6.0 * ih2 - m.cq_src * dE * rhoc - m.cq_pot * (1.0 + m.alpha) * px / (x * m.c2);
    return uc - r / dr;
  }
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Relax every cell of one colour ((i+j+k) % 2 == parity); one thread per cell.
template <int K>
__global__ void __launch_bounds__(kThreads) k_smooth64(ModelDev m, int n, double h, double* __restrict__ u,
                                                       const double* __restrict__ rho,
                                                       const double* __restrict__ S, int parity) {
  const int i = blockIdx.z, j = blockIdx.y;
  const int kk = blockIdx.x * blockDim.x + threadIdx.x;
  if (kk >= (n >> 1)) return;
  const int k = 2 * kk + ((i + j + parity) & 1);
  const size_t c = cidx(n, i, j, k);
  const double Lnb = nb_sum64<K>(u, n, i, j, k);
  u[c] = local_update64<K>(m, h, u[c], rho[c], S ? S[c] : 0.0, Lnb);
}

// d = N(u) - S on every cell; optional store of d; per-block partial sums of d^2.
template <int K>
__global__ void __launch_bounds__(kThreads) k_residual64(ModelDev m, int n, double h, const double* __restrict__ u,
                                                         const double* __restrict__ rho,
                                                         const double* __restrict__ S, double* __restrict__ d,
                                                         double* __restrict__ partials) {
  double acc = 0.0;
  // grid-stride over rows (i, j), threads along k
  for (int r = blockIdx.x; r < n * n; r += gridDim.x) {
    const int i = r / n, j = r - (r / n) * n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const size_t t = cidx(n, i, j, k);
      const double v = local_N64<K>(m, h, u[t], rho[t], nb_sum64<K>(u, n, i, j, k)) - (S ? S[t] : 0.0);
      if (d) d[t] = v;
      acc += v * v;
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Sum 'count' partials in a fixed order into *out (one block).
__global__ void k_finalize_sum(const double* __restrict__ partials, int count, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partials[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

// coarse = mean of the 8 children.
__global__ void k_restrict64(int nf, const double* __restrict__ fine, double* __restrict__ coarse) {
  const int nc = nf >> 1;
  const int I = blockIdx.z, J = blockIdx.y;
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= nc) return;
  double s = 0.0;
  for (int di = 0; di < 2; ++di)
    for (int dj = 0; dj < 2; ++dj)
      for (int dk = 0; dk < 2; ++dk) s += fine[cidx(nf, 2 * I + di, 2 * J + dj, 2 * K + dk)];
  coarse[cidx(nc, I, J, K)] = s * 0.125;
}

// Fused: for each coarse cell, the local residual of its 8 children is formed
// on the fly (the recomputation the paper also does, Sec. 3.2.2) and averaged
// into Rd; the children's solution is averaged into Ru and copied to uH.
template <int K>
__global__ void __launch_bounds__(kThreads) k_residual_restrict64(ModelDev m, int nf, double hf,
                                                                  const double* __restrict__ u,
                                                                  const double* __restrict__ rho,
                                                                  const double* __restrict__ S,
                                                                  double* __restrict__ Ru, double* __restrict__ uH,
                                                                  double* __restrict__ Rd) {
  const int nc = nf >> 1;
  const int I = blockIdx.z, J = blockIdx.y;
  const int K0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (K0 < nc) {
    const size_t t = cidx(nc, I, J, K0);
    double su = 0.0, sd = 0.0;
    for (int di = 0; di < 2; ++di)
      for (int dj = 0; dj < 2; ++dj)
        for (int dk = 0; dk < 2; ++dk) {
          const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K0 + dk;
          const size_t c = cidx(nf, i, j, k);
          const double uc = u[c];
          su += uc;
          sd += local_N64<K>(m, hf, uc, rho[c], nb_sum64<K>(u, nf, i, j, k)) - (S ? S[c] : 0.0);
        }
    const double ru = su * 0.125;
    Ru[t] = ru;
    uH[t] = ru;
    Rd[t] = sd * 0.125;
  }
}

// In place: S <- N^H(Ru) - S, where S holds R d on entry.
template <int K>
__global__ void __launch_bounds__(kThreads) k_fas_source64(ModelDev m, int n, double h, const double* __restrict__ Ru,
                                                           const double* __restrict__ rho, double* __restrict__ S) {
  const int i = blockIdx.z, j = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const size_t t = cidx(n, i, j, k);
  S[t] = local_N64<K>(m, h, Ru[t], rho[t], nb_sum64<K>(Ru, n, i, j, k)) - S[t];
}

// The prolongation weight stencil at fine cell (i,j,k) of coarse field c (side nc).
__device__ __forceinline__ double prolong_at64(const double* __restrict__ c, int nc, int i, int j, int k) {
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  const int I2 = wrapi(I + ((i & 1) ? 1 : -1), nc);
  const int J2 = wrapi(J + ((j & 1) ? 1 : -1), nc);
  const int K2 = wrapi(K + ((k & 1) ? 1 : -1), nc);
  const double v = 27.0 * c[cidx(nc, I, J, K)] +
                   9.0 * (c[cidx(nc, I2, J, K)] + c[cidx(nc, I, J2, K)] + c[cidx(nc, I, J, K2)]) +
                   3.0 * (c[cidx(nc, I2, J2, K)] + c[cidx(nc, I2, J, K2)] + c[cidx(nc, I, J2, K2)]) +
                   c[cidx(nc, I2, J2, K2)];
  return v * (1.0 / 64.0);
}

// u^h += P(u^H - R u^h); f(R): non-positive results fall back to half the old value.
template <bool FR>
__global__ void __launch_bounds__(kThreads) k_prolong_correct64(int nc, const double* __restrict__ uH,
                                                                const double* __restrict__ RuH,
                                                                double* __restrict__ uf,
                                                                unsigned long long* guard) {
  const int nf = nc << 1;
  const int i = blockIdx.z, j = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nf) {
    const size_t t = cidx(nf, i, j, k);
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const int I2 = wrapi(I + ((i & 1) ? 1 : -1), nc);
    const int J2 = wrapi(J + ((j & 1) ? 1 : -1), nc);
    const int K2 = wrapi(K + ((k & 1) ? 1 : -1), nc);
#define EH(a, b, c) (uH[cidx(nc, a, b, c)] - RuH[cidx(nc, a, b, c)])
    const double corr = (27.0 * EH(I, J, K) + 9.0 * (EH(I2, J, K) + EH(I, J2, K) + EH(I, J, K2)) +
                         3.0 * (EH(I2, J2, K) + EH(I2, J, K2) + EH(I, J2, K2)) + EH(I2, J2, K2)) *
                        (1.0 / 64.0);
#undef EH
    const double old = uf[t];
    double v = old + corr;
    if (FR && !(v > 0.0)) {
      v = 0.5 * old;
      count_guards(guard, 1u);
    }
    uf[t] = v;
  }
}

// Coarsest level: 'sweeps' red-black sweeps by one CTA (the level is tiny).
template <int K>
__global__ void __launch_bounds__(512) k_coarse64(ModelDev m, int n, double h, double* __restrict__ u,
                                                  const double* __restrict__ rho,
                                                  const double* __restrict__ S, int sweeps) {
  const int n3 = n * n * n;
  for (int s = 0; s < sweeps; ++s) {
    for (int parity = 0; parity < 2; ++parity) {
      for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int k = t % n, j = (t / n) % n, i = t / (n * n);
        if (((i + j + k) & 1) != parity) continue;
        const double Lnb = nb_sum64<K>(u, n, i, j, k);
        u[t] = local_update64<K>(m, h, u[t], rho[t], S ? S[t] : 0.0, Lnb);
      }
      __syncthreads();
    }
  }
}

__global__ void k_sum_f32(const float* __restrict__ x, long long n3, double* __restrict__ partials) {
  FloatFloat acc;  // FP32 arithmetic (GB300's FP64 rate is 1/64 of FP32), exact to ~1e-14
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    acc.add(x[t]);
  const double a = block_sum(acc.value());
  if (threadIdx.x == 0) partials[blockIdx.x] = a;
}

// rho64 = rho32 / mean, mean = sum / n3 read from device memory.
__global__ void k_density_to64(const float* __restrict__ rho32, long long n3, const double* __restrict__ sum,
                               double* __restrict__ rho64) {
  const double inv_mean = (double)n3 / *sum;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    rho64[t] = (double)rho32[t] * inv_mean;
}

// Sum of squares of the model's linear source term (relative-residual scale).
template <int K>
__global__ void k_src_sumsq(ModelDev m, const double* __restrict__ rho, long long n3, double* __restrict__ partials) {
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    const double delta = rho[t] - 1.0;
    double s;
    if constexpr (is_fr(K)) s = m.om_a * delta;
    else if constexpr (K == KSYM) s = m.msym * m.rat3 * delta * m.ubar;
    else s = m.cq_src * delta;
    acc += s * s;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// If field[0] is NaN, fill the field with the background value.
__global__ void k_init_background(double* __restrict__ field, long long n3, double ubar) {
  if (!isnan(field[0])) return;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    if (t != 0) field[t] = ubar;
}
__global__ void k_init_background_first(double* __restrict__ field, double ubar) {
  if (isnan(field[0])) field[0] = ubar;
}

// ---------------------------------------------------------------------------
// Launchers (dispatch on the model kind)
// ---------------------------------------------------------------------------

// 3D grid for kernels indexed (x: k, y: j, z: i) with k3dThreads threads along k.
constexpr int k3dThreads = 64;
static dim3 grid3d(int n_k, int n_j, int n_i) { return dim3((n_k + k3dThreads - 1) / k3dThreads, n_j, n_i); }

#define MG_DISPATCH(kind, KERNEL_CALL)                       \
  switch (kind) {                                            \
    case KFR0: { constexpr int KK = KFR0; KERNEL_CALL; note_launch(1); } break; \
    case KFR1: { constexpr int KK = KFR1; KERNEL_CALL; note_launch(1); } break; \
    case KFR2: { constexpr int KK = KFR2; KERNEL_CALL; note_launch(1); } break; \
    case KSYM: { constexpr int KK = KSYM; KERNEL_CALL; note_launch(1); } break; \
    case KCQ: { constexpr int KK = KCQ; KERNEL_CALL; note_launch(1); } break;   \
    default: return MGGLAM_ERR_ARG;                          \
  }

int launch_smooth64(const ModelDev& m, int n, double h, double* u, const double* rho, const double* S,
                    int sweeps, cudaStream_t st) {
  const dim3 g = grid3d(n / 2, n, n);
  for (int s = 0; s < sweeps; ++s)
    for (int parity = 0; parity < 2; ++parity) {
      MG_DISPATCH(m.kind, (k_smooth64<KK><<<g, k3dThreads, 0, st>>>(m, n, h, u, rho, S, parity)));
    }
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int launch_residual64(const ModelDev& m, int n, double h, const double* u, const double* rho,
                      const double* S, double* d, double* partials, double* out_sum, cudaStream_t st) {
  const long long n3 = (long long)n * n * n;
  const int g = n * n < 2048 ? n * n : 2048;
  const int bt = n >= 256 ? 256 : (n <= 32 ? 32 : ((n + 31) / 32) * 32);
  MG_DISPATCH(m.kind, (k_residual64<KK><<<g, bt, 0, st>>>(m, n, h, u, rho, S, d, partials)));
  k_finalize_sum<<<1, 1024, 0, st>>>(partials, g, out_sum);
  note_launch(1);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int launch_restrict64(int nf, const double* fine, double* coarse, cudaStream_t st) {
  const long long nc3 = (long long)(nf / 2) * (nf / 2) * (nf / 2);
  k_restrict64<<<grid3d(nf / 2, nf / 2, nf / 2), k3dThreads, 0, st>>>(nf, fine, coarse);
  note_launch(1);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int launch_prolong_correct64(const ModelDev& m, int nc, const double* uH, const double* RuH,
                             unsigned long long* guard, double* uf, cudaStream_t st) {
  const long long nf3 = 8LL * nc * nc * nc;
  const dim3 g = grid3d(2 * nc, 2 * nc, 2 * nc);
  if (is_fr(m.kind)) k_prolong_correct64<true><<<g, k3dThreads, 0, st>>>(nc, uH, RuH, uf, guard);
  else k_prolong_correct64<false><<<g, k3dThreads, 0, st>>>(nc, uH, RuH, uf, guard);
  note_launch(1);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int launch_coarse64(const ModelDev& m, int n, double h, double* u, const double* rho, const double* S,
                    int sweeps, cudaStream_t st) {
  if ((long long)n * n * n > 4096) return launch_smooth64(m, n, h, u, rho, S, sweeps, st);
  MG_DISPATCH(m.kind, (k_coarse64<KK><<<1, 512, 0, st>>>(m, n, h, u, rho, S, sweeps)));
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int launch_residual_restrict64(const ModelDev& m, int nf, double hf, const double* u, const double* rho,
                               const double* S, double* Ru, double* uH, double* Rd, cudaStream_t st) {
  const long long nc3 = (long long)(nf / 2) * (nf / 2) * (nf / 2);
  const dim3 g = grid3d(nf / 2, nf / 2, nf / 2);
  MG_DISPATCH(m.kind, (k_residual_restrict64<KK><<<g, k3dThreads, 0, st>>>(m, nf, hf, u, rho, S, Ru, uH, Rd)));
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int launch_fas_source64(const ModelDev& m, int nc, double hc, const double* Ru, const double* rho, double* S,
                        cudaStream_t st) {
  const long long n3 = (long long)nc * nc * nc;
  const int g = grid_for(n3, kThreads, 1 << 20);
  MG_DISPATCH(m.kind, (k_fas_source64<KK><<<grid3d(nc, nc, nc), k3dThreads, 0, st>>>(m, nc, hc, Ru, rho, S)));
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int launch_density_mean(const float* rho32, size_t n3, double* partials, double* out_sum, cudaStream_t st) {
  const int g = stream_grid((long long)n3);
  k_sum_f32<<<g, kThreads, 0, st>>>(rho32, (long long)n3, partials);
  k_finalize_sum<<<1, 1024, 0, st>>>(partials, g, out_sum);
  note_launch(2);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int launch_density_to64(const float* rho32, size_t n3, const double* sum, double* rho64, cudaStream_t st) {
  k_density_to64<<<stream_grid((long long)n3), kThreads, 0, st>>>(rho32, (long long)n3, sum, rho64);
  note_launch(1);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int launch_src_sumsq(const ModelDev& m, const double* rho64, size_t n3, double* partials, double* out,
                     cudaStream_t st) {
  const int g = grid_for((long long)n3);
  MG_DISPATCH(m.kind, (k_src_sumsq<KK><<<g, kThreads, 0, st>>>(m, rho64, (long long)n3, partials)));
  k_finalize_sum<<<1, 1024, 0, st>>>(partials, g, out);
  note_launch(1);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int launch_init_background(const ModelDev& m, double* field, size_t n3, cudaStream_t st) {
  k_init_background<<<stream_grid((long long)n3), kThreads, 0, st>>>(field, (long long)n3, m.ubar);
  k_init_background_first<<<1, 1, 0, st>>>(field, m.ubar);
  note_launch(2);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

// ---------------------------------------------------------------------------
// FP64 solver
// ---------------------------------------------------------------------------

// One multigrid cycle from level l (Sec. 3.2.1): mode 0 V, 1 F, 2 W.
static int vcycle64(const ModelDev& m, Workspace* ws, int l, const mgglam_params* prm, cudaStream_t st,
                    int mode = -1) {
  if (mode < 0) mode = prm->cycle;
  Level& L = ws->lev[l];
  int rc;
  if (l == ws->nlev - 1) return launch_coarse64(m, L.n, L.h, L.u, L.rho, L.S, prm->coarse_sweeps, st);
  if (l == 0) prof_begin(PC_SMOOTH64_FINE, st, 24.0 * L.n3 * prm->nu1);
  if ((rc = launch_smooth64(m, L.n, L.h, L.u, L.rho, L.S, prm->nu1, st))) return rc;
  if (l == 0) prof_end(st);
  Level& C = ws->lev[l + 1];
  // Ru -> C.Ru, u^H = Ru -> C.u, R d -> C.S (then C.S <- N^H(Ru) - R d)
  if (l == 0) prof_begin(PC_RESTRICT64_FINE, st, (16.0 + 3.0) * L.n3);
  if ((rc = launch_residual_restrict64(m, L.n, L.h, L.u, L.rho, L.S, C.Ru, C.u, C.S, st))) return rc;
  if (l == 0) { prof_end(st); prof_begin(PC_COARSE_LEVELS, st, 0.0); }
  if ((rc = launch_fas_source64(m, C.n, C.h, C.Ru, C.rho, C.S, st))) return rc;
  if ((rc = vcycle64(m, ws, l + 1, prm, st, mode))) return rc;
  if (mode != 0 && (rc = vcycle64(m, ws, l + 1, prm, st, mode == 2 ? 2 : 0))) return rc;
  if (l == 0) { prof_end(st); prof_begin(PC_PROLONG64_FINE, st, (16.0 + 2.0) * L.n3); }
  if ((rc = launch_prolong_correct64(m, C.n, C.u, C.Ru, guard_of(ws), L.u, st))) return rc;
  if (l == 0) { prof_end(st); prof_begin(PC_SMOOTH64_FINE, st, 24.0 * L.n3 * prm->nu2); }
  rc = launch_smooth64(m, L.n, L.h, L.u, L.rho, L.S, prm->nu2, st);
  if (l == 0) prof_end(st);
  return rc;
}

// Full-multigrid start (prm->fmg): every level poses N^H(u^H) = 0 on its restricted
// density; the coarsest level relaxes from the background value, and each finer
// level starts from the plain prolongation of the coarser result (the correction
// kernel applied to a zero field with a zero coarse reference) and takes one
// cycle.  Level 0 (the caller's field) holds the result.
static int fmg_start64(const ModelDev& m, Workspace* ws, const mgglam_params* prm, cudaStream_t st) {
  const int L = ws->nlev;
  Level& C = ws->lev[L - 1];
  int rc;
  if ((rc = launch_init_background(m, C.u, C.n3, st))) return rc;
  if (L > 1) MG_CUDA_TRY(cudaMemsetAsync(C.S, 0, C.n3 * sizeof(double), st));
  if ((rc = launch_coarse64(m, C.n, C.h, C.u, C.rho, L > 1 ? C.S : nullptr, prm->coarse_sweeps, st))) return rc;
  for (int l = L - 2; l >= 0; --l) {
    Level& F = ws->lev[l];
    Level& H = ws->lev[l + 1];
    MG_CUDA_TRY(cudaMemsetAsync(F.u, 0, F.n3 * sizeof(double), st));
    MG_CUDA_TRY(cudaMemsetAsync(H.Ru, 0, H.n3 * sizeof(double), st));
    if ((rc = launch_prolong_correct64(m, H.n, H.u, H.Ru, nullptr, F.u, st))) return rc;
    if (l > 0) MG_CUDA_TRY(cudaMemsetAsync(F.S, 0, F.n3 * sizeof(double), st));
    if ((rc = vcycle64(m, ws, l, prm, st, 0))) return rc;
  }
  return MGGLAM_OK;
}

int solve_fp64(const mgglam_params* prm, double a, const float* rho, int N, double* field, double tol,
               mgglam_stats* stats, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  ModelDev m;
  int rc = make_model(prm, a, N, &m);
  if (rc) return rc;
  Workspace* ws = nullptr;
  if ((rc = get_workspace(N, MGGLAM_FP64, prm->levels, &ws))) return rc;
  Level& F = ws->lev[0];
  F.u = field;
  const size_t n3 = F.n3;
  // density: FP64 mean (a2), normalised FP64 copy, restricted down the levels
  if ((rc = launch_density_mean(rho, n3, ws->partials, ws->scalars + SC_MEAN, st))) return rc;
  if ((rc = launch_density_to64(rho, n3, ws->scalars + SC_MEAN, F.rho, st))) return rc;
  for (int l = 1; l < ws->nlev; ++l)
    if ((rc = launch_restrict64(ws->lev[l - 1].n, ws->lev[l - 1].rho, ws->lev[l].rho, st))) return rc;
  if ((rc = launch_init_background(m, field, n3, st))) return rc;
  MG_CUDA_TRY(cudaMemsetAsync(guard_of(ws), 0, sizeof(unsigned long long), st));
  if ((rc = launch_src_sumsq(m, F.rho, n3, ws->partials, ws->scalars + SC_SRC, st))) return rc;
  if ((rc = launch_residual64(m, F.n, F.h, field, F.rho, nullptr, nullptr, ws->partials,
                              ws->scalars + SC_SUMSQ, st)))
    return rc;
  MG_CUDA_TRY(cudaMemcpyAsync(ws->h_scalars, ws->scalars, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
  MG_CUDA_TRY(cudaStreamSynchronize(st));
  const double src = sqrt(ws->h_scalars[SC_SRC] / (double)n3);
  const double snorm = source_norm(m, src);
  double eps = sqrt(ws->h_scalars[SC_SUMSQ] / (double)n3) / snorm;
  mgglam_stats local;
  mgglam_stats* S = stats ? stats : &local;
  memset(S, 0, sizeof(*S));
  S->resid0 = eps;
  S->resid_hist[0] = eps;
  int cyc = 0, nh = 1;
  const int every = prm->check_every > 0 ? prm->check_every : 1;
  int status = MGGLAM_OK;
  while (!(eps <= tol) && cyc < prm->max_cycles) {
    if (!isfinite(eps)) { status = MGGLAM_ERR_NONFINITE; break; }
    if (prm->fmg && m.kind != KCQ && cyc == 0) {
      if ((rc = fmg_start64(m, ws, prm, st))) return rc;
    } else if ((rc = vcycle64(m, ws, 0, prm, st))) {
      return rc;
    }
    ++cyc;
    if (cyc % every == 0 || cyc == prm->max_cycles) {
      if ((rc = launch_residual64(m, F.n, F.h, field, F.rho, nullptr, nullptr, ws->partials,
                                  ws->scalars + SC_SUMSQ, st)))
        return rc;
      MG_CUDA_TRY(cudaMemcpyAsync(ws->h_scalars + SC_SUMSQ, ws->scalars + SC_SUMSQ, sizeof(double),
                                  cudaMemcpyDeviceToHost, st));
      MG_CUDA_TRY(cudaStreamSynchronize(st));
      eps = sqrt(ws->h_scalars[SC_SUMSQ] / (double)n3) / snorm;
      if (nh < 64) S->resid_hist[nh++] = eps;
    }
  }
  if (status == MGGLAM_OK && !isfinite(eps)) status = MGGLAM_ERR_NONFINITE;
  MG_CUDA_TRY(cudaMemcpyAsync(ws->h_scalars + SC_GUARD, guard_of(ws), sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, st));
  MG_CUDA_TRY(cudaStreamSynchronize(st));
  S->guarded = (long long)*reinterpret_cast<const unsigned long long*>(ws->h_scalars + SC_GUARD);
  S->cycles = cyc;
  S->resid = eps;
  S->converged = eps <= tol;
  S->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (status == MGGLAM_OK && !S->converged) status = MGGLAM_ERR_NOT_CONVERGED;
  return status;
}

}  // namespace mg
