// mixed_common.cuh -- device helpers shared by the single and batched mixed-precision
// solvers: FP32 level constants, the correction operator M(e), neighbour sums,
// the FP64 source term and the tiled FP64 fine-level residual.
#pragma once
#include <math.h>
#include <string.h>

#include "mg_common.cuh"
#include "sweep32.cuh"

namespace mg {

static inline LevelF make_levelf(const ModelDev& m, double h) {
  LevelF f;
  memset(&f, 0, sizeof(f));
  f.c2_h2 = (float)(m.c2 / (h * h));
  f.ih2 = (float)(1.0 / (h * h));
  if (is_fr(m.kind)) {
    const double al = h * h / (6.0 * m.c2);
    const int np1 = m.kind + 1;  // n + 1
    const double sc = pow(al * m.K, 1.0 / (double)(np1 + 1));
    f.al = (float)al;
    f.K = (float)m.K;
    f.alK = (float)(al * m.K);
    f.fr_s = (float)sc;
    f.fr_is1 = (float)pow(sc, -(double)np1);
  } else if (m.kind == KSYM) {
    f.al = (float)(m.c2 * m.xi2_a2 / (h * h));
    f.msym = (float)m.msym;
    f.rat3 = (float)m.rat3;
  } else {
    f.cq_src = (float)m.cq_src;
    f.cq_pot = (float)m.cq_pot;
    f.alpha = (float)m.alpha;
    f.phibar = (float)m.phibar;
    f.inv_c2 = (float)(1.0 / m.c2);
    f.beta = (float)m.beta;
    f.keep_exp = m.keep_exp;
  }
  return f;
}

// M(e) at one cell, given the neighbours' nbq sum (accurate operations: this
// defines the residual and the coarse sources, not a relaxation).
template <int K>
__device__ __forceinline__ float local_M(const LevelF& f, float u, float e, float rho, float Lnb) {
  if constexpr (is_fr(K)) {
    return -f.c2_h2 * (Lnb - 6.f * dw<K>(u, e)) + f.K * e / (u * (u + e));
  } else if constexpr (K == KSYM) {
    return f.c2_h2 * (Lnb - 6.f * e) - f.msym * ((rho * f.rat3 - 1.f) * e + e * (3.f * u * u + 3.f * u * e + e * e));
  } else {
    const float x0 = f.phibar + u * f.inv_c2;
    const float dpow = powf(x0, -1.f - f.alpha) * expm1f((-1.f - f.alpha) * log1pf(e * f.inv_c2 / x0));
    float v = (Lnb - 6.f * e) * f.ih2 + f.cq_pot * dpow;
    if (f.keep_exp) v -= f.cq_src * rho * expf(f.beta * u * f.inv_c2) * expm1f(f.beta * e * f.inv_c2);
    return v;
  }
}

// nbq sum of the six neighbours of (i,j,k) read from global arrays.
template <int K>
__device__ __forceinline__ float nb_sum_g(const float* __restrict__ e, const float* __restrict__ ub, int n, int i,
                                          int j, int k) {
  const int ip = wrapi(i + 1, n), im = wrapi(i - 1, n);
  const int jp = wrapi(j + 1, n), jm = wrapi(j - 1, n);
  const int kp = wrapi(k + 1, n), km = wrapi(k - 1, n);
  const size_t c0 = cidx(n, ip, j, k), c1 = cidx(n, im, j, k), c2 = cidx(n, i, jp, k), c3 = cidx(n, i, jm, k),
               c4 = cidx(n, i, j, kp), c5 = cidx(n, i, j, km);
  if constexpr (is_fr(K)) {
    return dw<K>(ub[c0], e[c0]) + dw<K>(ub[c1], e[c1]) + dw<K>(ub[c2], e[c2]) + dw<K>(ub[c3], e[c3]) +
           dw<K>(ub[c4], e[c4]) + dw<K>(ub[c5], e[c5]);
  } else {
    return e[c0] + e[c1] + e[c2] + e[c3] + e[c4] + e[c5];
  }
}

// 1/x in FP64 by one Newton-Raphson refinement y1 = y0 (2 - x y0) of a
// single-precision reciprocal y0: the relative error of y0 (below 2^-22) is
// squared, leaving about 2^-44 ~ 6e-14, far below what the residual needs.
__device__ __forceinline__ double rcp_nr(double x, float xf) {
  const double y = (double)__frcp_rn(xf);
  const double t = fma(-x, y, 1.0);
  return fma(y, t, y);
}

// src64 = the part of N that does not depend on u, in FP64:
// f(R): Om (rho/mean - 1)/a + Rbar a^2/3; symmetron: rho/mean (the density
// itself, used in the u-dependent term); CQ: -3 beta Om e^{beta phibar}/a (rho/mean - 1).
template <int K>
__global__ void k_src64(ModelDev m, const float* __restrict__ rho32, long long n3, const double* __restrict__ rho_sum,
                        double* __restrict__ src) {
  const double inv_mean = (double)n3 / *rho_sum;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    const double r = (double)rho32[t] * inv_mean;
    if constexpr (is_fr(K)) src[t] = m.om_a * (r - 1.0) + m.K0;
    else if constexpr (K == KSYM) src[t] = r;
    else src[t] = r;
  }
}

// r = N(u64) on the fine level, z-marching tiles (each cell's transformed value
// formed once): writes ub = float(u64), tau = float(-r), and per-block partial
// sums of r^2 (accumulated from the float tau).
// Body for one CTA: tile index 'tile' over (j,k) tiles, chunk index 'cb' along i;
// returns the CTA's sum of tau^2 (valid in thread 0).
template <int K, int TJ, int TK>
__device__ __forceinline__ double outer_residual_tile(const ModelDev& m, int n, int chunk, const double* __restrict__ u,
                                                      const double* __restrict__ src, float* __restrict__ ub,
                                                      float* __restrict__ tau, int tile, int cb) {
  constexpr int PJ = TJ + 2, PK = TK + 2, PS = PJ * PK;
  __shared__ double s_w[3][PS];
  const int tiles_k = n / TK;
  const int k0 = (tile % tiles_k) * TK;
  const int j0 = (tile / tiles_k) * TJ;
  const int i0 = cb * chunk;
  const int i1 = min(i0 + chunk, n);
  const int t = threadIdx.x;
  const int tj = t / TK, tk = t - tj * TK;
  const int jg = j0 + tj, kg = k0 + tk;
  const int cc = (tj + 1) * PK + tk + 1;
  float acc = 0.f;
  auto load = [&](int p) {
    const int ig = p < 0 ? p + n : (p >= n ? p - n : p);
    const int slot = (p + 3) % 3;
    const size_t base = (size_t)ig * n * n;
    for (int c = t; c < PS; c += TJ * TK) {
      const int jj = c / PK, kk = c - jj * PK;
      const size_t g = base + (size_t)wrapi(j0 + jj - 1, n) * n + wrapi(k0 + kk - 1, n);
      s_w[slot][c] = fr_or_id<K>(u[g]);
    }
  };
  load(i0 - 1);
  load(i0);
  for (int i = i0; i < i1; ++i) {
    load(i + 1);
    __syncthreads();
    const int sl = (i + 3) % 3, sm = (i + 2) % 3, sp = (i + 4) % 3;
    const size_t g = ((size_t)i * n + jg) * n + kg;
    const double uc = u[g];
    const double L = s_w[sm][cc] + s_w[sp][cc] + s_w[sl][cc - PK] + s_w[sl][cc + PK] + s_w[sl][cc - 1] +
                     s_w[sl][cc + 1];
    const float uf = (float)uc;
    double v;
    if constexpr (is_fr(K)) {
      v = fma(-m.c2, L - 6.0 * s_w[sl][cc], src[g]) - m.K * rcp_nr(uc, uf);
    } else if constexpr (K == KSYM) {
      v = m.c2 * (L - 6.0 * uc) - m.msym * ((src[g] * m.rat3 - 1.0) * uc + uc * uc * uc);
    } else {
      const double E = m.keep_exp ? exp(m.beta * uc / m.c2) : 1.0;
      const double x = m.phibar + uc / m.c2;
      v = (L - 6.0 * uc) - m.cq_src * (E * src[g] - 1.0) + m.cq_pot * (pow(x, -1.0 - m.alpha) - m.pot0);
    }
    const float tv = (float)(-v);
    ub[g] = uf;
    tau[g] = tv;
    acc += tv * tv;
    __syncthreads();
  }
  return block_sum((double)acc);
}

template <int K, int TJ, int TK>
__global__ void __launch_bounds__(TJ* TK) k_outer_residual(ModelDev m, int n, int chunk, const double* __restrict__ u,
                                                           const double* __restrict__ src, float* __restrict__ ub,
                                                           float* __restrict__ tau, double* __restrict__ partials) {
  const double a = outer_residual_tile<K, TJ, TK>(m, n, chunk, u, src, ub, tau, blockIdx.x, blockIdx.y);
  if (threadIdx.x == 0) partials[blockIdx.x + blockIdx.y * gridDim.x] = a;
}


// ---- small whole-mesh kernels shared by the single and batched solvers ----

// rho32 normalised to mean 1 (FP64 mean), for the inner levels.
static __global__ void k_density_norm32(const float* __restrict__ rho, long long n3, const double* __restrict__ sum,
                                 float* __restrict__ out) {
  const double inv_mean = (double)n3 / *sum;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = (float)((double)rho[t] * inv_mean);
}

static __global__ void __launch_bounds__(128) k_restrict32(int nf, const float* __restrict__ fine, float* __restrict__ coarse) {
  const int nc = nf >> 1;
  const int I = blockIdx.z, J = blockIdx.y;
  const int Kc = blockIdx.x * blockDim.x + threadIdx.x;
  if (Kc >= nc) return;
  float s = 0.f;
  for (int di = 0; di < 2; ++di)
    for (int dj = 0; dj < 2; ++dj)
      for (int dk = 0; dk < 2; ++dk) s += fine[cidx(nf, 2 * I + di, 2 * J + dj, 2 * Kc + dk)];
  coarse[cidx(nc, I, J, Kc)] = 0.125f * s;
}

// Source scale from the FP32 input density (sum of squares of the linear source).
template <int K>
static __global__ void k_src_sumsq32(ModelDev m, const float* __restrict__ rho32, long long n3,
                              const double* __restrict__ rho_sum, double* __restrict__ partials) {
  const double inv_mean = (double)n3 / *rho_sum;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    const double delta = (double)rho32[t] * inv_mean - 1.0;
    double s;
    if constexpr (is_fr(K)) s = m.om_a * delta;
    else if constexpr (K == KSYM) s = m.msym * m.rat3 * delta * m.ubar;
    else s = m.cq_src * delta;
    acc += s * s;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

static __global__ void k_finalize_sum32(const double* __restrict__ partials, int count, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partials[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}


}  // namespace mg
