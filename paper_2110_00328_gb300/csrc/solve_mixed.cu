// solve_mixed.cu -- the FP32/FP64 mixed-precision solver.
//
// Outer loop (FP64, fine level only): r = N(u64) (Eq. residual_d), the
// convergence test, and u64 += e after each inner solve.
//
// Inner loop (FP32): FAS V-cycles (Sec. 3.2.1) for the correction e = U - u,
// where u = float(u64) is held fixed as a base field and U is the total field.
// Each level solves M(e) = S with M(e) = N(U) - N(u) evaluated in a form
// without cancellation (f(R): Delta w = (u+e)^{n+1} - u^{n+1} = e * sum_j ...;
// 1/(u+e) - 1/u = -e/(u(u+e)); symmetron: (u+e)^3 - u^3 = e(3u^2 + 3ue + e^2);
// CQ: powers and exponentials via expm1/log1p).  On the finest level
// S = -N(u64) (from the FP64 residual), on coarse levels the FAS source
// S^H = M^H(R e) - R d with base R u.  In exact arithmetic an inner V-cycle
// started from e = 0 produces exactly the iterate of one FAS V-cycle on the
// total field started from u64 (restriction and prolongation are linear, and
// the nonlinear Gauss-Seidel local solve of M(e)_i = S_i is the local solve of
// N(U)_i = 0); single precision then only limits how much each outer step
// reduces the FP64 residual.
//
// Local solves: f(R) and the symmetron use the closed-form root of the total
// field's local polynomial (Secs. 3.2.4-3.2.5, stable forms in mg_model.cuh),
// followed by one Newton step on the cancellation-free correction equation,
// which restores full relative precision of e; CQ takes one Newton step
// (Eq. relaxation_iteration).
#include <math.h>
#include <string.h>

#include <chrono>

#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

// FP32 constants of one level.
struct LevelF {
  float c2_h2;   // c~^2 / h^2
  float al;      // f(R): h^2 / (6 c~^2); symmetron: g = c~^2 xi^2 / (h^2 a^2)
  float K;       // f(R): Rbar a^2/3 * ubar
  float msym;    // symmetron a^2/(2 xi^2)
  float rat3;    // symmetron (a_star/a)^3
  float ih2;     // 1/h^2
  float fr_s;    // f(R): s = (al K)^{1/(n+2)}, the root's natural scale
  float fr_is1;  // f(R): 1 / s^{n+1}
  float cq_src, cq_pot, alpha, phibar, inv_c2, beta;
  int keep_exp;
};

static LevelF make_levelf(const ModelDev& m, double h) {
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

// Delta w = (u+e)^{n+1} - u^{n+1}, factored so that small e loses nothing.
template <int K>
__device__ __forceinline__ float dw(float u, float e) {
  if constexpr (K == KFR0) return e;
  else if constexpr (K == KFR1) return e * (2.f * u + e);
  else return e * (3.f * u * u + 3.f * u * e + e * e);
}

// The neighbour sum of the correction field that enters M: f(R) sum of Delta w,
// otherwise sum of e.
template <int K>
__device__ __forceinline__ float nb_sum_e(const float* __restrict__ e, const float* __restrict__ ub, int n, int i,
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

// M(e) at one cell, given the neighbour sum from nb_sum_e.
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

// Nonlinear Gauss-Seidel update of the correction at one cell.
template <int K>
__device__ __forceinline__ float local_update_e(const LevelF& f, float u, float e, float rho, float s, float Lnb) {
  if constexpr (is_fr(K)) {
    // total-field polynomial U^{n+2} + p U + q = 0 with p = -u^{n+1} + al K/u - (Lnb/6 + al s), q = -al K
    const float alK = f.al * f.K;
    const float B = Lnb * (1.f / 6.f) + f.al * s;
    const float p = -fr_w<K>(u) + alK / u - B;
    // scaled: U = s y with y^{n+2} + (p/s^{n+1}) y - 1 = 0 keeps single precision in range
    const float U = f.fr_s * fr_root<K>(p * f.fr_is1, -1.f);
    float x = U - u;
    // one Newton step on G(e) = Delta w(e) + al K e/(u(u+e)) - B
    const float Ue = u + x;
    const float G = dw<K>(u, x) + alK * x / (u * Ue) - B;
    float dG = alK / (Ue * Ue);
    if constexpr (K == KFR0) dG += 1.f;
    else if constexpr (K == KFR1) dG += 2.f * Ue;
    else dG += 3.f * Ue * Ue;
    const float xn = x - G / dG;
    return (u + xn > 0.f) ? xn : x;
  } else if constexpr (K == KSYM) {
    // total-field cubic U^3 + p U + q = 0, p = rho a*^3/a^3 - 1 + 12 g, q = -(p u + u^3 + 2 g Lnb - s/msym)
    const float p = rho * f.rat3 - 1.f + 12.f * f.al;
    const float B = 2.f * f.al * Lnb - s / f.msym;
    const float q = -(p * u + u * u * u + B);
    const float U = sym_root(p, q, u + e);
    float x = U - u;
    // Newton step on G(e) = p e + e(3u^2 + 3ue + e^2) - B
    const float G = p * x + x * (3.f * u * u + 3.f * u * x + x * x) - B;
    const float Ue = u + x;
    const float dG = p + 3.f * Ue * Ue;
    return dG != 0.f ? x - G / dG : x;
  } else {
    // Newton-Gauss-Seidel step on M(e) - s
    const float r = local_M<K>(f, u, e, rho, Lnb) - s;
    const float x = f.phibar + (u + e) * f.inv_c2;
    float dr = -6.f * f.ih2 - f.cq_pot * (1.f + f.alpha) * powf(x, -2.f - f.alpha) * f.inv_c2;
    if (f.keep_exp) dr -= f.cq_src * rho * f.beta * f.inv_c2 * expf(f.beta * (u + e) * f.inv_c2);
    return e - r / dr;
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_smooth32(LevelF f, int n, float* __restrict__ e,
                                                       const float* __restrict__ ub, const float* __restrict__ rho,
                                                       const float* __restrict__ S, int parity) {
  const int nh = n >> 1;
  const long long total = (long long)n * n * nh;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(t % nh);
    const long long r = t / nh;
    const int j = (int)(r % n), i = (int)(r / n);
    const int k = 2 * kk + ((i + j + parity) & 1);
    const size_t c = cidx(n, i, j, k);
    const float Lnb = nb_sum_e<K>(e, ub, n, i, j, k);
    e[c] = local_update_e<K>(f, ub[c], e[c], rho ? rho[c] : 1.f, S[c], Lnb);
  }
}

// For each coarse cell: d = M(e) - S at the 8 children, averaged into Rd (stored
// in SH); the children's e averaged into Re and eH; ub averaged into ubH.
template <int K>
__global__ void __launch_bounds__(kThreads) k_residual_restrict32(LevelF f, int nf, const float* __restrict__ e,
                                                                  const float* __restrict__ ub,
                                                                  const float* __restrict__ rho,
                                                                  const float* __restrict__ S,
                                                                  float* __restrict__ Re, float* __restrict__ eH,
                                                                  float* __restrict__ ubH, float* __restrict__ SH) {
  const int nc = nf >> 1;
  const long long total = (long long)nc * nc * nc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int K0 = (int)(t % nc);
    const long long r = t / nc;
    const int J = (int)(r % nc), I = (int)(r / nc);
    float se = 0.f, su = 0.f, sd = 0.f;
    for (int di = 0; di < 2; ++di)
      for (int dj = 0; dj < 2; ++dj)
        for (int dk = 0; dk < 2; ++dk) {
          const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K0 + dk;
          const size_t c = cidx(nf, i, j, k);
          const float ec = e[c], uc = ub[c];
          se += ec;
          su += uc;
          sd += local_M<K>(f, uc, ec, rho ? rho[c] : 1.f, nb_sum_e<K>(e, ub, nf, i, j, k)) - S[c];
        }
    Re[t] = 0.125f * se;
    eH[t] = 0.125f * se;
    ubH[t] = 0.125f * su;
    SH[t] = 0.125f * sd;
  }
}

// In place: S <- M^H(Re) - S (S holds R d on entry).
template <int K>
__global__ void __launch_bounds__(kThreads) k_fas_source32(LevelF f, int n, const float* __restrict__ Re,
                                                           const float* __restrict__ ub,
                                                           const float* __restrict__ rho, float* __restrict__ S) {
  const long long total = (long long)n * n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t % n);
    const long long r = t / n;
    const int j = (int)(r % n), i = (int)(r / n);
    S[t] = local_M<K>(f, ub[t], Re[t], rho ? rho[t] : 1.f, nb_sum_e<K>(Re, ub, n, i, j, k)) - S[t];
  }
}

// e^h += P(e^H - R e^h); f(R): if u + e would not be positive, e <- (e_old - u)/2
// (the total field halves, as in the FP64 path).
template <bool FR>
__global__ void __launch_bounds__(kThreads) k_prolong_correct32(int nc, const float* __restrict__ eH,
                                                                const float* __restrict__ Re,
                                                                const float* __restrict__ ub,
                                                                float* __restrict__ ef) {
  const int nf = nc << 1;
  const long long total = (long long)nf * nf * nf;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t % nf);
    const long long r = t / nf;
    const int j = (int)(r % nf), i = (int)(r / nf);
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const int I2 = wrapi(I + ((i & 1) ? 1 : -1), nc);
    const int J2 = wrapi(J + ((j & 1) ? 1 : -1), nc);
    const int K2 = wrapi(K + ((k & 1) ? 1 : -1), nc);
#define EH(a, b, c) (eH[cidx(nc, a, b, c)] - Re[cidx(nc, a, b, c)])
    const float corr = (27.f * EH(I, J, K) + 9.f * (EH(I2, J, K) + EH(I, J2, K) + EH(I, J, K2)) +
                        3.f * (EH(I2, J2, K) + EH(I2, J, K2) + EH(I, J2, K2)) + EH(I2, J2, K2)) *
                       (1.f / 64.f);
#undef EH
    const float old = ef[t];
    float v = old + corr;
    if (FR && !(ub[t] + v > 0.f)) v = 0.5f * (old - ub[t]);
    ef[t] = v;
  }
}

template <int K>
__global__ void __launch_bounds__(512) k_coarse32(LevelF f, int n, float* __restrict__ e, const float* __restrict__ ub,
                                                  const float* __restrict__ rho, const float* __restrict__ S,
                                                  int sweeps) {
  const int n3 = n * n * n;
  for (int s = 0; s < sweeps; ++s)
    for (int parity = 0; parity < 2; ++parity) {
      for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int k = t % n, j = (t / n) % n, i = t / (n * n);
        if (((i + j + k) & 1) != parity) continue;
        const float Lnb = nb_sum_e<K>(e, ub, n, i, j, k);
        e[t] = local_update_e<K>(f, ub[t], e[t], rho ? rho[t] : 1.f, S[t], Lnb);
      }
      __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP64 outer-loop kernels (fine level)
// ---------------------------------------------------------------------------

// 1/x in FP64 by Newton-Raphson refinement of a single-precision reciprocal:
// y1 = y0 (2 - x y0) squares the relative error of y0 (about 2^-24), giving
// about 2^-47; a second step reaches double rounding level.  Used where the
// residual needs K/u to ~1e-14 relative without a full-precision division.
__device__ __forceinline__ double rcp_nr(double x) {
  double y = (double)(1.0f / (float)x);
  double t = fma(-x, y, 1.0);
  y = fma(y, t, y);
  t = fma(-x, y, 1.0);
  return fma(y, t, y);
}

// r = N(u64) on the fine level (rho normalised by its FP64 mean): writes
// ub = float(u64), tau = float(-r), and per-block partial sums of r^2.
template <int K>
__global__ void __launch_bounds__(kThreads) k_outer_residual(ModelDev m, int n, const double* __restrict__ u,
                                                             const float* __restrict__ rho32,
                                                             const double* __restrict__ rho_sum, float* __restrict__ ub,
                                                             float* __restrict__ tau, double* __restrict__ partials) {
  const long long total = (long long)n * n * n;
  const double inv_mean = (double)total / *rho_sum;
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t % n);
    const long long r = t / n;
    const int j = (int)(r % n), i = (int)(r / n);
    const int ip = wrapi(i + 1, n), im = wrapi(i - 1, n);
    const int jp = wrapi(j + 1, n), jm = wrapi(j - 1, n);
    const int kp = wrapi(k + 1, n), km = wrapi(k - 1, n);
    const double uc = u[t];
    const double Lnb = fr_or_id<K>(u[cidx(n, ip, j, k)]) + fr_or_id<K>(u[cidx(n, im, j, k)]) +
                       fr_or_id<K>(u[cidx(n, i, jp, k)]) + fr_or_id<K>(u[cidx(n, i, jm, k)]) +
                       fr_or_id<K>(u[cidx(n, i, j, kp)]) + fr_or_id<K>(u[cidx(n, i, j, km)]);
    const double rhoc = (double)rho32[t] * inv_mean;
    double v;
    if constexpr (is_fr(K)) {
      v = -m.c2 * (Lnb - 6.0 * fr_w<K>(uc)) + m.om_a * (rhoc - 1.0) + m.K0 - m.K * rcp_nr(uc);
    } else if constexpr (K == KSYM) {
      v = m.c2 * (Lnb - 6.0 * uc) - m.msym * ((rhoc * m.rat3 - 1.0) * uc + uc * uc * uc);
    } else {
      const double E = m.keep_exp ? exp(m.beta * uc / m.c2) : 1.0;
      const double x = m.phibar + uc / m.c2;
      v = (Lnb - 6.0 * uc) - m.cq_src * (E * rhoc - 1.0) + m.cq_pot * (pow(x, -1.0 - m.alpha) - m.pot0);
    }
    ub[t] = (float)uc;
    tau[t] = (float)(-v);
    acc += v * v;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// u64 += e; e <- 0 (ready for the next inner solve).
__global__ void k_apply_correction(double* __restrict__ u, float* __restrict__ e, long long n3) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    u[t] += (double)e[t];
    e[t] = 0.f;
  }
}

// rho32 normalised to mean 1 (FP64 mean), for the inner levels.
__global__ void k_density_norm32(const float* __restrict__ rho, long long n3, const double* __restrict__ sum,
                                 float* __restrict__ out) {
  const double inv_mean = (double)n3 / *sum;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = (float)((double)rho[t] * inv_mean);
}

__global__ void k_restrict32(int nf, const float* __restrict__ fine, float* __restrict__ coarse) {
  const int nc = nf >> 1;
  const long long total = (long long)nc * nc * nc;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int K = (int)(t % nc);
    const long long r = t / nc;
    const int J = (int)(r % nc), I = (int)(r / nc);
    float s = 0.f;
    for (int di = 0; di < 2; ++di)
      for (int dj = 0; dj < 2; ++dj)
        for (int dk = 0; dk < 2; ++dk) s += fine[cidx(nf, 2 * I + di, 2 * J + dj, 2 * K + dk)];
    coarse[t] = 0.125f * s;
  }
}

// Source scale from the FP32 input density (sum of squares of the linear source).
template <int K>
__global__ void k_src_sumsq32(ModelDev m, const float* __restrict__ rho32, long long n3,
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

__global__ void k_finalize_sum32(const double* __restrict__ partials, int count, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partials[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------

#define MG_DISPATCH32(kind, CALL)                                  \
  switch (kind) {                                                  \
    case KFR0: { constexpr int KK = KFR0; CALL; note_launch(1); } break; \
    case KFR1: { constexpr int KK = KFR1; CALL; note_launch(1); } break; \
    case KFR2: { constexpr int KK = KFR2; CALL; note_launch(1); } break; \
    case KSYM: { constexpr int KK = KSYM; CALL; note_launch(1); } break; \
    case KCQ: { constexpr int KK = KCQ; CALL; note_launch(1); } break;   \
    default: return MGGLAM_ERR_ARG;                                \
  }

struct MixedCtx {
  ModelDev m;
  LevelF lf[kMaxLevels];
  Workspace* ws;
  const mgglam_params* prm;
  bool need_rho;
};

static int smooth32(const MixedCtx& C, int l, int sweeps, cudaStream_t st) {
  Level& L = C.ws->lev[l];
  const float* rho = C.need_rho ? L.rho32 : nullptr;
  const long long half = (long long)L.n * L.n * (L.n / 2);
  const int g = grid_for(half, kThreads, 1 << 20);
  for (int s = 0; s < sweeps; ++s)
    for (int parity = 0; parity < 2; ++parity)
      MG_DISPATCH32(C.m.kind, (k_smooth32<KK><<<g, kThreads, 0, st>>>(C.lf[l], L.n, L.e, L.ub, rho, L.S32, parity)));
  return MGGLAM_OK;
}

static int vcycle32(const MixedCtx& C, int l, cudaStream_t st) {
  Workspace* ws = C.ws;
  Level& L = ws->lev[l];
  const float* rho = C.need_rho ? L.rho32 : nullptr;
  int rc;
  if (l == ws->nlev - 1) {
    if ((long long)L.n3 > 4096) return smooth32(C, l, C.prm->coarse_sweeps, st);
    MG_DISPATCH32(C.m.kind, (k_coarse32<KK><<<1, 512, 0, st>>>(C.lf[l], L.n, L.e, L.ub, rho, L.S32,
                                                                 C.prm->coarse_sweeps)));
    return MGGLAM_OK;
  }
  if (l == 0) prof_begin(PC_SMOOTH32_FINE, st, 16.0 * L.n3 * C.prm->nu1);
  if ((rc = smooth32(C, l, C.prm->nu1, st))) return rc;
  if (l == 0) prof_end(st);
  Level& H = ws->lev[l + 1];
  const float* rhoH = C.need_rho ? H.rho32 : nullptr;
  const int gc = grid_for((long long)H.n3, kThreads, 1 << 20);
  if (l == 0) prof_begin(PC_RESTRICT32_FINE, st, 14.0 * L.n3);
  MG_DISPATCH32(C.m.kind, (k_residual_restrict32<KK><<<gc, kThreads, 0, st>>>(C.lf[l], L.n, L.e, L.ub, rho, L.S32,
                                                                               H.Re, H.e, H.ub, H.S32)));
  if (l == 0) { prof_end(st); prof_begin(PC_COARSE_LEVELS, st, 0.0); }
  MG_DISPATCH32(C.m.kind, (k_fas_source32<KK><<<gc, kThreads, 0, st>>>(C.lf[l + 1], H.n, H.Re, H.ub, rhoH, H.S32)));
  if ((rc = vcycle32(C, l + 1, st))) return rc;
  const int gf = grid_for((long long)L.n3, kThreads, 1 << 20);
  if (l == 0) { prof_end(st); prof_begin(PC_PROLONG32_FINE, st, 13.0 * L.n3); }
  if (is_fr(C.m.kind)) k_prolong_correct32<true><<<gf, kThreads, 0, st>>>(H.n, H.e, H.Re, L.ub, L.e);
  else k_prolong_correct32<false><<<gf, kThreads, 0, st>>>(H.n, H.e, H.Re, L.ub, L.e);
  note_launch(1);
  if (l == 0) { prof_end(st); prof_begin(PC_SMOOTH32_FINE, st, 16.0 * L.n3 * C.prm->nu2); }
  rc = smooth32(C, l, C.prm->nu2, st);
  if (l == 0) prof_end(st);
  return rc;
}

static int outer_residual(const MixedCtx& C, double* field, const float* rho_in, cudaStream_t st) {
  Workspace* ws = C.ws;
  Level& F = ws->lev[0];
  const int g = grid_for((long long)F.n3);
  prof_begin(PC_OUTER_RESID, st, 20.0 * F.n3);
  MG_DISPATCH32(C.m.kind, (k_outer_residual<KK><<<g, kThreads, 0, st>>>(C.m, F.n, field, rho_in,
                                                                          ws->scalars + SC_MEAN, F.ub, F.S32,
                                                                          ws->partials)));
  k_finalize_sum32<<<1, 1024, 0, st>>>(ws->partials, g, ws->scalars + SC_SUMSQ);
  note_launch(1);
  prof_end(st);
  return MGGLAM_OK;
}

int solve_mixed(const mgglam_params* prm, double a, const float* rho, int N, double* field, double tol,
                mgglam_stats* stats, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  MixedCtx C;
  int rc = make_model(prm, a, N, &C.m);
  if (rc) return rc;
  if ((rc = get_workspace(N, MGGLAM_MIXED, prm->levels, &C.ws))) return rc;
  C.prm = prm;
  C.need_rho = (C.m.kind == KSYM) || (C.m.kind == KCQ && C.m.keep_exp);
  Workspace* ws = C.ws;
  for (int l = 0; l < ws->nlev; ++l) C.lf[l] = make_levelf(C.m, ws->lev[l].h);
  Level& F = ws->lev[0];
  const long long n3 = (long long)F.n3;
  const int g = grid_for(n3);
  // FP64 density mean; FP32 normalised pyramid where the inner operator needs it
  if ((rc = launch_density_mean(rho, F.n3, ws->partials, ws->scalars + SC_MEAN, st))) return rc;
  if (C.need_rho) {
    k_density_norm32<<<grid_for(n3, kThreads, 1 << 20), kThreads, 0, st>>>(rho, n3, ws->scalars + SC_MEAN, F.rho32);
    note_launch(1);
    for (int l = 1; l < ws->nlev; ++l)
      k_restrict32<<<grid_for((long long)ws->lev[l].n3, kThreads, 1 << 20), kThreads, 0, st>>>(
          ws->lev[l - 1].n, ws->lev[l - 1].rho32, ws->lev[l].rho32);
    note_launch(ws->nlev - 1);
  }
  if ((rc = launch_init_background(C.m, field, F.n3, st))) return rc;
  MG_DISPATCH32(C.m.kind, (k_src_sumsq32<KK><<<g, kThreads, 0, st>>>(C.m, rho, n3, ws->scalars + SC_MEAN,
                                                                      ws->partials)));
  k_finalize_sum32<<<1, 1024, 0, st>>>(ws->partials, g, ws->scalars + SC_SRC);
  note_launch(1);
  MG_CUDA_TRY(cudaMemsetAsync(F.e, 0, F.n3 * sizeof(float), st));
  if ((rc = outer_residual(C, field, rho, st))) return rc;
  MG_CUDA_TRY(cudaMemcpyAsync(ws->h_scalars, ws->scalars, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
  MG_CUDA_TRY(cudaStreamSynchronize(st));
  MG_CUDA_TRY(cudaGetLastError());
  const double src = sqrt(ws->h_scalars[SC_SRC] / (double)n3);
  const double snorm = src > 0.0 ? src : 1.0;
  double eps = sqrt(ws->h_scalars[SC_SUMSQ] / (double)n3) / snorm;
  mgglam_stats local;
  mgglam_stats* S = stats ? stats : &local;
  memset(S, 0, sizeof(*S));
  S->resid0 = eps;
  S->resid_hist[0] = eps;
  int cyc = 0, outer = 0, nh = 1;
  const int inner = prm->inner_cycles > 0 ? prm->inner_cycles : 1;
  int status = MGGLAM_OK;
  while (!(eps <= tol) && cyc < prm->max_cycles) {
    if (!isfinite(eps)) { status = MGGLAM_ERR_NONFINITE; break; }
    for (int c = 0; c < inner && cyc < prm->max_cycles; ++c, ++cyc)
      if ((rc = vcycle32(C, 0, st))) return rc;
    prof_begin(PC_APPLY_CORR, st, 24.0 * n3);
    k_apply_correction<<<grid_for(n3, kThreads, 1 << 20), kThreads, 0, st>>>(field, F.e, n3);
    note_launch(1);
    prof_end(st);
    ++outer;
    if ((rc = outer_residual(C, field, rho, st))) return rc;
    MG_CUDA_TRY(cudaMemcpyAsync(ws->h_scalars + SC_SUMSQ, ws->scalars + SC_SUMSQ, sizeof(double),
                                cudaMemcpyDeviceToHost, st));
    MG_CUDA_TRY(cudaStreamSynchronize(st));
    MG_CUDA_TRY(cudaGetLastError());
    eps = sqrt(ws->h_scalars[SC_SUMSQ] / (double)n3) / snorm;
    if (nh < 64) S->resid_hist[nh++] = eps;
  }
  if (status == MGGLAM_OK && !isfinite(eps)) status = MGGLAM_ERR_NONFINITE;
  S->cycles = cyc;
  S->outer = outer;
  S->resid = eps;
  S->converged = eps <= tol;
  S->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (status == MGGLAM_OK && !S->converged) status = MGGLAM_ERR_NOT_CONVERGED;
  return status;
}

}  // namespace mg
