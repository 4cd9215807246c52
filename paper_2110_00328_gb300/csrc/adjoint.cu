// adjoint.cu -- gradients of a loss through the scalar-field solve.
//
// The solve defines u*(delta, theta) by N(u*; delta, theta) = 0 (the discrete
// equations of Eq. fR_eom_codeunit2 / Eq. sym_eom_code_unit, theta =
// ln|f_R0|).  For a loss l(u*) with g = dl/du*, the adjoint field lambda solves
// J^T lambda = g with J = dN/du at u*, and
//   dl/d delta = -(dN/d delta)^T lambda,   dl/d theta = -lambda . dN/d theta.
// With Delta_h the 7-point Laplacian (symmetric) the transposed problem takes
// one screened-Poisson form for both models,
//   -kappa Delta_h lambda + m lambda = sigma g,
//   f(R):      J = -c^2 Delta_h diag((n+1)u^n) + diag(K/u^2), so
//              kappa = c~^2, m = K/((n+1)u^{n+2}), sigma = 1/((n+1)u^n);
//   symmetron: J = c^2 Delta_h - diag(msym (rho a*^3/a^3 - 1 + 3u^2)), so
//              kappa = c~^2, m = msym (rho a*^3/a^3 - 1 + 3u^2), sigma = -1;
// m > 0 in both (the f(R) field is positive; in the symmetron's broken phase
// rho a*^3/a^3 - 1 + 3u^2 = 2u^2 at the local minimum), so the operator is
// symmetric positive definite and red-black Gauss-Seidel multigrid converges.
//
// Solver: FP64 outer residual r = sigma g - A lambda on the fine level, FP32
// correction-scheme V-cycles for A e = r (the same cycle shape, restriction
// and prolongation as the forward solve), lambda += e.  The coarse-level mass
// is the 8-child mean of the fine mass, rebuilt from u* on every call (no state
// of the forward V-cycles is kept).
#include <math.h>
#include <string.h>

#include <chrono>
#include <mutex>

#include "ff.cuh"
#include "mg_common.cuh"
#include "mg_internal.h"
#include "sweep32.cuh"

namespace mg {

// ---- per-cell coefficients from the converged field ----
// m64, m32 = mass; rhs = sigma * g (FP64); also the density-gradient factor
// gam (dl/d delta_i = gam_i lambda_i) and the theta factor tq (dl/d theta =
// sum lambda_i tq_i).
template <int K>
__global__ void k_adj_setup(ModelDev m, int n, const double* __restrict__ u, const float* __restrict__ rho32,
                            const double* __restrict__ rho_sum, const double* __restrict__ g,
                            double* __restrict__ m64, float* __restrict__ m32, double* __restrict__ rhs,
                            double* __restrict__ gam, double* __restrict__ tq) {
  const int i = blockIdx.z, j = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const size_t t = cidx(n, i, j, k);
  const double uc = u[t];
  double mass, sigma, gm, tqv;
  if constexpr (is_fr(K)) {
    constexpr int np1 = K + 1;
    double un = 1.0;  // u^n
    for (int q = 0; q < K; ++q) un *= uc;
    mass = m.K / ((double)np1 * un * uc * uc);
    sigma = 1.0 / ((double)np1 * un);
    gm = -m.om_a;                   // dN/d delta = Om/a
    tqv = m.K / ((double)np1 * uc);  // -dN/d theta = K/((n+1)u)
  } else {
    const double r = (double)rho32[t] * ((double)n * n * n / *rho_sum);
    mass = m.msym * (r * m.rat3 - 1.0 + 3.0 * uc * uc);
    sigma = -1.0;
    gm = m.msym * m.rat3 * uc;      // dN/d delta = -msym (a*/a)^3 u
    tqv = 0.0;
  }
  m64[t] = mass;
  m32[t] = (float)mass;
  rhs[t] = sigma * g[t];
  gam[t] = gm;
  tq[t] = tqv;
}

// r = rhs - (-kappa Delta_h lambda + m lambda) on the fine level (FP64);
// writes b = float(r) and per-block partial sums of r^2 and rhs^2.
__global__ void k_adj_residual64(int n, double kappa, const double* __restrict__ lam, const double* __restrict__ m64,
                                 const double* __restrict__ rhs, float* __restrict__ b,
                                 double* __restrict__ partials, double* __restrict__ partials2) {
  double acc = 0.0, acc2 = 0.0;
  for (int r = blockIdx.x; r < n * n; r += gridDim.x) {
    const int i = r / n, j = r - (r / n) * n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const size_t t = cidx(n, i, j, k);
      const double L = lam[cidx(n, wrapi(i + 1, n), j, k)] + lam[cidx(n, wrapi(i - 1, n), j, k)] +
                       lam[cidx(n, i, wrapi(j + 1, n), k)] + lam[cidx(n, i, wrapi(j - 1, n), k)] +
                       lam[cidx(n, i, j, wrapi(k + 1, n))] + lam[cidx(n, i, j, wrapi(k - 1, n))];
      const double lc = lam[t];
      const double v = rhs[t] - (-kappa * (L - 6.0 * lc) + m64[t] * lc);
      b[t] = (float)v;
      acc += v * v;
      acc2 += rhs[t] * rhs[t];
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  acc2 = block_sum(acc2);
  if (threadIdx.x == 0) partials2[blockIdx.x] = acc2;
}

// The same fine-level residual in float-float arithmetic (lambda, m and rhs
// split exactly from FP64; ~2^-48 per operation): z-marching 8 x 32 tiles with
// a three-plane ring of lambda in shared memory.  Writes b = float(r) and
// per-block partial sums of r^2.
template <int TJ, int TK>
__global__ void __launch_bounds__(TJ* TK) k_adj_residual_ff(int n, int chunk, ff kappa, const double* __restrict__ lam,
                                                            const double* __restrict__ m64,
                                                            const double* __restrict__ rhs, float* __restrict__ b,
                                                            double* __restrict__ partials) {
  constexpr int PJ = TJ + 2, PK = TK + 2, PS = PJ * PK, NT = TJ * TK;
  __shared__ float s_h[3][PS], s_l[3][PS];
  const int tiles_k = n / TK;
  const int tile = blockIdx.x, cb = blockIdx.y;
  const int k0 = (tile % tiles_k) * TK, j0 = (tile / tiles_k) * TJ;
  const int i0 = cb * chunk, i1 = min(i0 + chunk, n);
  const int t = threadIdx.x, tj = t / TK, tk = t - tj * TK;
  const int jg = j0 + tj, kg = k0 + tk, cc = (tj + 1) * PK + tk + 1;
  const size_t nn = (size_t)n * n;
  auto load = [&](int p) {
    const int ig = p < 0 ? p + n : (p >= n ? p - n : p);
    const int slot = (p + 3) % 3;
    for (int c = t; c < PS; c += NT) {
      const int jj = c / PK, kk = c - jj * PK;
      const ff v = ff_from_double(lam[(size_t)ig * nn + (size_t)wrapi(j0 + jj - 1, n) * n + wrapi(k0 + kk - 1, n)]);
      s_h[slot][c] = v.hi;
      s_l[slot][c] = v.lo;
    }
  };
  auto W = [&](int slot, int c) { return ff{s_h[slot][c], s_l[slot][c]}; };
  float acc = 0.f;
  load(i0 - 1);
  load(i0);
  for (int i = i0; i < i1; ++i) {
    load(i + 1);
    __syncthreads();
    const int sl = (i + 3) % 3, sm = (i + 2) % 3, sp = (i + 4) % 3;
    const size_t g = (size_t)i * nn + (size_t)jg * n + kg;
    const ff lc = W(sl, cc);
    ff L = ff_add(W(sm, cc), W(sp, cc));
    L = ff_add(L, ff_add(W(sl, cc - PK), W(sl, cc + PK)));
    L = ff_add(L, ff_add(W(sl, cc - 1), W(sl, cc + 1)));
    L = ff_sub(L, ff_mul_f(lc, 6.f));
    // r = rhs + kappa (L - 6 lambda) - m lambda
    ff r = ff_add(ff_from_double(rhs[g]), ff_mul(kappa, L));
    r = ff_sub(r, ff_mul(ff_from_double(m64[g]), lc));
    const float rv = ff_to_float(r);
    b[g] = rv;
    acc += rv * rv;
    __syncthreads();
  }
  const double a = block_sum((double)acc);
  if (threadIdx.x == 0) partials[blockIdx.x + blockIdx.y * gridDim.x] = a;
}

// sum of rhs^2 (once per solve: the residual's normaliser)
__global__ void k_adj_rhs_sumsq(long long n3, const double* __restrict__ rhs, double* __restrict__ partials) {
  double acc = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    acc += rhs[t] * rhs[t];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void k_adj_sum(const double* __restrict__ p, int count, double* __restrict__ out) {
  double a = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) a += p[i];
  a = block_sum(a);
  if (threadIdx.x == 0) *out = a;
}

__global__ void k_adj_finalize(const double* __restrict__ p, const double* __restrict__ p2, int count,
                               double* __restrict__ out) {
  double a = 0.0, a2 = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    a += p[i];
    a2 += p2[i];
  }
  a = block_sum(a);
  if (threadIdx.x == 0) out[0] = a;
  a2 = block_sum(a2);
  if (threadIdx.x == 0) out[1] = a2;
}

// 1 / (6 kh + m), the inverse diagonal of one level (kh = kappa/h^2).
__global__ void k_adj_dinv32(long long n3, float kh, const float* __restrict__ m32, float* __restrict__ dinv) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    dinv[t] = 1.f / (6.f * kh + m32[t]);
}

// Red-black Gauss-Seidel on one colour: x_i = (b_i + kh sum_nb x) / (6 kh + m_i), kh = kappa/h^2.
__global__ void __launch_bounds__(64) k_adj_smooth32(int n, float kh, float* __restrict__ x, const float* __restrict__ b,
                                                     const float* __restrict__ dinv, int parity) {
  const int i = blockIdx.z, j = blockIdx.y;
  const int kk = blockIdx.x * blockDim.x + threadIdx.x;
  if (kk >= (n >> 1)) return;
  const int k = 2 * kk + ((i + j + parity) & 1);
  const size_t c = cidx(n, i, j, k);
  const float L = x[cidx(n, wrapi(i + 1, n), j, k)] + x[cidx(n, wrapi(i - 1, n), j, k)] +
                  x[cidx(n, i, wrapi(j + 1, n), k)] + x[cidx(n, i, wrapi(j - 1, n), k)] +
                  x[cidx(n, i, j, wrapi(k + 1, n))] + x[cidx(n, i, j, wrapi(k - 1, n))];
  x[c] = (b[c] + kh * L) * dinv[c];
}

// The same colour step, four cells per lane (n % 4 == 0, n >= 8; as smooth_quad):
// block (32, 4), grid (ceil(n/128), n, n/4).
__global__ void __launch_bounds__(128) k_adj_smooth32q(int n, float kh, float* __restrict__ x,
                                                       const float* __restrict__ b, const float* __restrict__ dinv,
                                                       int parity) {
  const int i = blockIdx.z * 4 + threadIdx.y;
  if (i >= n) return;  // whole warps
  const int j = blockIdx.y, lane = threadIdx.x, tq = blockIdx.x * 32 + lane;
  const int nq = n >> 2;
  const bool act = tq < nq;
  const int k0 = 4 * (act ? tq : nq - 1);
  const long long nn = (long long)n * n;
  const long long c0 = (long long)i * nn + (long long)j * n + k0;
  const long long djp = (j + 1 < n) ? (long long)n : -(long long)(n - 1) * n;
  const long long djm = (j > 0) ? -(long long)n : (long long)(n - 1) * n;
  const long long dip = (i + 1 < n) ? nn : -(long long)(n - 1) * nn;
  const long long dim = (i > 0) ? -nn : (long long)(n - 1) * nn;
  float* x0 = x + c0;
  const float4 X = ld4(x0), B = ld4(b + c0), D = ld4(dinv + c0);
  const float4 P = ld4(x0 + djp), M = ld4(x0 + djm), Q = ld4(x0 + dip), R = ld4(x0 + dim);
  if (((i + j + parity) & 1) == 0) {
    // cells k0 and k0+2
    float km = __shfl_up_sync(0xffffffffu, X.w, 1);
    if (lane == 0) km = x[c0 + (k0 == 0 ? n - 1 : -1)];
    const float LA = (km + X.y) + (P.x + M.x) + (Q.x + R.x);
    const float LB = (X.y + X.w) + (P.z + M.z) + (Q.z + R.z);
    if (act) {
      x0[0] = (B.x + kh * LA) * D.x;
      x0[2] = (B.z + kh * LB) * D.z;
    }
  } else {
    // cells k0+1 and k0+3
    float kp = __shfl_down_sync(0xffffffffu, X.x, 1);
    if (lane == 31 || tq + 1 >= nq) kp = x[c0 + (k0 + 4 == n ? 4 - n : 4)];
    const float LA = (X.x + X.z) + (P.y + M.y) + (Q.y + R.y);
    const float LB = (X.z + kp) + (P.w + M.w) + (Q.w + R.w);
    if (act) {
      x0[1] = (B.y + kh * LA) * D.y;
      x0[3] = (B.w + kh * LB) * D.w;
    }
  }
}

__global__ void __launch_bounds__(512) k_adj_coarse32(int n, float kh, float* __restrict__ x,
                                                      const float* __restrict__ b, const float* __restrict__ dinv,
                                                      int sweeps) {
  const int n3 = n * n * n;
  for (int s = 0; s < sweeps; ++s)
    for (int parity = 0; parity < 2; ++parity) {
      for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int k = t % n, j = (t / n) % n, i = t / (n * n);
        if (((i + j + k) & 1) != parity) continue;
        const float L = x[cidx(n, wrapi(i + 1, n), j, k)] + x[cidx(n, wrapi(i - 1, n), j, k)] +
                        x[cidx(n, i, wrapi(j + 1, n), k)] + x[cidx(n, i, wrapi(j - 1, n), k)] +
                        x[cidx(n, i, j, wrapi(k + 1, n))] + x[cidx(n, i, j, wrapi(k - 1, n))];
        x[t] = (b[t] + kh * L) * dinv[t];
      }
      __syncthreads();
    }
}

// Coarse right-hand side: b^H = R (b - A x) over the 8 children; x^H = 0.
__global__ void __launch_bounds__(64) k_adj_restrict_resid32(int nf, float kh, const float* __restrict__ x,
                                                             const float* __restrict__ b,
                                                             const float* __restrict__ m32, float* __restrict__ bH,
                                                             float* __restrict__ xH) {
  const int nc = nf >> 1;
  const int I = blockIdx.z, J = blockIdx.y;
  const int Kc = blockIdx.x * blockDim.x + threadIdx.x;
  if (Kc >= nc) return;
  float s = 0.f;
  for (int di = 0; di < 2; ++di)
    for (int dj = 0; dj < 2; ++dj)
      for (int dk = 0; dk < 2; ++dk) {
        const int i = 2 * I + di, j = 2 * J + dj, k = 2 * Kc + dk;
        const size_t c = cidx(nf, i, j, k);
        const float L = x[cidx(nf, wrapi(i + 1, nf), j, k)] + x[cidx(nf, wrapi(i - 1, nf), j, k)] +
                        x[cidx(nf, i, wrapi(j + 1, nf), k)] + x[cidx(nf, i, wrapi(j - 1, nf), k)] +
                        x[cidx(nf, i, j, wrapi(k + 1, nf))] + x[cidx(nf, i, j, wrapi(k - 1, nf))];
        s += b[c] - (-kh * (L - 6.f * x[c]) + m32[c] * x[c]);
      }
  const size_t t = cidx(nc, I, J, Kc);
  bH[t] = 0.125f * s;
  xH[t] = 0.f;
}

// The same restriction, sixteen fine cells per lane (nf % 4 == 0, as
// restrict_quad): block (32, 4), grid (ceil(nf/128), nc [J], ceil(nc/4) [I]).
__global__ void __launch_bounds__(128) k_adj_restrict_resid32q(int nf, float kh, const float* __restrict__ x,
                                                               const float* __restrict__ b,
                                                               const float* __restrict__ m32, float* __restrict__ bH,
                                                               float* __restrict__ xH) {
  const int nc = nf >> 1, nq = nf >> 2;
  const int I = blockIdx.z * 4 + threadIdx.y;
  if (I >= nc) return;  // whole warps
  const int J = blockIdx.y, lane = threadIdx.x, tq = blockIdx.x * 32 + lane;
  const bool act = tq < nq;
  const int k0 = 4 * (act ? tq : nq - 1);
  const int i0 = 2 * I, j0 = 2 * J;
  const int iA = i0 == 0 ? nf - 1 : i0 - 1, iB = i0 + 2 == nf ? 0 : i0 + 2;
  const int jA = j0 == 0 ? nf - 1 : j0 - 1, jB = j0 + 2 == nf ? 0 : j0 + 2;
  auto row = [&](int i, int j) { return ((long long)i * nf + j) * nf + k0; };
  float4 X[2][2];
  long long co[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      co[a][c] = row(i0 + a, j0 + c);
      X[a][c] = ld4(x + co[a][c]);
    }
  float4 xi[2][2], xj[2][2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    xi[0][c] = ld4(x + row(iA, j0 + c));
    xi[1][c] = ld4(x + row(iB, j0 + c));
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    xj[a][0] = ld4(x + row(i0 + a, jA));
    xj[a][1] = ld4(x + row(i0 + a, jB));
  }
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float4 q = X[a][c];
      float qm = __shfl_up_sync(0xffffffffu, q.w, 1);
      float qp = __shfl_down_sync(0xffffffffu, q.x, 1);
      if (lane == 0) qm = x[co[a][c] + (k0 == 0 ? nf - 1 : -1)];
      if (lane == 31 || tq + 1 >= nq) qp = x[co[a][c] + (k0 + 4 == nf ? 4 - nf : 4)];
      const float4 ni = a == 0 ? xi[0][c] : X[0][c], pi = a == 0 ? X[1][c] : xi[1][c];
      const float4 nj = c == 0 ? xj[a][0] : X[a][0], pj = c == 0 ? X[a][1] : xj[a][1];
      const float4 Bv = ld4(b + co[a][c]), Mv = ld4(m32 + co[a][c]);
      auto d = [&](float bb, float mm, float xc, float L) { return bb + kh * (L - 6.f * xc) - mm * xc; };
      s0 += d(Bv.x, Mv.x, q.x, (qm + q.y) + (ni.x + pi.x) + (nj.x + pj.x)) +
            d(Bv.y, Mv.y, q.y, (q.x + q.z) + (ni.y + pi.y) + (nj.y + pj.y));
      s1 += d(Bv.z, Mv.z, q.z, (q.y + q.w) + (ni.z + pi.z) + (nj.z + pj.z)) +
            d(Bv.w, Mv.w, q.w, (q.z + qp) + (ni.w + pi.w) + (nj.w + pj.w));
    }
  if (act) {
    const long long t = ((long long)I * nc + J) * nc + (k0 >> 1);
    *reinterpret_cast<float2*>(bH + t) = make_float2(0.125f * s0, 0.125f * s1);
    *reinterpret_cast<float2*>(xH + t) = make_float2(0.f, 0.f);
  }
}

// x^h += P x^H, four fine cells per lane (as prolong_quad, without the
// restricted-solution term): block (32, 4), grid (ceil(nf/128), nf, nf/4).
__global__ void __launch_bounds__(128) k_adj_prolong32q(int nc, const float* __restrict__ xH, float* __restrict__ xf) {
  const int nf = nc << 1, nq = nf >> 2;
  const int i = blockIdx.z * 4 + threadIdx.y, j = blockIdx.y, lane = threadIdx.x, tq = blockIdx.x * 32 + lane;
  const bool act = tq < nq;
  const int t = act ? tq : nq - 1;
  const int k0 = 4 * t, K0 = 2 * t;
  const int I = i >> 1, J = j >> 1;
  int I2 = I + ((i & 1) ? 1 : -1), J2 = J + ((j & 1) ? 1 : -1);
  I2 = I2 < 0 ? nc - 1 : (I2 >= nc ? 0 : I2);
  J2 = J2 < 0 ? nc - 1 : (J2 >= nc ? 0 : J2);
  const long long rA = ((long long)I * nc + J) * nc, rB = ((long long)I2 * nc + J) * nc,
                  rC = ((long long)I * nc + J2) * nc, rD = ((long long)I2 * nc + J2) * nc;
  auto two = [&](long long r) { return *reinterpret_cast<const float2*>(xH + r + K0); };
  const float2 A = two(rA), B = two(rB), C = two(rC), D = two(rD);
  const float Rx = 9.f * A.x + 3.f * (B.x + C.x) + D.x;
  const float Ry = 9.f * A.y + 3.f * (B.y + C.y) + D.y;
  float Rm = __shfl_up_sync(0xffffffffu, Ry, 1);
  float Rp = __shfl_down_sync(0xffffffffu, Rx, 1);
  if (lane == 0) {
    const int Km = K0 == 0 ? nc - 1 : K0 - 1;
    Rm = 9.f * xH[rA + Km] + 3.f * (xH[rB + Km] + xH[rC + Km]) + xH[rD + Km];
  }
  if (lane == 31 || tq + 1 >= nq) {
    const int Kp = K0 + 2 == nc ? 0 : K0 + 2;
    Rp = 9.f * xH[rA + Kp] + 3.f * (xH[rB + Kp] + xH[rC + Kp]) + xH[rD + Kp];
  }
  constexpr float w = 1.f / 64.f;
  float* p = xf + ((long long)i * nf + j) * nf + k0;
  const float4 old = ld4(p);
  if (act)
    *reinterpret_cast<float4*>(p) = make_float4(old.x + (3.f * Rx + Rm) * w, old.y + (3.f * Rx + Ry) * w,
                                                old.z + (3.f * Ry + Rx) * w, old.w + (3.f * Ry + Rp) * w);
}

// x^h += P x^H (27/9/3/1 weights).
__global__ void __launch_bounds__(64) k_adj_prolong32(int nc, const float* __restrict__ xH, float* __restrict__ xf) {
  const int nf = nc << 1;
  const int i = blockIdx.z, j = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const int I = i >> 1, J = j >> 1, Kc = k >> 1;
  const int I2 = wrapi(I + ((i & 1) ? 1 : -1), nc);
  const int J2 = wrapi(J + ((j & 1) ? 1 : -1), nc);
  const int K2 = wrapi(Kc + ((k & 1) ? 1 : -1), nc);
#define XH(a, b, c) xH[cidx(nc, a, b, c)]
  const float corr = (27.f * XH(I, J, Kc) + 9.f * (XH(I2, J, Kc) + XH(I, J2, Kc) + XH(I, J, K2)) +
                      3.f * (XH(I2, J2, Kc) + XH(I2, J, K2) + XH(I, J2, K2)) + XH(I2, J2, K2)) *
                     (1.f / 64.f);
#undef XH
  xf[cidx(nf, i, j, k)] += corr;
}

__global__ void __launch_bounds__(64) k_adj_restrict_m32(int nf, const float* __restrict__ fine,
                                                         float* __restrict__ coarse) {
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

// lambda += e; grad_rho = gam * lambda (after the last step); partial sums of lambda * tq.
__global__ void k_adj_apply(long long n3, double* __restrict__ lam, const float* __restrict__ e) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    lam[t] += (double)e[t];
}

// Also partial sums of (dl/d delta_i) rho_i, the term the mean-1 normalisation
// of the density adds to the gradient with respect to the caller's rho.
__global__ void k_adj_outputs(long long n3, const double* __restrict__ lam, const double* __restrict__ gam,
                              const double* __restrict__ tq, const float* __restrict__ rho32,
                              double* __restrict__ grad_rho, double* __restrict__ partials,
                              double* __restrict__ partials2) {
  double acc = 0.0, acc2 = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    const double g = gam[t] * lam[t];
    grad_rho[t] = g;
    acc += lam[t] * tq[t];
    acc2 += g * (double)rho32[t];
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
  acc2 = block_sum(acc2);
  if (threadIdx.x == 0) partials2[blockIdx.x] = acc2;
}

// Chain rule through delta = rho / mu - 1, mu = sum(rho) / N^3:
//   dl/d rho_j = (dl/d delta_j - sum_i (dl/d delta_i) rho_i / sum(rho)) / mu.
__global__ void k_adj_grad_raw(long long n3, const double* __restrict__ g, const double* __restrict__ dot,
                               const double* __restrict__ rho_sum, double* __restrict__ out) {
  const double S = *rho_sum, shift = *dot / S, inv_mu = (double)n3 / S;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = (g[t] - shift) * inv_mu;
}

// ---------------------------------------------------------------------------
// Scratch: one allocation per (device, N): FP64 lambda, m, rhs, gam, tq on the
// fine level; FP32 x, b, m on every level; partial sums.
// ---------------------------------------------------------------------------

struct AdjWork {
  int device = -1, N = 0, nlev = 0;
  void* base = nullptr;
  double *lam = nullptr, *m64 = nullptr, *rhs = nullptr, *gam = nullptr, *tq = nullptr;
  double *partials = nullptr, *partials2 = nullptr, *scal = nullptr, *h_scal = nullptr;
  int n[kMaxLevels];
  float *x[kMaxLevels], *b[kMaxLevels], *m32[kMaxLevels], *dinv[kMaxLevels];
};

static std::mutex g_adj_mu;
static AdjWork* g_adj[32];
static int g_nadj = 0;

static int adj_work(int N, int levels, AdjWork** out) {
  int dev = 0;
  MG_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_adj_mu);
  const int nlev = count_levels(N, levels);
  for (int i = 0; i < g_nadj; ++i)
    if (g_adj[i]->device == dev && g_adj[i]->N == N && g_adj[i]->nlev == nlev) {
      *out = g_adj[i];
      return MGGLAM_OK;
    }
  if (g_nadj >= 32) return MGGLAM_ERR_OOM;
  AdjWork* w = new AdjWork();
  w->device = dev;
  w->N = N;
  w->nlev = nlev;
  const size_t n3 = (size_t)N * N * N;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
  const size_t o_lam = take(n3 * 8), o_m = take(n3 * 8), o_rhs = take(n3 * 8), o_gam = take(n3 * 8),
               o_tq = take(n3 * 8), o_p = take(kMaxReduceBlocks * 8), o_p2 = take(kMaxReduceBlocks * 8),
               o_s = take(64);
  size_t ox[kMaxLevels], ob[kMaxLevels], om[kMaxLevels], od[kMaxLevels];
  for (int l = 0, nn = N; l < nlev; ++l, nn /= 2) {
    const size_t c = (size_t)nn * nn * nn;
    w->n[l] = nn;
    ox[l] = take(c * 4);
    ob[l] = take(c * 4);
    om[l] = take(c * 4);
    od[l] = take(c * 4);
  }
  if (cudaMalloc(&w->base, off) != cudaSuccess) {
    cudaGetLastError();
    delete w;
    return MGGLAM_ERR_OOM;
  }
  if (cudaMallocHost((void**)&w->h_scal, 64) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(w->base);
    delete w;
    return MGGLAM_ERR_OOM;
  }
  char* b = (char*)w->base;
  w->lam = (double*)(b + o_lam);
  w->m64 = (double*)(b + o_m);
  w->rhs = (double*)(b + o_rhs);
  w->gam = (double*)(b + o_gam);
  w->tq = (double*)(b + o_tq);
  w->partials = (double*)(b + o_p);
  w->partials2 = (double*)(b + o_p2);
  w->scal = (double*)(b + o_s);
  for (int l = 0; l < nlev; ++l) {
    w->x[l] = (float*)(b + ox[l]);
    w->b[l] = (float*)(b + ob[l]);
    w->m32[l] = (float*)(b + om[l]);
    w->dinv[l] = (float*)(b + od[l]);
  }
  g_adj[g_nadj++] = w;
  *out = w;
  return MGGLAM_OK;
}

void release_adjoint_work() {
  std::lock_guard<std::mutex> lk(g_adj_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  int keep = 0;
  for (int i = 0; i < g_nadj; ++i) {
    if (g_adj[i]->device == dev) {
      cudaFree(g_adj[i]->base);
      cudaFreeHost(g_adj[i]->h_scal);
      delete g_adj[i];
    } else {
      g_adj[keep++] = g_adj[i];
    }
  }
  g_nadj = keep;
}

static dim3 grid_k(int n_k, int n_j, int n_i) { return dim3((n_k + 63) / 64, n_j, n_i); }

static void adj_smooth(AdjWork* w, int l, float kh, int sweeps, cudaStream_t st) {
  const int n = w->n[l];
  for (int s = 0; s < sweeps; ++s)
    for (int par = 0; par < 2; ++par) {
      if (n % 4 == 0 && n >= 8)
        k_adj_smooth32q<<<dim3((n / 4 + 31) / 32, n, n / 4), dim3(32, 4), 0, st>>>(n, kh, w->x[l], w->b[l],
                                                                                 w->dinv[l], par);
      else
        k_adj_smooth32<<<grid_k(n / 2, n, n), 64, 0, st>>>(n, kh, w->x[l], w->b[l], w->dinv[l], par);
      note_launch(1);
    }
}

static void adj_vcycle(AdjWork* w, int l, double kappa, const mgglam_params* prm, cudaStream_t st) {
  const int n = w->n[l];
  const float kh = (float)(kappa / ((double)(1 << l) * (double)(1 << l)));
  if (l == w->nlev - 1) {
    if ((long long)n * n * n <= 4096) {
      k_adj_coarse32<<<1, 512, 0, st>>>(n, kh, w->x[l], w->b[l], w->dinv[l], prm->coarse_sweeps);
      note_launch(1);
    } else {
      adj_smooth(w, l, kh, prm->coarse_sweeps, st);
    }
    return;
  }
  adj_smooth(w, l, kh, prm->nu1, st);
  const int nc = w->n[l + 1];
  if (n % 4 == 0 && n >= 8)
    k_adj_restrict_resid32q<<<dim3((n / 4 + 31) / 32, nc, (nc + 3) / 4), dim3(32, 4), 0, st>>>(
        n, kh, w->x[l], w->b[l], w->m32[l], w->b[l + 1], w->x[l + 1]);
  else
    k_adj_restrict_resid32<<<grid_k(nc, nc, nc), 64, 0, st>>>(n, kh, w->x[l], w->b[l], w->m32[l], w->b[l + 1],
                                                               w->x[l + 1]);
  note_launch(1);
  adj_vcycle(w, l + 1, kappa, prm, st);
  if (n % 4 == 0 && n >= 8)
    k_adj_prolong32q<<<dim3((n / 4 + 31) / 32, n, n / 4), dim3(32, 4), 0, st>>>(nc, w->x[l + 1], w->x[l]);
  else
    k_adj_prolong32<<<grid_k(n, n, n), 64, 0, st>>>(nc, w->x[l + 1], w->x[l]);
  note_launch(1);
  adj_smooth(w, l, kh, prm->nu2, st);
}

int solve_adjoint(const mgglam_params* prm, double a, const double* field, const float* rho, int N,
                  const double* grad_field, double* grad_rho, double* grad_rho_raw, double* grad_theta, double tol,
                  mgglam_stats* stats, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  ModelDev m;
  int rc = make_model(prm, a, N, &m);
  if (rc) return rc;
  if (!(is_fr(m.kind) || m.kind == KSYM)) return MGGLAM_ERR_ARG;
  AdjWork* w = nullptr;
  if ((rc = adj_work(N, prm->levels, &w))) return rc;
  Workspace* ws = nullptr;  // for the density mean scratch
  if ((rc = get_workspace(4, MGGLAM_FP64, 1, &ws))) return rc;
  const long long n3 = (long long)N * N * N;
  if ((rc = launch_density_mean(rho, (size_t)n3, ws->partials, ws->scalars + SC_MEAN, st))) return rc;
  const dim3 gf = grid_k(N, N, N);
  switch (m.kind) {
    case KFR0: k_adj_setup<KFR0><<<gf, 64, 0, st>>>(m, N, field, rho, ws->scalars + SC_MEAN, grad_field, w->m64, w->m32[0], w->rhs, w->gam, w->tq); break;
    case KFR1: k_adj_setup<KFR1><<<gf, 64, 0, st>>>(m, N, field, rho, ws->scalars + SC_MEAN, grad_field, w->m64, w->m32[0], w->rhs, w->gam, w->tq); break;
    case KFR2: k_adj_setup<KFR2><<<gf, 64, 0, st>>>(m, N, field, rho, ws->scalars + SC_MEAN, grad_field, w->m64, w->m32[0], w->rhs, w->gam, w->tq); break;
    default: k_adj_setup<KSYM><<<gf, 64, 0, st>>>(m, N, field, rho, ws->scalars + SC_MEAN, grad_field, w->m64, w->m32[0], w->rhs, w->gam, w->tq); break;
  }
  note_launch(1);
  for (int l = 1; l < w->nlev; ++l) {
    k_adj_restrict_m32<<<grid_k(w->n[l], w->n[l], w->n[l]), 64, 0, st>>>(w->n[l - 1], w->m32[l - 1], w->m32[l]);
    note_launch(1);
  }
  for (int l = 0; l < w->nlev; ++l) {
    const long long nl3 = (long long)w->n[l] * w->n[l] * w->n[l];
    const float kh = (float)(m.c2 / ((double)(1 << l) * (double)(1 << l)));
    k_adj_dinv32<<<stream_grid(nl3), kThreads, 0, st>>>(nl3, kh, w->m32[l], w->dinv[l]);
    note_launch(1);
  }
  MG_CUDA_TRY(cudaMemsetAsync(w->lam, 0, (size_t)n3 * 8, st));
  const double kappa = m.c2;
  const int gr = N * N < 2048 ? N * N : 2048;
  const int bt = N >= 256 ? 256 : (N <= 32 ? 32 : ((N + 31) / 32) * 32);
  // the fine residual in float-float on meshes its 8 x 32 tiles divide, else FP64
  const bool ffr = N % 32 == 0;
  const int chunk = ffr ? march_chunk(N, (long long)(N / 32) * (N / 8), (const void*)k_adj_residual_ff<8, 32>, 256) : N;
  const dim3 gff((N / 32) * (N / 8), (N + chunk - 1) / chunk);
  const ff kappa_ff = {(float)kappa, (float)(kappa - (double)(float)kappa)};
  if (ffr) {
    k_adj_rhs_sumsq<<<stream_grid(n3), kThreads, 0, st>>>(n3, w->rhs, w->partials2);
    k_adj_sum<<<1, 1024, 0, st>>>(w->partials2, stream_grid(n3), w->scal + 1);
    note_launch(2);
  }
  auto residual = [&]() -> int {
    if (ffr) {
      k_adj_residual_ff<8, 32><<<gff, 256, 0, st>>>(N, chunk, kappa_ff, w->lam, w->m64, w->rhs, w->b[0], w->partials);
      k_adj_sum<<<1, 1024, 0, st>>>(w->partials, (int)(gff.x * gff.y), w->scal);
    } else {
      k_adj_residual64<<<gr, bt, 0, st>>>(N, kappa, w->lam, w->m64, w->rhs, w->b[0], w->partials, w->partials2);
      k_adj_finalize<<<1, 1024, 0, st>>>(w->partials, w->partials2, gr, w->scal);
    }
    note_launch(2);
    MG_CUDA_TRY(cudaMemcpyAsync(w->h_scal, w->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MG_CUDA_TRY(cudaStreamSynchronize(st));
    MG_CUDA_TRY(cudaGetLastError());
    return MGGLAM_OK;
  };
  if ((rc = residual())) return rc;
  const double bnorm = sqrt(w->h_scal[1] / (double)n3);
  const double snorm = bnorm > 0.0 ? bnorm : 1.0;
  double eps = sqrt(w->h_scal[0] / (double)n3) / snorm;
  mgglam_stats local;
  mgglam_stats* S = stats ? stats : &local;
  memset(S, 0, sizeof(*S));
  S->resid0 = eps;
  S->resid_hist[0] = eps;
  int cyc = 0, outer = 0, nh = 1;
  // inner FP32 cycles per FP64/float-float step: fixed, or (inner_cycles = 0)
  // enough for tol at the observed contraction, capped where one single-
  // precision correction stops gaining (~1e-6), as in the forward solve
  double rho_est = kInitialContraction;
  int status = MGGLAM_OK;
  while (!(eps <= tol) && cyc < prm->max_cycles) {
    if (!isfinite(eps)) { status = MGGLAM_ERR_NONFINITE; break; }
    int inner = prm->inner_cycles;
    if (inner <= 0) {
      const double lr = log(rho_est);
      const int need = (int)ceil(log(fmax(tol, 1e-300) / eps) / lr - 1e-9);
      const int cap = (int)ceil(log(kFp32StepGain) / lr - 1e-9);
      inner = need < 1 ? 1 : (need > cap ? cap : need);
    }
    const double eps_before = eps;
    int done = 0;
    MG_CUDA_TRY(cudaMemsetAsync(w->x[0], 0, (size_t)n3 * 4, st));
    for (int c = 0; c < inner && cyc < prm->max_cycles; ++c, ++cyc, ++done) adj_vcycle(w, 0, kappa, prm, st);
    k_adj_apply<<<stream_grid(n3), kThreads, 0, st>>>(n3, w->lam, w->x[0]);
    note_launch(1);
    ++outer;
    if ((rc = residual())) return rc;
    eps = sqrt(w->h_scal[0] / (double)n3) / snorm;
    if (nh < 64) S->resid_hist[nh++] = eps;
    if (done > 0 && eps > 0.0 && eps < eps_before && eps / eps_before > kFp32StepGain)
      rho_est = fmin(0.5, fmax(0.01, pow(eps / eps_before, 1.0 / done)));
  }
  const int go = grid_for(n3);
  k_adj_outputs<<<go, kThreads, 0, st>>>(n3, w->lam, w->gam, w->tq, rho, grad_rho, w->partials, w->partials2);
  k_adj_finalize<<<1, 1024, 0, st>>>(w->partials, w->partials2, go, w->scal);
  note_launch(2);
  if (grad_rho_raw) {
    k_adj_grad_raw<<<stream_grid(n3), kThreads, 0, st>>>(n3, grad_rho, w->scal + 1, ws->scalars + SC_MEAN,
                                                          grad_rho_raw);
    note_launch(1);
  }
  MG_CUDA_TRY(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  MG_CUDA_TRY(cudaStreamSynchronize(st));
  MG_CUDA_TRY(cudaGetLastError());
  if (grad_theta) *grad_theta = w->h_scal[0];
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

extern "C" int mgglam_solve_adjoint(const mgglam_params* prm, double a, const double* field, const float* rho,
                                    int N, const double* grad_field, double* grad_rho, double* grad_rho_raw,
                                    double* grad_logfR0, double tol, mgglam_stats* stats, void* stream) {
  if (!prm || !field || !rho || !grad_field || !grad_rho || !(tol >= 0.0)) return MGGLAM_ERR_ARG;
  if (grad_rho_raw == grad_rho) return MGGLAM_ERR_ARG;
  if (N < 4 || N > 2048 || N % 2) return MGGLAM_ERR_SHAPE;
  if (prm->model != MGGLAM_FR && prm->model != MGGLAM_SYMMETRON) return MGGLAM_ERR_ARG;
  return mg::solve_adjoint(prm, a, field, rho, N, grad_field, grad_rho, grad_rho_raw, grad_logfR0, tol, stats,
                           (cudaStream_t)stream);
}
