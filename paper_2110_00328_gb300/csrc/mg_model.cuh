// mg_model.cuh -- device-side model description and the nonlinear
// Gauss-Seidel local solves of the three scalar-field models.
//
// Models (GLAM code units, Sec. 3.1.1), operator N_h at one cell with the
// six-neighbour sum L (Eq. Lijk):
//   f(R)  Eq. fR_eom_codeunit2, w = u^{n+1}:
//         N = -c^2 (L(w) - 6w)/h^2 + Om delta/a + Rb a^2/3 - (Rb a^2/3) ubar / u
//   symmetron  Eq. sym_eom_code_unit:
//         N = c^2 (L(u) - 6u)/h^2 - a^2/(2 xi^2) [(rho a*^3/a^3 - 1) u + u^3]
//   CQ    Eq. csf_eom_code (exp(beta phi/c^2) before (1+delta) optional):
//         N = (L - 6 phi)/h^2 - 3 beta Om e^{beta phibar}/a [E rho - 1]
//             + alpha lambda^2 a^2 [(phibar + phi/c^2)^{-1-alpha} - phibar^{-1-alpha}]
// Local residual d = N - S (S = FAS source, 0 on the finest level).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace mg {

// Kinds: one template instantiation per model (f(R) n is a compile-time constant).
enum Kind { KFR0 = 0, KFR1 = 1, KFR2 = 2, KSYM = 3, KCQ = 4 };

__host__ __device__ constexpr bool is_fr(int K) { return K <= KFR2; }

// Background scalars and model constants, computed on the host in FP64.
struct ModelDev {
  double c2;      // c~^2, c~ = (N_fine/L) c/H0
  double om_a;    // Omega_m / a
  double K0;      // f(R): Rbar(a) a^2 / 3
  double K;       // f(R): K0 * ubar
  double ubar;    // background field
  double msym;    // symmetron: a^2/(2 xi^2)
  double rat3;    // symmetron: (a_star/a)^3
  double xi2_a2;  // symmetron: xi^2/a^2
  double cq_src;  // CQ: 3 beta Om e^{beta phibar}/a
  double cq_pot;  // CQ: alpha lambda^2 a^2
  double alpha;   // CQ
  double phibar;  // CQ
  double beta;    // CQ
  double pot0;    // CQ: phibar^{-1-alpha}
  int keep_exp;   // CQ
  int kind;       // Kind
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <int K, typename T>
__device__ __forceinline__ T fr_w(T u) {
  if constexpr (K == KFR0) return u;
  else if constexpr (K == KFR1) return u * u;
  else return u * u * u;
}

// The field whose Laplacian enters N: w = u^{n+1} for f(R), u itself otherwise.
template <int K, typename T>
__device__ __forceinline__ T fr_or_id(T u) {
  if constexpr (is_fr(K)) return fr_w<K>(u);
  else return u;
}

// ---------------------------------------------------------------------------
// Closed-form local roots (Secs. 3.2.4-3.2.5), rearranged to avoid
// cancellation, followed by Newton polishing on the same polynomial.
// ---------------------------------------------------------------------------

// Positive root of x^3 + p x + q = 0 for q < 0 (Eq. fR_cubic_solns /
// Eq. sym_cubic_solns).  With D = (q/2)^2 + (p/3)^3:
//  D >= 0: Cardano x = A - (p/3)/A with A = cbrt(-q/2 + sqrt D) > 0, evaluated
//          as x = -q / (A^2 + p/3 + (p/(3A))^2) (same value; no subtraction of
//          nearly equal terms when p > 0, where the printed C formula divides 0/0);
//  D < 0:  the trigonometric branch x = 2 sqrt(-p/3) cos(theta/3),
//          cos(theta) = (-q/2) / (-p/3)^{3/2}, the largest (only positive) root.
template <typename T>
__device__ __forceinline__ T cubic_pos_root(T p, T q) {
  const T hq = T(-0.5) * q;
  const T p3 = p * T(1.0 / 3.0);
  const T D = hq * hq + p3 * p3 * p3;
  T x;
  if (D >= T(0)) {
    const T A = cbrt(hq + sqrt(D));
    const T B = p3 / A;
    x = (hq + hq) / (A * A + p3 + B * B);
  } else {
    const T r = sqrt(-p3);
    T c = hq / (r * r * r);
    c = c > T(1) ? T(1) : c;
    x = T(2) * r * cos(acos(c) * T(1.0 / 3.0));
  }
  // Newton polish (x > 0, P'(x) = 3x^2 + p > 0 at the root)
  const T f = (x * x + p) * x + q;
  const T df = T(3) * x * x + p;
  if (df > T(0)) x -= f / df;
  return x;
}

// Positive root of x^2 + p x + q = 0, q < 0 (Eq. fR_quadratic_solns), in the
// cancellation-free form when p > 0.
template <typename T>
__device__ __forceinline__ T quadratic_pos_root(T p, T q) {
  const T s = sqrt(p * p - T(4) * q);
  return p > T(0) ? (T(-2) * q) / (p + s) : T(0.5) * (s - p);
}

// Positive root of x^4 + p x + q = 0, q < 0 (Eq. fR_quartic_solns).
// With Delta0 = 12q < 0, Delta1 = 27 p^2, a = cbrt((sqrt(Delta1^2 - 4 Delta0^3) + Delta1)/2),
// b = |Delta0|/a: 12 S^2 = a - b = Delta1 / (a^2 + ab + b^2) (no cancellation).
// p > 0: x = -S + sqrt(p/(4S) - S^2) (evaluated as a ratio); p < 0:
// x = S + sqrt(-p/(4S) - S^2); p = 0: x = (-q)^{1/4}.  For p > 0 the root is
// also bounded by -q/p, which is the better start when p dominates; two
// Newton steps finish it.
template <typename T>
__device__ __forceinline__ T quartic_pos_root(T p, T q) {
  T x;
  if (p == T(0)) {
    x = sqrt(sqrt(-q));
  } else {
    const T d0 = T(-12) * q;  // |Delta0|
    const T d1 = T(27) * p * p;
    const T a = cbrt(T(0.5) * (sqrt(d1 * d1 + T(4) * d0 * d0 * d0) + d1));
    const T b = d0 / a;
    const T S = sqrt(d1 / (T(12) * (a * a + a * b + b * b)));
    if (p > T(0)) {
      const T r2 = p / (T(4) * S) - S * S;  // > 0 since 8 S^3 < p
      const T rr = sqrt(r2 > T(0) ? r2 : T(0));
      const T num = r2 - S * S;              // (rr - S)(rr + S)
      T xc = num / (rr + S);
      const T xl = -q / p;
      x = (xc > T(0) && xc < xl) ? xc : xl;
    } else {
      const T r2 = -p / (T(4) * S) - S * S;
      x = S + sqrt(r2 > T(0) ? r2 : T(0));
    }
  }
  for (int it = 0; it < 2; ++it) {
    const T x2 = x * x;
    const T f = x2 * x2 + p * x + q;
    const T df = T(4) * x2 * x + p;
    if (df > T(0)) {
      const T xn = x - f / df;
      x = xn > T(0) ? xn : T(0.5) * x;
    }
  }
  return x;
}

// f(R) local root of u^{n+2} + p u + q = 0 (q < 0): the unique positive root.
template <int K, typename T>
__device__ __forceinline__ T fr_root(T p, T q) {
  if constexpr (K == KFR0) return quadratic_pos_root(p, q);
  else if constexpr (K == KFR1) return cubic_pos_root(p, q);
  else return quartic_pos_root(p, q);
}

// Symmetron local root of u^3 + p u + q = 0: the root with sign opposite to q
// (the paper's positive branch for q < 0, mirrored by the cubic's odd symmetry
// for q > 0); for q = 0 the root 0 when p >= 0, else sqrt(-p) with the sign of
// the current value.
template <typename T>
__device__ __forceinline__ T sym_root(T p, T q, T u_old) {
  if (q < T(0)) return cubic_pos_root(p, q);
  if (q > T(0)) return -cubic_pos_root(p, -q);
  if (p >= T(0)) return T(0);
  return u_old < T(0) ? -sqrt(-p) : sqrt(-p);
}

}  // namespace mg
