// background.cu -- the coupled-quintessence background (Sec. 3.2.3,
// "background cosmology solver"): host code, run once per parameter set.
//
// Model (Eqs. csf_coupling_function, csf_potential, csf_param_lambda):
// A(phi) = exp(beta phi), V = Lambda^4 / phi^alpha with Lambda^4 / M_Pl^2 =
// H0^2 lambda^2, phi in units of M_Pl.  In N = ln a, with x = dphi/dN and
// E = H/H0 (cosmic time), the Friedmann constraint, the Raychaudhuri equation
// and the field equation (Eqs. csf_background_Friedmann, _Raychaudhuri, _eom)
// read
//   E^2 (1 - x^2/6) = Or e^{-4N} + e^{beta phi} Om e^{-3N} + (lambda^2/3) phi^{-alpha}
//   dlnH/dN         = -[2 Or e^{-4N} + (3/2) Om e^{-3N} e^{beta phi}] / E^2 - x^2/2
//   dx/dN           = -(3 + dlnH/dN) x + [alpha lambda^2 phi^{-alpha-1}
//                                         - 3 beta Om e^{-3N} e^{beta phi}] / E^2
// (multiplied by a^2 these are the paper's conformal-time code-unit forms,
// Eq. csf_background_eom_codeunit, whose potential amplitude is lambda^2/3).
// Radiation: CMB photons at 2.7255 K and 3.046 massless neutrino species.
//
// The system is integrated from z = 1e5 (phi = 1e-4, x = 0: any small start
// relaxes onto the same solution) with the adaptive Dormand-Prince 5(4)
// Runge-Kutta pair (the paper uses a fifth-sixth order continuous Runge-Kutta
// integrator), and lambda is found by shooting as in the paper: the predicted
// H(a=1) must equal H0; E(1) grows with lambda, so the root is bracketed and
// refined by safeguarded secant steps.
#include <math.h>
#include <string.h>

#include "../../include/mgglam.h"

namespace {

struct Cosmo {
  double alpha, beta, om, orad, lam2;
};

double E2_of(const Cosmo& c, double N, double phi, double x) {
  return (c.orad * exp(-4.0 * N) + exp(c.beta * phi) * c.om * exp(-3.0 * N) + c.lam2 / 3.0 * pow(phi, -c.alpha)) /
         (1.0 - x * x / 6.0);
}

void rhs(const Cosmo& c, double N, const double y[2], double dy[2]) {
  const double phi = y[0], x = y[1];
  const double E2 = E2_of(c, N, phi, x);
  const double em = exp(-3.0 * N) * exp(c.beta * phi);
  const double dlnH = -(2.0 * c.orad * exp(-4.0 * N) + 1.5 * c.om * em) / E2 - 0.5 * x * x;
  dy[0] = x;
  dy[1] = -(3.0 + dlnH) * x + (c.alpha * c.lam2 * pow(phi, -c.alpha - 1.0) - 3.0 * c.beta * c.om * em) / E2;
}

// Dormand-Prince 5(4) tableau
constexpr double C2 = 1.0 / 5, C3 = 3.0 / 10, C4 = 4.0 / 5, C5 = 8.0 / 9;
constexpr double A21 = 1.0 / 5;
constexpr double A31 = 3.0 / 40, A32 = 9.0 / 40;
constexpr double A41 = 44.0 / 45, A42 = -56.0 / 15, A43 = 32.0 / 9;
constexpr double A51 = 19372.0 / 6561, A52 = -25360.0 / 2187, A53 = 64448.0 / 6561, A54 = -212.0 / 729;
constexpr double A61 = 9017.0 / 3168, A62 = -355.0 / 33, A63 = 46732.0 / 5247, A64 = 49.0 / 176,
                 A65 = -5103.0 / 18656;
constexpr double B1 = 35.0 / 384, B3 = 500.0 / 1113, B4 = 125.0 / 192, B5 = -2187.0 / 6784, B6 = 11.0 / 84;
constexpr double E1 = 5179.0 / 57600, E3 = 7571.0 / 16695, E4 = 393.0 / 640, E5 = -92097.0 / 339200,
                 E6 = 187.0 / 2100, E7 = 1.0 / 40;

// Integrate y from N0 to N1 (N1 > N0); returns false if the step size collapses.
bool integrate(const Cosmo& c, double N0, double N1, double y[2]) {
  const double rtol = 1e-12, atol = 1e-15;
  double N = N0, h = 1e-3;
  double k1[2], k2[2], k3[2], k4[2], k5[2], k6[2], k7[2], t[2], y5[2];
  rhs(c, N, y, k1);
  for (int guard = 0; guard < 2000000 && N < N1; ++guard) {
    if (N + h > N1) h = N1 - N;
    for (int i = 0; i < 2; ++i) t[i] = y[i] + h * A21 * k1[i];
    rhs(c, N + C2 * h, t, k2);
    for (int i = 0; i < 2; ++i) t[i] = y[i] + h * (A31 * k1[i] + A32 * k2[i]);
    rhs(c, N + C3 * h, t, k3);
    for (int i = 0; i < 2; ++i) t[i] = y[i] + h * (A41 * k1[i] + A42 * k2[i] + A43 * k3[i]);
    rhs(c, N + C4 * h, t, k4);
    for (int i = 0; i < 2; ++i) t[i] = y[i] + h * (A51 * k1[i] + A52 * k2[i] + A53 * k3[i] + A54 * k4[i]);
    rhs(c, N + C5 * h, t, k5);
    for (int i = 0; i < 2; ++i)
      t[i] = y[i] + h * (A61 * k1[i] + A62 * k2[i] + A63 * k3[i] + A64 * k4[i] + A65 * k5[i]);
    rhs(c, N + h, t, k6);
    for (int i = 0; i < 2; ++i) y5[i] = y[i] + h * (B1 * k1[i] + B3 * k3[i] + B4 * k4[i] + B5 * k5[i] + B6 * k6[i]);
    rhs(c, N + h, y5, k7);
    double err = 0.0;
    for (int i = 0; i < 2; ++i) {
      const double y4 = y[i] + h * (E1 * k1[i] + E3 * k3[i] + E4 * k4[i] + E5 * k5[i] + E6 * k6[i] + E7 * k7[i]);
      const double sc = atol + rtol * fmax(fabs(y[i]), fabs(y5[i]));
      err = fmax(err, fabs(y5[i] - y4) / sc);
    }
    if (!(err == err)) return false;  // NaN
    if (err <= 1.0) {
      N += h;
      y[0] = y5[0];
      y[1] = y5[1];
      k1[0] = k7[0];  // first-same-as-last
      k1[1] = k7[1];
    }
    const double fac = err > 0.0 ? 0.9 * pow(err, -0.2) : 5.0;
    h *= fmin(5.0, fmax(0.2, fac));
    if (h < 1e-14) return false;
  }
  return N >= N1;
}

constexpr double kZInit = 1e5, kPhiInit = 1e-4;

// E(a=1) - 1 for lambda; false if the integration failed
bool mismatch(Cosmo& c, double lam, double* f) {
  c.lam2 = lam * lam;
  double y[2] = {kPhiInit, 0.0};
  if (!integrate(c, -log1p(kZInit), 0.0, y)) return false;
  *f = sqrt(E2_of(c, 0.0, y[0], y[1])) - 1.0;
  return true;
}

}  // namespace

extern "C" double mgglam_radiation_density(double h) {
  // Omega_r = rho_gamma / rho_crit * (1 + N_eff (7/8)(4/11)^{4/3}), rho_gamma = 4 sigma T^4 / c^3
  const double sigma_sb = 5.670374419e-8, c = 299792458.0, G = 6.67430e-11, mpc = 3.0856775814913673e22;
  const double T = 2.7255, Neff = 3.046;
  const double H0 = 100.0 * h * 1e3 / mpc;
  const double rho_gamma = 4.0 * sigma_sb / (c * c * c) * T * T * T * T;
  const double rho_crit = 3.0 * H0 * H0 / (8.0 * M_PI * G);
  return rho_gamma / rho_crit * (1.0 + Neff * 7.0 / 8.0 * pow(4.0 / 11.0, 4.0 / 3.0));
}

extern "C" int mgglam_cq_background(double alpha, double beta, double omega_m, double h, double a, double* lambda,
                                    double* phibar, double* dphibar_dlna, double* E) {
  if (!lambda || !phibar || !dphibar_dlna || !E) return MGGLAM_ERR_ARG;
  if (!(alpha > 0.0) || !(omega_m > 0.0 && omega_m < 1.0) || !(h > 0.0) || !(a > 0.0 && a <= 1.0) ||
      !(beta == beta))
    return MGGLAM_ERR_ARG;
  Cosmo c = {alpha, beta, omega_m, mgglam_radiation_density(h), 0.0};
  // bracket: E(1) increases with lambda
  double lo = 1.0, hi = 1.0, flo, fhi;
  if (!mismatch(c, lo, &flo)) return MGGLAM_ERR_NONFINITE;
  fhi = flo;
  for (int k = 0; flo > 0.0 && k < 60; ++k) {
    hi = lo;
    fhi = flo;
    lo *= 0.5;
    if (!mismatch(c, lo, &flo)) return MGGLAM_ERR_NONFINITE;
  }
  for (int k = 0; fhi < 0.0 && k < 60; ++k) {
    lo = hi;
    flo = fhi;
    hi *= 2.0;
    if (!mismatch(c, hi, &fhi)) return MGGLAM_ERR_NONFINITE;
  }
  if (!(flo <= 0.0 && fhi >= 0.0)) return MGGLAM_ERR_NOT_CONVERGED;
  // safeguarded secant (regula falsi with the Illinois halving)
  double lam = lo;
  int side = 0;
  for (int it = 0; it < 200 && hi - lo > 1e-13 * hi; ++it) {
    lam = (lo * fhi - hi * flo) / (fhi - flo);
    if (!(lam > lo && lam < hi)) lam = 0.5 * (lo + hi);
    double f;
    if (!mismatch(c, lam, &f)) return MGGLAM_ERR_NONFINITE;
    if (fabs(f) < 1e-15) break;
    if (f > 0.0) {
      hi = lam;
      fhi = f;
      if (side == 1) flo *= 0.5;
      side = 1;
    } else {
      lo = lam;
      flo = f;
      if (side == -1) fhi *= 0.5;
      side = -1;
    }
  }
  c.lam2 = lam * lam;
  double y[2] = {kPhiInit, 0.0};
  const double Na = log(a);
  if (Na > -log1p(kZInit) && !integrate(c, -log1p(kZInit), Na, y)) return MGGLAM_ERR_NONFINITE;
  *lambda = lam;
  *phibar = y[0];
  *dphibar_dlna = y[1];
  *E = sqrt(E2_of(c, Na, y[0], y[1]));
  return MGGLAM_OK;
}
