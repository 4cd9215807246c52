/*
 * mgoracle.c -- plain, slow FP64 CPU reference ("oracle") for the MG-GLAM
 * scalar-field solve (arXiv:2110.00328).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path: every formula below is written
 * out again from the paper.
 *
 * What it computes
 * ----------------
 *  - Background scalars in GLAM code units (Sec. 3.1.1, Eqs. code_units,
 *    code_units2; f(R): Eq. R_bar, Eq. fR_HS; symmetron: Eq. varphi_min_symm).
 *  - The discrete operator N_h(u) of each model, cell by cell, with
 *    L_ijk = sum of the six face neighbours (Eq. Lijk) on a periodic mesh:
 *      f(R)      Eq. fR_eom_codeunit2 with w = u^{n+1}:
 *                N = -c^2 (L(w) - 6w)/h^2 + Om delta/a + Rb a^2/3 - (Rb a^2/3) ubar/u
 *      symmetron Eq. sym_eom_code_unit:
 *                N = c^2 (L(u) - 6u)/h^2 - a^2/(2 xi^2) [ (rho a*^3/a^3 - 1) u + u^3 ]
 *      CQ        Eq. csf_eom_code (the exp(beta phi/c^2) factor in front of
 *                (1+delta) dropped as in Sec. 3.2.3 unless keep_exp is set):
 *                N = (L(phi) - 6 phi)/h^2 - 3 beta Om e^{beta phibar}/a [E (1+delta) - 1]
 *                    + alpha lambda^2 a^2 [ (phibar + phi/c^2)^{-1-alpha} - phibar^{-1-alpha} ]
 *    The local residual is d = N(u) - S (Eq. residual_d with f^h = S, S = 0 on
 *    the finest mesh) and the global residual is its root-mean-square.
 *  - Red-black ("black first, then red") Gauss-Seidel sweeps (Sec. 3.2.1).
 *    kind 0 = nonlinear Gauss-Seidel: each cell's local equation is solved
 *    exactly for that cell given its neighbours (Secs. 3.2.4, 3.2.5); the
 *    unique admissible root is found here by safeguarded Newton-bisection, not
 *    by the closed forms.  kind 1 = Newton-Gauss-Seidel: one step of
 *    Eq. relaxation_iteration per cell (Sec. 3.2.1; the paper's CQ method).
 *  - Optionally a full-multigrid start (fmg_start): the coarse problems first,
 *    each level starting from the prolonged coarser solution.
 *  - FAS multigrid V-cycles (Sec. 3.2.1): restriction = mean of the 8 children,
 *    coarse equation Eq. general_pde_numerical_coarse, coarse initial guess =
 *    restricted fine solution, correction Eq. solution_correction with the
 *    27/9/3/1 (/64) trilinear prolongation.
 *  - CIC mass assignment and the three-point-difference force interpolated back
 *    to particles with the same CIC weights (Sec. 3.1).
 *
 * Readings taken where the paper leaves a point open:
 *  black cells are those with (i+j+k) even (0-based); the coarsest level is
 *  relaxed with a fixed number of sweeps; for f(R) a cell whose value is not
 *  positive after the coarse-grid correction is set to half its value before
 *  the correction; for the symmetron the admissible root is the one with the
 *  sign opposite to q (the paper's positive branch when q < 0).
 *
 * Layout: a level-n mesh is a contiguous array of n^3 doubles indexed
 * (i*n + j)*n + k, k fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_FR 0
#define OR_SYMMETRON 1
#define OR_CQ 2

/* Model and numerical parameters (code units; box in Mpc/h). */
typedef struct {
  int model;
  int n;            /* f(R) Hu-Sawicki index n = 0, 1, 2 */
  int keep_exp;     /* CQ: keep exp(beta phi / c^2) in front of (1+delta) */
  int pad0;
  double fR0_abs, omega_m, omega_l, box;
  double a_star, xi, beta_star;
  double alpha, beta, lambda, phibar;
  double a;
} or_params;

/* Background scalars derived from or_params at scale factor a. */
typedef struct {
  double ctilde;    /* c~ = (N_g / (H0 L)) c, Sec. 3.1.1 */
  double c2;        /* c~^2 */
  double Rbar;      /* R~bar(a) = 3 (Om a^-3 + 4 OL), Sec. 3.2.5 */
  double fRbar;     /* fbar_R(a) = -|fR0| (Rbar(1)/Rbar(a))^{n+1}, Eq. fR_HS */
  double ubar;      /* background field: f(R) (-fbar_R)^{1/(n+1)}; symmetron sqrt(1-(a_star/a)^3) */
  double K0;        /* f(R): Rbar a^2 / 3 */
  double K;         /* f(R): K0 * ubar */
  double msym;      /* symmetron: a^2 / (2 xi^2) */
  double cq_src;    /* CQ: 3 beta Om e^{beta phibar} / a */
  double cq_pot;    /* CQ: alpha lambda^2 a^2 */
} or_background;

/* Speed of light over H0 in Mpc/h: c / (100 km/s/Mpc). */
static const double OR_C_OVER_H0_MPCH = 299792.458 / 100.0;

void or_compute_background(const or_params* p, int N, or_background* b) {
  double a = p->a;
  memset(b, 0, sizeof(*b));
  b->ctilde = ((double)N / p->box) * OR_C_OVER_H0_MPCH;
  b->c2 = b->ctilde * b->ctilde;
  if (p->model == OR_FR) {
    double Rbar_a = 3.0 * (p->omega_m / (a * a * a) + 4.0 * p->omega_l);
    double Rbar_1 = 3.0 * (p->omega_m + 4.0 * p->omega_l);
    b->Rbar = Rbar_a;
    b->fRbar = -p->fR0_abs * pow(Rbar_1 / Rbar_a, (double)(p->n + 1));
    b->ubar = pow(-b->fRbar, 1.0 / (double)(p->n + 1));
    b->K0 = Rbar_a * a * a / 3.0;
    b->K = b->K0 * b->ubar;
  } else if (p->model == OR_SYMMETRON) {
    double r = p->a_star / a;
    double s = 1.0 - r * r * r;
    b->ubar = s > 0.0 ? sqrt(s) : 0.0;
    b->msym = a * a / (2.0 * p->xi * p->xi);
  } else {
    b->ubar = 0.0;
    b->cq_src = 3.0 * p->beta * p->omega_m * exp(p->beta * p->phibar) / a;
    b->cq_pot = p->alpha * p->lambda * p->lambda * a * a;
  }
}

static inline size_t IDX(int n, int i, int j, int k) {
  return ((size_t)i * n + j) * n + k;
}
static inline int WRAP(int i, int n) { return (i + n) % n; }

/* Sum of the six face neighbours of cell (i,j,k) of field f (Eq. Lijk). */
static double neighbour_sum(const double* f, int n, int i, int j, int k) {
  return f[IDX(n, WRAP(i + 1, n), j, k)] + f[IDX(n, WRAP(i - 1, n), j, k)] +
         f[IDX(n, i, WRAP(j + 1, n), k)] + f[IDX(n, i, WRAP(j - 1, n), k)] +
         f[IDX(n, i, j, WRAP(k + 1, n))] + f[IDX(n, i, j, WRAP(k - 1, n))];
}

/* The transform whose Laplacian appears in N: f(R) w = u^{n+1}; else the field itself. */
static inline double field_w(const or_params* p, double u) {
  if (p->model == OR_FR) {
    double w = u;
    for (int m = 0; m < p->n; ++m) w *= u;
    return w;
  }
  return u;
}

/*
 * Local operator at one cell, given its own value u, its density rho (mean 1),
 * and Lnb = sum of the neighbours of the transformed field w (f(R)) or of u.
 */
static double local_N(const or_params* p, const or_background* b, double h, double u,
                      double rho, double Lnb) {
  double a = p->a, delta = rho - 1.0, ih2 = 1.0 / (h * h);
  if (p->model == OR_FR) {
    double w = field_w(p, u);
    return -b->c2 * (Lnb - 6.0 * w) * ih2 + p->omega_m * delta / a + b->K0 - b->K / u;
  } else if (p->model == OR_SYMMETRON) {
    double a3 = a * a * a, as3 = p->a_star * p->a_star * p->a_star;
    return b->c2 * (Lnb - 6.0 * u) * ih2 - b->msym * ((rho * as3 / a3 - 1.0) * u + u * u * u);
  } else {
    double E = p->keep_exp ? exp(p->beta * u / b->c2) : 1.0;
    double x = p->phibar + u / b->c2;
    return (Lnb - 6.0 * u) * ih2 - b->cq_src * (E * rho - 1.0) +
           b->cq_pot * (pow(x, -1.0 - p->alpha) - pow(p->phibar, -1.0 - p->alpha));
  }
}

/* d(local_N)/du at fixed neighbours (the denominator of Eq. relaxation_iteration). */
static double local_dN(const or_params* p, const or_background* b, double h, double u,
                       double rho) {
  double a = p->a, ih2 = 1.0 / (h * h);
  if (p->model == OR_FR) {
    double dw = (double)(p->n + 1);
    for (int m = 0; m < p->n; ++m) dw *= u;
    return 6.0 * b->c2 * dw * ih2 + b->K / (u * u);
  } else if (p->model == OR_SYMMETRON) {
    double a3 = a * a * a, as3 = p->a_star * p->a_star * p->a_star;
    return -6.0 * b->c2 * ih2 - b->msym * ((rho * as3 / a3 - 1.0) + 3.0 * u * u);
  } else {
    double dE = p->keep_exp ? (p->beta / b->c2) * exp(p->beta * u / b->c2) : 0.0;
    double x = p->phibar + u / b->c2;
    return -6.0 * ih2 - b->cq_src * dE * rho +
           b->cq_pot * (-1.0 - p->alpha) * pow(x, -2.0 - p->alpha) / b->c2;
  }
}

/*
 * The local polynomial of the nonlinear Gauss-Seidel update, P(u) = 0.
 *  f(R) (Eq. fR_eom_codeunit): u^{n+2} + p u + q with
 *    p = h^2/(6c^2) [Om delta/a + Rb a^2/3 - S] - Lnb/6,   q = -h^2/(6c^2) K
 *  symmetron (Eq. sym_cubic_eqn): u^3 + p u + q with
 *    p = rho a*^3/a^3 - 1 + 12 c^2 xi^2/(h^2 a^2),  q = -2 c^2 xi^2 Lnb/(h^2 a^2) + (2 xi^2/a^2) S
 * The S terms are the coarse-level FAS source carried into the same polynomial.
 */
static void local_pq(const or_params* p, const or_background* b, double h, double rho,
                     double Lnb, double S, double* pp, double* qq) {
  double a = p->a;
  if (p->model == OR_FR) {
    double al = h * h / (6.0 * b->c2);
    *pp = al * (p->omega_m * (rho - 1.0) / a + b->K0 - S) - Lnb / 6.0;
    *qq = -al * b->K;
  } else {
    double a3 = a * a * a, as3 = p->a_star * p->a_star * p->a_star;
    double g = b->c2 * p->xi * p->xi / (h * h * a * a);
    *pp = rho * as3 / a3 - 1.0 + 12.0 * g;
    *qq = -2.0 * g * Lnb + (2.0 * p->xi * p->xi / (a * a)) * S;
  }
}

static inline double poly(int deg, double p, double q, double u) {
  double v = u;
  for (int m = 1; m < deg; ++m) v *= u;
  return v + p * u + q;
}
static inline double dpoly(int deg, double p, double u) {
  double v = (double)deg;
  for (int m = 1; m < deg; ++m) v *= u;
  return v + p;
}

/*
 * Root of u^deg + p u + q on the positive half-line, given q < 0.  P(0) = q < 0
 * and P -> +inf, and P has exactly one positive zero (for p >= 0 P is increasing;
 * for p < 0 it first decreases from q then increases).  Safeguarded Newton
 * inside a bracket [lo, hi] with P(lo) < 0 < P(hi), halving when a Newton step
 * leaves the bracket; stops when the bracket is one ulp wide.
 */
static double positive_root(int deg, double p, double q, double guess) {
  double lo = 0.0, hi = guess > 0.0 ? guess : 1.0;
  int it;
  for (it = 0; it < 2100 && poly(deg, p, q, hi) <= 0.0; ++it) { lo = hi; hi *= 2.0; }
  double x = 0.5 * (lo + hi);
  for (it = 0; it < 400; ++it) {
    double f = poly(deg, p, q, x);
    if (f == 0.0) return x;
    if (f < 0.0) lo = x; else hi = x;
    double df = dpoly(deg, p, x);
    double xn = (df > 0.0) ? x - f / df : 0.5 * (lo + hi);
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (xn == x || hi - lo <= 2.0 * 2.2204460492503131e-16 * hi) {
      x = xn;
      break;
    }
    x = xn;
  }
  return x;
}

/* Nonlinear Gauss-Seidel local solve: the admissible root of P(u) = 0. */
static double local_root(const or_params* p, double pp, double qq, double u_old) {
  int deg = (p->model == OR_FR) ? p->n + 2 : 3;
  if (qq < 0.0) return positive_root(deg, pp, qq, fabs(u_old));
  if (qq > 0.0) return -positive_root(deg, pp, -qq, fabs(u_old)); /* odd cubic mirror (symmetron) */
  if (pp >= 0.0) return 0.0;
  return (u_old < 0.0) ? -sqrt(-pp) : sqrt(-pp);
}

/* Residual d = N(u) - S on an n^3 level of spacing h; returns sum of d^2. */
double or_residual(const or_params* p, const or_background* b, int n, double h,
                   const double* u, const double* rho, const double* S, double* d) {
  size_t n3 = (size_t)n * n * n;
  double* w = (double*)malloc(n3 * sizeof(double));
  for (size_t c = 0; c < n3; ++c) w[c] = field_w(p, u[c]);
  double ss = 0.0;
#pragma omp parallel for reduction(+ : ss) schedule(static)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        size_t c = IDX(n, i, j, k);
        double r = local_N(p, b, h, u[c], rho[c], neighbour_sum(w, n, i, j, k)) - (S ? S[c] : 0.0);
        if (d) d[c] = r;
        ss += r * r;
      }
  free(w);
  return ss;
}

/* Relax the cells of one colour (parity = (i+j+k) % 2) in place. */
static void relax_colour(const or_params* p, const or_background* b, int n, double h,
                         double* u, const double* rho, const double* S, int parity, int kind) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        if (((i + j + k) & 1) != parity) continue;
        size_t c = IDX(n, i, j, k);
        double Lnb;
        if (p->model == OR_FR) {
          /* neighbours of w = u^{n+1}, transformed on the fly */
          Lnb = field_w(p, u[IDX(n, WRAP(i + 1, n), j, k)]) + field_w(p, u[IDX(n, WRAP(i - 1, n), j, k)]) +
                field_w(p, u[IDX(n, i, WRAP(j + 1, n), k)]) + field_w(p, u[IDX(n, i, WRAP(j - 1, n), k)]) +
                field_w(p, u[IDX(n, i, j, WRAP(k + 1, n))]) + field_w(p, u[IDX(n, i, j, WRAP(k - 1, n))]);
        } else {
          Lnb = neighbour_sum(u, n, i, j, k);
        }
        double s = S ? S[c] : 0.0;
        if (kind == 0 && p->model != OR_CQ) {
          double pp, qq;
          local_pq(p, b, h, rho[c], Lnb, s, &pp, &qq);
          u[c] = local_root(p, pp, qq, u[c]);
        } else {
          double r = local_N(p, b, h, u[c], rho[c], Lnb) - s;
          u[c] = u[c] - r / local_dN(p, b, h, u[c], rho[c]);
        }
      }
}

/* 'sweeps' red-black sweeps: black ((i+j+k) even) first, then red. */
void or_smooth(const or_params* p, const or_background* b, int n, double h, double* u,
               const double* rho, const double* S, int sweeps, int kind) {
  for (int s = 0; s < sweeps; ++s) {
    relax_colour(p, b, n, h, u, rho, S, 0, kind);
    relax_colour(p, b, n, h, u, rho, S, 1, kind);
  }
}

/* Restriction: coarse cell = arithmetic mean of its 8 fine children (Sec. 3.2.1). */
void or_restrict(int nf, const double* fine, double* coarse) {
  int nc = nf / 2;
  for (int I = 0; I < nc; ++I)
    for (int J = 0; J < nc; ++J)
      for (int K = 0; K < nc; ++K) {
        double s = 0.0;
        for (int di = 0; di < 2; ++di)
          for (int dj = 0; dj < 2; ++dj)
            for (int dk = 0; dk < 2; ++dk) s += fine[IDX(nf, 2 * I + di, 2 * J + dj, 2 * K + dk)];
        coarse[IDX(nc, I, J, K)] = s / 8.0;
      }
}

/*
 * Prolongation of a coarse field to one fine cell (Sec. 3.2.1): the parent has
 * weight 27/64, each of the 3 face neighbours 9/64, each of the 3 edge
 * neighbours 3/64 and the vertex neighbour 1/64, the neighbours being on the
 * side of the parent towards which the fine cell lies.
 */
static double prolong_at(int nc, const double* c, int i, int j, int k) {
  int I = i / 2, J = j / 2, K = k / 2;
  int si = (i & 1) ? 1 : -1, sj = (j & 1) ? 1 : -1, sk = (k & 1) ? 1 : -1;
  int I2 = WRAP(I + si, nc), J2 = WRAP(J + sj, nc), K2 = WRAP(K + sk, nc);
  double v = 27.0 * c[IDX(nc, I, J, K)] +
             9.0 * (c[IDX(nc, I2, J, K)] + c[IDX(nc, I, J2, K)] + c[IDX(nc, I, J, K2)]) +
             3.0 * (c[IDX(nc, I2, J2, K)] + c[IDX(nc, I2, J, K2)] + c[IDX(nc, I, J2, K2)]) +
             1.0 * c[IDX(nc, I2, J2, K2)];
  return v / 64.0;
}

/* Plain prolongation of a coarse field into an nf^3 fine field (for tests). */
void or_prolong(int nc, const double* coarse, double* fine) {
  int nf = 2 * nc;
  for (int i = 0; i < nf; ++i)
    for (int j = 0; j < nf; ++j)
      for (int k = 0; k < nf; ++k) fine[IDX(nf, i, j, k)] = prolong_at(nc, coarse, i, j, k);
}

/*
 * Coarse-grid correction, Eq. solution_correction: u^h += P(u^H - R u^h).
 * f(R) positivity reading: a fine value that is not positive afterwards is
 * replaced by half its value before the correction.  Returns the number of
 * such replacements.
 */
long or_prolong_correct(const or_params* p, int nc, const double* uH, const double* RuH, double* uh) {
  size_t nc3 = (size_t)nc * nc * nc;
  double* e = (double*)malloc(nc3 * sizeof(double));
  for (size_t c = 0; c < nc3; ++c) e[c] = uH[c] - RuH[c];
  int nf = 2 * nc;
  long guarded = 0;
  for (int i = 0; i < nf; ++i)
    for (int j = 0; j < nf; ++j)
      for (int k = 0; k < nf; ++k) {
        size_t c = IDX(nf, i, j, k);
        double old = uh[c];
        double v = old + prolong_at(nc, e, i, j, k);
        if (p->model == OR_FR && !(v > 0.0)) {
          v = 0.5 * old;
          ++guarded;
        }
        uh[c] = v;
      }
  free(e);
  return guarded;
}

/* ---------------------------------------------------------------------- */
/* FAS V-cycle solver                                                       */
/* ---------------------------------------------------------------------- */

typedef struct {
  int nlev;
  int n[32];
  double h[32];
  double *u[32], *rho[32], *S[32], *Ru[32], *d[32];
} or_hier;

typedef struct {
  int nu1, nu2, coarse_sweeps, kind, levels;
} or_cycle_opts;

/* One multigrid cycle from level l (Sec. 3.2.1, Fig. multigrid_cycles): the
 * coarse-grid correction of level l calls the cycle of level l+1 once
 * (mode 0, V-cycle), twice as W-cycles (mode 2, W-cycle), or once as an
 * F-cycle and then once as a V-cycle (mode 1, F-cycle).  The second call
 * continues from the coarse solution the first one left, with the same
 * coarse source. */
static void vcycle(const or_params* p, const or_background* b, or_hier* H, int l,
                   const or_cycle_opts* o, long* guarded, int mode) {
  int n = H->n[l];
  double h = H->h[l];
  if (l == H->nlev - 1) {
    or_smooth(p, b, n, h, H->u[l], H->rho[l], H->S[l], o->coarse_sweeps, o->kind);
    return;
  }
  or_smooth(p, b, n, h, H->u[l], H->rho[l], H->S[l], o->nu1, o->kind);
  /* fine residual d^l, restricted solution and residual */
  or_residual(p, b, n, h, H->u[l], H->rho[l], H->S[l], H->d[l]);
  int nc = H->n[l + 1];
  size_t nc3 = (size_t)nc * nc * nc;
  double* Rd = (double*)malloc(nc3 * sizeof(double));
  or_restrict(n, H->u[l], H->Ru[l + 1]);
  or_restrict(n, H->d[l], Rd);
  /* coarse source S^H = N^H(R u^h) - R d^h (Eq. general_pde_numerical_coarse) */
  or_residual(p, b, nc, H->h[l + 1], H->Ru[l + 1], H->rho[l + 1], NULL, H->S[l + 1]);
  for (size_t c = 0; c < nc3; ++c) H->S[l + 1][c] -= Rd[c];
  free(Rd);
  /* coarse initial guess = R u^h */
  memcpy(H->u[l + 1], H->Ru[l + 1], nc3 * sizeof(double));
  vcycle(p, b, H, l + 1, o, guarded, mode);
  if (mode == 2) vcycle(p, b, H, l + 1, o, guarded, 2);
  if (mode == 1) vcycle(p, b, H, l + 1, o, guarded, 0);
  *guarded += or_prolong_correct(p, nc, H->u[l + 1], H->Ru[l + 1], H->u[l]);
  or_smooth(p, b, n, h, H->u[l], H->rho[l], H->S[l], o->nu2, o->kind);
}

/*
 * Full-multigrid start (the nested-iteration use of the same FAS cycles,
 * Sec. 3.2.1): the problem is posed on every level (the density restricted by
 * 8-child means, no FAS source: N^H(u^H) = 0), relaxed on the coarsest level
 * from the background value, and each finer level starts from the plain
 * 27/9/3/1 prolongation of the coarser level's result and takes one cycle.
 * On return level 0 holds the FMG iterate.
 */
static void fmg_start(const or_params* p, const or_background* b, or_hier* H, const or_cycle_opts* o,
                      long* guarded) {
  const int L = H->nlev;
  const size_t nL3 = (size_t)H->n[L - 1] * H->n[L - 1] * H->n[L - 1];
  for (size_t c = 0; c < nL3; ++c) H->u[L - 1][c] = b->ubar;
  if (L - 1 > 0) memset(H->S[L - 1], 0, nL3 * sizeof(double));
  or_smooth(p, b, H->n[L - 1], H->h[L - 1], H->u[L - 1], H->rho[L - 1], H->S[L - 1], o->coarse_sweeps, o->kind);
  for (int l = L - 2; l >= 0; --l) {
    const size_t n3 = (size_t)H->n[l] * H->n[l] * H->n[l];
    or_prolong(H->n[l + 1], H->u[l + 1], H->u[l]);
    if (l > 0) memset(H->S[l], 0, n3 * sizeof(double));
    vcycle(p, b, H, l, o, guarded, 0);
  }
}

/* Source scale used to make the global residual relative (reading C5). */
static double source_rms(const or_params* p, const or_background* b, int N, const double* rho) {
  size_t n3 = (size_t)N * N * N;
  double ss = 0.0;
  for (size_t c = 0; c < n3; ++c) {
    double delta = rho[c] - 1.0, s;
    if (p->model == OR_FR) s = p->omega_m * delta / p->a;
    else if (p->model == OR_SYMMETRON) {
      double r = p->a_star / p->a;
      s = b->msym * r * r * r * delta * b->ubar;
    } else s = b->cq_src * delta;
    ss += s * s;
  }
  double r = sqrt(ss / (double)n3);
  return r > 0.0 ? r : 1.0;
}

/* Number of levels: halve while the mesh stays even and above 4 cells (or 'levels' if > 0). */
static int count_levels(int N, int levels) {
  int nl = 1, n = N;
  if (levels > 0) {
    for (int l = 1; l < levels; ++l) {
      if (n % 2 != 0 || n / 2 < 2) break;
      n /= 2;
      ++nl;
    }
    return nl;
  }
  while (n % 2 == 0 && n / 2 >= 4 && (n / 2) % 2 == 0) { n /= 2; ++nl; }
  return nl;
}

/*
 * Solve N_h(u; rho) = 0 on the periodic N^3 mesh (h = 1) by FAS V-cycles.
 * rho: input density (any positive mean; normalised here to mean 1 in FP64).
 * u:   in: initial guess (if u[0] is NaN the background value is used); out: solution.
 * hist[0..max_cycles]: relative global residual before each cycle and at the end.
 * Returns the number of V-cycles run; *eps_out = final relative residual.
 */
int or_solve_cycle(const or_params* p, int N, const double* rho_in, double* u, double tol,
                   int max_cycles, int nu1, int nu2, int coarse_sweeps, int kind, int levels, int cycle,
                   int fmg, double* hist, double* eps_out, long* guarded_out) {
  or_background b;
  or_compute_background(p, N, &b);
  or_hier H;
  memset(&H, 0, sizeof(H));
  H.nlev = count_levels(N, levels);
  for (int l = 0, n = N; l < H.nlev; ++l, n /= 2) {
    size_t n3 = (size_t)n * n * n;
    H.n[l] = n;
    H.h[l] = (double)(1 << l);
    H.u[l] = (l == 0) ? u : (double*)calloc(n3, sizeof(double));
    H.rho[l] = (double*)malloc(n3 * sizeof(double));
    H.S[l] = (l == 0) ? NULL : (double*)calloc(n3, sizeof(double));
    H.Ru[l] = (double*)calloc(n3, sizeof(double));
    H.d[l] = (double*)calloc(n3, sizeof(double));
  }
  /* density normalised to mean 1 (reading C12), then restricted down the levels */
  size_t N3 = (size_t)N * N * N;
  double mean = 0.0;
  for (size_t c = 0; c < N3; ++c) mean += rho_in[c];
  mean /= (double)N3;
  for (size_t c = 0; c < N3; ++c) H.rho[0][c] = rho_in[c] / mean;
  for (int l = 1; l < H.nlev; ++l) or_restrict(H.n[l - 1], H.rho[l - 1], H.rho[l]);
  if (isnan(u[0]))
    for (size_t c = 0; c < N3; ++c) u[c] = b.ubar;

  or_cycle_opts o = {nu1, nu2, coarse_sweeps, kind, levels};
  double snorm = source_rms(p, &b, N, H.rho[0]);
  long guarded = 0;
  int cyc = 0;
  double eps = sqrt(or_residual(p, &b, N, 1.0, u, H.rho[0], NULL, NULL) / (double)N3) / snorm;
  if (hist) hist[0] = eps;
  while (cyc < max_cycles && !(eps <= tol)) {
    /* fmg: the first cycle is the full-multigrid start (it ends with one cycle on level 0) */
    if (fmg && cyc == 0) fmg_start(p, &b, &H, &o, &guarded);
    else vcycle(p, &b, &H, 0, &o, &guarded, cycle);
    ++cyc;
    eps = sqrt(or_residual(p, &b, N, 1.0, u, H.rho[0], NULL, NULL) / (double)N3) / snorm;
    if (hist) hist[cyc] = eps;
  }
  for (int l = 0; l < H.nlev; ++l) {
    if (l > 0) { free(H.u[l]); free(H.S[l]); }
    free(H.rho[l]); free(H.Ru[l]); free(H.d[l]);
  }
  if (eps_out) *eps_out = eps;
  if (guarded_out) *guarded_out = guarded;
  return cyc;
}

int or_solve(const or_params* p, int N, const double* rho_in, double* u, double tol,
             int max_cycles, int nu1, int nu2, int coarse_sweeps, int kind, int levels,
             double* hist, double* eps_out, long* guarded_out) {
  return or_solve_cycle(p, N, rho_in, u, tol, max_cycles, nu1, nu2, coarse_sweeps, kind, levels, 0, 0, hist,
                        eps_out, guarded_out);
}

/* Relative-residual normaliser, exposed so tests can form the same ratio. */
double or_source_rms(const or_params* p, int N, const double* rho) {
  or_background b;
  or_compute_background(p, N, &b);
  return source_rms(p, &b, N, rho);
}

/* ---------------------------------------------------------------------- */
/* Cloud-in-cell (Sec. 3.1)                                                 */
/* ---------------------------------------------------------------------- */

/*
 * CIC mass assignment: cell c spans [c, c+1) with centre c + 1/2.  A particle
 * at x contributes (1 - |x - (c + 1/2)|) per axis to the two nearest cell
 * centres, periodic.  Each particle carries mass N^3/np so the mean is 1.
 */
void or_deposit_cic(const float* pos, long long np, int N, double* rho) {
  size_t N3 = (size_t)N * N * N;
  for (size_t c = 0; c < N3; ++c) rho[c] = 0.0;
  double m = (double)N3 / (double)np;
  for (long long q = 0; q < np; ++q) {
    int i0[3];
    double f[3];
    for (int d = 0; d < 3; ++d) {
      double x = (double)pos[3 * q + d] - 0.5;
      double fl = floor(x);
      i0[d] = (int)fl;
      f[d] = x - fl;
    }
    for (int di = 0; di < 2; ++di)
      for (int dj = 0; dj < 2; ++dj)
        for (int dk = 0; dk < 2; ++dk) {
          double wgt = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) * (dk ? f[2] : 1.0 - f[2]);
          int i = WRAP(((i0[0] + di) % N), N), j = WRAP(((i0[1] + dj) % N), N), k = WRAP(((i0[2] + dk) % N), N);
          rho[IDX(N, i, j, k)] += m * wgt;
        }
  }
}

/*
 * Force on particles: the three-point central difference (T_{c+1} - T_{c-1})/2
 * of a mesh scalar T at each cell centre, interpolated to the particle with the
 * CIC weights of the deposit, times 'scale'.  T is formed from the solved field:
 *   f(R): T = f_R = -u^{n+1}, scale = c^2/2            (Eq. F5_fR_codeunit)
 *   symmetron: T = u^2, scale = -3 xi^2 Om beta*^2 c^2 a*^-3 (Eq. F_5_codeunit)
 *   CQ: T = phi (plus an optional Newtonian potential), scale = -beta
 *       (the fifth-force part of Eq. csf_particle_geodesic_code2)
 * The result is multiplied by 'prefactor' (the caller's time factor, e.g. H0/adot).
 */
void or_gather_force(const or_params* p, int N, const double* u, const double* phiN,
                     const float* pos, long long np, double prefactor, double* force) {
  or_background b;
  or_compute_background(p, N, &b);
  size_t N3 = (size_t)N * N * N;
  double* T = (double*)malloc(N3 * sizeof(double));
  double scale;
  if (p->model == OR_FR) {
    for (size_t c = 0; c < N3; ++c) T[c] = -field_w(p, u[c]);
    scale = 0.5 * b.c2;
  } else if (p->model == OR_SYMMETRON) {
    for (size_t c = 0; c < N3; ++c) T[c] = u[c] * u[c];
    scale = -3.0 * p->xi * p->xi * p->omega_m * p->beta_star * p->beta_star * b.c2 /
            (p->a_star * p->a_star * p->a_star);
  } else {
    for (size_t c = 0; c < N3; ++c) T[c] = p->beta * u[c] + (phiN ? phiN[c] : 0.0);
    scale = -1.0;
  }
  for (long long q = 0; q < np; ++q) {
    int i0[3];
    double f[3];
    for (int d = 0; d < 3; ++d) {
      double x = (double)pos[3 * q + d] - 0.5;
      double fl = floor(x);
      i0[d] = (int)fl;
      f[d] = x - fl;
    }
    double F[3] = {0.0, 0.0, 0.0};
    for (int di = 0; di < 2; ++di)
      for (int dj = 0; dj < 2; ++dj)
        for (int dk = 0; dk < 2; ++dk) {
          double wgt = (di ? f[0] : 1.0 - f[0]) * (dj ? f[1] : 1.0 - f[1]) * (dk ? f[2] : 1.0 - f[2]);
          int i = WRAP((i0[0] + di) % N, N), j = WRAP((i0[1] + dj) % N, N), k = WRAP((i0[2] + dk) % N, N);
          double gx = 0.5 * (T[IDX(N, WRAP(i + 1, N), j, k)] - T[IDX(N, WRAP(i - 1, N), j, k)]);
          double gy = 0.5 * (T[IDX(N, i, WRAP(j + 1, N), k)] - T[IDX(N, i, WRAP(j - 1, N), k)]);
          double gz = 0.5 * (T[IDX(N, i, j, WRAP(k + 1, N))] - T[IDX(N, i, j, WRAP(k - 1, N))]);
          F[0] += wgt * gx;
          F[1] += wgt * gy;
          F[2] += wgt * gz;
        }
    for (int d = 0; d < 3; ++d) force[3 * q + d] = prefactor * scale * F[d];
  }
  free(T);
}

/* Threads the oracle will use (1 without OpenMP). */
int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Set the number of threads of later parallel loops (no effect without OpenMP). */
void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Test export: the nonlinear Gauss-Seidel local root for given p, q. */
double or_local_root(int model, int n, double pp, double qq, double u_old) {
  or_params p;
  memset(&p, 0, sizeof(p));
  p.model = model;
  p.n = n;
  return local_root(&p, pp, qq, u_old);
}

/*
 * Coupled-quintessence background (Sec. 3.2.3, "background cosmology solver").
 *
 * The paper's equations in N = ln a, conformal form:
 *   H^2/H0^2  = [1 - x^2/6]^{-1} [Or e^{-2N} + e^{beta phi} Om e^{-N} + L e^{2N} phi^{-alpha}]
 *   H'/H0^2   = -x^2/3 H^2/H0^2 + L e^{2N} phi^{-alpha} - Or e^{-2N} - Om e^{-N} e^{beta phi}/2
 *   (H^2/H0^2) phi_NN + [2 H^2/H0^2 + H'/H0^2] phi_N - 3 alpha L e^{2N} phi^{-(1+alpha)}
 *        + 3 beta e^{-N} Om e^{beta phi} = 0        (Eq. csf_background_eom_codeunit)
 * with x = dphi/dN and H the conformal Hubble rate.  L is the potential
 * amplitude of these code-unit equations; reading: L = lambda^2/3 with lambda
 * of Eq. csf_param_lambda (V = Lambda^4/phi^alpha, Lambda^4/M_Pl^2 = H0^2
 * lambda^2), which is what the physical Friedmann and field equations give
 * for this potential.
 *
 * Integration: classical fourth-order Runge-Kutta with a fixed step in N from
 * z_init to the requested a.  lambda is found as in the paper by shooting: the
 * H(a=1) the integration predicts must equal H0 (E(N=0) = 1), and E(0) grows
 * with lambda; the root is bracketed and bisected.
 */
typedef struct { double alpha, beta, om, orad, L; } cq_bg;

static double cq_H2(const cq_bg* c, double N, double phi, double x) {
  return (c->orad * exp(-2.0 * N) + exp(c->beta * phi) * c->om * exp(-N) + c->L * exp(2.0 * N) * pow(phi, -c->alpha)) /
         (1.0 - x * x / 6.0);
}

static void cq_rhs(const cq_bg* c, double N, const double y[2], double dy[2]) {
  const double phi = y[0], x = y[1];
  const double H2 = cq_H2(c, N, phi, x);
  const double Hp = -x * x / 3.0 * H2 + c->L * exp(2.0 * N) * pow(phi, -c->alpha) - c->orad * exp(-2.0 * N) -
                    0.5 * c->om * exp(-N) * exp(c->beta * phi);
  dy[0] = x;
  dy[1] = (3.0 * c->alpha * c->L * exp(2.0 * N) * pow(phi, -(1.0 + c->alpha)) -
           3.0 * c->beta * exp(-N) * c->om * exp(c->beta * phi) - (2.0 * H2 + Hp) * x) /
          H2;
}

/* Integrate from N0 to N1 with 'steps' RK4 steps; y in/out. */
static void cq_integrate(const cq_bg* c, double N0, double N1, int steps, double y[2]) {
  const double h = (N1 - N0) / steps;
  double N = N0;
  for (int s = 0; s < steps; ++s) {
    double k1[2], k2[2], k3[2], k4[2], t[2];
    cq_rhs(c, N, y, k1);
    t[0] = y[0] + 0.5 * h * k1[0]; t[1] = y[1] + 0.5 * h * k1[1];
    cq_rhs(c, N + 0.5 * h, t, k2);
    t[0] = y[0] + 0.5 * h * k2[0]; t[1] = y[1] + 0.5 * h * k2[1];
    cq_rhs(c, N + 0.5 * h, t, k3);
    t[0] = y[0] + h * k3[0]; t[1] = y[1] + h * k3[1];
    cq_rhs(c, N + h, t, k4);
    y[0] += h / 6.0 * (k1[0] + 2.0 * k2[0] + 2.0 * k3[0] + k4[0]);
    y[1] += h / 6.0 * (k1[1] + 2.0 * k2[1] + 2.0 * k3[1] + k4[1]);
    N += h;
  }
}

/* E(a=1) - 1 for a trial lambda. */
static double cq_mismatch(cq_bg* c, double lambda, double Ni, double phi_i, double x_i, int steps) {
  c->L = lambda * lambda / 3.0;
  double y[2] = {phi_i, x_i};
  cq_integrate(c, Ni, 0.0, steps, y);
  /* E^2 = H^2/H0^2 at N = 0 (conformal and cosmic rates agree at a = 1) */
  return sqrt(cq_H2(c, 0.0, y[0], y[1])) - 1.0;
}

/* lambda, and at scale factor a: phibar, dphibar/dlna, E = H/H0.  Returns the
 * number of bisection steps, or -1 if no bracket was found. */
int or_cq_background(double alpha, double beta, double omega_m, double omega_r, double a, double z_init,
                     double phi_init, double dphi_init, int steps, double* lambda, double* phibar,
                     double* dphibar, double* E) {
  cq_bg c = {alpha, beta, omega_m, omega_r, 0.0};
  const double Ni = -log(1.0 + z_init);
  double lo = 1.0, hi = 1.0;
  double flo = cq_mismatch(&c, lo, Ni, phi_init, dphi_init, steps), fhi = flo;
  int k = 0;
  while (flo > 0.0 && k++ < 60) { hi = lo; fhi = flo; lo *= 0.5; flo = cq_mismatch(&c, lo, Ni, phi_init, dphi_init, steps); }
  k = 0;
  while (fhi < 0.0 && k++ < 60) { lo = hi; flo = fhi; hi *= 2.0; fhi = cq_mismatch(&c, hi, Ni, phi_init, dphi_init, steps); }
  if (!(flo <= 0.0 && fhi >= 0.0)) return -1;
  int it = 0;
  while (hi - lo > 1e-14 * hi && it < 200) {
    const double mid = 0.5 * (lo + hi);
    const double f = cq_mismatch(&c, mid, Ni, phi_init, dphi_init, steps);
    if (f > 0.0) hi = mid; else lo = mid;
    ++it;
  }
  const double lam = 0.5 * (lo + hi);
  c.L = lam * lam / 3.0;
  double y[2] = {phi_init, dphi_init};
  const double Na = log(a);
  cq_integrate(&c, Ni, Na, (int)ceil(steps * (Na - Ni) / (0.0 - Ni)), y);
  *lambda = lam;
  *phibar = y[0];
  *dphibar = y[1];
  *E = sqrt(cq_H2(&c, Na, y[0], y[1])) * exp(-Na);  /* conformal H / a = H */
  return it;
}
