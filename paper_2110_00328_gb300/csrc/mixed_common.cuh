// mixed_common.cuh -- device helpers shared by the single and batched mixed-precision
// solvers: FP32 level constants, the correction operator M(e), neighbour sums,
// the FP64 source term and the tiled FP64 fine-level residual.
#pragma once
#include <math.h>
#include <string.h>

#include "ff.cuh"
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
    return -f.c2_h2 * (Lnb - 6.f * dw<K>(u, e)) + f.K * e * frcp(u * (u + e));
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

__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// ---------------------------------------------------------------------------
// Restriction of the defect, four fine cells per lane (fine side nf % 4 == 0)
// ---------------------------------------------------------------------------
//
// A lane owns the coarse cells (I, J, 2tq) and (I, J, 2tq+1), whose children
// are the fine quads k0 = 4tq .. k0+3 of the four fine rows (2I+a, 2J+b),
// a, b in {0, 1}.  It reads those rows and the eight rows around them that
// the Laplacian of their cells touches (2I-1, 2I+2 in i; 2J-1, 2J+2 in j) as
// 16-byte quads, forms d = M(e) - S at the sixteen children and writes the
// 8-child means of e, u and d (Eq. restriction) as float2 pairs.  The two
// k-neighbours outside the quad come from the adjacent lanes by shuffles.  All
// 32 lanes of a warp take part (same I, J); lanes past the row end work on a
// clamped quad and store nothing.
// QH (f(R) n = 1, 2 on a split level with stored q, in qf): the halo rows'
// neighbour quantities are read from qf instead of formed from e and u.
// ZR (f(R), symmetron, after pre-smoothing): the second colour ((i+j+k) odd)
// was relaxed last and satisfies its local equations, so its defect is taken as
// zero and only the first colour's is formed (see restrict_split_zr).
template <int K, class FL = NatLayout, bool QH = false, bool ZR = false>
__device__ __forceinline__ void restrict_quad(const LevelF& f, int nf, const float* __restrict__ e,
                                              const float* __restrict__ ub, const float* __restrict__ rho,
                                              const float* __restrict__ S, float* __restrict__ Re,
                                              float* __restrict__ eH, float* __restrict__ ubH,
                                              float* __restrict__ SH, int I, int J, int tq, int lane,
                                              const float* __restrict__ qf = nullptr) {
  constexpr bool FR = is_fr(K);
  constexpr bool RHO = (K == KSYM) || (K == KCQ);
  const int nc = nf >> 1, nq = nf >> 2;
  const bool act = tq < nq;
  const int k0 = 4 * (act ? tq : nq - 1);
  const int i0 = 2 * I, j0 = 2 * J;
  const int iA = i0 == 0 ? nf - 1 : i0 - 1, iB = i0 + 2 == nf ? 0 : i0 + 2;
  const int jA = j0 == 0 ? nf - 1 : j0 - 1, jB = j0 + 2 == nf ? 0 : j0 + 2;
  auto q4 = [&](int i, int j) {
    if constexpr (QH) {
      static_assert(K == KFR1 || K == KFR2, "stored q: f(R) n = 1, 2");
      return FL::q(qf, nf, i, j, k0);
    }
    const float4 E = FL::q(e, nf, i, j, k0);
    if constexpr (FR) {
      const float4 U = FL::q(ub, nf, i, j, k0);
      return make_float4(dw<K>(U.x, E.x), dw<K>(U.y, E.y), dw<K>(U.z, E.z), dw<K>(U.w, E.w));
    } else {
      return E;
    }
  };
  auto q1 = [&](int i, int j, int k) {
    const typename FL::index_t c = FL::idx(nf, i, j, k);
    return nbq<K>(FR ? ub[c] : 0.f, e[c]);
  };
  // own rows (a, b) and their quads
  float4 E[2][2], U[2][2], Q[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      E[a][b] = FL::q(e, nf, i0 + a, j0 + b, k0);
      U[a][b] = FL::q(ub, nf, i0 + a, j0 + b, k0);
      Q[a][b] = FR ? make_float4(dw<K>(U[a][b].x, E[a][b].x), dw<K>(U[a][b].y, E[a][b].y),
                                 dw<K>(U[a][b].z, E[a][b].z), dw<K>(U[a][b].w, E[a][b].w))
                   : E[a][b];
    }
  // halo rows: qi[0][b] = row (2I-1, 2J+b), qi[1][b] = row (2I+2, 2J+b); qj[a][0], qj[a][1] likewise in j
  float4 qi[2][2], qj[2][2];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    qi[0][b] = q4(iA, j0 + b);
    qi[1][b] = q4(iB, j0 + b);
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    qj[a][0] = q4(i0 + a, jA);
    qj[a][1] = q4(i0 + a, jB);
  }
  float se0 = 0.f, se1 = 0.f, su0 = 0.f, su1 = 0.f, sd0 = 0.f, sd1 = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float4 q = Q[a][b];
      float qm = __shfl_up_sync(0xffffffffu, q.w, 1);
      float qp = __shfl_down_sync(0xffffffffu, q.x, 1);
      if (lane == 0) qm = q1(i0 + a, j0 + b, k0 == 0 ? nf - 1 : k0 - 1);
      if (lane == 31 || tq + 1 >= nq) qp = q1(i0 + a, j0 + b, k0 + 4 == nf ? 0 : k0 + 4);
      const float4 ni = a == 0 ? qi[0][b] : Q[0][b];   // i - 1
      const float4 pi = a == 0 ? Q[1][b] : qi[1][b];   // i + 1
      const float4 nj = b == 0 ? qj[a][0] : Q[a][0];   // j - 1
      const float4 pj = b == 0 ? Q[a][1] : qj[a][1];   // j + 1
      const float4 Sv = FL::q(S, nf, i0 + a, j0 + b, k0);
      float4 R = make_float4(1.f, 1.f, 1.f, 1.f);
      if constexpr (RHO) {
        if (rho) R = FL::q(rho, nf, i0 + a, j0 + b, k0);
      }
      const float4 Ev = E[a][b], Uv = U[a][b];
      // with ZR the cells k0 + c of colour (a + b + c) & 1 = 1 have zero defect (k0, 2I, 2J even)
      static_assert(!ZR || K != KCQ, "CQ relaxes by one Newton step: its defect is not zero");
      const bool odd = (a + b) & 1;
      float dx = 0.f, dy = 0.f, dz = 0.f, dv = 0.f;
      if (!ZR || !odd) {
        dx = local_M<K>(f, Uv.x, Ev.x, R.x, (qm + q.y) + (ni.x + pi.x) + (nj.x + pj.x)) - Sv.x;
        dz = local_M<K>(f, Uv.z, Ev.z, R.z, (q.y + q.w) + (ni.z + pi.z) + (nj.z + pj.z)) - Sv.z;
      }
      if (!ZR || odd) {
        dy = local_M<K>(f, Uv.y, Ev.y, R.y, (q.x + q.z) + (ni.y + pi.y) + (nj.y + pj.y)) - Sv.y;
        dv = local_M<K>(f, Uv.w, Ev.w, R.w, (q.z + qp) + (ni.w + pi.w) + (nj.w + pj.w)) - Sv.w;
      }
      se0 += Ev.x + Ev.y;
      se1 += Ev.z + Ev.w;
      su0 += Uv.x + Uv.y;
      su1 += Uv.z + Uv.w;
      sd0 += dx + dy;
      sd1 += dz + dv;
    }
  if (act) {
    using IT = typename FL::index_t;
    const IT t = ((IT)I * nc + J) * nc + (k0 >> 1);
    const float2 me = make_float2(0.125f * se0, 0.125f * se1);
    *reinterpret_cast<float2*>(Re + t) = me;
    *reinterpret_cast<float2*>(eH + t) = me;
    *reinterpret_cast<float2*>(ubH + t) = make_float2(0.125f * su0, 0.125f * su1);
    *reinterpret_cast<float2*>(SH + t) = make_float2(0.125f * sd0, 0.125f * sd1);
  }
}

// ---------------------------------------------------------------------------
// FAS source of a coarse level, four cells per lane (side % 4 == 0)
// ---------------------------------------------------------------------------
//
// S <- M(Re) - S at the four cells k0 .. k0+3 of row (i, j) (S holds R d on
// entry; Eq. general_pde_numerical_coarse), with the neighbour quantities of
// Re read as 16-byte quads from the row and the four rows around it and the
// two k-neighbours outside the quad from the adjacent lanes.  All 32 lanes of a
// warp take part; lanes past the row end work on a clamped quad and store
// nothing.
template <int K, typename IT = long long>
__device__ __forceinline__ void fas_quad(const LevelF& f, int n, const float* __restrict__ Re,
                                         const float* __restrict__ ub, const float* __restrict__ rho,
                                         float* __restrict__ S, int i, int j, int tq, int lane) {
  constexpr bool FR = is_fr(K);
  constexpr bool RHO = (K == KSYM) || (K == KCQ);
  const int nq = n >> 2;
  const bool act = tq < nq;
  const int k0 = 4 * (act ? tq : nq - 1);
  const IT nn = (IT)n * n;
  const IT c0 = (IT)i * nn + (IT)j * n + k0;
  const IT djp = (j + 1 < n) ? (IT)n : -(IT)(n - 1) * n;
  const IT djm = (j > 0) ? -(IT)n : (IT)(n - 1) * n;
  const IT dip = (i + 1 < n) ? nn : -(IT)(n - 1) * nn;
  const IT dim = (i > 0) ? -nn : (IT)(n - 1) * nn;
  auto q4 = [&](IT c) {
    const float4 E = ld4(Re + c);
    if constexpr (FR) {
      const float4 U = ld4(ub + c);
      return make_float4(dw<K>(U.x, E.x), dw<K>(U.y, E.y), dw<K>(U.z, E.z), dw<K>(U.w, E.w));
    } else {
      return E;
    }
  };
  const float4 E = ld4(Re + c0), U = ld4(ub + c0), Sv = ld4(S + c0);
  const float4 q = FR ? make_float4(dw<K>(U.x, E.x), dw<K>(U.y, E.y), dw<K>(U.z, E.z), dw<K>(U.w, E.w)) : E;
  const float4 P = q4(c0 + djp), M = q4(c0 + djm), A = q4(c0 + dip), B = q4(c0 + dim);
  float4 R = make_float4(1.f, 1.f, 1.f, 1.f);
  if constexpr (RHO) {
    if (rho) R = ld4(rho + c0);
  }
  float qm = __shfl_up_sync(0xffffffffu, q.w, 1);
  float qp = __shfl_down_sync(0xffffffffu, q.x, 1);
  if (lane == 0) {
    const IT c = c0 + (k0 == 0 ? n - 1 : -1);
    qm = nbq<K>(FR ? ub[c] : 0.f, Re[c]);
  }
  if (lane == 31 || tq + 1 >= nq) {
    const IT c = c0 + (k0 + 4 == n ? 4 - n : 4);
    qp = nbq<K>(FR ? ub[c] : 0.f, Re[c]);
  }
  float4 out;
  out.x = local_M<K>(f, U.x, E.x, R.x, (qm + q.y) + (P.x + M.x) + (A.x + B.x)) - Sv.x;
  out.y = local_M<K>(f, U.y, E.y, R.y, (q.x + q.z) + (P.y + M.y) + (A.y + B.y)) - Sv.y;
  out.z = local_M<K>(f, U.z, E.z, R.z, (q.y + q.w) + (P.z + M.z) + (A.z + B.z)) - Sv.z;
  out.w = local_M<K>(f, U.w, E.w, R.w, (q.z + qp) + (P.w + M.w) + (A.w + B.w)) - Sv.w;
  if (act) *reinterpret_cast<float4*>(S + c0) = out;
}

// Restriction of the defect after pre-smoothing on a split finest level with
// stored q (f(R) n = 1, 2): the last pre-smoothing pass relaxed the second
// colour, and each of its cells then satisfies its own local equation (the
// closed-form root polished by Newton steps, or the warm-started Newton
// steps), so the defect d = M(e) - S vanishes there up to the local solve's
// rounding; it is formed at the first colour's cells only.  The lane mapping
// is restrict_quad's (coarse cells (I, J, 2tq), (I, J, 2tq+1); fine quads
// k0 = 4tq .. k0+3 of the rows (2I+a, 2J+b)).  In the split layout a row's quad
// is one float2 per colour half; the first colour's two cells of row (i, j)
// sit at k0 + p and k0 + p + 2, p = (i + j) & 1, one in each coarse cell, and
// all six neighbours of a first-colour cell are second-colour cells, whose
// stored q lies in the second colour's half at the same index (the i and j
// neighbours) or the adjacent ones (the k neighbours).
// IT: the index type of the cell offsets (int where the fine level has < 2^31 cells).
template <int K, typename IT = long long>
__device__ __forceinline__ void restrict_split_zr(const LevelF& f, int nf, const float* __restrict__ e,
                                                  const float* __restrict__ ub, const float* __restrict__ S,
                                                  const float* __restrict__ qf, float* __restrict__ Re,
                                                  float* __restrict__ eH, float* __restrict__ ubH,
                                                  float* __restrict__ SH, int I, int J, int tq, int lane) {
  static_assert(K == KFR1 || K == KFR2, "stored q: f(R) n = 1, 2");
  const int nc = nf >> 1, nq = nf >> 2, h = nf >> 1;
  const bool act = tq < nq;
  const int m0 = 2 * (act ? tq : nq - 1);  // index of the quad in a colour half-row
  const IT H = (IT)nf * nf * h;
  const int i0 = 2 * I, j0 = 2 * J;
  const int iA = i0 == 0 ? nf - 1 : i0 - 1, iB = i0 + 2 == nf ? 0 : i0 + 2;
  const int jA = j0 == 0 ? nf - 1 : j0 - 1, jB = j0 + 2 == nf ? 0 : j0 + 2;
  auto row = [&](int i, int j) { return ((IT)i * nf + j) * h + m0; };
  const float* q1 = qf + H;  // second-colour half of q
  // second-colour q of the own rows and of the halo rows around them
  float2 Q[2][2], qi[2][2], qj[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) Q[a][b] = ld2(q1 + row(i0 + a, j0 + b));
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    qi[0][b] = ld2(q1 + row(iA, j0 + b));
    qi[1][b] = ld2(q1 + row(iB, j0 + b));
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    qj[a][0] = ld2(q1 + row(i0 + a, jA));
    qj[a][1] = ld2(q1 + row(i0 + a, jB));
  }
  float se0 = 0.f, se1 = 0.f, su0 = 0.f, su1 = 0.f, sd0 = 0.f, sd1 = 0.f;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const IT r = row(i0 + a, j0 + b);
      const float2 E0 = ld2(e + r), E1 = ld2(e + H + r), U0 = ld2(ub + r), U1 = ld2(ub + H + r);
      const float2 S0 = ld2(S + r);
      se0 += E0.x + E1.x;
      se1 += E0.y + E1.y;
      su0 += U0.x + U1.x;
      su1 += U0.y + U1.y;
      // k neighbours of the first-colour cells k0 + p + 2m: p = 0 -> (m - 1/2 +- 1/2) in the
      // second colour's half-row, the one before the quad from the previous lane; p = 1 ->
      // (m, m + 1), the one after the quad from the next lane
      const int p = (a + b) & 1;
      const float2 q = Q[a][b];
      float qm = __shfl_up_sync(0xffffffffu, q.y, 1);
      float qp = __shfl_down_sync(0xffffffffu, q.x, 1);
      if (p == 0 && lane == 0) qm = q1[row(i0 + a, j0 + b) + (m0 == 0 ? h - 1 : -1)];
      if (p == 1 && (lane == 31 || tq + 1 >= nq)) qp = q1[row(i0 + a, j0 + b) + (m0 + 2 == h ? 2 - h : 2)];
      const float k0s = p ? q.x + q.y : qm + q.x;
      const float k1s = p ? q.y + qp : q.x + q.y;
      const float2 ni = a == 0 ? qi[0][b] : Q[0][b], pi = a == 0 ? Q[1][b] : qi[1][b];
      const float2 nj = b == 0 ? qj[a][0] : Q[a][0], pj = b == 0 ? Q[a][1] : qj[a][1];
      const float dx = local_M<K>(f, U0.x, E0.x, 1.f, k0s + (ni.x + pi.x) + (nj.x + pj.x)) - S0.x;
      const float dy = local_M<K>(f, U0.y, E0.y, 1.f, k1s + (ni.y + pi.y) + (nj.y + pj.y)) - S0.y;
      sd0 += dx;
      sd1 += dy;
    }
  if (act) {
    const IT t = ((IT)I * nc + J) * nc + m0;
    const float2 me = make_float2(0.125f * se0, 0.125f * se1);
    *reinterpret_cast<float2*>(Re + t) = me;
    *reinterpret_cast<float2*>(eH + t) = me;
    *reinterpret_cast<float2*>(ubH + t) = make_float2(0.125f * su0, 0.125f * su1);
    *reinterpret_cast<float2*>(SH + t) = make_float2(0.125f * sd0, 0.125f * sd1);
  }
}

// ---------------------------------------------------------------------------
// Prolongation-correction, four fine cells per lane (fine side % 4 == 0)
// ---------------------------------------------------------------------------
//
// e_h += P(e_H - R e_h) with the 27/9/3/1 (/64) weights of Eq. prolongation,
// which factor into (3/4, 1/4) per axis: the lane first combines the four
// coarse rows (I, J) 9, (I2, J) 3, (I, J2) 3, (I2, J2) 1 at its two coarse k
// (2tq, 2tq+1), takes the combinations at 2tq-1 and 2tq+2 from the adjacent
// lanes, and weights (3, 1) along k.  f(R): where u + e would not be positive
// the total field is halved instead (e <- (e_old - u)/2).
// QK >= 0 (split layout, f(R) n = QK): also writes the second colour's stored
// neighbour quantity q = Delta w(u, e) into qf (smooth_split with QS), so that
// the next first-colour pass sees the corrected values.
// SECOND_ONLY (with QK >= 0, when post-smoothing follows): corrects the second
// colour only.  The f(R) local solve of the first-colour pass that comes next
// does not read a cell's old value (the closed-form root from u, S and the
// neighbours, then the polish), so the first colour's corrected values would be
// overwritten unread; skipping them leaves the iterates unchanged and moves
// 8 instead of 14 bytes per fine cell.
template <bool FR, class FL = NatLayout, int QK = -1, bool SECOND_ONLY = false>
__device__ __forceinline__ void prolong_quad(int nc, const float* __restrict__ eH, const float* __restrict__ Re,
                                             const float* __restrict__ ub, float* __restrict__ ef, int i, int j,
                                             int tq, int lane, unsigned long long* guard,
                                             float* __restrict__ qf = nullptr) {
  static_assert(QK < 0 || (FR && QK != KFR0), "stored q: f(R) n = 1, 2");
  static_assert(!SECOND_ONLY || QK >= 0, "second-colour-only prolongation: split layout with stored q");
  const int nf = nc << 1, nq = nf >> 2;
  const bool act = tq < nq;
  const int t = act ? tq : nq - 1;
  const int k0 = 4 * t, K0 = 2 * t;
  const int I = i >> 1, J = j >> 1;
  int I2 = I + ((i & 1) ? 1 : -1), J2 = J + ((j & 1) ? 1 : -1);
  I2 = I2 < 0 ? nc - 1 : (I2 >= nc ? 0 : I2);
  J2 = J2 < 0 ? nc - 1 : (J2 >= nc ? 0 : J2);
  using IT = typename FL::index_t;  // the coarse level is the fine one's half: the same index range fits
  const IT rA = ((IT)I * nc + J) * nc, rB = ((IT)I2 * nc + J) * nc, rC = ((IT)I * nc + J2) * nc,
           rD = ((IT)I2 * nc + J2) * nc;
  auto d2 = [&](IT r) {
    const float2 a = ld2(eH + r + K0), b = ld2(Re + r + K0);
    return make_float2(a.x - b.x, a.y - b.y);
  };
  auto d1 = [&](IT r, int Kc) { return eH[r + Kc] - Re[r + Kc]; };
  const float2 A = d2(rA), B = d2(rB), C = d2(rC), D = d2(rD);
  const float Rx = 9.f * A.x + 3.f * (B.x + C.x) + D.x;
  const float Ry = 9.f * A.y + 3.f * (B.y + C.y) + D.y;
  float Rm = __shfl_up_sync(0xffffffffu, Ry, 1);    // coarse k = K0 - 1
  float Rp = __shfl_down_sync(0xffffffffu, Rx, 1);  // coarse k = K0 + 2
  if (lane == 0) {
    const int Km = K0 == 0 ? nc - 1 : K0 - 1;
    Rm = 9.f * d1(rA, Km) + 3.f * (d1(rB, Km) + d1(rC, Km)) + d1(rD, Km);
  }
  if (lane == 31 || tq + 1 >= nq) {
    const int Kp = K0 + 2 == nc ? 0 : K0 + 2;
    Rp = 9.f * d1(rA, Kp) + 3.f * (d1(rB, Kp) + d1(rC, Kp)) + d1(rD, Kp);
  }
  constexpr float w = 1.f / 64.f;
  if constexpr (SECOND_ONLY) {
    // the second colour's two cells of the quad: k0 and k0+2 where i + j is odd, else k0+1 and k0+3;
    // they are consecutive in the second colour's half-row
    const bool odd = (i + j) & 1;
    const float cA = odd ? (3.f * Rx + Rm) * w : (3.f * Rx + Ry) * w;
    const float cB = odd ? (3.f * Ry + Rx) * w : (3.f * Ry + Rp) * w;
    const int h = nf >> 1;
    const long long o1 = (long long)nf * nf * h + ((long long)i * nf + j) * h + (k0 >> 1);
    const float2 old = ld2(ef + o1), u = ld2(ub + o1);
    float vA = old.x + cA, vB = old.y + cB;
    const bool gA = !(u.x + vA > 0.f), gB = !(u.y + vB > 0.f);
    if (gA) vA = 0.5f * (old.x - u.x);
    if (gB) vB = 0.5f * (old.y - u.y);
    if (act) count_guards(guard, (unsigned)gA + (unsigned)gB);
    if (act) {
      *reinterpret_cast<float2*>(ef + o1) = make_float2(vA, vB);
      *reinterpret_cast<float2*>(qf + o1) = make_float2(dw<QK>(u.x, vA), dw<QK>(u.y, vB));
    }
    return;
  }
  const float4 old = FL::q(ef, nf, i, j, k0);
  float4 v = make_float4(old.x + (3.f * Rx + Rm) * w, old.y + (3.f * Rx + Ry) * w, old.z + (3.f * Ry + Rx) * w,
                         old.w + (3.f * Ry + Rp) * w);
  float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (FR) {
    u = FL::q(ub, nf, i, j, k0);
    const bool gx = !(u.x + v.x > 0.f), gy = !(u.y + v.y > 0.f), gz = !(u.z + v.z > 0.f),
               gw = !(u.w + v.w > 0.f);
    if (gx) v.x = 0.5f * (old.x - u.x);
    if (gy) v.y = 0.5f * (old.y - u.y);
    if (gz) v.z = 0.5f * (old.z - u.z);
    if (gw) v.w = 0.5f * (old.w - u.w);
    if (act) count_guards(guard, (unsigned)gx + (unsigned)gy + (unsigned)gz + (unsigned)gw);
  }
  if (act) FL::st(ef, nf, i, j, k0, v);
  if constexpr (QK >= 0) {
    // second-colour cells of the quad: k odd where i + j is even, else k even
    if (act) {
      const int h = nf >> 1;
      const long long H = (long long)nf * nf * h, r = ((long long)i * nf + j) * h + (k0 >> 1);
      *reinterpret_cast<float2*>(qf + H + r) = ((i + j) & 1)
                                                   ? make_float2(dw<QK>(u.x, v.x), dw<QK>(u.z, v.z))
                                                   : make_float2(dw<QK>(u.y, v.y), dw<QK>(u.w, v.w));
    }
  }
}

// Prolongation-correction of the second colour on a split finest level with
// stored q (f(R) n = QK), four fine rows per lane: the lane owns the quad
// k0 = 4tq .. k0+3 of the fine rows (2I+a, 2J+b), a, b in {0, 1} -- the children
// of the coarse row pair (I, J) -- which interpolate from the nine coarse rows
// (I-1..I+1, J-1..J+1); prolong_quad reads four coarse rows for each fine row.
// Each fine row's second-colour pair is corrected (and its q written) exactly
// as prolong_quad<true, SplitLayout, QK, true> does it.  Grid as the
// restriction's: (ceil(nf/128), nc [J], ceil(nc/4) [I]), block (32, 4).
// DD: eH holds the coarse difference eH - Re itself (written by the coarse
// level's last post-smoothing pass, smooth_quad's WD), and Re is not read.
template <int QK, bool DD = false, typename IT = long long>
__device__ __forceinline__ void prolong_split2x2_second(int nc, const float* __restrict__ eH,
                                                        const float* __restrict__ Re, const float* __restrict__ ub,
                                                        float* __restrict__ ef, int I, int J, int tq, int lane,
                                                        unsigned long long* guard, float* __restrict__ qf) {
  static_assert(QK == KFR1 || QK == KFR2, "stored q: f(R) n = 1, 2");
  const int nf = nc << 1, nq = nf >> 2, h = nf >> 1;
  const bool act = tq < nq;
  const int t = act ? tq : nq - 1;
  const int k0 = 4 * t, K0 = 2 * t;
  const int Km = K0 == 0 ? nc - 1 : K0 - 1, Kp = K0 + 2 == nc ? 0 : K0 + 2;
  const int Iv[3] = {I == 0 ? nc - 1 : I - 1, I, I + 1 == nc ? 0 : I + 1};
  const int Jv[3] = {J == 0 ? nc - 1 : J - 1, J, J + 1 == nc ? 0 : J + 1};
  const bool edge_m = lane == 0, edge_p = lane == 31 || tq + 1 >= nq;
  // coarse differences eH - Re of the nine rows at K0, K0+1 (and K0-1, K0+2 at the row ends)
  float2 d[3][3];
  float dm[3][3], dp[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) {
      const IT r = ((IT)Iv[x] * nc + Jv[y]) * nc;
      if constexpr (DD) {
        d[x][y] = ld2(eH + r + K0);
        dm[x][y] = edge_m ? eH[r + Km] : 0.f;
        dp[x][y] = edge_p ? eH[r + Kp] : 0.f;
      } else {
        const float2 a = ld2(eH + r + K0), b = ld2(Re + r + K0);
        d[x][y] = make_float2(a.x - b.x, a.y - b.y);
        dm[x][y] = edge_m ? eH[r + Km] - Re[r + Km] : 0.f;
        dp[x][y] = edge_p ? eH[r + Kp] - Re[r + Kp] : 0.f;
      }
    }
  constexpr float w = 1.f / 64.f;
  const IT H = (IT)nf * nf * h;
  unsigned ng = 0;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int x2 = a ? 2 : 0, y2 = b ? 2 : 0;  // the coarse neighbour rows of fine row (2I+a, 2J+b)
      const float2 A = d[1][1], B = d[x2][1], Cc = d[1][y2], D = d[x2][y2];
      const float Rx = 9.f * A.x + 3.f * (B.x + Cc.x) + D.x;
      const float Ry = 9.f * A.y + 3.f * (B.y + Cc.y) + D.y;
      float Rm = __shfl_up_sync(0xffffffffu, Ry, 1);
      float Rp = __shfl_down_sync(0xffffffffu, Rx, 1);
      if (edge_m) Rm = 9.f * dm[1][1] + 3.f * (dm[x2][1] + dm[1][y2]) + dm[x2][y2];
      if (edge_p) Rp = 9.f * dp[1][1] + 3.f * (dp[x2][1] + dp[1][y2]) + dp[x2][y2];
      const bool odd = (a + b) & 1;  // (i + j) & 1 of the fine row
      const float cA = odd ? (3.f * Rx + Rm) * w : (3.f * Rx + Ry) * w;
      const float cB = odd ? (3.f * Ry + Rx) * w : (3.f * Ry + Rp) * w;
      const int i = 2 * I + a, j = 2 * J + b;
      const IT o1 = H + ((IT)i * nf + j) * h + (k0 >> 1);
      const float2 old = ld2(ef + o1), u = ld2(ub + o1);
      float vA = old.x + cA, vB = old.y + cB;
      const bool gA = !(u.x + vA > 0.f), gB = !(u.y + vB > 0.f);
      if (gA) vA = 0.5f * (old.x - u.x);
      if (gB) vB = 0.5f * (old.y - u.y);
      ng += (unsigned)gA + (unsigned)gB;
      if (act) {
        *reinterpret_cast<float2*>(ef + o1) = make_float2(vA, vB);
        *reinterpret_cast<float2*>(qf + o1) = make_float2(dw<QK>(u.x, vA), dw<QK>(u.y, vB));
      }
    }
  if (act) count_guards(guard, ng);
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
  // f(R): Om/a (rho/mean - 1) + K0 = c1 rho + c0, one FMA per cell
  const double c1 = is_fr(K) ? m.om_a * inv_mean : inv_mean;
  const double c0 = is_fr(K) ? m.K0 - m.om_a : 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    src[t] = fma(c1, (double)rho32[t], c0);
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

// ---------------------------------------------------------------------------
// The same residual in float-float arithmetic (f(R) and symmetron)
// ---------------------------------------------------------------------------

// Constants of the float-float residual, written once per solve on the device
// (the source slope depends on the density mean computed there).
struct FFC {
  ff c2;      // c~^2
  ff K;       // f(R): K0 ubar
  ff c1, c0;  // source term c1 rho + c0: f(R) Om/(a mean), K0 - Om/a; symmetron 1/mean, 0
  ff msym, rat3;
};

__device__ __forceinline__ ff ff_split_dev(double d) {
  const float hi = (float)d;
  return ff{hi, (float)(d - (double)hi)};
}

static __global__ void k_ff_consts(ModelDev m, long long n3, const double* __restrict__ rho_sum,
                                   FFC* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double inv_mean = (double)n3 / *rho_sum;
  FFC c;
  c.c2 = ff_split_dev(m.c2);
  c.K = ff_split_dev(m.K);
  const bool fr = m.kind <= KFR2;
  c.c1 = ff_split_dev(fr ? m.om_a * inv_mean : inv_mean);
  c.c0 = ff_split_dev(fr ? m.K0 - m.om_a : 0.0);
  c.msym = ff_split_dev(m.msym);
  c.rat3 = ff_split_dev(m.rat3);
  *out = c;
}

// f(R): w = u^{n+1}; symmetron: w = u
template <int K>
__device__ __forceinline__ ff ff_w(ff u) {
  if constexpr (K == KFR1) return ff_sqr(u);
  else if constexpr (K == KFR2) return ff_mul(ff_sqr(u), u);
  else return u;
}

// r = N(u64) at every cell of one tile, as outer_residual_tile, with the
// arithmetic in float-float (~2^-48 relative per operation; the terms of N are
// at most ~10^3 times the residual's scale, so the result keeps ~1e-12 of it).
// The source is formed from the FP32 density on the fly.
// The CTA marches up its chunk of planes with a three-plane ring of w and u in
// shared memory; the doubles of plane i+2 are loaded into registers while
// plane i is computed, so the global-load latency overlaps the arithmetic.
// zero_e, zero_q (may be null): arrays of the level's layout set to zero at every
// cell, the next inner solve's initial correction and its stored Delta w(u, 0).
template <int K, int TJ, int TK, bool SPLIT = false>
__device__ __forceinline__ double outer_residual_tile_ff(const FFC& C, int n, int chunk, const double* __restrict__ u,
                                                         const float* __restrict__ rho, float* __restrict__ ub,
                                                         float* __restrict__ tau, int tile, int cb,
                                                         float* __restrict__ zero_e = nullptr,
                                                         float* __restrict__ zero_q = nullptr) {
  static_assert(K != KCQ, "CQ keeps the FP64 residual");
  constexpr int PJ = TJ + 2, PK = TK + 2, PS = PJ * PK, NT = TJ * TK, NE = (PS + NT - 1) / NT;
  __shared__ float s_wh[3][PS], s_wl[3][PS], s_uh[3][PS], s_ul[3][PS];
  const int tiles_k = n / TK;
  const int k0 = (tile % tiles_k) * TK;
  const int j0 = (tile / tiles_k) * TJ;
  const int i0 = cb * chunk;
  const int i1 = min(i0 + chunk, n);
  const int t = threadIdx.x;
  const int tj = t / TK, tk = t - tj * TK;
  const int jg = j0 + tj, kg = k0 + tk;
  const int cc = (tj + 1) * PK + tk + 1;
  const size_t nn = (size_t)n * n;
  // in-plane offsets of this thread's ring elements (fixed for the whole march)
  size_t off[NE];
#pragma unroll
  for (int m = 0; m < NE; ++m) {
    const int c = t + m * NT;
    const int jj = c / PK, kk = c - jj * PK;
    off[m] = c < PS ? (size_t)wrapi(j0 + jj - 1, n) * n + wrapi(k0 + kk - 1, n) : 0;
  }
  double pre[NE];
  auto fetch = [&](int p) {
    const int ig = p < 0 ? p + n : (p >= n ? p - n : p);
    const double* base = u + (size_t)ig * nn;
#pragma unroll
    for (int m = 0; m < NE; ++m) pre[m] = (t + m * NT < PS) ? base[off[m]] : 0.0;
  };
  auto commit = [&](int p) {
    const int slot = (p + 3) % 3;
#pragma unroll
    for (int m = 0; m < NE; ++m) {
      const int c = t + m * NT;
      if (c < PS) {
        const ff uu = ff_from_double(pre[m]);
        const ff w = ff_w<K>(uu);
        s_wh[slot][c] = w.hi;
        s_wl[slot][c] = w.lo;
        s_uh[slot][c] = uu.hi;
        s_ul[slot][c] = uu.lo;
      }
    }
  };
  auto W = [&](int slot, int c) { return ff{s_wh[slot][c], s_wl[slot][c]}; };
  float acc = 0.f;
  fetch(i0 - 1);
  commit(i0 - 1);
  fetch(i0);
  commit(i0);
  fetch(i0 + 1);
  for (int i = i0; i < i1; ++i) {
    commit(i + 1);
    __syncthreads();
    if (i + 2 <= i1) fetch(i + 2);
    const int sl = (i + 3) % 3, sm = (i + 2) % 3, sp = (i + 4) % 3;
    const size_t g = (size_t)i * nn + (size_t)jg * n + kg;
    const float r = rho[g];
    const ff uc = ff{s_uh[sl][cc], s_ul[sl][cc]};
    const ff wc = W(sl, cc);
    // sum of the six neighbours - 6 w, accumulated unnormalised
    ffacc La = acc_of(W(sm, cc));
    acc_add(La, W(sp, cc));
    acc_add(La, W(sl, cc - PK));
    acc_add(La, W(sl, cc + PK));
    acc_add(La, W(sl, cc - 1));
    acc_add(La, W(sl, cc + 1));
    {
      const ff w6 = two_prod(wc.hi, -6.f);
      acc_add(La, w6.hi, __fmaf_rn(wc.lo, -6.f, w6.lo));
    }
    const ff L = acc_ff(La);
    float tv;
    if constexpr (is_fr(K)) {
      // c1 rho + c0 - c2 (L - 6w) - K/u, each product kept as an exact leading
      // product plus its first-order low part
      ffacc v = acc_of(C.c0);
      const ff p1 = two_prod(C.c1.hi, r);
      acc_add(v, p1.hi, __fmaf_rn(C.c1.lo, r, p1.lo));
      const ff p2 = two_prod(C.c2.hi, L.hi);
      acc_add(v, -p2.hi, -__fmaf_rn(C.c2.hi, L.lo, __fmaf_rn(C.c2.lo, L.hi, p2.lo)));
      const ff q = ff_div(C.K, uc);
      acc_add(v, -q.hi, -q.lo);
      tv = -acc_float(v);
    } else {
      // c2 (L - 6u) - msym ((rho/mean rat3 - 1) u + u^3)
      const ff a = ff_sub(ff_mul(ff_mul_f(C.c1, r), C.rat3), ff{1.f, 0.f});
      const ff b = ff_add(ff_mul(a, uc), ff_mul(ff_sqr(uc), uc));
      tv = -ff_to_float(ff_sub(ff_mul(C.c2, L), ff_mul(C.msym, b)));
    }
    const long long o = SPLIT ? split_idx(n, i, jg, kg) : (long long)g;  // the level's layout
    ub[o] = ff_to_float(uc);
    tau[o] = tv;
    if (zero_e) zero_e[o] = 0.f;
    if (zero_q) zero_q[o] = 0.f;
    acc += tv * tv;
    __syncthreads();
  }
  return block_sum((double)acc);
}

// The same residual for two adjacent cells per thread (k = k0 + 2x and
// k0 + 2x + 1) on a TJ x 64 tile, TJ x 32 threads.  The three-plane ring holds
// w and u as (hi, lo) pairs, rows padded so that a thread's two cells are one
// 16-byte shared-memory access; the halo (TJ + 2) x 66 is converted once per
// plane (1.29 conversions a cell instead of 1.33 with 8 x 32 tiles of one cell
// a thread), and the two cells share the per-plane bookkeeping, the address
// arithmetic and, on a split level, one index into both colours (cells 2m and
// 2m + 1 of a row sit at the same k/2 of the two colour arrays).  The six-
// neighbour sum and the source terms of each cell are formed in the same order
// as in outer_residual_tile_ff, so each cell's residual is the same float.
// IT: the index type of the cell offsets (int where n^3 < 2^31).
template <int K, int TJ, bool SPLIT, typename IT = long long>
__global__ void __launch_bounds__(TJ * 32, 5) k_outer_residual_ff2(const FFC* __restrict__ Cp, int n, int chunk,
                                                               const double* __restrict__ u,
                                                               const float* __restrict__ rho, float* __restrict__ ub,
                                                               float* __restrict__ tau, double* __restrict__ partials,
                                                               const int* __restrict__ skip,
                                                               float* __restrict__ zero_e, float* __restrict__ zero_q) {
  static_assert(K != KCQ, "CQ keeps the FP64 residual");
  if (skip && *skip) return;
  const FFC C = *Cp;
  constexpr int TK = 64, NT = TJ * 32;
  constexpr int RW = TK + 2;         // halo row: k0 - 1 .. k0 + 64
  constexpr int RS = RW + 2;         // slot row stride; element x of a halo row at x + 1
  constexpr int PE = (TJ + 2) * RW;  // halo elements a plane
  constexpr int PS = (TJ + 2) * RS;
  constexpr int NE = (PE + NT - 1) / NT;
  __shared__ __align__(16) float2 s_w[4][PS];
  __shared__ __align__(16) float2 s_u[4][PS];
  const int tiles_k = n / TK;
  const int k0 = (blockIdx.x % tiles_k) * TK;
  const int j0 = (blockIdx.x / tiles_k) * TJ;
  const int i0 = blockIdx.y * chunk;
  const int i1 = min(i0 + chunk, n);
  const int t = threadIdx.x;
  const int ty = t >> 5, tx = t & 31;
  const int jg = j0 + ty, kg = k0 + 2 * tx;
  const int cc = (ty + 1) * RS + 2 * tx + 2;  // slot index of cell kg; cell kg + 1 at cc + 1
  const IT nn = (IT)n * n;
  IT off[NE];
  int pos[NE];
#pragma unroll
  for (int m = 0; m < NE; ++m) {
    const int c = t + m * NT;
    const int y = c / RW, x = c - y * RW;
    off[m] = c < PE ? (IT)wrapi(j0 + y - 1, n) * n + wrapi(k0 + x - 1, n) : 0;
    pos[m] = c < PE ? y * RS + x + 1 : -1;
  }
  double pre[NE];
  auto fetch = [&](int p) {
    const int ig = p < 0 ? p + n : (p >= n ? p - n : p);
    const double* base = u + (IT)ig * nn;
#pragma unroll
    for (int m = 0; m < NE; ++m) pre[m] = pos[m] >= 0 ? base[off[m]] : 0.0;
  };
  auto commit = [&](int slot) {
#pragma unroll
    for (int m = 0; m < NE; ++m)
      if (pos[m] >= 0) {
        const ff uu = ff_from_double(pre[m]);
        const ff w = ff_w<K>(uu);
        s_w[slot][pos[m]] = make_float2(w.hi, w.lo);
        s_u[slot][pos[m]] = make_float2(uu.hi, uu.lo);
      }
  };
  auto lds4 = [](const float2* p) { return *reinterpret_cast<const float4*>(p); };
  // the residual of one cell from its ring values (outer_residual_tile_ff's order)
  auto cell = [&](ff uc, ff wc, ff wim, ff wip, ff wjm, ff wjp, ff wkm, ff wkp, float r) -> float {
    ffacc La = acc_of(wim);
    acc_add(La, wip);
    acc_add(La, wjm);
    acc_add(La, wjp);
    acc_add(La, wkm);
    acc_add(La, wkp);
    {
      const ff w6 = two_prod(wc.hi, -6.f);
      acc_add(La, w6.hi, __fmaf_rn(wc.lo, -6.f, w6.lo));
    }
    const ff L = acc_ff(La);
    if constexpr (is_fr(K)) {
      ffacc v = acc_of(C.c0);
      const ff p1 = two_prod(C.c1.hi, r);
      acc_add(v, p1.hi, __fmaf_rn(C.c1.lo, r, p1.lo));
      const ff p2 = two_prod(C.c2.hi, L.hi);
      acc_add(v, -p2.hi, -__fmaf_rn(C.c2.hi, L.lo, __fmaf_rn(C.c2.lo, L.hi, p2.lo)));
      const ff q = ff_div(C.K, uc);
      acc_add(v, -q.hi, -q.lo);
      return -acc_float(v);
    } else {
      const ff a = ff_sub(ff_mul(ff_mul_f(C.c1, r), C.rat3), ff{1.f, 0.f});
      const ff b = ff_add(ff_mul(a, uc), ff_mul(ff_sqr(uc), uc));
      return -ff_to_float(ff_sub(ff_mul(C.c2, L), ff_mul(C.msym, b)));
    }
  };
  float acc = 0.f;
  // four ring slots: plane p in slot p & 3, so the slot written for plane i + 1
  // was last read two planes earlier and one barrier a plane suffices
  const IT nh = (IT)n * (n >> 1);
  const IT H = (IT)nn * (n >> 1);
  IT o0, o1;  // the two cells of plane i0 in the level's layout
  if constexpr (SPLIT) {
    const IT idx = ((IT)i0 * n + jg) * (n >> 1) + (kg >> 1);
    const bool c0 = ((i0 + jg) & 1) != 0;  // colour of the even cell kg
    o0 = c0 ? H + idx : idx;
    o1 = c0 ? idx : H + idx;
  } else {
    o0 = (IT)i0 * (IT)nn + (IT)jg * n + kg;
    o1 = o0 + 1;
  }
  const float* rp = rho + (IT)i0 * nn + (IT)jg * n + kg;
  fetch(i0 - 1);
  commit((i0 - 1) & 3);
  fetch(i0);
  commit(i0 & 3);
  fetch(i0 + 1);
  for (int i = i0; i < i1; ++i) {
    commit((i + 1) & 3);
    __syncthreads();
    if (i + 2 <= i1) fetch(i + 2);
    const int sm = (i - 1) & 3, sl = i & 3, sp = (i + 1) & 3;
    const float2 r2 = *reinterpret_cast<const float2*>(rp);
    const float4 U = lds4(&s_u[sl][cc]);
    const float4 Wc = lds4(&s_w[sl][cc]);
    const float2 Wkm = s_w[sl][cc - 1], Wkp = s_w[sl][cc + 2];
    const float4 Wjm = lds4(&s_w[sl][cc - RS]), Wjp = lds4(&s_w[sl][cc + RS]);
    const float4 Wim = lds4(&s_w[sm][cc]), Wip = lds4(&s_w[sp][cc]);
    const ff u0{U.x, U.y}, u1{U.z, U.w}, w0{Wc.x, Wc.y}, w1{Wc.z, Wc.w};
    const float t0 = cell(u0, w0, ff{Wim.x, Wim.y}, ff{Wip.x, Wip.y}, ff{Wjm.x, Wjm.y}, ff{Wjp.x, Wjp.y},
                          ff{Wkm.x, Wkm.y}, w1, r2.x);
    const float t1 = cell(u1, w1, ff{Wim.z, Wim.w}, ff{Wip.z, Wip.w}, ff{Wjm.z, Wjm.w}, ff{Wjp.z, Wjp.w}, w0,
                          ff{Wkp.x, Wkp.y}, r2.y);
    ub[o0] = ff_to_float(u0);
    ub[o1] = ff_to_float(u1);
    tau[o0] = t0;
    tau[o1] = t1;
    if (zero_e) {
      zero_e[o0] = 0.f;
      zero_e[o1] = 0.f;
    }
    if (zero_q) {
      zero_q[o0] = 0.f;
      zero_q[o1] = 0.f;
    }
    acc += t0 * t0;
    acc += t1 * t1;
    rp += nn;
    if constexpr (SPLIT) {
      // the next plane: one row block on, the colours of the two cells swapped
      const IT a = o0;
      o0 = o1 + nh;
      o1 = a + nh;
    } else {
      o0 += (IT)nn;
      o1 += (IT)nn;
    }
  }
  const double a = block_sum((double)acc);
  if (t == 0) partials[blockIdx.x + blockIdx.y * gridDim.x] = a;
}

// skip (may be nullptr): set when k_background_residual_ff has already formed
// this residual (the solve started from the background field).
template <int K, int TJ, int TK, bool SPLIT = false>
__global__ void __launch_bounds__(TJ* TK) k_outer_residual_ff(const FFC* __restrict__ C, int n, int chunk,
                                                              const double* __restrict__ u,
                                                              const float* __restrict__ rho,
                                                              float* __restrict__ ub, float* __restrict__ tau,
                                                              double* __restrict__ partials,
                                                              const int* __restrict__ skip = nullptr,
                                                              float* __restrict__ zero_e = nullptr,
                                                              float* __restrict__ zero_q = nullptr) {
  if (skip && *skip) return;
  const FFC c = *C;
  const double a = outer_residual_tile_ff<K, TJ, TK, SPLIT>(c, n, chunk, u, rho, ub, tau, blockIdx.x, blockIdx.y,
                                                            zero_e, zero_q);
  if (threadIdx.x == 0) partials[blockIdx.x + blockIdx.y * gridDim.x] = a;
}

// The start from the background field (its first element NaN on entry): the
// residual at the uniform field ubar is formed without reading or writing the
// field, which keeps its NaN mark; the first correction writes ubar + e over it
// (k_apply_correction<true>), or the solve fills it with ubar if it ends before
// one.  k_background_first raises the flag, after every CTA has read cell 0.  There the six-neighbour sum of w
// equals 6w exactly, so r = N(ubar) is the source term alone, which the
// float-float operations of outer_residual_tile_ff give to the same accuracy:
//   f(R): c1 rho + c0 - K/ubar;  symmetron: -msym ((rho/mean rat3 - 1) ubar + ubar^3).
// Writes ub = float(ubar), tau = -float(r) in the level's layout and one
// partial sum of tau^2 per CTA, for a grid of the general kernel's shape.
// When the field is not NaN-marked it returns at once (the general kernel runs).
template <int K, bool SPLIT>
__global__ void __launch_bounds__(256) k_background_residual_ff(const FFC* __restrict__ C, int n,
                                                                const double* __restrict__ u, double ubar,
                                                                const float* __restrict__ rho,
                                                                float* __restrict__ ub, float* __restrict__ tau,
                                                                double* __restrict__ partials,
                                                                float* __restrict__ zero_e = nullptr,
                                                                float* __restrict__ zero_q = nullptr) {
  static_assert(K != KCQ, "CQ keeps the FP64 residual");
  if (!isnan(u[0])) return;
  const FFC c = *C;
  const ff uc = ff_from_double(ubar);
  const float ubf = ff_to_float(uc);
  const int nb = gridDim.x * gridDim.y;
  const int b = blockIdx.x + blockIdx.y * gridDim.x;
  const int rows = n * n;
  const ff Kdu = ff_div(c.K, uc);              // f(R): K / ubar, the same in every cell
  const ff ub3 = ff_mul(ff_sqr(uc), uc);       // symmetron: ubar^3
  float acc = 0.f;
  // rows (i, j) over the CTAs, k over the threads: one division per row
  for (int row = b; row < rows; row += nb) {
    const int i = row / n, j = row - i * n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const long long t = (long long)row * n + k;
      const float r = rho[t];
      float tv;
      if constexpr (is_fr(K)) {
        ffacc v = acc_of(c.c0);
        const ff p1 = two_prod(c.c1.hi, r);
        acc_add(v, p1.hi, __fmaf_rn(c.c1.lo, r, p1.lo));
        acc_add(v, -Kdu.hi, -Kdu.lo);
        tv = -acc_float(v);
      } else {
        const ff a = ff_sub(ff_mul(ff_mul_f(c.c1, r), c.rat3), ff{1.f, 0.f});
        tv = ff_to_float(ff_mul(c.msym, ff_add(ff_mul(a, uc), ub3)));
      }
      const long long o = SPLIT ? split_idx(n, i, j, k) : t;
      ub[o] = ubf;
      tau[o] = tv;
      if (zero_e) zero_e[o] = 0.f;
      if (zero_q) zero_q[o] = 0.f;
      acc += tv * tv;
    }
  }
  const double a = block_sum((double)acc);
  if (threadIdx.x == 0) partials[b] = a;
}

// k_background_residual_ff with four consecutive cells a thread (n % 4 == 0,
// rho 16-byte aligned): one 16-byte density load a thread, and on a split
// level two 8-byte stores per colour
// array (cells 4m, 4m + 2 and 4m + 1, 4m + 3 of a row sit at 2m, 2m + 1 of the
// two colours).  Same per-cell arithmetic; grid as the general kernel's.
template <int K, bool SPLIT>
__global__ void __launch_bounds__(256) k_background_residual_ff4(const FFC* __restrict__ C, int n,
                                                                 const double* __restrict__ u, double ubar,
                                                                 const float* __restrict__ rho,
                                                                 float* __restrict__ ub, float* __restrict__ tau,
                                                                 double* __restrict__ partials,
                                                                 float* __restrict__ zero_e = nullptr,
                                                                 float* __restrict__ zero_q = nullptr) {
  static_assert(K != KCQ, "CQ keeps the FP64 residual");
  if (!isnan(u[0])) return;
  const FFC c = *C;
  const ff uc = ff_from_double(ubar);
  const float ubf = ff_to_float(uc);
  const int nb = gridDim.x * gridDim.y;
  const int b = blockIdx.x + blockIdx.y * gridDim.x;
  const int rows = n * n, h = n >> 1;
  const unsigned q = (unsigned)(n >> 2), quads = (unsigned)rows * q;  // 32-bit index: <= 2^30 for n <= 2048
  const long long H = (long long)rows * h;
  const ff Kdu = ff_div(c.K, uc);         // f(R): K / ubar, the same in every cell
  const ff ub3 = ff_mul(ff_sqr(uc), uc);  // symmetron: ubar^3
  auto resid = [&](float r) -> float {
    if constexpr (is_fr(K)) {
      ffacc v = acc_of(c.c0);
      const ff p1 = two_prod(c.c1.hi, r);
      acc_add(v, p1.hi, __fmaf_rn(c.c1.lo, r, p1.lo));
      acc_add(v, -Kdu.hi, -Kdu.lo);
      return -acc_float(v);
    } else {
      const ff a = ff_sub(ff_mul(ff_mul_f(c.c1, r), c.rat3), ff{1.f, 0.f});
      return ff_to_float(ff_mul(c.msym, ff_add(ff_mul(a, uc), ub3)));
    }
  };
  float acc = 0.f;
  for (unsigned Q = (unsigned)b * blockDim.x + threadIdx.x; Q < quads; Q += (unsigned)nb * blockDim.x) {
    const int row = (int)(Q / q), m = (int)(Q - (unsigned)row * q);
    const long long t = (long long)row * n + 4 * m;
    const float4 r4 = *reinterpret_cast<const float4*>(rho + t);
    const float t0 = resid(r4.x), t1 = resid(r4.y), t2 = resid(r4.z), t3 = resid(r4.w);
    if constexpr (SPLIT) {
      const int i = row / n, j = row - i * n;
      const long long idx = (long long)row * h + 2 * m;
      const int c0 = (i + j) & 1;  // colour of cell 4m
      const long long a = c0 ? H + idx : idx, o = c0 ? idx : H + idx;
      *reinterpret_cast<float2*>(ub + idx) = make_float2(ubf, ubf);
      *reinterpret_cast<float2*>(ub + H + idx) = make_float2(ubf, ubf);
      *reinterpret_cast<float2*>(tau + a) = make_float2(t0, t2);
      *reinterpret_cast<float2*>(tau + o) = make_float2(t1, t3);
      if (zero_e) {
        *reinterpret_cast<float2*>(zero_e + idx) = make_float2(0.f, 0.f);
        *reinterpret_cast<float2*>(zero_e + H + idx) = make_float2(0.f, 0.f);
      }
      if (zero_q) {
        *reinterpret_cast<float2*>(zero_q + idx) = make_float2(0.f, 0.f);
        *reinterpret_cast<float2*>(zero_q + H + idx) = make_float2(0.f, 0.f);
      }
    } else {
      *reinterpret_cast<float4*>(ub + t) = make_float4(ubf, ubf, ubf, ubf);
      *reinterpret_cast<float4*>(tau + t) = make_float4(t0, t1, t2, t3);
    }
    acc += t0 * t0;
    acc += t1 * t1;
    acc += t2 * t2;
    acc += t3 * t3;
  }
  const double a = block_sum((double)acc);
  if (threadIdx.x == 0) partials[b] = a;
}

// The flag that tells the general residual kernel its work is done, and the
// host that the field still holds the background mark (flag = 0 when the
// caller gave an initial field).
static __global__ void k_background_first(const double* __restrict__ u, int* __restrict__ flag) {
  *flag = isnan(u[0]) ? 1 : 0;
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
  const float im = (float)((double)n3 / *sum);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    out[t] = rho[t] * im;
}

// rho32 normalised to mean 1 into a red-black split fine level (n % 8 == 0).
static __global__ void k_density_norm32_split(const float* __restrict__ rho, int n, const double* __restrict__ sum,
                                              float* __restrict__ out) {
  const long long n3 = (long long)n * n * n;
  const float im = (float)((double)n3 / *sum);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(t % n), j = (int)((t / n) % n), i = (int)(t / ((long long)n * n));
    out[split_idx(n, i, j, k)] = rho[t] * im;
  }
}

// 8-child mean from a split fine level into a natural coarse level.
static __global__ void __launch_bounds__(128) k_restrict32_from_split(int nf, const float* __restrict__ fine,
                                                                      float* __restrict__ coarse) {
  const int nc = nf >> 1;
  const int I = blockIdx.z, J = blockIdx.y;
  const int Kc = blockIdx.x * blockDim.x + threadIdx.x;
  if (Kc >= nc) return;
  float s = 0.f;
  for (int di = 0; di < 2; ++di)
    for (int dj = 0; dj < 2; ++dj)
      for (int dk = 0; dk < 2; ++dk) s += fine[split_idx(nf, 2 * I + di, 2 * J + dj, 2 * Kc + dk)];
  coarse[cidx(nc, I, J, Kc)] = 0.125f * s;
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
  // a normalisation scale: single precision per cell is ample.  delta =
  // rho/mean - 1 is formed with an FMA against the two-float 1/mean, so it
  // keeps its relative precision where rho is close to the mean.
  const double inv_mean = (double)n3 / *rho_sum;
  const float im_hi = (float)inv_mean, im_lo = (float)(inv_mean - (double)im_hi);
  float acc = 0.f;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    const float r = rho32[t];
    const float delta = fmaf(r, im_hi, -1.f) + r * im_lo;
    acc = fmaf(delta, delta, acc);
  }
  double f;
  if constexpr (is_fr(K)) f = m.om_a;
  else if constexpr (K == KSYM) f = m.msym * m.rat3 * m.ubar;
  else f = m.cq_src;
  const double a = block_sum((double)acc * (f * f));
  if (threadIdx.x == 0) partials[blockIdx.x] = a;
}

static __global__ void k_finalize_sum32(const double* __restrict__ partials, int count, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partials[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}


}  // namespace mg
