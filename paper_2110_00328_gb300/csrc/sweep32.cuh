// sweep32.cuh -- the FP32 correction-form nonlinear Gauss-Seidel sweep, both
// colours fused in one pass over the level (the hot kernel of the mixed path).
//
// Work decomposition: a CTA owns a TJ x TK tile of (j,k) columns and a chunk
// of planes [i0, i1) along i (the slowest index).  It marches up the chunk
// keeping a ring of four planes in shared memory, each with a two-cell halo in
// j and k.  At step s it loads plane s+1 (old values), updates the first
// colour ((i+j+k) even, the paper's first sweep) on plane s over the tile plus
// a one-cell ring, then the second colour on plane s-1 over the tile.  The ring
// cells' first-colour values are recomputed from old values exactly as their
// owner computes them, so each CTA sees the true red-black ordering.  All
// reads come from e_in and all writes go to e_out (ping-pong), so no CTA can
// observe another's new values: the result equals one red-black sweep for
// any CTA schedule.
//
// Per cell the stencil uses a precomputed neighbour quantity q (f(R): Delta w
// = (u+e)^{n+1} - u^{n+1}; symmetron, CQ: e), refreshed whenever e changes.
#pragma once
#include "mg_common.cuh"

namespace mg {

// FP32 constants of one level (correction form).
struct LevelF {
  float c2_h2;   // c~^2 / h^2
  float al;      // f(R): h^2 / (6 c~^2); symmetron: g = c~^2 xi^2 / (h^2 a^2)
  float K;       // f(R): Rbar a^2/3 * ubar
  float alK;     // f(R): al * K
  float msym;    // symmetron a^2/(2 xi^2)
  float rat3;    // symmetron (a_star/a)^3
  float ih2;     // 1/h^2
  float fr_s;    // f(R): s = (al K)^{1/(n+2)}, the root's natural scale
  float fr_is1;  // f(R): 1 / s^{n+1}
  float cq_src, cq_pot, alpha, phibar, inv_c2, beta;
  int keep_exp;
};

// ---- fast single-precision building blocks ----
// The PTX approximate instructions with subnormals flushed (.ftz): one special-
// function-unit operation each, no subnormal rescaling around it.  Every value
// they see in the local solve is a normal float (fields, corrections and their
// squares stay far above 1e-38), and the exact Newton polish that follows each
// closed-form start removes their few-ulp errors.
// reciprocal, relative error below 2^-23
__device__ __forceinline__ float frcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float fdiv(float a, float b) { return a * frcp(b); }
// x^{1/3} for x > 0 as 2^(log2(x)/3): absolute error of the base-2 log below
// 2^-22, so the result carries ~1e-7 relative error
__device__ __forceinline__ float fcbrt_pos(float x) {
  float l, y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
  l *= (1.0f / 3.0f);
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(l));
  return y;
}
// sqrt(max(x, 0))
__device__ __forceinline__ float fsqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(fmaxf(x, 0.f)));
  return y;
}
// sqrt(x) for x known to be >= 0
__device__ __forceinline__ float fsqrt_nn(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Newton polishing steps after the closed-form start of the local solve.  The
// start inherits the single-precision cancellation in the polynomial's
// coefficient p (-u^{n+1} + al K/u - B): in strongly screened cells its
// relative error reaches ~1e-4, which two steps (error squared twice) remove.
// With one step (or one Halley step) the mixed solve stalls: above 1e-8 on the
// 256^3, |fR0| = 1e-6 workload, above 1e-11 on small meshes.
constexpr int kPolishSteps = 2;

// Delta w = (u+e)^{n+1} - u^{n+1}, factored so that small e loses nothing.
template <int K>
__device__ __forceinline__ float dw(float u, float e) {
  if constexpr (K == KFR0) return e;
  else if constexpr (K == KFR1) return e * (2.f * u + e);
  else return e * (3.f * u * u + 3.f * u * e + e * e);
}

// Neighbour quantity of a cell in the stencil sum.
template <int K>
__device__ __forceinline__ float nbq(float u, float e) {
  if constexpr (is_fr(K)) return dw<K>(u, e);
  else return e;
}

// Positive root y of y^{m} + p y - 1 = 0 (m = n+2) by the closed forms of
// Sec. 3.2.5 in fast single precision, as the start for the exact polish.
template <int K>
__device__ __forceinline__ float fr_root_scaled_fast(float p) {
  if constexpr (K == KFR0) {
    // y^2 + p y - 1 = 0
    const float s = fsqrt(p * p + 4.f);
    return p > 0.f ? fdiv(2.f, p + s) : 0.5f * (s - p);
  } else if constexpr (K == KFR1) {
    // y^3 + p y - 1 = 0, D = 1/4 + (p/3)^3
    const float p3 = p * (1.f / 3.f);
    const float D = 0.25f + p3 * p3 * p3;
    if (D >= 0.f) {
      const float A = fcbrt_pos(0.5f + fsqrt_nn(D));
      const float B = fdiv(p3, A);
      return frcp(A * A + p3 + B * B);
    }
    // three real roots: the largest lies in [sqrt(3) r, 2 r), r = sqrt(-p/3);
    // Newton from 2r converges monotonically (P convex there).  Three steps
    // (error <= 15% -> ~1e-6): with two, the solves to 1e-11 stall.
    float y = 2.f * fsqrt_nn(-p3);
#pragma unroll
    for (int it = 0; it < 3; ++it) y -= fdiv((y * y + p) * y - 1.f, 3.f * y * y + p);
    return y;
  } else {
    // y^4 + p y - 1 = 0 (Eq. fR_quartic_solns with q = -1): Delta0 = -12, Delta1 = 27 p^2
    if (p == 0.f) return 1.f;
    const float d1 = 27.f * p * p;
    const float a = fcbrt_pos(0.5f * (fsqrt(d1 * d1 + 6912.f) + d1));
    const float b = fdiv(12.f, a);
    const float S = fsqrt(fdiv(d1, 12.f * (a * a + a * b + b * b)));
    if (p > 0.f) {
      const float r2 = fdiv(p, 4.f * S) - S * S;
      const float xc = fdiv(r2 - S * S, fsqrt(fmaxf(r2, 0.f)) + S);
      const float xl = frcp(p);
      return (xc > 0.f && xc < xl) ? xc : xl;
    }
    return S + fsqrt(fmaxf(fdiv(-p, 4.f * S) - S * S, 0.f));
  }
}

// Symmetron total-field root of U^3 + p U + q = 0 with the sign rule of the
// FP64 path, fast single precision (start for the polish).
__device__ __forceinline__ float sym_root_fast(float p, float q, float u_old) {
  if (q == 0.f) return p >= 0.f ? 0.f : (u_old < 0.f ? -fsqrt(-p) : fsqrt(-p));
  const float sg = q < 0.f ? 1.f : -1.f;
  const float hq = 0.5f * fabsf(q);
  const float p3 = p * (1.f / 3.f);
  const float D = hq * hq + p3 * p3 * p3;
  float x;
  if (D >= 0.f) {
    const float A = fcbrt_pos(hq + fsqrt(D));
    const float B = fdiv(p3, A);
    x = fdiv(hq + hq, A * A + p3 + B * B);
  } else {
    const float aq = -2.f * hq;  // q of the positive-side problem
    x = 2.f * fsqrt_nn(-p3);
#pragma unroll
    for (int it = 0; it < 3; ++it) x -= fdiv((x * x + p) * x + aq, 3.f * x * x + p);
  }
  return sg * x;
}

// Nonlinear Gauss-Seidel update of the correction e at one cell.
//  u: base field, e: current correction, rho: density (symmetron/CQ), s: source,
//  Lnb: sum of the six neighbours' nbq.
template <int K>
__device__ __forceinline__ float update_e_fast(const LevelF& f, float u, float e, float rho, float s, float Lnb) {
  if constexpr (is_fr(K)) {
    // total-field polynomial U^{n+2} + p U - al K = 0, p = -u^{n+1} + al K/u - B
    const float B = Lnb * (1.f / 6.f) + f.al * s;
    const float p = -fr_w<K>(u) + f.alK * frcp(u) - B;
    const float U = f.fr_s * fr_root_scaled_fast<K>(p * f.fr_is1);
    float x = U - u;
    // Newton steps on G(x) = Delta w(x) + al K x/(u(u+x)) - B (no cancellation
    // in x) bring x to single-precision relative accuracy.  From the closed-form
    // start (relative error <= ~1e-4) they stay on the positive branch; should
    // the result not be a positive total field, the closed-form root is kept.
    const float ru = frcp(u);
    const float x0 = x;
#pragma unroll
    for (int it = 0; it < kPolishSteps; ++it) {
      const float Ue = u + x;
      const float rU = frcp(Ue);
      const float G = dw<K>(u, x) + f.alK * x * ru * rU - B;
      float dG = f.alK * rU * rU;
      if constexpr (K == KFR0) dG += 1.f;
      else if constexpr (K == KFR1) dG += 2.f * Ue;
      else dG += 3.f * Ue * Ue;
      x -= fdiv(G, dG);
    }
    return (u + x > 0.f) ? x : x0;
  } else if constexpr (K == KSYM) {
    const float p = rho * f.rat3 - 1.f + 12.f * f.al;
    const float B = 2.f * f.al * Lnb - fdiv(s, f.msym);
    const float q = -(p * u + u * u * u + B);
    const float U = sym_root_fast(p, q, u + e);
    float x = U - u;
#pragma unroll
    for (int it = 0; it < kPolishSteps; ++it) {
      const float G = p * x + x * (3.f * u * u + 3.f * u * x + x * x) - B;
      const float Ue = u + x;
      const float dG = p + 3.f * Ue * Ue;
      x = dG != 0.f ? x - fdiv(G, dG) : x;
    }
    return x;
  } else {
    // Newton-Gauss-Seidel step (Eq. relaxation_iteration) on M(e) - s
    const float x0 = f.phibar + u * f.inv_c2;
    const float dpow = powf(x0, -1.f - f.alpha) * expm1f((-1.f - f.alpha) * log1pf(e * f.inv_c2 / x0));
    float r = (Lnb - 6.f * e) * f.ih2 + f.cq_pot * dpow - s;
    const float x = x0 + e * f.inv_c2;
    float dr = -6.f * f.ih2 - f.cq_pot * (1.f + f.alpha) * powf(x, -2.f - f.alpha) * f.inv_c2;
    if (f.keep_exp) {
      const float Eu = expf(f.beta * u * f.inv_c2);
      r -= f.cq_src * rho * Eu * expm1f(f.beta * e * f.inv_c2);
      dr -= f.cq_src * rho * f.beta * f.inv_c2 * Eu * expf(f.beta * e * f.inv_c2);
    }
    return e - r / dr;
  }
}

// Largest Newton step, relative to the current total field u + e, from which
// the warm-started update below finishes without the closed form.
constexpr float kWarmStep = 1e-2f;

// f(R) n = 1, 2 update started from the cell's current correction e.  The
// local root is the zero of G(x) = Delta w(x) + al K x/(u(u+x)) - B, and
// |G''| / (2 G') <= 1/(u+x) on the positive branch, so a Newton step from a
// start that is eps (relative to u + x) from the root leaves at most eps^2.
// When the first step of every lane of the warp is at most kWarmStep (u + e),
// a second step leaves at most eps^4 <= 1e-8: an error of at most ~1e-6 of the
// update itself, which shrinks with it as the iteration converges.  Otherwise
// the warp takes the closed-form start and its polish (update_e_fast).  The
// lanes named in warp_mask (all 32 by default) call this together.
template <int K>
__device__ __forceinline__ float update_e_warm(const LevelF& f, float u, float e, float s, float Lnb,
                                               unsigned warp_mask = 0xffffffffu) {
  static_assert(K == KFR1 || K == KFR2, "warm start: f(R) n = 1, 2");
  const float B = Lnb * (1.f / 6.f) + f.al * s;
  const float c = f.alK * frcp(u);
  // Newton step G/G' with numerator and denominator multiplied by U^2 (U = u + x),
  // so that one reciprocal serves: G U^2 = (Delta w(x) - B) U^2 + (al K/u) x U and
  // G' U^2 = w'(U) U^2 + al K, with w'(U) = 2U (n = 1) or 3U^2 (n = 2).
  auto newton = [&](float x, float* Ue_out) {
    const float Ue = u + x;
    const float U2 = Ue * Ue;
    const float num = fmaf(c * x, Ue, (dw<K>(u, x) - B) * U2);
    float den;
    if constexpr (K == KFR1) den = fmaf(2.f * Ue, U2, f.alK);
    else den = fmaf(3.f * U2, U2, f.alK);
    *Ue_out = Ue;
    return num * frcp(den);
  };
  float Ue;
  const float dx = newton(e, &Ue);
  const bool near = Ue > 0.f && fabsf(dx) <= kWarmStep * Ue;
  if (__all_sync(warp_mask, near)) {
    const float x = e - dx;
    return x - newton(x, &Ue);
  }
  return update_e_fast<K>(f, u, 0.f, 1.f, s, Lnb);
}

// ---------------------------------------------------------------------------
// One colour of a red-black sweep, four consecutive cells per thread
// ---------------------------------------------------------------------------
//
// A warp covers 32 quads (128 cells) of one row (i, j) of a level whose side n
// is a multiple of 4; each lane owns the quad k0 = 4 tq .. k0+3, of which two
// cells have the colour being updated: k0+o and k0+o+2 with o = (i+j+parity)&1.
// The lane reads its quad of e (and u, S, rho) and the same quad of the four
// rows (i, j+-1) and (i+-1, j) as 16-byte loads; the k-neighbours come from the
// lane's own quad except one, which the adjacent lane hands over by a shuffle
// (lanes at a warp or row end load it).  Cells of the other colour are only
// read, so the update is the red-black Gauss-Seidel colour step for any
// schedule.  All 32 lanes of the warp must call this together (the shuffles);
// lanes past the row end (tq >= n/4) work on a clamped quad and store nothing.

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Local update of the quad smoother: f(R) n = 1, 2 warm-started from the cell's
// current correction (update_e_warm, the whole warp together), else the closed
// form (update_e_fast).
template <int K>
__device__ __forceinline__ float update_quad(const LevelF& f, float u, float e, float rho, float s, float Lnb) {
  if constexpr (K == KFR1 || K == KFR2) return update_e_warm<K>(f, u, e, s, Lnb);
  else return update_e_fast<K>(f, u, e, rho, s, Lnb);
}

// WD: also store D = e - Re at the cells this pass updates (the coarse difference
// that the finest level's prolongation then reads in place of e and Re).
// IT: the index type (int where n^3 < 2^31, which shortens the address
// arithmetic every lane runs before its first load).
template <int K, bool WD = false, typename IT = long long>
__device__ __forceinline__ void smooth_quad(const LevelF& f, int n, float* __restrict__ e,
                                            const float* __restrict__ ub, const float* __restrict__ rho,
                                            const float* __restrict__ S, int i, int j, int tq, int lane,
                                            int parity, const float* __restrict__ Re = nullptr,
                                            float* __restrict__ D = nullptr) {
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
  float* e0 = e + c0;
  const float* u0 = ub + c0;
  const float4 E = ld4(e0), U = ld4(u0), Sv = ld4(S + c0);
  const float4 Ejp = ld4(e0 + djp), Ejm = ld4(e0 + djm), Eip = ld4(e0 + dip), Eim = ld4(e0 + dim);
  float4 Ujp = make_float4(0.f, 0.f, 0.f, 0.f), Ujm = Ujp, Uip = Ujp, Uim = Ujp;
  if constexpr (FR) {
    Ujp = ld4(u0 + djp);
    Ujm = ld4(u0 + djm);
    Uip = ld4(u0 + dip);
    Uim = ld4(u0 + dim);
  }
  float4 R = make_float4(1.f, 1.f, 1.f, 1.f);
  if constexpr (RHO) {
    if (rho) R = ld4(rho + c0);  // CQ without the exponential coupling passes no density
  }
  float4 Rq = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (WD) Rq = ld4(Re + c0);
  if (((i + j + parity) & 1) == 0) {
    // cells k0 (x) and k0+2 (z); k-neighbours k0-1 (previous lane's w), y, w
    const float qy = nbq<K>(U.y, E.y), qw = nbq<K>(U.w, E.w);
    float qm = __shfl_up_sync(0xffffffffu, qw, 1);
    if (lane == 0) {
      const IT cm = c0 + (k0 == 0 ? n - 1 : -1);
      qm = nbq<K>(FR ? ub[cm] : 0.f, e[cm]);
    }
    const float LA = (qm + qy) + (nbq<K>(Ujp.x, Ejp.x) + nbq<K>(Ujm.x, Ejm.x)) +
                     (nbq<K>(Uip.x, Eip.x) + nbq<K>(Uim.x, Eim.x));
    const float LB = (qy + qw) + (nbq<K>(Ujp.z, Ejp.z) + nbq<K>(Ujm.z, Ejm.z)) +
                     (nbq<K>(Uip.z, Eip.z) + nbq<K>(Uim.z, Eim.z));
    const float eA = update_quad<K>(f, U.x, E.x, R.x, Sv.x, LA);
    const float eB = update_quad<K>(f, U.z, E.z, R.z, Sv.z, LB);
    if (act) {
      e0[0] = eA;
      e0[2] = eB;
      if constexpr (WD) {
        D[c0] = eA - Rq.x;
        D[c0 + 2] = eB - Rq.z;
      }
    }
  } else {
    // cells k0+1 (y) and k0+3 (w); k-neighbours x, z, k0+4 (next lane's x)
    const float qx = nbq<K>(U.x, E.x), qz = nbq<K>(U.z, E.z);
    float qp = __shfl_down_sync(0xffffffffu, qx, 1);
    if (lane == 31 || tq + 1 >= nq) {
      const IT cp = c0 + (k0 + 4 == n ? 4 - n : 4);
      qp = nbq<K>(FR ? ub[cp] : 0.f, e[cp]);
    }
    const float LA = (qx + qz) + (nbq<K>(Ujp.y, Ejp.y) + nbq<K>(Ujm.y, Ejm.y)) +
                     (nbq<K>(Uip.y, Eip.y) + nbq<K>(Uim.y, Eim.y));
    const float LB = (qz + qp) + (nbq<K>(Ujp.w, Ejp.w) + nbq<K>(Ujm.w, Ejm.w)) +
                     (nbq<K>(Uip.w, Eip.w) + nbq<K>(Uim.w, Eim.w));
    const float eA = update_quad<K>(f, U.y, E.y, R.y, Sv.y, LA);
    const float eB = update_quad<K>(f, U.w, E.w, R.w, Sv.w, LB);
    if (act) {
      e0[1] = eA;
      e0[3] = eB;
      if constexpr (WD) {
        D[c0 + 1] = eA - Rq.y;
        D[c0 + 3] = eB - Rq.w;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Red-black split layout (the finest level)
// ---------------------------------------------------------------------------
//
// A level of side n (n % 8 == 0) stores each colour contiguously: cell
// (i, j, k) of colour c = (i+j+k) & 1 at c H + (i n + j) h + k/2, with h = n/2
// and H = n^2 h.  A colour pass then reads only that colour's u and S and the
// other colour's e and u (its neighbours): ~10 bytes a cell instead of the
// ~14 a pass over interleaved colours moves.  The neighbours (i, j+-1, k) and
// (i+-1, j, k) of a cell sit at the same k/2 of the other colour's adjacent
// rows; (i, j, k+-1) at k/2 - 1 + p and k/2 + p of the same row, p = k & 1.

__device__ __forceinline__ long long split_idx(int n, int i, int j, int k) {
  const int h = n >> 1;
  return (long long)((i + j + k) & 1) * ((long long)n * n * h) + ((long long)i * n + j) * h + (k >> 1);
}

__device__ __forceinline__ float2 ld2s(const float* p) { return *reinterpret_cast<const float2*>(p); }

// The interleaved quad k0 .. k0+3 (k0 % 4 == 0) of row (i, j) of a split array.
__device__ __forceinline__ float4 ld4_split(const float* a, int n, int i, int j, int k0) {
  const int h = n >> 1;
  const long long H = (long long)n * n * h, r = ((long long)i * n + j) * h + (k0 >> 1);
  const float2 b = ld2s(a + r), q = ld2s(a + H + r);
  return ((i + j) & 1) ? make_float4(q.x, b.x, q.y, b.y) : make_float4(b.x, q.x, b.y, q.y);
}

__device__ __forceinline__ void st4_split(float* a, int n, int i, int j, int k0, float4 v) {
  const int h = n >> 1;
  const long long H = (long long)n * n * h, r = ((long long)i * n + j) * h + (k0 >> 1);
  float2 b, q;
  if ((i + j) & 1) {
    q = make_float2(v.x, v.z);
    b = make_float2(v.y, v.w);
  } else {
    b = make_float2(v.x, v.z);
    q = make_float2(v.y, v.w);
  }
  *reinterpret_cast<float2*>(a + r) = b;
  *reinterpret_cast<float2*>(a + H + r) = q;
}

// Lane -> (row, position in row) of a split-level colour pass over np planes:
// rows of nq = n/8 lanes packed 32/nq to a warp (nq <= 32), or spread over
// ceil(nq/32) warps.  Lanes with nothing to do get act = false and a valid
// (clamped) cell, since all 32 lanes take part in the pass's shuffles.
__device__ __forceinline__ void split_lane(int n, int np, long long warp, int lane, long long* r, int* seg,
                                           bool* act) {
  const int nq = n >> 3;
  const long long rows = (long long)np * n;
  if (nq <= 32) {
    const bool pow2 = (nq & (nq - 1)) == 0;  // shifts instead of divisions (the usual meshes)
    const int sh = __ffs(nq) - 1;
    const int per = pow2 ? 32 >> sh : 32 / nq, sub = pow2 ? lane >> sh : lane / nq;
    *r = warp * per + sub;
    *seg = lane - sub * nq;
    *act = sub < per;
    if (!*act) {
      *r = warp * per + per - 1;
      *seg = nq - 1;
    }
  } else {
    const int W = (nq + 31) / 32;
    *r = warp / W;
    *seg = (int)(warp % W) * 32 + lane;
    *act = *seg < nq;
    if (!*act) *seg = nq - 1;
  }
  if (*r >= rows) {
    *r = rows - 1;
    *act = false;
  }
}

// Warps of one split-level colour pass over np planes.
static inline long long split_warps(int n, int np) {
  const int nq = n >> 3;
  const long long rows = (long long)np * n;
  if (nq <= 32) {
    const int per = 32 / nq;
    return (rows + per - 1) / per;
  }
  return rows * ((nq + 31) / 32);
}

// Access to a level as interleaved quads: natural layout or red-black split.
struct NatLayout {
  using index_t = long long;
  static __device__ __forceinline__ float4 q(const float* a, int n, int i, int j, int k0) {
    return ld4(a + ((long long)i * n + j) * n + k0);
  }
  static __device__ __forceinline__ void st(float* a, int n, int i, int j, int k0, float4 v) {
    *reinterpret_cast<float4*>(a + ((long long)i * n + j) * n + k0) = v;
  }
  static __device__ __forceinline__ long long idx(int n, int i, int j, int k) { return ((long long)i * n + j) * n + k; }
};
// NatLayout with 32-bit offsets, for levels with n^3 < 2^31 (n <= 1024 here).
struct NatLayout32 {
  using index_t = int;
  static __device__ __forceinline__ float4 q(const float* a, int n, int i, int j, int k0) {
    return ld4(a + (i * n + j) * n + k0);
  }
  static __device__ __forceinline__ void st(float* a, int n, int i, int j, int k0, float4 v) {
    *reinterpret_cast<float4*>(a + (i * n + j) * n + k0) = v;
  }
  static __device__ __forceinline__ int idx(int n, int i, int j, int k) { return (i * n + j) * n + k; }
};
struct SplitLayout {
  using index_t = long long;
  static __device__ __forceinline__ float4 q(const float* a, int n, int i, int j, int k0) {
    return ld4_split(a, n, i, j, k0);
  }
  static __device__ __forceinline__ void st(float* a, int n, int i, int j, int k0, float4 v) {
    st4_split(a, n, i, j, k0, v);
  }
  static __device__ __forceinline__ long long idx(int n, int i, int j, int k) { return split_idx(n, i, j, k); }
};

// One colour pass on a split level: a lane owns four consecutive cells
// m0 .. m0+3 (k = 2m + p, p = (i+j+colour) & 1) of the colour being updated
// in row (i, j).  Rows are packed into warps in segments of nq = n/8 lanes
// ('seg' = the lane's position in its row, 'nq' lanes per row; a row longer
// than a warp continues in the next warp); all 32 lanes call this together
// (the shuffles), idle lanes with act = false and a valid (clamped) cell.  Reads: the
// colour's u, S (and e, rho where the model uses them) at m0 .. m0+3, the other
// colour's e and u at m0 .. m0+3 of the same row and of the rows (i, j+-1),
// (i+-1, j); the one k-neighbour outside that window comes from the adjacent
// lane (p = 0: m0 - 1; p = 1: m0 + 4), or a load at a row end.
//
// Stored neighbour quantity (QS, f(R) n = 1, 2): the level also keeps
// q = Delta w(u, e) of every cell in the same layout, written with e by the
// pass that updates the cell (and by the prolongation for the second colour).
// A pass then reads the other colour's q instead of its e and u -- five rows
// of loads and five Delta w evaluations fewer per cell, the same DRAM bytes
// (q written beside e).  q is formed by the same expression from the same
// values, so the sweep computes what it computes without it, up to where the
// compiler fuses a product into the neighbouring sum.
// IT: the index type of the cell offsets (int where 2 n^2 (n/2) < 2^31).
template <int K, bool QS = false, int FRESH = 0, typename IT = long long>
__device__ __forceinline__ void smooth_split(const LevelF& f, int n, float* __restrict__ e,
                                             const float* __restrict__ ub, const float* __restrict__ rho,
                                             const float* __restrict__ S, int i, int j, int seg, bool act,
                                             int colour, int lane, float* __restrict__ q = nullptr, int pdl = 0) {
  constexpr bool FR = is_fr(K);
  static_assert(!QS || K == KFR1 || K == KFR2, "the stored neighbour quantity differs from e for f(R) n = 1, 2 only");
  constexpr bool RHO = (K == KSYM) || (K == KCQ);
  const int h = n >> 1, nq = h >> 2;
  const int m0 = 4 * seg;
  const IT H = (IT)n * n * h;
  const IT r0 = ((IT)i * n + j) * h + m0;
  const IT djp = (j + 1 < n) ? (IT)h : -(IT)(n - 1) * h;
  const IT djm = (j > 0) ? -(IT)h : (IT)(n - 1) * h;
  const IT nh = (IT)n * h;
  const IT dip = (i + 1 < n) ? nh : -(IT)(n - 1) * nh;
  const IT dim = (i > 0) ? -nh : (IT)(n - 1) * nh;
  const int p = (i + j + colour) & 1;
  float* eo = e + (IT)colour * H + r0;               // own colour
  const float* e1 = e + (IT)(colour ^ 1) * H + r0;   // other colour
  const float* uo = ub + (IT)colour * H + r0;
  const float* u1 = ub + (IT)(colour ^ 1) * H + r0;
  if constexpr (QS) {
    // pdl (programmatic dependent launch): 1 = the previous kernel is a colour
    // pass, which writes only its own colour's e and q, so this colour's u and S
    // (constant through the sweeps) are loaded before waiting for it; 2 = wait
    // first.  The next pass may start only once every CTA here has waited, so
    // when its own early loads run, every kernel before this one has finished.
    // The colour's own e (the Newton start of update_e_warm) is written only by
    // passes of this colour and by the prolongation, both finished by then.
    // FRESH (the first sweep of an inner solve, whose correction starts at
    // zero): bit 0, this colour's e is zero and is not read; bit 1, the other
    // colour's q = Delta w(u, 0) is zero too and is not read.  The result is the
    // one the zero arrays would give.
    const float* q1 = q + (IT)(colour ^ 1) * H + r0;  // other colour's q
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pdl == 2) asm volatile("griddepcontrol.wait;" ::: "memory");
    const float4 U = ld4(uo), Sv = ld4(S + (IT)colour * H + r0), E = (FRESH & 1) ? z4 : ld4(eo);
    if (pdl == 1) asm volatile("griddepcontrol.wait;" ::: "memory");
    if (pdl) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    float4 Q = z4, Qjp = z4, Qjm = z4, Qip = z4, Qim = z4;
    if constexpr (!(FRESH & 2)) {
      Q = ld4(q1);
      Qjp = ld4(q1 + djp);
      Qjm = ld4(q1 + djm);
      Qip = ld4(q1 + dip);
      Qim = ld4(q1 + dim);
    }
    float qm = __shfl_up_sync(0xffffffffu, Q.w, 1);
    float qp = __shfl_down_sync(0xffffffffu, Q.x, 1);
    if constexpr (!(FRESH & 2)) {
      if (p == 0 && (seg == 0 || lane == 0)) qm = q1[m0 == 0 ? h - 1 : -1];
      if (p == 1 && (seg == nq - 1 || lane == 31)) qp = q1[m0 + 4 == h ? 4 - h : 4];
    }
    const float k0s = p ? Q.x + Q.y : qm + Q.x;
    const float k1s = p ? Q.y + Q.z : Q.x + Q.y;
    const float k2s = p ? Q.z + Q.w : Q.y + Q.z;
    const float k3s = p ? Q.w + qp : Q.z + Q.w;
    const float L0 = k0s + (Qjp.x + Qjm.x) + (Qip.x + Qim.x);
    const float L1 = k1s + (Qjp.y + Qjm.y) + (Qip.y + Qim.y);
    const float L2 = k2s + (Qjp.z + Qjm.z) + (Qip.z + Qim.z);
    const float L3 = k3s + (Qjp.w + Qjm.w) + (Qip.w + Qim.w);
    float4 out;
    out.x = update_e_warm<K>(f, U.x, E.x, Sv.x, L0);
    out.y = update_e_warm<K>(f, U.y, E.y, Sv.y, L1);
    out.z = update_e_warm<K>(f, U.z, E.z, Sv.z, L2);
    out.w = update_e_warm<K>(f, U.w, E.w, Sv.w, L3);
    if (act) {
      *reinterpret_cast<float4*>(eo) = out;
      *reinterpret_cast<float4*>(q + (IT)colour * H + r0) =
          make_float4(nbq<K>(U.x, out.x), nbq<K>(U.y, out.y), nbq<K>(U.z, out.z), nbq<K>(U.w, out.w));
    }
    return;
  }
  const float4 U = ld4(uo), Sv = ld4(S + (IT)colour * H + r0);
  float4 E = make_float4(0.f, 0.f, 0.f, 0.f);
  if constexpr (!FR) E = ld4(eo);
  float4 R = make_float4(1.f, 1.f, 1.f, 1.f);
  if constexpr (RHO) {
    if (rho) R = ld4(rho + (IT)colour * H + r0);
  }
  const float4 Er = ld4(e1);
  const float4 Ejp = ld4(e1 + djp), Ejm = ld4(e1 + djm), Eip = ld4(e1 + dip), Eim = ld4(e1 + dim);
  float4 Ur = make_float4(0.f, 0.f, 0.f, 0.f), Ujp = Ur, Ujm = Ur, Uip = Ur, Uim = Ur;
  if constexpr (FR) {
    Ur = ld4(u1);
    Ujp = ld4(u1 + djp);
    Ujm = ld4(u1 + djm);
    Uip = ld4(u1 + dip);
    Uim = ld4(u1 + dim);
  }
  const float4 Q = make_float4(nbq<K>(Ur.x, Er.x), nbq<K>(Ur.y, Er.y), nbq<K>(Ur.z, Er.z), nbq<K>(Ur.w, Er.w));
  float qm = __shfl_up_sync(0xffffffffu, Q.w, 1);    // other colour at m0 - 1
  float qp = __shfl_down_sync(0xffffffffu, Q.x, 1);  // other colour at m0 + 4
  if (p == 0 && (seg == 0 || lane == 0)) {
    const IT c = r0 + (m0 == 0 ? h - 1 : -1);
    qm = nbq<K>(FR ? ub[(IT)(colour ^ 1) * H + c] : 0.f, e[(IT)(colour ^ 1) * H + c]);
  }
  if (p == 1 && (seg == nq - 1 || lane == 31)) {
    const IT c = r0 + (m0 + 4 == h ? 4 - h : 4);
    qp = nbq<K>(FR ? ub[(IT)(colour ^ 1) * H + c] : 0.f, e[(IT)(colour ^ 1) * H + c]);
  }
  // the two k-neighbours of own cell t: other-colour m0+t-1+p and m0+t+p
  const float k0s = p ? Q.x + Q.y : qm + Q.x;
  const float k1s = p ? Q.y + Q.z : Q.x + Q.y;
  const float k2s = p ? Q.z + Q.w : Q.y + Q.z;
  const float k3s = p ? Q.w + qp : Q.z + Q.w;
  const float L0 = k0s + (nbq<K>(Ujp.x, Ejp.x) + nbq<K>(Ujm.x, Ejm.x)) + (nbq<K>(Uip.x, Eip.x) + nbq<K>(Uim.x, Eim.x));
  const float L1 = k1s + (nbq<K>(Ujp.y, Ejp.y) + nbq<K>(Ujm.y, Ejm.y)) + (nbq<K>(Uip.y, Eip.y) + nbq<K>(Uim.y, Eim.y));
  const float L2 = k2s + (nbq<K>(Ujp.z, Ejp.z) + nbq<K>(Ujm.z, Ejm.z)) + (nbq<K>(Uip.z, Eip.z) + nbq<K>(Uim.z, Eim.z));
  const float L3 = k3s + (nbq<K>(Ujp.w, Ejp.w) + nbq<K>(Ujm.w, Ejm.w)) + (nbq<K>(Uip.w, Eip.w) + nbq<K>(Uim.w, Eim.w));
  float4 out;
  out.x = update_e_fast<K>(f, U.x, E.x, R.x, Sv.x, L0);
  out.y = update_e_fast<K>(f, U.y, E.y, R.y, Sv.y, L1);
  out.z = update_e_fast<K>(f, U.z, E.z, R.z, Sv.z, L2);
  out.w = update_e_fast<K>(f, U.w, E.w, R.w, Sv.w, L3);
  if (act) *reinterpret_cast<float4*>(eo) = out;
}

// Red-black split fine level (n % 8 == 0), one colour on the planes
// i0 .. i0+np-1 (mod n): rows of n/8 lanes packed into warps (several short rows
// per warp, a long row over several warps), four cells per lane; block (32, 4),
// 1D grid over warps.
// QS: f(R) n = 1, 2 with the neighbour quantity q stored beside e (smooth_split).
template <int K, bool QS = false, int FRESH = 0, typename IT = long long>
__global__ void __launch_bounds__(128, QS ? 10 : 1) k_smooth32s(LevelF f, int n, float* __restrict__ e,
                                                   const float* __restrict__ ub, const float* __restrict__ rho,
                                                   const float* __restrict__ S, int colour, int i0, int np,
                                                   float* __restrict__ q, int pdl) {
  const int lane = threadIdx.x;
  const long long warp = (long long)blockIdx.x * 4 + threadIdx.y;
  long long r;
  int seg;
  bool act;
  split_lane(n, np, warp, lane, &r, &seg, &act);
  const bool pow2 = (n & (n - 1)) == 0;
  const int sh = __ffs(n) - 1;
  int i = i0 + (int)(pow2 ? r >> sh : r / n);
  if (i >= n) i -= n;
  const int j = (int)(pow2 ? r & (n - 1) : r % n);
  smooth_split<K, QS, FRESH, IT>(f, n, e, ub, rho, S, i, j, seg, act, colour, lane, q, pdl);
}

}  // namespace mg

namespace mg {

// ---------------------------------------------------------------------------
// k_sweep32: one full red-black sweep of the correction equation on one level
// ---------------------------------------------------------------------------
//
// Shared-memory plane layout: a (TJ+4) x (TK+4) plane (two-cell halo) stored
// row by row, each row split into its even-k half followed by its odd-k half.
// The cells of one colour in a row then sit at unit stride in one half and
// their k-neighbours at unit stride in the other half, so a warp's accesses are
// free of bank conflicts.  Each thread computes its load and update offsets
// once; only the plane base changes as the CTA marches along i.
template <int K, int TJ, int TK>
__global__ void __launch_bounds__(TJ* TK / 2) k_sweep32(LevelF f, int n, int chunk, const float* __restrict__ e_in,
                                                        float* __restrict__ e_out, const float* __restrict__ ub,
                                                        const float* __restrict__ rho, const float* __restrict__ S) {
  constexpr int PJ = TJ + 4, PK = TK + 4, LS = PJ * PK;  // logical plane with a two-cell halo
  // each row stored as its even-k half then its odd-k half; for f(R) the halves
  // are padded to a 16-bank offset so that the two halves never share a bank
  constexpr int HP0 = PK / 2;
  constexpr int HP = is_fr(K) ? (HP0 <= 16 ? 16 : ((HP0 - 16 + 31) / 32) * 32 + 16) : HP0;
  constexpr int RS = 2 * HP, PS = PJ * RS;  // row stride and stored plane size
  constexpr int NT = TJ * TK / 2;          // threads: one second-colour cell each
  constexpr int NE = (LS + NT - 1) / NT;   // plane elements loaded per thread
  constexpr int RW = (TK + 2) / 2;         // first-colour cells per row of the one-cell ring
  constexpr int NA = ((TJ + 2) * RW + NT - 1) / NT;  // first-colour cells per thread
  constexpr bool FR = is_fr(K);
  constexpr bool RHO = (K == KSYM) || (K == KCQ);
  __shared__ float s_q[4][PS];             // neighbour quantity, planes s-2 .. s+1
  __shared__ float s_u[3][PS];             // base field, planes s-1 .. s+1
  __shared__ float s_s[3][PS];             // source
  __shared__ float s_r[RHO ? 3 : 1][RHO ? PS : 1];

  const int tiles_k = n / TK;
  const int k0 = (blockIdx.x % tiles_k) * TK;
  const int j0 = (blockIdx.x / tiles_k) * TJ;
  const int i0 = blockIdx.y * chunk;
  const int i1 = min(i0 + chunk, n);
  const int t = threadIdx.x;
  const size_t nn = (size_t)n * n;

  // ---- per-thread offsets, computed once ----
  int l_sx[NE];      // split shared index of each loaded element (-1: none)
  int l_g[NE];       // in-plane global offset
  bool l_h1[NE];     // inside the one-cell halo (source/density needed)
#pragma unroll
  for (int m = 0; m < NE; ++m) {
    const int c = t + m * NT;
    l_sx[m] = -1;
    l_g[m] = 0;
    l_h1[m] = false;
    if (c < LS) {
      const int jj = c / PK, kk = c - jj * PK;
      l_sx[m] = jj * RS + (kk >> 1) + (kk & 1) * HP;
      l_g[m] = wrapi(j0 + jj - 2, n) * n + wrapi(k0 + kk - 2, n);
      l_h1[m] = jj >= 1 && jj <= TJ + 2 && kk >= 1 && kk <= TK + 2;
    }
  }
  // first-colour cells on the ring rows: row jj (1..TJ+2) and index q (0..RW-1);
  // kk = 1 + 2q + d with d = parity offset, which alternates with the plane
  int a_jj[NA], a_q[NA], a_d0[NA];
#pragma unroll
  for (int m = 0; m < NA; ++m) {
    const int c = t + m * NT;
    a_jj[m] = -1;
    a_q[m] = 0;
    a_d0[m] = 0;
    if (c < (TJ + 2) * RW) {
      const int r = c / RW;
      a_jj[m] = r + 1;
      a_q[m] = c - r * RW;
      // (i + j + k) even with k = k0 - 1 + 2q + d and i even: d = (j + k0 - 1) & 1
      a_d0[m] = ((j0 + a_jj[m] - 2 + k0 - 1) % 2 + 2) & 1;
    }
  }
  // second-colour cell: row jj = t/(TK/2) + 2, index q = t % (TK/2), kk = 2 + 2q + d
  const int b_jj = t / (TK / 2) + 2, b_q = t % (TK / 2);
  const int b_d0 = (j0 + b_jj - 2 + k0 + 1) & 1;  // for i even: (i + j + k) odd

  float pe[NE], pu[NE], ps[NE], pr[RHO ? NE : 1];
  auto fetch = [&](int p) {
    const int ig = p < 0 ? p + n : (p >= n ? p - n : p);
    const size_t base = (size_t)ig * nn;
#pragma unroll
    for (int m = 0; m < NE; ++m) {
      if (l_sx[m] >= 0) {
        const size_t g = base + l_g[m];
        pe[m] = e_in[g];
        pu[m] = ub[g];
        if (l_h1[m]) {
          ps[m] = S[g];
          if constexpr (RHO) pr[m] = rho ? rho[g] : 1.f;
        }
      }
    }
  };
  auto sl3 = [](int p) { return (p + 6) % 3; };
  auto commit = [&](int p) {
    const int slot = p & 3, s3 = sl3(p);
#pragma unroll
    for (int m = 0; m < NE; ++m) {
      if (l_sx[m] >= 0) {
        s_u[s3][l_sx[m]] = pu[m];
        s_q[slot][l_sx[m]] = nbq<K>(pu[m], pe[m]);
        if (l_h1[m]) {
          s_s[s3][l_sx[m]] = ps[m];
          if constexpr (RHO) s_r[s3][l_sx[m]] = pr[m];
        }
      }
    }
  };
  // relax the cell at row jj, tile column kk of plane p; returns the new correction
  auto relax = [&](int p, int jj, int kk) -> float {
    const int slot = p & 3, sm = (p - 1) & 3, sp = (p + 1) & 3, s3 = sl3(p);
    const int own = jj * RS + (kk >> 1) + (kk & 1) * HP;
    const int oth = jj * RS + (1 - (kk & 1)) * HP;  // other half of the row
    const float Lnb = s_q[sm][own] + s_q[sp][own] + s_q[slot][own - RS] + s_q[slot][own + RS] +
                      s_q[slot][oth + ((kk - 1) >> 1)] + s_q[slot][oth + ((kk + 1) >> 1)];
    float rv = 1.f, eo = 0.f;
    if constexpr (RHO) rv = s_r[s3][own];
    if constexpr (!FR) eo = s_q[slot][own];
    const float uv = s_u[s3][own];
    const float en = update_e_fast<K>(f, uv, eo, rv, s_s[s3][own], Lnb);
    s_q[slot][own] = nbq<K>(uv, en);
    return en;
  };

  fetch(i0 - 2);
  commit(i0 - 2);
  fetch(i0 - 1);
  commit(i0 - 1);
  fetch(i0);
  for (int s = i0 - 1; s <= i1; ++s) {
    commit(s + 1);
    if (s + 2 <= i1 + 1) fetch(s + 2);
    __syncthreads();
    // first colour ((i+j+k) even) on plane s over the tile plus a one-cell ring
    {
      const int ig = s < 0 ? s + n : (s >= n ? s - n : s);
      const bool store = s >= i0 && s < i1;
      const size_t pbase = (size_t)ig * nn;
#pragma unroll
      for (int m = 0; m < NA; ++m) {
        if (a_jj[m] < 0) continue;
        const int kk = 1 + 2 * a_q[m] + (a_d0[m] ^ (ig & 1));
        const float en = relax(s, a_jj[m], kk);
        if (store && a_jj[m] >= 2 && a_jj[m] < TJ + 2 && kk >= 2 && kk < TK + 2)
          e_out[pbase + (size_t)(j0 + a_jj[m] - 2) * n + (k0 + kk - 2)] = en;
      }
    }
    __syncthreads();
    // second colour on plane s-1 over the tile
    if (s - 1 >= i0) {
      const int p = s - 1;
      const int kk = 2 + 2 * b_q + (b_d0 ^ (p & 1));
      const float en = relax(p, b_jj, kk);
      e_out[(size_t)p * nn + (size_t)(j0 + b_jj - 2) * n + (k0 + kk - 2)] = en;
    }
    __syncthreads();
  }
}

}  // namespace mg
