// tail32.cuh -- the coarsest levels of an FP32 correction-form V-cycle in one
// thread block.
//
// Below ~16^3 cells a level's kernels are bound by launch latency, not by work
// (a 16^3 colour pass is 2048 updates).  From the first level with at most
// kTailMaxCells cells down to the coarsest, the whole V-cycle -- pre-smoothing,
// restriction of the defect, FAS source, the coarsest relaxation, prolongation-
// correction and post-smoothing (Sec. 3.2.1) -- runs inside one CTA with the
// levels held in shared memory and __syncthreads() between the steps.  Every
// step applies the same per-cell arithmetic as the one-kernel-per-step path
// (update_e_fast, local_M, the 8-child mean and the 27/9/3/1 prolongation), in
// the same red-black order, so the result is the same iterate.
#pragma once
#include "mixed_common.cuh"

namespace mg {

constexpr int kTailMaxCells = 4096;  // the first tail level has at most this many cells
constexpr int kTailMaxLevels = 6;
constexpr int kTailThreads = 512;

struct TailArgs {
  int T;                              // tail levels (first, ..., coarsest)
  int n[kTailMaxLevels];              // their sides
  LevelF lf[kTailMaxLevels];
  float* e;                           // first tail level, global: correction (in/out)
  const float* ub;                    // base field
  const float* S;                     // FAS source
  const float* rho[kTailMaxLevels];   // density pyramid (nullptr when the operator takes none)
  int nu1, nu2, coarse_sweeps;
  unsigned long long* guard;          // positivity-guard replacements (counted), or nullptr
};

// Shared-memory bytes of a tail: e, u, S per level, R e on all but the first,
// the density where used.
static inline size_t tail_smem_bytes(const TailArgs& A) {
  size_t cells = 0;
  for (int m = 0; m < A.T; ++m) {
    const size_t n3 = (size_t)A.n[m] * A.n[m] * A.n[m];
    cells += n3 * (3 + (m > 0 ? 1 : 0) + (A.rho[m] ? 1 : 0));
  }
  return cells * sizeof(float);
}

// nb_sum_g's sum (same terms, same order) with 32-bit shared-memory offsets.
template <int K>
__device__ __forceinline__ float tail_nb_sum(const float* e, const float* ub, int n, int i, int j, int k) {
  const int nn = n * n, c = (i * n + j) * n + k;
  const int ip = i + 1 < n ? nn : nn - n * nn, im = i > 0 ? -nn : n * nn - nn;
  const int jp = j + 1 < n ? n : n - nn, jm = j > 0 ? -n : nn - n;
  const int kp = k + 1 < n ? 1 : 1 - n, km = k > 0 ? -1 : n - 1;
  const int c0 = c + ip, c1 = c + im, c2 = c + jp, c3 = c + jm, c4 = c + kp, c5 = c + km;
  if constexpr (is_fr(K)) {
    return dw<K>(ub[c0], e[c0]) + dw<K>(ub[c1], e[c1]) + dw<K>(ub[c2], e[c2]) + dw<K>(ub[c3], e[c3]) +
           dw<K>(ub[c4], e[c4]) + dw<K>(ub[c5], e[c5]);
  } else {
    return e[c0] + e[c1] + e[c2] + e[c3] + e[c4] + e[c5];
  }
}

template <int K>
__device__ __forceinline__ void tail_smooth(const LevelF& f, int n, float* e, const float* ub, const float* rho,
                                            const float* S, int sweeps) {
  const int h = n >> 1, half = h * n * n;
  const bool p2 = (n & (n - 1)) == 0;  // power-of-two side: index by shifts
  const int sh = __ffs(n) - 1;
  for (int s = 0; s < sweeps; ++s)
    for (int parity = 0; parity < 2; ++parity) {
      for (int t = threadIdx.x; t < half; t += blockDim.x) {
        int kk, r, j, i;
        if (p2) {
          kk = t & (h - 1), r = t >> (sh - 1), j = r & (n - 1), i = r >> sh;
        } else {
          kk = t % h, r = t / h, j = r % n, i = r / n;
        }
        const int k = 2 * kk + ((i + j + parity) & 1);
        const int c = (i * n + j) * n + k;
        const float Lnb = tail_nb_sum<K>(e, ub, n, i, j, k);
        if constexpr (K == KFR1 || K == KFR2)
          e[c] = update_e_warm<K>(f, ub[c], e[c], S[c], Lnb, __activemask());  // the lanes still in the loop
        else
          e[c] = update_e_fast<K>(f, ub[c], e[c], rho ? rho[c] : 1.f, S[c], Lnb);
      }
      __syncthreads();
    }
}

// d = M(e) - S at the 8 children of each coarse cell, averaged; coarse e starts at R e.
template <int K>
__device__ __forceinline__ void tail_restrict(const LevelF& f, int nf, const float* e, const float* ub,
                                              const float* rho, const float* S, float* Re, float* eH, float* ubH,
                                              float* SH) {
  const int nc = nf >> 1, nc3 = nc * nc * nc;
  for (int t = threadIdx.x; t < nc3; t += blockDim.x) {
    const int Kc = t % nc, J = (t / nc) % nc, I = t / (nc * nc);
    float se = 0.f, su = 0.f, sd = 0.f;
    for (int di = 0; di < 2; ++di)
      for (int dj = 0; dj < 2; ++dj)
        for (int dk = 0; dk < 2; ++dk) {
          const int i = 2 * I + di, j = 2 * J + dj, k = 2 * Kc + dk;
          const int c = (i * nf + j) * nf + k;
          const float ec = e[c], uc = ub[c];
          se += ec;
          su += uc;
          sd += local_M<K>(f, uc, ec, rho ? rho[c] : 1.f, tail_nb_sum<K>(e, ub, nf, i, j, k)) - S[c];
        }
    Re[t] = 0.125f * se;
    eH[t] = 0.125f * se;
    ubH[t] = 0.125f * su;
    SH[t] = 0.125f * sd;
  }
  __syncthreads();
}

// S <- M(Re) - S (S holds R d on entry)
template <int K>
__device__ __forceinline__ void tail_fas(const LevelF& f, int n, const float* Re, const float* ub, const float* rho,
                                         float* S) {
  const int n3 = n * n * n;
  for (int t = threadIdx.x; t < n3; t += blockDim.x) {
    const int k = t % n, j = (t / n) % n, i = t / (n * n);
    S[t] = local_M<K>(f, ub[t], Re[t], rho ? rho[t] : 1.f, tail_nb_sum<K>(Re, ub, n, i, j, k)) - S[t];
  }
  __syncthreads();
}

template <bool FR>
__device__ __forceinline__ void tail_prolong(int nc, const float* eH, const float* Re, const float* ub, float* ef,
                                             unsigned long long* guard) {
  const int nf = nc << 1, nf3 = nf * nf * nf;
  for (int t = threadIdx.x; t < nf3; t += blockDim.x) {
    const int k = t % nf, j = (t / nf) % nf, i = t / (nf * nf);
    const int I = i >> 1, J = j >> 1, Kc = k >> 1;
    const int I2 = wrapi(I + ((i & 1) ? 1 : -1), nc);
    const int J2 = wrapi(J + ((j & 1) ? 1 : -1), nc);
    const int K2 = wrapi(Kc + ((k & 1) ? 1 : -1), nc);
    auto d = [&](int a, int b, int c) {
      const int o = (a * nc + b) * nc + c;
      return eH[o] - Re[o];
    };
    const float corr = (27.f * d(I, J, Kc) + 9.f * (d(I2, J, Kc) + d(I, J2, Kc) + d(I, J, K2)) +
                        3.f * (d(I2, J2, Kc) + d(I2, J, K2) + d(I, J2, K2)) + d(I2, J2, K2)) *
                       (1.f / 64.f);
    const float old = ef[t];
    float v = old + corr;
    if (FR && !(ub[t] + v > 0.f)) {
      v = 0.5f * (old - ub[t]);
      count_guards(guard, 1u);
    }
    ef[t] = v;
  }
  __syncthreads();
}

template <int K>
__global__ void __launch_bounds__(kTailThreads) k_tail32(TailArgs A) {
  extern __shared__ float sm[];
  float *e[kTailMaxLevels], *ub[kTailMaxLevels], *S[kTailMaxLevels], *Re[kTailMaxLevels], *rh[kTailMaxLevels];
  float* p = sm;
  for (int m = 0; m < A.T; ++m) {
    const int n3 = A.n[m] * A.n[m] * A.n[m];
    e[m] = p; p += n3;
    ub[m] = p; p += n3;
    S[m] = p; p += n3;
    Re[m] = nullptr;
    if (m > 0) { Re[m] = p; p += n3; }
    rh[m] = nullptr;
    if (A.rho[m]) { rh[m] = p; p += n3; }
  }
  {
    const int n3 = A.n[0] * A.n[0] * A.n[0];
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
      e[0][t] = A.e[t];
      ub[0][t] = A.ub[t];
      S[0][t] = A.S[t];
    }
    for (int m = 0; m < A.T; ++m)
      if (A.rho[m]) {
        const int nm = A.n[m] * A.n[m] * A.n[m];
        for (int t = threadIdx.x; t < nm; t += blockDim.x) rh[m][t] = A.rho[m][t];
      }
  }
  __syncthreads();
  for (int m = 0; m + 1 < A.T; ++m) {
    tail_smooth<K>(A.lf[m], A.n[m], e[m], ub[m], rh[m], S[m], A.nu1);
    tail_restrict<K>(A.lf[m], A.n[m], e[m], ub[m], rh[m], S[m], Re[m + 1], e[m + 1], ub[m + 1], S[m + 1]);
    tail_fas<K>(A.lf[m + 1], A.n[m + 1], Re[m + 1], ub[m + 1], rh[m + 1], S[m + 1]);
  }
  tail_smooth<K>(A.lf[A.T - 1], A.n[A.T - 1], e[A.T - 1], ub[A.T - 1], rh[A.T - 1], S[A.T - 1], A.coarse_sweeps);
  for (int m = A.T - 2; m >= 0; --m) {
    tail_prolong<is_fr(K)>(A.n[m + 1], e[m + 1], Re[m + 1], ub[m], e[m], A.guard);
    tail_smooth<K>(A.lf[m], A.n[m], e[m], ub[m], rh[m], S[m], A.nu2);
  }
  const int n3 = A.n[0] * A.n[0] * A.n[0];
  for (int t = threadIdx.x; t < n3; t += blockDim.x) A.e[t] = e[0][t];
}

}  // namespace mg
