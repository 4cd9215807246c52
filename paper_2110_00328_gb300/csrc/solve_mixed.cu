// solve_mixed.cu -- the FP32/FP64 mixed-precision solver.
//
// Outer loop (FP64, fine level only): r = N(u64) (Eq. residual_d), the
// convergence test, and u64 += e after each inner solve.
//
// Inner loop (FP32): FAS V-cycles (Sec. 3.2.1) for the correction e = U - u,
// where u = float(u64) is held fixed as a base field and U is the total field.
// Each level solves M(e) = S with M(e) = N(U) - N(u) evaluated in a form
// without cancellation (f(R): Delta w = (u+e)^{n+1} - u^{n+1} factored;
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
// Local solves: f(R) and the symmetron take the closed-form root of the total
// field's local polynomial (Secs. 3.2.4-3.2.5) in fast single precision as a
// starting point, then one Newton step on the cancellation-free correction
// equation, which restores full relative precision of e; CQ takes one Newton
// step (Eq. relaxation_iteration).
#include <math.h>
#include <string.h>

#include <chrono>

#include <mutex>

#include "mg_common.cuh"
#include "mg_internal.h"
#include "mixed_common.cuh"
#include "sweep32.cuh"
#include "tail32.cuh"

namespace mg {

// Level constants, M(e), neighbour sums and the FP64 residual live in mixed_common.cuh.


// The fused sweep kernel k_sweep32 lives in sweep32.cuh.

// ---------------------------------------------------------------------------
// Per-colour sweep for levels the fused kernel does not tile
// ---------------------------------------------------------------------------

template <int K>
__global__ void __launch_bounds__(64) k_smooth32(LevelF f, int n, float* __restrict__ e, const float* __restrict__ ub,
                                                 const float* __restrict__ rho, const float* __restrict__ S,
                                                 int parity) {
  const int i = blockIdx.z, j = blockIdx.y;
  const int kk = blockIdx.x * blockDim.x + threadIdx.x;
  if (kk >= (n >> 1)) return;
  const int k = 2 * kk + ((i + j + parity) & 1);
  const size_t c = cidx(n, i, j, k);
  const float Lnb = nb_sum_g<K>(e, ub, n, i, j, k);
  e[c] = update_e_fast<K>(f, ub[c], e[c], rho ? rho[c] : 1.f, S[c], Lnb);
}

// Quad version (levels with n % 4 == 0) on the planes i0 .. i0+np-1 (mod n):
// block (32, 4) = four rows (i, j), grid (ceil(n/128), n, ceil(np/4)).
template <int K, bool WD = false, typename IT = long long>
__global__ void __launch_bounds__(128) k_smooth32q(LevelF f, int n, float* __restrict__ e,
                                                   const float* __restrict__ ub, const float* __restrict__ rho,
                                                   const float* __restrict__ S, int parity, int i0, int np,
                                                   const float* __restrict__ Re = nullptr,
                                                   float* __restrict__ D = nullptr) {
  const int z = blockIdx.z * 4 + threadIdx.y;
  if (z >= np) return;  // whole warps: z is uniform in a warp
  int i = i0 + z;
  if (i >= n) i -= n;
  smooth_quad<K, WD, IT>(f, n, e, ub, rho, S, i, blockIdx.y, blockIdx.x * 32 + threadIdx.x, threadIdx.x, parity,
                         Re, D);
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
        const float Lnb = nb_sum_g<K>(e, ub, n, i, j, k);
        e[t] = update_e_fast<K>(f, ub[t], e[t], rho ? rho[t] : 1.f, S[t], Lnb);
      }
      __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Transfers (3D grids: x over k, y over j, z over i)
// ---------------------------------------------------------------------------

// For each coarse cell: d = M(e) - S at the 8 children, averaged into Rd (stored
// in SH); the children's e averaged into Re and eH; ub averaged into ubH.
template <int K>
__global__ void __launch_bounds__(128) k_residual_restrict32(LevelF f, int nf, const float* __restrict__ e,
                                                             const float* __restrict__ ub,
                                                             const float* __restrict__ rho,
                                                             const float* __restrict__ S, float* __restrict__ Re,
                                                             float* __restrict__ eH, float* __restrict__ ubH,
                                                             float* __restrict__ SH) {
  const int nc = nf >> 1;
  const int I = blockIdx.z, J = blockIdx.y;
  const int Kc = blockIdx.x * blockDim.x + threadIdx.x;
  if (Kc >= nc) return;
  float se = 0.f, su = 0.f, sd = 0.f;
#pragma unroll
  for (int di = 0; di < 2; ++di)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int dk = 0; dk < 2; ++dk) {
        const int i = 2 * I + di, j = 2 * J + dj, k = 2 * Kc + dk;
        const size_t c = cidx(nf, i, j, k);
        const float ec = e[c], uc = ub[c];
        se += ec;
        su += uc;
        sd += local_M<K>(f, uc, ec, rho ? rho[c] : 1.f, nb_sum_g<K>(e, ub, nf, i, j, k)) - S[c];
      }
  const size_t t = cidx(nc, I, J, Kc);
  Re[t] = 0.125f * se;
  eH[t] = 0.125f * se;
  ubH[t] = 0.125f * su;
  SH[t] = 0.125f * sd;
}

// Quad versions (fine side % 4 == 0): block (32, 4), lanes along k; FL is the
// fine level's layout.  Restriction: grid (ceil(nf/128), nc [J], ceil(nc/4) [I]).
template <int K, class FL = NatLayout, bool QH = false, bool ZR = false>
__global__ void __launch_bounds__(128) k_residual_restrict32q(LevelF f, int nf, const float* __restrict__ e,
                                                              const float* __restrict__ ub,
                                                              const float* __restrict__ rho,
                                                              const float* __restrict__ S, float* __restrict__ Re,
                                                              float* __restrict__ eH, float* __restrict__ ubH,
                                                              float* __restrict__ SH,
                                                              const float* __restrict__ qf) {
  const int I = blockIdx.z * 4 + threadIdx.y;
  if (I >= (nf >> 1)) return;  // whole warps
  restrict_quad<K, FL, QH, ZR>(f, nf, e, ub, rho, S, Re, eH, ubH, SH, I, blockIdx.y, blockIdx.x * 32 + threadIdx.x,
                               threadIdx.x, qf);
}

// Prolongation: grid (ceil(nf/128), nf [j], nf/4 [i]).
template <bool FR, class FL = NatLayout, int QK = -1, bool SECOND_ONLY = false>
__global__ void __launch_bounds__(128) k_prolong_correct32q(int nc, const float* __restrict__ eH,
                                                            const float* __restrict__ Re,
                                                            const float* __restrict__ ub, float* __restrict__ ef,
                                                            unsigned long long* guard,
                                                            float* __restrict__ qf = nullptr) {
  prolong_quad<FR, FL, QK, SECOND_ONLY>(nc, eH, Re, ub, ef, blockIdx.z * 4 + threadIdx.y, blockIdx.y,
                                        blockIdx.x * 32 + threadIdx.x, threadIdx.x, guard, qf);
}

// Second-colour prolongation on a split finest level with stored q, four fine
// rows per lane (prolong_split2x2_second); grid as the restriction's.
template <int QK, bool DD = false, typename IT = long long>
__global__ void __launch_bounds__(128) k_prolong32_split2x2(int nc, const float* __restrict__ eH,
                                                            const float* __restrict__ Re, const float* __restrict__ ub,
                                                            float* __restrict__ ef, unsigned long long* guard,
                                                            float* __restrict__ qf) {
  const int I = blockIdx.z * 4 + threadIdx.y;
  if (I >= nc) return;  // whole warps
  prolong_split2x2_second<QK, DD, IT>(nc, eH, Re, ub, ef, I, blockIdx.y, blockIdx.x * 32 + threadIdx.x,
                                      threadIdx.x, guard, qf);
}

// Restriction after pre-smoothing on a split finest level with stored q, the
// defect formed at the first colour only (restrict_split_zr); grid as above.
template <int K, typename IT = long long>
__global__ void __launch_bounds__(128) k_restrict32_split_zr(LevelF f, int nf, const float* __restrict__ e,
                                                             const float* __restrict__ ub,
                                                             const float* __restrict__ S, const float* __restrict__ qf,
                                                             float* __restrict__ Re, float* __restrict__ eH,
                                                             float* __restrict__ ubH, float* __restrict__ SH) {
  const int I = blockIdx.z * 4 + threadIdx.y;
  if (I >= (nf >> 1)) return;  // whole warps
  restrict_split_zr<K, IT>(f, nf, e, ub, S, qf, Re, eH, ubH, SH, I, blockIdx.y, blockIdx.x * 32 + threadIdx.x,
                           threadIdx.x);
}

// FAS source, four cells per lane (n % 4 == 0, n >= 8): grid (ceil(n/128), n, n/4).
template <int K, typename IT = long long>
__global__ void __launch_bounds__(128) k_fas_source32q(LevelF f, int n, const float* __restrict__ Re,
                                                       const float* __restrict__ ub, const float* __restrict__ rho,
                                                       float* __restrict__ S) {
  fas_quad<K, IT>(f, n, Re, ub, rho, S, blockIdx.z * 4 + threadIdx.y, blockIdx.y, blockIdx.x * 32 + threadIdx.x,
              threadIdx.x);
}

// In place: S <- M^H(Re) - S (S holds R d on entry).
template <int K>
__global__ void __launch_bounds__(128) k_fas_source32(LevelF f, int n, const float* __restrict__ Re,
                                                      const float* __restrict__ ub, const float* __restrict__ rho,
                                                      float* __restrict__ S) {
  const int i = blockIdx.z, j = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const size_t t = cidx(n, i, j, k);
  S[t] = local_M<K>(f, ub[t], Re[t], rho ? rho[t] : 1.f, nb_sum_g<K>(Re, ub, n, i, j, k)) - S[t];
}

// e^h += P(e^H - R e^h); f(R): if u + e would not be positive, e <- (e_old - u)/2
// (the total field halves, as in the FP64 path).
template <bool FR>
__global__ void __launch_bounds__(128) k_prolong_correct32(int nc, const float* __restrict__ eH,
                                                           const float* __restrict__ Re, const float* __restrict__ ub,
                                                           float* __restrict__ ef, unsigned long long* guard) {
  const int nf = nc << 1;
  const int i = blockIdx.z, j = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const int I = i >> 1, J = j >> 1, Kc = k >> 1;
  const int I2 = wrapi(I + ((i & 1) ? 1 : -1), nc);
  const int J2 = wrapi(J + ((j & 1) ? 1 : -1), nc);
  const int K2 = wrapi(Kc + ((k & 1) ? 1 : -1), nc);
#define EH(a, b, c) (eH[cidx(nc, a, b, c)] - Re[cidx(nc, a, b, c)])
  const float corr = (27.f * EH(I, J, Kc) + 9.f * (EH(I2, J, Kc) + EH(I, J2, Kc) + EH(I, J, K2)) +
                      3.f * (EH(I2, J2, Kc) + EH(I2, J, K2) + EH(I, J2, K2)) + EH(I2, J2, K2)) *
                     (1.f / 64.f);
#undef EH
  const size_t t = cidx(nf, i, j, k);
  const float old = ef[t];
  float v = old + corr;
  if (FR && !(ub[t] + v > 0.f)) {
    v = 0.5f * (old - ub[t]);
    count_guards(guard, 1u);
  }
  ef[t] = v;
}


// ---------------------------------------------------------------------------
// FP64 outer-loop kernels (fine level)
// ---------------------------------------------------------------------------

// u64 += e with e in the split layout; BG: u64 = ubar + e (the first correction
// of a solve from the background, whose field still holds only its NaN mark).
// Thread w of row (i, j) takes cells 4w .. 4w+3 (h even), whose corrections sit
// at row h + 2w, 2w+1 of the two colour halves: two 8-byte loads of e and two
// 16-byte accesses of u (16-byte aligned) a thread, grid-stride over all rows.
template <bool BG>
__global__ void k_apply_correction_split(double* __restrict__ u, const float* __restrict__ e, int n, double ubar) {
  const int h = n >> 1;
  const unsigned q = (unsigned)(h >> 1), items = (unsigned)n * (unsigned)n * q;  // <= 2^31 for n <= 2048
  const long long H = (long long)n * n * h;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < items; t += gridDim.x * blockDim.x) {
    const int row = (int)(t / q), w = (int)(t - (unsigned)row * q);
    const int i = row / n, j = row - i * n;
    const long long c0 = ((i + j) & 1) ? H : 0;  // colour half of the even-k cells
    double2* ur = reinterpret_cast<double2*>(u + (long long)row * n) + 2 * w;
    const float2 a = reinterpret_cast<const float2*>(e + c0 + (long long)row * h)[w];
    const float2 b = reinterpret_cast<const float2*>(e + (H - c0) + (long long)row * h)[w];
    double2 lo = BG ? make_double2(ubar, ubar) : ur[0], hi = BG ? make_double2(ubar, ubar) : ur[1];
    lo.x += (double)a.x;
    lo.y += (double)b.x;
    hi.x += (double)a.y;
    hi.y += (double)b.y;
    ur[0] = lo;
    ur[1] = hi;
  }
}

// k_apply_correction_split for a field that is not 16-byte aligned: thread m
// takes the pair k = 2m, 2m+1.
template <bool BG>
__global__ void k_apply_correction_split_scalar(double* __restrict__ u, const float* __restrict__ e, int n,
                                                double ubar) {
  const int h = n >> 1, rows = n * n;
  const long long H = (long long)n * n * h;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int i = row / n, j = row - i * n;
    const long long c0 = ((i + j) & 1) ? H : 0;
    double* ur = u + (long long)row * n;
    const float* ev = e + c0 + (long long)row * h;
    const float* od = e + (H - c0) + (long long)row * h;
    for (int m = threadIdx.x; m < h; m += blockDim.x) {
      ur[2 * m] = (BG ? ubar : ur[2 * m]) + (double)ev[m];
      ur[2 * m + 1] = (BG ? ubar : ur[2 * m + 1]) + (double)od[m];
    }
  }
}

// u64 += e (the correction of one inner solve); BG: u64 = ubar + e.
template <bool BG>
__global__ void k_apply_correction(double* __restrict__ u, const float* __restrict__ e, long long n3, double ubar) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    u[t] = (BG ? ubar : u[t]) + (double)e[t];
}




// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------

#define MG_DISPATCH32(kind, CALL)                                        \
  switch (kind) {                                                        \
    case KFR0: { constexpr int KK = KFR0; CALL; note_launch(1); } break; \
    case KFR1: { constexpr int KK = KFR1; CALL; note_launch(1); } break; \
    case KFR2: { constexpr int KK = KFR2; CALL; note_launch(1); } break; \
    case KSYM: { constexpr int KK = KSYM; CALL; note_launch(1); } break; \
    case KCQ: { constexpr int KK = KCQ; CALL; note_launch(1); } break;   \
    default: return MGGLAM_ERR_ARG;                                      \
  }

static dim3 grid3(int n_k, int n_j, int n_i, int bx) { return dim3((n_k + bx - 1) / bx, n_j, n_i); }
static int bx_for(int n) { return n >= 128 ? 128 : (n < 32 ? 32 : n); }

struct MixedCtx {
  ModelDev m;
  LevelF lf[kMaxLevels];
  Workspace* ws;
  const mgglam_params* prm;
  bool need_rho;
  int chunk;          // planes per CTA of the fused sweep
  const float* rho;   // the caller's density (the float-float residual forms its source from it)
  bool split;         // the finest level in the red-black split layout
  bool ff_resid;      // fine residual in float-float (f(R), symmetron) rather than FP64 (CQ)
  int tail_level;     // first level (>= 1) run by the one-block tail kernel, or -1
  float* qs;          // split f(R) n = 1, 2: the finest level's stored neighbour quantity, else nullptr
  unsigned long long* guard;  // positivity-guard replacements of this solve (workspace scalar)
  const struct L2Window* l2 = nullptr;  // persisting L2 window over qs for the colour passes, or nullptr
  // set: the finest level's e and q were not zeroed for the inner solve that
  // starts next, and its first stored-q sweep takes them as zero (smooth32 clears it)
  bool* fresh = nullptr;
};

static FFC* ffc_of(Workspace* ws) { return reinterpret_cast<FFC*>(ws->scalars + SC_FFC); }

// Fused-sweep tile width along k for a level side n (0 = per-colour kernels).
static int sweep_tile_k(int n) {
  if (n >= 64 && n % 64 == 0) return 64;
  if (n >= 32 && n % 32 == 0) return 32;
  if (n >= 16 && n % 16 == 0) return 16;
  return 0;
}

template <int K, int TK>
static void launch_sweep_t(const MixedCtx& C, int l, const float* rho, cudaStream_t st) {
  constexpr int TJ = 8;
  Level& L = C.ws->lev[l];
  const int chunk = C.chunk < L.n ? C.chunk : L.n;
  dim3 grid((L.n / TK) * (L.n / TJ), (L.n + chunk - 1) / chunk);
  k_sweep32<K, TJ, TK><<<grid, TJ * TK / 2, 0, st>>>(C.lf[l], L.n, chunk, L.e, L.e_alt, L.ub, rho, L.S32);
}

// The fused sweep runs only when the caller asks for it (sweep_chunk > 0) on a
// level its tile divides.  Both kernels are bound by instruction issue on
// GB300 (the local root costs ~120 instructions per cell); measured at 256^3,
// one kernel per colour is ~8% faster than the fused pass, whose ring
// recomputation and per-plane barriers cost more than the DRAM traffic they
// save.
static bool use_fused(const MixedCtx& C, int n) {
  const int tk = sweep_tile_k(n);
  if (!tk || n % 8 != 0) return false;
  return C.prm->sweep_chunk > 0;
}

// Planes per L2 slab of the per-colour sweep on a level of side n (0 = one
// pass per colour), on request only, on levels whose e, u and S (12 bytes a
// cell) do not fit in L2 (n >= 256).
static int slab_planes(const MixedCtx& C, int n) {
  const int P = C.prm->sweep_slab;
  if (P <= 0 || n < 256) return 0;
  return P >= n ? 0 : (P < 2 ? 2 : P);
}

// L2 residency of the stored neighbour quantity q on the split finest level:
// each colour pass reads the other colour's q and writes its own, and the
// restriction reads q of its halo rows, so keeping q in L2 (a persisting
// access-policy window on the colour-pass launches) spares those DRAM round
// trips (measured at 256^3: 60.6 instead of 66.7 us per sweep, 37 instead of
// 43 us per restriction).  The L2 set-aside for persisting lines
// (cudaLimitPersistingL2CacheSize, a per-context setting) takes that capacity
// from every other kernel of the process, so a solve raises it to the size of
// q only for its own duration and restores the previous value at its end
// (with its persisting lines returned to normal status); meshes whose q does
// not fit in the device's persisting capacity go without.
struct L2Window {
  bool ok = false;
  cudaAccessPolicyWindow w = {};
  size_t prev_limit = 0;  // the set-aside before the solve
};

// Device capacities, read once per device.
struct L2Caps {
  int state = 0;  // 0 unknown, 1 usable, -1 not offered
  size_t max_persist = 0, max_window = 0;
};
static bool l2_caps(int dev, L2Caps* out) {
  static std::mutex mu;
  static L2Caps caps[64];
  if (dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lk(mu);
  L2Caps& c = caps[dev];
  if (c.state == 0) {
    int mp = 0, mw = 0;
    const bool got = cudaDeviceGetAttribute(&mp, cudaDevAttrMaxPersistingL2CacheSize, dev) == cudaSuccess &&
                     cudaDeviceGetAttribute(&mw, cudaDevAttrMaxAccessPolicyWindowSize, dev) == cudaSuccess;
    if (!got) cudaGetLastError();
    c.state = got && mp > 0 && mw > 0 ? 1 : -1;
    c.max_persist = (size_t)mp;
    c.max_window = (size_t)mw;
  }
  *out = c;
  return c.state > 0;
}

// At the start of a solve: the window over q and the raised set-aside, if q fits.
static L2Window q_window_begin(const MixedCtx& C) {
  L2Window r;
  if (!C.qs) return r;
  int dev = 0;
  L2Caps caps;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return r;
  }
  if (!l2_caps(dev, &caps)) return r;
  const size_t bytes = C.ws->lev[0].n3 * sizeof(float);
  if (bytes > caps.max_persist || bytes > caps.max_window) return r;
  if (cudaDeviceGetLimit(&r.prev_limit, cudaLimitPersistingL2CacheSize) != cudaSuccess ||
      (r.prev_limit < bytes && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes) != cudaSuccess)) {
    cudaGetLastError();
    return r;
  }
  r.w.base_ptr = C.qs;
  r.w.num_bytes = bytes;
  r.w.hitRatio = 1.f;
  r.w.hitProp = cudaAccessPropertyPersisting;
  r.w.missProp = cudaAccessPropertyStreaming;
  r.ok = true;
  return r;
}

// At the end of a solve (every return path): q's lines back to normal, the
// set-aside as it was.
struct L2Scope {
  L2Window w;
  explicit L2Scope(const L2Window& v) : w(v) {}
  L2Scope(const L2Scope&) = delete;
  L2Scope& operator=(const L2Scope&) = delete;
  ~L2Scope() {
    if (!w.ok) return;
    cudaCtxResetPersistingL2Cache();
    size_t now = 0;
    if (cudaDeviceGetLimit(&now, cudaLimitPersistingL2CacheSize) == cudaSuccess && now != w.prev_limit)
      cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, w.prev_limit);
    cudaGetLastError();
  }
};

// wd: the last sweep's passes also store D = e - Re (smooth_quad's WD) in the
// level's second buffer, for the finest level's prolongation (fine_reads_d).
static int smooth32(const MixedCtx& C, int l, int sweeps, cudaStream_t st, bool wd = false) {
  Level& L = C.ws->lev[l];
  const float* rho = C.need_rho ? L.rho32 : nullptr;
  const int tk = sweep_tile_k(L.n);
  const bool fused = use_fused(C, L.n);
  int passes = 0;  // stored-q colour passes launched so far in this call
  for (int s = 0; s < sweeps; ++s) {
    const bool first_fresh = l == 0 && C.qs && C.fresh && *C.fresh;
    if (fused && L.e_alt) {
      switch (tk) {
        case 64: MG_DISPATCH32(C.m.kind, (launch_sweep_t<KK, 64>(C, l, rho, st))); break;
        case 32: MG_DISPATCH32(C.m.kind, (launch_sweep_t<KK, 32>(C, l, rho, st))); break;
        default: MG_DISPATCH32(C.m.kind, (launch_sweep_t<KK, 16>(C, l, rho, st))); break;
      }
      float* tmp = L.e;
      L.e = L.e_alt;
      L.e_alt = tmp;
    } else if (L.n % 4 == 0 && L.n >= 16) {
      const int P = slab_planes(C, L.n);
      const bool split = l == 0 && C.split;
      auto colour = [&](int parity, int i0, int np) -> int {
        if (np <= 0) return MGGLAM_OK;
        if (split) {
          const unsigned blocks = (unsigned)((split_warps(L.n, np) + 3) / 4);
          if (C.qs) {
            // programmatic dependent launch: a pass overlaps its start with the
            // previous pass's last wave (the first pass of the call waits first)
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(blocks);
            cfg.blockDim = dim3(32, 4);
            cfg.stream = st;
            cudaLaunchAttribute attr[2];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (C.l2 && C.l2->ok) {
              attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
              attr[1].val.accessPolicyWindow = C.l2->w;
              cfg.numAttrs = 2;
            }
            const int pdl = passes++ > 0 ? 1 : 2;
            const float *ubc = L.ub, *Sc = L.S32, *no_rho = nullptr;
            // the first sweep from e = 0: the first colour reads neither e nor the
            // other colour's q, the second not its own e
            const int fresh = first_fresh ? (parity == 0 ? 3 : 1) : 0;
            auto go = [&](auto kern) {
              return cudaLaunchKernelEx(&cfg, kern, C.lf[l], L.n, L.e, ubc, no_rho, Sc, parity, i0, np, C.qs, pdl);
            };
            const bool f1 = C.m.kind == KFR1, i32 = L.n <= 1024;  // 32-bit cell offsets where n^3 <= 2^30
            if (fresh == 3)
              MG_CUDA_TRY(f1 ? go(i32 ? k_smooth32s<KFR1, true, 3, int> : k_smooth32s<KFR1, true, 3>)
                             : go(i32 ? k_smooth32s<KFR2, true, 3, int> : k_smooth32s<KFR2, true, 3>));
            else if (fresh == 1)
              MG_CUDA_TRY(f1 ? go(i32 ? k_smooth32s<KFR1, true, 1, int> : k_smooth32s<KFR1, true, 1>)
                             : go(i32 ? k_smooth32s<KFR2, true, 1, int> : k_smooth32s<KFR2, true, 1>));
            else
              MG_CUDA_TRY(f1 ? go(i32 ? k_smooth32s<KFR1, true, 0, int> : k_smooth32s<KFR1, true>)
                             : go(i32 ? k_smooth32s<KFR2, true, 0, int> : k_smooth32s<KFR2, true>));
            note_launch(1);
            return MGGLAM_OK;
          }
          MG_DISPATCH32(C.m.kind, (k_smooth32s<KK><<<blocks, dim3(32, 4), 0, st>>>(C.lf[l], L.n, L.e, L.ub, rho,
                                                                                   L.S32, parity, i0, np, nullptr, 0)));
          return MGGLAM_OK;
        }
        const dim3 g((L.n / 4 + 31) / 32, L.n, (np + 3) / 4);
        const bool i32 = L.n <= 1024;  // n^3 <= 2^30: 32-bit cell offsets
        if (wd && s == sweeps - 1) {
          MG_DISPATCH32(C.m.kind, (k_smooth32q<KK, true, int><<<g, dim3(32, 4), 0, st>>>(
                                       C.lf[l], L.n, L.e, L.ub, rho, L.S32, parity, i0, np, L.Re, L.e_alt)));
        } else if (i32) {
          MG_DISPATCH32(C.m.kind, (k_smooth32q<KK, false, int><<<g, dim3(32, 4), 0, st>>>(
                                       C.lf[l], L.n, L.e, L.ub, rho, L.S32, parity, i0, np)));
        } else {
          MG_DISPATCH32(C.m.kind, (k_smooth32q<KK><<<g, dim3(32, 4), 0, st>>>(C.lf[l], L.n, L.e, L.ub, rho, L.S32,
                                                                              parity, i0, np)));
        }
        return MGGLAM_OK;
      };
      if (P <= 0) {
        colour(0, 0, L.n);
        colour(1, 0, L.n);
      } else {
        // first colour on planes [a, a+P), then the second colour on the planes
        // whose first-colour neighbours are all final, one plane behind; planes
        // n-1 and 0 (which see each other periodically) last
        for (int a = 0; a < L.n; a += P) {
          const int b = a + P < L.n ? a + P : L.n;
          colour(0, a, b - a);
          const int r0 = a == 0 ? 1 : a - 1;
          colour(1, r0, (b - 1) - r0);
        }
        colour(1, L.n - 1, 2);
      }
    } else {
      const dim3 g = grid3(L.n / 2, L.n, L.n, 64);
      for (int parity = 0; parity < 2; ++parity)
        MG_DISPATCH32(C.m.kind, (k_smooth32<KK><<<g, 64, 0, st>>>(C.lf[l], L.n, L.e, L.ub, rho, L.S32, parity)));
    }
    if (first_fresh) *C.fresh = false;
  }
  return MGGLAM_OK;
}

static int vcycle32(const MixedCtx& C, int l, cudaStream_t st, int mode);

// Whether the finest level's second-colour prolongation reads the coarse
// difference eH - Re that level 1's last post-smoothing sweep stores in its
// second buffer (unused there: the split layout excludes the fused sweep): a
// split f(R) n = 1, 2 finest level with post-smoothing, whose level 1 is smoothed
// by the quad kernel (neither the coarsest, a tail, nor slab-scheduled).
static bool fine_reads_d(const MixedCtx& C) {
  const Workspace* ws = C.ws;
  if (!(C.split && C.qs && C.prm->nu2 >= 1 && ws->nlev > 2 && C.tail_level != 1)) return false;
  const int n1 = ws->lev[1].n;
  return n1 % 4 == 0 && n1 >= 16 && !use_fused(C, n1) && slab_planes(C, n1) == 0 && ws->lev[1].e_alt;
}

// The FAS source on level l (natural layout).
static int fas_source(const MixedCtx& C, int l, cudaStream_t st) {
  Level& H = C.ws->lev[l];
  const float* rhoH = C.need_rho ? H.rho32 : nullptr;
  if (H.n % 4 == 0 && H.n >= 8) {
    const dim3 g((H.n / 4 + 31) / 32, H.n, H.n / 4);
    if (H.n <= 1024) {  // 32-bit cell offsets
      MG_DISPATCH32(C.m.kind,
                    (k_fas_source32q<KK, int><<<g, dim3(32, 4), 0, st>>>(C.lf[l], H.n, H.Re, H.ub, rhoH, H.S32)));
    } else {
      MG_DISPATCH32(C.m.kind, (k_fas_source32q<KK><<<g, dim3(32, 4), 0, st>>>(C.lf[l], H.n, H.Re, H.ub, rhoH, H.S32)));
    }
  } else {
    const int bh = bx_for(H.n);
    MG_DISPATCH32(C.m.kind, (k_fas_source32<KK><<<grid3(H.n, H.n, H.n, bh), bh, 0, st>>>(C.lf[l], H.n, H.Re, H.ub,
                                                                                        rhoH, H.S32)));
  }
  return MGGLAM_OK;
}

// Coarse-grid correction seen from the finest level: the FAS source on level 1
// and the cycle(s) on levels >= 1 (V: one; W: two W; F: F then V), enqueued directly.
static int coarse_part_direct(const MixedCtx& C, cudaStream_t st) {
  int rc = fas_source(C, 1, st);
  if (rc) return rc;
  const int mode = C.prm->cycle;
  rc = vcycle32(C, 1, st, mode);
  if (rc || mode == 0) return rc;
  return vcycle32(C, 1, st, mode == 2 ? 2 : 0);
}

// Signature of everything the coarse graph bakes in (kernel constants and the
// cycle shape); buffers are fixed per workspace.
static unsigned long long coarse_signature(const MixedCtx& C) {
  unsigned long long h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  };
  mix(&C.m.kind, sizeof(int));
  mix(C.lf, sizeof(LevelF) * C.ws->nlev);
  const int shape[8] = {C.prm->nu1, C.prm->nu2, C.prm->coarse_sweeps, C.chunk, C.need_rho ? 1 : 0,
                        C.prm->sweep_slab, C.tail_level, C.prm->cycle};
  mix(shape, sizeof(shape));
  const int forced = C.prm->sweep_chunk > 0;
  mix(&forced, sizeof(int));
  return h;
}

// The coarse part as one CUDA graph launch: the ~10 small kernels per level on
// levels >= 1 are launch-rate bound when enqueued one by one.  The graph is
// captured once per parameter signature on a private stream and replayed on
// the caller's stream; if capture fails, or the cycle would not leave the
// ping-pong buffers as it found them, the kernels are enqueued directly.
static int coarse_part(const MixedCtx& C, cudaStream_t st) {
  Workspace* ws = C.ws;
  const unsigned long long sig = coarse_signature(C);
  if (!(ws->coarse_exec && ws->coarse_sig == sig)) {
    if (ws->coarse_exec) {
      cudaGraphExecDestroy(ws->coarse_exec);
      ws->coarse_exec = nullptr;
    }
    if (!ws->cap_stream && cudaStreamCreateWithFlags(&ws->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return coarse_part_direct(C, st);
    }
    float* e0[kMaxLevels];
    float* ea0[kMaxLevels];
    for (int l = 0; l < ws->nlev; ++l) { e0[l] = ws->lev[l].e; ea0[l] = ws->lev[l].e_alt; }
    const long long n0 = launch_count();
    cudaGraph_t g = nullptr;
    int rc = MGGLAM_OK;
    bool ok = cudaStreamBeginCapture(ws->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      rc = coarse_part_direct(C, ws->cap_stream);
      ok = cudaStreamEndCapture(ws->cap_stream, &g) == cudaSuccess && rc == MGGLAM_OK && g != nullptr;
    }
    const long long captured = launch_count() - n0;
    note_launch((int)-captured);  // nothing ran during capture
    bool same = true;
    for (int l = 0; l < ws->nlev; ++l) same = same && ws->lev[l].e == e0[l] && ws->lev[l].e_alt == ea0[l];
    if (ok && same) ok = cudaGraphInstantiate(&ws->coarse_exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    for (int l = 0; l < ws->nlev; ++l) { ws->lev[l].e = e0[l]; ws->lev[l].e_alt = ea0[l]; }
    if (!ok || !same) {
      if (ws->coarse_exec) cudaGraphExecDestroy(ws->coarse_exec);
      ws->coarse_exec = nullptr;
      return coarse_part_direct(C, st);
    }
    ws->coarse_sig = sig;
    ws->coarse_launches = captured;
  }
  MG_CUDA_TRY(cudaGraphLaunch(ws->coarse_exec, st));
  note_launch((int)ws->coarse_launches);
  return MGGLAM_OK;
}

// Levels tail_level .. coarsest in one CTA (tail32.cuh).
template <int K>
static void launch_tail_t(const TailArgs& A, cudaStream_t st) {
  k_tail32<K><<<1, kTailThreads, tail_smem_bytes(A), st>>>(A);
}

static int launch_tail(const MixedCtx& C, int l, cudaStream_t st) {
  Workspace* ws = C.ws;
  TailArgs A;
  memset(&A, 0, sizeof(A));
  A.T = ws->nlev - l;
  for (int m = 0; m < A.T; ++m) {
    A.n[m] = ws->lev[l + m].n;
    A.lf[m] = C.lf[l + m];
    A.rho[m] = C.need_rho ? ws->lev[l + m].rho32 : nullptr;
  }
  A.e = ws->lev[l].e;
  A.ub = ws->lev[l].ub;
  A.S = ws->lev[l].S32;
  A.nu1 = C.prm->nu1;
  A.nu2 = C.prm->nu2;
  A.coarse_sweeps = C.prm->coarse_sweeps;
  A.guard = C.guard;
  MG_DISPATCH32(C.m.kind, (launch_tail_t<KK>(A, st)));
  return MGGLAM_OK;
}

// The tail's shared memory can exceed the 48 KB default (at most ~94 KB).
static void tail_allow_smem() {
  const int bytes = 96 * 1024;
  cudaFuncSetAttribute(k_tail32<KFR0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_tail32<KFR1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_tail32<KFR2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_tail32<KSYM>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_tail32<KCQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// The natural-layout restriction after pre-smoothing (ZR), per model kind.
template <class FL, bool ZR>
static void launch_restrict_nat(const MixedCtx& C, int l, const float* rho, dim3 g, cudaStream_t st) {
  Level& L = C.ws->lev[l];
  Level& H = C.ws->lev[l + 1];
  switch (C.m.kind) {
    case KFR0: k_residual_restrict32q<KFR0, FL, false, ZR><<<g, dim3(32, 4), 0, st>>>(
                   C.lf[l], L.n, L.e, L.ub, rho, L.S32, H.Re, H.e, H.ub, H.S32, nullptr); break;
    case KFR1: k_residual_restrict32q<KFR1, FL, false, ZR><<<g, dim3(32, 4), 0, st>>>(
                   C.lf[l], L.n, L.e, L.ub, rho, L.S32, H.Re, H.e, H.ub, H.S32, nullptr); break;
    case KFR2: k_residual_restrict32q<KFR2, FL, false, ZR><<<g, dim3(32, 4), 0, st>>>(
                   C.lf[l], L.n, L.e, L.ub, rho, L.S32, H.Re, H.e, H.ub, H.S32, nullptr); break;
    default: k_residual_restrict32q<KSYM, FL, false, ZR><<<g, dim3(32, 4), 0, st>>>(
                   C.lf[l], L.n, L.e, L.ub, rho, L.S32, H.Re, H.e, H.ub, H.S32, nullptr); break;
  }
}

// Residual and restriction from level l to l+1: H.Re = R e, H.e = R e (the coarse
// start), H.ub = R ub, H.S32 = R (M(e) - S); the FAS source follows (fas_source).
// relaxed: the level's second colour was the last one relaxed (pre-smoothing
// ran), so on a split finest level with stored q the defect is formed at the
// first colour only (restrict_split_zr).
static int restrict_level(const MixedCtx& C, int l, cudaStream_t st, bool relaxed = false) {
  Workspace* ws = C.ws;
  Level& L = ws->lev[l];
  const float* rho = C.need_rho ? L.rho32 : nullptr;
  Level& H = ws->lev[l + 1];
  const int bh = bx_for(H.n);
  if (l == 0 && C.split) {
    const dim3 g((L.n / 4 + 31) / 32, H.n, (H.n + 3) / 4);
    if (C.qs && relaxed) {
      // 32-bit cell offsets where the level has at most 2^30 cells
      auto kern = C.m.kind == KFR1 ? (L.n <= 1024 ? k_restrict32_split_zr<KFR1, int> : k_restrict32_split_zr<KFR1>)
                                   : (L.n <= 1024 ? k_restrict32_split_zr<KFR2, int> : k_restrict32_split_zr<KFR2>);
      kern<<<g, dim3(32, 4), 0, st>>>(C.lf[l], L.n, L.e, L.ub, L.S32, C.qs, H.Re, H.e, H.ub, H.S32);
      note_launch(1);
    } else if (C.qs && C.m.kind == KFR1) {
      k_residual_restrict32q<KFR1, SplitLayout, true><<<g, dim3(32, 4), 0, st>>>(C.lf[l], L.n, L.e, L.ub, rho, L.S32,
                                                                                 H.Re, H.e, H.ub, H.S32, C.qs);
      note_launch(1);
    } else if (C.qs) {
      k_residual_restrict32q<KFR2, SplitLayout, true><<<g, dim3(32, 4), 0, st>>>(C.lf[l], L.n, L.e, L.ub, rho, L.S32,
                                                                                 H.Re, H.e, H.ub, H.S32, C.qs);
      note_launch(1);
    } else {
      MG_DISPATCH32(C.m.kind, (k_residual_restrict32q<KK, SplitLayout><<<g, dim3(32, 4), 0, st>>>(
                                   C.lf[l], L.n, L.e, L.ub, rho, L.S32, H.Re, H.e, H.ub, H.S32, nullptr)));
    }
  } else if (L.n % 4 == 0 && L.n >= 8) {
    const dim3 g((L.n / 4 + 31) / 32, H.n, (H.n + 3) / 4);
    // 32-bit cell offsets where n^3 < 2^31
    if (relaxed && C.m.kind != KCQ) {
      if (L.n <= 1024) launch_restrict_nat<NatLayout32, true>(C, l, rho, g, st);
      else launch_restrict_nat<NatLayout, true>(C, l, rho, g, st);
      note_launch(1);
    } else {
      if (L.n <= 1024) {
        MG_DISPATCH32(C.m.kind, (k_residual_restrict32q<KK, NatLayout32><<<g, dim3(32, 4), 0, st>>>(
                                     C.lf[l], L.n, L.e, L.ub, rho, L.S32, H.Re, H.e, H.ub, H.S32, nullptr)));
      } else {
        MG_DISPATCH32(C.m.kind, (k_residual_restrict32q<KK><<<g, dim3(32, 4), 0, st>>>(
                                     C.lf[l], L.n, L.e, L.ub, rho, L.S32, H.Re, H.e, H.ub, H.S32, nullptr)));
      }
    }
  } else {
    MG_DISPATCH32(C.m.kind, (k_residual_restrict32<KK><<<grid3(H.n, H.n, H.n, bh), bh, 0, st>>>(
                                 C.lf[l], L.n, L.e, L.ub, rho, L.S32, H.Re, H.e, H.ub, H.S32)));
  }
  return MGGLAM_OK;
}

// Coarse-grid correction of level l from l+1 (e += P(H.e - H.Re)).  both: correct
// both colours of a split finest level even when post-smoothing follows.
static int prolong_level(const MixedCtx& C, int l, cudaStream_t st, bool both = false) {
  Workspace* ws = C.ws;
  Level& L = ws->lev[l];
  Level& H = ws->lev[l + 1];
  const int bf = bx_for(L.n);
  if (l == 0 && C.split) {
    const dim3 g((L.n / 4 + 31) / 32, L.n, L.n / 4);
    // with post-smoothing the first colour's corrections would be overwritten unread (prolong_quad)
    const bool second_only = !both && C.prm->nu2 >= 1;
    const dim3 g2((L.n / 4 + 31) / 32, H.n, (H.n + 3) / 4);
    const bool dd = second_only && fine_reads_d(C);  // H.e_alt holds eH - Re
    const bool i32 = L.n <= 1024;  // 32-bit cell offsets
    if (C.qs && C.m.kind == KFR1 && dd)
      (i32 ? k_prolong32_split2x2<KFR1, true, int> : k_prolong32_split2x2<KFR1, true>)<<<g2, dim3(32, 4), 0, st>>>(
          H.n, H.e_alt, H.Re, L.ub, L.e, C.guard, C.qs);
    else if (C.qs && C.m.kind == KFR2 && dd)
      (i32 ? k_prolong32_split2x2<KFR2, true, int> : k_prolong32_split2x2<KFR2, true>)<<<g2, dim3(32, 4), 0, st>>>(
          H.n, H.e_alt, H.Re, L.ub, L.e, C.guard, C.qs);
    else if (C.qs && C.m.kind == KFR1 && second_only)
      k_prolong32_split2x2<KFR1><<<g2, dim3(32, 4), 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard, C.qs);
    else if (C.qs && C.m.kind == KFR2 && second_only)
      k_prolong32_split2x2<KFR2><<<g2, dim3(32, 4), 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard, C.qs);
    else if (C.qs && C.m.kind == KFR1)
      k_prolong_correct32q<true, SplitLayout, KFR1><<<g, dim3(32, 4), 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard,
                                                                                C.qs);
    else if (C.qs)
      k_prolong_correct32q<true, SplitLayout, KFR2><<<g, dim3(32, 4), 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard,
                                                                                C.qs);
    else if (is_fr(C.m.kind))
      k_prolong_correct32q<true, SplitLayout><<<g, dim3(32, 4), 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard);
    else k_prolong_correct32q<false, SplitLayout><<<g, dim3(32, 4), 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard);
  } else if (L.n % 4 == 0 && L.n >= 8) {
    const dim3 g((L.n / 4 + 31) / 32, L.n, L.n / 4);
    const bool i32 = L.n <= 1024;  // 32-bit cell offsets
    if (is_fr(C.m.kind) && i32)
      k_prolong_correct32q<true, NatLayout32><<<g, dim3(32, 4), 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard);
    else if (is_fr(C.m.kind))
      k_prolong_correct32q<true><<<g, dim3(32, 4), 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard);
    else if (i32)
      k_prolong_correct32q<false, NatLayout32><<<g, dim3(32, 4), 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard);
    else
      k_prolong_correct32q<false><<<g, dim3(32, 4), 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard);
  } else if (is_fr(C.m.kind)) {
    k_prolong_correct32<true><<<grid3(L.n, L.n, L.n, bf), bf, 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard);
  } else {
    k_prolong_correct32<false><<<grid3(L.n, L.n, L.n, bf), bf, 0, st>>>(H.n, H.e, H.Re, L.ub, L.e, C.guard);
  }
  note_launch(1);
  return MGGLAM_OK;
}

// One multigrid cycle from level l: mode 0 V, 1 F, 2 W (Sec. 3.2.1).
static int vcycle32(const MixedCtx& C, int l, cudaStream_t st, int mode) {
  Workspace* ws = C.ws;
  Level& L = ws->lev[l];
  const float* rho = C.need_rho ? L.rho32 : nullptr;
  int rc;
  if (l == C.tail_level) return launch_tail(C, l, st);
  if (l == ws->nlev - 1) {
    if ((long long)L.n3 > 4096) return smooth32(C, l, C.prm->coarse_sweeps, st);
    MG_DISPATCH32(C.m.kind, (k_coarse32<KK><<<1, 512, 0, st>>>(C.lf[l], L.n, L.e, L.ub, rho, L.S32,
                                                                 C.prm->coarse_sweeps)));
    return MGGLAM_OK;
  }
  if (l == 0) prof_begin(PC_SMOOTH32_FINE, st, 16.0 * L.n3 * C.prm->nu1);
  if ((rc = smooth32(C, l, C.prm->nu1, st))) return rc;
  if (l == 0) prof_end(st);
  if (l == 0) prof_begin(PC_RESTRICT32_FINE, st, 14.0 * L.n3);
  if ((rc = restrict_level(C, l, st, C.prm->nu1 > 0))) return rc;
  if (l == 0) {
    prof_end(st);
    prof_begin(PC_COARSE_LEVELS, st, 0.0);
    if ((rc = coarse_part(C, st))) return rc;
  } else {
    if ((rc = fas_source(C, l + 1, st))) return rc;
    if ((rc = vcycle32(C, l + 1, st, mode))) return rc;
    if (mode != 0 && (rc = vcycle32(C, l + 1, st, mode == 2 ? 2 : 0))) return rc;
  }
  // algorithmic bytes per fine cell: e, u read and e written (12), the coarse pair (1); the
  // second-colour-only form reads and writes half of e and u and writes half of q (9)
  if (l == 0) { prof_end(st); prof_begin(PC_PROLONG32_FINE, st, (C.qs && C.prm->nu2 >= 1 ? 9.0 : 13.0) * L.n3); }
  if ((rc = prolong_level(C, l, st))) return rc;
  if (l == 0) { prof_end(st); prof_begin(PC_SMOOTH32_FINE, st, 16.0 * L.n3 * C.prm->nu2); }
  rc = smooth32(C, l, C.prm->nu2, st, l == 1 && fine_reads_d(C));
  if (l == 0) prof_end(st);
  return rc;
}

// Full-multigrid start of the first outer step (prm->fmg), on the correction
// problem M(e) = S.  With e = 0 on every level, the residual-restriction and FAS-
// source kernels hand each coarser level the restricted base field and the
// restricted source (M(0) = 0, so S^H = M^H(0) - R(M(0) - S) = R S, and R e = 0).
// The coarsest level relaxes from e = 0; every finer level starts from the
// prolonged coarser correction (e = 0 + P(e^H - 0), both colours) and takes one
// V-cycle, the coarse stages without the one-block tail (so that each stage is
// the oracle's: relax the coarsest, prolong, cycle), the last one (level 0)
// as every other cycle of the solve.  From a uniform base field (the
// background start) this is the FMG of the total-field problem.
static int fmg_start32(const MixedCtx& C, cudaStream_t st) {
  Workspace* ws = C.ws;
  MixedCtx Cs = C;
  Cs.tail_level = -1;
  const int base = ws->nlev - 1;
  int rc;
  for (int l = 0; l < base; ++l) {
    if ((rc = restrict_level(C, l, st))) return rc;
    if ((rc = fas_source(C, l + 1, st))) return rc;
  }
  if ((rc = vcycle32(Cs, base, st, 0))) return rc;
  for (int l = base - 1; l >= 0; --l) {
    if ((rc = prolong_level(C, l, st, true))) return rc;
    if ((rc = vcycle32(l == 0 ? C : Cs, l, st, 0))) return rc;
  }
  return MGGLAM_OK;
}

// Tile of the FP64 outer-residual kernel.
constexpr int kRTJ = 8, kRTK = 32;

// bg_first: the first residual of the solve, with the background start fused
// into it (k_background_residual_ff); the tiled meshes only.
static bool bg_residual_tiled(int n) { return n % kRTK == 0 && n % kRTJ == 0; }

template <int K>
static int launch_outer_residual_ff(const MixedCtx& C, double* field, int* blocks, cudaStream_t st, bool bg_first,
                                    bool zero) {
  Workspace* ws = C.ws;
  Level& F = ws->lev[0];
  const FFC* ffc = ffc_of(ws);
  float* ze = zero ? F.e : nullptr;   // the split kernels' zeroing of e and q
  float* zq = zero ? C.qs : nullptr;
  if (bg_residual_tiled(F.n)) {
    // two cells a thread on 8 x 64 tiles where the side and the density's
    // alignment allow (8-byte pair loads), else one on 8 x 32
    const bool pair = F.n % 64 == 0 && (uintptr_t)C.rho % 8 == 0;
    const long long tiles = (long long)(F.n / (pair ? 64 : kRTK)) * (F.n / kRTJ);
    const bool i32 = F.n <= 1024;  // 32-bit cell offsets
    auto pk_split = i32 ? k_outer_residual_ff2<K, kRTJ, true, int> : k_outer_residual_ff2<K, kRTJ, true>;
    auto pk_nat = i32 ? k_outer_residual_ff2<K, kRTJ, false, int> : k_outer_residual_ff2<K, kRTJ, false>;
    const void* kern = pair ? (C.split ? (const void*)pk_split : (const void*)pk_nat)
                            : (C.split ? (const void*)k_outer_residual_ff<K, kRTJ, kRTK, true>
                                       : (const void*)k_outer_residual_ff<K, kRTJ, kRTK>);
    const int chunk = march_chunk(F.n, tiles, kern, kRTJ * (pair ? 32 : kRTK));
    dim3 grid((unsigned)tiles, (F.n + chunk - 1) / chunk);
    *blocks = grid.x * grid.y;
    if (*blocks > kMaxReduceBlocks) return MGGLAM_ERR_SHAPE;
    const int* skip = nullptr;
    if (bg_first) {
      int* flag = reinterpret_cast<int*>(ws->scalars + SC_FLAG);
      // four cells a thread when the caller's density and field allow 16-byte accesses
      const bool vec = ((uintptr_t)C.rho % 16 == 0) && ((uintptr_t)field % 16 == 0);
      if (vec && C.split)
        k_background_residual_ff4<K, true><<<grid, 256, 0, st>>>(ffc, F.n, field, C.m.ubar, C.rho, F.ub, F.S32,
                                                                  ws->partials, ze, zq);
      else if (vec)
        k_background_residual_ff4<K, false><<<grid, 256, 0, st>>>(ffc, F.n, field, C.m.ubar, C.rho, F.ub, F.S32,
                                                                   ws->partials);
      else if (C.split)
        k_background_residual_ff<K, true><<<grid, 256, 0, st>>>(ffc, F.n, field, C.m.ubar, C.rho, F.ub, F.S32,
                                                                 ws->partials, ze, zq);
      else
        k_background_residual_ff<K, false><<<grid, 256, 0, st>>>(ffc, F.n, field, C.m.ubar, C.rho, F.ub, F.S32,
                                                                  ws->partials);
      k_background_first<<<1, 1, 0, st>>>(field, flag);
      note_launch(2);
      skip = flag;
    }
    if (pair && C.split)
      pk_split<<<grid, kRTJ * 32, 0, st>>>(ffc, F.n, chunk, field, C.rho, F.ub, F.S32,
                                                                      ws->partials, skip, ze, zq);
    else if (pair)
      pk_nat<<<grid, kRTJ * 32, 0, st>>>(ffc, F.n, chunk, field, C.rho, F.ub, F.S32,
                                                                       ws->partials, skip, nullptr, nullptr);
    else if (C.split)
      k_outer_residual_ff<K, kRTJ, kRTK, true><<<grid, kRTJ * kRTK, 0, st>>>(ffc, F.n, chunk, field, C.rho, F.ub,
                                                                             F.S32, ws->partials, skip, ze, zq);
    else
      k_outer_residual_ff<K, kRTJ, kRTK><<<grid, kRTJ * kRTK, 0, st>>>(ffc, F.n, chunk, field, C.rho, F.ub, F.S32,
                                                                       ws->partials, skip);
    return MGGLAM_OK;
  }
  const int tk = (F.n % 16 == 0) ? 16 : ((F.n % 8 == 0) ? 8 : ((F.n % 4 == 0) ? 4 : 2));
  dim3 grid((F.n / tk) * (F.n / 2), 1);
  *blocks = grid.x;
  if (*blocks > kMaxReduceBlocks) return MGGLAM_ERR_SHAPE;
  switch (tk) {
    case 16: k_outer_residual_ff<K, 2, 16><<<grid, 32, 0, st>>>(ffc, F.n, F.n, field, C.rho, F.ub, F.S32, ws->partials); break;
    case 8: k_outer_residual_ff<K, 2, 8><<<grid, 16, 0, st>>>(ffc, F.n, F.n, field, C.rho, F.ub, F.S32, ws->partials); break;
    case 4: k_outer_residual_ff<K, 2, 4><<<grid, 8, 0, st>>>(ffc, F.n, F.n, field, C.rho, F.ub, F.S32, ws->partials); break;
    default: k_outer_residual_ff<K, 2, 2><<<grid, 4, 0, st>>>(ffc, F.n, F.n, field, C.rho, F.ub, F.S32, ws->partials); break;
  }
  return MGGLAM_OK;
}

template <int K>
static int launch_outer_residual_t(const MixedCtx& C, double* field, int* blocks, cudaStream_t st, bool bg_first,
                                   bool zero) {
  Workspace* ws = C.ws;
  Level& F = ws->lev[0];
  if constexpr (K != KCQ) {
    if (C.ff_resid) return launch_outer_residual_ff<K>(C, field, blocks, st, bg_first, zero);
  }
  if (F.n % kRTK == 0 && F.n % kRTJ == 0) {
    const int chunk = march_chunk(F.n, (long long)(F.n / kRTK) * (F.n / kRTJ),
                                  (const void*)k_outer_residual<K, kRTJ, kRTK>, kRTJ * kRTK);
    dim3 grid((F.n / kRTK) * (F.n / kRTJ), (F.n + chunk - 1) / chunk);
    *blocks = grid.x * grid.y;
    if (*blocks > kMaxReduceBlocks) return MGGLAM_ERR_SHAPE;
    k_outer_residual<K, kRTJ, kRTK><<<grid, kRTJ * kRTK, 0, st>>>(C.m, F.n, chunk, field, ws->src64, F.ub, F.S32,
                                                                  ws->partials);
  } else {
    // small or non-tiling meshes: two rows of the widest dividing k-tile per CTA
    const int tk = (F.n % 16 == 0) ? 16 : ((F.n % 8 == 0) ? 8 : ((F.n % 4 == 0) ? 4 : 2));
    dim3 grid((F.n / tk) * (F.n / 2), 1);
    *blocks = grid.x;
    if (*blocks > kMaxReduceBlocks) return MGGLAM_ERR_SHAPE;
    switch (tk) {
      case 16: k_outer_residual<K, 2, 16><<<grid, 32, 0, st>>>(C.m, F.n, F.n, field, ws->src64, F.ub, F.S32, ws->partials); break;
      case 8: k_outer_residual<K, 2, 8><<<grid, 16, 0, st>>>(C.m, F.n, F.n, field, ws->src64, F.ub, F.S32, ws->partials); break;
      case 4: k_outer_residual<K, 2, 4><<<grid, 8, 0, st>>>(C.m, F.n, F.n, field, ws->src64, F.ub, F.S32, ws->partials); break;
      default: k_outer_residual<K, 2, 2><<<grid, 4, 0, st>>>(C.m, F.n, F.n, field, ws->src64, F.ub, F.S32, ws->partials); break;
    }
  }
  return MGGLAM_OK;
}

// Whether the outer residual pass can zero the finest level's e and q when the
// next inner solve needs them zeroed (the split tiled float-float kernels write
// the zeros beside ub and tau; otherwise the outer step clears them with
// memsets).  On stored-q levels the next solve's first sweep takes them as zero
// by itself (fresh) and nothing is zeroed, except before an FMG start.
static bool residual_zeroes_e(const MixedCtx& C) { return C.split && C.ff_resid && bg_residual_tiled(C.ws->lev[0].n); }

// bg_first: the solve's first residual, on a mesh where the background start is
// fused into it (fused_background_start): the residual at ubar is formed there and
// the field keeps its NaN mark until the first correction (bg_pending).
static bool fused_background_start(const MixedCtx& C) { return C.ff_resid && bg_residual_tiled(C.ws->lev[0].n); }

// zero: the split tiled residual also zeroes e and q for the next inner solve
// (not needed when that solve's first sweep starts from e = 0 by itself).
static int outer_residual(const MixedCtx& C, double* field, cudaStream_t st, bool bg_first, bool zero) {
  Workspace* ws = C.ws;
  Level& F = ws->lev[0];
  // bytes per cell: u (8) and the source (float-float: the FP32 density, 4; FP64: src64, 8) in, ub and tau (4 + 4) out
  prof_begin(PC_OUTER_RESID, st, (C.ff_resid ? 20.0 : 24.0) * F.n3);
  int g = 0, rc = MGGLAM_OK;
  MG_DISPATCH32(C.m.kind, (rc = launch_outer_residual_t<KK>(C, field, &g, st, bg_first, zero)));
  if (rc) return rc;
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
  C.chunk = prm->sweep_chunk > 0 ? prm->sweep_chunk : 16;  // < 0: per-colour kernels only
  C.rho = rho;
  C.ff_resid = C.m.kind != KCQ;
  // red-black split fine level: float-float residual with its 8 x 32 tiles, per-colour smoothing
  C.split = C.ff_resid && prm->sweep_chunk <= 0 && C.ws->lev[0].n % 32 == 0;
  // the split level never runs the fused sweep, so its second buffer holds q
  C.qs = C.split && (C.m.kind == KFR1 || C.m.kind == KFR2) ? C.ws->lev[0].e_alt : nullptr;
  C.guard = guard_of(C.ws);
  const L2Scope l2s(q_window_begin(C));
  C.l2 = &l2s.w;
  C.tail_level = -1;  // the one-block tail runs V-cycles only
  const long long tail_cells = prm->tail_cells == 0 ? 512 : (prm->tail_cells > kTailMaxCells ? kTailMaxCells : prm->tail_cells);
  for (int l = 1; l < C.ws->nlev && tail_cells > 0 && prm->cycle == 0; ++l)
    if ((long long)C.ws->lev[l].n3 <= tail_cells && C.ws->nlev - l <= kTailMaxLevels) {
      C.tail_level = l;
      break;
    }
  if (C.tail_level > 0) tail_allow_smem();
  Workspace* ws = C.ws;
  for (int l = 0; l < ws->nlev; ++l) C.lf[l] = make_levelf(C.m, ws->lev[l].h);
  Level& F = ws->lev[0];
  const long long n3 = (long long)F.n3;
  const int g = stream_grid(n3);
  // FP64 density mean and source term; FP32 normalised pyramid where the inner operator needs it
  if ((rc = launch_density_mean(rho, F.n3, ws->partials, ws->scalars + SC_MEAN, st))) return rc;
  if (C.ff_resid) {
    k_ff_consts<<<1, 32, 0, st>>>(C.m, n3, ws->scalars + SC_MEAN, ffc_of(ws));
    note_launch(1);
  } else {
    MG_DISPATCH32(C.m.kind, (k_src64<KK><<<stream_grid(n3), kThreads, 0, st>>>(
                                 C.m, rho, n3, ws->scalars + SC_MEAN, ws->src64)));
  }
  if (C.need_rho) {
    if (C.split) k_density_norm32_split<<<stream_grid(n3), kThreads, 0, st>>>(rho, F.n, ws->scalars + SC_MEAN, F.rho32);
    else k_density_norm32<<<stream_grid(n3), kThreads, 0, st>>>(rho, n3, ws->scalars + SC_MEAN, F.rho32);
    note_launch(1);
    for (int l = 1; l < ws->nlev; ++l) {
      const int b = bx_for(ws->lev[l].n);
      if (l == 1 && C.split)
        k_restrict32_from_split<<<grid3(ws->lev[l].n, ws->lev[l].n, ws->lev[l].n, b), b, 0, st>>>(
            ws->lev[l - 1].n, ws->lev[l - 1].rho32, ws->lev[l].rho32);
      else
        k_restrict32<<<grid3(ws->lev[l].n, ws->lev[l].n, ws->lev[l].n, b), b, 0, st>>>(
            ws->lev[l - 1].n, ws->lev[l - 1].rho32, ws->lev[l].rho32);
      note_launch(1);
    }
  }
  // the background start (a NaN first element) is filled here, or inside the first residual
  const bool fused_bg = fused_background_start(C);
  if (!fused_bg && (rc = launch_init_background(C.m, field, F.n3, st))) return rc;
  MG_CUDA_TRY(cudaMemsetAsync(C.guard, 0, sizeof(unsigned long long), st));
  MG_DISPATCH32(C.m.kind, (k_src_sumsq32<KK><<<g, kThreads, 0, st>>>(C.m, rho, n3, ws->scalars + SC_MEAN,
                                                                      ws->partials)));
  k_finalize_sum32<<<1, 1024, 0, st>>>(ws->partials, g, ws->scalars + SC_SRC);
  note_launch(1);
  // The first stored-q sweep of an inner solve can take e = q = 0 by itself
  // (split f(R) n = 1, 2 with pre-smoothing), so the residual passes need not
  // zero them -- except before an FMG start, which restricts e before any sweep.
  const bool fresh_ok = residual_zeroes_e(C) && C.qs && prm->nu1 >= 1;
  const bool fmg_first = prm->fmg && C.m.kind != KCQ;
  bool fresh = false;
  C.fresh = &fresh;
  if ((rc = outer_residual(C, field, st, fused_bg, !fresh_ok || fmg_first))) return rc;
  MG_CUDA_TRY(cudaMemcpyAsync(ws->h_scalars, ws->scalars, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
  MG_CUDA_TRY(cudaStreamSynchronize(st));
  MG_CUDA_TRY(cudaGetLastError());
  // background start fused into the first residual: the field keeps its NaN mark
  // until the first correction writes ubar + e (or the fill below, without one)
  bool bg_pending = fused_bg && *reinterpret_cast<const int*>(ws->h_scalars + SC_FLAG) != 0;
  const double src = sqrt(ws->h_scalars[SC_SRC] / (double)n3);
  const double snorm = source_norm(C.m, src);
  double eps = sqrt(ws->h_scalars[SC_SUMSQ] / (double)n3) / snorm;
  mgglam_stats local;
  mgglam_stats* S = stats ? stats : &local;
  memset(S, 0, sizeof(*S));
  S->resid0 = eps;
  S->resid_hist[0] = eps;
  int cyc = 0, outer = 0, nh = 1;
  // Inner cycles per outer step: fixed (prm->inner_cycles > 0), or adaptive:
  // enough cycles to reach tol at the contraction rho observed so far, but no
  // more than single precision can use in one step (kFp32StepGain).
  double rho_est = kInitialContraction;
  int status = MGGLAM_OK;
  while (!(eps <= tol) && cyc < prm->max_cycles) {
    if (!isfinite(eps)) { status = MGGLAM_ERR_NONFINITE; break; }
    // the first cycle of the first outer step is the FMG start (fmg_start32),
    // planned as a gain of kFmgGain followed by cycles at the estimated contraction
    const bool fmg = prm->fmg && C.m.kind != KCQ && outer == 0;
    int inner = prm->inner_cycles;
    if (inner <= 0) {
      const double lr = log(rho_est), lg = fmg ? log(kFmgGain) : 0.0;
      const int need = (fmg ? 1 : 0) + (int)ceil((log(fmax(tol, 1e-300) / eps) - lg) / lr - 1e-9);
      const int cap = (fmg ? 1 : 0) + (int)ceil((log(kFp32StepGain) - lg) / lr - 1e-9);
      inner = need < 1 ? 1 : (need > cap ? cap : need);
    }
    const double eps_before = eps;
    int done = 0;
    if (!residual_zeroes_e(C)) {
      MG_CUDA_TRY(cudaMemsetAsync(F.e, 0, F.n3 * sizeof(float), st));
      if (C.qs) MG_CUDA_TRY(cudaMemsetAsync(C.qs, 0, F.n3 * sizeof(float), st));  // Delta w(u, 0) = 0
    }
    fresh = fresh_ok && !fmg;
    for (int c = 0; c < inner && cyc < prm->max_cycles; ++c, ++cyc, ++done)
      if ((rc = (fmg && c == 0) ? fmg_start32(C, st) : vcycle32(C, 0, st, C.prm->cycle))) return rc;
    prof_begin(PC_APPLY_CORR, st, 20.0 * n3);
    const bool vec = C.split && (uintptr_t)field % 16 == 0;  // the split layout has n % 32 == 0
    if (vec && bg_pending)
      k_apply_correction_split<true><<<kStreamBlocks, kThreads, 0, st>>>(field, F.e, F.n, C.m.ubar);
    else if (vec)
      k_apply_correction_split<false><<<kStreamBlocks, kThreads, 0, st>>>(field, F.e, F.n, C.m.ubar);
    else if (C.split && bg_pending)
      k_apply_correction_split_scalar<true><<<kStreamBlocks, 128, 0, st>>>(field, F.e, F.n, C.m.ubar);
    else if (C.split)
      k_apply_correction_split_scalar<false><<<kStreamBlocks, 128, 0, st>>>(field, F.e, F.n, C.m.ubar);
    else if (bg_pending)
      k_apply_correction<true><<<stream_grid(n3), kThreads, 0, st>>>(field, F.e, n3, C.m.ubar);
    else
      k_apply_correction<false><<<stream_grid(n3), kThreads, 0, st>>>(field, F.e, n3, C.m.ubar);
    note_launch(1);
    bg_pending = false;
    prof_end(st);
    ++outer;
    if ((rc = outer_residual(C, field, st, false, !fresh_ok))) return rc;
    MG_CUDA_TRY(cudaMemcpyAsync(ws->h_scalars + SC_SUMSQ, ws->scalars + SC_SUMSQ, sizeof(double),
                                cudaMemcpyDeviceToHost, st));
    MG_CUDA_TRY(cudaStreamSynchronize(st));
    MG_CUDA_TRY(cudaGetLastError());
    eps = sqrt(ws->h_scalars[SC_SUMSQ] / (double)n3) / snorm;
    if (nh < 64) S->resid_hist[nh++] = eps;
    const int vdone = fmg ? done - 1 : done;  // V-cycles after the FMG start
    if (vdone > 0 && eps > 0.0 && eps < eps_before) {
      // per-cycle contraction of this step, when it was not limited by single precision
      const double g = (eps / eps_before) / (fmg ? kFmgGain : 1.0);
      const double r = pow(g, 1.0 / vdone);
      if (eps / eps_before > kFp32StepGain) rho_est = fmin(0.5, fmax(0.01, r));
    }
  }
  if (status == MGGLAM_OK && !isfinite(eps)) status = MGGLAM_ERR_NONFINITE;
  // no correction was applied to a background start: the solution is ubar
  if (bg_pending && (rc = launch_init_background(C.m, field, F.n3, st))) return rc;
  MG_CUDA_TRY(cudaMemcpyAsync(ws->h_scalars + SC_GUARD, C.guard, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                              st));
  MG_CUDA_TRY(cudaStreamSynchronize(st));
  S->guarded = (long long)*reinterpret_cast<const unsigned long long*>(ws->h_scalars + SC_GUARD);
  S->cycles = cyc;
  S->outer = outer;
  S->resid = eps;
  S->converged = eps <= tol;
  S->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (status == MGGLAM_OK && !S->converged) status = MGGLAM_ERR_NOT_CONVERGED;
  return status;
}

}  // namespace mg
