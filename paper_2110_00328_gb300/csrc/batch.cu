// batch.cu -- many independent solves (uneven meshes, models, parameters) at once.
//
// All solves of a batch follow the mixed-precision scheme of solve_mixed.cu
// (FP64 outer residual and update, FP32 correction-form FAS V-cycles) in lock
// step.  Each phase of a V-cycle (one colour of smoothing on level l,
// restriction l -> l+1, coarse source on l+1, coarsest-level relaxation,
// prolongation l+1 -> l) is one kernel launch covering the blocks of every
// solve that takes part in it: a block finds its solve by binary search in a
// prefix table of per-solve block counts and then works exactly as the single-
// solve kernel does.  One V-cycle of the whole batch is captured once as a CUDA
// graph and replayed.  Solves that have converged are masked by a device flag
// (their blocks exit at once), so the graph never needs re-capturing.  The
// smoother's block width is chosen by timing the candidates on the batch's
// finest levels on first use (a small autotuner), and cached with the batch.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <vector>

#include "mg_common.cuh"
#include "mg_internal.h"
#include "mixed_common.cuh"
#include "sweep32.cuh"

namespace mg {

// One level of one solve.
struct BDesc {
  int n;      // level side
  int solve;  // index of the solve in the batch
  int split;  // this level (the finest) in the red-black split layout
  LevelF lf;  // constants of this level
  float *e, *ub, *S, *rho, *Re;      // this level
  float* q;                          // split f(R) n = 1, 2: the stored neighbour quantity, else nullptr
  float *eH, *ubH, *SH, *ReH;        // next coarser level (if any)
};

// Finest-level descriptor for the FP64 outer kernels.
struct BFine {
  int n, solve;
  ModelDev m;
  double* u;
  const double* src;   // CQ: FP64 source term
  const FFC* ffc;      // f(R), symmetron: float-float residual constants
  const float* rho;    // f(R), symmetron: the caller's density
  float *ub, *tau, *e;
  float* q;            // the finest level's stored neighbour quantity (zeroed with e), or nullptr
};

// Level layouts of the batched kernels: the quad kernels take levels whose side
// is a multiple of 4 (>= 8); others fall back to one cell per thread.
__host__ __device__ __forceinline__ bool quad_level(int n) { return (n & 3) == 0 && n >= 8; }

__device__ __forceinline__ int find_slot(const int* __restrict__ prefix, int cnt, int b) {
  int lo = 0, hi = cnt - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---- batched phase kernels (bodies as in solve_mixed.cu) ----

// Block (32, ROWS).  Quad levels: ceil(n/128) x n x ceil(n/ROWS) blocks per
// solve (lanes along k, ROWS planes i per block); others: one cell of the
// colour per thread, flat.
template <int K, int ROWS>
__global__ void __launch_bounds__(32 * ROWS) kb_smooth(const BDesc* __restrict__ D, const int* __restrict__ prefix,
                                                       int cnt, const int* __restrict__ active, int parity) {
  const int s = find_slot(prefix, cnt, blockIdx.x);
  const BDesc& d = D[s];
  if (!active[d.solve]) return;
  const int n = d.n;
  const int b = blockIdx.x - prefix[s];
  if (d.split) {
    long long r;
    int seg;
    bool act;
    split_lane(n, n, (long long)b * ROWS + threadIdx.y, threadIdx.x, &r, &seg, &act);
    if constexpr (K == KFR1 || K == KFR2) {
      if (d.q) {
        smooth_split<K, true>(d.lf, n, d.e, d.ub, d.rho, d.S, (int)(r / n), (int)(r % n), seg, act, parity,
                              threadIdx.x, d.q);
        return;
      }
    }
    smooth_split<K>(d.lf, n, d.e, d.ub, d.rho, d.S, (int)(r / n), (int)(r % n), seg, act, parity, threadIdx.x);
    return;
  }
  if (quad_level(n)) {
    const int nbx = ((n >> 2) + 31) / 32;
    const int xb = b % nbx, r = b / nbx, j = r % n, i = (r / n) * ROWS + threadIdx.y;
    if (i >= n) return;  // whole warps
    smooth_quad<K>(d.lf, n, d.e, d.ub, d.rho, d.S, i, j, xb * 32 + threadIdx.x, threadIdx.x, parity);
    return;
  }
  const long long t = (long long)b * (32 * ROWS) + threadIdx.y * 32 + threadIdx.x;
  const int h = n >> 1;
  if (t >= (long long)h * n * n) return;
  const int kk = (int)(t % h), j = (int)((t / h) % n), i = (int)(t / ((long long)h * n));
  const int k = 2 * kk + ((i + j + parity) & 1);
  const size_t c = cidx(n, i, j, k);
  const float Lnb = nb_sum_g<K>(d.e, d.ub, n, i, j, k);
  d.e[c] = update_e_fast<K>(d.lf, d.ub[c], d.e[c], d.rho ? d.rho[c] : 1.f, d.S[c], Lnb);
}

static int smooth_blocks(int n, int rows, bool split) {
  if (split) return (int)((split_warps(n, n) + rows - 1) / rows);
  if (quad_level(n)) return (((n >> 2) + 31) / 32) * n * ((n + rows - 1) / rows);
  return (int)(((long long)(n >> 1) * n * n + 32 * rows - 1) / (32 * rows));
}

// Restriction of level l into l+1, d = M(e) - S at 8 children; block (32, 4).
// Quad levels: ceil(nf/128) x nc x ceil(nc/4) blocks per solve; others: one
// coarse cell per thread, flat.
template <int K>
__global__ void __launch_bounds__(128) kb_restrict(const BDesc* __restrict__ D, const int* __restrict__ prefix, int cnt,
                                                   const int* __restrict__ active) {
  const int s = find_slot(prefix, cnt, blockIdx.x);
  const BDesc& d = D[s];
  if (!active[d.solve]) return;
  const int nf = d.n, nc = nf >> 1;
  const int b = blockIdx.x - prefix[s];
  if (quad_level(nf)) {
    const int nbx = ((nf >> 2) + 31) / 32;
    const int xb = b % nbx, r = b / nbx, J = r % nc, I = (r / nc) * 4 + threadIdx.y;
    if (I >= nc) return;  // whole warps
    if constexpr (K == KFR1 || K == KFR2) {
      if (d.split && d.q) {
        restrict_quad<K, SplitLayout, true>(d.lf, nf, d.e, d.ub, d.rho, d.S, d.ReH, d.eH, d.ubH, d.SH, I, J,
                                            xb * 32 + threadIdx.x, threadIdx.x, d.q);
        return;
      }
    }
    if (d.split)
      restrict_quad<K, SplitLayout>(d.lf, nf, d.e, d.ub, d.rho, d.S, d.ReH, d.eH, d.ubH, d.SH, I, J,
                                    xb * 32 + threadIdx.x, threadIdx.x);
    else
      restrict_quad<K>(d.lf, nf, d.e, d.ub, d.rho, d.S, d.ReH, d.eH, d.ubH, d.SH, I, J, xb * 32 + threadIdx.x,
                       threadIdx.x);
    return;
  }
  const long long t = (long long)b * 128 + threadIdx.y * 32 + threadIdx.x;
  if (t >= (long long)nc * nc * nc) return;
  const int Kc = (int)(t % nc), J = (int)((t / nc) % nc), I = (int)(t / ((long long)nc * nc));
  float se = 0.f, su = 0.f, sd = 0.f;
  for (int di = 0; di < 2; ++di)
    for (int dj = 0; dj < 2; ++dj)
      for (int dk = 0; dk < 2; ++dk) {
        const int i = 2 * I + di, j = 2 * J + dj, k = 2 * Kc + dk;
        const size_t c = cidx(nf, i, j, k);
        const float ec = d.e[c], uc = d.ub[c];
        se += ec;
        su += uc;
        sd += local_M<K>(d.lf, uc, ec, d.rho ? d.rho[c] : 1.f, nb_sum_g<K>(d.e, d.ub, nf, i, j, k)) - d.S[c];
      }
  const size_t o = cidx(nc, I, J, Kc);
  d.ReH[o] = 0.125f * se;
  d.eH[o] = 0.125f * se;
  d.ubH[o] = 0.125f * su;
  d.SH[o] = 0.125f * sd;
}

static int restrict_blocks(int nf) {
  const int nc = nf >> 1;
  if (quad_level(nf)) return (((nf >> 2) + 31) / 32) * nc * ((nc + 3) / 4);
  return (int)(((long long)nc * nc * nc + 127) / 128);
}

// Coarse source on level l (descriptors of level l): S <- M(Re) - S.
template <int K>
__global__ void __launch_bounds__(64) kb_fas(const BDesc* __restrict__ D, const int* __restrict__ prefix, int cnt,
                                             const int* __restrict__ active) {
  const int s = find_slot(prefix, cnt, blockIdx.x);
  const BDesc& d = D[s];
  if (!active[d.solve]) return;
  const int n = d.n, nxb = (n + 63) / 64;
  const int b = blockIdx.x - prefix[s];
  const int xb = b % nxb, r = b / nxb, j = r % n, i = r / n;
  const int k = xb * 64 + threadIdx.x;
  if (k >= n) return;
  const size_t t = cidx(n, i, j, k);
  d.S[t] = local_M<K>(d.lf, d.ub[t], d.Re[t], d.rho ? d.rho[t] : 1.f, nb_sum_g<K>(d.Re, d.ub, n, i, j, k)) - d.S[t];
}

// Prolongation-correction of level l from l+1; block (32, 4).  Quad levels:
// ceil(nf/128) x nf x ceil(nf/4) blocks per solve; others: one fine cell per
// thread, flat.
// QK >= 0 (f(R) n = QK): levels with a stored q get it written (prolong_quad),
// only for the second colour when SO (post-smoothing follows).
template <bool FR, int QK = -1, bool SO = false>
__global__ void __launch_bounds__(128) kb_prolong(const BDesc* __restrict__ D, const int* __restrict__ prefix, int cnt,
                                                  const int* __restrict__ active, unsigned long long* guards) {
  const int s = find_slot(prefix, cnt, blockIdx.x);
  const BDesc& d = D[s];
  if (!active[d.solve]) return;
  unsigned long long* guard = guards + d.solve;
  const int nf = d.n, nc = nf >> 1;
  const int b = blockIdx.x - prefix[s];
  if (quad_level(nf)) {
    const int nbx = ((nf >> 2) + 31) / 32;
    const int xb = b % nbx, r = b / nbx, j = r % nf, i = (r / nf) * 4 + threadIdx.y;
    if (i >= nf) return;  // whole warps
    if constexpr (QK >= 0) {
      if (d.split && d.q) {
        prolong_quad<FR, SplitLayout, QK, SO>(nc, d.eH, d.ReH, d.ub, d.e, i, j, xb * 32 + threadIdx.x, threadIdx.x,
                                              guard, d.q);
        return;
      }
    }
    if (d.split)
      prolong_quad<FR, SplitLayout>(nc, d.eH, d.ReH, d.ub, d.e, i, j, xb * 32 + threadIdx.x, threadIdx.x, guard);
    else prolong_quad<FR>(nc, d.eH, d.ReH, d.ub, d.e, i, j, xb * 32 + threadIdx.x, threadIdx.x, guard);
    return;
  }
  const long long t = (long long)b * 128 + threadIdx.y * 32 + threadIdx.x;
  if (t >= (long long)nf * nf * nf) return;
  const int k = (int)(t % nf), j = (int)((t / nf) % nf), i = (int)(t / ((long long)nf * nf));
  const int I = i >> 1, J = j >> 1, Kc = k >> 1;
  const int I2 = wrapi(I + ((i & 1) ? 1 : -1), nc);
  const int J2 = wrapi(J + ((j & 1) ? 1 : -1), nc);
  const int K2 = wrapi(Kc + ((k & 1) ? 1 : -1), nc);
#define EH(a, b, c) (d.eH[cidx(nc, a, b, c)] - d.ReH[cidx(nc, a, b, c)])
  const float corr = (27.f * EH(I, J, Kc) + 9.f * (EH(I2, J, Kc) + EH(I, J2, Kc) + EH(I, J, K2)) +
                      3.f * (EH(I2, J2, Kc) + EH(I2, J, K2) + EH(I, J2, K2)) + EH(I2, J2, K2)) *
                     (1.f / 64.f);
#undef EH
  const size_t o = cidx(nf, i, j, k);
  const float old = d.e[o];
  float v = old + corr;
  if (FR && !(d.ub[o] + v > 0.f)) {
    v = 0.5f * (old - d.ub[o]);
    count_guards(guard, 1u);
  }
  d.e[o] = v;
}

static int prolong_blocks(int nf) {
  if (quad_level(nf)) return (((nf >> 2) + 31) / 32) * nf * ((nf + 3) / 4);
  return (int)(((long long)nf * nf * nf + 127) / 128);
}

// Coarsest levels: one CTA per solve.
template <int K>
__global__ void __launch_bounds__(512) kb_coarse(const BDesc* __restrict__ D, const int* __restrict__ active,
                                                 int sweeps) {
  const BDesc& d = D[blockIdx.x];
  if (!active[d.solve]) return;
  const int n = d.n, n3 = n * n * n;
  for (int s = 0; s < sweeps; ++s)
    for (int parity = 0; parity < 2; ++parity) {
      for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int k = t % n, j = (t / n) % n, i = t / (n * n);
        if (((i + j + k) & 1) != parity) continue;
        const float Lnb = nb_sum_g<K>(d.e, d.ub, n, i, j, k);
        d.e[t] = update_e_fast<K>(d.lf, d.ub[t], d.e[t], d.rho ? d.rho[t] : 1.f, d.S[t], Lnb);
      }
      __syncthreads();
    }
}

// FP64 fine residual of every active solve (tiles of 8 x 32, chunks of 64 planes).
template <int K>
__global__ void __launch_bounds__(256) kb_outer_residual(const BFine* __restrict__ F, const int* __restrict__ prefix,
                                                         int cnt, const int* __restrict__ active,
                                                         double* __restrict__ partials) {
  const int s = find_slot(prefix, cnt, blockIdx.x);
  const BFine& f = F[s];
  const int b = blockIdx.x - prefix[s];
  double a = 0.0;
  if (active[f.solve]) {
    const int tiles = (f.n / 32) * (f.n / 8);
    if constexpr (K == KCQ) {
      a = outer_residual_tile<K, 8, 32>(f.m, f.n, 64, f.u, f.src, f.ub, f.tau, b % tiles, b / tiles);
    } else {
      const FFC c = *f.ffc;
      a = outer_residual_tile_ff<K, 8, 32, true>(c, f.n, 64, f.u, f.rho, f.ub, f.tau, b % tiles, b / tiles);
    }
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = a;
}

// Per-solve sums of the partials: out[solve] = sum over its blocks.
__global__ void kb_finalize(const BFine* __restrict__ F, const int* __restrict__ prefix, int cnt,
                            const double* __restrict__ partials, double* __restrict__ out) {
  const int s = blockIdx.x;
  double a = 0.0;
  for (int i = prefix[s] + threadIdx.x; i < prefix[s + 1]; i += blockDim.x) a += partials[i];
  a = block_sum(a);
  if (threadIdx.x == 0) out[F[s].solve] = a;
}

// u64 += e and e <- 0 (and the stored q <- 0) for every active solve (fine-cell grid).
__global__ void __launch_bounds__(256) kb_apply(const BFine* __restrict__ F, const int* __restrict__ prefix, int cnt,
                                                const int* __restrict__ active, int clear_only) {
  const int s = find_slot(prefix, cnt, blockIdx.x);
  const BFine& f = F[s];
  if (!active[f.solve]) return;
  const size_t n3 = (size_t)f.n * f.n * f.n;
  const size_t t = (size_t)(blockIdx.x - prefix[s]) * 256 + threadIdx.x;
  if (t >= n3) return;
  // f(R) and symmetron fine levels are split (float-float residual); CQ keeps the natural layout
  const long long c = f.m.kind == KCQ ? (long long)t
                                      : split_idx(f.n, (int)(t / ((size_t)f.n * f.n)), (int)((t / f.n) % f.n),
                                                  (int)(t % f.n));
  if (!clear_only) f.u[t] += (double)f.e[c];
  f.e[c] = 0.f;
  if (f.q) f.q[c] = 0.f;  // Delta w(u, 0)
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct Phase {            // one batched launch: kind group, descriptor table, block prefix
  int kind = 0, cnt = 0, blocks = 0;
  BDesc* d = nullptr;     // device
  int* prefix = nullptr;  // device, cnt + 1
};

struct Batch {
  int device = -1;
  std::vector<int> Ns, levels_req;   // signature
  int count = 0;
  void* base = nullptr;
  size_t bytes = 0;
  // per solve
  struct S {
    int N, nlev, kind;
    double* src64;
    float *e[kMaxLevels], *ub[kMaxLevels], *S32[kMaxLevels], *Re[kMaxLevels], *rho32[kMaxLevels];
    float* q0;  // the finest level's stored neighbour quantity (used for f(R) n = 1, 2)
  };
  std::vector<S> sv;
  double* partials = nullptr;  // outer-residual partials
  double* sums = nullptr;      // per solve: sum r^2
  double* ssum = nullptr;      // per solve: source sum of squares
  double* rmean = nullptr;     // per solve: density sum
  int* active = nullptr;       // per solve flag (device)
  unsigned long long* guards = nullptr;    // per solve: positivity-guard replacements (device)
  unsigned long long* h_guards = nullptr;  // pinned host mirror
  int* h_active = nullptr;     // pinned host mirror
  double* h_sums = nullptr;    // pinned host mirror of sums (count) and ssum (count)
  void* tables = nullptr;      // descriptor tables and prefixes
  size_t tables_bytes = 0;
  cudaGraphExec_t vexec = nullptr;
  cudaStream_t cap = nullptr;
  unsigned long long vsig = 0;
  long long vlaunches = 0;
  int rows = 0;                // autotuned smoother block height (planes per block)
  FFC* ffc = nullptr;          // per solve: float-float residual constants
};

static std::mutex g_bmu;
static std::vector<Batch*> g_batches;

static void free_batch(Batch* b) {
  if (b->vexec) cudaGraphExecDestroy(b->vexec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->tables) cudaFree(b->tables);
  if (b->base) cudaFree(b->base);
  if (b->h_active) cudaFreeHost(b->h_active);
  if (b->h_sums) cudaFreeHost(b->h_sums);
  if (b->h_guards) cudaFreeHost(b->h_guards);
  delete b;
}

void release_batches() {
  std::lock_guard<std::mutex> lk(g_bmu);
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<Batch*> keep;
  for (Batch* b : g_batches) {
    if (b->device == dev) free_batch(b);
    else keep.push_back(b);
  }
  g_batches = keep;
}

static int get_batch(int count, const int* N, const mgglam_params* prm, Batch** out) {
  int dev = 0;
  MG_CUDA_TRY(cudaGetDevice(&dev));
  std::vector<int> ns(N, N + count), lv(count);
  for (int s = 0; s < count; ++s) lv[s] = prm[s].levels;
  std::lock_guard<std::mutex> lk(g_bmu);
  for (Batch* b : g_batches)
    if (b->device == dev && b->Ns == ns && b->levels_req == lv) {
      *out = b;
      return MGGLAM_OK;
    }
  Batch* b = new Batch();
  b->device = dev;
  b->Ns = ns;
  b->levels_req = lv;
  b->count = count;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
  struct O { size_t src, q0, e[kMaxLevels], ub[kMaxLevels], S[kMaxLevels], Re[kMaxLevels], rho[kMaxLevels]; };
  std::vector<O> o(count);
  size_t total_blocks = 0;
  b->sv.resize(count);
  for (int s = 0; s < count; ++s) {
    Batch::S& v = b->sv[s];
    v.N = N[s];
    v.nlev = count_levels(N[s], prm[s].levels);
    o[s].src = take((size_t)N[s] * N[s] * N[s] * 8);
    o[s].q0 = take((size_t)N[s] * N[s] * N[s] * 4);  // the plan is cached per mesh set, the models may change
    for (int l = 0, n = N[s]; l < v.nlev; ++l, n /= 2) {
      const size_t c = (size_t)n * n * n * 4;
      o[s].e[l] = take(c);
      o[s].ub[l] = take(c);
      o[s].S[l] = take(c);
      o[s].Re[l] = take(c);
      o[s].rho[l] = take(c);
    }
    total_blocks += (size_t)(N[s] / 32) * (N[s] / 8) * ((N[s] + 63) / 64);
  }
  const size_t o_part = take(std::max<size_t>(total_blocks, kMaxReduceBlocks) * 8);
  const size_t o_sums = take(count * 8), o_ssum = take(count * 8), o_rmean = take(count * 8), o_act = take(count * 4);
  const size_t o_ffc = take(count * sizeof(FFC));
  const size_t o_guard = take(count * sizeof(unsigned long long));
  if (cudaMalloc(&b->base, off) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return MGGLAM_ERR_OOM;
  }
  if (cudaMallocHost((void**)&b->h_active, count * 4) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_sums, count * 16) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_guards, count * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return MGGLAM_ERR_OOM;
  }
  b->bytes = off;
  char* base = (char*)b->base;
  for (int s = 0; s < count; ++s) {
    Batch::S& v = b->sv[s];
    v.src64 = (double*)(base + o[s].src);
    v.q0 = (float*)(base + o[s].q0);
    for (int l = 0; l < v.nlev; ++l) {
      v.e[l] = (float*)(base + o[s].e[l]);
      v.ub[l] = (float*)(base + o[s].ub[l]);
      v.S32[l] = (float*)(base + o[s].S[l]);
      v.Re[l] = (float*)(base + o[s].Re[l]);
      v.rho32[l] = (float*)(base + o[s].rho[l]);
    }
  }
  b->partials = (double*)(base + o_part);
  b->sums = (double*)(base + o_sums);
  b->ssum = (double*)(base + o_ssum);
  b->rmean = (double*)(base + o_rmean);
  b->active = (int*)(base + o_act);
  b->ffc = (FFC*)(base + o_ffc);
  b->guards = (unsigned long long*)(base + o_guard);
  g_batches.push_back(b);
  *out = b;
  return MGGLAM_OK;
}

// Kernel-group dispatch for batched launches.
#define MG_BDISPATCH(kind, CALL)                                        \
  switch (kind) {                                                       \
    case KFR0: { constexpr int KK = KFR0; CALL; } break;                \
    case KFR1: { constexpr int KK = KFR1; CALL; } break;                \
    case KFR2: { constexpr int KK = KFR2; CALL; } break;                \
    case KSYM: { constexpr int KK = KSYM; CALL; } break;                \
    default: { constexpr int KK = KCQ; CALL; } break;                   \
  }

struct Plan {
  // per level l: phases for kinds present; smooth/restrict/prolong over solves with
  // last level > l; fas over level l+1 of the same solves; coarse for last level == l
  struct LevelPhases {
    std::vector<Phase> smooth, restrict_, fas, prolong, coarse;
  };
  std::vector<LevelPhases> lv;
  std::vector<Phase> outer;  // fine levels, per kind (tiled residual)
  std::vector<Phase> apply;  // fine levels, per kind (256 cells per block)
  std::vector<BFine*> fine_desc;
  std::vector<int*> fine_prefix;
};

// Build all descriptor tables in one device allocation.
static int build_plan(Batch* B, const std::vector<ModelDev>& models, const std::vector<std::vector<LevelF>>& lfs,
                      const std::vector<const float*>& rho_in, double* const* field, const mgglam_params* prm,
                      bool need_rho_any, int rows, Plan* P, cudaStream_t st) {
  (void)need_rho_any;
  (void)prm;
  const int count = B->count;
  int Lmax = 0;
  for (auto& v : B->sv) Lmax = std::max(Lmax, v.nlev);
  // host staging buffer of descriptors + prefixes
  std::vector<char> host;
  struct Pending { Phase* ph; size_t d_off, p_off; };
  std::vector<Pending> pend;
  auto align = [&](size_t x) { return (x + 255) & ~(size_t)255; };
  auto add_phase = [&](Phase& ph, const std::vector<BDesc>& ds, const std::vector<int>& blocks) {
    ph.cnt = (int)ds.size();
    size_t d_off = align(host.size());
    host.resize(d_off + ds.size() * sizeof(BDesc));
    memcpy(host.data() + d_off, ds.data(), ds.size() * sizeof(BDesc));
    size_t p_off = align(host.size());
    host.resize(p_off + (ds.size() + 1) * sizeof(int));
    int* pf = (int*)(host.data() + p_off);
    int acc = 0;
    for (size_t i = 0; i < ds.size(); ++i) { pf[i] = acc; acc += blocks[i]; }
    pf[ds.size()] = acc;
    ph.blocks = acc;
    pend.push_back({&ph, d_off, p_off});
  };
  auto desc = [&](int s, int l) {
    const Batch::S& v = B->sv[s];
    BDesc d;
    memset(&d, 0, sizeof(d));
    d.n = v.N >> l;
    d.solve = s;
    d.split = (l == 0 && models[s].kind != KCQ) ? 1 : 0;  // split finest level (float-float residual)
    d.q = (l == 0 && (models[s].kind == KFR1 || models[s].kind == KFR2)) ? v.q0 : nullptr;
    d.lf = lfs[s][l];
    d.e = v.e[l];
    d.ub = v.ub[l];
    d.S = v.S32[l];
    const bool rho_needed = models[s].kind == KSYM || (models[s].kind == KCQ && models[s].keep_exp);
    d.rho = rho_needed ? v.rho32[l] : nullptr;
    d.Re = v.Re[l];
    if (l + 1 < v.nlev) {
      d.eH = v.e[l + 1];
      d.ubH = v.ub[l + 1];
      d.SH = v.S32[l + 1];
      d.ReH = v.Re[l + 1];
    }
    return d;
  };
  P->lv.assign(Lmax, {});
  std::vector<int> kinds;
  for (auto& m : models)
    if (std::find(kinds.begin(), kinds.end(), m.kind) == kinds.end()) kinds.push_back(m.kind);
  for (int l = 0; l < Lmax; ++l) {
    for (int kind : kinds) {
      std::vector<BDesc> sm, fa, co;
      std::vector<int> bsm, bre, bfa, bpr, bco;
      for (int s = 0; s < count; ++s) {
        if (models[s].kind != kind) continue;
        const int last = B->sv[s].nlev - 1;
        const int n = B->sv[s].N >> l;
        if (l < last) {
          sm.push_back(desc(s, l));
          bsm.push_back(smooth_blocks(n, rows, l == 0 && models[s].kind != KCQ));
          bre.push_back(restrict_blocks(n));
          bpr.push_back(prolong_blocks(n));
          fa.push_back(desc(s, l + 1));
          bfa.push_back(((n / 2 + 63) / 64) * (n / 2) * (n / 2));
        } else if (l == last) {
          co.push_back(desc(s, l));
          bco.push_back(1);
        }
      }
      if (!sm.empty()) {
        Phase a, b, c, d;
        a.kind = b.kind = c.kind = d.kind = kind;
        P->lv[l].smooth.push_back(a);
        P->lv[l].restrict_.push_back(b);
        P->lv[l].fas.push_back(c);
        P->lv[l].prolong.push_back(d);
      }
      if (!co.empty()) {
        Phase e;
        e.kind = kind;
        P->lv[l].coarse.push_back(e);
      }
    }
  }
  // second pass now that the vectors no longer move: fill tables
  for (int l = 0; l < Lmax; ++l) {
    int is = 0, ic = 0;
    for (int kind : kinds) {
      std::vector<BDesc> sm, fa, co;
      std::vector<int> bsm, bre, bfa, bpr, bco;
      for (int s = 0; s < count; ++s) {
        if (models[s].kind != kind) continue;
        const int last = B->sv[s].nlev - 1;
        const int n = B->sv[s].N >> l;
        if (l < last) {
          sm.push_back(desc(s, l));
          bsm.push_back(smooth_blocks(n, rows, l == 0 && models[s].kind != KCQ));
          bre.push_back(restrict_blocks(n));
          bpr.push_back(prolong_blocks(n));
          fa.push_back(desc(s, l + 1));
          bfa.push_back(((n / 2 + 63) / 64) * (n / 2) * (n / 2));
        } else if (l == last) {
          co.push_back(desc(s, l));
          bco.push_back(1);
        }
      }
      if (!sm.empty()) {
        add_phase(P->lv[l].smooth[is], sm, bsm);
        add_phase(P->lv[l].restrict_[is], sm, bre);
        add_phase(P->lv[l].fas[is], fa, bfa);
        add_phase(P->lv[l].prolong[is], sm, bpr);
        ++is;
      }
      if (!co.empty()) add_phase(P->lv[l].coarse[ic++], co, bco);
    }
  }
  // fine-level tables for the FP64 kernels (outer residual tiles; apply in 256-cell blocks)
  std::vector<std::vector<BFine>> fk(kinds.size());
  P->outer.assign(kinds.size(), {});
  P->apply.assign(kinds.size(), {});
  std::vector<size_t> fine_off(kinds.size()), fpo(kinds.size()), fpa(kinds.size());
  for (size_t g = 0; g < kinds.size(); ++g) {
    std::vector<int> bo, ba;
    for (int s = 0; s < count; ++s) {
      if (models[s].kind != kinds[g]) continue;
      BFine f;
      memset(&f, 0, sizeof(f));
      const Batch::S& v = B->sv[s];
      f.n = v.N;
      f.solve = s;
      f.m = models[s];
      f.u = field[s];
      f.src = v.src64;
      f.ffc = B->ffc + s;
      f.rho = rho_in[s];
      f.ub = v.ub[0];
      f.tau = v.S32[0];
      f.e = v.e[0];
      f.q = (models[s].kind == KFR1 || models[s].kind == KFR2) ? v.q0 : nullptr;
      fk[g].push_back(f);
      bo.push_back((v.N / 32) * (v.N / 8) * ((v.N + 63) / 64));
      ba.push_back((int)(((size_t)v.N * v.N * v.N + 255) / 256));
    }
    P->outer[g].kind = P->apply[g].kind = kinds[g];
    // stage BFine tables with the same layout helper (reinterpret as bytes)
    size_t d_off = align(host.size());
    host.resize(d_off + fk[g].size() * sizeof(BFine));
    memcpy(host.data() + d_off, fk[g].data(), fk[g].size() * sizeof(BFine));
    fine_off[g] = d_off;
    auto put_prefix = [&](const std::vector<int>& bl, Phase& ph) {
      size_t p_off = align(host.size());
      host.resize(p_off + (bl.size() + 1) * sizeof(int));
      int* pf = (int*)(host.data() + p_off);
      int acc = 0;
      for (size_t i = 0; i < bl.size(); ++i) { pf[i] = acc; acc += bl[i]; }
      pf[bl.size()] = acc;
      ph.blocks = acc;
      ph.cnt = (int)bl.size();
      return p_off;
    };
    fpo[g] = put_prefix(bo, P->outer[g]);
    fpa[g] = put_prefix(ba, P->apply[g]);
  }
  // upload
  if (B->tables) cudaFree(B->tables);
  B->tables = nullptr;
  if (cudaMalloc(&B->tables, host.size() + 256) != cudaSuccess) {
    cudaGetLastError();
    return MGGLAM_ERR_OOM;
  }
  B->tables_bytes = host.size();
  MG_CUDA_TRY(cudaMemcpyAsync(B->tables, host.data(), host.size(), cudaMemcpyHostToDevice, st));
  MG_CUDA_TRY(cudaStreamSynchronize(st));
  char* tb = (char*)B->tables;
  for (auto& pd : pend) {
    pd.ph->d = (BDesc*)(tb + pd.d_off);
    pd.ph->prefix = (int*)(tb + pd.p_off);
  }
  P->fine_desc.resize(kinds.size());
  P->fine_prefix.resize(kinds.size());
  for (size_t g = 0; g < kinds.size(); ++g) {
    P->fine_desc[g] = (BFine*)(tb + fine_off[g]);
    P->outer[g].prefix = (int*)(tb + fpo[g]);
    P->apply[g].prefix = (int*)(tb + fpa[g]);
  }
  return MGGLAM_OK;
}

static void launch_smooth_phase(const Phase& ph, int rows, const int* active, int parity, cudaStream_t st) {
  if (ph.blocks == 0) return;
  switch (rows) {
    case 2: MG_BDISPATCH(ph.kind, (kb_smooth<KK, 2><<<ph.blocks, dim3(32, 2), 0, st>>>(ph.d, ph.prefix, ph.cnt, active, parity))); break;
    case 8: MG_BDISPATCH(ph.kind, (kb_smooth<KK, 8><<<ph.blocks, dim3(32, 8), 0, st>>>(ph.d, ph.prefix, ph.cnt, active, parity))); break;
    default: MG_BDISPATCH(ph.kind, (kb_smooth<KK, 4><<<ph.blocks, dim3(32, 4), 0, st>>>(ph.d, ph.prefix, ph.cnt, active, parity))); break;
  }
  note_launch(1);
}

// One V-cycle of every active solve.
static void batch_vcycle(const Plan& P, const int* active, unsigned long long* guards, const mgglam_params& prm,
                         int rows, cudaStream_t st) {
  const int Lmax = (int)P.lv.size();
  for (int l = 0; l < Lmax; ++l) {
    const auto& L = P.lv[l];
    for (size_t g = 0; g < L.smooth.size(); ++g) {
      for (int s = 0; s < prm.nu1; ++s)
        for (int par = 0; par < 2; ++par) launch_smooth_phase(L.smooth[g], rows, active, par, st);
      const Phase& r = L.restrict_[g];
      MG_BDISPATCH(r.kind, (kb_restrict<KK><<<r.blocks, dim3(32, 4), 0, st>>>(r.d, r.prefix, r.cnt, active)));
      const Phase& f = L.fas[g];
      MG_BDISPATCH(f.kind, (kb_fas<KK><<<f.blocks, 64, 0, st>>>(f.d, f.prefix, f.cnt, active)));
      note_launch(2);
    }
    for (const Phase& c : L.coarse) {
      MG_BDISPATCH(c.kind, (kb_coarse<KK><<<c.cnt, 512, 0, st>>>(c.d, active, prm.coarse_sweeps)));
      note_launch(1);
    }
  }
  for (int l = Lmax - 2; l >= 0; --l) {
    const auto& L = P.lv[l];
    for (size_t g = 0; g < L.prolong.size(); ++g) {
      const Phase& p = L.prolong[g];
      const bool so = prm.nu2 >= 1;  // the same for every solve of the batch
      const dim3 b4(32, 4);
      if (p.kind == KFR1 && so) kb_prolong<true, KFR1, true><<<p.blocks, b4, 0, st>>>(p.d, p.prefix, p.cnt, active, guards);
      else if (p.kind == KFR1) kb_prolong<true, KFR1><<<p.blocks, b4, 0, st>>>(p.d, p.prefix, p.cnt, active, guards);
      else if (p.kind == KFR2 && so) kb_prolong<true, KFR2, true><<<p.blocks, b4, 0, st>>>(p.d, p.prefix, p.cnt, active, guards);
      else if (p.kind == KFR2) kb_prolong<true, KFR2><<<p.blocks, b4, 0, st>>>(p.d, p.prefix, p.cnt, active, guards);
      else if (is_fr(p.kind)) kb_prolong<true><<<p.blocks, b4, 0, st>>>(p.d, p.prefix, p.cnt, active, guards);
      else kb_prolong<false><<<p.blocks, b4, 0, st>>>(p.d, p.prefix, p.cnt, active, guards);
      note_launch(1);
      for (int s = 0; s < prm.nu2; ++s)
        for (int par = 0; par < 2; ++par) launch_smooth_phase(L.smooth[g], rows, active, par, st);
    }
  }
}

int solve_batch(int count, const mgglam_params* prm, const double* a, const float* const* rho, const int* N,
                double* const* field, double tol, mgglam_stats* stats, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  // models and constants
  std::vector<ModelDev> models(count);
  std::vector<std::vector<LevelF>> lfs(count);
  int rc;
  for (int s = 0; s < count; ++s) {
    if ((rc = make_model(&prm[s], a[s], N[s], &models[s]))) return rc;
    const int nl = count_levels(N[s], prm[s].levels);
    for (int l = 0; l < nl; ++l) lfs[s].push_back(make_levelf(models[s], (double)(1 << l)));
  }
  Batch* B = nullptr;
  if ((rc = get_batch(count, N, prm, &B))) return rc;
  // per-solve setup (density mean, FP64 source, density pyramid, background, source norm)
  for (int s = 0; s < count; ++s) {
    const Batch::S& v = B->sv[s];
    const long long n3 = (long long)v.N * v.N * v.N;
    if ((rc = launch_density_mean(rho[s], (size_t)n3, B->partials, B->rmean + s, st))) return rc;
    if (models[s].kind == KCQ) {
      MG_BDISPATCH(models[s].kind, (k_src64<KK><<<stream_grid(n3), kThreads, 0, st>>>(
                                       models[s], rho[s], n3, B->rmean + s, v.src64)));
    } else {
      k_ff_consts<<<1, 32, 0, st>>>(models[s], n3, B->rmean + s, B->ffc + s);
    }
    const bool split = models[s].kind != KCQ;
    if (split) k_density_norm32_split<<<stream_grid(n3), kThreads, 0, st>>>(rho[s], v.N, B->rmean + s, v.rho32[0]);
    else k_density_norm32<<<stream_grid(n3), kThreads, 0, st>>>(rho[s], n3, B->rmean + s, v.rho32[0]);
    for (int l = 1; l < v.nlev; ++l) {
      const int nc = v.N >> l;
      if (l == 1 && split)
        k_restrict32_from_split<<<dim3((nc + 63) / 64, nc, nc), 64, 0, st>>>(v.N, v.rho32[0], v.rho32[1]);
      else
        k_restrict32<<<dim3((nc + 63) / 64, nc, nc), 64, 0, st>>>(v.N >> (l - 1), v.rho32[l - 1], v.rho32[l]);
    }
    if ((rc = launch_init_background(models[s], field[s], (size_t)n3, st))) return rc;
    MG_BDISPATCH(models[s].kind, (k_src_sumsq32<KK><<<stream_grid(n3), kThreads, 0, st>>>(
                                     models[s], rho[s], n3, B->rmean + s, B->partials)));
    k_finalize_sum32<<<1, 1024, 0, st>>>(B->partials, stream_grid(n3), B->ssum + s);
    MG_CUDA_TRY(cudaMemsetAsync(v.e[0], 0, (size_t)n3 * 4, st));
    MG_CUDA_TRY(cudaMemsetAsync(v.q0, 0, (size_t)n3 * 4, st));  // Delta w(u, 0) = 0
    note_launch(5 + v.nlev);
  }
  Plan P;
  if ((rc = build_plan(B, models, lfs, std::vector<const float*>(rho, rho + count), field, prm, false,
                       B->rows ? B->rows : 4, &P, st)))
    return rc;
  const int ng = (int)P.outer.size();
  auto outer_residual = [&]() -> int {
    for (int g = 0; g < ng; ++g) {
      const Phase& o = P.outer[g];
      // partial slots: each group's blocks start after the previous groups'
      int base = 0;
      for (int h = 0; h < g; ++h) base += P.outer[h].blocks;
      MG_BDISPATCH(o.kind, (kb_outer_residual<KK><<<o.blocks, 256, 0, st>>>(P.fine_desc[g], o.prefix, o.cnt,
                                                                             B->active, B->partials + base)));
      kb_finalize<<<o.cnt, 256, 0, st>>>(P.fine_desc[g], o.prefix, o.cnt, B->partials + base, B->sums);
      note_launch(2);
    }
    MG_CUDA_TRY(cudaMemcpyAsync(B->h_sums, B->sums, count * 8, cudaMemcpyDeviceToHost, st));
    MG_CUDA_TRY(cudaMemcpyAsync(B->h_sums + count, B->ssum, count * 8, cudaMemcpyDeviceToHost, st));
    MG_CUDA_TRY(cudaStreamSynchronize(st));
    MG_CUDA_TRY(cudaGetLastError());
    return MGGLAM_OK;
  };
  for (int s = 0; s < count; ++s) B->h_active[s] = 1;
  MG_CUDA_TRY(cudaMemcpyAsync(B->active, B->h_active, count * 4, cudaMemcpyHostToDevice, st));
  MG_CUDA_TRY(cudaMemsetAsync(B->guards, 0, count * sizeof(unsigned long long), st));
  if ((rc = outer_residual())) return rc;
  // autotune the smoother's block height once per batch (timed on the fine
  // levels' sweeps, after the first residual has set the base field and source)
  if (B->rows == 0) {
    int best = 4;
    float best_ms = 1e30f;
    for (int cand : {2, 4, 8}) {
      Plan Pt;
      if ((rc = build_plan(B, models, lfs, std::vector<const float*>(rho, rho + count), field, prm, false, cand, &Pt, st)))
        return rc;
      for (int s = 0; s < count; ++s) B->h_active[s] = 1;
      MG_CUDA_TRY(cudaMemcpyAsync(B->active, B->h_active, count * 4, cudaMemcpyHostToDevice, st));
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      for (const Phase& ph : Pt.lv[0].smooth) launch_smooth_phase(ph, cand, B->active, 0, st);  // warm
      cudaEventRecord(e0, st);
      for (int rep = 0; rep < 3; ++rep)
        for (const Phase& ph : Pt.lv[0].smooth) launch_smooth_phase(ph, cand, B->active, rep & 1, st);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (ms < best_ms) { best_ms = ms; best = cand; }
    }
    B->rows = best;
    // the timing sweeps changed e on the fine levels: start again from zero
    for (int s = 0; s < count; ++s) {
      const size_t bytes = (size_t)B->sv[s].N * B->sv[s].N * B->sv[s].N * 4;
      MG_CUDA_TRY(cudaMemsetAsync(B->sv[s].e[0], 0, bytes, st));
      MG_CUDA_TRY(cudaMemsetAsync(B->sv[s].q0, 0, bytes, st));
    }
    if ((rc = build_plan(B, models, lfs, std::vector<const float*>(rho, rho + count), field, prm, false, B->rows, &P,
                         st)))
      return rc;
  }
  std::vector<double> snorm(count), eps(count);
  std::vector<mgglam_stats> lst(count);
  for (int s = 0; s < count; ++s) {
    const double n3 = (double)B->sv[s].N * B->sv[s].N * B->sv[s].N;
    const double src = sqrt(B->h_sums[count + s] / n3);
    snorm[s] = source_norm(models[s], src);
    eps[s] = sqrt(B->h_sums[s] / n3) / snorm[s];
    memset(&lst[s], 0, sizeof(mgglam_stats));
    lst[s].resid0 = eps[s];
    lst[s].resid_hist[0] = eps[s];
  }
  // graph of one batched V-cycle (captured per plan signature)
  if (!B->cap && cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess) return MGGLAM_ERR_CUDA;
  unsigned long long sig = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* bb = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) sig = (sig ^ bb[i]) * 1099511628211ull;
  };
  for (int s = 0; s < count; ++s) {
    mix(lfs[s].data(), lfs[s].size() * sizeof(LevelF));
    mix(&models[s].kind, sizeof(int));
    mix(&field[s], sizeof(double*));
  }
  const int shape[4] = {prm[0].nu1, prm[0].nu2, prm[0].coarse_sweeps, B->rows};
  mix(shape, sizeof(shape));
  mix(&B->tables, sizeof(void*));
  if (!(B->vexec && B->vsig == sig)) {
    if (B->vexec) { cudaGraphExecDestroy(B->vexec); B->vexec = nullptr; }
    const long long n0 = launch_count();
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      batch_vcycle(P, B->active, B->guards, prm[0], B->rows, B->cap);
      ok = cudaStreamEndCapture(B->cap, &g) == cudaSuccess && g;
    }
    B->vlaunches = launch_count() - n0;
    note_launch((int)-B->vlaunches);
    if (ok) ok = cudaGraphInstantiate(&B->vexec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) { cudaGetLastError(); B->vexec = nullptr; return MGGLAM_ERR_CUDA; }
    B->vsig = sig;
  }
  int cyc = 0, outer = 0, status = MGGLAM_OK;
  double rho_est = kInitialContraction;
  const int maxc = prm[0].max_cycles;
  auto worst = [&]() {
    double w = 0.0;
    for (int s = 0; s < count; ++s)
      if (B->h_active[s]) w = fmax(w, eps[s] / fmax(tol, 1e-300));
    return w;
  };
  while (cyc < maxc) {
    bool any = false;
    for (int s = 0; s < count; ++s) {
      const bool act = !(eps[s] <= tol) && isfinite(eps[s]);
      B->h_active[s] = act ? 1 : 0;
      any = any || act;
    }
    if (!any) break;
    MG_CUDA_TRY(cudaMemcpyAsync(B->active, B->h_active, count * 4, cudaMemcpyHostToDevice, st));
    // e <- 0 on the fine levels of the active solves
    for (int g = 0; g < ng; ++g) {
      kb_apply<<<P.apply[g].blocks, 256, 0, st>>>(P.fine_desc[g], P.apply[g].prefix, P.apply[g].cnt, B->active, 1);
      note_launch(1);
    }
    int inner = prm[0].inner_cycles;
    if (inner <= 0) {
      const double lr = log(rho_est);
      const int need = (int)ceil(log(1.0 / worst()) / lr - 1e-9);
      const int cap = (int)ceil(log(kFp32StepGain) / lr - 1e-9);
      inner = need < 1 ? 1 : (need > cap ? cap : need);
    }
    double worst_before = worst();
    int done = 0;
    for (int c = 0; c < inner && cyc < maxc; ++c, ++cyc, ++done) {
      MG_CUDA_TRY(cudaGraphLaunch(B->vexec, st));
      note_launch((int)B->vlaunches);
      for (int s = 0; s < count; ++s)
        if (B->h_active[s]) ++lst[s].cycles;
    }
    for (int g = 0; g < ng; ++g) {
      kb_apply<<<P.apply[g].blocks, 256, 0, st>>>(P.fine_desc[g], P.apply[g].prefix, P.apply[g].cnt, B->active, 0);
      note_launch(1);
    }
    ++outer;
    if ((rc = outer_residual())) return rc;
    for (int s = 0; s < count; ++s) {
      if (!B->h_active[s]) continue;
      const double n3 = (double)B->sv[s].N * B->sv[s].N * B->sv[s].N;
      eps[s] = sqrt(B->h_sums[s] / n3) / snorm[s];
      ++lst[s].outer;
      if (lst[s].outer < 64) lst[s].resid_hist[lst[s].outer] = eps[s];
    }
    const double worst_after = worst();
    if (done > 0 && worst_after > 0.0 && worst_after < worst_before && worst_after / worst_before > kFp32StepGain)
      rho_est = fmin(0.5, fmax(0.01, pow(worst_after / worst_before, 1.0 / done)));
  }
  MG_CUDA_TRY(cudaMemcpyAsync(B->h_guards, B->guards, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                              st));
  MG_CUDA_TRY(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int s = 0; s < count; ++s) {
    lst[s].guarded = (long long)B->h_guards[s];
    lst[s].resid = eps[s];
    lst[s].converged = eps[s] <= tol;
    lst[s].seconds = secs;
    if (!isfinite(eps[s])) status = MGGLAM_ERR_NONFINITE;
    else if (status == MGGLAM_OK && !lst[s].converged) status = MGGLAM_ERR_NOT_CONVERGED;
    if (stats) stats[s] = lst[s];
  }
  return status;
}

}  // namespace mg

extern "C" int mgglam_solve_batch(int count, const mgglam_params* prm, const double* a, const float* const* rho,
                                  const int* N, double* const* field, double tol, mgglam_stats* stats, void* stream) {
  if (count < 1 || !prm || !a || !rho || !N || !field || !(tol >= 0.0)) return MGGLAM_ERR_ARG;
  for (int s = 0; s < count; ++s) {
    if (!rho[s] || !field[s]) return MGGLAM_ERR_ARG;
    if (N[s] < 32 || N[s] > 2048 || N[s] % 32) return MGGLAM_ERR_SHAPE;
    if (prm[s].nu1 != prm[0].nu1 || prm[s].nu2 != prm[0].nu2 || prm[s].coarse_sweeps != prm[0].coarse_sweeps)
      return MGGLAM_ERR_ARG;
    if (prm[s].nu1 < 0 || prm[s].nu2 < 0 || prm[s].coarse_sweeps < 0) return MGGLAM_ERR_ARG;
    if (prm[s].cycle != 0) return MGGLAM_ERR_ARG;  // batched solves run V-cycles
  }
  return mg::solve_batch(count, prm, a, rho, N, field, tol, stats, (cudaStream_t)stream);
}
