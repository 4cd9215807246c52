// particles.cu -- CIC density assignment and the fifth-force gather (Sec. 3.1).
//
// Deposit: each particle spreads mass N^3/np over the 8 nearest cell centres
// (centre of cell c at c + 1/2) with weights prod_d (1 - |x_d - c_d - 1/2|),
// periodic.  The weights are accumulated as 64-bit fixed-point integers
// (units of 2^-32 of one particle's weight) with integer atomics, so the sum is
// independent of the order in which particles arrive: the mesh is bitwise
// reproducible.  A second pass scales to float32 density.
//
// Gather: the field transform T (f(R): f_R = -u^{n+1}; symmetron: u^2; CQ:
// beta phi) is formed once per cell in FP64 and stored as the FP32 perturbation
// T - Tbar (Tbar = T of the background field), which keeps the central
// difference (T_{c+1} - T_{c-1})/2 free of cancellation in single precision.
// Each particle then interpolates the three-point differences of the 8 cells
// around it with its CIC weights.
#include <math.h>

#include <mutex>

#include "cic.cuh"
#include "ff.cuh"
#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

// round(x * 2^31) for 0 <= x < 2^32 by integer operations on the float's bits
// (exact for x >= 2^-8, whose bits all lie at or above 2^-31).
__device__ __forceinline__ unsigned long long fix31(float x) {
  const unsigned b = __float_as_uint(x);
  const int ex = (int)(b >> 23);
  if (ex == 0) return 0ull;  // zero (or subnormal: far below 2^-31)
  const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = ex - 127 - 23 + 31;  // x * 2^31 = m * 2^sh
  if (sh >= 0) return m << sh;
  if (sh < -25) return 0ull;
  return (m + (1ull << (-sh - 1))) >> (-sh);
}

// CIC along one axis in fixed point: cells c0 = floor(x - 1/2), c1 = c0 + 1
// (periodic) and weights W0 = 1 - f, W1 = f in units of 2^-31, f = the
// fractional part of x - 1/2 -- the same numbers the FP64 definition gives,
// without double-precision arithmetic (GB300's FP64 rate is 1/64 of FP32).
__device__ __forceinline__ void cic_axis_fixed(float x, int N, int& c0, int& c1, unsigned long long& W0,
                                               unsigned long long& W1) {
  const long long xs = (long long)fix31(wrap_pos(x, N)) - (1ll << 30);
  const int c = (int)(xs >> 31);  // -1 .. N-1 (arithmetic shift = floor)
  const unsigned long long F = (unsigned long long)(xs & 0x7FFFFFFFll);
  c0 = c < 0 ? c + N : c;
  c1 = c + 1 >= N ? c + 1 - N : c + 1;
  W1 = F;
  W0 = (1ull << 31) - F;
}

// round(P W / 2^61) for P <= 2^62, W <= 2^31: a product of three axis weights
// (units 2^-93) rounded to the accumulator's unit 2^-32, exactly.
__device__ __forceinline__ unsigned long long wmul(unsigned long long P, unsigned long long W) {
  const unsigned long long lo = P * W, hi = __umul64hi(P, W);
  return ((hi << 3) | (lo >> 61)) + ((lo >> 60) & 1ull);
}

// One particle per lane, warps over consecutive particles.  A lane's four
// cells in its upper k plane are the next lane's lower-plane cells whenever
// the two particles share (i0, j0) and sit in adjacent k cells (neighbours in
// a lattice-ordered particle array do): the next lane then adds them to its
// own and this lane skips those atomics.  Integer sums are exact, so the mesh
// does not depend on which lane issues an update.
template <typename IT>
__global__ void __launch_bounds__(kThreads) k_deposit_fixed(const float* __restrict__ pos, long long np, int N,
                                                            unsigned long long* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < np; base += stride) {
    const long long q = base + lane;
    const bool ok = q < np;
    int i0 = 0, i1 = 0, j0 = 0, j1 = 0, k0 = -1, k1 = -2;
    unsigned long long X0 = 0, X1 = 0, Y0 = 0, Y1 = 0, Z0 = 0, Z1 = 0;
    if (ok) {
      cic_axis_fixed(pos[3 * q + 0], N, i0, i1, X0, X1);
      cic_axis_fixed(pos[3 * q + 1], N, j0, j1, Y0, Y1);
      cic_axis_fixed(pos[3 * q + 2], N, k0, k1, Z0, Z1);
    }
    const unsigned long long P[4] = {X0 * Y0, X0 * Y1, X1 * Y0, X1 * Y1};  // (a, b) = 00, 01, 10, 11
    unsigned long long lo[4], up[4];                                          // k0 and k1 planes
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      lo[s] = wmul(P[s], Z0);
      up[s] = wmul(P[s], Z1);
    }
    const int pi = __shfl_up_sync(0xffffffffu, i0, 1), pj = __shfl_up_sync(0xffffffffu, j0, 1);
    const int pk = __shfl_up_sync(0xffffffffu, k1, 1);
    const bool take = lane > 0 && ok && pi == i0 && pj == j0 && pk == k0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const unsigned long long w = __shfl_up_sync(0xffffffffu, up[s], 1);
      if (take) lo[s] += w;
    }
    const bool given = __shfl_down_sync(0xffffffffu, (int)take, 1) != 0 && lane < 31;
    if (ok) {
      const IT ri[2] = {(IT)i0 * N, (IT)i1 * N};
      const int jj[2] = {j0, j1};
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const IT row = (ri[s >> 1] + jj[s & 1]) * N;
        if (lo[s]) atomicAdd(&acc[row + k0], lo[s]);
        if (!given && up[s]) atomicAdd(&acc[row + k1], up[s]);
      }
    }
  }
}

__global__ void k_deposit_finish(const unsigned long long* __restrict__ acc, long long n3, double mass,
                                 float* __restrict__ rho) {
  // single-precision scaling of the correctly rounded float of the sum (the
  // output is FP32): within one ulp of the exact product
  const float s = (float)(mass / 4294967296.0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    rho[t] = __ull2float_rn(acc[t]) * s;
}

// Scratch for the fixed-point accumulator, cached per (device, N).
static int deposit_scratch(int N, unsigned long long** acc) {
  Workspace* ws = nullptr;
  int rc = get_workspace(N < 4 ? 4 : (N % 2 ? N + 1 : N), MGGLAM_FP64, 1, &ws);
  if (rc) return rc;
  const size_t need = (size_t)N * N * N * sizeof(unsigned long long);
  if (ws->cic_bytes < need) {
    if (ws->cic_acc) cudaFree(ws->cic_acc);
    ws->cic_acc = nullptr;
    ws->cic_bytes = 0;
    if (cudaMalloc((void**)&ws->cic_acc, need) != cudaSuccess) {
      cudaGetLastError();
      return MGGLAM_ERR_OOM;
    }
    ws->cic_bytes = need;
  }
  *acc = (unsigned long long*)ws->cic_acc;
  return MGGLAM_OK;
}

int deposit_cic(const float* pos, long long np, int N, float* rho, cudaStream_t st) {
  unsigned long long* acc = nullptr;
  int rc = deposit_scratch(N, &acc);
  if (rc) return rc;
  const long long n3 = (long long)N * N * N;
  MG_CUDA_TRY(cudaMemsetAsync(acc, 0, (size_t)n3 * sizeof(unsigned long long), st));
  prof_begin(PC_DEPOSIT, st, 12.0 * np);
  // 32-bit cell offsets where the mesh has at most 2^30 cells
  (N <= 1024 ? k_deposit_fixed<int> : k_deposit_fixed<long long>)<<<grid_for(np, kThreads, 1 << 20), kThreads, 0,
                                                                     st>>>(pos, np, N, acc);
  prof_end(st);
  prof_begin(PC_DEPOSIT_FINISH, st, 12.0 * n3);
  k_deposit_finish<<<stream_grid(n3), kThreads, 0, st>>>(acc, n3, (double)n3 / (double)np, rho);
  prof_end(st);
  note_launch(2);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

// ---------------------------------------------------------------------------
// Gather
// ---------------------------------------------------------------------------

// T - Tbar per cell, stored in FP32.  f(R) and the symmetron form it in
// float-float (FP32 instructions; the exact split of the FP64 field, v - ubar
// exact to first order, ~48-bit products), which rounds to the same float as
// FP64 would at 1/64 of FP32's rate; CQ (one product) stays in FP64.
template <int K>
__global__ void k_transform(const double* __restrict__ u, long long n3, double ubar, double beta,
                            float* __restrict__ T) {
  const ff ub = ff_from_double(ubar);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    if constexpr (K == KCQ) {
      T[t] = (float)(beta * u[t]);
    } else {
      const ff v = ff_from_double(u[t]);
      const ff dv = ff_sub(v, ub);  // v - ubar
      ff d;
      if constexpr (K == KFR0) d = ff_neg(dv);
      else if constexpr (K == KFR1) d = ff_neg(ff_mul(dv, ff_add(v, ub)));
      else if constexpr (K == KFR2) d = ff_neg(ff_mul(dv, ff_add(ff_add(ff_sqr(v), ff_mul(v, ub)), ff_sqr(ub))));
      else d = ff_mul(dv, ff_add(v, ub));  // symmetron: u^2 - ubar^2
      T[t] = ff_to_float(d);
    }
  }
}

// One particle per thread (cic_grad: the 32 distinct cells its three central
// differences at the 8 CIC cells touch).
template <typename IT>
__global__ void __launch_bounds__(kThreads) k_gather(const float* __restrict__ T, int N, const float* __restrict__ pos,
                                                     long long np, float scale, float* __restrict__ force) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < np;
       q += (long long)gridDim.x * blockDim.x) {
    const float3 g = cic_grad<IT>(T, N, pos[3 * q + 0], pos[3 * q + 1], pos[3 * q + 2]);
    force[3 * q + 0] = scale * g.x;
    force[3 * q + 1] = scale * g.y;
    force[3 * q + 2] = scale * g.z;
  }
}

// Force prefactor of the gather (the spatial factor of the model's fifth force, times the caller's).
static double force_scale(const ModelDev& m, int kind, const mgglam_params* prm) {
  if (is_fr(kind)) return 0.5 * m.c2;  // F = (c~^2/2) grad f_R
  if (kind == KSYM)
    return -3.0 * prm->xi * prm->xi * prm->omega_m * prm->beta_star * prm->beta_star * m.c2 /
           (prm->a_star * prm->a_star * prm->a_star);
  return -1.0;  // F = -grad(beta phi)
}

// The gather of a range of particles on the mesh T the last gather_force call
// on this stream formed (the workspace's scratch mesh).
int gather_chunk(const ModelDev& m, int kind, const mgglam_params* prm, int N, const float* pos, long long np,
                 float* force, double prefactor, cudaStream_t st) {
  Workspace* ws = nullptr;
  int rc = get_workspace(N, MGGLAM_MIXED, 0, &ws);
  if (rc) return rc;
  const float* T = ws->lev[0].ub;
  prof_begin(PC_GATHER, st, 24.0 * np);
  (N <= 1024 ? k_gather<int> : k_gather<long long>)<<<grid_for(np, kThreads, 1 << 20), kThreads, 0, st>>>(
      T, N, pos, np, (float)(force_scale(m, kind, prm) * prefactor), force);
  prof_end(st);
  note_launch(1);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int gather_force(const ModelDev& m, int kind, int n_fr, const mgglam_params* prm, const double* field, int N,
                 const float* pos, long long np, float* force, double prefactor, cudaStream_t st) {
  (void)n_fr;
  Workspace* ws = nullptr;
  int rc = get_workspace(N, MGGLAM_MIXED, 0, &ws);
  if (rc) return rc;
  float* T = ws->lev[0].ub;  // scratch mesh of N^3 floats
  const long long n3 = (long long)N * N * N;
  const int g = stream_grid(n3);
  double scale;
  prof_begin(PC_TRANSFORM, st, 12.0 * n3);
  switch (kind) {
    case KFR0: k_transform<KFR0><<<g, kThreads, 0, st>>>(field, n3, m.ubar, 0.0, T); break;
    case KFR1: k_transform<KFR1><<<g, kThreads, 0, st>>>(field, n3, m.ubar, 0.0, T); break;
    case KFR2: k_transform<KFR2><<<g, kThreads, 0, st>>>(field, n3, m.ubar, 0.0, T); break;
    case KSYM: k_transform<KSYM><<<g, kThreads, 0, st>>>(field, n3, m.ubar, 0.0, T); break;
    default: k_transform<KCQ><<<g, kThreads, 0, st>>>(field, n3, 0.0, prm->beta, T); break;
  }
  prof_end(st);
  scale = force_scale(m, kind, prm);
  prof_begin(PC_GATHER, st, 24.0 * np + 4.0 * n3);
  // 32-bit cell offsets where the mesh has at most 2^30 cells
  (N <= 1024 ? k_gather<int> : k_gather<long long>)<<<grid_for(np, kThreads, 1 << 20), kThreads, 0, st>>>(
      T, N, pos, np, (float)(scale * prefactor), force);
  prof_end(st);
  note_launch(2);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

// ---------------------------------------------------------------------------
// Host input / output overlapped with the kernels
// ---------------------------------------------------------------------------
//
// The particles live in page-locked host memory.  The deposit copies them to a
// device buffer in chunks on a second stream, and deposits chunk c as soon as
// its copy has landed (stream-ordered by an event), so the host-link copy and
// the atomics overlap; the gather computes chunk c and copies its forces back
// while chunk c+1 is computed.  One copy stream and an event pool per device.

constexpr int kMaxIoChunks = 32;

struct HostIo {
  int device = -1;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev[kMaxIoChunks + 2] = {};
};

static int host_io(HostIo** out) {
  static std::mutex mu;
  static HostIo io[16];
  int dev = 0;
  MG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 16) return MGGLAM_ERR_CUDA;
  std::lock_guard<std::mutex> lk(mu);
  HostIo& h = io[dev];
  if (h.device != dev) {
    MG_CUDA_TRY(cudaStreamCreateWithFlags(&h.cs, cudaStreamNonBlocking));
    for (int i = 0; i < kMaxIoChunks + 2; ++i)
      MG_CUDA_TRY(cudaEventCreateWithFlags(&h.ev[i], cudaEventDisableTiming));
    h.device = dev;
  }
  *out = &h;
  return MGGLAM_OK;
}

int deposit_cic_host(const float* pos_host, float* pos_dev, long long np, int N, float* rho, int chunks,
                     cudaStream_t st) {
  unsigned long long* acc = nullptr;
  int rc = deposit_scratch(N, &acc);
  if (rc) return rc;
  HostIo* io = nullptr;
  if ((rc = host_io(&io))) return rc;
  const long long n3 = (long long)N * N * N;
  const long long per = (np + chunks - 1) / chunks;
  MG_CUDA_TRY(cudaMemsetAsync(acc, 0, (size_t)n3 * sizeof(unsigned long long), st));
  // the copies must not overwrite pos_dev before earlier work on st is done with it
  MG_CUDA_TRY(cudaEventRecord(io->ev[kMaxIoChunks], st));
  MG_CUDA_TRY(cudaStreamWaitEvent(io->cs, io->ev[kMaxIoChunks], 0));
  prof_begin(PC_DEPOSIT, st, 12.0 * np);
  for (int c = 0; c < chunks; ++c) {
    const long long q0 = c * per, cnt = q0 >= np ? 0 : (np - q0 < per ? np - q0 : per);
    if (cnt <= 0) break;
    MG_CUDA_TRY(cudaMemcpyAsync(pos_dev + 3 * q0, pos_host + 3 * q0, (size_t)cnt * 12, cudaMemcpyHostToDevice,
                                io->cs));
    MG_CUDA_TRY(cudaEventRecord(io->ev[c], io->cs));
    MG_CUDA_TRY(cudaStreamWaitEvent(st, io->ev[c], 0));
    (N <= 1024 ? k_deposit_fixed<int> : k_deposit_fixed<long long>)<<<grid_for(cnt, kThreads, 1 << 20), kThreads, 0,
                                                                       st>>>(pos_dev + 3 * q0, cnt, N, acc);
    note_launch(1);
  }
  prof_end(st);
  prof_begin(PC_DEPOSIT_FINISH, st, 12.0 * n3);
  k_deposit_finish<<<stream_grid(n3), kThreads, 0, st>>>(acc, n3, (double)n3 / (double)np, rho);
  prof_end(st);
  note_launch(1);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int gather_force_host(const ModelDev& m, int kind, const mgglam_params* prm, const double* field, int N,
                      const float* pos_dev, long long np, float* force_dev, float* force_host, double prefactor,
                      int chunks, cudaStream_t st) {
  HostIo* io = nullptr;
  int rc = host_io(&io);
  if (rc) return rc;
  // the transform and the first chunk's gather, then per chunk: gather, hand the chunk to the copy stream
  const long long per = (np + chunks - 1) / chunks;
  for (int c = 0; c < chunks; ++c) {
    const long long q0 = c * per, cnt = q0 >= np ? 0 : (np - q0 < per ? np - q0 : per);
    if (cnt <= 0) break;
    if (c == 0) {
      // transform + gather of the first chunk through the common path
      if ((rc = gather_force(m, kind, prm->n, prm, field, N, pos_dev, cnt, force_dev, prefactor, st))) return rc;
    } else {
      if ((rc = gather_chunk(m, kind, prm, N, pos_dev + 3 * q0, cnt, force_dev + 3 * q0, prefactor, st))) return rc;
    }
    MG_CUDA_TRY(cudaEventRecord(io->ev[c], st));
    MG_CUDA_TRY(cudaStreamWaitEvent(io->cs, io->ev[c], 0));
    MG_CUDA_TRY(cudaMemcpyAsync(force_host + 3 * q0, force_dev + 3 * q0, (size_t)cnt * 12, cudaMemcpyDeviceToHost,
                                io->cs));
  }
  // the caller's stream completes after the last copy
  MG_CUDA_TRY(cudaEventRecord(io->ev[kMaxIoChunks + 1], io->cs));
  MG_CUDA_TRY(cudaStreamWaitEvent(st, io->ev[kMaxIoChunks + 1], 0));
  return MGGLAM_OK;
}

}  // namespace mg

// ---------------------------------------------------------------------------
// Deposit without allocation (mgglam_deposit_cic_static)
// ---------------------------------------------------------------------------
//
// The accumulator lives in a fixed file-scope device array instead of the
// scratch cache, so this entry point never calls cudaMalloc.  The array's name
// is only a host-side stand-in in host code; the device address comes from
// cudaGetSymbolAddress, looked up once per device (with that device current)
// on the first call and cached until mgglam_release runs on that device (a
// reset device reloads the module, which may move the array).

namespace mg {

constexpr int kStaticDepositMaxN = 128;
constexpr size_t kStaticDepositCells = (size_t)kStaticDepositMaxN * kStaticDepositMaxN * kStaticDepositMaxN;
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_static_deposit_acc[kStaticDepositCells];

static std::mutex g_static_mu;
static unsigned long long* g_static_acc_ptr[kStaticMaxDevices];

static int static_deposit_scratch(unsigned long long** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MGGLAM_ERR_CUDA;
  }
  if (dev < 0 || dev >= kStaticMaxDevices) return MGGLAM_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_acc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_deposit_acc);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return MGGLAM_ERR_CUDA;
    }
    g_static_acc_ptr[dev] = (unsigned long long*)p;
  }
  *out = g_static_acc_ptr[dev];
  return MGGLAM_OK;
}

void forget_static_deposit_address() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (dev < 0 || dev >= kStaticMaxDevices) return;
  std::lock_guard<std::mutex> lk(g_static_mu);
  g_static_acc_ptr[dev] = nullptr;
}

}  // namespace mg

extern "C" int mgglam_deposit_cic_static(const float* pos, long long np, int N, float* rho, void* stream) {
  using namespace mg;
  if (!pos || !rho || np < 1) return MGGLAM_ERR_ARG;
  if (N < 2 || N > kStaticDepositMaxN) return MGGLAM_ERR_SHAPE;
  unsigned long long* acc = nullptr;
  int rc = static_deposit_scratch(&acc);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const long long n3 = (long long)N * N * N;
  // the array keeps the previous call's sums: clear the part this call uses
  MG_CUDA_TRY(cudaMemsetAsync(acc, 0, (size_t)n3 * sizeof(unsigned long long), st));
  // 32-bit cell offsets where the mesh has at most 2^30 cells
  (N <= 1024 ? k_deposit_fixed<int> : k_deposit_fixed<long long>)<<<grid_for(np, kThreads, 1 << 20), kThreads, 0,
                                                                     st>>>(pos, np, N, acc);
  k_deposit_finish<<<stream_grid(n3), kThreads, 0, st>>>(acc, n3, (double)n3 / (double)np, rho);
  note_launch(2);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}
