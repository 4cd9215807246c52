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

#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

// Periodic cell index and weight pair along one axis for coordinate x.
__device__ __forceinline__ void cic_axis(float x, int N, int& i0, int& i1, double& w0, double& w1) {
  // wrap into [0, N)
  float xf = fmodf(x, (float)N);
  if (xf < 0.f) xf += (float)N;
  if (xf >= (float)N) xf = 0.f;
  const double xs = (double)xf - 0.5;
  const double fl = floor(xs);
  const double f = xs - fl;
  int i = (int)fl;  // -1 .. N-1
  i0 = i < 0 ? i + N : i;
  i1 = i + 1 >= N ? i + 1 - N : i + 1;
  w0 = 1.0 - f;
  w1 = f;
}

__global__ void __launch_bounds__(kThreads) k_deposit_fixed(const float* __restrict__ pos, long long np, int N,
                                                            unsigned long long* __restrict__ acc) {
  const double scale = 4294967296.0;  // 2^32
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < np;
       q += (long long)gridDim.x * blockDim.x) {
    int i0, i1, j0, j1, k0, k1;
    double wx0, wx1, wy0, wy1, wz0, wz1;
    cic_axis(pos[3 * q + 0], N, i0, i1, wx0, wx1);
    cic_axis(pos[3 * q + 1], N, j0, j1, wy0, wy1);
    cic_axis(pos[3 * q + 2], N, k0, k1, wz0, wz1);
    const int ii[2] = {i0, i1}, jj[2] = {j0, j1}, kk[2] = {k0, k1};
    const double wx[2] = {wx0, wx1}, wy[2] = {wy0, wy1}, wz[2] = {wz0, wz1};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const double w = wx[a] * wy[b] * wz[c];
          const unsigned long long v = (unsigned long long)llrint(w * scale);
          if (v) atomicAdd(&acc[cidx(N, ii[a], jj[b], kk[c])], v);
        }
  }
}

__global__ void k_deposit_finish(const unsigned long long* __restrict__ acc, long long n3, double mass,
                                 float* __restrict__ rho) {
  const double s = mass / 4294967296.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x)
    rho[t] = (float)((double)acc[t] * s);
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
  k_deposit_fixed<<<grid_for(np, kThreads, 1 << 20), kThreads, 0, st>>>(pos, np, N, acc);
  prof_end(st);
  prof_begin(PC_DEPOSIT_FINISH, st, 12.0 * n3);
  k_deposit_finish<<<grid_for(n3, kThreads, 1 << 20), kThreads, 0, st>>>(acc, n3, (double)n3 / (double)np, rho);
  prof_end(st);
  note_launch(2);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

// ---------------------------------------------------------------------------
// Gather
// ---------------------------------------------------------------------------

// T - Tbar per cell, formed in FP64 and stored in FP32.
template <int K>
__global__ void k_transform(const double* __restrict__ u, long long n3, double ubar, double beta,
                            float* __restrict__ T) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    const double v = u[t];
    double d;
    if constexpr (K == KFR0) d = -(v - ubar);
    else if constexpr (K == KFR1) d = -(v - ubar) * (v + ubar);
    else if constexpr (K == KFR2) d = -(v - ubar) * (v * v + v * ubar + ubar * ubar);
    else if constexpr (K == KSYM) d = (v - ubar) * (v + ubar);
    else d = beta * v;
    T[t] = (float)d;
  }
}

__global__ void __launch_bounds__(kThreads) k_gather(const float* __restrict__ T, int N, const float* __restrict__ pos,
                                                     long long np, float scale, float* __restrict__ force) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < np;
       q += (long long)gridDim.x * blockDim.x) {
    int i0, i1, j0, j1, k0, k1;
    double wx0, wx1, wy0, wy1, wz0, wz1;
    cic_axis(pos[3 * q + 0], N, i0, i1, wx0, wx1);
    cic_axis(pos[3 * q + 1], N, j0, j1, wy0, wy1);
    cic_axis(pos[3 * q + 2], N, k0, k1, wz0, wz1);
    const int ii[2] = {i0, i1}, jj[2] = {j0, j1}, kk[2] = {k0, k1};
    const float wx[2] = {(float)wx0, (float)wx1}, wy[2] = {(float)wy0, (float)wy1}, wz[2] = {(float)wz0, (float)wz1};
    float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int i = ii[a], j = jj[b], k = kk[c];
          const int ip = i + 1 == N ? 0 : i + 1, im = i == 0 ? N - 1 : i - 1;
          const int jp = j + 1 == N ? 0 : j + 1, jm = j == 0 ? N - 1 : j - 1;
          const int kp = k + 1 == N ? 0 : k + 1, km = k == 0 ? N - 1 : k - 1;
          const float w = wx[a] * wy[b] * wz[c];
          fx += w * (T[cidx(N, ip, j, k)] - T[cidx(N, im, j, k)]);
          fy += w * (T[cidx(N, i, jp, k)] - T[cidx(N, i, jm, k)]);
          fz += w * (T[cidx(N, i, j, kp)] - T[cidx(N, i, j, km)]);
        }
    force[3 * q + 0] = 0.5f * scale * fx;
    force[3 * q + 1] = 0.5f * scale * fy;
    force[3 * q + 2] = 0.5f * scale * fz;
  }
}

int gather_force(const ModelDev& m, int kind, int n_fr, const mgglam_params* prm, const double* field, int N,
                 const float* pos, long long np, float* force, double prefactor, cudaStream_t st) {
  (void)n_fr;
  Workspace* ws = nullptr;
  int rc = get_workspace(N, MGGLAM_MIXED, 0, &ws);
  if (rc) return rc;
  float* T = ws->lev[0].ub;  // scratch mesh of N^3 floats
  const long long n3 = (long long)N * N * N;
  const int g = grid_for(n3, kThreads, 1 << 20);
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
  if (is_fr(kind)) scale = 0.5 * m.c2;  // F = (c~^2/2) grad f_R
  else if (kind == KSYM)
    scale = -3.0 * prm->xi * prm->xi * prm->omega_m * prm->beta_star * prm->beta_star * m.c2 /
            (prm->a_star * prm->a_star * prm->a_star);
  else
    scale = -1.0;  // F = -grad(beta phi)
  prof_begin(PC_GATHER, st, 24.0 * np + 4.0 * n3);
  k_gather<<<grid_for(np, kThreads, 1 << 20), kThreads, 0, st>>>(T, N, pos, np, (float)(scale * prefactor), force);
  prof_end(st);
  note_launch(2);
  MG_CUDA_TRY(cudaGetLastError());
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
// on the first call and cached.

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
  k_deposit_fixed<<<grid_for(np, kThreads, 1 << 20), kThreads, 0, st>>>(pos, np, N, acc);
  k_deposit_finish<<<grid_for(n3, kThreads, 1 << 20), kThreads, 0, st>>>(acc, n3, (double)n3 / (double)np, rho);
  note_launch(2);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}
