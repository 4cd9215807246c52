// fft.cu -- the PM gravity solver: the periodic Poisson equation by FFT
// (Sec. 3.1: FFTs along x, y and z, multiplication by the Green's function of
// the discrete Laplacian, inverse FFTs; Eq. GR_poisson_codeunit).
//
//   grad_h^2 Phi = coef (rho/mean - 1),   Phi_k = -coef delta_k / K_h^2,
//   K_h^2 = sum_d 4 sin^2(pi k_d / N)   (the 7-point Laplacian's eigenvalues),
//   Phi_0 = 0 (the mean of Phi is not fixed by the equation).
//
// Single-precision complex FFTs of power-of-two length N = R1 R2 (R1, R2 <= 32)
// by one Cooley-Tukey split: with n = R2 n1 + n2 and k = k1 + R1 k2,
//   X[k1 + R1 k2] = sum_n2 W_R2^{n2 k2} [ W_N^{n2 k1} sum_n1 x[R2 n1 + n2] W_R1^{n1 k1} ],
// so a thread computes an R1-point DFT in registers, applies the twiddle
// W_N^{n2 k1} (table formed in double on the host), exchanges through shared
// memory once, and computes an R2-point DFT in registers.  Five passes over the
// mesh, each one read and one write:
//   z forward (real density in) -> y forward -> x forward, times the Green's
//   function, x inverse (one kernel) -> y inverse -> z inverse (real Phi out).
// z is the contiguous axis: a CTA transforms whole rows.  For y and x a CTA
// holds an N x TC tile (TC consecutive z columns of one plane or row), so each
// of its global accesses is a contiguous run of TC complex values.
#include <math.h>

#include <mutex>

#include "mg_common.cuh"
#include "mg_internal.h"

namespace mg {

constexpr int kFftThreads = 256;

// exp(-2 pi i m / 32), m = 0..15: the twiddles of the register DFTs (R <= 32)
__constant__ float2 c_w32[16] = {
    {1.0f, 0.0f}, {0.980785251f, -0.195090324f}, {0.923879504f, -0.382683426f}, {0.831469595f, -0.555570245f},
    {0.707106769f, -0.707106769f}, {0.555570245f, -0.831469595f}, {0.382683426f, -0.923879504f},
    {0.195090324f, -0.980785251f}, {0.0f, -1.0f}, {-0.195090324f, -0.980785251f}, {-0.382683426f, -0.923879504f},
    {-0.555570245f, -0.831469595f}, {-0.707106769f, -0.707106769f}, {-0.831469595f, -0.555570245f},
    {-0.923879504f, -0.382683426f}, {-0.980785251f, -0.195090324f}};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__host__ __device__ constexpr int bitrev(int k, int R) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) {
    r = (r << 1) | (k & 1);
    k >>= 1;
  }
  return r;
}

// R-point DFT in registers (R a power of two <= 32): radix-2 decimation in
// frequency, natural input, bit-reversed output (X[k] in v[bitrev(k, R)]).
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
#pragma unroll
  for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int s = 0; s < R; s += 2 * span) {
#pragma unroll
      for (int j = 0; j < span; ++j) {
        const float2 a = v[s + j], b = v[s + j + span];
        v[s + j] = make_float2(a.x + b.x, a.y + b.y);
        float2 d = make_float2(a.x - b.x, a.y - b.y);
        if (j != 0) {  // W_{2 span}^j = W_32^{j 32 / (2 span)}
          float2 w = c_w32[j * (32 / (2 * span))];
          if (INV) w.y = -w.y;
          d = cmul(d, w);
        }
        v[s + j + span] = d;
      }
    }
  }
}

template <int R1, int R2>
__host__ __device__ constexpr int fft_threads_per_line() {
  return R1 > R2 ? R1 : R2;
}

// Resident CTAs per SM the register allocation is bounded for: four (64
// registers a thread) while a thread's DFT holds at most 16 complex values,
// two for the 32-point factors, whose 64 values would otherwise spill.
template <int R1, int R2>
__host__ __device__ constexpr int fft_min_ctas() {
  return (R1 > 16 || R2 > 16) ? 2 : 4;
}

// Phase 1 of a transform of length N = R1 R2 for the thread owning n2 (< R2):
// v holds x[R2 n1 + n2], n1 = 0..R1-1 (natural order); writes the twiddled
// R1-point DFT, W_N^{n2 k1} X1[k1], to ex(k1).
template <int R1, int R2, bool INV, class EX>
__device__ __forceinline__ void fft_phase1(float2 (&v)[R1], int n2, const float2* __restrict__ twN, EX ex) {
  dft_reg<R1, INV>(v);
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    float2 w = __ldg(&twN[n2 * k1]);
    if (INV) w.y = -w.y;
    ex(k1) = cmul(v[bitrev(k1, R1)], w);
  }
}

// Phase 3 for the thread owning k1 (< R1): u holds the twiddled values of all
// n2 (< R2); on return u[k2] = X[k1 + R1 k2] in natural order of k2.
template <int R2, bool INV>
__device__ __forceinline__ void fft_phase3(float2 (&u)[R2]) {
  dft_reg<R2, INV>(u);
  float2 t[R2];
#pragma unroll
  for (int k2 = 0; k2 < R2; ++k2) t[k2] = u[bitrev(k2, R2)];
#pragma unroll
  for (int k2 = 0; k2 < R2; ++k2) u[k2] = t[k2];
}

// Contiguous axis (z), L whole rows per CTA, T = max(R1, R2) threads per row:
// thread (l, r) loads x[R2 n1 + r] of its row straight into registers (runs of
// R2 consecutive values across the threads), exchanges once through shared
// memory (Y[n2][k1] at l R1 (R2+1) + k1 (R2+1) + n2: the padding keeps a
// half-warp's column reads on distinct banks) and stores X[r + R1 k2].
// MODE 1: forward, the real density in (times N^3 / sum rho, i.e. rho / mean);
// MODE 2: inverse, the real part out times 'scale'; MODE 0: complex in and out.
template <int R1, int R2, bool INV, int MODE>
__global__ void __launch_bounds__(kFftThreads, fft_min_ctas<R1, R2>()) k_fft_rows(const float* __restrict__ rin, float2* __restrict__ data,
                                                             float* __restrict__ rout, int L, float scale,
                                                             const double* __restrict__ rho_sum, long long n3,
                                                             const float2* __restrict__ twN) {
  constexpr int N = R1 * R2;
  constexpr int T = fft_threads_per_line<R1, R2>();
  extern __shared__ float2 fft_sm[];
  const int l = threadIdx.x / T, r = threadIdx.x - l * T;
  const long long lb = ((long long)blockIdx.x * L + l) * N;
  float2* Y = fft_sm + l * (R1 * (R2 + 1));
  float s = scale;
  if constexpr (MODE == 1) s = (float)((double)n3 / *rho_sum);
  if (r < R2) {
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      if constexpr (MODE == 1) v[n1] = make_float2(rin[lb + R2 * n1 + r] * s, 0.f);
      else v[n1] = data[lb + R2 * n1 + r];
    }
    fft_phase1<R1, R2, INV>(v, r, twN, [&](int k1) -> float2& { return Y[k1 * (R2 + 1) + r]; });
  }
  __syncthreads();
  if (r < R1) {
    float2 u[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) u[n2] = Y[r * (R2 + 1) + n2];
    fft_phase3<R2, INV>(u);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      if constexpr (MODE == 2) rout[lb + r + R1 * k2] = u[k2].x * s;
      else data[lb + r + R1 * k2] = u[k2];
    }
  }
}

// Strided axis: element m of column c at base + m * stride_axis + c with
// base = blockIdx.y * stride_other + z0, z0 = blockIdx.x * TC; thread (c, r) =
// (t % TC, t / TC), so a warp's global accesses are runs of TC consecutive
// values.  Exchange buffer Y[n2][k1] at (k1 R2 + n2) TC + c.
// GREEN (the x pass): the forward result X[k1 + R1 k2] stays in the registers
// of thread k1, is multiplied by -coef / K_h^2 (k_x = k1 + R1 k2, k_y =
// blockIdx.y, k_z = z0 + c) and transformed back with the two factors' roles
// swapped (input index R1 k2 + k1: phase 1 of length R2 over k2 by the thread
// owning k1, phase 3 of length R1), so the inverse starts from the registers;
// its output index is j1 + R2 j2.
template <int R1, int R2, bool INV, bool GREEN>
__global__ void __launch_bounds__(kFftThreads, fft_min_ctas<R1, R2>()) k_fft_cols(float2* __restrict__ data, int TC, long long stride_axis,
                                                             long long stride_other, const float2* __restrict__ twN,
                                                             const float* __restrict__ s2, float coef) {
  extern __shared__ float2 fft_sm[];
  const int c = threadIdx.x % TC, r = threadIdx.x / TC;
  const int z0 = blockIdx.x * TC;
  const int o = blockIdx.y;
  float2* col = data + (long long)o * stride_other + z0 + c;
  if (r < R2) {
    float2 v[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = col[(long long)(R2 * n1 + r) * stride_axis];
    fft_phase1<R1, R2, INV>(v, r, twN, [&](int k1) -> float2& { return fft_sm[(k1 * R2 + r) * TC + c]; });
  }
  __syncthreads();
  float2 u[R2];
  if (r < R1) {
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) u[n2] = fft_sm[(r * R2 + n2) * TC + c];
    fft_phase3<R2, INV>(u);
    if constexpr (!GREEN) {
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) col[(long long)(r + R1 * k2) * stride_axis] = u[k2];
    }
  }
  if constexpr (GREEN) {
    __syncthreads();  // every phase-3 read of the exchange buffer is done
    if (r < R1) {
      const float sc = s2[o] + s2[z0 + c];
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const float K2 = s2[r + R1 * k2] + sc;
        // fast division (a few ulp): far below the transforms' own rounding
        const float g = K2 > 0.f ? __fdividef(-coef, K2) : 0.f;
        u[k2] = make_float2(u[k2].x * g, u[k2].y * g);
      }
      // inverse, roles swapped: length-R2 DFTs over k2, twiddle W_N^{-r j1}
      fft_phase1<R2, R1, true>(u, r, twN, [&](int j1) -> float2& { return fft_sm[(j1 * R1 + r) * TC + c]; });
    }
    __syncthreads();
    if (r < R2) {
      float2 w[R1];
#pragma unroll
      for (int n2 = 0; n2 < R1; ++n2) w[n2] = fft_sm[(r * R1 + n2) * TC + c];
      fft_phase3<R1, true>(w);
#pragma unroll
      for (int j2 = 0; j2 < R1; ++j2) col[(long long)(r + R2 * j2) * stride_axis] = w[j2];
    }
  }
}

// Per-device, per-N plan: the complex work mesh, twiddles and K_h^2 terms.
struct FftPlan {
  int device = -1;
  int N = 0;
  float2* buf = nullptr;
  float2* tw = nullptr;
  float* s2 = nullptr;
  double* partials = nullptr;
  double* sum = nullptr;
};

constexpr int kMaxFftPlans = 8;
static std::mutex g_fft_mu;
static FftPlan* g_fft[kMaxFftPlans];
static int g_nfft = 0;

static int fft_plan(int N, FftPlan** out) {
  int dev = 0;
  MG_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_fft_mu);
  for (int i = 0; i < g_nfft; ++i)
    if (g_fft[i]->device == dev && g_fft[i]->N == N) {
      *out = g_fft[i];
      return MGGLAM_OK;
    }
  if (g_nfft == kMaxFftPlans) return MGGLAM_ERR_OOM;
  FftPlan* p = new FftPlan;
  p->device = dev;
  p->N = N;
  const size_t n3 = (size_t)N * N * N;
  bool ok = cudaMalloc(&p->buf, n3 * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&p->tw, (size_t)N * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&p->s2, (size_t)N * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&p->partials, kMaxReduceBlocks * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&p->sum, sizeof(double)) == cudaSuccess;
  if (ok) {
    float2* tw = new float2[N];
    float* s2 = new float[N];
    for (int m = 0; m < N; ++m) {
      const double ang = -2.0 * M_PI * (double)m / (double)N;
      tw[m] = make_float2((float)cos(ang), (float)sin(ang));
    }
    for (int k = 0; k < N; ++k) {
      const double s = sin(M_PI * (double)k / (double)N);
      s2[k] = (float)(4.0 * s * s);
    }
    ok = cudaMemcpy(p->tw, tw, (size_t)N * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(p->s2, s2, (size_t)N * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
    delete[] tw;
    delete[] s2;
  }
  if (!ok) {
    cudaGetLastError();
    cudaFree(p->buf);
    cudaFree(p->tw);
    cudaFree(p->s2);
    cudaFree(p->partials);
    cudaFree(p->sum);
    delete p;
    return MGGLAM_ERR_OOM;
  }
  g_fft[g_nfft++] = p;
  *out = p;
  return MGGLAM_OK;
}

void release_fft_plans() {
  std::lock_guard<std::mutex> lk(g_fft_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  int keep = 0;
  for (int i = 0; i < g_nfft; ++i) {
    FftPlan* p = g_fft[i];
    if (p->device == dev) {
      cudaFree(p->buf);
      cudaFree(p->tw);
      cudaFree(p->s2);
      cudaFree(p->partials);
      cudaFree(p->sum);
      delete p;
    } else {
      g_fft[keep++] = p;
    }
  }
  g_nfft = keep;
}

static bool pow2_mesh(int N) { return N >= 8 && N <= 1024 && (N & (N - 1)) == 0; }

// The five passes for N = R1 R2.  Rows kernel: L = 256/T rows per CTA (at most
// N^2); columns kernel: TC = 256/T z columns per tile (at most N).  Dynamic
// shared memory: the exchange buffer (about 33 KB at N = 256, 66 KB at 1024).
template <int R1, int R2>
static int poisson_passes(const float* rho, float* phi, double coef, const FftPlan* p, cudaStream_t st) {
  constexpr int N = R1 * R2;
  constexpr int T = fft_threads_per_line<R1, R2>();
  const long long NN = (long long)N * N, n3 = NN * N;
  const int L = (int)(kFftThreads / T < NN ? kFftThreads / T : NN);
  const int TC = kFftThreads / T < N ? kFftThreads / T : N;
  const size_t rows_smem = (size_t)L * R1 * (R2 + 1) * sizeof(float2);
  const size_t cols_smem = (size_t)N * TC * sizeof(float2);
  static bool attr_set[64] = {};  // per device: the opt-in above 48 KB, once
  if (p->device < 64 && !attr_set[p->device]) {
    MG_CUDA_TRY(cudaFuncSetAttribute(k_fft_rows<R1, R2, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)rows_smem));
    MG_CUDA_TRY(cudaFuncSetAttribute(k_fft_rows<R1, R2, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)rows_smem));
    MG_CUDA_TRY(cudaFuncSetAttribute(k_fft_cols<R1, R2, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cols_smem));
    MG_CUDA_TRY(cudaFuncSetAttribute(k_fft_cols<R1, R2, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cols_smem));
    MG_CUDA_TRY(cudaFuncSetAttribute(k_fft_cols<R1, R2, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cols_smem));
    attr_set[p->device] = true;
  }
  const unsigned rows_grid = (unsigned)(NN / L);
  const dim3 cols_grid(N / TC, N);
  prof_begin(PC_POISSON_FFT, st, 72.0 * n3);
  k_fft_rows<R1, R2, false, 1><<<rows_grid, L * T, rows_smem, st>>>(rho, p->buf, nullptr, L, 1.f, p->sum, n3, p->tw);
  k_fft_cols<R1, R2, false, false><<<cols_grid, TC * T, cols_smem, st>>>(p->buf, TC, N, NN, p->tw, p->s2, 0.f);
  k_fft_cols<R1, R2, false, true><<<cols_grid, TC * T, cols_smem, st>>>(p->buf, TC, NN, N, p->tw, p->s2, (float)coef);
  k_fft_cols<R1, R2, true, false><<<cols_grid, TC * T, cols_smem, st>>>(p->buf, TC, N, NN, p->tw, p->s2, 0.f);
  k_fft_rows<R1, R2, true, 2><<<rows_grid, L * T, rows_smem, st>>>(nullptr, p->buf, phi, L, (float)(1.0 / (double)n3),
                                                                    nullptr, n3, p->tw);
  prof_end(st);
  note_launch(5);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

int poisson_fft(const float* rho, int N, double coef, float* phi, cudaStream_t st) {
  if (!pow2_mesh(N)) return MGGLAM_ERR_SHAPE;
  FftPlan* p = nullptr;
  int rc = fft_plan(N, &p);
  if (rc) return rc;
  if ((rc = launch_density_mean(rho, (size_t)N * N * N, p->partials, p->sum, st))) return rc;
  switch (N) {
    case 8: return poisson_passes<4, 2>(rho, phi, coef, p, st);
    case 16: return poisson_passes<4, 4>(rho, phi, coef, p, st);
    case 32: return poisson_passes<8, 4>(rho, phi, coef, p, st);
    case 64: return poisson_passes<8, 8>(rho, phi, coef, p, st);
    case 128: return poisson_passes<16, 8>(rho, phi, coef, p, st);
    case 256: return poisson_passes<16, 16>(rho, phi, coef, p, st);
    case 512: return poisson_passes<32, 16>(rho, phi, coef, p, st);
    default: return poisson_passes<32, 32>(rho, phi, coef, p, st);
  }
}

}  // namespace mg
