// fft.cu -- the PM gravity solver: the periodic Poisson equation by FFT
// (Sec. 3.1: FFTs along x, y and z, multiplication by the Green's function of
// the discrete Laplacian, inverse FFTs; Eq. GR_poisson_codeunit).
//
//   grad_h^2 Phi = coef (rho/mean - 1),   Phi_k = -coef delta_k / K_h^2,
//   K_h^2 = sum_d 4 sin^2(pi k_d / N)   (the 7-point Laplacian's eigenvalues),
//   Phi_0 = 0 (the mean of Phi is not fixed by the equation).
//
// Single-precision complex FFTs of power-of-two length, radix-2 Stockham
// (self-sorting) stages in shared memory; twiddles formed in double on the host.
// Five passes over the mesh, each one read and one write:
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
constexpr int kFftRowElems = 2048;   // complex values per buffer, contiguous-axis kernel (2 x 16 KB)
constexpr int kFftTileElems = 4096;  // complex values per buffer, strided-axis kernel (2 x 32 KB)

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// log2(N) radix-2 Stockham stages on L lines of length N in shared memory,
// ping-ponging between a and b; returns the buffer holding the transform
// (natural order).  LINE_MAJOR: element m of line l at l N + m, else at m L + l
// (threads are mapped so that consecutive threads touch consecutive words).
// Stage with span Ns: for j < N/2, k = j mod Ns,
//   x0 = in[j], x1 = in[j + N/2] w^k  (w = exp(-+2 pi i / (2 Ns)))
//   out[2(j - k) + k] = x0 + x1,  out[2(j - k) + k + Ns] = x0 - x1.
template <bool INV, bool LINE_MAJOR>
__device__ __forceinline__ float2* stockham(float2* a, float2* b, int N, int L, const float2* __restrict__ tw) {
  const int half = N >> 1;
  for (int Ns = 1; Ns < N; Ns <<= 1) {
    const int step = N / (2 * Ns);
    for (int t = threadIdx.x; t < L * half; t += blockDim.x) {
      const int l = LINE_MAJOR ? t / half : t % L;
      const int j = LINE_MAJOR ? t - l * half : t / L;
      const int k = j & (Ns - 1);
      float2 w = __ldg(&tw[k * step]);
      if (INV) w.y = -w.y;
      const int o = ((j - k) << 1) + k;
      const float2 x0 = LINE_MAJOR ? a[l * N + j] : a[j * L + l];
      const float2 x1 = cmul(LINE_MAJOR ? a[l * N + j + half] : a[(j + half) * L + l], w);
      const float2 s = make_float2(x0.x + x1.x, x0.y + x1.y), d = make_float2(x0.x - x1.x, x0.y - x1.y);
      if (LINE_MAJOR) {
        b[l * N + o] = s;
        b[l * N + o + Ns] = d;
      } else {
        b[o * L + l] = s;
        b[(o + Ns) * L + l] = d;
      }
    }
    __syncthreads();
    float2* tmp = a;
    a = b;
    b = tmp;
  }
  return a;
}

// Contiguous axis (z), L whole rows per CTA.  MODE 1: forward, the real density
// in (times N^3 / sum rho, i.e. rho / mean); MODE 2: inverse, the real part out
// times 'scale'; MODE 0: complex in and out.
template <bool INV, int MODE>
__global__ void __launch_bounds__(kFftThreads) k_fft_rows(const float* __restrict__ rin, float2* __restrict__ data,
                                                          float* __restrict__ rout, int N, int L, float scale,
                                                          const double* __restrict__ rho_sum, long long n3,
                                                          const float2* __restrict__ tw) {
  extern __shared__ float2 fft_sm[];
  float2* A = fft_sm;
  float2* B = fft_sm + L * N;
  const long long base = (long long)blockIdx.x * L * N;
  float s = scale;
  if constexpr (MODE == 1) s = (float)((double)n3 / *rho_sum);
  for (int e = threadIdx.x; e < L * N; e += blockDim.x) {
    if constexpr (MODE == 1) A[e] = make_float2(rin[base + e] * s, 0.f);
    else A[e] = data[base + e];
  }
  __syncthreads();
  const float2* r = stockham<INV, true>(A, B, N, L, tw);
  for (int e = threadIdx.x; e < L * N; e += blockDim.x) {
    if constexpr (MODE == 2) rout[base + e] = r[e].x * s;
    else data[base + e] = r[e];
  }
}

// Strided axis: element m of column t at base + m * stride_axis + t, with
// base = blockIdx.y * stride_other + z0, z0 = blockIdx.x * TC.  GREEN: forward
// transform, multiplication by -coef / K_h^2 (k_axis = m, k_other = blockIdx.y,
// k_z = z0 + t; the x pass), inverse transform.
template <bool INV, bool GREEN>
__global__ void __launch_bounds__(kFftThreads) k_fft_cols(float2* __restrict__ data, int N, int TC,
                                                          long long stride_axis, long long stride_other,
                                                          const float2* __restrict__ tw, const float* __restrict__ s2,
                                                          float coef) {
  extern __shared__ float2 fft_sm[];
  float2* A = fft_sm;
  float2* B = fft_sm + N * TC;
  const int z0 = blockIdx.x * TC;
  const int o = blockIdx.y;
  const long long base = (long long)o * stride_other + z0;
  for (int e = threadIdx.x; e < N * TC; e += blockDim.x) {
    const int m = e / TC, t = e - m * TC;
    A[e] = data[base + (long long)m * stride_axis + t];
  }
  __syncthreads();
  float2* r = stockham<INV, false>(A, B, N, TC, tw);
  if constexpr (GREEN) {
    const float so = s2[o];
    for (int e = threadIdx.x; e < N * TC; e += blockDim.x) {
      const int m = e / TC, t = e - m * TC;
      const float K2 = s2[m] + so + s2[z0 + t];
      const float g = K2 > 0.f ? -coef / K2 : 0.f;
      r[e] = make_float2(r[e].x * g, r[e].y * g);
    }
    __syncthreads();
    float2* other = r == A ? B : A;
    r = stockham<true, false>(r, other, N, TC, tw);
  }
  for (int e = threadIdx.x; e < N * TC; e += blockDim.x) {
    const int m = e / TC, t = e - m * TC;
    data[base + (long long)m * stride_axis + t] = r[e];
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
            cudaMalloc(&p->tw, (size_t)(N / 2) * sizeof(float2)) == cudaSuccess &&
            cudaMalloc(&p->s2, (size_t)N * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&p->partials, kMaxReduceBlocks * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&p->sum, sizeof(double)) == cudaSuccess;
  // the shared-memory opt-in of the strided kernels (2 x 32 KB)
  const int bytes = 2 * kFftTileElems * (int)sizeof(float2);
  ok = ok && cudaFuncSetAttribute(k_fft_cols<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
                 cudaSuccess &&
       cudaFuncSetAttribute(k_fft_cols<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess &&
       cudaFuncSetAttribute(k_fft_cols<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
  if (ok) {
    float2* tw = new float2[N / 2];
    float* s2 = new float[N];
    for (int m = 0; m < N / 2; ++m) {
      const double ang = -2.0 * M_PI * (double)m / (double)N;
      tw[m] = make_float2((float)cos(ang), (float)sin(ang));
    }
    for (int k = 0; k < N; ++k) {
      const double s = sin(M_PI * (double)k / (double)N);
      s2[k] = (float)(4.0 * s * s);
    }
    ok = cudaMemcpy(p->tw, tw, (size_t)(N / 2) * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
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

int poisson_fft(const float* rho, int N, double coef, float* phi, cudaStream_t st) {
  if (!pow2_mesh(N)) return MGGLAM_ERR_SHAPE;
  FftPlan* p = nullptr;
  int rc = fft_plan(N, &p);
  if (rc) return rc;
  const long long n3 = (long long)N * N * N;
  if ((rc = launch_density_mean(rho, (size_t)n3, p->partials, p->sum, st))) return rc;
  const long long NN = (long long)N * N;
  const int L = kFftRowElems / N < NN ? kFftRowElems / N : (int)NN;  // rows per CTA (N <= 1024: >= 2)
  const int TC = kFftTileElems / N < N ? kFftTileElems / N : N;       // z columns per tile (>= 4)
  const unsigned rows_grid = (unsigned)(NN / L);
  const size_t rows_smem = 2 * (size_t)L * N * sizeof(float2);
  const size_t cols_smem = 2 * (size_t)N * TC * sizeof(float2);
  const dim3 cols_grid(N / TC, N);
  prof_begin(PC_POISSON_FFT, st, 72.0 * n3);
  k_fft_rows<false, 1><<<rows_grid, kFftThreads, rows_smem, st>>>(rho, p->buf, nullptr, N, L, 1.f, p->sum, n3, p->tw);
  k_fft_cols<false, false><<<cols_grid, kFftThreads, cols_smem, st>>>(p->buf, N, TC, N, NN, p->tw, p->s2, 0.f);
  k_fft_cols<false, true><<<cols_grid, kFftThreads, cols_smem, st>>>(p->buf, N, TC, NN, N, p->tw, p->s2, (float)coef);
  k_fft_cols<true, false><<<cols_grid, kFftThreads, cols_smem, st>>>(p->buf, N, TC, N, NN, p->tw, p->s2, 0.f);
  k_fft_rows<true, 2><<<rows_grid, kFftThreads, rows_smem, st>>>(nullptr, p->buf, phi, N, L, (float)(1.0 / (double)n3),
                                                                 nullptr, n3, p->tw);
  prof_end(st);
  note_launch(5);
  MG_CUDA_TRY(cudaGetLastError());
  return MGGLAM_OK;
}

}  // namespace mg
