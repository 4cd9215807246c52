// mg_common.cuh -- shared device helpers: indexing, deterministic block
// reductions, launch geometry.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mg_model.cuh"

namespace mg {

constexpr int kThreads = 256;
constexpr int kMaxReduceBlocks = 8192;  // size of the partial-sum array
// Grid cap of the grid-stride elementwise kernels: about two waves of
// 256-thread blocks on 152 SMs, so that per-thread setup (a division, a
// scalar read) is paid once per ~30 cells, not once per cell.
constexpr int kStreamBlocks = 2432;

__host__ __device__ __forceinline__ size_t cidx(int n, int i, int j, int k) {
  return ((size_t)i * n + j) * n + k;
}

// Block-wide sum of one double per thread; result valid in thread 0.  Fixed
// shuffle/tree order, so the result is deterministic for a fixed launch shape.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Positivity-guard replacements (reading C11): each thread adds its own count to
// the solve's counter (a 64-bit integer in the workspace scalars); the guard is
// rare, so the atomic is almost never issued.  guard may be null (not counted).
__device__ __forceinline__ void count_guards(unsigned long long* guard, unsigned c) {
  if (c && guard) atomicAdd(guard, (unsigned long long)c);
}

// Grid for a grid-stride loop over 'work' items, capped so that partial sums fit.
inline int grid_for(long long work, int threads = kThreads, int cap = kMaxReduceBlocks) {
  long long g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// Grid for a grid-stride elementwise kernel.
inline int stream_grid(long long work) { return grid_for(work, kThreads, kStreamBlocks); }

// Error-free accumulation of single-precision values (Knuth's two-sum): after
// any number of steps hi + lo equals the exact sum up to the rounding of lo,
// i.e. to ~2^-46 relative, without double-precision arithmetic.
struct FloatFloat {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace mg
