// cic.cuh -- cloud-in-cell interpolation shared by the force gather and the
// particle push (Sec. 3.1: CIC assignment and interpolation, three-point
// finite differences at cell centres, periodic mesh, centre of cell c at c + 1/2).
#pragma once
#include <cuda_runtime.h>

namespace mg {

// Position wrapped into [0, N).
__device__ __forceinline__ float wrap_pos(float x, int N) {
  if (x >= 0.f && x < (float)N) return x;
  float xf = fmodf(x, (float)N);
  if (xf < 0.f) xf += (float)N;
  if (xf >= (float)N) xf = 0.f;
  return xf;
}

// Single-precision CIC along one axis (for the gather, whose output is FP32).
__device__ __forceinline__ void cic_axis_f(float x, int N, int& c0, int& c1, float& w0, float& w1) {
  const float xs = wrap_pos(x, N) - 0.5f;
  const float fl = floorf(xs);
  const float f = xs - fl;
  const int c = (int)fl;
  c0 = c < 0 ? c + N : c;
  c1 = c + 1 >= N ? c + 1 - N : c + 1;
  w0 = 1.f - f;
  w1 = f;
}

// The CIC-weighted central differences of a mesh scalar around one particle:
// Tv(a, b, c) returns T at the cell with per-axis positions a, b, c in 0..3,
// meaning (c0 - 1, c0, c1, c1 + 1) of that axis.  Shared by the gather from
// global memory and the gather from a tile staged in shared memory, so that
// both form the same sums in the same order.
template <class Tv>
__device__ __forceinline__ float3 cic_grad_core(const Tv& Tat, const float wx[2], const float wy[2],
                                                const float wz[2]) {
  float C[2][2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 2; ++c) C[a][b][c] = Tat(a + 1, b + 1, c + 1);
  float fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float xm = Tat(0, b + 1, c + 1), xp = Tat(3, b + 1, c + 1);
      const float w = wy[b] * wz[c];
      fx += w * (wx[0] * (C[1][b][c] - xm) + wx[1] * (xp - C[0][b][c]));
    }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float ym = Tat(a + 1, 0, c + 1), yp = Tat(a + 1, 3, c + 1);
      const float w = wx[a] * wz[c];
      fy += w * (wy[0] * (C[a][1][c] - ym) + wy[1] * (yp - C[a][0][c]));
    }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float zm = Tat(a + 1, b + 1, 0), zp = Tat(a + 1, b + 1, 3);
      const float w = wx[a] * wy[b];
      fz += w * (wz[0] * (C[a][b][1] - zm) + wz[1] * (zp - C[a][b][0]));
    }
  return make_float3(0.5f * fx, 0.5f * fy, 0.5f * fz);
}

// Gradient of the mesh scalar T at (x, y, z): the central differences
// (T_{c+1} - T_{c-1})/2 at the 8 CIC cells, weighted with the particle's CIC
// weights.  Reads the 32 distinct cells those differences touch: the 2x2x2
// core and a one-cell extension on each side along each axis.  IT: the index
// type of the cell offsets (int where N^3 < 2^31).
template <typename IT = long long>
__device__ __forceinline__ float3 cic_grad(const float* __restrict__ T, int N, float x, float y, float z) {
  int i0, i1, j0, j1, k0, k1;
  float wx[2], wy[2], wz[2];
  cic_axis_f(x, N, i0, i1, wx[0], wx[1]);
  cic_axis_f(y, N, j0, j1, wy[0], wy[1]);
  cic_axis_f(z, N, k0, k1, wz[0], wz[1]);
  const IT NN = (IT)N * N;
  // offsets: x[0..3] = i0-1, i0, i1, i1+1 (times N^2), likewise y (times N) and z
  const IT ox[4] = {(IT)(i0 == 0 ? N - 1 : i0 - 1) * NN, (IT)i0 * NN, (IT)i1 * NN,
                    (IT)(i1 + 1 == N ? 0 : i1 + 1) * NN};
  const IT oy[4] = {(IT)(j0 == 0 ? N - 1 : j0 - 1) * N, (IT)j0 * N, (IT)j1 * N, (IT)(j1 + 1 == N ? 0 : j1 + 1) * N};
  const int oz[4] = {k0 == 0 ? N - 1 : k0 - 1, k0, k1, k1 + 1 == N ? 0 : k1 + 1};
  auto Tat = [&](int a, int b, int c) { return T[ox[a] + oy[b] + oz[c]]; };
  return cic_grad_core(Tat, wx, wy, wz);
}

}  // namespace mg
