// FP32 step of a CTA-resident chain (n <= 81): the CTA's propagator
// D = P - I and its nb states live in shared memory as interleaved complex
// FP32 (row-major, a state is a row of n values), and one step is
//   Y[q][i] = X[q][i] + sum_j D[i][j] X[q][j].
// Work unit = (row i, group of RS states): a thread keeps 2 RS independent
// accumulators (the dot products of row i with RS states), reads D[i][j] once
// per j for all of them and the states' X[q][j] as warp broadcasts, so the
// loop issues RS + 1 8-byte shared loads per 4 RS FMAs and no FMA waits on
// the one before it.
#pragma once

#include <cuda_runtime.h>

namespace lb {

// With C given, the outputs of state q are multiplied by C[q] = 1 / Tr X[q]
// (the renormalisation of the previous step, applied one step late: the same
// states up to rounding; res32_traces writes C after the step's barrier).
// After the last step the states still need one division by their trace
// (res32_renorm).
template <int RS>
__device__ __forceinline__ void res32_step(int n, int nb, const float2* __restrict__ D,
                                           const float2* __restrict__ X, float2* __restrict__ Y, int tid,
                                           int nthreads, const float2* __restrict__ C = nullptr) {
  const int G = (nb + RS - 1) / RS;
  for (int u = tid; u < n * G; u += nthreads) {
    const int i = u % n, g = u / n, q0 = g * RS;
    const int qn = min(RS, nb - q0);
    float2 cs[RS];
#pragma unroll
    for (int r = 0; r < RS; r++) cs[r] = (C != nullptr && r < qn) ? C[q0 + r] : make_float2(1.f, 0.f);
    float ar[RS], ai[RS];
#pragma unroll
    for (int r = 0; r < RS; r++) ar[r] = ai[r] = 0.f;
    const float2* drow = D + i * n;
    const float2* xq = X + q0 * n;
#pragma unroll 9  // measured at n = 81: 10 % faster than 3; 27 is slower
    for (int j = 0; j < n; j++) {
      const float2 a = drow[j];
#pragma unroll
      for (int r = 0; r < RS; r++) {
        const float2 x = xq[(r < qn ? r : 0) * n + j];  // a valid state; unused results for r >= qn
        ar[r] = fmaf(a.x, x.x, ar[r]);
        ar[r] = fmaf(-a.y, x.y, ar[r]);
        ai[r] = fmaf(a.x, x.y, ai[r]);
        ai[r] = fmaf(a.y, x.x, ai[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < RS; r++) {
      if (r < qn) {
        const int e = (q0 + r) * n + i;
        const float2 x = X[e];
        const float vr = x.x + ar[r], vi = x.y + ai[r];
        Y[e] = make_float2(vr * cs[r].x - vi * cs[r].y, vr * cs[r].y + vi * cs[r].x);
      }
    }
  }
}

// C[q] = 1 / Tr(Y[q]) for the nb states (no barrier inside).
__device__ __forceinline__ void res32_traces(int n, int d, int nb, const float2* __restrict__ Y,
                                             float2* __restrict__ C, int tid, int nthreads) {
  for (int q = tid; q < nb; q += nthreads) {
    float sr = 0.f, si = 0.f;
    for (int k = 0; k < d; k++) {
      const float2 v = Y[q * n + k * (d + 1)];
      sr += v.x;
      si += v.y;
    }
    const float m2 = sr * sr + si * si;
    C[q] = make_float2(sr / m2, -si / m2);
  }
}

// Y[q] /= Tr(Y[q]) for the nb states (Tr = sum of the d diagonal entries of
// the d x d matrix), C (nb complex) as scratch; two CTA barriers.
__device__ __forceinline__ void res32_renorm(int n, int d, int nb, float2* __restrict__ Y, float2* __restrict__ C,
                                             int tid, int nthreads) {
  for (int q = tid; q < nb; q += nthreads) {
    float sr = 0.f, si = 0.f;
    for (int k = 0; k < d; k++) {
      const float2 v = Y[q * n + k * (d + 1)];
      sr += v.x;
      si += v.y;
    }
    const float m2 = sr * sr + si * si;
    C[q] = make_float2(sr / m2, -si / m2);
  }
  __syncthreads();
  for (int e = tid; e < nb * n; e += nthreads) {
    const float2 c = C[e / n], v = Y[e];
    Y[e] = make_float2(v.x * c.x - v.y * c.y, v.x * c.y + v.y * c.x);
  }
}

}  // namespace lb
