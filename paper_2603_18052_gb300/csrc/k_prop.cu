// Propagation kernels: chained steps rho <- P rho (Algorithm 2), batched over
// states that share P (Algorithm 3's batch), for the sizes where P fits in
// shared memory (n <= 81, i.e. d <= 9).  The whole chain runs inside one
// launch: states are independent, so each CTA owns a slice of the batch,
// keeps P and its states on chip for every step and synchronises only
// within the CTA.  Larger n (d = 27) goes through the grouped GEMM, one
// launch per step.
//
// FP64 form: Gauss three-real-product complex multiply-add, P held as the
// planes (re, im, re + im).
// FP32 form: D = P - I held in FP32 planes, states in FP32, each step
// rho <- rho + D rho with FP32 accumulation (the identity part is applied
// exactly, so the rounding of the stored propagator scales with |D| rather
// than with |P| ~ 1), optional per-step division by the trace.
#include "lb_internal.cuh"
#include "res32.cuh"

#include <algorithm>

namespace lb {

namespace {

constexpr int kResThreads = 256;

size_t resident_f64_smem(int n, int chunk) {
  return sizeof(double) * (3ull * n * n + 5ull * chunk * n);
}
size_t resident_f32_smem(int n, int chunk) {
  return sizeof(float) * (2ull * n * n + 4ull * chunk * n) + sizeof(float) * 2 * chunk;
}

// adjoint: apply P^+ (load conj(P[j][i]) as row i) with the slices in reverse
// order.  hist (optional): the states before the first step and after every
// step, indexed t = 0..T forward or T - k after k adjoint steps.
// Several independent problems (blockIdx.y = problem k): its propagators at
// P + k p_stride, states at states + k x_stride, history at hist + k h_stride.
// hcompact: the history keeps only what the gradient reads, T entries per
// problem: forward X_0 .. X_{T-1} at t, adjoint Lam_1 .. Lam_T at t - 1.
__global__ void __launch_bounds__(kResThreads)
    prop_resident_f64_kernel(int n, int nslices, const z64* __restrict__ P, int steps_per_slice, int B,
                             int chunk, z64* __restrict__ states, int adjoint, z64* __restrict__ hist,
                             long long p_stride, long long x_stride, long long h_stride, int hcompact) {
  extern __shared__ __align__(16) double sm[];
  double* Pr = sm;
  double* Pi = Pr + n * n;
  double* Ps = Pi + n * n;
  double* xr = Ps + n * n;      // chunk x n
  double* xi = xr + chunk * n;
  double* xs = xi + chunk * n;
  double* yr = xs + chunk * n;
  double* yi = yr + chunk * n;
  const int b0 = blockIdx.x * chunk;
  if (b0 >= B) return;
  P += blockIdx.y * p_stride;
  states += blockIdx.y * x_stride;
  if (hist != nullptr) hist += blockIdx.y * h_stride;
  const int nb = min(chunk, B - b0);
  const int tid = threadIdx.x;
  const long long nn = (long long)n * n;
  for (int e = tid; e < nb * n; e += blockDim.x) {
    const z64 v = states[(long long)b0 * n + e];
    xr[e] = v.x;
    xi[e] = v.y;
    xs[e] = v.x + v.y;
  }
  const int work = nb * n;
  const long long T = (long long)nslices * steps_per_slice;
  long long hidx = adjoint ? T : 0;
  // where the state after hidx steps goes in the history (-1: not kept)
  auto hpos = [&](long long h) -> long long {
    if (!hcompact) return h;
    if (adjoint) return h >= 1 ? h - 1 : -1;
    return h <= T - 1 ? h : -1;
  };
  if (hist != nullptr && hpos(hidx) >= 0)
    for (int e = tid; e < work; e += blockDim.x)
      hist[(hpos(hidx) * B + b0) * n + e] = states[(long long)b0 * n + e];
  for (int si = 0; si < nslices; si++) {
    const int s = adjoint ? nslices - 1 - si : si;
    __syncthreads();
    for (int e = tid; e < n * n; e += blockDim.x) {
      z64 v;
      if (adjoint) {
        const int i = e / n, j = e - (e / n) * n;
        v = P[s * nn + (long long)j * n + i];
        v.y = -v.y;
      } else {
        v = P[s * nn + e];
      }
      Pr[e] = v.x;
      Pi[e] = v.y;
      Ps[e] = v.x + v.y;
    }
    __syncthreads();
    for (int t = 0; t < steps_per_slice; t++) {
      for (int e = tid; e < work; e += blockDim.x) {
        const int q = e / n, i = e - (e / n) * n;
        const double* pr = Pr + i * n;
        const double* pi = Pi + i * n;
        const double* ps = Ps + i * n;
        const double* ar = xr + q * n;
        const double* ai = xi + q * n;
        const double* as = xs + q * n;
        double a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll 3
        for (int j = 0; j < n; j++) {
          a1 = fma(pr[j], ar[j], a1);
          a2 = fma(pi[j], ai[j], a2);
          a3 = fma(ps[j], as[j], a3);
        }
        yr[e] = a1 - a2;
        yi[e] = a3 - a1 - a2;
      }
      __syncthreads();
      hidx += adjoint ? -1 : 1;
      for (int e = tid; e < work; e += blockDim.x) {
        const double r = yr[e], im = yi[e];
        xr[e] = r;
        xi[e] = im;
        xs[e] = r + im;
        if (hist != nullptr && hpos(hidx) >= 0) hist[(hpos(hidx) * B + b0) * n + e] = make_double2(r, im);
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < nb * n; e += blockDim.x) states[(long long)b0 * n + e] = make_double2(xr[e], xi[e]);
}

// Latency form for tiny n (n <= 16, d <= 4): one warp per state, no shared
// memory and no block barrier in the step loop.  K = 32 / n lanes share a
// row of P, each holding C = ceil(n / K) of its entries in registers (three
// planes for the Gauss form); a step is C chained FMAs, a K-lane shuffle sum
// and a shuffle broadcast of the new state to the lanes that need it.
template <int MAXC>
__global__ void __launch_bounds__(128)
    prop_warp_f64_kernel(int n, int nslices, const z64* __restrict__ P, int steps_per_slice, int B,
                         z64* __restrict__ states) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= B) return;  // whole warps leave together
  const int K = 32 / n, C = (n + K - 1) / K;
  const int r = lane / K, part = lane - (lane / K) * K;
  const bool rowok = r < n;
  const int j0 = part * C;
  z64* x = states + (long long)w * n;
  const long long nn = (long long)n * n;
  double xr[MAXC], xi[MAXC], xs[MAXC], pr[MAXC], pi[MAXC], ps[MAXC];
#pragma unroll
  for (int c = 0; c < MAXC; c++) {
    const int j = j0 + c;
    z64 v = make_double2(0.0, 0.0);
    if (c < C && j < n) v = x[j];
    xr[c] = v.x;
    xi[c] = v.y;
    xs[c] = v.x + v.y;
  }
  double re = 0.0, im = 0.0;
  for (int s = 0; s < nslices; s++) {
#pragma unroll
    for (int c = 0; c < MAXC; c++) {
      const int j = j0 + c;
      z64 v = make_double2(0.0, 0.0);
      if (rowok && c < C && j < n) v = P[s * nn + (long long)r * n + j];
      pr[c] = v.x;
      pi[c] = v.y;
      ps[c] = v.x + v.y;
    }
    for (int t = 0; t < steps_per_slice; t++) {
      double a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
      for (int c = 0; c < MAXC; c++) {
        if (c < C) {
          a1 = fma(pr[c], xr[c], a1);
          a2 = fma(pi[c], xi[c], a2);
          a3 = fma(ps[c], xs[c], a3);
        }
      }
      double vr = a1 - a2, vi = a3 - a1 - a2;
      // sum of the K parts of the row, at the row's first lane
      re = vr;
      im = vi;
      for (int q = 1; q < K; q++) {
        re += __shfl_down_sync(FULL, vr, q);
        im += __shfl_down_sync(FULL, vi, q);
      }
      // every lane fetches the new entries of its columns from their rows' first lanes
#pragma unroll
      for (int c = 0; c < MAXC; c++) {
        if (c < C) {
          const int j = j0 + c;
          const int src = (j < n ? j : 0) * K;
          const double nr = __shfl_sync(FULL, re, src), ni = __shfl_sync(FULL, im, src);
          xr[c] = (j < n) ? nr : 0.0;
          xi[c] = (j < n) ? ni : 0.0;
          xs[c] = xr[c] + xi[c];
        }
      }
    }
  }
  if (rowok && part == 0 && (long long)nslices * steps_per_slice > 0) x[r] = make_double2(re, im);
}

// Latency form for one state per CTA (n <= 16, few states).  FP64 runs at
// 1/64 of the FP32 rate here: a warp-wide FP64 instruction occupies its SM
// sub-partition for 64 cycles however many lanes are active, so the step time
// is the number of FP64 instructions a warp issues.  The 2n real outputs
// (Re and Im of each row) each sum 2n real products; an output is split over
// K lanes of one warp with C products each (C FMAs), the K partial sums meet
// in a log2(K)-level shuffle tree, and the outputs are spread over four warps
// (one per sub-partition).  The new state goes through shared memory (double
// buffered, one barrier per step).  n = 9: C = 3, K = 6, six FP64
// instructions per warp per step instead of about twenty for one warp.
template <int CMAX>
__global__ void __launch_bounds__(128)
    prop_lat_f64_kernel(int n, int C, int K, int nslices, const z64* __restrict__ P, int steps_per_slice,
                        z64* __restrict__ states) {
  __shared__ double X[2][32];  // [xr(0..n-1), xi(0..n-1)], double buffered
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n2 = 2 * n;
  const int gpw = 32 / K;                 // output groups per warp
  const int g = lane / K, part = lane - g * K;
  const int o = g * 4 + warp;             // this lane's output (round robin over the warps)
  const bool active = g < gpw && o < n2;
  z64* x = states + (long long)blockIdx.x * n;
  if (tid < n) {
    const z64 v = x[tid];
    X[0][tid] = v.x;
    X[0][n + tid] = v.y;
  }
  // coefficient and state index of each of this lane's C terms
  const int i = o < n ? o : o - n;
  int xidx[CMAX];
  double cf[CMAX];
  const long long nn = (long long)n * n;
  int cur = 0;
  __syncthreads();
  for (int s = 0; s < nslices; s++) {
#pragma unroll
    for (int k = 0; k < CMAX; k++) {
      const int t = part * C + k;
      double c = 0.0;
      int xi_ = 0;
      if (active && k < C && t < n2) {
        const int j = t < n ? t : t - n;
        const z64 pv = P[s * nn + (long long)i * n + j];
        if (o < n) {  // Re_i = sum_j pr xr - pi xi
          c = t < n ? pv.x : -pv.y;
          xi_ = t;
        } else {      // Im_i = sum_j pr xi + pi xr
          c = t < n ? pv.x : pv.y;
          xi_ = t < n ? n + t : t - n;
        }
      }
      cf[k] = c;
      xidx[k] = xi_;
    }
    for (int st = 0; st < steps_per_slice; st++) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < CMAX; k++)
        if (k < C) acc = fma(cf[k], X[cur][xidx[k]], acc);
      // segmented tree over the K lanes of the group; the first lane ends with the sum
      if (K == 6) {
        // after the pairwise level the first lane needs the pair sums of
        // lanes 2 and 4: both are fetched at once, and the additions are the
        // tree's, ((a0 + a1) + (a2 + a3)) + (a4 + a5)
        const double v = __shfl_down_sync(0xffffffffu, acc, 1);
        if (part + 1 < K) acc += v;
        const double v2 = __shfl_down_sync(0xffffffffu, acc, 2);
        const double v4 = __shfl_down_sync(0xffffffffu, acc, 4);
        if (part == 0) acc = (acc + v2) + v4;
      } else {
        for (int off = 1; off < K; off <<= 1) {
          const double v = __shfl_down_sync(0xffffffffu, acc, off);
          if (part + off < K) acc += v;
        }
      }
      if (active && part == 0) X[cur ^ 1][o] = acc;
      __syncthreads();
      cur ^= 1;
    }
  }
  if (tid < n && (long long)nslices * steps_per_slice > 0) x[tid] = make_double2(X[cur][tid], X[cur][n + tid]);
}

// Split of 2n products per output for the latency form: C products per lane,
// K = ceil(2n / C) lanes per output, at most four warps of 32 lanes; the
// choice minimises C + ceil(log2 K) (FP64 instructions per step).
bool lat_split(int n, int* C, int* K) {
  int best = 1 << 30;
  for (int c = 1; c <= 8; c++) {
    const int k = (2 * n + c - 1) / c;
    if (k > 32 || 2 * n > 4 * (32 / k)) continue;
    int lg = 0;
    while ((1 << lg) < k) lg++;
    if (c + lg < best) {
      best = c + lg;
      *C = c;
      *K = k;
    }
  }
  return best < (1 << 30);
}

// FP32 resident chain (n <= 81): D = P - I and the CTA's states in shared
// memory for the whole chain, one register-blocked step per barrier
// (res32.cuh), optional trace renormalisation after every step.
__global__ void __launch_bounds__(1024)
    prop_resident_f32_kernel(int n, int d, int nslices, const float* __restrict__ Dr,
                             const float* __restrict__ Di, int steps_per_slice, int B, int chunk,
                             int renorm, z64* __restrict__ states) {
  extern __shared__ __align__(16) float2 sm2[];
  float2* D = sm2;
  float2* X = D + n * n;
  float2* Y = X + chunk * n;
  float2* C = Y + chunk * n;
  const int b0 = blockIdx.x * chunk;
  if (b0 >= B) return;
  const int nb = min(chunk, B - b0);
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long nn = (long long)n * n;
  for (int e = tid; e < nb * n; e += nt) {
    const z64 v = states[(long long)b0 * n + e];
    X[e] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  if (renorm) res32_traces(n, d, nb, X, C, tid, nt);
  for (int s = 0; s < nslices; s++) {
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) D[e] = make_float2(Dr[s * nn + e], Di[s * nn + e]);
    __syncthreads();
    for (int t = 0; t < steps_per_slice; t++) {
      res32_step<2>(n, nb, D, X, Y, tid, nt, renorm ? C : nullptr);  // trace factor of X applied to Y
      __syncthreads();
      if (renorm) {
        res32_traces(n, d, nb, Y, C, tid, nt);
        __syncthreads();
      }
      float2* tmp = X;
      X = Y;
      Y = tmp;
    }
  }
  if (renorm && (long long)nslices * steps_per_slice > 0) {  // the last step's trace factor
    res32_renorm(n, d, nb, X, C, tid, nt);
    __syncthreads();
  }
  for (int e = tid; e < nb * n; e += nt) states[(long long)b0 * n + e] = make_double2((double)X[e].x, (double)X[e].y);
}

__global__ void make_delta_f32_kernel(int n, long long total, const z64* __restrict__ P,
                                      float* __restrict__ Dr, float* __restrict__ Di) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long o = e % nn;
    const int i = (int)(o / n), j = (int)(o - (o / n) * n);
    z64 v = P[e];
    if (i == j) v.x -= 1.0;
    Dr[e] = (float)v.x;
    Di[e] = (float)v.y;
  }
}



// Out[b][i] = R[b][i] + sum_j D[i][j] R[b][j]; planar FP32.  BM x BN output
// tile (states x rows), TM x TN outputs per thread.  32 x 32 tiles give 184
// CTAs for 256 states x 729 rows, all resident at once on 152 SMs.


int isqrt_exact(int n) {
  int d = 1;
  while ((d + 1) * (d + 1) <= n) d++;
  return d;
}

unsigned grid_for(long long total, int threads, int sm_count) {
  long long g = (total + threads - 1) / threads;
  long long cap = (long long)sm_count * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

int pick_chunk(int B, int sm_count) { return std::max(1, (B + sm_count - 1) / sm_count); }

}  // namespace

bool resident_f64_fits(int n) { return n <= 81 && resident_f64_smem(n, 8) <= 227 * 1024; }
bool resident_f32_fits(int n) { return n <= 81; }

cudaError_t launch_propagate_resident_f64(int n, int nslices, const z64* P, int steps_per_slice, int B,
                                          z64* states, int sm_count, cudaStream_t st) {
  return launch_propagate_resident_f64_hist(n, nslices, P, steps_per_slice, B, states, 0, nullptr, sm_count, st);
}

cudaError_t launch_propagate_resident_f64_hist(int n, int nslices, const z64* P, int steps_per_slice, int B,
                                               z64* states, int adjoint, z64* hist, int sm_count,
                                               cudaStream_t st) {
  int lc = 0, lk = 0;
  if (n <= 16 && !adjoint && hist == nullptr && B <= sm_count && lat_split(n, &lc, &lk)) {
    // few states: one CTA of four warps per state (latency form)
    count_launch();
    if (lc <= 2)
      prop_lat_f64_kernel<2><<<B, 128, 0, st>>>(n, lc, lk, nslices, P, steps_per_slice, states);
    else if (lc <= 4)
      prop_lat_f64_kernel<4><<<B, 128, 0, st>>>(n, lc, lk, nslices, P, steps_per_slice, states);
    else
      prop_lat_f64_kernel<8><<<B, 128, 0, st>>>(n, lc, lk, nslices, P, steps_per_slice, states);
    return cudaGetLastError();
  }
  if (n <= 16 && !adjoint && hist == nullptr) {
    const int grid = (B * 32 + 127) / 128;
    const int K = 32 / n, C = (n + K - 1) / K;
    count_launch();
    if (C <= 1)
      prop_warp_f64_kernel<1><<<grid, 128, 0, st>>>(n, nslices, P, steps_per_slice, B, states);
    else if (C <= 3)
      prop_warp_f64_kernel<3><<<grid, 128, 0, st>>>(n, nslices, P, steps_per_slice, B, states);
    else
      prop_warp_f64_kernel<8><<<grid, 128, 0, st>>>(n, nslices, P, steps_per_slice, B, states);
    return cudaGetLastError();
  }
  int chunk = pick_chunk(B, sm_count);
  size_t smem = resident_f64_smem(n, chunk);
  while (smem > 227 * 1024 && chunk > 1) {
    chunk = (chunk + 1) / 2;
    smem = resident_f64_smem(n, chunk);
  }
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = set_smem_once((const void*)prop_resident_f64_kernel, smem);
  if (e != cudaSuccess) return e;
  const int grid = (B + chunk - 1) / chunk;
  count_launch();
  prop_resident_f64_kernel<<<grid, kResThreads, smem, st>>>(n, nslices, P, steps_per_slice, B, chunk,
                                                            states, adjoint, hist, 0, 0, 0, 0);
  return cudaGetLastError();
}

cudaError_t launch_propagate_resident_f64_multi(int n, int K, int nslices, const z64* P, int steps_per_slice, int B,
                                                z64* states, int adjoint, z64* hist, int sm_count, cudaStream_t st) {
  if (K < 1 || K > 65535) return cudaErrorInvalidValue;
  const long long nn = (long long)n * n, T = (long long)nslices * steps_per_slice;
  int chunk = std::max(1, std::min(B, (B * K + sm_count - 1) / sm_count));
  size_t smem = resident_f64_smem(n, chunk);
  while (smem > 227 * 1024 && chunk > 1) {
    chunk = (chunk + 1) / 2;
    smem = resident_f64_smem(n, chunk);
  }
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = set_smem_once((const void*)prop_resident_f64_kernel, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((B + chunk - 1) / chunk, K);
  count_launch();
  prop_resident_f64_kernel<<<grid, kResThreads, smem, st>>>(n, nslices, P, steps_per_slice, B, chunk, states,
                                                            adjoint, hist, nslices * nn, (long long)B * n,
                                                            T * B * n, 1);
  return cudaGetLastError();
}

cudaError_t launch_make_delta_f32(int n, int S, const z64* P, float* Dr, float* Di, cudaStream_t st) {
  const long long total = (long long)n * n * S;
  count_launch();
  make_delta_f32_kernel<<<grid_for(total, 256, 152), 256, 0, st>>>(n, total, P, Dr, Di);
  return cudaGetLastError();
}

cudaError_t launch_propagate_resident_f32(int n, int nslices, const float* Dr, const float* Di,
                                          int steps_per_slice, int B, z64* states, int renorm,
                                          int sm_count, cudaStream_t st) {
  int chunk = pick_chunk(B, sm_count);
  size_t smem = resident_f32_smem(n, chunk);
  while (smem > 227 * 1024 && chunk > 1) {
    chunk = (chunk + 1) / 2;
    smem = resident_f32_smem(n, chunk);
  }
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = set_smem_once((const void*)prop_resident_f32_kernel, smem);
  if (e != cudaSuccess) return e;
  const int grid = (B + chunk - 1) / chunk;
  // one thread per (row, pair of states) of the register-blocked step
  int threads = (n * ((chunk + 1) / 2) + 31) / 32 * 32;
  threads = std::max(64, std::min(1024, threads));
  count_launch();
  prop_resident_f32_kernel<<<grid, threads, smem, st>>>(n, isqrt_exact(n), nslices, Dr, Di, steps_per_slice, B,
                                                        chunk, renorm, states);
  return cudaGetLastError();
}





}  // namespace lb
