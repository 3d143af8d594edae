// FP64 propagation of density matrices on their real coordinates (the
// LB_FP64_HERMITIAN form of Algorithm 2, Sec. 3.2).
//
// A density matrix is Hermitian, and every propagator exp(L dt) of a
// Lindbladian maps Hermitian matrices to Hermitian matrices.  A Hermitian
// d x d matrix is fixed by n = d^2 real numbers, its coordinates
//   c = ( rho_00, ..., rho_{d-1,d-1},  Re rho_kl, Im rho_kl for k < l ),
// the pairs (k, l) in row-major order of the upper triangle; on them the
// step rho <- P rho is the real n x n map
//   R[a][b] = d(out_a) / d(c_b),
// with, for an output entry (k, l) and an input coordinate b,
//   b = rho_ii   :  P[kl][ii]
//   b = Re rho_ij:  P[kl][ij] + P[kl][ji]
//   b = Im rho_ij:  i (P[kl][ij] - P[kl][ji])
// and out_a the real part (diagonal and Re coordinates) or the imaginary
// part (Im coordinates) of that derivative.  A step then costs n^2 real
// multiply-adds instead of the 4 n^2 of the complex product: on a part whose
// FP64 instructions take 64 cycles per warp, that is what matters.  The
// result equals the complex product for Hermitian inputs up to rounding; the
// state is read from its diagonal and upper triangle, and written back
// exactly Hermitian.
//
// Shared-memory form (9 < n <= 81): R and the CTA's states in shared
// memory, one thread per output coordinate, like the complex resident form
// with a third of its FP64 instructions.
//
// Latency form (n <= 9, d <= 3): one warp per state.  Output coordinate o is
// summed by K lanes with C products each (C + ceil(log2 K) dependent FP64
// instructions, five at n = 9 against six for the complex step), and the new
// coordinates reach the lanes that need them by warp shuffles, so a step has
// no shared-memory exchange and no barrier.
#include "lb_internal.cuh"

#include <algorithm>

namespace lb {
namespace {

// a CTA per row a of R[s], its threads along the row
__global__ void herm_matrix_kernel(int n, int d, int S, const z64* __restrict__ P, double* __restrict__ R) {
  const long long nn = (long long)n * n, rows = (long long)S * n;
  for (long long rw = blockIdx.x; rw < rows; rw += gridDim.x) {
    const long long s = rw / n;
    const int a = (int)(rw - s * n);
    int k, l, pa;
    herm_coord(a, d, &k, &l, &pa);
    const z64* row = P + s * nn + (long long)(k * d + l) * n;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
      int i, j, pb;
      herm_coord(b, d, &i, &j, &pb);
      z64 v;
      if (pb == 0) {
        v = row[i * d + i];
      } else {
        const z64 pij = row[i * d + j], pji = row[j * d + i];
        v = pb == 1 ? make_double2(pij.x + pji.x, pij.y + pji.y)      // Re rho_ij
                    : make_double2(-(pij.y - pji.y), pij.x - pji.x);  // Im rho_ij: i (P_ij - P_ji)
      }
      R[rw * n + b] = pa == 2 ? v.y : v.x;
    }
  }
}

constexpr unsigned kFullMask = 0xffffffffu;

template <int CMAX>
__global__ void __launch_bounds__(32)
    prop_herm_lat_kernel(int n, int d, int C, int K, int nslices, const double* __restrict__ R, int steps_per_slice,
                         z64* __restrict__ states) {
  __shared__ double cst[32];
  const int lane = threadIdx.x;
  const int o = lane / K, p = lane - (lane / K) * K;
  const bool active = o < n;
  z64* x = states + (long long)blockIdx.x * n;
  if (lane < n) {  // the state's real coordinates
    int k, l, part;
    herm_coord(lane, d, &k, &l, &part);
    const z64 v = x[k * d + l];
    cst[lane] = part == 2 ? v.y : v.x;
  }
  __syncwarp();
  // this lane's C inputs (coordinate indices), their values, the lane holding
  // each of them after a step
  int xin[CMAX];
  double xv[CMAX];
#pragma unroll
  for (int c = 0; c < CMAX; c++) {
    const int j = p * C + c;
    xin[c] = (active && c < C && j < n) ? j : -1;
    xv[c] = xin[c] >= 0 ? cst[xin[c]] : 0.0;
  }
  const long long nn = (long long)n * n;
  double out = 0.0;
  for (int s = 0; s < nslices; s++) {
    double cf[CMAX];
#pragma unroll
    for (int c = 0; c < CMAX; c++) cf[c] = xin[c] >= 0 ? R[s * nn + (long long)o * n + xin[c]] : 0.0;
    for (int t = 0; t < steps_per_slice; t++) {
      double acc = cf[0] * xv[0];
#pragma unroll
      for (int c = 1; c < CMAX; c++)
        if (c < C) acc = fma(cf[c], xv[c], acc);
      // sum over the K lanes of output o; lane o*K ends with it.  For K = 3
      // both neighbours' sums are fetched at once and added in order
      // ((a0 + a1) + a2, as the two-level tree does), which takes one shuffle
      // off the dependent chain
      if (K == 3) {
        const double v1 = __shfl_down_sync(kFullMask, acc, 1);
        const double v2 = __shfl_down_sync(kFullMask, acc, 2);
        if (p == 0) acc = (acc + v1) + v2;
      } else {
        for (int off = 1; off < K; off <<= 1) {
          const double v = __shfl_down_sync(kFullMask, acc, off);
          if (p + off < K) acc += v;
        }
      }
      out = acc;
#pragma unroll
      for (int c = 0; c < CMAX; c++) {
        const double v = __shfl_sync(kFullMask, acc, xin[c] >= 0 ? xin[c] * K : 0);
        if (xin[c] >= 0) xv[c] = v;
      }
    }
  }
  if ((long long)nslices * steps_per_slice == 0) return;
  if (active && p == 0) cst[o] = out;
  __syncwarp();
  if (lane < n) {  // back to the complex matrix, exactly Hermitian
    const int r = lane / d, c = lane - (lane / d) * d;
    z64 v;
    if (r == c) {
      v = make_double2(cst[r], 0.0);
    } else {
      const int k = r < c ? r : c, l = r < c ? c : r;
      int q = 0;
      for (int rr = 0; rr < k; rr++) q += d - 1 - rr;
      q += l - k - 1;
      const double re = cst[d + 2 * q], im = cst[d + 2 * q + 1];
      v = make_double2(re, r < c ? im : -im);
    }
    x[lane] = v;
  }
}

// Shared-memory form (9 < n <= 81): R of the current slice and the CTA's
// states (real coordinates, ping-pong) in shared memory for the whole
// chain, one thread per (state, coordinate) output, one barrier per step.
__global__ void __launch_bounds__(1024)
    prop_herm_resident_kernel(int n, int d, int nslices, const double* __restrict__ R, int steps_per_slice, int B,
                              int chunk, z64* __restrict__ states) {
  extern __shared__ __align__(16) double hsm[];
  double* Rs = hsm;
  double* x = Rs + n * n;  // chunk x n
  double* y = x + chunk * n;
  const int b0 = blockIdx.x * chunk;
  if (b0 >= B) return;
  const int nb = min(chunk, B - b0);
  const int tid = threadIdx.x, nt = blockDim.x, work = nb * n;
  const long long nn = (long long)n * n;
  z64* X = states + (long long)b0 * n;
  for (int e = tid; e < work; e += nt) {
    const int q = e / n, a = e - (e / n) * n;
    int k, l, part;
    herm_coord(a, d, &k, &l, &part);
    const z64 v = X[(long long)q * n + k * d + l];
    x[e] = part == 2 ? v.y : v.x;
  }
  for (int s = 0; s < nslices; s++) {
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) Rs[e] = R[s * nn + e];
    __syncthreads();
    for (int t = 0; t < steps_per_slice; t++) {
      for (int e = tid; e < work; e += nt) {
        const int q = e / n, a = e - (e / n) * n;
        const double* r = Rs + a * n;
        const double* xq = x + q * n;
        double acc = 0.0;
#pragma unroll 9
        for (int b = 0; b < n; b++) acc = fma(r[b], xq[b], acc);
        y[e] = acc;
      }
      __syncthreads();
      double* tmp = x;
      x = y;
      y = tmp;
    }
  }
  __syncthreads();
  for (int e = tid; e < work; e += nt) {  // back to complex matrices, exactly Hermitian
    const int q = e / n, m = e - (e / n) * n;
    const int r = m / d, c = m - (m / d) * d;
    const double* xq = x + q * n;
    z64 v;
    if (r == c) {
      v = make_double2(xq[r], 0.0);
    } else {
      const int k = r < c ? r : c, l = r < c ? c : r;
      int qq = 0;
      for (int rr = 0; rr < k; rr++) qq += d - 1 - rr;
      qq += l - k - 1;
      const double re = xq[d + 2 * qq], im = xq[d + 2 * qq + 1];
      v = make_double2(re, r < c ? im : -im);
    }
    X[e] = v;
  }
}

// states (complex B x n) <-> real coordinates (B x n)
__global__ void herm_coords_in_kernel(int n, int d, long long total, const z64* __restrict__ X, double* __restrict__ Y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / n;
    const int a = (int)(t - b * n);
    int k, l, part;
    herm_coord(a, d, &k, &l, &part);
    const z64 v = X[b * n + k * d + l];
    Y[t] = part == 2 ? v.y : v.x;
  }
}

__global__ void herm_coords_out_kernel(int n, int d, long long total, const double* __restrict__ Y, z64* __restrict__ X) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / n;
    const int m = (int)(t - b * n), r = m / d, c = m - (m / d) * d;
    const double* y = Y + b * n;
    if (r == c) {
      X[t] = make_double2(y[r], 0.0);
    } else {
      const int idx = herm_pair_coord(r < c ? r : c, r < c ? c : r, d);
      X[t] = make_double2(y[idx], r < c ? y[idx + 1] : -y[idx + 1]);
    }
  }
}

// Largest column abs-sum of S real n x n matrices into *norm_bits (bits of a
// non-negative double, integer max); 8 columns x 32 row groups per CTA, the
// partial sums of a column added in a fixed order.
__global__ void __launch_bounds__(256) real_colnorm_kernel(int n, int S, const double* __restrict__ G,
                                                          unsigned long long* __restrict__ norm_bits) {
  __shared__ double part[32][8];
  const long long nn = (long long)n * n;
  const int c = threadIdx.x % 8, rg = threadIdx.x / 8;
  const int cblocks = (n + 7) / 8;
  for (long long t = blockIdx.x; t < (long long)S * cblocks; t += gridDim.x) {
    const int s = (int)(t / cblocks), j = (int)(t - (t / cblocks) * cblocks) * 8 + c;
    double sum = 0.0;
    if (j < n)
      for (int i = rg; i < n; i += 32) sum += fabs(G[s * nn + (long long)i * n + j]);
    part[rg][c] = sum;
    __syncthreads();
    if (rg == 0 && j < n) {
      double col = 0.0;
      for (int r = 0; r < 32; r++) col += part[r][c];
      if (!(col == col)) col = INFINITY;
      atomicMax(norm_bits, (unsigned long long)__double_as_longlong(col));
    }
    __syncthreads();
  }
}

unsigned grid_cap(long long work, int per_block, int sm_count) {
  long long g = (work + per_block - 1) / per_block;
  const long long cap = (long long)sm_count * 8;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_herm_coords_in(int n, int d, int B, const z64* X, double* Y, int sm_count, cudaStream_t st) {
  const long long total = (long long)B * n;
  count_launch();
  herm_coords_in_kernel<<<grid_cap(total, 256, sm_count), 256, 0, st>>>(n, d, total, X, Y);
  return cudaGetLastError();
}

cudaError_t launch_herm_coords_out(int n, int d, int B, const double* Y, z64* X, int sm_count, cudaStream_t st) {
  const long long total = (long long)B * n;
  count_launch();
  herm_coords_out_kernel<<<grid_cap(total, 256, sm_count), 256, 0, st>>>(n, d, total, Y, X);
  return cudaGetLastError();
}

cudaError_t launch_real_colnorm(int n, int S, const double* G, unsigned long long* norm_bits, int sm_count,
                                cudaStream_t st) {
  const long long tiles = (long long)S * ((n + 7) / 8);
  count_launch();
  real_colnorm_kernel<<<grid_cap(tiles, 1, sm_count), 256, 0, st>>>(n, S, G, norm_bits);
  return cudaGetLastError();
}

size_t herm_resident_smem(int n, int chunk) { return sizeof(double) * ((size_t)n * n + 2ull * chunk * n); }

bool herm_resident_fits(int n) { return n <= 81 && herm_resident_smem(n, 1) <= 227 * 1024; }

cudaError_t launch_prop_herm_resident(int n, int d, int nslices, const double* R, int steps_per_slice, int B,
                                      z64* X, int sm_count, cudaStream_t st) {
  int chunk = std::max(1, (B + sm_count - 1) / sm_count);
  chunk = std::min(chunk, std::max(1, 1024 / n));  // one thread per output
  while (chunk > 1 && herm_resident_smem(n, chunk) > 227 * 1024) chunk = (chunk + 1) / 2;
  const size_t smem = herm_resident_smem(n, chunk);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = set_smem_once((const void*)prop_herm_resident_kernel, smem);
  if (e != cudaSuccess) return e;
  const int threads = std::min(1024, (chunk * n + 31) / 32 * 32);
  const int grid = (B + chunk - 1) / chunk;
  count_launch();
  prop_herm_resident_kernel<<<grid, threads, smem, st>>>(n, d, nslices, R, steps_per_slice, B, chunk, X);
  return cudaGetLastError();
}

// Split of the n real products of an output over K lanes with C each: at
// most 32 lanes for the n outputs, fewest dependent FP64 instructions
// (C + ceil(log2 K)), then the fewest lanes.
bool herm_lat_split(int n, int* C, int* K) {
  if (n < 1 || n > 9) return false;
  int best = 1 << 30;
  for (int k = 1; k * n <= 32; k++) {
    const int c = (n + k - 1) / k;
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

cudaError_t launch_herm_matrix(int n, int d, int S, const z64* P, double* R, int sm_count, cudaStream_t st) {
  long long blocks = (long long)S * n;
  if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
  count_launch();
  herm_matrix_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, d, S, P, R);
  return cudaGetLastError();
}

cudaError_t launch_prop_herm_lat(int n, int d, int nslices, const double* R, int steps_per_slice, int B, z64* X,
                                 cudaStream_t st) {
  int C = 0, K = 0;
  if (!herm_lat_split(n, &C, &K)) return cudaErrorInvalidValue;
  count_launch();
  if (C <= 3)
    prop_herm_lat_kernel<3><<<B, 32, 0, st>>>(n, d, C, K, nslices, R, steps_per_slice, X);
  else
    prop_herm_lat_kernel<9><<<B, 32, 0, st>>>(n, d, C, K, nslices, R, steps_per_slice, X);
  return cudaGetLastError();
}

}  // namespace lb
