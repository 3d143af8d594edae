// Small-batch FP64 complex matrix-vector products: one propagation step
// (Algorithm 2, Sec. 3.2) or one Taylor term of the action of the
// exponential, for B <= 8 states at once.
//
//   V[b][i]     = alpha * sum_j A[i][j] X[b][j]
//   Yacc[b][i] += alpha * sum_j A[i][j] X[b][j]      (optional)
//
// With few states a tiled GEMM leaves most of the GPU idle (a 64-row tile
// holds one state; n = 729 gives 12 CTAs), and FP64 runs at 1/64 of the FP32
// rate, so the work has to reach every SM sub-partition.  A warp owns one
// output row i (or, for n > 256, half of it) for all B states: its lanes
// stride over j, so each load of A's row is coalesced (the transpose of the
// paper's gather, Algorithm alg:gpu), A[i][j] is read once for all B states,
// and the states (B x n, at most 94 KB) stay in L1 and L2.  The lane sums
// meet in a butterfly of shuffles that leaves the same bits in every lane;
// lane b writes state b.  n = 729 gives 1458 half-row warps over the 608
// sub-partitions.  The summation order is fixed, so the result is the same
// on every run.
#include "lb_internal.cuh"

namespace lb {
namespace {

constexpr int kGemvWarps = 4;
constexpr unsigned kFull = 0xffffffffu;

// Row i is split into H contiguous parts, one warp each (H = 2 for long
// rows: 2n parts over the 608 sub-partitions balance better than n rows);
// the parts of a row sit in one CTA and meet in shared memory, part 0 adding
// the others in order.  U row loads of A per lane are issued before their
// products: with a few warps per SM nothing else hides the latency of a load
// from L2 or HBM.
template <int BB, int U, int H>
__global__ void __launch_bounds__(kGemvWarps * 32)
    zgemv_f64_kernel(int n, int B, const z64* __restrict__ A, long long lda, const z64* __restrict__ X,
                     long long ldx, z64* __restrict__ V, long long ldv, double alpha, z64* __restrict__ Yacc,
                     long long ldacc) {
  __shared__ double red[kGemvWarps][2 * BB];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row = blockIdx.x * (kGemvWarps / H) + w / H, part = w % H;
  const bool rowok = row < n;  // no early return: the parts meet at a barrier
  const int seg = (n + H - 1) / H;
  const int jb = part * seg, je = min(n, jb + seg);
  double ar[BB], ai[BB];
#pragma unroll
  for (int b = 0; b < BB; b++) ar[b] = ai[b] = 0.0;
  const z64* a = A + (long long)(rowok ? row : 0) * lda;
  for (int j0 = jb + lane; rowok && j0 < je; j0 += 32 * U) {
    z64 p[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      const int j = j0 + 32 * k;
      p[k] = j < je ? a[j] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int k = 0; k < U; k++) {
      const int j = j0 + 32 * k;
      if (j < je) {
#pragma unroll
        for (int b = 0; b < BB; b++) {
          if (b < B) {
            const z64 x = X[b * ldx + j];
            ar[b] = fma(p[k].x, x.x, ar[b]);
            ar[b] = fma(-p[k].y, x.y, ar[b]);
            ai[b] = fma(p[k].x, x.y, ai[b]);
            ai[b] = fma(p[k].y, x.x, ai[b]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int b = 0; b < BB; b++) {
      if (b < B) {
        ar[b] += __shfl_xor_sync(kFull, ar[b], off);
        ai[b] += __shfl_xor_sync(kFull, ai[b], off);
      }
    }
  }
  if (H > 1) {
    if (lane == 0) {
#pragma unroll
      for (int b = 0; b < BB; b++) {
        red[w][2 * b] = ar[b];
        red[w][2 * b + 1] = ai[b];
      }
    }
    __syncthreads();
    if (part == 0) {
#pragma unroll
      for (int b = 0; b < BB; b++) {
        for (int h = 1; h < H; h++) {
          ar[b] += red[w + h][2 * b];
          ai[b] += red[w + h][2 * b + 1];
        }
      }
    }
  }
#pragma unroll
  for (int b = 0; b < BB; b++) {
    if (rowok && part == 0 && b < B && lane == b) {
      V[b * ldv + row] = make_double2(alpha * ar[b], alpha * ai[b]);
      if (Yacc != nullptr) {
        z64* y = Yacc + b * ldacc + row;
        const z64 y0 = *y;
        *y = make_double2(fma(alpha, ar[b], y0.x), fma(alpha, ai[b], y0.y));
      }
    }
  }
}

// The same product for real matrices and states (the Hermitian coordinates
// of density matrices): V[b][i] = alpha sum_j A[i][j] X[b][j], Yacc += it.
template <int BB, int U, int H>
__global__ void __launch_bounds__(kGemvWarps * 32)
    dgemv_f64_kernel(int n, int B, const double* __restrict__ A, long long lda, const double* __restrict__ X,
                     long long ldx, double* __restrict__ V, long long ldv, double alpha, double* __restrict__ Yacc,
                     long long ldacc) {
  __shared__ double red[kGemvWarps][BB];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row = blockIdx.x * (kGemvWarps / H) + w / H, part = w % H;
  const bool rowok = row < n;  // no early return: the parts meet at a barrier
  const int seg = (n + H - 1) / H;
  const int jb = part * seg, je = min(n, jb + seg);
  double acc[BB];
#pragma unroll
  for (int b = 0; b < BB; b++) acc[b] = 0.0;
  const double* a = A + (long long)(rowok ? row : 0) * lda;
  for (int j0 = jb + lane; rowok && j0 < je; j0 += 32 * U) {
    double p[U];
#pragma unroll
    for (int k = 0; k < U; k++) {
      const int j = j0 + 32 * k;
      p[k] = j < je ? a[j] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < U; k++) {
      const int j = j0 + 32 * k;
      if (j < je) {
#pragma unroll
        for (int b = 0; b < BB; b++)
          if (b < B) acc[b] = fma(p[k], X[b * ldx + j], acc[b]);
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int b = 0; b < BB; b++)
      if (b < B) acc[b] += __shfl_xor_sync(kFull, acc[b], off);
  }
  if (H > 1) {
    if (lane == 0) {
#pragma unroll
      for (int b = 0; b < BB; b++) red[w][b] = acc[b];
    }
    __syncthreads();
    if (part == 0) {
#pragma unroll
      for (int b = 0; b < BB; b++)
        for (int h = 1; h < H; h++) acc[b] += red[w + h][b];
    }
  }
#pragma unroll
  for (int b = 0; b < BB; b++) {
    if (rowok && part == 0 && b < B && lane == b) {
      V[b * ldv + row] = alpha * acc[b];
      if (Yacc != nullptr) Yacc[b * ldacc + row] = fma(alpha, acc[b], Yacc[b * ldacc + row]);
    }
  }
}

}  // namespace

cudaError_t launch_dgemv_f64(int n, int B, const double* A, long long lda, const double* X, long long ldx, double* V,
                             long long ldv, double alpha, double* Yacc, long long ldacc, cudaStream_t st) {
  if (B < 1 || B > kGemvMaxB || n < 1) return cudaErrorInvalidValue;
  const int threads = kGemvWarps * 32;
  count_launch();
  if (n > 256) {  // two warps per row
    const unsigned grid = (unsigned)((n + kGemvWarps / 2 - 1) / (kGemvWarps / 2));
    if (B <= 2)
      dgemv_f64_kernel<2, 12, 2><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
    else
      dgemv_f64_kernel<8, 4, 2><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
  } else {
    const unsigned grid = (unsigned)((n + kGemvWarps - 1) / kGemvWarps);
    if (B <= 2)
      dgemv_f64_kernel<2, 8, 1><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
    else
      dgemv_f64_kernel<8, 4, 1><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
  }
  return cudaGetLastError();
}

cudaError_t launch_zgemv_f64(int n, int B, const z64* A, long long lda, const z64* X, long long ldx, z64* V,
                             long long ldv, double alpha, z64* Yacc, long long ldacc, cudaStream_t st) {
  if (B < 1 || B > kGemvMaxB || n < 1) return cudaErrorInvalidValue;
  const int threads = kGemvWarps * 32;
  count_launch();
  if (n > 256) {  // two warps per row
    const unsigned grid = (unsigned)((n + kGemvWarps / 2 - 1) / (kGemvWarps / 2));
    if (B == 1)
      zgemv_f64_kernel<1, 12, 2><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
    else if (B == 2)
      zgemv_f64_kernel<2, 12, 2><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
    else if (B <= 4)
      zgemv_f64_kernel<4, 4, 2><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
    else
      zgemv_f64_kernel<8, 4, 2><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
  } else {
    const unsigned grid = (unsigned)((n + kGemvWarps - 1) / kGemvWarps);
    if (B == 1)
      zgemv_f64_kernel<1, 8, 1><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
    else if (B == 2)
      zgemv_f64_kernel<2, 8, 1><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
    else if (B <= 4)
      zgemv_f64_kernel<4, 4, 1><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
    else
      zgemv_f64_kernel<8, 4, 1><<<grid, threads, 0, st>>>(n, B, A, lda, X, ldx, V, ldv, alpha, Yacc, ldacc);
  }
  return cudaGetLastError();
}

bool gemv_f64_preferred(int n, int B) {
  // Against the resident kernels (n <= 81: one SM per group of states) and
  // the tiled GEMM: few states at n <= 16 stay with the latency kernel.
  if (n <= 16) return false;
  if (n <= 81) return B <= 4;
  return B <= kGemvMaxB;
}

}  // namespace lb
