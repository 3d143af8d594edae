// Grouped, batched REAL GEMM on the CUDA cores, FP64 and FP32.
//
// The real-coordinate ("Hermitian") forms of the propagator build and of the
// propagation run every product of Algorithm 1 (the three powers, the three
// U/V products, the LU updates, the substitutions, the squarings) and of
// Algorithm 2 on real n x n matrices: a density matrix is Hermitian and
// exp(L dt) maps Hermitian matrices to Hermitian matrices, so on the n = d^2
// real coordinates of a Hermitian matrix both L dt and exp(L dt) are real
// n x n matrices.  A real multiply-add is one FMA, against three (Gauss form)
// or four for a complex one, which on GB300, where FP64 runs at 1/64 of the
// FP32 rate, is what bounds the build.
//
//   r_w   = alpha[w] acc + beta[w] O_w(old) + sum_t coef[w][t] X_t + gamma[w] I   (arithmetic in T)
//   O_w   = r_w                                          (T, when O[w] != null)
//   Od_w  = double(r_w) + dcoef[w] Xd + dgamma[w] I      (FP64, when Od[w] != null)
// for w = 0, 1, with acc = opA(A) opB(B) accumulated in T.  FP64 (T = double)
// uses O; FP32 (T = float: operands and accumulation in FP32, as in the
// reduced-precision forms) writes FP32 results for the next product and
// widens the ones the FP64 LU consumes, with the terms that must stay exact
// (the identity, b_1 A, 2P) added in FP64.
//
// The kernel is the same flat list of output tiles over problems x batch,
// walked by a persistent grid, as the complex GEMM.  FP64 tiles are 32 x 32
// (2 x 2 per thread; at n = 729 the ragged edge wastes 2 % against 11 % for
// 64 x 64), FP32 tiles 64 x 64 (4 x 4 per thread, vector loads of the shared
// tiles, so the FMA pipe and not shared memory is the limit).  The K loop is
// double-buffered: the next 16-wide K block is fetched into registers while
// the current one is multiplied out of shared memory.
#include "lb_internal.cuh"

#include <algorithm>

namespace lb {

namespace {

template <typename T>
struct RGroup {
  RGemmProblem<T> p[4];
  long long tile_start[5];
  int tiles_m[4];
  int tiles_n[4];
  int nprob;
};

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ double flip(double v, unsigned long long m) {
  return __longlong_as_double(__double_as_longlong(v) ^ (long long)m);
}
__device__ __forceinline__ float flip(float v, unsigned long long m) {
  return __int_as_float(__float_as_int(v) ^ (int)(m >> 32));
}

template <typename T, int TM>
struct Vec;
template <>
struct Vec<double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double* r) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    r[0] = v.x;
    r[1] = v.y;
  }
};
template <>
struct Vec<double, 1> {
  static __device__ __forceinline__ void ld(const double* p, double* r) { r[0] = p[0]; }
};
template <>
struct Vec<double, 4> {
  static __device__ __forceinline__ void ld(const double* p, double* r) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    r[0] = a.x;
    r[1] = a.y;
    r[2] = b.x;
    r[3] = b.y;
  }
};
template <>
struct Vec<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float* r) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    r[0] = v.x;
    r[1] = v.y;
    r[2] = v.z;
    r[3] = v.w;
  }
};
template <>
struct Vec<float, 2> {
  static __device__ __forceinline__ void ld(const float* p, float* r) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    r[0] = v.x;
    r[1] = v.y;
  }
};

// The epilogue of one output element (see the header comment): r_w in T,
// then the FP64 widened outputs with their exact FP64 terms.
template <typename T>
__device__ __forceinline__ void store_out(const RGemmProblem<T>& P, long long b, int gm, int gn, T accv) {
  const long long off = (long long)gm * P.ldc + gn;
  const long long idx = b * P.sC + off;
#pragma unroll
  for (int w = 0; w < 2; w++) {
    if (P.O[w] == nullptr && P.Od[w] == nullptr) continue;
    T v = T(P.alpha[w]) * accv;
    if (P.beta[w] != 0.0 && P.O[w] != nullptr) v = fma_t(T(P.beta[w]), P.O[w][idx], v);
    for (int q = 0; q < P.nterms; q++) v = fma_t(T(P.coef[w][q]), P.X[q][b * P.sX[q] + off], v);
    if (gm == gn) v += T(P.gamma[w]);
    if (P.O[w] != nullptr) P.O[w][idx] = v;
    if (P.Od[w] != nullptr) {
      double vd = double(v);
      if (P.dcoef[w] != 0.0) vd = fma(P.dcoef[w], P.Xd[b * P.sXd + off], vd);
      if (gm == gn) vd += P.dgamma[w];
      P.Od[w][idx] = vd;
    }
  }
}

// Resident CTAs per SM the register allocation is held to: 1 x 1 thread
// tiles (small problems, many tiles) keep enough CTAs for every tile to be
// resident at once; larger thread tiles two.
template <int TM, int TN>
constexpr int rgemm_min_ctas() {
  return TM * TN == 1 ? 6 : 2;
}

template <typename T, int BM, int BN, int TM, int TN, bool DB>
__global__ void __launch_bounds__((BM / TM) * (BN / TN), rgemm_min_ctas<TM, TN>())
    rgemm_kernel(const __grid_constant__ RGroup<T> g) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int BK = 16;
  constexpr int LA = BM * BK / NT, LB = BK * BN / NT;  // tile elements each thread stages
  static_assert(LA * NT == BM * BK && LB * NT == BK * BN, "tile must divide over the threads");
  // DB: two shared-memory stages, the next K block fetched into registers
  // while the current one is multiplied, then stored into the other stage
  __shared__ __align__(16) T As[DB ? 2 : 1][BK][BM];
  __shared__ __align__(16) T Bs[DB ? 2 : 1][BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN);
  const int ty = tid / (BN / TN);
  const long long total = g.tile_start[g.nprob];

  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    int pi = 0;
    while (pi + 1 < g.nprob && t >= g.tile_start[pi + 1]) pi++;
    const RGemmProblem<T>& P = g.p[pi];
    const long long lt = t - g.tile_start[pi];
    const int tpb = g.tiles_m[pi] * g.tiles_n[pi];
    const long long b = lt / tpb;
    const int r = (int)(lt - b * tpb);
    const int tm = r / g.tiles_n[pi];
    const int tn = r - tm * g.tiles_n[pi];
    if (P.active != nullptr && P.active[b] <= P.active_iter) continue;
    if (P.active_lo != nullptr && P.active_lo[b] > P.active_iter) continue;
    if (P.pick != nullptr && P.pick[b] != P.pick_val) continue;
    const int m0 = tm * BM, n0 = tn * BN;
    const T* __restrict__ A = P.A + b * P.sA;
    const T* __restrict__ B = P.B + b * P.sB;
    const int M = P.M, N = P.N, K = P.K;

    // O_0 +- A B and nothing else (the LU updates): start the accumulators
    // from O_0 and fold the sign into A, so the epilogue is a plain store.
    const bool fastC = P.beta[0] == 1.0 && (P.alpha[0] == 1.0 || P.alpha[0] == -1.0) && P.nterms == 0 &&
                       P.gamma[0] == 0.0 && P.O[0] != nullptr && P.Od[0] == nullptr && P.O[1] == nullptr &&
                       P.Od[1] == nullptr;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
      for (int j = 0; j < TN; j++) {
        acc[i][j] = T(0);
        if (fastC) {
          const int gm = m0 + ty * TM + i, gn = n0 + tx * TN + j;
          if (gm < M && gn < N) acc[i][j] = P.O[0][b * P.sC + (long long)gm * P.ldc + gn];
        }
      }
    const unsigned long long aneg = (fastC && P.alpha[0] < 0.0) ? 0x8000000000000000ull : 0ull;
    const T shA = T(P.shiftA), shB = T(P.shiftB);
    const bool bT = P.transB != 0;

    T ra[LA], rb[LB];
    // global -> registers for the K block at k0 (zero outside the matrices)
    auto fetch = [&](int k0) {
#pragma unroll
      for (int q = 0; q < LA; q++) {
        const int e = tid + q * NT;
        const int m = e / BK, k = e - (e / BK) * BK;
        const int gm = m0 + m, gk = k0 + k;
        T v = T(0);
        if (gm < M && gk < K) {
          v = A[(long long)gm * P.lda + gk];
          if (gm == gk) v -= shA;
        }
        ra[q] = flip(v, aneg);
      }
#pragma unroll
      for (int q = 0; q < LB; q++) {
        const int e = tid + q * NT;
        int k, c;
        if (bT) {
          c = e / BK;
          k = e - c * BK;
        } else {
          k = e / BN;
          c = e - k * BN;
        }
        const int gk = k0 + k, gn = n0 + c;
        T v = T(0);
        if (gk < K && gn < N) {
          v = bT ? B[(long long)gn * P.ldb + gk] : B[(long long)gk * P.ldb + gn];
          if (gk == gn) v -= shB;
        }
        rb[q] = v;
      }
    };
    auto stash = [&](int st) {
#pragma unroll
      for (int q = 0; q < LA; q++) {
        const int e = tid + q * NT;
        As[st][e - (e / BK) * BK][e / BK] = ra[q];
      }
#pragma unroll
      for (int q = 0; q < LB; q++) {
        const int e = tid + q * NT;
        if (bT)
          Bs[st][e - (e / BK) * BK][e / BK] = rb[q];
        else
          Bs[st][e / BN][e - (e / BN) * BN] = rb[q];
      }
    };

    auto multiply = [&](int st) {
#pragma unroll
      for (int k = 0; k < BK; k++) {
        T a[TM], bb[TN];
        Vec<T, TM>::ld(&As[st][k][ty * TM], a);
        Vec<T, TN>::ld(&Bs[st][k][tx * TN], bb);
#pragma unroll
        for (int i = 0; i < TM; i++)
#pragma unroll
          for (int j = 0; j < TN; j++) acc[i][j] = fma_t(a[i], bb[j], acc[i][j]);
      }
    };
    if (DB) {
      fetch(0);
      stash(0);
      __syncthreads();
      int st = 0;
      for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) fetch(k0 + BK);  // loads in flight during the products below
        multiply(st);
        if (more) stash(st ^ 1);
        __syncthreads();
        st ^= 1;
      }
    } else {  // one stage: fewer registers, more resident CTAs
      for (int k0 = 0; k0 < K; k0 += BK) {
        fetch(k0);
        stash(0);
        __syncthreads();
        multiply(0);
        __syncthreads();
      }
    }

#pragma unroll
    for (int i = 0; i < TM; i++) {
      const int gm = m0 + ty * TM + i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; j++) {
        const int gn = n0 + tx * TN + j;
        if (gn >= N) continue;
        if (fastC) {
          P.O[0][b * P.sC + (long long)gm * P.ldc + gn] = acc[i][j];
          continue;
        }
        store_out(P, b, gm, gn, acc[i][j]);
      }
    }
  }
}

// Row-sparse left operand (the zero-skip of the paper's Pade products,
// Sec. 3.1): one warp per output row gm of batch element b, lane l owning
// the columns l + 32 q (q < NQ, all N of them); A's row is scanned 32
// entries at a time (coalesced), a ballot marks the nonzeros, and only those
// rows of B are multiplied in (coalesced row reads).  For a row with z
// nonzeros that is z N multiply-adds instead of K N; the low powers of a
// local Lindbladian have a few percent of nonzeros.
template <typename T, int NQ>
__global__ void __launch_bounds__(256) rgemm_rowskip_kernel(const __grid_constant__ RGemmProblem<T> P) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long rows = (long long)P.batch * P.M;
  const T shA = T(P.shiftA);
  for (long long t = wid; t < rows; t += nw) {
    const long long b = t / P.M;
    const int gm = (int)(t - b * P.M);
    // batch-element tests are the same for every lane of the warp
    if (P.pick != nullptr && P.pick[b] != P.pick_val) continue;
    if (P.active != nullptr && P.active[b] <= P.active_iter) continue;
    if (P.active_lo != nullptr && P.active_lo[b] > P.active_iter) continue;
    const T* __restrict__ arow = P.A + b * P.sA + (long long)gm * P.lda;
    const T* __restrict__ B = P.B + b * P.sB;
    T acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) acc[q] = T(0);
    for (int k0 = 0; k0 < P.K; k0 += 32) {
      const int k = k0 + lane;
      T v = T(0);
      if (k < P.K) {
        v = arow[k];
        if (k == gm) v -= shA;
      }
      unsigned mask = __ballot_sync(kFull, v != T(0));
      while (mask != 0u) {
        const int bit = __ffs(mask) - 1;
        mask &= mask - 1u;
        const T a = __shfl_sync(kFull, v, bit);
        const T* __restrict__ brow = B + (long long)(k0 + bit) * P.ldb;
        T bv[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
          const int j = lane + 32 * q;
          bv[q] = j < P.N ? brow[j] : T(0);
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) acc[q] = fma_t(a, bv[q], acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; q++) {
      const int j = lane + 32 * q;
      if (j < P.N) store_out(P, b, gm, j, acc[q]);
    }
  }
}

// The same product with A's nonzero pattern given by rows (the column
// indices of row r in increasing order at cols[rowbeg[r] .. rowend[r])), a
// superset of every batch element's nonzeros: one warp per output row, the
// row's pattern read 32 entries at a time, an entry that is zero in this
// batch element skipped, so the terms and their order are those of
// rgemm_rowskip_kernel.  Two rows of B are in flight at a time.
template <typename T, int NQ>
__global__ void __launch_bounds__(256) rgemm_csr_kernel(const __grid_constant__ RGemmProblem<T> P,
                                                        const int* __restrict__ rowbeg, const int* __restrict__ rowend,
                                                        const int* __restrict__ cols) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long rows = (long long)P.batch * P.M;
  for (long long t = wid; t < rows; t += nw) {
    const long long b = t / P.M;
    const int gm = (int)(t - b * P.M);
    if (P.pick != nullptr && P.pick[b] != P.pick_val) continue;
    if (P.active != nullptr && P.active[b] <= P.active_iter) continue;
    if (P.active_lo != nullptr && P.active_lo[b] > P.active_iter) continue;
    const T* __restrict__ arow = P.A + b * P.sA + (long long)gm * P.lda;
    const T* __restrict__ B = P.B + b * P.sB;
    T acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) acc[q] = T(0);
    const int j0 = rowbeg[gm], j1 = rowend[gm];
    for (int jb = j0; jb < j1; jb += 32) {
      int k = 0;
      T v = T(0);
      if (jb + lane < j1) {
        k = cols[jb + lane];
        v = arow[k];
      }
      unsigned mask = __ballot_sync(kFull, v != T(0));
      while (mask != 0u) {
        const int bit0 = __ffs(mask) - 1;
        mask &= mask - 1u;
        const int bit1 = mask != 0u ? __ffs(mask) - 1 : -1;
        if (bit1 >= 0) mask &= mask - 1u;
        const T a0 = __shfl_sync(kFull, v, bit0);
        const int k0 = __shfl_sync(kFull, k, bit0);
        const T a1 = __shfl_sync(kFull, v, bit1 < 0 ? 0 : bit1);
        const int k1 = __shfl_sync(kFull, k, bit1 < 0 ? 0 : bit1);
        const T* __restrict__ b0 = B + (long long)k0 * P.ldb;
        const T* __restrict__ b1 = B + (long long)k1 * P.ldb;
        T u0[NQ], u1[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
          const int j = lane + 32 * q;
          u0[q] = j < P.N ? b0[j] : T(0);
          u1[q] = (bit1 >= 0 && j < P.N) ? b1[j] : T(0);
        }
#pragma unroll
        for (int q = 0; q < NQ; q++) acc[q] = fma_t(a0, u0[q], acc[q]);
        if (bit1 >= 0) {
#pragma unroll
          for (int q = 0; q < NQ; q++) acc[q] = fma_t(a1, u1[q], acc[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; q++) {
      const int j = lane + 32 * q;
      if (j < P.N) store_out(P, b, gm, j, acc[q]);
    }
  }
}

// The union nonzero pattern of two n x n matrices (X1 may be null) by rows:
// a warp per row writes the row's column indices, increasing, at
// cols[r n ..] (ballots over 32 columns at a time), rowbeg[r] = r n,
// rowend[r] = r n + its count, and adds the count to *total.
__global__ void __launch_bounds__(256) csr_rows_kernel(int n, const double* __restrict__ X0,
                                                       const double* __restrict__ X1, int* __restrict__ rowbeg,
                                                       int* __restrict__ rowend, int* __restrict__ cols,
                                                       unsigned long long* __restrict__ total) {
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int r = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (r >= n) return;
  const long long base = (long long)r * n;
  int pos = 0;
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int k = k0 + lane;
    const bool z = k < n && (X0[base + k] != 0.0 || (X1 != nullptr && X1[base + k] != 0.0));
    const unsigned m = __ballot_sync(kFull, z);
    if (z) cols[base + pos + __popc(m & ((1u << lane) - 1u))] = k;
    pos += __popc(m);
  }
  if (lane == 0) {
    rowbeg[r] = (int)base;
    rowend[r] = (int)base + pos;
    atomicAdd(total, (unsigned long long)pos);
  }
}

// flag[0 .. S) = 1 when the pattern has at most max_nnz entries, else 0
__global__ void csr_flags_kernel(const unsigned long long* __restrict__ total, long long max_nnz, int S,
                                 int* __restrict__ flag) {
  const int ok = *total <= (unsigned long long)max_nnz ? 1 : 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) flag[s] = ok;
}

// Counts of nonzero entries per matrix, one CTA per matrix, then the flag.
template <typename T>
__global__ void __launch_bounds__(256) sparse_flags_kernel(int n, int S, const T* __restrict__ M, long long max_nnz,
                                                          int* __restrict__ flag) {
  __shared__ int part[8];
  const long long nn = (long long)n * n;
  for (int s = blockIdx.x; s < S; s += gridDim.x) {
    int c = 0;
    for (long long e = threadIdx.x; e < nn; e += blockDim.x) c += M[s * nn + e] != T(0);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += part[w];
      flag[s] = tot <= max_nnz ? 1 : 0;
    }
    __syncthreads();
  }
}

template <typename T, int BM, int BN, int TM, int TN, bool DB>
cudaError_t launch_rcfg(const RGemmProblem<T>* probs, int nprob, int sm_count, cudaStream_t st) {
  RGroup<T> g;
  g.nprob = nprob;
  long long acc = 0;
  for (int i = 0; i < nprob; i++) {
    g.p[i] = probs[i];
    g.tiles_m[i] = (probs[i].M + BM - 1) / BM;
    g.tiles_n[i] = (probs[i].N + BN - 1) / BN;
    g.tile_start[i] = acc;
    if (probs[i].M > 0 && probs[i].N > 0 && probs[i].batch > 0)
      acc += (long long)g.tiles_m[i] * g.tiles_n[i] * probs[i].batch;
    else
      g.tiles_m[i] = g.tiles_n[i] = 1;  // empty problem: zero tiles
  }
  for (int i = nprob; i <= 4; i++) g.tile_start[i] = acc;
  if (acc == 0) return cudaSuccess;
  constexpr int NT = (BM / TM) * (BN / TN);
  static int occ = -1;  // resident CTAs per SM for this configuration
  if (occ < 0) {
    int o = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, rgemm_kernel<T, BM, BN, TM, TN, DB>, NT, 0);
    if (e != cudaSuccess) return e;
    occ = std::max(1, o);
  }
  const long long grid = std::min<long long>(acc, (long long)sm_count * occ);
  count_launch();
  rgemm_kernel<T, BM, BN, TM, TN, DB><<<(unsigned)grid, NT, 0, st>>>(g);
  return cudaGetLastError();
}

template <typename T>
double rpad(const RGemmProblem<T>* probs, int nprob, int BM, int BN) {
  double padded = 0.0, real = 0.0;
  for (int i = 0; i < nprob; i++) {
    if (probs[i].M <= 0 || probs[i].N <= 0) continue;
    padded += (double)((probs[i].M + BM - 1) / BM * BM) * ((probs[i].N + BN - 1) / BN * BN) * probs[i].batch;
    real += (double)probs[i].M * probs[i].N * probs[i].batch;
  }
  return real > 0.0 ? padded / real : 1.0;
}

template <typename T>
long long rtiles(const RGemmProblem<T>* probs, int nprob, int BM, int BN) {
  long long acc = 0;
  for (int i = 0; i < nprob; i++)
    if (probs[i].M > 0 && probs[i].N > 0)
      acc += (long long)((probs[i].M + BM - 1) / BM) * ((probs[i].N + BN - 1) / BN) * probs[i].batch;
  return acc;
}

template <typename T>
TuneKey rshape_key(const RGemmProblem<T>* p, int np) {
  TuneKey k{};
  k[0] = 2;  // family: real GEMM
  k[1] = sizeof(T) * 8;
  k[2] = np;
  for (int i = 0; i < np && i < 4; i++) {
    k[3 + 5 * i] = p[i].M;
    k[4 + 5 * i] = p[i].N;
    k[5 + 5 * i] = p[i].K;
    k[6 + 5 * i] = p[i].batch;
    k[7 + 5 * i] = p[i].transB * 4 + (p[i].beta[0] != 0.0 ? 2 : 0) + (p[i].active != nullptr ? 1 : 0);
  }
  return k;
}

template <typename T>
struct RArgs {
  cudaError_t (*const* cands)(const RGemmProblem<T>*, int, int, cudaStream_t);
  const RGemmProblem<T>* probs;
  int nprob, sm_count;
};

template <typename T>
cudaError_t rrun(int cand, const void* a, cudaStream_t st) {
  const RArgs<T>* r = (const RArgs<T>*)a;
  return r->cands[cand](r->probs, r->nprob, r->sm_count, st);
}

}  // namespace

cudaError_t rgemm_f64(const RGemmProblem<double>* probs, int nprob, int sm_count, cudaStream_t st) {
  if (nprob <= 0 || nprob > 4) return cudaErrorInvalidValue;
  typedef cudaError_t (*fn)(const RGemmProblem<double>*, int, int, cudaStream_t);
  static const fn cands[5] = {launch_rcfg<double, 16, 16, 1, 1, false>, launch_rcfg<double, 32, 32, 2, 2, true>,
                              launch_rcfg<double, 64, 64, 4, 4, true>, launch_rcfg<double, 16, 16, 1, 1, true>,
                              launch_rcfg<double, 32, 32, 2, 2, false>};
  // 32 x 32 tiles (two stages) when there are enough of them to balance the
  // persistent grid, else 16 x 16 (one stage, more resident CTAs)
  const long long t32 = rtiles(probs, nprob, 32, 32);
  const bool big = t32 >= 8LL * sm_count && rpad(probs, nprob, 32, 32) <= 1.25 * rpad(probs, nprob, 16, 16);
  const RArgs<double> a{cands, probs, nprob, sm_count};
  return tuned_launch(rshape_key(probs, nprob), 5, big ? 1 : 0, rrun<double>, &a, st);
}

cudaError_t rgemm_f32(const RGemmProblem<float>* probs, int nprob, int sm_count, cudaStream_t st) {
  if (nprob <= 0 || nprob > 4) return cudaErrorInvalidValue;
  typedef cudaError_t (*fn)(const RGemmProblem<float>*, int, int, cudaStream_t);
  static const fn cands[2] = {launch_rcfg<float, 32, 32, 2, 2, true>, launch_rcfg<float, 64, 64, 4, 4, true>};
  const long long t64 = rtiles(probs, nprob, 64, 64);
  const bool big = t64 >= 2LL * sm_count && rpad(probs, nprob, 64, 64) <= 1.25 * rpad(probs, nprob, 32, 32);
  const RArgs<float> a{cands, probs, nprob, sm_count};
  return tuned_launch(rshape_key(probs, nprob), 2, big ? 1 : 0, rrun<float>, &a, st);
}

template <typename T, int NQ>
cudaError_t launch_rowskip(const RGemmProblem<T>& p, int sm_count, cudaStream_t st) {
  static int occ = -1;
  if (occ < 0) {
    int o = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, rgemm_rowskip_kernel<T, NQ>, 256, 0);
    if (e != cudaSuccess) return e;
    occ = std::max(1, o);
  }
  const long long warps = (long long)p.batch * p.M;
  const long long grid = std::min<long long>((warps + 7) / 8, (long long)sm_count * occ);
  count_launch();
  rgemm_rowskip_kernel<T, NQ><<<(unsigned)grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t rgemm_rowskip(const RGemmProblem<T>& p, int sm_count, cudaStream_t st) {
  if (p.transB != 0 || p.shiftB != 0.0 || p.N > 736 || p.N < 1) return cudaErrorInvalidValue;
  if (p.M < 1 || p.batch < 1) return cudaSuccess;
  if (p.N <= 128) return launch_rowskip<T, 4>(p, sm_count, st);
  if (p.N <= 256) return launch_rowskip<T, 8>(p, sm_count, st);
  return launch_rowskip<T, 23>(p, sm_count, st);
}
template <typename T, int NQ>
cudaError_t launch_csr(const RGemmProblem<T>& p, const int* rowbeg, const int* rowend, const int* cols, int sm_count,
                       cudaStream_t st) {
  static int occ = -1;
  if (occ < 0) {
    int o = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, rgemm_csr_kernel<T, NQ>, 256, 0);
    if (e != cudaSuccess) return e;
    occ = std::max(1, o);
  }
  const long long warps = (long long)p.batch * p.M;
  const long long grid = std::min<long long>((warps + 7) / 8, (long long)sm_count * occ);
  count_launch();
  rgemm_csr_kernel<T, NQ><<<(unsigned)grid, 256, 0, st>>>(p, rowbeg, rowend, cols);
  return cudaGetLastError();
}

template <typename T>
cudaError_t rgemm_csr(const RGemmProblem<T>& p, const int* rowbeg, const int* rowend, const int* cols, int sm_count,
                      cudaStream_t st) {
  if (p.transB != 0 || p.shiftA != 0.0 || p.shiftB != 0.0 || p.N > 736 || p.N < 1) return cudaErrorInvalidValue;
  if (p.M < 1 || p.batch < 1) return cudaSuccess;
  if (p.N <= 128) return launch_csr<T, 4>(p, rowbeg, rowend, cols, sm_count, st);
  if (p.N <= 256) return launch_csr<T, 8>(p, rowbeg, rowend, cols, sm_count, st);
  return launch_csr<T, 23>(p, rowbeg, rowend, cols, sm_count, st);
}
template cudaError_t rgemm_csr<double>(const RGemmProblem<double>&, const int*, const int*, const int*, int,
                                       cudaStream_t);

cudaError_t launch_csr_union(int n, const double* X0, const double* X1, long long max_nnz, int S, CsrPattern pat,
                             int* flag, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(pat.total, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  count_launch();
  csr_rows_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(n, X0, X1, pat.rowbeg, pat.rowend, pat.cols, pat.total);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  csr_flags_kernel<<<1, 256, 0, st>>>(pat.total, max_nnz, S, flag);
  return cudaGetLastError();
}

template cudaError_t rgemm_rowskip<double>(const RGemmProblem<double>&, int, cudaStream_t);
template cudaError_t rgemm_rowskip<float>(const RGemmProblem<float>&, int, cudaStream_t);

template <typename T>
cudaError_t launch_sparse_flags(int n, int S, const T* M, long long max_nnz, int* flag, int sm_count,
                                cudaStream_t st) {
  const int grid = std::min(S, sm_count * 8);
  if (grid < 1) return cudaSuccess;
  count_launch();
  sparse_flags_kernel<T><<<grid, 256, 0, st>>>(n, S, M, max_nnz, flag);
  return cudaGetLastError();
}
template cudaError_t launch_sparse_flags<double>(int, int, const double*, long long, int*, int, cudaStream_t);
template cudaError_t launch_sparse_flags<float>(int, int, const float*, long long, int*, int, cudaStream_t);

}  // namespace lb
