// Grouped, batched complex GEMM on the CUDA cores.
//
// Every dense complex product of the propagator build (Algorithm 1: the three
// power products, the three U/V products, the LU panel and trailing updates,
// the back substitution and the squarings) and the large-n FP64 propagation
// step (Algorithm 2 batched over states) goes through this kernel.
//
// FP64 form: on GB300 FP64 runs at 1/64 of the FP32 rate, so the kernel is
// bound by the FP64 pipe and the design goal is the fewest FP64 instructions
// with every SM busy.  It uses Gauss's three-real-product form of the complex
// product, C_re = A_re B_re - A_im B_im and
// C_im = (A_re + A_im)(B_re + B_im) - A_re B_re - A_im B_im, with the operand
// sums formed once per shared-memory tile: 3 DFMA per complex multiply-add
// instead of 4.  Work is a flat list of output tiles over all problems and
// batch elements, walked by a persistent grid of (SMs x resident CTAs), so
// 200-slice batches and ragged LU updates balance across the 152 SMs.
//
// FP32 form (mixed-precision Pade products): the same tiling with FP32
// operands and FP32 accumulation, four real products per complex
// multiply-add and larger register tiles; the epilogue (the linear
// combinations of the Pade step) stays FP64.
#include "lb_internal.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

namespace lb {

namespace {

struct GroupArgs {
  ZGemmProblem p[4];
  long long tile_start[5];
  int tiles_m[4];
  int tiles_n[4];
  int nprob;
};

template <typename T>
__device__ __forceinline__ T fmaT(T a, T b, T c);
template <>
__device__ __forceinline__ double fmaT<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fmaT<float>(float a, float b, float c) { return fmaf(a, b, c); }

// NPL = number of operand planes kept in shared memory (3 for Gauss, 2 otherwise).
template <typename T, int BM, int BN, int TM, int TN, bool GAUSS>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    zgemm_kernel(const __grid_constant__ GroupArgs g) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int BK = 16;
  constexpr int NPL = GAUSS ? 3 : 2;
  __shared__ __align__(16) T As[NPL][BK][BM];
  __shared__ __align__(16) T Bs[NPL][BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN);
  const int ty = tid / (BN / TN);
  const long long total = g.tile_start[g.nprob];

  for (long long t = blockIdx.x; t < total; t += gridDim.x) {
    int pi = 0;
    while (pi + 1 < g.nprob && t >= g.tile_start[pi + 1]) pi++;
    const ZGemmProblem& P = g.p[pi];
    const long long lt = t - g.tile_start[pi];
    const int tpb = g.tiles_m[pi] * g.tiles_n[pi];
    const long long b = lt / tpb;
    const int r = (int)(lt - b * tpb);
    const int tm = r / g.tiles_n[pi];
    const int tn = r - tm * g.tiles_n[pi];
    if (P.active != nullptr && P.active[b] <= P.active_iter) continue;
    if (P.active_lo != nullptr && P.active_lo[b] > P.active_iter) continue;
    const int m0 = tm * BM, n0 = tn * BN;
    const z64* __restrict__ A = P.A + b * P.sA;
    const z64* __restrict__ B = P.B + b * P.sB;
    const int M = P.M, N = P.N, K = P.K;

    // C +- A B with nothing else in the epilogue (the LU updates): start the
    // Gauss accumulators from C and fold the sign into A, so the epilogue is
    // the plain recombination (fewer FP64 instructions on a 1/64-rate pipe).
    const bool fastC = GAUSS && P.beta == 1.0 && (P.alpha == 1.0 || P.alpha == -1.0) && P.nterms == 0 &&
                       P.C2 == nullptr && P.gamma == 0.0;
    T acc1[TM][TN], acc2[TM][TN], acc3[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; i++)
#pragma unroll
      for (int j = 0; j < TN; j++) {
        acc1[i][j] = T(0);
        acc2[i][j] = T(0);
        acc3[i][j] = T(0);
        if (fastC) {
          const int gm = m0 + ty * TM + i, gn = n0 + tx * TN + j;
          if (gm < M && gn < N) {
            const z64 c0 = P.C[b * P.sC + (long long)gm * P.ldc + gn];
            acc1[i][j] = T(c0.x);
            acc3[i][j] = T(c0.x + c0.y);
          }
        }
      }

    // signs applied by flipping the sign bit (integer work, no FP64 multiply)
    const unsigned long long SGN = 0x8000000000000000ull;
    const bool bT = (P.opB & 1) != 0;
    const unsigned long long bneg_im = (P.opB & 2) ? SGN : 0ull;
    const unsigned long long aneg_re = (fastC && P.alpha < 0.0) ? SGN : 0ull;
    const unsigned long long aneg_im = aneg_re ^ (P.conjA ? SGN : 0ull);

    for (int k0 = 0; k0 < K; k0 += BK) {
      // A tile (BM x BK), k contiguous in memory.
      for (int e = tid; e < BM * BK; e += NT) {
        const int m = e / BK, k = e - (e / BK) * BK;
        const int gm = m0 + m, gk = k0 + k;
        z64 v = make_double2(0.0, 0.0);
        if (gm < M && gk < K) {
          v = A[(long long)gm * P.lda + gk];
          if (gm == gk) v.x -= P.shiftA;
        }
        const T re = T(__longlong_as_double(__double_as_longlong(v.x) ^ aneg_re));
        const T im = T(__longlong_as_double(__double_as_longlong(v.y) ^ aneg_im));
        As[0][k][m] = re;
        As[1][k][m] = im;
        if (GAUSS) As[NPL - 1][k][m] = re + im;
      }
      // B tile (BK x BN).
      if (!bT) {
        for (int e = tid; e < BK * BN; e += NT) {
          const int k = e / BN, nn = e - (e / BN) * BN;
          const int gk = k0 + k, gn = n0 + nn;
          z64 v = make_double2(0.0, 0.0);
          if (gk < K && gn < N) {
            v = B[(long long)gk * P.ldb + gn];
            if (gk == gn) v.x -= P.shiftB;
          }
          const T re = T(v.x), im = T(__longlong_as_double(__double_as_longlong(v.y) ^ bneg_im));
          Bs[0][k][nn] = re;
          Bs[1][k][nn] = im;
          if (GAUSS) Bs[NPL - 1][k][nn] = re + im;
        }
      } else {
        for (int e = tid; e < BK * BN; e += NT) {
          const int nn = e / BK, k = e - (e / BK) * BK;
          const int gk = k0 + k, gn = n0 + nn;
          z64 v = make_double2(0.0, 0.0);
          if (gk < K && gn < N) {
            v = B[(long long)gn * P.ldb + gk];
            if (gk == gn) v.x -= P.shiftB;
          }
          const T re = T(v.x), im = T(__longlong_as_double(__double_as_longlong(v.y) ^ bneg_im));
          Bs[0][k][nn] = re;
          Bs[1][k][nn] = im;
          if (GAUSS) Bs[NPL - 1][k][nn] = re + im;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BK; k++) {
        T ar[TM], ai[TM], br[TN], bi[TN];
#pragma unroll
        for (int i = 0; i < TM; i++) {
          ar[i] = As[0][k][ty * TM + i];
          ai[i] = As[1][k][ty * TM + i];
        }
#pragma unroll
        for (int j = 0; j < TN; j++) {
          br[j] = Bs[0][k][tx * TN + j];
          bi[j] = Bs[1][k][tx * TN + j];
        }
        if (GAUSS) {
          T as[TM], bs[TN];
#pragma unroll
          for (int i = 0; i < TM; i++) as[i] = As[NPL - 1][k][ty * TM + i];
#pragma unroll
          for (int j = 0; j < TN; j++) bs[j] = Bs[NPL - 1][k][tx * TN + j];
#pragma unroll
          for (int i = 0; i < TM; i++)
#pragma unroll
            for (int j = 0; j < TN; j++) {
              acc1[i][j] = fmaT(ar[i], br[j], acc1[i][j]);
              acc2[i][j] = fmaT(ai[i], bi[j], acc2[i][j]);
              acc3[i][j] = fmaT(as[i], bs[j], acc3[i][j]);
            }
        } else {
          // acc1 = re, acc2 = im
#pragma unroll
          for (int i = 0; i < TM; i++)
#pragma unroll
            for (int j = 0; j < TN; j++) {
              acc1[i][j] = fmaT(ar[i], br[j], acc1[i][j]);
              acc1[i][j] = fmaT(-ai[i], bi[j], acc1[i][j]);
              acc2[i][j] = fmaT(ar[i], bi[j], acc2[i][j]);
              acc2[i][j] = fmaT(ai[i], br[j], acc2[i][j]);
            }
        }
      }
      __syncthreads();
    }

    // Epilogue in FP64.
#pragma unroll
    for (int i = 0; i < TM; i++) {
      const int gm = m0 + ty * TM + i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; j++) {
        const int gn = n0 + tx * TN + j;
        if (gn >= N) continue;
        double pre, pim;
        if (GAUSS) {
          pre = double(acc1[i][j]) - double(acc2[i][j]);
          pim = double(acc3[i][j]) - double(acc1[i][j]) - double(acc2[i][j]);
        } else {
          pre = double(acc1[i][j]);
          pim = double(acc2[i][j]);
        }
        const long long off = (long long)gm * P.ldc + gn;
        const long long idx = b * P.sC + off;
        if (fastC) {  // C was folded into the accumulators
          P.C[idx] = make_double2(pre, pim);
          continue;
        }
        double cr = P.alpha * pre, ci = P.alpha * pim;
        if (P.beta != 0.0) {
          const z64 c0 = P.C[idx];
          cr = fma(P.beta, c0.x, cr);
          ci = fma(P.beta, c0.y, ci);
        }
        for (int q = 0; q < P.nterms; q++) {
          const z64 x = P.X[q][b * P.sX[q] + off];
          cr = fma(P.coef[q], x.x, cr);
          ci = fma(P.coef[q], x.y, ci);
        }
        if (gm == gn) cr += P.gamma;
        P.C[idx] = make_double2(cr, ci);
        if (P.C2 != nullptr) {
          const z64 x2 = P.X2[b * P.sX2 + off];
          P.C2[idx] = make_double2(fma(P.alpha2, pre, x2.x), fma(P.alpha2, pim, x2.y));
        }
      }
    }
  }
}

template <typename T, int BM, int BN, int TM, int TN, bool GAUSS>
cudaError_t launch_cfg(const ZGemmProblem* probs, int nprob, int sm_count, cudaStream_t st) {
  GroupArgs g;
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
  g.tile_start[nprob] = acc;
  for (int i = nprob; i < 4; i++) g.tile_start[i + 1 > 4 ? 4 : i + 1] = acc;
  if (acc == 0) return cudaSuccess;
  constexpr int NT = (BM / TM) * (BN / TN);
  static int occ = -1;  // resident CTAs per SM for this configuration
  if (occ < 0) {
    int o = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &o, zgemm_kernel<T, BM, BN, TM, TN, GAUSS>, NT, 0);
    if (e != cudaSuccess) return e;
    occ = std::max(1, o);
  }
  long long grid = std::min<long long>(acc, (long long)sm_count * occ);
  count_launch();
  zgemm_kernel<T, BM, BN, TM, TN, GAUSS><<<(unsigned)grid, NT, 0, st>>>(g);
  return cudaGetLastError();
}

// Padded output area of BM x BN tiles over the problems' real output area:
// large tiles on small matrices (9 x 9, 81 x 81) compute mostly zeros.
double pad_ratio(const ZGemmProblem* probs, int nprob, int BM, int BN) {
  double padded = 0.0, real = 0.0;
  for (int i = 0; i < nprob; i++) {
    if (probs[i].M <= 0 || probs[i].N <= 0) continue;
    padded += (double)((probs[i].M + BM - 1) / BM * BM) * ((probs[i].N + BN - 1) / BN * BN) * probs[i].batch;
    real += (double)probs[i].M * probs[i].N * probs[i].batch;
  }
  return real > 0.0 ? padded / real : 1.0;
}

long long count_tiles(const ZGemmProblem* probs, int nprob, int BM, int BN) {
  long long acc = 0;
  for (int i = 0; i < nprob; i++)
    if (probs[i].M > 0 && probs[i].N > 0)
      acc += (long long)((probs[i].M + BM - 1) / BM) * ((probs[i].N + BN - 1) / BN) * probs[i].batch;
  return acc;
}

}  // namespace

namespace {

// ------------------------------------------------------------ autotuner --
// A launch "shape" is the GEMM family, its precision, the number of problems
// and each problem's (M, N, K, batch, opB, beta).  In tuning mode (set for
// the calling host thread only, by lb_autotune) every launch times each
// candidate tile configuration (one untimed and three timed runs, CUDA
// events, host wait) and records the fastest for its shape; afterwards launches of a recorded shape use it, and
// other shapes use the caller's tile-count heuristic.
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
thread_local bool t_tuning = false;

// Both events of a timing pair, destroyed on every exit path.
struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok() {
    return cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  }
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

}  // namespace

cudaError_t tuned_launch(const TuneKey& key, int ncand, int heuristic, TuneCand run, const void* args,
                         cudaStream_t st) {
  int choice = heuristic;
  if (!t_tuning) {
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) choice = it->second;
    }
    return run(choice, args, st);
  }
  EventPair ev;
  if (!ev.ok()) return cudaErrorUnknown;
  float best = 1e30f;
  int besti = heuristic;
  for (int c = 0; c < ncand; c++) {
    cudaError_t e = run(c, args, st);  // warm-up
    if (e != cudaSuccess) return e;
    for (int rep = 0; rep < 3; rep++) {  // the fastest of three timed runs
      if (cudaEventRecord(ev.e0, st) != cudaSuccess) return cudaErrorUnknown;
      e = run(c, args, st);
      if (e != cudaSuccess) return e;
      if (cudaEventRecord(ev.e1, st) != cudaSuccess || cudaEventSynchronize(ev.e1) != cudaSuccess)
        return cudaErrorUnknown;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev.e0, ev.e1);
      if (ms < best) {
        best = ms;
        besti = c;
      }
    }
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = besti;
  return cudaSuccess;
}

void set_tuning(bool on) { t_tuning = on; }

int tuned_shapes() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)g_tune.size();
}

namespace {

TuneKey zshape_key(int prec, const ZGemmProblem* p, int np) {
  TuneKey k{};
  k[0] = 1;  // family: complex GEMM
  k[1] = prec;
  k[2] = np;
  for (int i = 0; i < np && i < 4; i++) {
    k[3 + 5 * i] = p[i].M;
    k[4 + 5 * i] = p[i].N;
    k[5 + 5 * i] = p[i].K;
    k[6 + 5 * i] = p[i].batch;
    k[7 + 5 * i] = p[i].opB * 4 + (p[i].beta != 0.0 ? 2 : 0) + (p[i].active != nullptr ? 1 : 0);
  }
  return k;
}

typedef cudaError_t (*cfg_fn)(const ZGemmProblem*, int, int, cudaStream_t);

struct ZArgs {
  const cfg_fn* cands;
  const ZGemmProblem* probs;
  int nprob, sm_count;
};

cudaError_t zrun(int cand, const void* a, cudaStream_t st) {
  const ZArgs* z = (const ZArgs*)a;
  return z->cands[cand](z->probs, z->nprob, z->sm_count, st);
}

}  // namespace

cudaError_t zgemm_f64(const ZGemmProblem* probs, int nprob, int sm_count, cudaStream_t st) {
  if (nprob <= 0 || nprob > 4) return cudaErrorInvalidValue;
  static const cfg_fn cands[3] = {launch_cfg<double, 16, 16, 1, 1, true>, launch_cfg<double, 32, 32, 2, 2, true>,
                                  launch_cfg<double, 64, 64, 4, 4, true>};
  // heuristic: 32x32 tiles when there are enough of them to balance the
  // persistent grid and they pad little more than 16x16 tiles, else 16x16
  const long long t32 = count_tiles(probs, nprob, 32, 32);
  const bool big = t32 >= 8LL * sm_count &&
                   pad_ratio(probs, nprob, 32, 32) <= 1.25 * pad_ratio(probs, nprob, 16, 16);
  const ZArgs a{cands, probs, nprob, sm_count};
  return tuned_launch(zshape_key(64, probs, nprob), 3, big ? 1 : 0, zrun, &a, st);
}

cudaError_t zgemm_f32(const ZGemmProblem* probs, int nprob, int sm_count, cudaStream_t st) {
  if (nprob <= 0 || nprob > 4) return cudaErrorInvalidValue;
  static const cfg_fn cands[2] = {launch_cfg<float, 32, 32, 2, 2, false>, launch_cfg<float, 64, 64, 4, 4, false>};
  const long long t64 = count_tiles(probs, nprob, 64, 64);
  const bool big = t64 >= 4LL * sm_count &&
                   pad_ratio(probs, nprob, 64, 64) <= 1.25 * pad_ratio(probs, nprob, 32, 32);
  const ZArgs a{cands, probs, nprob, sm_count};
  return tuned_launch(zshape_key(32, probs, nprob), 2, big ? 1 : 0, zrun, &a, st);
}

}  // namespace lb
