// FP64 matrix products on the BF16 tensor cores through exact slices (the
// Ozaki scheme: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Row r of the left operand A (M x K) is written in fixed point against its
// own exponent e_r (every |A[r][k]| < 2^e_r) as signed base-2^BETA digits,
//   A[r][k] = 2^e_r ( sum_{i=1..NS} a_i[r][k] 2^(-i BETA) + rho ),
//   |a_1| <= 2^BETA, |a_i| <= 2^(BETA-1) (i >= 2), |rho| <= 2^(-NS BETA - 1),
// and column c of B (K x N) likewise against f_c with digits b_j.  Every
// digit is an integer of at most seven significant bits, exact in BF16, and
// every digit product is exact in FP32.  The digit products of one "group"
// g = i + j share the unit 2^(-g BETA), so
//   G_g[r][c] = sum_{i+j=g} sum_k a_i[r][k] b_j[k][c]
// is an integer; with BETA = 6 every partial sum stays below 2^24 in
// magnitude for K <= kOzMaxK, so the tensor cores' FP32 accumulation of a
// group is exact whatever the order.  The product is
//   (A B)[r][c] = 2^(e_r + f_c) sum_{g=2..NS+1} G_g[r][c] 2^(-g BETA) + err,
// where err (the pairs with i + j > NS + 1 and the residuals rho) is below
// K 2^(e_r + f_c) 2^(-NS BETA) (1 + NS / 4).  With NS = 9 (54 bits) that is
// the size of the FP64 product's own rounding bound, K 2^-53 |A| |B|, for
// rows and columns whose entries are of one magnitude.  The group sums are
// combined in exact integer arithmetic and rounded to FP64 once.
//
// Data path (one CTA per 128 x OZ_BN output tile and batch element):
//  * an operand's digits ("slices") sit in a tile-blocked layout: for each
//    batch element, tile of rows (128 for A, OZ_BN of B's columns for B) and
//    16-wide block of K, the NS digit planes follow each other, each plane
//    in 8 x 8 core matrices (8 rows x 16 bytes) ordered row group, then K
//    half: one block of a stage is one contiguous run of bytes, copied with
//    one plain bulk copy, and lands in shared memory in the tensor cores'
//    no-swizzle K-major layout.  Padding rows and K are zero digits.
//  * warp 0 copies the A and B blocks of a K block into a four-stage ring;
//  * one thread of warp 1 issues, per K block and digit i of A, MMAs of A_i
//    against the stacked planes B_1 .. B_{NS+1-i} (N = (NS+1-i) OZ_BN, at
//    most 240 per instruction) into the TMEM columns of the groups
//    i+1 .. NS+1: the accumulator is NS groups x OZ_BN columns of FP32;
//  * all eight warps read the groups out of TMEM (warp w: lanes 32 (w % 4),
//    column chunks of half w / 4), combine them and write FP64
//    C = alpha (A B) + beta C.
// Every mbarrier wait is bounded; a wait that gives up sets the error word,
// the CTA waits (bounded) for its copies in flight and frees its TMEM.
#include "lb_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace lb {

namespace {

constexpr int OZ_BETA = 6;
constexpr int OZ_TBM = 128;       // rows per A tile (M of one MMA)
constexpr int OZ_KB = 16;         // K per block and stage (one MMA K step)
constexpr int OZ_NSTAGE = 4;
constexpr int OZ_THREADS = 256;
constexpr int OZ_ZERO_EXP = -2000;  // exponent of an all-zero row
constexpr long long kOzWaitCycles = 4000000000LL;

template <int NS, int BN>
struct OzCfg {
  static constexpr int A_BYTES = NS * OZ_TBM * OZ_KB * 2;  // one K block of all A planes
  static constexpr int B_BYTES = NS * BN * OZ_KB * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int SMEM = OZ_NSTAGE * STAGE + 1024;
  static constexpr int TCOLS = NS * BN;
  static constexpr int TALLOC = TCOLS <= 32 ? 32 : TCOLS <= 64 ? 64 : TCOLS <= 128 ? 128 : TCOLS <= 256 ? 256 : 512;
  static constexpr int NMAX = (256 / BN) * BN;  // rows of stacked B per MMA (a multiple of BN)
  static_assert(TCOLS <= 512, "TMEM columns");
  static_assert(SMEM <= 232448, "shared memory");
  static_assert(BN % 16 == 0 && NMAX % 16 == 0, "MMA N");
  static_assert(STAGE % 128 == 0 && A_BYTES % 128 == 0, "copy alignment");
};

__device__ __forceinline__ uint32_t oz_su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool oz_try(uint32_t bar, uint32_t ph) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(ph)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t ph) {
  if (oz_try(bar, ph)) return true;
  const long long t0 = clock64();
  while (!oz_try(bar, ph))
    if (clock64() - t0 > kOzWaitCycles) return false;
  return true;
}

// shared-memory matrix descriptor, K-major without swizzle: core matrices of
// 8 rows x 16 bytes, the two K halves of a block 128 bytes apart (leading
// offset), 8-row groups 256 bytes apart (stride offset); Blackwell version
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M = 128
__host__ __device__ constexpr uint32_t oz_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(OZ_TBM >> 4) << 24);
}

__device__ __forceinline__ void oz_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void oz_bulk(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void oz_ld8(uint32_t ta, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

// 2^s as a double for s in [-1022, 1023]; 0 below
__device__ __forceinline__ double oz_pow2(int s) {
  if (s < -1022) return 0.0;
  return __longlong_as_double((long long)(s + 1023) << 52);
}

// (hi 2^30 + lo) 2^e rounded to the nearest double (ties to even), for
// |hi| < 2^44, |lo| < 2^50, in integer arithmetic only (the FP64 pipe is
// slow on this part); *ok = false where the result would leave the normal
// range (the caller then takes the FP64 route).
__device__ __forceinline__ double oz_round(long long hi, long long lo, int e, bool* ok) {
  const __int128 T = (__int128)hi * ((__int128)1 << 30) + (__int128)lo;
  const bool neg = T < 0;
  const unsigned __int128 U = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
  const unsigned long long uh = (unsigned long long)(U >> 64), ul = (unsigned long long)U;
  *ok = true;
  if ((uh | ul) == 0ull) return 0.0;
  const int p = uh != 0ull ? 127 - __clzll((long long)uh) : 63 - __clzll((long long)ul);  // leading bit
  unsigned long long mant;
  int E = p + e;
  if (p <= 52) {
    mant = ul << (52 - p);
  } else {
    const int sh = p - 52;  // 1 .. 75
    const unsigned __int128 m = U >> sh;
    const unsigned __int128 rem = U - (m << sh);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    mant = (unsigned long long)m;
    if (rem > half || (rem == half && (mant & 1ull))) {
      mant++;
      if (mant == (1ull << 53)) {
        mant >>= 1;
        E++;
      }
    }
  }
  if (E < -1022 || E > 1023) {
    *ok = false;
    return 0.0;
  }
  const unsigned long long bits =
      ((unsigned long long)neg << 63) | ((unsigned long long)(E + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

template <int NS, int BN>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    ozgemm_kernel(const __grid_constant__ OzGemm P, const __nv_bfloat16* __restrict__ QA,
                  const __nv_bfloat16* __restrict__ QB, int kblocks) {
  using Cfg = OzCfg<NS, BN>;
  const int b = blockIdx.z;
  if (P.active != nullptr && P.active[b] <= P.active_iter) return;  // whole CTA, before any setup
  extern __shared__ __align__(1024) uint8_t oz_smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[OZ_NSTAGE], empty_bar[OZ_NSTAGE], acc_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int give_up;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * OZ_TBM;
  const int nk = kblocks;
  // this CTA's K blocks of A (tile blockIdx.y) and of B (tile blockIdx.x)
  const uint8_t* srcA =
      (const uint8_t*)QA + ((long long)b * gridDim.y + blockIdx.y) * (long long)kblocks * Cfg::A_BYTES;
  const uint8_t* srcB =
      (const uint8_t*)QB + ((long long)b * gridDim.x + blockIdx.x) * (long long)kblocks * Cfg::B_BYTES;

  if (tid == 0) {
    for (int s = 0; s < OZ_NSTAGE; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(&empty_bar[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(&acc_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    give_up = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(oz_su32(&tmem_base)),
                 "r"(Cfg::TALLOC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tacc = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer: the A and B blocks of each K block, one bulk copy each
    for (int kb = 0; kb < nk; kb++) {
      const int s = kb % OZ_NSTAGE;
      if (kb >= OZ_NSTAGE && !oz_wait(oz_su32(&empty_bar[s]), ((kb - OZ_NSTAGE) / OZ_NSTAGE) & 1)) {
        atomicOr(P.err, ERR_TIMEOUT);
        give_up = 1;
        break;
      }
      const uint32_t base = oz_su32(sm + s * Cfg::STAGE);
      const uint32_t fb = oz_su32(&full_bar[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(Cfg::STAGE) : "memory");
      oz_bulk(base, srcA + (long long)kb * Cfg::A_BYTES, Cfg::A_BYTES, fb);
      oz_bulk(base + Cfg::A_BYTES, srcB + (long long)kb * Cfg::B_BYTES, Cfg::B_BYTES, fb);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: digit i of A (0-based) against B digits 0 .. NS-1-i into
    // group columns [i BN, NS BN)
    bool ok = true;
    for (int kb = 0; kb < nk; kb++) {
      const int s = kb % OZ_NSTAGE;
      if (!oz_wait(oz_su32(&full_bar[s]), (kb / OZ_NSTAGE) & 1)) {
        atomicOr(P.err, ERR_TIMEOUT);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t abase = oz_su32(sm + s * Cfg::STAGE);
      const uint32_t bbase = abase + Cfg::A_BYTES;
#pragma unroll
      for (int i = 0; i < NS; i++) {
        const uint64_t ad = oz_desc(abase + i * (OZ_TBM * OZ_KB * 2));
        const int rows = (NS - i) * BN;  // stacked B rows of digits 0 .. NS-1-i
#pragma unroll
        for (int r0 = 0; r0 < rows; r0 += Cfg::NMAX) {
          const int nr = rows - r0 < Cfg::NMAX ? rows - r0 : Cfg::NMAX;
          const uint32_t acc = (kb > 0 || i > 0) ? 1u : 0u;
          oz_mma(tacc + i * BN + r0, ad, oz_desc(bbase + r0 * (OZ_KB * 2)), oz_idesc(nr), acc);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       oz_su32(&empty_bar[s]))
                   : "memory");
    }
    if (!ok) give_up = 1;
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     oz_su32(&acc_bar))
                 : "memory");
  }
  __syncwarp();
  // while the MMAs run: this thread's exponents of B's columns and, for
  // beta != 0, its entries of C (row r, the 8-column chunks of its half),
  // all loads in flight at once
  constexpr int NCH = (BN / 8 + 1) / 2;  // chunks per half
  const int quad = warp & 3, half = warp >> 2;
  const int r = m0 + quad * 32 + lane;
  int ebv[NCH][8];
  double cpre[NCH][8];
#pragma unroll
  for (int h = 0; h < NCH; h++) {
    const int c0 = half * 8 + 16 * h;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int c = n0 + c0 + j;
      const bool in = c0 < BN && c < P.N;
      ebv[h][j] = in ? __ldg(P.EB + (long long)b * P.N + c) : 0;
      cpre[h][j] = (in && r < P.M && P.beta != 0.0) ? P.C[(long long)b * P.sC + (long long)r * P.ldc + c] : 0.0;
    }
  }
  const bool have = oz_wait(oz_su32(&acc_bar), 0);
  if (!have && tid == 0) atomicOr(P.err, ERR_TIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool good = __syncthreads_and(have ? 1 : 0) && !give_up;
  if (!good && tid == 0) {
    // copies may still be in flight after a give-up: wait (bounded) for the
    // last use of each stage before the shared memory is released
    for (int s = 0; s < OZ_NSTAGE; s++) {
      const int uses = (nk - s + OZ_NSTAGE - 1) / OZ_NSTAGE;
      if (uses > 0) oz_wait(oz_su32(&full_bar[s]), (uses - 1) & 1);
    }
  }
  if (good) {
    // warp w: TMEM lanes 32 (w % 4) .. (its rows), 8-column chunks
    // half w / 4, half w / 4 + 2, ...
    const int ea = r < P.M ? P.EA[(long long)b * P.M + r] : OZ_ZERO_EXP;
    double* crow = P.C + (long long)b * P.sC + (long long)r * P.ldc;
#pragma unroll
    for (int h = 0; h < NCH; h++) {
      const int c0 = half * 8 + 16 * h;
      if (c0 >= BN) break;
      // groups 2 .. 5 in hi (units 2^-30), groups 6 .. NS+1 in lo: exact
      // integers below 2^43 and 2^49
      long long hi[8], lo[8];
#pragma unroll
      for (int j = 0; j < 8; j++) hi[j] = lo[j] = 0;
#pragma unroll
      for (int g = 0; g < NS; g++) {
        float v[8];
        oz_ld8(tacc + ((uint32_t)(quad * 32) << 16) + g * BN + c0, v);
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const long long q = (long long)__float2int_rn(v[j]);
          if (g < 4)
            hi[j] = hi[j] * (1 << OZ_BETA) + q;
          else
            lo[j] = lo[j] * (1 << OZ_BETA) + q;
        }
      }
      if (r < P.M) {
        static_assert(NS == 9, "the integer rounding takes lo in units of 2^-30 of hi");
        constexpr int LO_SHIFT = (NS - 4) * OZ_BETA;  // lo's unit relative to hi's
        const bool unit = P.alpha == 1.0 || P.alpha == -1.0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const int c = n0 + c0 + j;
          if (c >= P.N) break;
          const int eb = ebv[h][j];
          // value = (hi 2^30 + lo) 2^(ea + eb - 60): one rounding to FP64
          bool ok = false;
          double v = unit ? oz_round(hi[j], lo[j], ea + eb - 2 * LO_SHIFT, &ok) : 0.0;
          if (ok) {
            if (P.alpha < 0.0) v = -v;
          } else {
            const double u = fma((double)lo[j], oz_pow2(-LO_SHIFT), (double)hi[j]);
            v = P.alpha * (u * oz_pow2(ea + eb - 5 * OZ_BETA));
          }
          if (P.beta == 1.0)
            v += cpre[h][j];
          else if (P.beta != 0.0)
            v = fma(P.beta, cpre[h][j], v);
          crow[c] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tacc), "r"(Cfg::TALLOC));
}

// Exponent of each row of an operand: e with max_k |X(r, k)| < 2^e (frexp's
// exponent of the largest magnitude), OZ_ZERO_EXP for a zero row.  Element
// (r, k) of batch b at X[b sb + r sr + k sk].  Magnitudes are compared as the
// integer bit patterns of |x| (the order of nonnegative doubles).
__device__ __forceinline__ int oz_exp_of(unsigned long long mx) {
  if (mx == 0) return OZ_ZERO_EXP;
  const int ex = (int)(mx >> 52);
  return ex == 0 ? -1022 : ex - 1022;
}

__device__ __forceinline__ bool oz_skip(const int* active, int active_iter, int b) {
  return active != nullptr && active[b] <= active_iter;
}

__global__ void oz_exp_kcontig_kernel(int R, int K, int batch, const double* __restrict__ X, long long sr,
                                      long long sb, int* __restrict__ E, const int* __restrict__ active,
                                      int active_iter) {
  // one warp per row, K contiguous
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long long)R * batch) return;
  const int b = (int)(w / R), r = (int)(w % R);
  if (oz_skip(active, active_iter, b)) return;
  const double* x = X + (long long)b * sb + (long long)r * sr;
  unsigned long long mx = 0;
  for (int k = lane; k < K; k += 32) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(__ldg(x + k)) & 0x7FFFFFFFFFFFFFFFull;
    mx = a > mx ? a : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  if (lane == 0) E[(long long)b * R + r] = oz_exp_of(mx);
}

__global__ void oz_exp_rcontig_kernel(int R, int K, int batch, const double* __restrict__ X, long long sr,
                                      long long sk, long long sb, int* __restrict__ E,
                                      const int* __restrict__ active, int active_iter) {
  // 32 rows x 8 K-strips per block: with rows contiguous (sr = 1) a warp
  // reads 32 consecutive values at each k; the eight strips are combined
  // through shared memory
  __shared__ unsigned long long part[8][32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int b = blockIdx.y, r = blockIdx.x * 32 + tx;
  if (oz_skip(active, active_iter, b)) return;
  unsigned long long mx = 0;
  if (r < R) {
    const double* x = X + (long long)b * sb + (long long)r * sr;
    for (int k = ty; k < K; k += 8) {
      const unsigned long long a =
          (unsigned long long)__double_as_longlong(__ldg(x + (long long)k * sk)) & 0x7FFFFFFFFFFFFFFFull;
      mx = a > mx ? a : mx;
    }
  }
  part[ty][tx] = mx;
  __syncthreads();
  if (ty == 0 && r < R) {
#pragma unroll
    for (int j = 1; j < 8; j++) mx = part[j][tx] > mx ? part[j][tx] : mx;
    E[(long long)b * R + r] = oz_exp_of(mx);
  }
}

// Digits of x against exponent e: x 2^(62 - e) in 64-bit fixed point
// (truncated below 2^(e - 62)), then NS signed base-2^BETA digits by
// rounding from the top.
template <int NS>
__device__ __forceinline__ void oz_digits(double x, int e, int* d) {
  long long F = 0;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = bits & 0x7FFFFFFFFFFFFFFFull;
  if (mag != 0 && e != OZ_ZERO_EXP) {
    const int ex = (int)(mag >> 52);
    const unsigned long long m = ex == 0 ? (mag & 0xFFFFFFFFFFFFFull) : ((mag & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    const int sh = (ex == 0 ? 1 : ex) - 1075 + 62 - e;  // x = m 2^(ex - 1075); F = m 2^sh
    unsigned long long f;
    if (sh >= 0)
      f = m << sh;  // < 2^62 because |x| < 2^e
    else
      f = sh > -64 ? (m >> (-sh)) : 0ull;
    F = (bits >> 63) ? -(long long)f : (long long)f;
  }
#pragma unroll
  for (int i = 0; i < NS; i++) {
    const int s = 62 - (i + 1) * OZ_BETA;
    const long long q = (F + (1ll << (s - 1))) >> s;  // round half up
    d[i] = (int)q;
    F -= q * (1ll << s);
  }
}

// Digit planes of an operand in the tile-blocked layout (see the head of
// the file): a block of 32 rows x 32 K is read through shared memory (along
// whichever of r and k is contiguous) and written in address order, 64
// consecutive elements (one core matrix) per half warp.  Rows up to the
// padded tile count and K up to the padded block count are written, zero
// where outside the operand.
template <int NS>
__global__ void oz_slice_kernel(int R, int K, const double* __restrict__ X, long long sr, long long sk, long long sb,
                                const int* __restrict__ E, __nv_bfloat16* __restrict__ Q, int tile_rows, int ntiles,
                                int kblocks, const int* __restrict__ active, int active_iter) {
  __shared__ double tile[32][33];
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32, b = blockIdx.z;
  if (oz_skip(active, active_iter, b)) return;
  const int tid = threadIdx.x;  // 256
  const double* x = X + (long long)b * sb;
  if (sk == 1) {
    for (int e = tid; e < 1024; e += 256) {
      const int rr = e >> 5, kk = e & 31, r = r0 + rr, k = k0 + kk;
      tile[rr][kk] = (r < R && k < K) ? __ldg(x + (long long)r * sr + k) : 0.0;
    }
  } else {
    for (int e = tid; e < 1024; e += 256) {
      const int kk = e >> 5, rr = e & 31, r = r0 + rr, k = k0 + kk;
      tile[rr][kk] = (r < R && k < K) ? __ldg(x + (long long)r * sr + (long long)k * sk) : 0.0;
    }
  }
  __syncthreads();
  const int rpad = ntiles * tile_rows, kpad = kblocks * OZ_KB;
  const long long plane = (long long)tile_rows * OZ_KB;  // elements of one plane of one block
  for (int e = tid; e < 1024; e += 256) {
    // address order: k8, r8, K half, row group, K block
    const int k8 = e & 7, r8 = (e >> 3) & 7, kh = (e >> 6) & 1, rgl = (e >> 7) & 3, kbl = e >> 9;
    const int rr = rgl * 8 + r8, kk = kbl * 16 + kh * 8 + k8;
    const int r = r0 + rr, k = k0 + kk;
    if (r >= rpad || k >= kpad) continue;
    int d[NS];
    oz_digits<NS>(tile[rr][kk], r < R ? E[(long long)b * R + r] : OZ_ZERO_EXP, d);
    const int t = r / tile_rows, rt = r - t * tile_rows;
    const int kb = k / OZ_KB;
    __nv_bfloat16* q = Q + (((long long)b * ntiles + t) * kblocks + kb) * NS * plane +
                       ((rt >> 3) * 2 + kh) * 64 + r8 * 8 + k8;
#pragma unroll
    for (int i = 0; i < NS; i++) q[i * plane] = __int2bfloat16_rn(d[i]);
  }
}

unsigned oz_grid(long long total, int per) { return (unsigned)((total + per - 1) / per); }

}  // namespace

int oz_tiles(int rows, int tile_rows) { return (rows + tile_rows - 1) / tile_rows; }
int oz_kblocks(int K) { return (K + OZ_KB - 1) / OZ_KB; }

size_t oz_sliced_bytes(int rows, int K, int batch, int tile_rows) {
  const size_t planes = (size_t)kOzSlices * batch * oz_tiles(rows, tile_rows) * tile_rows * oz_kblocks(K) * OZ_KB * 2;
  return (planes + 255) / 256 * 256 + ((size_t)batch * rows * sizeof(int) + 255) / 256 * 256;
}

OzSliced oz_carve(void* base, int rows, int K, int batch, int tile_rows) {
  OzSliced o;
  o.rows = rows;
  o.K = K;
  o.batch = batch;
  o.tile_rows = tile_rows;
  o.Q = (__nv_bfloat16*)base;
  const size_t planes = (size_t)kOzSlices * batch * oz_tiles(rows, tile_rows) * tile_rows * oz_kblocks(K) * OZ_KB * 2;
  o.E = (int*)((uint8_t*)base + (planes + 255) / 256 * 256);
  return o;
}

OzSliced oz_view(const OzSliced& o, int b) {
  OzSliced v = o;
  v.batch = 1;
  v.Q = o.Q + (size_t)b * kOzSlices * oz_tiles(o.rows, o.tile_rows) * o.tile_rows * oz_kblocks(o.K) * OZ_KB;
  v.E = o.E + (size_t)b * o.rows;
  return v;
}

cudaError_t oz_slice(const double* X, long long sr, long long sk, long long sb, const OzSliced& o, const int* active,
                     int active_iter, cudaStream_t st) {
  if (o.rows <= 0 || o.batch <= 0) return cudaSuccess;
  const long long rows = (long long)o.rows * o.batch;
  count_launch();
  if (sk == 1)
    oz_exp_kcontig_kernel<<<oz_grid(rows * 32, 256), 256, 0, st>>>(o.rows, o.K, o.batch, X, sr, sb, o.E, active,
                                                                   active_iter);
  else
    oz_exp_rcontig_kernel<<<dim3(oz_grid(o.rows, 32), o.batch), dim3(32, 8), 0, st>>>(o.rows, o.K, o.batch, X, sr, sk,
                                                                                       sb, o.E, active, active_iter);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nt = oz_tiles(o.rows, o.tile_rows), kbl = oz_kblocks(o.K);
  dim3 grid(oz_grid((long long)kbl * OZ_KB, 32), oz_grid((long long)nt * o.tile_rows, 32), o.batch);
  count_launch();
  oz_slice_kernel<kOzSlices><<<grid, 256, 0, st>>>(o.rows, o.K, X, sr, sk, sb, o.E, o.Q, o.tile_rows, nt, kbl, active,
                                                   active_iter);
  return cudaGetLastError();
}

namespace {
template <int BN>
cudaError_t oz_launch(const OzSliced& A, const OzSliced& B, OzGemm p, cudaStream_t st) {
  constexpr int NS = kOzSlices;
  using Cfg = OzCfg<NS, BN>;
  p.EA = A.E;
  p.EB = B.E;
  cudaError_t e = set_smem_once((const void*)ozgemm_kernel<NS, BN>, Cfg::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(oz_tiles(p.N, BN), oz_tiles(p.M, OZ_TBM), p.batch);
  count_launch();
  ozgemm_kernel<NS, BN><<<grid, OZ_THREADS, Cfg::SMEM, st>>>(p, A.Q, B.Q, oz_kblocks(p.K));
  return cudaGetLastError();
}
}  // namespace

cudaError_t oz_multiply(const OzSliced& A, const OzSliced& B, const OzGemm& p, cudaStream_t st) {
  if (p.M <= 0 || p.N <= 0 || p.batch <= 0) return cudaSuccess;
  if (A.tile_rows != OZ_TBM || A.rows != p.M || B.rows != p.N || A.K != p.K || B.K != p.K || A.batch != p.batch ||
      B.batch != p.batch || p.K > kOzMaxK)
    return cudaErrorInvalidValue;
  if (B.tile_rows == kOzBN) return oz_launch<kOzBN>(A, B, p, st);
  if (B.tile_rows == kOzBNSmall) return oz_launch<kOzBNSmall>(A, B, p, st);
  return cudaErrorInvalidValue;
}

size_t oz_scratch_bytes(int M, int N, int K, int batch) {
  return oz_sliced_bytes(M, K, batch, OZ_TBM) + oz_sliced_bytes(N, K, batch, kOzBN);
}

cudaError_t ozgemm_f64(const OzGemm& p, void* scratch, size_t scratch_bytes, int sm_count, cudaStream_t st) {
  (void)sm_count;
  if (p.M <= 0 || p.N <= 0 || p.batch <= 0) return cudaSuccess;
  if (p.K <= 0 || p.K > kOzMaxK) return cudaErrorInvalidValue;
  if (scratch_bytes < oz_scratch_bytes(p.M, p.N, p.K, p.batch)) return cudaErrorInvalidValue;
  const OzSliced A = oz_carve(scratch, p.M, p.K, p.batch, OZ_TBM);
  const OzSliced B = oz_carve((uint8_t*)scratch + oz_sliced_bytes(p.M, p.K, p.batch, OZ_TBM), p.N, p.K, p.batch, kOzBN);
  // A's rows; B's columns (B element (k, c) is row c, position k of B^T)
  cudaError_t e = oz_slice(p.A, p.a_sm, p.a_sk, p.sA, A, p.active, p.active_iter, st);
  if (e == cudaSuccess) e = oz_slice(p.B, p.b_sn, p.b_sk, p.sB, B, p.active, p.active_iter, st);
  if (e != cudaSuccess) return e;
  return oz_multiply(A, B, p, st);
}

}  // namespace lb
