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
// Data path (one CTA per 128 x BN output tile and batch element):
//  * the digits are "slice planes" bf16 [batch][NS][rows][Kp] (K contiguous,
//    Kp = K rounded up to 8) with the exponents int [batch][rows]; for B the
//    rows are B's columns (the K-major B operand of the MMA);
//  * warp 0 copies 32-wide K blocks of all NS planes of A (128 rows) and of
//    B (BN rows) with one 3-D TMA each (64-byte swizzle) into a two-stage
//    ring;
//  * one thread of warp 1 issues, per 16-wide K step and digit i of A, one
//    MMA of A_i against the stacked planes B_1 .. B_{NS+1-i} (N = (NS+1-i)
//    BN, at most 256 per instruction) into the TMEM columns of the groups
//    i+1 .. NS+1: the accumulator is NS groups x BN columns of FP32;
//  * all eight warps read the groups out of TMEM (warp w: lanes 32 (w % 4),
//    columns of half w / 4), combine them and write FP64
//    C = alpha (A B) + beta C.
// Every mbarrier wait is bounded; a wait that gives up sets the error word,
// the CTA waits (bounded) for its copies in flight and frees its TMEM.
#include "lb_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

namespace lb {

namespace {

constexpr int OZ_BETA = 6;
constexpr int OZ_TBM = 128;       // rows per tile (M of one MMA)
constexpr int OZ_TBK = 32;        // K per stage: 64 bytes of BF16 per row
constexpr int OZ_NSTAGE = 2;
constexpr int OZ_THREADS = 256;
constexpr int OZ_ZERO_EXP = -2000;  // exponent of an all-zero row
constexpr long long kOzWaitCycles = 4000000000LL;

template <int NS, int BN>
struct OzCfg {
  static constexpr int A_BYTES = NS * OZ_TBM * OZ_TBK * 2;
  static constexpr int B_BYTES = NS * BN * OZ_TBK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int SMEM = OZ_NSTAGE * STAGE + 1024;
  static constexpr int TCOLS = NS * BN;
  static constexpr int TALLOC = TCOLS <= 32 ? 32 : TCOLS <= 64 ? 64 : TCOLS <= 128 ? 128 : TCOLS <= 256 ? 256 : 512;
  static_assert(TCOLS <= 512, "TMEM columns");
  static_assert(SMEM <= 232448, "shared memory");
  static_assert(A_BYTES % 1024 == 0 && B_BYTES % 512 == 0, "swizzle atoms");
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

// shared-memory matrix descriptor: K-major, 64-byte swizzle (8-row atoms of
// 512 bytes), Blackwell descriptor version
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
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

__device__ __forceinline__ void oz_tma3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void oz_ld16(uint32_t ta, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// 2^s as a double for s in [-1022, 1023]; 0 below
__device__ __forceinline__ double oz_pow2(int s) {
  if (s < -1022) return 0.0;
  return __longlong_as_double((long long)(s + 1023) << 52);
}

template <int NS, int BN>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    ozgemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ OzGemm P) {
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
  const int nk = (P.K + OZ_TBK - 1) / OZ_TBK;

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
    // producer: all NS planes of a K block of A and of B, one TMA each
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
      oz_tma3(base, &mapA, kb * OZ_TBK, m0, b * NS, fb);
      oz_tma3(base + Cfg::A_BYTES, &mapB, kb * OZ_TBK, n0, b * NS, fb);
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
      for (int kk = 0; kk < OZ_TBK / 16; kk++) {
        const uint32_t o = kk * 32;
#pragma unroll
        for (int i = 0; i < NS; i++) {
          const uint64_t ad = oz_desc(abase + i * (OZ_TBM * OZ_TBK * 2) + o);
          const int rows = (NS - i) * BN;  // stacked B rows of digits 0 .. NS-1-i
#pragma unroll
          for (int r0 = 0; r0 < rows; r0 += 256) {
            const int nr = rows - r0 < 256 ? rows - r0 : 256;
            const uint32_t acc = (kb > 0 || kk > 0 || i > 0) ? 1u : 0u;
            oz_mma(tacc + i * BN + r0, ad, oz_desc(bbase + r0 * (OZ_TBK * 2) + o), oz_idesc(nr), acc);
          }
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
    // warp w: TMEM lanes 32 (w % 4) .. (its rows), columns of half w / 4
    const int quad = warp & 3, half = warp >> 2;
    const int r = m0 + quad * 32 + lane;
    const int ea = r < P.M ? P.EA[(long long)b * P.M + r] : OZ_ZERO_EXP;
    double* crow = P.C + (long long)b * P.sC + (long long)r * P.ldc;
    for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
      // groups 2 .. 5 in hi (units 2^-30), groups 6 .. NS+1 in lo: exact
      // integers below 2^43 and 2^49
      long long hi[16], lo[16];
#pragma unroll
      for (int j = 0; j < 16; j++) hi[j] = lo[j] = 0;
#pragma unroll
      for (int g = 0; g < NS; g++) {
        float v[16];
        oz_ld16(tacc + ((uint32_t)(quad * 32) << 16) + g * BN + c0, v);
#pragma unroll
        for (int j = 0; j < 16; j++) {
          const long long q = (long long)__float2int_rn(v[j]);
          if (g < 4)
            hi[j] = hi[j] * (1 << OZ_BETA) + q;
          else
            lo[j] = lo[j] * (1 << OZ_BETA) + q;
        }
      }
      if (r < P.M) {
        constexpr int LO_SHIFT = (NS - 4) * OZ_BETA;  // lo's unit relative to hi's
#pragma unroll
        for (int j = 0; j < 16; j++) {
          const int c = n0 + c0 + j;
          if (c >= P.N) break;
          const int eb = P.EB[(long long)b * P.N + c];
          const double u = fma((double)lo[j], oz_pow2(-LO_SHIFT), (double)hi[j]);
          const double v = u * oz_pow2(ea + eb - 5 * OZ_BETA);
          double out = P.alpha * v;
          if (P.beta != 0.0) out = fma(P.beta, crow[c], out);
          crow[c] = out;
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

__global__ void oz_exp_kcontig_kernel(int R, int K, int batch, const double* __restrict__ X, long long sr,
                                      long long sb, int* __restrict__ E) {
  // one warp per row, K contiguous
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long long)R * batch) return;
  const int b = (int)(w / R), r = (int)(w % R);
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
                                      long long sk, long long sb, int* __restrict__ E) {
  // one thread per row; with rows contiguous (sr = 1) the threads of a warp
  // read consecutive addresses at every k
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)R * batch) return;
  const int b = (int)(t / R), r = (int)(t % R);
  const double* x = X + (long long)b * sb + (long long)r * sr;
  unsigned long long mx = 0;
  for (int k = 0; k < K; k++) {
    const unsigned long long a =
        (unsigned long long)__double_as_longlong(__ldg(x + (long long)k * sk)) & 0x7FFFFFFFFFFFFFFFull;
    mx = a > mx ? a : mx;
  }
  E[(long long)b * R + r] = oz_exp_of(mx);
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

// Slice planes of an operand: Q[b][i][r][k] (row stride Kp, plane stride
// R Kp) for rows r < R and k < K, through a 32 x 32 tile in shared memory so
// that reads (along whichever of r and k is contiguous) and writes (along k)
// are coalesced.
template <int NS>
__global__ void oz_split_kernel(int R, int K, int batch, const double* __restrict__ X, long long sr, long long sk,
                                long long sb, const int* __restrict__ E, __nv_bfloat16* __restrict__ Q,
                                long long Kp) {
  __shared__ double tile[32][33];
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32, b = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const double* x = X + (long long)b * sb;
  if (sk == 1) {
    for (int rr = ty; rr < 32; rr += 8) {
      const int r = r0 + rr, k = k0 + tx;
      tile[rr][tx] = (r < R && k < K) ? __ldg(x + (long long)r * sr + k) : 0.0;
    }
  } else {
    for (int kk = ty; kk < 32; kk += 8) {
      const int r = r0 + tx, k = k0 + kk;
      tile[tx][kk] = (r < R && k < K) ? __ldg(x + (long long)r * sr + (long long)k * sk) : 0.0;
    }
  }
  __syncthreads();
  const long long plane = (long long)R * Kp;
  for (int rr = ty; rr < 32; rr += 8) {
    const int r = r0 + rr, k = k0 + tx;
    if (r >= R || k >= K) continue;
    int d[NS];
    oz_digits<NS>(tile[rr][tx], E[(long long)b * R + r], d);
    __nv_bfloat16* q = Q + (long long)b * NS * plane + (long long)r * Kp + k;
#pragma unroll
    for (int i = 0; i < NS; i++) q[i * plane] = __int2bfloat16_rn(d[i]);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 oz_encode_fn = nullptr;
std::once_flag oz_encode_once;

bool oz_encode(CUtensorMap* m, const __nv_bfloat16* base, int rows, int K, long long Kp, int planes, int box_rows,
               int box_planes) {
  std::call_once(oz_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      oz_encode_fn = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    else
      cudaGetLastError();
  });
  if (oz_encode_fn == nullptr) return false;
  if ((Kp * 2) % 16 != 0 || ((uintptr_t)base & 15) != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * 2), (cuuint64_t)(Kp * 2 * rows)};
  cuuint32_t box[3] = {(cuuint32_t)OZ_TBK, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
  cuuint32_t es[3] = {1, 1, 1};
  return oz_encode_fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

unsigned oz_grid(long long total, int per) { return (unsigned)((total + per - 1) / per); }

cudaError_t oz_exponents(int R, int K, int batch, const double* X, long long sr, long long sk, long long sb, int* E,
                         cudaStream_t st) {
  const long long rows = (long long)R * batch;
  count_launch();
  if (sk == 1)
    oz_exp_kcontig_kernel<<<oz_grid(rows * 32, 256), 256, 0, st>>>(R, K, batch, X, sr, sb, E);
  else
    oz_exp_rcontig_kernel<<<oz_grid(rows, 256), 256, 0, st>>>(R, K, batch, X, sr, sk, sb, E);
  return cudaGetLastError();
}

template <int NS>
cudaError_t oz_split(int R, int K, int batch, const double* X, long long sr, long long sk, long long sb, const int* E,
                     __nv_bfloat16* Q, long long Kp, cudaStream_t st) {
  dim3 grid((K + 31) / 32, (R + 31) / 32, batch);
  count_launch();
  oz_split_kernel<NS><<<grid, dim3(32, 8), 0, st>>>(R, K, batch, X, sr, sk, sb, E, Q, Kp);
  return cudaGetLastError();
}

}  // namespace

long long oz_kpad(int K) { return ((long long)K + 7) / 8 * 8; }

size_t oz_scratch_bytes(int M, int N, int K, int batch) {
  const long long Kp = oz_kpad(K);
  const size_t slices = (size_t)kOzSlices * batch * ((size_t)M + N) * Kp * 2;
  return (slices + 255) / 256 * 256 + (size_t)batch * (M + N) * sizeof(int) + 256;
}

cudaError_t ozgemm_f64(const OzGemm& p0, void* scratch, size_t scratch_bytes, int sm_count, cudaStream_t st) {
  (void)sm_count;
  OzGemm p = p0;
  if (p.M <= 0 || p.N <= 0 || p.batch <= 0) return cudaSuccess;
  if (p.K <= 0 || p.K > kOzMaxK) return cudaErrorInvalidValue;
  if (scratch_bytes < oz_scratch_bytes(p.M, p.N, p.K, p.batch)) return cudaErrorInvalidValue;
  constexpr int NS = kOzSlices, BN = 32;
  using Cfg = OzCfg<NS, BN>;
  const long long Kp = oz_kpad(p.K);
  __nv_bfloat16* QA = (__nv_bfloat16*)scratch;
  __nv_bfloat16* QB = QA + (size_t)NS * p.batch * p.M * Kp;
  const size_t slices = (size_t)NS * p.batch * ((size_t)p.M + p.N) * Kp * 2;
  int* EA = (int*)((uint8_t*)scratch + (slices + 255) / 256 * 256);
  int* EB = EA + (size_t)p.batch * p.M;
  // A's rows; B's columns (B element (k, c) is row c, position k of B^T)
  cudaError_t e = oz_exponents(p.M, p.K, p.batch, p.A, p.a_sm, p.a_sk, p.sA, EA, st);
  if (e == cudaSuccess) e = oz_exponents(p.N, p.K, p.batch, p.B, p.b_sn, p.b_sk, p.sB, EB, st);
  if (e == cudaSuccess) e = oz_split<NS>(p.M, p.K, p.batch, p.A, p.a_sm, p.a_sk, p.sA, EA, QA, Kp, st);
  if (e == cudaSuccess) e = oz_split<NS>(p.N, p.K, p.batch, p.B, p.b_sn, p.b_sk, p.sB, EB, QB, Kp, st);
  if (e != cudaSuccess) return e;
  p.EA = EA;
  p.EB = EB;
  CUtensorMap ma, mb;
  if (!oz_encode(&ma, QA, p.M, p.K, Kp, NS * p.batch, OZ_TBM, NS) ||
      !oz_encode(&mb, QB, p.N, p.K, Kp, NS * p.batch, BN, NS))
    return cudaErrorInvalidValue;
  e = set_smem_once((const void*)ozgemm_kernel<NS, BN>, Cfg::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid((p.N + BN - 1) / BN, (p.M + OZ_TBM - 1) / OZ_TBM, p.batch);
  count_launch();
  ozgemm_kernel<NS, BN><<<grid, OZ_THREADS, Cfg::SMEM, st>>>(ma, mb, p);
  return cudaGetLastError();
}

}  // namespace lb
