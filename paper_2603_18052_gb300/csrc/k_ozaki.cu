// FP64 matrix products on the BF16 tensor cores through exact slices (the
// Ozaki scheme: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Row r of the left operand A (M x K) is written in fixed point against its
// own exponent e_r (every |A[r][k]| < 2^e_r) as signed base-2^BETA digits,
//   A[r][k] = 2^e_r ( sum_{i=1..NS} a_i[r][k] 2^(-i BETA) + rho ),
//   |a_1| <= 2^BETA, -2^(BETA-1) <= a_i < 2^(BETA-1) (i >= 2),
//   |rho| <= 2^(-NS BETA - 1),
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
//    C = alpha (A B) + beta C; a variant (XO) also writes further outputs
//    formed from the product and two matrices laid out like C (OzExtra).
// Every mbarrier wait is bounded; a wait that gives up sets the error word,
// the CTA waits (bounded) for its copies in flight and frees its TMEM.
//
// The digits are made by oz_slice: one pass per row group (exponents and
// digits) when K or the rows of the operand are contiguous, else an
// exponent pass and a pass over 32 x 32 blocks.
#include "lb_internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace lb {

namespace {

constexpr int OZ_BETA = 6;
constexpr int OZ_TBM = 128;       // rows per A tile (M of one MMA)
constexpr int OZ_KB = 16;         // K per block and stage (one MMA K step)
constexpr int OZ_NSTAGE = 4;
constexpr int OZ_THREADS = 320;  // producer warp, MMA warp, eight epilogue warps (at most 168 registers:
                                 // three warps share one scheduler's 16K registers)
constexpr int OZ_ZERO_EXP = -2000;  // exponent of an all-zero row
constexpr long long kOzWaitCycles = 4000000000LL;
constexpr long long kOzSliceCtas = 304;  // slicing CTAs wanted at least (two per SM of 152)

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

// Eight columns of each of the nine groups of this thread's lane (group g
// at TMEM column ta + g stride), all loads in flight, one wait.
__device__ __forceinline__ void oz_ld8x9(uint32_t ta, uint32_t stride, float* v) {
  uint32_t r[72];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%72];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%73];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%74];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%75];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32,%33,%34,%35,%36,%37,%38,%39}, [%76];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%40,%41,%42,%43,%44,%45,%46,%47}, [%77];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%48,%49,%50,%51,%52,%53,%54,%55}, [%78];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%56,%57,%58,%59,%60,%61,%62,%63}, [%79];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%64,%65,%66,%67,%68,%69,%70,%71}, [%80];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63]), "=r"(r[64]), "=r"(r[65]), "=r"(r[66]), "=r"(r[67]), "=r"(r[68]), "=r"(r[69]), "=r"(r[70]), "=r"(r[71])
      : "r"(ta + 0 * stride), "r"(ta + 1 * stride), "r"(ta + 2 * stride), "r"(ta + 3 * stride), "r"(ta + 4 * stride), "r"(ta + 5 * stride), "r"(ta + 6 * stride), "r"(ta + 7 * stride), "r"(ta + 8 * stride)
      : "memory");
#pragma unroll
  for (int i = 0; i < 72; i++) v[i] = __uint_as_float(r[i]);
}

// x 2^e as a double, exactly, for |x| < 2^53, with sgn xor-ed into the sign;
// false where the result would not be a normal double.
__device__ __forceinline__ bool oz_i2d(long long x, int e, unsigned long long sgn, double* out) {
  if (x == 0) {
    *out = 0.0;
    return true;
  }
  const unsigned long long neg = x < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  const int p = 63 - __clzll((long long)a);  // leading bit, <= 52
  const int E = p + e;
  if (E < -1022 || E > 1023) return false;
  const unsigned long long mant = (a << (52 - p)) & 0xFFFFFFFFFFFFFull;
  *out = __longlong_as_double((long long)((neg ^ sgn) | ((unsigned long long)(E + 1023) << 52) | mant));
  return true;
}

// 2^s as a double for s in [-1022, 1023]; 0 below
__device__ __forceinline__ double oz_pow2(int s) {
  if (s < -1022) return 0.0;
  return __longlong_as_double((long long)(s + 1023) << 52);
}

// Persistent: CTA c takes tiles c, c + gridDim.x, ... (tile = (batch, row
// tile, column tile), column tile fastest).  Warp 0 (one lane) copies K
// blocks into the ring, running ahead into the next tile; warp 1 (one lane)
// issues the MMAs of a tile once the epilogue has emptied TMEM; warps 2 .. 9
// are the epilogue: they read the groups of a finished tile out of TMEM,
// fold them into two exact integers per output, release TMEM (so the next
// tile's MMAs start) and only then round, add beta C and store.
template <int NS, int BN, bool XO>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    ozgemm_kernel(const __grid_constant__ OzGemm P, const __nv_bfloat16* __restrict__ QA,
                  const __nv_bfloat16* __restrict__ QB, int kblocks) {
  using Cfg = OzCfg<NS, BN>;
  constexpr int NCH = (BN / 8 + 1) / 2;  // 8-column chunks per epilogue thread
  static_assert(BN % 16 == 0 && 16 * (NCH - 1) + 8 < BN, "both halves take NCH whole chunks");
  extern __shared__ __align__(1024) uint8_t oz_smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[OZ_NSTAGE], empty_bar[OZ_NSTAGE], acc_bar, tfree_bar, done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int give_up;
  __shared__ int issued_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NT = (P.N + BN - 1) / BN, MT = (P.M + OZ_TBM - 1) / OZ_TBM;
  const int tiles = NT * MT * P.batch;
  const int nk = kblocks;
  auto tile_of = [&](int t, int& b, int& mt, int& nt) {
    nt = t % NT;
    mt = (t / NT) % MT;
    b = t / (NT * MT);
  };
  auto skipped = [&](int b) { return P.active != nullptr && P.active[b] <= P.active_iter; };

  if (tid == 0) {
    for (int s = 0; s < OZ_NSTAGE; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(&empty_bar[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(&acc_bar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(oz_su32(&tfree_bar)));  // one arrival per epilogue warp
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(oz_su32(&done_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    give_up = 0;
    issued_s = 0;
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

  if (warp == 0) {
    if (lane == 0) {
      // producer: K blocks of this CTA's tiles in order, it = running block count
      int it = 0;
      for (int t = blockIdx.x; t < tiles && !give_up; t += gridDim.x) {
        int b, mt, nt;
        tile_of(t, b, mt, nt);
        if (skipped(b)) continue;
        const uint8_t* srcA = (const uint8_t*)QA + ((long long)b * MT + mt) * (long long)nk * Cfg::A_BYTES;
        const uint8_t* srcB = (const uint8_t*)QB + ((long long)b * NT + nt) * (long long)nk * Cfg::B_BYTES;
        for (int kb = 0; kb < nk; kb++, it++) {
          const int s = it % OZ_NSTAGE;
          if (it >= OZ_NSTAGE && !oz_wait(oz_su32(&empty_bar[s]), ((it - OZ_NSTAGE) / OZ_NSTAGE) & 1)) {
            atomicOr(P.err, ERR_TIMEOUT);
            give_up = 1;
            break;
          }
          const uint32_t base = oz_su32(sm + s * Cfg::STAGE);
          const uint32_t fb = oz_su32(&full_bar[s]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(Cfg::STAGE)
                       : "memory");
          oz_bulk(base, srcA + (long long)kb * Cfg::A_BYTES, Cfg::A_BYTES, fb);
          oz_bulk(base + Cfg::A_BYTES, srcB + (long long)kb * Cfg::B_BYTES, Cfg::B_BYTES, fb);
          issued_s = it + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: digit i of A against B digits 0 .. NS-1-i into group
      // columns [i BN, NS BN); one commit to acc_bar per tile
      int it = 0, j = 0;
      for (int t = blockIdx.x; t < tiles && !give_up; t += gridDim.x) {
        int b, mt, nt;
        tile_of(t, b, mt, nt);
        if (skipped(b)) continue;
        if (j > 0 && !oz_wait(oz_su32(&tfree_bar), (j - 1) & 1)) {  // TMEM read out by the epilogue
          atomicOr(P.err, ERR_TIMEOUT);
          give_up = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        bool ok = true;
        for (int kb = 0; kb < nk; kb++, it++) {
          const int s = it % OZ_NSTAGE;
          if (!oz_wait(oz_su32(&full_bar[s]), (it / OZ_NSTAGE) & 1)) {
            atomicOr(P.err, ERR_TIMEOUT);
            give_up = 1;
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t abase = oz_su32(sm + s * Cfg::STAGE);
          const uint32_t bbase = abase + Cfg::A_BYTES;
#pragma unroll
          for (int i = 0; i < NS; i++) {
            const uint64_t ad = oz_desc(abase + i * (OZ_TBM * OZ_KB * 2));
            const int rows = (NS - i) * BN;
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
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         oz_su32(&acc_bar))
                     : "memory");
        j++;
      }
      // every MMA issued so far complete before TMEM is released at exit
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       oz_su32(&done_bar))
                   : "memory");
    }
  } else {
    // epilogue warps 2 .. 9: TMEM lane quadrant warp % 4, column half (warp - 2) / 4
    static_assert(NS == 9, "the group split below is for nine groups");
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const bool unit = P.alpha == 1.0 || P.alpha == -1.0;
    const unsigned long long sgn = P.alpha < 0.0 ? (1ull << 63) : 0ull;
    const int bmode = P.beta == 0.0 ? 0 : (P.beta == 1.0 ? 1 : 2);
    int j = 0;
    for (int t = blockIdx.x; t < tiles && !give_up; t += gridDim.x) {
      int b, mt, nt;
      tile_of(t, b, mt, nt);
      if (skipped(b)) continue;
      const int n0 = nt * BN, r = mt * OZ_TBM + quad * 32 + lane;
      const int ea = r < P.M ? __ldg(P.EA + (long long)b * P.M + r) : OZ_ZERO_EXP;
      // every lane waits; the verdict is made warp-uniform (the TMEM loads
      // below need the whole warp)
      if (!__all_sync(0xffffffffu, oz_wait(oz_su32(&acc_bar), j & 1) ? 1 : 0)) {
        if (lane == 0) atomicOr(P.err, ERR_TIMEOUT);
        give_up = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // the product is 2^(ea + eb - 12) sum_g G_g 2^(-6 g) (G_g exact
      // integers below 2^24): H = groups 2 .. 6 (below 2^49) and L = groups
      // 7 .. 10 (below 2^43), both exact
      long long Hs[NCH][8], Ls[NCH][8];
#pragma unroll
      for (int h = 0; h < NCH; h++) {
        const int c0 = half * 8 + 16 * h;
        float v[NS * 8];
        oz_ld8x9(tacc + ((uint32_t)(quad * 32) << 16) + c0, BN, v);
#pragma unroll
        for (int jj = 0; jj < 8; jj++) {
          int q[NS];
#pragma unroll
          for (int g = 0; g < NS; g++) q[g] = __float2int_rn(v[g * 8 + jj]);
          Hs[h][jj] = ((((long long)(q[0] * 64 + q[1]) * 64 + q[2]) * 64 + q[3]) * 64) + q[4];
          Ls[h][jj] = ((long long)(q[5] * 64 + q[6]) * 64 + q[7]) * 64 + q[8];
        }
      }
      // TMEM free for the next tile's MMAs
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(oz_su32(&tfree_bar)) : "memory");
      j++;
      if (r < P.M) {
        // C element (r, c) at crow[c * cstep]: row-major, or transposed
        // (consecutive rows of a warp then hit consecutive addresses)
        const long long coff = (long long)b * P.sC + (P.transC ? (long long)r : (long long)r * P.ldc);
        double* crow = (!XO || P.C != nullptr) ? P.C + coff : nullptr;
        const long long cstep = P.transC ? P.ldc : 1;
#pragma unroll
        for (int h = 0; h < NCH; h++) {
          const int c0 = half * 8 + 16 * h;
          double cold[8];
          int ebv[8];
#pragma unroll
          for (int jj = 0; jj < 8; jj++) {
            const int c = n0 + c0 + jj;
            cold[jj] = (bmode != 0 && c < P.N) ? crow[c * cstep] : 0.0;
            ebv[jj] = c < P.N ? __ldg(P.EB + (long long)b * P.N + c) : 0;
          }
#pragma unroll
          for (int jj = 0; jj < 8; jj++) {
            const int c = n0 + c0 + jj;
            if (c >= P.N) break;
            const int E = ea + ebv[jj];
            double hd, ld, out;
            if (unit && oz_i2d(Hs[h][jj], E - 36, sgn, &hd) && oz_i2d(Ls[h][jj], E - 60, sgn, &ld)) {
              out = hd + ld;  // the one rounding
            } else {
              const double u = fma((double)Ls[h][jj], oz_pow2(-24), (double)Hs[h][jj]);
              out = P.alpha * (u * oz_pow2(E - 36));
            }
            if (bmode == 1)
              out += cold[jj];
            else if (bmode == 2)
              out = fma(P.beta, cold[jj], out);
            if (!XO) {
              crow[c * cstep] = out;
            } else {
              if (crow != nullptr) crow[c * cstep] = out;
              // the further outputs (row-major only)
              const long long e = coff + c;
              const double t1 = P.x.T1 != nullptr ? P.x.T1[e] : 0.0;
              if (P.x.pm) {
                P.x.X[0][e] = t1 - out;
                P.x.X[1][e] = t1 + out;
              } else {
                const double t2 = P.x.T2 != nullptr ? P.x.T2[e] : 0.0;
#pragma unroll
                for (int w = 0; w < 4; w++) {
                  if (w >= P.x.nx) break;
                  double v = P.x.c[w][0] * out + (P.x.c[w][1] * t1 + P.x.c[w][2] * t2);
                  if (r == c) v += P.x.g[w];
                  P.x.X[w][e] = v;
                }
              }
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    // MMAs complete (bounded) and, after a give-up, the copies in flight
    if (!oz_wait(oz_su32(&done_bar), 0)) atomicOr(P.err, ERR_TIMEOUT);
    if (give_up) {
      const int issued = issued_s;
      for (int s = 0; s < OZ_NSTAGE && s < issued; s++) {
        const int last = s + (issued - 1 - s) / OZ_NSTAGE * OZ_NSTAGE;  // the last block copied into stage s
        oz_wait(oz_su32(&full_bar[s]), (last / OZ_NSTAGE) & 1);
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

// Fixed-point form of x against exponent e: F = x 2^(62 - e), |F| < 2^62,
// truncated below 2^(e - 62); 0 for x = 0 or a zero row.
__device__ __forceinline__ long long oz_fixed(double x, int e) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = bits & 0x7FFFFFFFFFFFFFFFull;
  if (mag == 0 || e == OZ_ZERO_EXP) return 0;
  const int ex = (int)(mag >> 52);
  const unsigned long long m = ex == 0 ? (mag & 0xFFFFFFFFFFFFFull) : ((mag & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  const int sh = (ex == 0 ? 1 : ex) - 1075 + 62 - e;  // x = m 2^(ex - 1075); F = m 2^sh
  unsigned long long f;
  if (sh >= 0)
    f = m << sh;  // < 2^62 because |x| < 2^e
  else
    f = sh > -64 ? (m >> (-sh)) : 0ull;
  return (bits >> 63) ? -(long long)f : (long long)f;
}

// The NS = 9 signed base-64 digits of F (digit i at bit 56 - 6 i), as BF16
// bit patterns: with the balancing offsets sum_i 32 2^(56 - 6 i) and half of
// the last digit's unit added, digit i >= 1 is its 6-bit field minus 32
// (in [-32, 31]) and digit 0 everything above minus 32 (in [-64, 64]); the
// remainder F - sum_i d_i 2^(56 - 6 i) lies in [-128, 127].  A small
// integer d becomes a float through the 2^23 magic number (exact), and its
// BF16 pattern is the float's upper half (at most seven significant bits).
__device__ __forceinline__ uint32_t oz_bf16_of(int d) {
  const float f = __int_as_float(0x4B000000 | (d + 0x400000)) - 12582912.0f;
  return __float_as_uint(f) >> 16;
}

__host__ __device__ constexpr long long oz_offsets() {
  long long c = 1ll << (62 - 9 * OZ_BETA - 1);
  for (int i = 0; i < 9; i++) c += 1ll << (62 - (i + 1) * OZ_BETA + OZ_BETA - 1);
  return c;
}
static_assert(oz_offsets() == 0x2082082082082080ll, "digit offsets");

__device__ __forceinline__ void oz_digit_bits(long long F, uint32_t* h) {
  constexpr long long CR = oz_offsets();  // sum_i 2^(61 - 6 i) + 2^7
  const long long G = F + CR;
  const int hi = (int)(G >> 32);
  const unsigned lo = (unsigned)G;
  h[0] = oz_bf16_of((hi >> 24) - 32);
  h[1] = oz_bf16_of((int)((hi >> 18) & 63) - 32);
  h[2] = oz_bf16_of((int)((hi >> 12) & 63) - 32);
  h[3] = oz_bf16_of((int)((hi >> 6) & 63) - 32);
  h[4] = oz_bf16_of((int)(hi & 63) - 32);
  h[5] = oz_bf16_of((int)((lo >> 26) & 63) - 32);
  h[6] = oz_bf16_of((int)((lo >> 20) & 63) - 32);
  h[7] = oz_bf16_of((int)((lo >> 14) & 63) - 32);
  h[8] = oz_bf16_of((int)((lo >> 8) & 63) - 32);
}

// Digit planes of an operand in the tile-blocked layout (see the head of
// the file): a block of 32 rows x 32 K is read through shared memory (along
// whichever of r and k is contiguous) and written in address order, two
// consecutive elements per thread and plane (one 4-byte store), 64
// consecutive elements (one core matrix) per 32 threads.  Rows up to the
// padded tile count and K up to the padded block count are written, zero
// where outside the operand.
template <int NS>
__global__ void oz_slice_kernel(int R, int K, const double* __restrict__ X, long long sr, long long sk, long long sb,
                                const int* __restrict__ E, __nv_bfloat16* __restrict__ Q, int tile_rows, int ntiles,
                                int kblocks, const int* __restrict__ active, int active_iter) {
  static_assert(NS == 9, "nine digits per value");
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
  for (int p = tid; p < 512; p += 256) {
    // element pairs in address order: k8 (even), r8, K half, row group, K block
    const int e = 2 * p;
    const int k8 = e & 7, r8 = (e >> 3) & 7, kh = (e >> 6) & 1, rgl = (e >> 7) & 3, kbl = e >> 9;
    const int rr = rgl * 8 + r8, kk = kbl * 16 + kh * 8 + k8;
    const int r = r0 + rr, k = k0 + kk;
    if (r >= rpad || k >= kpad) continue;  // kpad is a multiple of 16: the pair is whole
    const int er = r < R ? E[(long long)b * R + r] : OZ_ZERO_EXP;
    uint32_t h0[NS], h1[NS];
    oz_digit_bits(oz_fixed(tile[rr][kk], er), h0);
    oz_digit_bits(oz_fixed(tile[rr][kk + 1], er), h1);
    const int t = r / tile_rows, rt = r - t * tile_rows;
    const int kb = k / OZ_KB;
    uint32_t* q = (uint32_t*)(Q + (((long long)b * ntiles + t) * kblocks + kb) * NS * plane +
                              ((rt >> 3) * 2 + kh) * 64 + r8 * 8 + k8);
#pragma unroll
    for (int i = 0; i < NS; i++) q[i * plane / 2] = h0[i] | (h1[i] << 16);
  }
}

// Exponents and digit planes of an operand, in one pass, where either K is
// contiguous (element (r, k) at X[b sb + r sr + k], RC = false) or the rows
// are (at X[b sb + r + k sk], RC = true): a CTA takes one row group (8 rows)
// whole.  With K contiguous each warp reads one row; with the rows
// contiguous each K position's 8 values (64 bytes) are read by 8
// consecutive threads.  The values go to shared memory and each row's
// largest magnitude is reduced; then the CTA writes the group's digits core
// matrix by core matrix (two elements per thread and plane, 128 contiguous
// bytes per 32 threads).  Rows past R (the padding of the last tile) are
// zero digits.  With gridDim.z > 1 (few row groups) the K blocks are shared
// out over the z CTAs of a group, each reading the whole rows for their
// exponents.
template <int NS, bool RC>
__global__ void __launch_bounds__(256) oz_slice_rows_kernel(int R, int K, const double* __restrict__ X, long long sx,
                                                            long long sb, int* __restrict__ E,
                                                            __nv_bfloat16* __restrict__ Q, int tile_rows, int ntiles,
                                                            int kblocks, const int* __restrict__ active,
                                                            int active_iter) {
  static_assert(NS == 9, "nine digits per value");
  extern __shared__ double oz_rows[];
  __shared__ int es[8];
  __shared__ unsigned long long part[8][8];
  const int b = blockIdx.y, r0 = blockIdx.x * 8;
  if (oz_skip(active, active_iter, b)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kpad = kblocks * OZ_KB, ld = kpad + 1;
  if (!RC) {
    // sx: the row stride
    const int r = r0 + warp;
    const double* x = X + (long long)b * sb + (long long)r * sx;
    unsigned long long mx = 0;
    for (int k = lane; k < kpad; k += 32) {
      const double v = (r < R && k < K) ? __ldg(x + k) : 0.0;
      oz_rows[warp * ld + k] = v;
      const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
      mx = a > mx ? a : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = t > mx ? t : mx;
    }
    const int e = r < R ? oz_exp_of(mx) : OZ_ZERO_EXP;
    if (lane == 0) {
      es[warp] = e;
      if (r < R && blockIdx.z == 0) E[(long long)b * R + r] = e;
    }
  } else {
    // sx: the K stride; thread t reads row r0 + t % 8 at K positions t / 8 + 32 j
    const int r8 = threadIdx.x & 7, r = r0 + r8;
    const double* x = X + (long long)b * sb + r;
    unsigned long long mx = 0;
    for (int k = threadIdx.x >> 3; k < kpad; k += 32) {
      const double v = (r < R && k < K) ? __ldg(x + (long long)k * sx) : 0.0;
      oz_rows[r8 * ld + k] = v;
      const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
      mx = a > mx ? a : mx;
    }
    // lanes with the same row: lane % 8 equal
#pragma unroll
    for (int o = 8; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = t > mx ? t : mx;
    }
    if (lane < 8) part[warp][lane] = mx;
    __syncthreads();
    if (threadIdx.x < 8) {
      const int rr = r0 + threadIdx.x;
      unsigned long long m = 0;
#pragma unroll
      for (int w = 0; w < 8; w++) m = part[w][threadIdx.x] > m ? part[w][threadIdx.x] : m;
      const int e = rr < R ? oz_exp_of(m) : OZ_ZERO_EXP;
      es[threadIdx.x] = e;
      if (rr < R && blockIdx.z == 0) E[(long long)b * R + rr] = e;
    }
  }
  __syncthreads();
  const int t = r0 / tile_rows, rt = r0 - t * tile_rows;
  const long long plane = (long long)tile_rows * OZ_KB;
  __nv_bfloat16* qb = Q + ((long long)b * ntiles + t) * kblocks * NS * plane + (rt >> 3) * 2 * 64;
  const int kb0 = (int)((long long)kblocks * blockIdx.z / gridDim.z),
            kb1 = (int)((long long)kblocks * (blockIdx.z + 1) / gridDim.z);
  for (int p = kb0 * 64 + threadIdx.x; p < kb1 * 64; p += 256) {
    // element pairs in address order: k8 (even), r8, K half, K block
    const int e = 2 * p;
    const int k8 = e & 7, r8 = (e >> 3) & 7, ci = e >> 6;
    const int kb = ci >> 1, kh = ci & 1, k = kb * 16 + kh * 8 + k8;
    const int er = es[r8];
    uint32_t h0[NS], h1[NS];
    oz_digit_bits(oz_fixed(oz_rows[r8 * ld + k], er), h0);
    oz_digit_bits(oz_fixed(oz_rows[r8 * ld + k + 1], er), h1);
    uint32_t* q = (uint32_t*)(qb + (long long)kb * NS * plane + kh * 64 + r8 * 8 + k8);
#pragma unroll
    for (int i = 0; i < NS; i++) q[i * plane / 2] = h0[i] | (h1[i] << 16);
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
  const int nt = oz_tiles(o.rows, o.tile_rows), kbl = oz_kblocks(o.K);
  if ((sk == 1 || sr == 1) && o.K <= kOzMaxK) {
    // K or the rows contiguous: exponents and digits in one pass, one row
    // group per CTA
    const size_t smem = (size_t)8 * (kbl * OZ_KB + 1) * sizeof(double);
    const long long groups = (long long)(nt * o.tile_rows) / 8 * o.batch;
    const int zs = (int)std::max<long long>(1, std::min<long long>(kbl, (kOzSliceCtas + groups - 1) / groups));
    const dim3 grid((nt * o.tile_rows) / 8, o.batch, zs);
    cudaError_t e;
    if (sk == 1) {
      e = set_smem_once((const void*)oz_slice_rows_kernel<kOzSlices, false>, smem);
      if (e != cudaSuccess) return e;
      count_launch();
      oz_slice_rows_kernel<kOzSlices, false><<<grid, 256, smem, st>>>(o.rows, o.K, X, sr, sb, o.E, o.Q, o.tile_rows,
                                                                      nt, kbl, active, active_iter);
    } else {
      e = set_smem_once((const void*)oz_slice_rows_kernel<kOzSlices, true>, smem);
      if (e != cudaSuccess) return e;
      count_launch();
      oz_slice_rows_kernel<kOzSlices, true><<<grid, 256, smem, st>>>(o.rows, o.K, X, sk, sb, o.E, o.Q, o.tile_rows,
                                                                     nt, kbl, active, active_iter);
    }
    return cudaGetLastError();
  }
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
  dim3 grid(oz_grid((long long)kbl * OZ_KB, 32), oz_grid((long long)nt * o.tile_rows, 32), o.batch);
  count_launch();
  oz_slice_kernel<kOzSlices><<<grid, 256, 0, st>>>(o.rows, o.K, X, sr, sk, sb, o.E, o.Q, o.tile_rows, nt, kbl, active,
                                                   active_iter);
  return cudaGetLastError();
}

namespace {
template <int BN, bool XO>
cudaError_t oz_launch(const OzSliced& A, const OzSliced& B, OzGemm p, int sm_count, cudaStream_t st, cudaEvent_t ev0,
                      cudaEvent_t ev1) {
  constexpr int NS = kOzSlices;
  using Cfg = OzCfg<NS, BN>;
  p.EA = A.E;
  p.EB = B.E;
  cudaError_t e = set_smem_once((const void*)ozgemm_kernel<NS, BN, XO>, Cfg::SMEM);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)oz_tiles(p.N, BN) * oz_tiles(p.M, OZ_TBM) * p.batch;
  const int grid = (int)std::min<long long>(tiles, sm_count > 0 ? sm_count : 1);
  if (ev0 != nullptr) {
    e = cudaEventRecord(ev0, st);
    if (e != cudaSuccess) return e;
  }
  count_launch();
  ozgemm_kernel<NS, BN, XO><<<grid, OZ_THREADS, Cfg::SMEM, st>>>(p, A.Q, B.Q, oz_kblocks(p.K));
  e = cudaGetLastError();
  if (e == cudaSuccess && ev1 != nullptr) e = cudaEventRecord(ev1, st);
  return e;
}
}  // namespace

cudaError_t oz_multiply(const OzSliced& A, const OzSliced& B, const OzGemm& p, int sm_count, cudaStream_t st,
                        cudaEvent_t ev0, cudaEvent_t ev1) {
  if (p.M <= 0 || p.N <= 0 || p.batch <= 0) return cudaSuccess;
  if (A.tile_rows != OZ_TBM || A.rows != p.M || B.rows != p.N || A.K != p.K || B.K != p.K || A.batch != p.batch ||
      B.batch != p.batch || p.K > kOzMaxK)
    return cudaErrorInvalidValue;
  if (p.x.nx < 0 || p.x.nx > 4 || (p.x.nx > 0 && p.transC) || (p.C == nullptr && (p.x.nx == 0 || p.beta != 0.0)))
    return cudaErrorInvalidValue;
  for (int w = 0; w < p.x.nx; w++)
    if (p.x.X[w] == nullptr) return cudaErrorInvalidValue;
  if (p.x.nx > 0) {
    if (B.tile_rows == kOzBN) return oz_launch<kOzBN, true>(A, B, p, sm_count, st, ev0, ev1);
    if (B.tile_rows == kOzBNMid) return oz_launch<kOzBNMid, true>(A, B, p, sm_count, st, ev0, ev1);
    if (B.tile_rows == kOzBNSmall) return oz_launch<kOzBNSmall, true>(A, B, p, sm_count, st, ev0, ev1);
    return cudaErrorInvalidValue;
  }
  if (B.tile_rows == kOzBN) return oz_launch<kOzBN, false>(A, B, p, sm_count, st, ev0, ev1);
  if (B.tile_rows == kOzBNMid) return oz_launch<kOzBNMid, false>(A, B, p, sm_count, st, ev0, ev1);
  if (B.tile_rows == kOzBNSmall) return oz_launch<kOzBNSmall, false>(A, B, p, sm_count, st, ev0, ev1);
  return cudaErrorInvalidValue;
}

int oz_bn_for(int N) { return N <= 16 ? kOzBNSmall : (N <= 64 ? kOzBNMid : kOzBN); }

size_t oz_scratch_bytes(int M, int N, int K, int batch) {
  return oz_sliced_bytes(M, K, batch, OZ_TBM) + oz_sliced_bytes(N, K, batch, oz_bn_for(N));
}

cudaError_t ozgemm_f64(const OzGemm& p, void* scratch, size_t scratch_bytes, int sm_count, cudaStream_t st,
                       cudaEvent_t ev0, cudaEvent_t ev1) {
  if (p.M <= 0 || p.N <= 0 || p.batch <= 0) return cudaSuccess;
  if (p.K <= 0 || p.K > kOzMaxK) return cudaErrorInvalidValue;
  if (scratch_bytes < oz_scratch_bytes(p.M, p.N, p.K, p.batch)) return cudaErrorInvalidValue;
  const OzSliced A = oz_carve(scratch, p.M, p.K, p.batch, OZ_TBM);
  const OzSliced B =
      oz_carve((uint8_t*)scratch + oz_sliced_bytes(p.M, p.K, p.batch, OZ_TBM), p.N, p.K, p.batch, oz_bn_for(p.N));
  // A's rows; B's columns (B element (k, c) is row c, position k of B^T)
  cudaError_t e = oz_slice(p.A, p.a_sm, p.a_sk, p.sA, A, p.active, p.active_iter, st);
  if (e == cudaSuccess) e = oz_slice(p.B, p.b_sn, p.b_sk, p.sB, B, p.active, p.active_iter, st);
  if (e != cudaSuccess) return e;
  return oz_multiply(A, B, p, sm_count, st, ev0, ev1);
}

}  // namespace lb
