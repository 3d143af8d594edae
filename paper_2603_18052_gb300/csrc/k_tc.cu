// Batched complex GEMM on the 5th-generation tensor cores (tcgen05), in the
// split-BF16 x3 form:  every FP64 operand x is stored as two BF16 numbers,
// x ~ hi + lo (hi = bf16(x), lo = bf16(x - hi)), and a real product is
// A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in TMEM.  A
// complex product needs the four real products of (Ar + i Ai)(Br + i Bi):
// with the real and imaginary planes of a B piece stacked along N, one MMA
// of width 2 BN gives Ar [Br | Bi] and one gives Ai [Br | Bi] (two TMEM
// accumulators), and the epilogue forms Re = Ar Br - Ai Bi and
// Im = Ar Bi + Ai Br; 2 MMAs per piece pair and K step.
//
// Operands are pre-split "plane" tensors: for a batch of S complex R x K
// matrices, bf16 [S][4][R][ld] with planes (re_hi, re_lo, im_hi, im_lo) and
// K contiguous (K-major).  For C = X Y the A operand is X and the B operand
// is Y^T (both K-major).  TMA loads 64-wide K blocks with the 128-byte swizzle
// into a two-stage shared-memory ring: warp 0 issues the copies, one thread of
// warp 1 issues the MMAs, and after the last K block all eight warps read the
// 128 x BN accumulator tile out of TMEM and apply the epilogue (FP32
// arithmetic, FP64 outputs by exact widening)
//   C  = alpha acc + sum_t coef_t X_t + gamma I + beta C
//   C2 = alpha2 acc + sum_t coef2_t X_t + gamma2 I          (optional)
// and optionally write the split planes of C (row-major and/or transposed)
// for the next product.  Every mbarrier wait is bounded; a wait that gives up
// sets the error word and the CTA still frees its TMEM.
#include "lb_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

namespace lb {

namespace {

constexpr int TBM = 128;           // rows per tile (M of one MMA)
constexpr int TBK = 64;            // K per stage (128 bytes of BF16)
constexpr int NSTAGE = 2;
constexpr int TC_THREADS = 256;   // warps 0-3 and 4-7 share the epilogue
constexpr int A_PLANE = TBM * 128;  // bytes per A plane per stage
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

// Shared memory of one configuration: NPA / NPB BF16 pieces per real value of
// the A / B operand (re and im planes each), BN columns per tile.
template <int NPA, int NPB, int BN>
struct TcCfg {
  static constexpr int B_PLANE = BN * 128;
  static constexpr int STAGE_BYTES = 2 * NPA * A_PLANE + 2 * NPB * B_PLANE;
  static constexpr int SMEM = NSTAGE * STAGE_BYTES + 1024;
  static_assert(TBM * (BN + 1) * 8 <= NSTAGE * STAGE_BYTES, "epilogue tile must fit in the ring");
  // residual tile prefetched behind the ring (light epilogue), if it fits
  static constexpr int XTILE = TBM * BN * 8;
  static constexpr bool XPRE_FITS = SMEM + XTILE + 4096 <= 232448;
  // split-K partials staged in the ring behind the epilogue tile
  static constexpr int PART_OFF = (TBM * (BN + 1) * 8 + 1023) / 1024 * 1024;
  static constexpr int PART_SMEM = (NSTAGE * STAGE_BYTES - PART_OFF) / (TBM * BN * 8);
};

__device__ __forceinline__ void cpa8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((uint32_t)__cvta_generic_to_shared(s)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cpa16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(s)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cpa_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Programmatic dependent launch (propagation steps): the B operand (D
// planes, written before the chain) is fetched before griddep_wait(); the
// states, the X term and every global write come after it.  Both are no-ops
// for an ordinary launch.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t ph) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(ph)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t ph) {
  if (mbar_try(bar, ph)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, ph))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__host__ __device__ constexpr uint32_t idesc(int negA, int bn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)negA << 13) | ((uint32_t)(bn >> 3) << 17) |
         ((uint32_t)(TBM >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void tma3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, float* v) {
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

// x ~ hi + lo, both BF16, computed in FP32 (the residual x - hi is exact).
__device__ __forceinline__ void split2f(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Exact FP32 -> FP64 widening with integer operations only (FP64 arithmetic
// runs at 1/64 of the FP32 rate on this part).  FP32 subnormals become 0.
__device__ __forceinline__ double widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint32_t ex = (u >> 23) & 0xFFu;
  const uint64_t man = (uint64_t)(u & 0x7FFFFFu) << 29;
  uint64_t d;
  if (ex == 0)
    d = sign;
  else if (ex == 255)
    d = sign | 0x7FF0000000000000ull | man;
  else
    d = sign | ((uint64_t)(ex + 896) << 52) | man;
  return __longlong_as_double((long long)d);
}

__device__ __forceinline__ void put_planes(__nv_bfloat16* base, long long idx, long long plane, float re, float im) {
  __nv_bfloat16 h, l;
  split2f(re, h, l);
  base[idx] = h;
  base[idx + plane] = l;
  split2f(im, h, l);
  base[idx + 2 * plane] = h;
  base[idx + 3 * plane] = l;
}

// Planes of four consecutive elements (idx a multiple of 4, 8-byte aligned):
// one 8-byte store per plane.
__device__ __forceinline__ void put_planes4(__nv_bfloat16* base, long long idx, long long plane, const float* re,
                                            const float* im) {
  __nv_bfloat16 h[4], l[4], hi_[4], li_[4];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    split2f(re[j], h[j], l[j]);
    split2f(im[j], hi_[j], li_[j]);
  }
  auto pack = [](const __nv_bfloat16* v) {
    uint2 w;
    w.x = (uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16);
    w.y = (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16);
    return w;
  };
  *(uint2*)(base + idx) = pack(h);
  *(uint2*)(base + idx + plane) = pack(l);
  *(uint2*)(base + idx + 2 * plane) = pack(hi_);
  *(uint2*)(base + idx + 3 * plane) = pack(li_);
}

// Products kept: pieces (i, j) with i + j < max(NPA, NPB): for two pieces
// each, hi*hi + hi*lo + lo*hi; for a three-piece B also the two products
// that carry B's third piece.
template <int NPA, int NPB, int TBN, bool LIGHT>
__global__ void __launch_bounds__(TC_THREADS) zgemm_tc_kernel(const __grid_constant__ CUtensorMap mapA,
                                                       const __grid_constant__ CUtensorMap mapB,
                                                       const __grid_constant__ TcProblem P, int ksplit, int kbps) {
  using Cfg = TcCfg<NPA, NPB, TBN>;
  constexpr int B_PLANE = Cfg::B_PLANE;
  constexpr int STAGE_BYTES = Cfg::STAGE_BYTES;
  constexpr int NPMAX = NPA > NPB ? NPA : NPB;
  if (P.active != nullptr && P.active[blockIdx.z / ksplit] <= P.active_iter) return;  // whole CTA, before any setup
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[NSTAGE], empty_bar[NSTAGE], acc_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int give_up, last_cta;
  __shared__ float2 rscale[TBM];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * TBN, m0 = blockIdx.y * TBM, b = blockIdx.z / ksplit, zs = blockIdx.z % ksplit;
  const int nkt = (P.K + TBK - 1) / TBK;
  // B planes sit in the ring as [Br_0, Bi_0, Br_1, Bi_1, ...]: each piece's
  // [Br; Bi] is one 2 TBN-row operand (tensor plane p: Re pieces first)
  auto bslot = [](int p) { return p < NPB ? 2 * p : 2 * (p - NPB) + 1; };
  const int kb0 = zs * kbps;                           // this CTA's K blocks [kb0, kb0 + nk)
  const int nk = min(nkt, kb0 + kbps) - kb0;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty_bar[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&acc_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    give_up = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(4 * TBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tacc = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer: TMA copies of the K blocks into the ring; the B planes of
    // the first stages go out before the wait for the previous grid
    const int pre = nk < NSTAGE ? nk : NSTAGE;
    for (int kb = 0; kb < pre; kb++) {
      const uint32_t base = su32(sm + kb * STAGE_BYTES);
      const uint32_t fb = su32(&full_bar[kb]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE_BYTES) : "memory");
      for (int p = 0; p < 2 * NPB; p++)
        tma3(base + 2 * NPA * A_PLANE + bslot(p) * B_PLANE, &mapB, (kb0 + kb) * TBK, n0, b * 2 * NPB + p, fb);
    }
    griddep_wait();
    for (int kb = 0; kb < pre; kb++) {
      const uint32_t base = su32(sm + kb * STAGE_BYTES);
      const uint32_t fb = su32(&full_bar[kb]);
      for (int p = 0; p < 2 * NPA; p++) tma3(base + p * A_PLANE, &mapA, (kb0 + kb) * TBK, m0, b * 2 * NPA + p, fb);
    }
    for (int kb = pre; kb < nk; kb++) {
      const int s = kb % NSTAGE;
      const int kx = (kb0 + kb) * TBK;
      if (!mbar_wait(su32(&empty_bar[s]), ((kb - NSTAGE) / NSTAGE) & 1)) {
        atomicOr(P.err, ERR_TIMEOUT);
        give_up = 1;
        break;
      }
      const uint32_t base = su32(sm + s * STAGE_BYTES);
      const uint32_t fb = su32(&full_bar[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE_BYTES) : "memory");
      for (int p = 0; p < 2 * NPA; p++) tma3(base + p * A_PLANE, &mapA, kx, m0, b * 2 * NPA + p, fb);
      for (int p = 0; p < 2 * NPB; p++)
        tma3(base + 2 * NPA * A_PLANE + bslot(p) * B_PLANE, &mapB, kx, n0, b * 2 * NPB + p, fb);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    // accumulators: Ar [Br | Bi] in columns [0, 2 TBN), Ai [Br | Bi] in [2 TBN, 4 TBN)
    const uint32_t tA = tacc, tB = tacc + 2 * TBN;
    bool ok = true;
    for (int kb = 0; kb < nk && ok; kb++) {
      const int s = kb % NSTAGE;
      if (!mbar_wait(su32(&full_bar[s]), (kb / NSTAGE) & 1)) {
        atomicOr(P.err, ERR_TIMEOUT);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = su32(sm + s * STAGE_BYTES);
      const uint32_t bb = base + 2 * NPA * A_PLANE;
#pragma unroll
      for (int k = 0; k < TBK / 16; k++) {
        const uint32_t o = k * 32;
        const uint32_t first = (kb > 0 || k > 0) ? 1u : 0u;
        bool started = false;
#pragma unroll
        for (int i = 0; i < NPA; i++)
#pragma unroll
          for (int j = 0; j < NPB; j++) {
            if (i + j >= NPMAX) continue;
            const uint64_t Ar = desc_sw128(base + i * A_PLANE + o), Ai = desc_sw128(base + (NPA + i) * A_PLANE + o);
            const uint64_t Bj = desc_sw128(bb + 2 * j * B_PLANE + o);  // [Br_j ; Bi_j], 2 TBN rows
            const uint32_t acc = started ? 1u : first;
            mma(tA, Ar, Bj, idesc(0, 2 * TBN), acc);
            mma(tB, Ai, Bj, idesc(0, 2 * TBN), acc);
            started = true;
          }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       su32(&empty_bar[s]))
                   : "memory");
    }
    if (!ok) give_up = 1;
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&acc_bar))
                 : "memory");
  }
  constexpr bool XPRE = LIGHT && Cfg::XPRE_FITS;
  float2* xs = (float2*)(sm + NSTAGE * STAGE_BYTES);  // residual tile (XPRE)
  if (warp >= 2) griddep_wait();  // the X tile and the trace read the previous grid's output
  if (XPRE && warp >= 2 && P.nterms > 0) {
    // the residual tile X[0] (rows m0.., columns n0..) into shared memory,
    // copied by the two warps that are idle while the K loop runs
    const float2* x0 = P.X[0] + (long long)b * P.sX[0];
    if (P.ldc % 2 == 0 && P.sX[0] % 2 == 0 && ((uintptr_t)P.X[0] & 15) == 0) {
      for (int e = 2 * (tid - 64); e < TBM * TBN; e += 2 * (TC_THREADS - 64)) {  // pairs: 16-byte copies
        const int row = m0 + e / TBN, col = n0 + e % TBN;
        if (row >= P.M || col >= P.N) continue;
        if (col + 1 < P.N)
          cpa16(xs + e, x0 + (long long)row * P.ldc + col);
        else
          cpa8(xs + e, x0 + (long long)row * P.ldc + col);
      }
    } else {
      for (int e = tid - 64; e < TBM * TBN; e += TC_THREADS - 64) {
        const int row = m0 + e / TBN, col = n0 + e % TBN;
        if (row < P.M && col < P.N) cpa8(xs + e, x0 + (long long)row * P.ldc + col);
      }
    }
    cpa_wait_all();
  }
  if (warp >= 2 && P.rs_src != nullptr) {
    // per-row factor 1 / Tr (rows m0 .. m0 + 127), computed by the warps
    // that are idle while the K loop runs
    for (int r = tid - 64; r < TBM; r += TC_THREADS - 64) {
      float2 c = make_float2(1.f, 0.f);
      const int row = m0 + r;
      if (row < P.M) {
        const float2* x = P.rs_src + (long long)b * P.sC + (long long)row * P.ldc;
        const int step = P.rs_d + 1;
        float sr = 0.f, si = 0.f;
        int i = 0;
        for (; i + 4 <= P.rs_d; i += 4) {
          const float2 v0 = __ldg(x + i * step), v1 = __ldg(x + (i + 1) * step);
          const float2 v2 = __ldg(x + (i + 2) * step), v3 = __ldg(x + (i + 3) * step);
          sr += (v0.x + v1.x) + (v2.x + v3.x);
          si += (v0.y + v1.y) + (v2.y + v3.y);
        }
        for (; i < P.rs_d; i++) {
          const float2 v = __ldg(x + i * step);
          sr += v.x;
          si += v.y;
        }
        const float m2 = sr * sr + si * si;
        c = make_float2(sr / m2, -si / m2);
      }
      rscale[r] = c;
    }
  }
  __syncwarp();
  // all warps: wait for the accumulator
  const bool have = mbar_wait(su32(&acc_bar), 0);
  if (!have && tid == 0) atomicOr(P.err, ERR_TIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool good = __syncthreads_and(have ? 1 : 0) && !give_up;  // uniform across the CTA
  griddep_wait();    // every thread: global writes below go to the previous grid's inputs
  griddep_launch();  // the next grid may start its prologue
  // the producer may still have copies in flight after a give-up: wait for
  // them (bounded) before the shared memory is released
  if (!good && tid == 0) {
    for (int s = 0; s < NSTAGE; s++) {
      const int uses = (nk - s + NSTAGE - 1) / NSTAGE;
      if (uses > 0) mbar_wait(su32(&full_bar[s]), (uses - 1) & 1);
    }
  }
  if (good) {
    // The shared-memory ring is idle now (every copy was consumed by an MMA
    // that has completed).  Stage the accumulator tile through it so that the
    // global reads and writes of the epilogue are coalesced.
    constexpr int LDS = TBN + 1;  // padded row of float2
    float2* tile = (float2*)sm;
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its lane quadrant), half
    // w / 4 of the columns
    const int quad = warp & 3, half = warp >> 2;
    for (int c0 = half * (TBN / 2); c0 < (half + 1) * (TBN / 2); c0 += 16) {
      float rr[16], ri[16], ir[16], ii[16];  // Ar Br, Ar Bi, Ai Br, Ai Bi
      const uint32_t ta = tacc + ((uint32_t)(quad * 32) << 16) + c0;
      tmem_ld16(ta, rr);
      tmem_ld16(ta + TBN, ri);
      tmem_ld16(ta + 2 * TBN, ir);
      tmem_ld16(ta + 3 * TBN, ii);
      const int r = quad * 32 + lane;
#pragma unroll
      for (int j = 0; j < 16; j++) tile[r * LDS + c0 + j] = make_float2(rr[j] - ii[j], ri[j] + ir[j]);
    }
    __syncthreads();
  }
  bool emit = good;
  if (ksplit > 1) {
    // split K: every CTA of the tile leaves its partial; the one that takes
    // the last ticket sums them in split order (independent of arrival order)
    constexpr int LDS = TBN + 1;
    float2* tile = (float2*)sm;
    const int tile_id = (b * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    float2* part = P.part + (long long)tile_id * ksplit * TBM * TBN;
    if (good) {
      float4* mine = (float4*)(part + (long long)zs * TBM * TBN);
      for (int e = tid; e < TBM * TBN / 2; e += TC_THREADS) {
        const float2 u = tile[(2 * e / TBN) * LDS + (2 * e) % TBN], v = tile[(2 * e / TBN) * LDS + (2 * e) % TBN + 1];
        mine[e] = make_float4(u.x, u.y, v.x, v.y);
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last_cta = atomicAdd(&P.cnt[tile_id], 1u) == (unsigned)(ksplit - 1);
    __syncthreads();
    emit = good && last_cta;
    if (last_cta) {
      __threadfence();
      constexpr int E4 = TBM * TBN / 2;  // float4 (two complex values) per partial tile
      if (good && ksplit <= Cfg::PART_SMEM) {
        // all partials into the idle ring with every copy in flight, then
        // summed in split order from shared memory
        float4* ps = (float4*)(sm + Cfg::PART_OFF);
        const float4* p4 = (const float4*)part;
        for (int e = tid; e < ksplit * E4; e += TC_THREADS) cpa16(ps + e, p4 + e);
        cpa_wait_all();
        __syncthreads();
        for (int e = tid; e < E4; e += TC_THREADS) {
          float4 a = ps[e];
          for (int z = 1; z < ksplit; z++) {
            const float4 v = ps[z * E4 + e];
            a.x += v.x;
            a.y += v.y;
            a.z += v.z;
            a.w += v.w;
          }
          const int r = 2 * e / TBN, cc = (2 * e) % TBN;
          tile[r * LDS + cc] = make_float2(a.x, a.y);
          tile[r * LDS + cc + 1] = make_float2(a.z, a.w);
        }
      } else if (good) {
        const float4* p4 = (const float4*)part;
#pragma unroll 4
        for (int e = tid; e < E4; e += TC_THREADS) {
          float4 a = __ldcg(p4 + e);
#pragma unroll
          for (int z = 1; z < 8; z++) {  // ksplit <= 8
            if (z < ksplit) {
              const float4 v = __ldcg(p4 + (long long)z * E4 + e);
              a.x += v.x;
              a.y += v.y;
              a.z += v.z;
              a.w += v.w;
            }
          }
          const int r = 2 * e / TBN, cc = (2 * e) % TBN;
          tile[r * LDS + cc] = make_float2(a.x, a.y);
          tile[r * LDS + cc + 1] = make_float2(a.z, a.w);
        }
      }
      if (tid == 0) P.cnt[tile_id] = 0u;
      __syncthreads();
    }
  }
  if (emit) {
    constexpr int LDS = TBN + 1;
    float2* tile = (float2*)sm;
    const long long bs = (long long)b;
    // row-major pass: consecutive threads take consecutive columns.  FP32
    // arithmetic only; FP64 outputs are exact widenings plus the FP64
    // diagonal term.  The X terms of EU elements are loaded before any of
    // them is stored (the outputs may alias nothing the compiler can prove),
    // so one L2 round trip covers EU elements.
    // Each thread takes quads of four consecutive columns of one row, so the
    // FP32 output and the BF16 planes go out as 16- and 8-byte stores (one
    // store instruction per quad and plane instead of one per element);
    // ragged or misaligned quads fall back to element stores.  The X terms of
    // QU quads are read before any of them is stored.
    constexpr int QR = TBN / 4;          // quads per row
    constexpr int QU = LIGHT ? 4 : 2;    // quads per thread per batch
    static_assert((TBM * QR) % (TC_THREADS * QU) == 0, "epilogue batches");
    const int nterms = LIGHT ? (P.nterms > 0 ? 1 : 0) : P.nterms;
    const bool cf_vec = P.Cf != nullptr && P.ldc % 2 == 0 && P.sC % 2 == 0 && ((uintptr_t)P.Cf & 15) == 0;
    const bool sp_vec = P.sp != nullptr && P.sp_ld % 4 == 0 && P.sp_plane % 4 == 0 && ((uintptr_t)P.sp & 7) == 0;
    for (int e0 = tid; e0 < TBM * QR; e0 += TC_THREADS * QU) {
      float2 xv[4][QU][4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        if (q < nterms) {  // uniform: X[q] is set
          const float2* xq = P.X[q] + bs * P.sX[q];
#pragma unroll
          for (int u = 0; u < QU; u++) {
            const int e4 = e0 + TC_THREADS * u;
            const int r = e4 / QR, cq = (e4 % QR) * 4;
#pragma unroll
            for (int j = 0; j < 4; j++) {
              if (XPRE) {
                xv[q][u][j] = xs[r * TBN + cq + j];
              } else {
                const int row = min(m0 + r, P.M - 1), col = min(n0 + cq + j, P.N - 1);  // in bounds
                xv[q][u][j] = __ldg(xq + (long long)row * P.ldc + col);
              }
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < QU; u++) {
        const int e4 = e0 + TC_THREADS * u;
        const int r = e4 / QR, cq = (e4 % QR) * 4;
        const int row = m0 + r, col = n0 + cq;
        if (row >= P.M || col >= P.N) continue;
        const bool full = col + 3 < P.N;
        float cr[4], ci[4], dr[4], di[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const float2 a2 = tile[r * LDS + cq + j];
          cr[j] = P.alpha * a2.x;
          ci[j] = P.alpha * a2.y;
          dr[j] = P.alpha2 * a2.x;
          di[j] = P.alpha2 * a2.y;
#pragma unroll
          for (int q = 0; q < 4; q++) {
            if (q < nterms) {
              cr[j] = fmaf(P.coef[q], xv[q][u][j].x, cr[j]);
              ci[j] = fmaf(P.coef[q], xv[q][u][j].y, ci[j]);
              if (!LIGHT) {
                dr[j] = fmaf(P.coef2[q], xv[q][u][j].x, dr[j]);
                di[j] = fmaf(P.coef2[q], xv[q][u][j].y, di[j]);
              }
            }
          }
          if (P.rs_src != nullptr) {
            const float2 c = rscale[r];
            const float t = cr[j] * c.x - ci[j] * c.y;
            ci[j] = cr[j] * c.y + ci[j] * c.x;
            cr[j] = t;
          }
        }
        const long long off = bs * P.sC + (long long)row * P.ldc + col;
        if (P.Cf != nullptr) {
          if (cf_vec && full) {
            float4* d4 = (float4*)(P.Cf + off);
            d4[0] = make_float4(cr[0], ci[0], cr[1], ci[1]);
            d4[1] = make_float4(cr[2], ci[2], cr[3], ci[3]);
          } else {
#pragma unroll
            for (int j = 0; j < 4; j++)
              if (col + j < P.N) P.Cf[off + j] = make_float2(cr[j], ci[j]);
          }
        }
        if (!LIGHT) {
          // FP64 outputs: exact widening only; the diagonal terms are added
          // in a separate pass (FP64 arithmetic costs 64 cycles per warp
          // instruction, taken or not)
#pragma unroll
          for (int j = 0; j < 4; j++) {
            if (col + j >= P.N) continue;
            if (P.Cd != nullptr) P.Cd[off + j] = make_double2(widen(cr[j]), widen(ci[j]));
            if (P.C2d != nullptr) P.C2d[off + j] = make_double2(widen(dr[j]), widen(di[j]));
          }
        }
        if (P.sp != nullptr) {
          float pr[4];
#pragma unroll
          for (int j = 0; j < 4; j++) pr[j] = (row == col + j) ? cr[j] - P.sp_shift : cr[j];
          const long long idx = bs * 4 * P.sp_plane + (long long)row * P.sp_ld + col;
          if (sp_vec && full) {
            put_planes4(P.sp, idx, P.sp_plane, pr, ci);
          } else {
#pragma unroll
            for (int j = 0; j < 4; j++)
              if (col + j < P.N) put_planes(P.sp, idx + j, P.sp_plane, pr[j], ci[j]);
          }
        }
        if (!LIGHT && P.spT != nullptr) {
#pragma unroll
          for (int j = 0; j < 4; j++)
            tile[r * LDS + cq + j] = make_float2(row == col + j ? cr[j] - P.spT_shift : cr[j], ci[j]);
        }
      }
    }
    if (!LIGHT && (P.Cd != nullptr || P.C2d != nullptr)) {
      // diagonal of the tile: + gamma, + gamma2 (this thread's own stores
      // above are visible to the CTA after the barrier)
      __syncthreads();
      const int dg = m0 + tid;
      if (tid < TBM && dg >= n0 && dg < n0 + TBN && dg < P.M && dg < P.N) {
        const long long off = bs * P.sC + (long long)dg * P.ldc + dg;
        if (P.Cd != nullptr) P.Cd[off].x += P.gamma;
        if (P.C2d != nullptr) P.C2d[off].x += P.gamma2;
      }
    }
    if (!LIGHT && P.spT != nullptr) {
      // transposed planes (B-operand layout): consecutive threads take
      // consecutive rows, which are contiguous in the transpose
      __syncthreads();
      for (int e = tid; e < TBM * TBN; e += TC_THREADS) {
        const int cc = e / TBM, r = e - (e / TBM) * TBM;
        const int row = m0 + r, col = n0 + cc;
        if (row >= P.M || col >= P.N) continue;
        const float2 v = tile[r * LDS + cc];
        put_planes(P.spT, bs * 4 * P.spT_plane + (long long)col * P.spT_ld + row, P.spT_plane, v.x, v.y);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tacc), "r"(4 * TBN));
}

// Split planes of a batch of complex FP64 matrices: dst[s][p][r][c] for the
// row-major form, or of the transpose (dst[s][p][c][r]) when trans != 0,
// with `shift` subtracted from the diagonal first; np BF16 pieces per value
// (the value is rounded to FP32 once, then split in FP32).  f32 (optional)
// receives the FP32 copy, row-major.
__global__ void split_kernel(int R, int Kc, long long total, const z64* __restrict__ src, long long lds,
                             long long ss, double shift, int trans, __nv_bfloat16* __restrict__ dst, long long ldd,
                             long long plane, int np, float2* __restrict__ f32) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long per = (long long)R * Kc;
    const long long s = e / per;
    const long long o = e - s * per;
    long long r, c;
    if (trans) {  // consecutive threads along r: coalesced writes of the transpose
      c = o / R;
      r = o - c * R;
    } else {
      r = o / Kc;
      c = o - r * Kc;
    }
    z64 v = src[s * ss + r * lds + c];
    if (r == c) v.x -= shift;
    float xr = (float)v.x, xi = (float)v.y;
    if (f32 != nullptr) f32[s * per + r * Kc + c] = make_float2(xr, xi);
    const long long d = s * 2 * np * plane + (trans ? c * ldd + r : r * ldd + c);
    for (int p = 0; p < np; p++) {  // x = sum of np BF16 pieces, each the rounding of what is left
      const __nv_bfloat16 hr = __float2bfloat16_rn(xr), hi = __float2bfloat16_rn(xi);
      dst[d + p * plane] = hr;
      dst[d + (np + p) * plane] = hi;
      xr -= __bfloat162float(hr);
      xi -= __bfloat162float(hi);
    }
  }
}

// Z = c0 X0 + c1 X1 + c2 X2 (FP32, n x n per slice), written only as the
// two-piece planes of its transpose (B-operand layout).
__global__ void lincomb_splitT_kernel(int n, long long total, const float2* __restrict__ X0,
                                      const float2* __restrict__ X1, const float2* __restrict__ X2, float c0, float c1,
                                      float c2, __nv_bfloat16* __restrict__ dst, long long ldd, long long plane) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / nn;
    const long long o = e - s * nn;
    const long long c = o / n, r = o - (o / n) * n;  // consecutive threads along r
    const long long i = s * nn + r * n + c;
    const float2 a = X0[i], b = X1[i], g = X2[i];
    const float zr = fmaf(c0, a.x, fmaf(c1, b.x, c2 * g.x)), zi = fmaf(c0, a.y, fmaf(c1, b.y, c2 * g.y));
    put_planes(dst, s * 4 * plane + c * ldd + r, plane, zr, zi);
  }
}

// One warp per state (FP32): optional division by the trace, then the
// state's two-piece planes (row b of the [4][B][ld] plane tensor).
__global__ void renorm_split_kernel(int n, int d, int B, int renorm, float2* __restrict__ X, long long xld,
                                    __nv_bfloat16* __restrict__ planes, long long ld, long long plane) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= B) return;
  float2* x = X + (long long)w * xld;
  float cr = 1.f, ci = 0.f;
  if (renorm) {
    float sr = 0.f, si = 0.f;
    for (int k = lane; k < d; k += 32) {
      sr += x[k * (d + 1)].x;
      si += x[k * (d + 1)].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    const float m2 = sr * sr + si * si;
    cr = sr / m2;
    ci = -si / m2;
  }
  for (int e = lane; e < n; e += 32) {
    float2 v = x[e];
    if (renorm) {
      v = make_float2(v.x * cr - v.y * ci, v.x * ci + v.y * cr);
      x[e] = v;
    }
    put_planes(planes, (long long)w * ld + e, plane, v.x, v.y);
  }
}

// states: complex128 rows of n (stride n) <-> FP32 rows of n (stride ld >= n)
__global__ void states_c64_to_f32_kernel(int n, long long total, const z64* __restrict__ a, float2* __restrict__ b,
                                         long long ld) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n, c = e - (e / n) * n;
    b[r * ld + c] = make_float2((float)a[e].x, (float)a[e].y);
  }
}

__global__ void states_f32_to_c64_kernel(int n, long long total, const float2* __restrict__ a, long long ld,
                                         z64* __restrict__ b) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / n, c = e - (e / n) * n;
    const float2 v = a[r * ld + c];
    b[e] = make_double2(widen(v.x), widen(v.y));
  }
}

unsigned grid_for(long long total) {
  long long g = (total + 255) / 256;
  return (unsigned)(g > 152LL * 16 ? 152LL * 16 : (g < 1 ? 1 : g));
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool encode_planes(CUtensorMap* m, const __nv_bfloat16* base, int rows, int K, long long ld, long long plane,
                   int nplanes, int box_rows) {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    else
      cudaGetLastError();
  });
  if (g_encode == nullptr) return false;
  if ((ld * 2) % 16 != 0 || (plane * 2) % 16 != 0 || ((uintptr_t)base & 15) != 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(plane * 2)};
  cuuint32_t box[3] = {(cuuint32_t)TBK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

long long plane_ld(int K) { return ((long long)K + 7) / 8 * 8; }

cudaError_t launch_split(int R, int Kc, int S, const z64* src, long long lds, long long ss, double shift, int trans,
                         __nv_bfloat16* dst, long long ldd, long long plane, cudaStream_t st, int np, float2* f32) {
  const long long total = (long long)R * Kc * S;
  count_launch();
  split_kernel<<<grid_for(total), 256, 0, st>>>(R, Kc, total, src, lds, ss, shift, trans, dst, ldd, plane, np, f32);
  return cudaGetLastError();
}

cudaError_t launch_lincomb_splitT(int n, int S, const float2* X0, const float2* X1, const float2* X2, float c0,
                                  float c1, float c2, __nv_bfloat16* dst, long long ldd, long long plane,
                                  cudaStream_t st) {
  const long long total = (long long)n * n * S;
  count_launch();
  lincomb_splitT_kernel<<<grid_for(total), 256, 0, st>>>(n, total, X0, X1, X2, c0, c1, c2, dst, ldd, plane);
  return cudaGetLastError();
}

cudaError_t launch_renorm_split(int n, int d, int B, int renorm, float2* X, long long xld, __nv_bfloat16* planes,
                                long long ld, long long plane, cudaStream_t st) {
  const int grid = (B * 32 + 255) / 256;
  count_launch();
  renorm_split_kernel<<<grid, 256, 0, st>>>(n, d, B, renorm, X, xld, planes, ld, plane);
  return cudaGetLastError();
}

cudaError_t launch_states_c64_f32(int n, int B, const z64* a, float2* b, long long ld, cudaStream_t st) {
  const long long count = (long long)n * B;
  count_launch();
  states_c64_to_f32_kernel<<<grid_for(count), 256, 0, st>>>(n, count, a, b, ld);
  return cudaGetLastError();
}

cudaError_t launch_states_f32_c64(int n, int B, const float2* a, long long ld, z64* b, cudaStream_t st) {
  const long long count = (long long)n * B;
  count_launch();
  states_f32_to_c64_kernel<<<grid_for(count), 256, 0, st>>>(n, count, a, ld, b);
  return cudaGetLastError();
}

namespace {
template <int NPA, int NPB, int BN, bool LIGHT>
cudaError_t launch_tc(const TcProblem& p, cudaStream_t st) {
  using Cfg = TcCfg<NPA, NPB, BN>;
  static_assert(Cfg::SMEM <= 232448, "shared memory");
  CUtensorMap ma, mb;
  if (!encode_planes(&ma, p.Aop, p.M, p.K, p.a_ld, p.a_plane, 2 * NPA * p.batch, TBM) ||
      !encode_planes(&mb, p.Bop, p.N, p.K, p.b_ld, p.b_plane, 2 * NPB * p.batch, BN))
    return cudaErrorInvalidValue;
  constexpr int SMEM = Cfg::SMEM + ((LIGHT && Cfg::XPRE_FITS) ? Cfg::XTILE : 0);
  cudaError_t e = set_smem_once((const void*)zgemm_tc_kernel<NPA, NPB, BN, LIGHT>, SMEM);
  if (e != cudaSuccess) return e;
  const int gx = (p.N + BN - 1) / BN, gy = (p.M + TBM - 1) / TBM;
  const int tiles = gx * gy * p.batch, nk = (p.K + TBK - 1) / TBK;
  int ksplit = 1;
  if (p.part != nullptr && p.cnt != nullptr && tiles < p.max_ctas)
    ksplit = std::max(1, std::min({p.max_ctas / tiles, nk / 2, 8}));
  const int kbps = (nk + ksplit - 1) / ksplit;
  ksplit = (nk + kbps - 1) / kbps;
  dim3 grid(gx, gy, p.batch * ksplit);
  count_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = p.pdl ? 1 : 0;
  e = cudaLaunchKernelEx(&cfg, zgemm_tc_kernel<NPA, NPB, BN, LIGHT>, ma, mb, p, ksplit, kbps);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}
}  // namespace

cudaError_t zgemm_tc(const TcProblem& p, cudaStream_t st) {
  if (p.M <= 0 || p.N <= 0 || p.batch <= 0) return cudaSuccess;
  // the light epilogue (one X term, FP32 output, row-major planes, row
  // factor) serves the propagation steps
  const bool light = p.nterms <= 1 && p.Cd == nullptr && p.C2d == nullptr && p.spT == nullptr;
  if (p.npa == 2 && p.npb == 2) return light ? launch_tc<2, 2, 64, true>(p, st) : launch_tc<2, 2, 64, false>(p, st);
  if (p.npa == 2 && p.npb == 3) return light ? launch_tc<2, 3, 32, true>(p, st) : launch_tc<2, 3, 32, false>(p, st);
  return cudaErrorInvalidValue;
}

}  // namespace lb
