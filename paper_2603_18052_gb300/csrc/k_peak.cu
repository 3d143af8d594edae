// Arithmetic peak probes: the measured ceilings against which the roofline
// fractions of the benchmark are taken (the paper measures its ceilings with
// probes too, Sec. 3.6, Tables tab:probes_cpu and tab:probes_gpu).
//
//   lb_probe_dfma     FP64 FMA on the CUDA cores (DFMA), the pipe that bounds
//                     every FP64 product of the build and the propagation
//   lb_probe_ffma     FP32 FMA on the CUDA cores (FFMA)
//   lb_probe_dmma     FP64 tensor-core MMA (mma.sync m8n8k4 f64)
//   lb_probe_bf16_tc  BF16 tcgen05 MMA (kind::f16, M = 128, N = 256, K = 16,
//                     FP32 accumulation in TMEM)
//
// The FMA probes run 8 independent dependent chains per thread, 32 warps per
// SM, so the pipe and not the latency is the limit; the MMA probes issue
// back-to-back MMAs on operands that stay in registers (DMMA) or shared
// memory (tcgen05), so no memory traffic enters.  Each probe runs one
// untimed and five timed launches (CUDA events on `stream`) and reports the
// best rate in TFLOP/s (2 FLOPs per multiply-add).  Results that cannot
// occur are the only values stored, into a file-scope sink, so nothing is
// optimised away; no device memory is allocated.  The tcgen05 probe's wait
// for its MMAs is bounded (about 2 s): a wait that gives up reports
// LB_ETIMEOUT and frees the CTA's TMEM.
#include "lb_internal.cuh"

#include <cstdint>

namespace lb {
namespace {

__device__ double g_sink_d;
__device__ float g_sink_f;
__device__ unsigned int g_probe_err;

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 4;

template <typename T>
__device__ __forceinline__ T fma_p(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_p<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_p<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(T x, T y, int iters) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; i++) a[i] = T(threadIdx.x % 7 + i) * T(0.125);
#pragma unroll 4
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = fma_p(a[i], x, y);
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; i++) s += a[i];
  if (s == T(-1.25e-30)) {  // never: every chain converges to y / (1 - x) > 0
    if (sizeof(T) == 8)
      g_sink_d = (double)s;
    else
      g_sink_f = (float)s;
  }
}

__global__ void __launch_bounds__(kProbeThreads) dmma_probe_kernel(double x, int iters) {
  double c[4][2];
#pragma unroll
  for (int q = 0; q < 4; q++) c[q][0] = c[q][1] = 0.0;
  const double a = x, b = x * 0.5;
  for (int it = 0; it < iters; it++)
#pragma unroll
    for (int q = 0; q < 4; q++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[q][0]), "+d"(c[q][1])
                   : "d"(a), "d"(b));
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 4; q++) s += c[q][0] + c[q][1];
  if (s == -1.25e-30) g_sink_d = s;  // never: every accumulator is a sum of positive products
}

// ------------------------------------------------------------- tcgen05 ----
constexpr int kTcM = 128, kTcN = 256, kTcK = 16;
constexpr int kTcOperandBytes = (kTcM + kTcN) * 128;  // one 64-wide K block of A and B (SW128)
// more shared memory than two CTAs fit in, so that one CTA runs per SM and
// its 256 TMEM columns never wait for another CTA's
constexpr int kTcSmem = 120 * 1024;
constexpr long long kTcWaitCycles = 4000000000LL;     // about 2 s

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  // K-major operand, 128-byte swizzle, 8-row groups 1024 bytes apart
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t ph) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(ph)
      : "memory");
  return ok != 0;
}

// One CTA per SM: BF16 operands of one K block in shared memory (zeros),
// `iters` x 4 MMAs of 128 x 256 x 16 into one TMEM accumulator, one commit,
// a bounded wait for it, then the TMEM is freed.
__global__ void __launch_bounds__(128) tc_probe_kernel(int iters) {
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < kTcOperandBytes / 16; e += blockDim.x) ((uint4*)sm)[e] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s32(&done_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(&tmem_base)),
                 "r"(kTcN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeros, visible to the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tacc = tmem_base;
  if (tid == 0) {
    // instruction descriptor: FP32 accumulator, BF16 A and B, K-major both,
    // N = 256, M = 128
    const uint32_t id = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                        ((uint32_t)(kTcM >> 4) << 24);
    const uint32_t a0 = s32(sm), b0 = s32(sm + kTcM * 128);
    for (int it = 0; it < iters; it++)
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const uint64_t da = sw128_desc(a0 + k * 32), db = sw128_desc(b0 + k * 32);
        const uint32_t acc = (it > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
                "r"(tacc),
            "l"(da), "l"(db), "r"(id), "r"(acc));
      }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s32(&done_bar))
                 : "memory");
    bool ok = bar_try(s32(&done_bar), 0);
    if (!ok) {
      const long long t0 = clock64();
      while (!(ok = bar_try(s32(&done_bar), 0)))
        if (clock64() - t0 > kTcWaitCycles) break;
    }
    if (!ok) atomicOr(&g_probe_err, ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tacc), "r"(kTcN));
}

// Best of five timed launches of `launch` (after one untimed), in ms.
template <typename F>
lb_status time_best(F launch, cudaStream_t st, float* best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess) return LB_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LB_ECUDA;
  }
  lb_status r = LB_OK;
  float best = 1e30f;
  for (int rep = 0; rep < 6 && r == LB_OK; rep++) {
    if (cudaEventRecord(e0, st) != cudaSuccess) r = LB_ECUDA;
    if (r == LB_OK && launch() != cudaSuccess) r = LB_ECUDA;
    if (r == LB_OK && cudaEventRecord(e1, st) != cudaSuccess) r = LB_ECUDA;
    if (r == LB_OK && cudaEventSynchronize(e1) != cudaSuccess) r = LB_ECUDA;
    float ms = 0.f;
    if (r == LB_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) r = LB_ECUDA;
    if (r == LB_OK && rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_ms = best;
  return r;
}

}  // namespace
}  // namespace lb

using namespace lb;

extern "C" {

lb_status lb_probe_dfma(double* tflops_out, void* stream) {
  if (tflops_out == nullptr) return LB_EINVAL;
  int dev = 0, sms = 0;
  lb_status r = current_device_sm103(&dev, &sms);
  if (r != LB_OK) return r;
  const int iters = 2048, blocks = sms * kProbeCtasPerSm;
  cudaStream_t st = (cudaStream_t)stream;
  float ms = 0.f;
  r = time_best(
      [&]() {
        count_launch();
        fma_probe_kernel<double><<<blocks, kProbeThreads, 0, st>>>(0.999999, 1e-6, iters);
        return cudaGetLastError();
      },
      st, &ms);
  if (r != LB_OK) return r;
  *tflops_out = 2.0 * kChains * (double)iters * blocks * kProbeThreads / (ms * 1e-3) / 1e12;
  return LB_OK;
}

lb_status lb_probe_ffma(double* tflops_out, void* stream) {
  if (tflops_out == nullptr) return LB_EINVAL;
  int dev = 0, sms = 0;
  lb_status r = current_device_sm103(&dev, &sms);
  if (r != LB_OK) return r;
  const int iters = 65536, blocks = sms * kProbeCtasPerSm;
  cudaStream_t st = (cudaStream_t)stream;
  float ms = 0.f;
  r = time_best(
      [&]() {
        count_launch();
        fma_probe_kernel<float><<<blocks, kProbeThreads, 0, st>>>(0.999f, 1e-3f, iters);
        return cudaGetLastError();
      },
      st, &ms);
  if (r != LB_OK) return r;
  *tflops_out = 2.0 * kChains * (double)iters * blocks * kProbeThreads / (ms * 1e-3) / 1e12;
  return LB_OK;
}

lb_status lb_probe_dmma(double* tflops_out, void* stream) {
  if (tflops_out == nullptr) return LB_EINVAL;
  int dev = 0, sms = 0;
  lb_status r = current_device_sm103(&dev, &sms);
  if (r != LB_OK) return r;
  const int iters = 1024, blocks = sms * kProbeCtasPerSm;
  cudaStream_t st = (cudaStream_t)stream;
  float ms = 0.f;
  r = time_best(
      [&]() {
        count_launch();
        dmma_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(1e-3, iters);
        return cudaGetLastError();
      },
      st, &ms);
  if (r != LB_OK) return r;
  // 4 MMAs of 8 x 8 x 4 per warp per iteration
  const double warps = (double)blocks * kProbeThreads / 32;
  *tflops_out = 2.0 * 8 * 8 * 4 * 4 * (double)iters * warps / (ms * 1e-3) / 1e12;
  return LB_OK;
}

lb_status lb_probe_bf16_tc(double* tflops_out, void* stream) {
  if (tflops_out == nullptr) return LB_EINVAL;
  int dev = 0, sms = 0;
  lb_status r = current_device_sm103(&dev, &sms);
  if (r != LB_OK) return r;
  const int iters = 4096;
  cudaStream_t st = (cudaStream_t)stream;
  if (set_smem_once((const void*)tc_probe_kernel, kTcSmem) != cudaSuccess) return LB_ECUDA;
  const unsigned int zero = 0;
  if (cudaMemcpyToSymbolAsync(g_probe_err, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return LB_ECUDA;
  float ms = 0.f;
  r = time_best(
      [&]() {
        count_launch();
        tc_probe_kernel<<<sms, 128, kTcSmem, st>>>(iters);
        return cudaGetLastError();
      },
      st, &ms);
  if (r != LB_OK) return r;
  unsigned int err = 0;
  if (cudaMemcpyFromSymbol(&err, g_probe_err, sizeof(err)) != cudaSuccess) return LB_ECUDA;
  if (err != 0) return LB_ETIMEOUT;
  *tflops_out = 2.0 * kTcM * kTcN * kTcK * 4.0 * iters * sms / (ms * 1e-3) / 1e12;
  return LB_OK;
}

}  // extern "C"
