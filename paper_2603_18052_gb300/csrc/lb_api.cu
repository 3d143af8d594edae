// C ABI of liblb: context management, argument checks and the host-side
// orchestration of the propagator build (Algorithm 1), the propagation chain
// (Algorithm 2, batched as in Algorithm 3) and the GRAPE gradient (Sec. 2.5).
#include "lb_internal.cuh"

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

using namespace lb;

#include <map>
#include <mutex>

namespace lb {
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

lb_status current_device_sm103(int* dev, int* sms) {
  int d = -1, major = 0, minor = 0, s = 0;
  if (cudaGetDevice(&d) != cudaSuccess ||
      cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, d) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, d) != cudaSuccess ||
      cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, d) != cudaSuccess) {
    cudaGetLastError();
    return LB_ENODEV;
  }
  if (major != 10 || minor != 3 || s <= 0) return LB_ENODEV;
  *dev = d;
  *sms = s;
  return LB_OK;
}

cudaError_t set_smem_once(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = done[std::make_pair(dev, kernel)];
  if (bytes <= cur) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}
}  // namespace lb

namespace {
cudaError_t accumulate_slot(lb_ctx* c, int r);

// fold every recorded sliced-product event pair into the totals (waits for them)
cudaError_t accumulate_kernels(lb_ctx* c) {
  for (int r = 0; r < lb_ctx::kKRing; r++) {
    if (!c->kern_used[r]) continue;
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(c->ev_kern[r][1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev_kern[r][0], c->ev_kern[r][1]);
    if (e != cudaSuccess) return e;
    c->kern_ms += ms;
    c->kern_fl += c->kern_flops[r];
    c->kern_launches++;
    c->kern_used[r] = 0;
  }
  return cudaSuccess;
}
}

namespace lb {
cudaError_t kernel_events(lb_ctx* c, double flops, cudaEvent_t* ev0, cudaEvent_t* ev1) {
  *ev0 = *ev1 = nullptr;
  if (!c->timing) return cudaSuccess;
  const int r = c->kern_next;
  c->kern_next = (r + 1) % lb_ctx::kKRing;
  if (c->kern_used[r]) {  // the ring has wrapped: fold the oldest pair in (waits for it)
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(c->ev_kern[r][1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->ev_kern[r][0], c->ev_kern[r][1]);
    if (e != cudaSuccess) return e;
    c->kern_ms += ms;
    c->kern_fl += c->kern_flops[r];
    c->kern_launches++;
    c->kern_used[r] = 0;
  }
  c->kern_used[r] = 1;
  c->kern_flops[r] = flops;
  *ev0 = c->ev_kern[r][0];
  *ev1 = c->ev_kern[r][1];
  return cudaSuccess;
}

lb_status stage_events_begin(lb_ctx* c, cudaStream_t st, cudaEvent_t** ev_out) {
  *ev_out = nullptr;
  if (!c->timing) return LB_OK;
  const int r = c->ring_next;
  c->ring_next = (r + 1) % lb_ctx::kRing;
  LB_CUDA(accumulate_slot(c, r));  // only waits if the ring has wrapped
  cudaEvent_t* ev = c->ev_stage[r];
  c->ring_used[r] = 1;
  LB_CUDA(cudaEventRecord(ev[0], st));
  *ev_out = ev;
  return LB_OK;
}
}  // namespace lb

namespace {

// [13/13] Pade coefficients of exp from the recurrence of the closed form
// b_j = (2m-j)! m! / ((2m)! j! (m-j)!):  b_j = b_{j-1} (m - j + 1) / (j (2m - j + 1)).
void pade13(double* b) {
  const int m = 13;
  b[0] = 1.0;
  for (int j = 1; j <= m; j++) b[j] = b[j - 1] * double(m - j + 1) / (double(j) * double(2 * m - j + 1));
}

int nblocks(int n) { return (n + kLuNb - 1) / kLuNb; }

// Fold the stage times of one ring slot into the totals (waits for its last event).
cudaError_t accumulate_slot(lb_ctx* c, int r) {
  if (!c->ring_used[r]) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(c->ev_stage[r][5]);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < 5; i++) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, c->ev_stage[r][i], c->ev_stage[r][i + 1]);
    if (e != cudaSuccess) return e;
    c->stage_ms[i] += ms;
  }
  c->stage_chunks++;
  c->ring_used[r] = 0;
  return cudaSuccess;
}

bool is_square(int n, int* d_out) {
  int d = 1;
  while (d * d < n) d++;
  if (d_out) *d_out = d;
  return d * d == n;
}

}  // namespace

extern "C" {

int lb_version(void) { return 100; }

const char* lb_status_str(int s) {
  switch (s) {
    case LB_OK: return "LB_OK";
    case LB_EINVAL: return "LB_EINVAL: invalid argument";
    case LB_ENODEV: return "LB_ENODEV: no usable sm_103 CUDA device";
    case LB_ENOMEM: return "LB_ENOMEM: device allocation failed";
    case LB_ECUDA: return "LB_ECUDA: CUDA runtime error";
    case LB_ENONFINITE: return "LB_ENONFINITE: NaN or Inf on the device";
    case LB_ESINGULAR: return "LB_ESINGULAR: zero pivot in the LU factorisation";
    case LB_ETIMEOUT: return "LB_ETIMEOUT: a device-side wait timed out";
    case LB_EUNSUPPORTED: return "LB_EUNSUPPORTED: request outside what this build supports";
    default: return "unknown lb_status";
  }
}

lb_status lb_create(lb_ctx** out, int device, int max_n, int max_batch, int max_slices) {
  if (out == nullptr) return LB_EINVAL;
  *out = nullptr;
  if (max_n < 1 || max_n > kMaxN || max_batch < 1 || max_slices < 1) return LB_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return LB_ENODEV;
  }
  if (device < 0 || device >= ndev) return LB_ENODEV;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return LB_ENODEV;
  if (prop.major != 10 || prop.minor != 3) return LB_ENODEV;  // sm_103 only
  DeviceGuard g(device);
  lb_ctx* c = new (std::nothrow) lb_ctx();
  if (!c) return LB_ENOMEM;
  c->device = device;
  c->max_n = max_n;
  c->max_batch = max_batch;
  c->max_slices = max_slices;
  c->sm_count = prop.multiProcessorCount;
  pade13(c->pade_b);

  const size_t nn = (size_t)max_n * max_n;
  const size_t S = (size_t)max_slices;
  const size_t zb = sizeof(z64);
  const int nb = kLuNb, nbk = nblocks(max_n);
  size_t need = 0;
  auto add = [&](size_t b) { need = ((need + 255) & ~size_t(255)) + b; };
  for (int i = 0; i < 9; i++) add(nn * S * zb);            // A A2 A4 A6 Z1 Z2 V W Mx
  add(S * nb * nb * zb);                                    // Linv
  add(S * (size_t)nbk * nb * nb * zb);                      // Uinv
  add(S * sizeof(unsigned long long));                      // norm bits
  add((S + 1) * sizeof(int));                               // sc
  add(S * sizeof(int));                                     // kmix
  add(2 * S * sizeof(int));                                 // spflag
  add((2 * (size_t)max_n + 2 + nn) * sizeof(int));        // csr
  add(sizeof(z64) * 64 * 64);                               // G
  add((size_t)max_batch * max_n * zb);                      // Rtmp
  add((size_t)max_batch * max_n * zb);                      // Xh
  const size_t plane_elems = (size_t)max_n * (size_t)plane_ld(max_n);
  // split planes (6 + 8 x 4); also the sliced-FP64 scratch: both operands of
  // a squaring of all slices, or the propagators' and the states' slices
  const size_t oz_need = std::max(oz_scratch_bytes(max_n, max_n, max_n, max_slices),
                                  oz_sliced_bytes(max_n, max_n, max_slices, kOzBNSmall) +
                                      oz_sliced_bytes(max_batch, max_n, 1, kOzTileM));
  const size_t sp_bytes = std::max(38 * plane_elems * S * sizeof(__nv_bfloat16), oz_need);
  add(sp_bytes);
  for (int i = 0; i < 2; i++) add(4 * (size_t)max_batch * plane_ld(max_n) * sizeof(__nv_bfloat16));
  const size_t dpl = std::max(chain32_dplane_floats(max_n), 2 * nn) * S;
  add(dpl * sizeof(float));                                 // Dpl (Dr, Di inside)
  for (int i = 0; i < 2; i++) add(chain32_state_floats(max_n, max_batch) * sizeof(float));  // C32a, C32b
  add(chain32_part_floats(prop.multiProcessorCount) * sizeof(float));                       // part32
  add((size_t)(prop.multiProcessorCount + 1) * sizeof(unsigned));                           // cnt32, barrier
  add(nn * S * zb);                                          // Ginst
  add(nn * S * zb);                                          // Pinst
  add(inst_table_bytes());                                   // instance tables
  const size_t gbytes = grape_ws_bytes(max_n, max_batch, max_slices);
  add(gbytes);
  add(sizeof(unsigned int));                                // error word
  need += 256;

  if (cudaMalloc(&c->ws, need) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return LB_ENOMEM;
  }
  c->ws_bytes = need;
  Arena ar;
  ar.base = c->ws;
  ar.cap = need;
  auto Z = [&](size_t elems) { return (z64*)ar.take(elems * zb); };
  c->A = Z(nn * S);
  c->A2 = Z(nn * S);
  c->A4 = Z(nn * S);
  c->A6 = Z(nn * S);
  c->Z1 = Z(nn * S);
  c->Z2 = Z(nn * S);
  c->V = Z(nn * S);
  c->W = Z(nn * S);
  c->Mx = Z(nn * S);
  c->Linv = Z(S * nb * nb);
  c->Uinv = Z(S * (size_t)nbk * nb * nb);
  c->norm_bits = (unsigned long long*)ar.take(S * sizeof(unsigned long long));
  c->sc = (int*)ar.take((S + 1) * sizeof(int));
  c->kmix = (int*)ar.take(S * sizeof(int));
  c->spflag = (int*)ar.take(2 * S * sizeof(int));
  c->csr = (int*)ar.take((2 * (size_t)max_n + 2 + nn) * sizeof(int));
  c->G = Z(64 * 64);
  c->Rtmp = Z((size_t)max_batch * max_n);
  c->Xh = Z((size_t)max_batch * max_n);
  c->oz_bytes = sp_bytes;
  c->oz_scratch = ar.take(c->oz_bytes);
  for (int i = 0; i < 9; i++)
    c->sp[i] = (__nv_bfloat16*)c->oz_scratch + (i == 0 ? 0 : 6 + 4 * (i - 1)) * plane_elems * S;
  for (int i = 0; i < 2; i++)
    c->spR[i] = (__nv_bfloat16*)ar.take(4 * (size_t)max_batch * plane_ld(max_n) * sizeof(__nv_bfloat16));
  c->Dpl = (float*)ar.take(dpl * sizeof(float));
  c->Dr = c->Dpl;
  c->Di = c->Dpl + nn * S;
  c->C32a = (float*)ar.take(chain32_state_floats(max_n, max_batch) * sizeof(float));
  c->C32b = (float*)ar.take(chain32_state_floats(max_n, max_batch) * sizeof(float));
  c->part32 = (float*)ar.take(chain32_part_floats(c->sm_count) * sizeof(float));
  c->cnt32 = (unsigned*)ar.take((size_t)(c->sm_count + 1) * sizeof(unsigned));
  c->Ginst = Z(nn * S);
  c->Pinst = Z(nn * S);
  c->inst_tab_bytes = inst_table_bytes();
  c->inst_tab_dev = ar.take(c->inst_tab_bytes);
  c->grape = (z64*)ar.take(gbytes);
  c->grape_bytes = gbytes;
  c->err_dev = (unsigned int*)ar.take(sizeof(unsigned int));
  if (!c->err_dev || cudaMemset(c->err_dev, 0, sizeof(unsigned int)) != cudaSuccess ||
      cudaMemset(c->cnt32, 0, (size_t)c->sm_count * sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&c->err_host, sizeof(unsigned int)) != cudaSuccess ||
      cudaMallocHost(&c->scmax_host, sizeof(int)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_scmax, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_tab, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(c->ev_tab, 0) != cudaSuccess ||
      cudaMallocHost(&c->inst_tab_host, c->inst_tab_bytes) != cudaSuccess) {
    cudaGetLastError();
    lb_destroy(c);
    return LB_ENOMEM;
  }
  for (int r = 0; r < lb_ctx::kRing; r++)
    for (int i = 0; i < 6; i++) {
      if (cudaEventCreate(&c->ev_stage[r][i]) != cudaSuccess) {
        cudaGetLastError();
        lb_destroy(c);
        return LB_ENOMEM;
      }
    }
  for (int r = 0; r < lb_ctx::kKRing; r++)
    for (int i = 0; i < 2; i++) {
      if (cudaEventCreate(&c->ev_kern[r][i]) != cudaSuccess) {
        cudaGetLastError();
        lb_destroy(c);
        return LB_ENOMEM;
      }
    }
  *out = c;
  return LB_OK;
}

lb_status lb_destroy(lb_ctx* c) {
  if (c == nullptr) return LB_OK;
  DeviceGuard g(c->device);
  if (c->ev_scmax) cudaEventDestroy(c->ev_scmax);
  if (c->ev_tab) cudaEventDestroy(c->ev_tab);
  if (c->inst_tab_host) cudaFreeHost(c->inst_tab_host);
  for (int r = 0; r < lb_ctx::kRing; r++)
    for (int i = 0; i < 6; i++)
      if (c->ev_stage[r][i]) cudaEventDestroy(c->ev_stage[r][i]);
  for (int r = 0; r < lb_ctx::kKRing; r++)
    for (int i = 0; i < 2; i++)
      if (c->ev_kern[r][i]) cudaEventDestroy(c->ev_kern[r][i]);
  if (c->err_host) cudaFreeHost(c->err_host);
  if (c->scmax_host) cudaFreeHost(c->scmax_host);
  if (c->ws) cudaFree(c->ws);
  delete c;
  return LB_OK;
}

unsigned long long lb_workspace_bytes(const lb_ctx* c) { return c ? (unsigned long long)c->ws_bytes : 0ull; }

unsigned long long lb_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

lb_status lb_set_stage_timing(lb_ctx* c, int enable) {
  if (c == nullptr) return LB_EINVAL;
  DeviceGuard g(c->device);
  for (int r = 0; r < lb_ctx::kRing; r++)
    if (accumulate_slot(c, r) != cudaSuccess) return LB_ECUDA;
  if (accumulate_kernels(c) != cudaSuccess) return LB_ECUDA;
  c->timing = enable ? 1 : 0;
  for (int i = 0; i < 5; i++) c->stage_ms[i] = 0.0;
  c->stage_chunks = 0;
  c->kern_ms = c->kern_fl = 0.0;
  c->kern_launches = 0;
  return LB_OK;
}

lb_status lb_kernel_times(lb_ctx* c, double* ms_out, double* flops_out, long long* launches_out) {
  if (c == nullptr || ms_out == nullptr) return LB_EINVAL;
  DeviceGuard g(c->device);
  if (accumulate_kernels(c) != cudaSuccess) return LB_ECUDA;
  *ms_out = c->kern_ms;
  if (flops_out) *flops_out = c->kern_fl;
  if (launches_out) *launches_out = c->kern_launches;
  return LB_OK;
}

lb_status lb_stage_times(lb_ctx* c, double* ms_out, long long* chunks_out) {
  if (c == nullptr || ms_out == nullptr) return LB_EINVAL;
  DeviceGuard g(c->device);
  for (int r = 0; r < lb_ctx::kRing; r++)
    if (accumulate_slot(c, r) != cudaSuccess) return LB_ECUDA;
  for (int i = 0; i < 5; i++) ms_out[i] = c->stage_ms[i];
  if (chunks_out) *chunks_out = c->stage_chunks;
  return LB_OK;
}

lb_status lb_sync_status(lb_ctx* c, void* stream) {
  if (c == nullptr) return LB_EINVAL;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(c->err_host, c->err_dev, sizeof(unsigned int), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess)
    return LB_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LB_ECUDA;
  const unsigned int w = *c->err_host;
  if (w != 0) {
    if (cudaMemsetAsync(c->err_dev, 0, sizeof(unsigned int), st) != cudaSuccess) return LB_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LB_ECUDA;
  }
  if (w & ERR_NONFINITE) return LB_ENONFINITE;
  if (w & ERR_SINGULAR) return LB_ESINGULAR;
  if (w & ERR_TIMEOUT) return LB_ETIMEOUT;
  if (w & ERR_SQUARING_BOUND) return LB_EUNSUPPORTED;
  return LB_OK;
}

lb_status lb_autotune(lb_ctx* c, int n, int nslices, int B, int* shapes_out, void* stream) {
  if (c == nullptr || n < 1 || n > c->max_n || nslices < 1 || nslices > c->max_slices || B < 1 ||
      B > c->max_batch)
    return LB_EINVAL;
  DeviceGuard g(c->device);
  return lb::autotune_impl(c, n, nslices, B, (cudaStream_t)stream, shapes_out);
}

lb_status lb_set_max_squarings(lb_ctx* c, int bound) {
  if (c == nullptr || bound > 64) return LB_EINVAL;
  c->max_squarings = bound < 0 ? -1 : bound;
  return LB_OK;
}

lb_status lb_assemble(lb_ctx* c, int d, const lb_c64* H, int K, const lb_c64* Ls, lb_c64* L_out,
                      void* stream) {
  if (c == nullptr || H == nullptr || L_out == nullptr) return LB_EINVAL;
  if (d < 1 || d * d > c->max_n || K < 0 || K > 64 || (K > 0 && Ls == nullptr)) return LB_EINVAL;
  DeviceGuard g(c->device);
  LB_CUDA(launch_assemble(d, (const z64*)H, K, (const z64*)Ls, (z64*)L_out, c->G, c->sm_count,
                          (cudaStream_t)stream));
  return LB_OK;
}

}  // extern "C"

namespace lb {

ZGemmProblem sq(int n, int S, const z64* A, const z64* B, z64* C) {
  ZGemmProblem p;
  const long long nn = (long long)n * n;
  p.M = p.N = p.K = n;
  p.A = A;
  p.lda = n;
  p.sA = nn;
  p.B = B;
  p.ldb = n;
  p.sB = nn;
  p.C = C;
  p.ldc = n;
  p.sC = nn;
  p.batch = S;
  return p;
}

// Blocked LU of Mx[s] (no pivot search) applied to the right-hand sides held in
// N[s] (n x nrhs, leading dimension ldN, slice stride sN), then back
// substitution into N[s]:  N <- Mx^{-1} N.  Uf (U), Lp (L) and Y (same shape
// as N) are n x n-per-slice scratch.
//
// Left-looking (Crout) order: at block step k the block row and the block
// column of Mx are first brought up to date with everything factored so far,
// each in one GEMM whose K is all previous blocks (K = k0), together with
// the block row of the right-hand sides; then the 32 x 32 diagonal block is
// factored and inverted in shared memory (lu_diag) and the new U row panel,
// L column panel and forward-substituted rows follow from the block
// inverses (K = 32).  The back substitution is left-looking too.  The
// FLOPs are those of the right-looking form; almost all of them now sit in
// GEMMs with long K loops instead of K = 32 updates, whose fixed costs
// (operand loads before the first multiply, the complex epilogue in FP64,
// one round trip per tile) are paid once per output tile instead of once
// per block step.
lb_status lu_solve_blocked(lb_ctx* c, int n, int S, z64* Mx, z64* N, int nrhs, long long ldN, long long sN,
                           z64* Uf, z64* Y, z64* Lp, cudaStream_t st) {
  const long long nn = (long long)n * n;
  const int nb = kLuNb, nbk = nblocks(n);
  const long long sLinv = (long long)nb * nb, sUinv = (long long)nbk * nb * nb;
  for (int k = 0; k < nbk; k++) {
    const int k0 = k * nb, kb = (n - k0 < nb) ? n - k0 : nb, rest = n - k0 - kb;
    z64* Uinv_k = c->Uinv + (long long)k * nb * nb;
    if (k0 > 0) {
      ZGemmProblem pr[3];
      int np = 0;
      {  // block row k, columns k0..n-1:  Mx[k0:k0+kb, k0:] -= L[k0:k0+kb, :k0] U[:k0, k0:]
        ZGemmProblem& a = pr[np++];
        a.M = kb; a.N = n - k0; a.K = k0;
        a.A = Lp + (long long)k0 * n; a.lda = n; a.sA = nn;
        a.B = Uf + k0; a.ldb = n; a.sB = nn;
        a.C = Mx + (long long)k0 * n + k0; a.ldc = n; a.sC = nn;
        a.alpha = -1.0; a.beta = 1.0; a.batch = S;
      }
      if (rest > 0) {  // block column k below the diagonal:  Mx[k0+kb:, k0:k0+kb] -= L[k0+kb:, :k0] U[:k0, k0:k0+kb]
        ZGemmProblem& b = pr[np++];
        b.M = rest; b.N = kb; b.K = k0;
        b.A = Lp + (long long)(k0 + kb) * n; b.lda = n; b.sA = nn;
        b.B = Uf + k0; b.ldb = n; b.sB = nn;
        b.C = Mx + (long long)(k0 + kb) * n + k0; b.ldc = n; b.sC = nn;
        b.alpha = -1.0; b.beta = 1.0; b.batch = S;
      }
      {  // right-hand sides, block row k:  N[k0:k0+kb, :] -= L[k0:k0+kb, :k0] Y[:k0, :]
        ZGemmProblem& q = pr[np++];
        q.M = kb; q.N = nrhs; q.K = k0;
        q.A = Lp + (long long)k0 * n; q.lda = n; q.sA = nn;
        q.B = Y; q.ldb = ldN; q.sB = sN;
        q.C = N + (long long)k0 * ldN; q.ldc = ldN; q.sC = sN;
        q.alpha = -1.0; q.beta = 1.0; q.batch = S;
      }
      LB_CUDA(zgemm_f64(pr, np, c->sm_count, st));
    }
    LB_CUDA(launch_lu_diag(n, S, k0, kb, Mx, Uf, c->Linv, sLinv, Uinv_k, sUinv, c->err_dev, st));
    {
      ZGemmProblem pr[3];
      int np = 0;
      if (rest > 0) {
        // U[k0:k0+kb, k0+kb:] = Linv_k Mx[k0:k0+kb, k0+kb:]
        ZGemmProblem& u = pr[np++];
        u.M = kb; u.N = rest; u.K = kb;
        u.A = c->Linv; u.lda = nb; u.sA = sLinv;
        u.B = Mx + (long long)k0 * n + k0 + kb; u.ldb = n; u.sB = nn;
        u.C = Uf + (long long)k0 * n + k0 + kb; u.ldc = n; u.sC = nn;
        u.batch = S;
        // L[k0+kb:, k0:k0+kb] = Mx[k0+kb:, k0:k0+kb] Uinv_k
        ZGemmProblem& l = pr[np++];
        l.M = rest; l.N = kb; l.K = kb;
        l.A = Mx + (long long)(k0 + kb) * n + k0; l.lda = n; l.sA = nn;
        l.B = Uinv_k; l.ldb = nb; l.sB = sUinv;
        l.C = Lp + (long long)(k0 + kb) * n + k0; l.ldc = n; l.sC = nn;
        l.batch = S;
      }
      // Y[k0:k0+kb, :] = Linv_k N[k0:k0+kb, :]
      ZGemmProblem& y = pr[np++];
      y.M = kb; y.N = nrhs; y.K = kb;
      y.A = c->Linv; y.lda = nb; y.sA = sLinv;
      y.B = N + (long long)k0 * ldN; y.ldb = ldN; y.sB = sN;
      y.C = Y + (long long)k0 * ldN; y.ldc = ldN; y.sC = sN;
      y.batch = S;
      LB_CUDA(zgemm_f64(pr, np, c->sm_count, st));
    }
  }
  // back substitution: X_k = Uinv_k (Y_k - U[k0:k0+kb, k0+kb:] X[k0+kb:]), X into N
  for (int k = nbk - 1; k >= 0; k--) {
    const int k0 = k * nb, kb = (n - k0 < nb) ? n - k0 : nb, rest = n - k0 - kb;
    z64* Uinv_k = c->Uinv + (long long)k * nb * nb;
    if (rest > 0) {
      ZGemmProblem g;
      g.M = kb; g.N = nrhs; g.K = rest;
      g.A = Uf + (long long)k0 * n + k0 + kb; g.lda = n; g.sA = nn;
      g.B = N + (long long)(k0 + kb) * ldN; g.ldb = ldN; g.sB = sN;
      g.C = Y + (long long)k0 * ldN; g.ldc = ldN; g.sC = sN;
      g.alpha = -1.0; g.beta = 1.0; g.batch = S;
      LB_CUDA(zgemm_f64(&g, 1, c->sm_count, st));
    }
    ZGemmProblem f;
    f.M = kb; f.N = nrhs; f.K = kb;
    f.A = Uinv_k; f.lda = nb; f.sA = sUinv;
    f.B = Y + (long long)k0 * ldN; f.ldb = ldN; f.sB = sN;
    f.C = N + (long long)k0 * ldN; f.ldc = ldN; f.sC = sN;
    f.batch = S;
    LB_CUDA(zgemm_f64(&f, 1, c->sm_count, st));
  }
  return LB_OK;
}

}  // namespace lb

namespace {

typedef cudaError_t (*gemm_fn)(const ZGemmProblem*, int, int, cudaStream_t);

// The six Pade products in split-BF16 x3 on the tensor cores, with every
// intermediate kept in FP32 (FP64 arithmetic is 1/64 rate here):
//   A2, A4, A6 = powers (FP32 copies + planes),  V = I + Vs,  W' = b1 I + Ws,
//   Vs = A6 Z1 + b6 A6 + b4 A4 + b2 A2,  Ws = A6 Z2 + b7 A6 + b5 A4 + b3 A2,
//   U = b1 A + A Ws, so the BF16 rounding touches only the O(A^3) part of U;
//   V - U and V + U are written in FP64 with the identity added in FP64.
lb_status pade_products_tc(lb_ctx* c, int n, int S, z64* P, cudaStream_t st) {
  const long long nn = (long long)n * n;
  const double* b = c->pade_b;
  const long long ld = plane_ld(n), pl = (long long)n * ld;
  __nv_bfloat16 *Aop = c->sp[0], *AopT = c->sp[1], *A2op = c->sp[2], *A2opT = c->sp[3], *A4op = c->sp[4],
                *A6op = c->sp[5], *Z1T = c->sp[6], *Z2T = c->sp[7], *WT = c->sp[8];
  // FP32 copies live in the (unused here) FP64 buffers
  float2 *Af = (float2*)c->Z1, *A2f = (float2*)c->A2, *A4f = (float2*)c->A4, *A6f = (float2*)c->A6,
         *Vsf = (float2*)c->V;
  LB_CUDA(launch_split(n, n, S, c->A, n, nn, 0.0, 0, Aop, ld, pl, st, 2, Af));
  LB_CUDA(launch_split(n, n, S, c->A, n, nn, 0.0, 1, AopT, ld, pl, st, 2));
  auto prob = [&](const __nv_bfloat16* a, const __nv_bfloat16* bo) {
    TcProblem t;
    t.M = t.N = t.K = n;
    t.batch = S;
    t.Aop = a; t.a_ld = ld; t.a_plane = pl;
    t.Bop = bo; t.b_ld = ld; t.b_plane = pl;
    t.ldc = n; t.sC = nn;
    t.err = c->err_dev;
    return t;
  };
  TcProblem t = prob(Aop, AopT);
  t.Cf = A2f;
  t.sp = A2op; t.sp_ld = ld; t.sp_plane = pl;
  t.spT = A2opT; t.spT_ld = ld; t.spT_plane = pl;
  LB_CUDA(zgemm_tc(t, st));
  t = prob(A2op, A2opT);
  t.Cf = A4f;
  t.sp = A4op; t.sp_ld = ld; t.sp_plane = pl;
  LB_CUDA(zgemm_tc(t, st));
  t = prob(A4op, A2opT);
  t.Cf = A6f;
  t.sp = A6op; t.sp_ld = ld; t.sp_plane = pl;
  LB_CUDA(zgemm_tc(t, st));
  LB_CUDA(launch_lincomb_splitT(n, S, A6f, A4f, A2f, (float)b[12], (float)b[10], (float)b[8], Z1T, ld, pl, st));
  LB_CUDA(launch_lincomb_splitT(n, S, A6f, A4f, A2f, (float)b[13], (float)b[11], (float)b[9], Z2T, ld, pl, st));
  auto with3 = [&](TcProblem q, double c0, double c1, double c2) {
    q.nterms = 3;
    q.X[0] = A6f; q.X[1] = A4f; q.X[2] = A2f;
    q.sX[0] = q.sX[1] = q.sX[2] = nn;
    q.coef[0] = (float)c0; q.coef[1] = (float)c1; q.coef[2] = (float)c2;
    return q;
  };
  t = with3(prob(A6op, Z1T), b[6], b[4], b[2]);
  t.Cf = Vsf;
  LB_CUDA(zgemm_tc(t, st));
  t = with3(prob(A6op, Z2T), b[7], b[5], b[3]);
  t.spT = WT; t.spT_ld = ld; t.spT_plane = pl;
  LB_CUDA(zgemm_tc(t, st));
  // acc = A Ws:  V - U = b0 I + Vs - b1 A - acc,  V + U = b0 I + Vs + b1 A + acc
  t = prob(Aop, WT);
  t.alpha = -1.f; t.alpha2 = 1.f;
  t.nterms = 2;
  t.X[0] = Vsf; t.X[1] = Af;
  t.sX[0] = t.sX[1] = nn;
  t.coef[0] = 1.f; t.coef[1] = (float)(-b[1]);
  t.coef2[0] = 1.f; t.coef2[1] = (float)b[1];
  t.Cd = c->Mx; t.gamma = b[0];
  t.C2d = P; t.gamma2 = b[0];
  LB_CUDA(zgemm_tc(t, st));
  return LB_OK;
}

// One chunk of slices of lb_expm_pade.
lb_status expm_chunk(lb_ctx* c, int n, int S, const z64* Lbase, const z64* Ldrv, const double* u,
                     double dt, lb_precision prec, z64* P, int* s_out, cudaStream_t st) {
  const long long nn = (long long)n * n;
  const double* b = c->pade_b;
  gemm_fn gemm = (prec == LB_FP64) ? zgemm_f64 : zgemm_f32;
  cudaEvent_t* ev = nullptr;
  {
    lb_status r = stage_events_begin(c, st, &ev);
    if (r != LB_OK) return r;
  }
  LB_CUDA(launch_slice_prepare(n, S, Lbase, Ldrv, u, dt, c->A, c->norm_bits, c->sc, c->kmix, s_out,
                               c->err_dev, c->sm_count, st));
  if (c->max_squarings < 0) {
    LB_CUDA(cudaMemcpyAsync(c->scmax_host, c->sc + S, sizeof(int), cudaMemcpyDeviceToHost, st));
    LB_CUDA(cudaEventRecord(c->ev_scmax, st));
  } else {
    LB_CUDA(launch_check_bound(c->sc + S, c->max_squarings, c->err_dev, st));
  }
  if (ev) LB_CUDA(cudaEventRecord(ev[1], st));
  if (prec == LB_BF16X3) {
    lb_status r = pade_products_tc(c, n, S, P, st);
    if (r != LB_OK) return r;
  } else {
  // three power products
  ZGemmProblem p = sq(n, S, c->A, c->A, c->A2);
  LB_CUDA(gemm(&p, 1, c->sm_count, st));
  p = sq(n, S, c->A2, c->A2, c->A4);
  LB_CUDA(gemm(&p, 1, c->sm_count, st));
  p = sq(n, S, c->A4, c->A2, c->A6);
  LB_CUDA(gemm(&p, 1, c->sm_count, st));
  LB_CUDA(launch_lincomb3((int)nn, S, c->A6, c->A4, c->A2, b[12], b[10], b[8], c->Z1, st));
  LB_CUDA(launch_lincomb3((int)nn, S, c->A6, c->A4, c->A2, b[13], b[11], b[9], c->Z2, st));
  // V = A6 Z1 + b6 A6 + b4 A4 + b2 A2 + b0 I ;  W' = A6 Z2 + b7 A6 + b5 A4 + b3 A2 + b1 I
  ZGemmProblem vw[2];
  vw[0] = sq(n, S, c->A6, c->Z1, c->V);
  vw[0].nterms = 3;
  vw[0].X[0] = c->A6; vw[0].X[1] = c->A4; vw[0].X[2] = c->A2;
  vw[0].sX[0] = vw[0].sX[1] = vw[0].sX[2] = nn;
  vw[0].coef[0] = b[6]; vw[0].coef[1] = b[4]; vw[0].coef[2] = b[2];
  vw[0].gamma = b[0];
  vw[1] = sq(n, S, c->A6, c->Z2, c->W);
  vw[1].nterms = 3;
  vw[1].X[0] = c->A6; vw[1].X[1] = c->A4; vw[1].X[2] = c->A2;
  vw[1].sX[0] = vw[1].sX[1] = vw[1].sX[2] = nn;
  vw[1].coef[0] = b[7]; vw[1].coef[1] = b[5]; vw[1].coef[2] = b[3];
  vw[1].gamma = b[1];
  LB_CUDA(gemm(vw, 2, c->sm_count, st));
  // U = A W';  Mx = V - U, P = V + U
  p = sq(n, S, c->A, c->W, c->Mx);
  p.alpha = -1.0;
  p.nterms = 1;
  p.X[0] = c->V; p.sX[0] = nn; p.coef[0] = 1.0;
  p.C2 = P; p.X2 = c->V; p.sX2 = nn; p.alpha2 = 1.0;
  LB_CUDA(gemm(&p, 1, c->sm_count, st));
  }
  if (ev) LB_CUDA(cudaEventRecord(ev[2], st));
  // (V - U) P = (V + U), FP64.  Uf, Y, Lp reuse A2, A4, A6.
  lb_status s = lu_solve_blocked(c, n, S, c->Mx, P, n, n, nn, c->A2, c->A4, c->A6, st);
  if (s != LB_OK) return s;
  if (ev) LB_CUDA(cudaEventRecord(ev[3], st));
  // squarings, FP64.  The count is known on the host once the event that
  // follows the norm kernel has completed (long before the LU finishes).
  int smax = c->max_squarings;
  if (smax < 0) {
    LB_CUDA(cudaEventSynchronize(c->ev_scmax));
    smax = *c->scmax_host;
  }
  // In the mixed forms a squaring whose operand is still close to I (the
  // leading kmix[s] ones, while ||A||_1 2^(j-s) <= 1) runs on D = P - I:
  // P^2 = 2P - I + D D, with only D D in the product precision; later
  // squarings (large ||L dt||) stay FP64.
  for (int it = 0; it < smax; it++) {
    ZGemmProblem q = sq(n, S, P, P, c->Z1);
    q.active = c->sc;
    q.active_iter = it;
    if (prec == LB_BF16X3) {
      // D D on the tensor cores (D = P - I: rows in two BF16 pieces, D^T in
      // three), Z1 = D D - I widened to FP64, then Z1 = 2P + Z1 in FP64
      const long long ld = plane_ld(n), pl = (long long)n * ld;
      LB_CUDA(launch_split(n, n, S, P, n, nn, 1.0, 0, c->sp[1], ld, pl, st, 2));
      LB_CUDA(launch_split(n, n, S, P, n, nn, 1.0, 1, c->sp[0], ld, pl, st, 3));
      TcProblem t;
      t.M = t.N = t.K = n;
      t.batch = S;
      t.npa = 2; t.npb = 3;
      t.Aop = c->sp[1]; t.a_ld = ld; t.a_plane = pl;
      t.Bop = c->sp[0]; t.b_ld = ld; t.b_plane = pl;
      t.ldc = n; t.sC = nn;
      t.Cd = c->Z1; t.gamma = -1.0;
      t.active = c->kmix; t.active_iter = it;
      t.err = c->err_dev;
      LB_CUDA(zgemm_tc(t, st));
      LB_CUDA(launch_add_twice(nn, S, P, c->Z1, st));
      q.active_lo = c->kmix;
    } else if (prec != LB_FP64) {
      ZGemmProblem qm = sq(n, S, P, P, c->Z1);
      qm.shiftA = qm.shiftB = 1.0;
      qm.nterms = 1;
      qm.X[0] = P; qm.sX[0] = nn; qm.coef[0] = 2.0;
      qm.gamma = -1.0;
      qm.active = c->kmix;
      qm.active_iter = it;
      LB_CUDA((prec == LB_FP32 ? gemm : zgemm_f32)(&qm, 1, c->sm_count, st));
      q.active_lo = c->kmix;
    }
    LB_CUDA(zgemm_f64(&q, 1, c->sm_count, st));
    LB_CUDA(launch_copy_active(nn, S, c->Z1, P, c->sc, it, st));
  }
  if (ev) LB_CUDA(cudaEventRecord(ev[4], st));
  LB_CUDA(launch_check_finite(nn * S, P, c->err_dev, st));
  if (ev) LB_CUDA(cudaEventRecord(ev[5], st));
  return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_expm_pade(lb_ctx* c, int n, int nslices, const lb_c64* Lbase, const lb_c64* Ldrv,
                       const double* u, double dt, lb_precision prec, lb_c64* P_out, int* s_out,
                       void* stream) {
  if (c == nullptr || Lbase == nullptr || P_out == nullptr) return LB_EINVAL;
  if (n < 1 || n > c->max_n || nslices < 0) return LB_EINVAL;
  if (Ldrv != nullptr && u == nullptr) return LB_EINVAL;
  if (!std::isfinite(dt)) return LB_EINVAL;
  const bool herm = prec == LB_FP64_HERMITIAN || prec == LB_FP32_HERMITIAN || prec == LB_FP64_SLICED;
  if (prec != LB_FP64 && prec != LB_FP32 && prec != LB_BF16X3 && !herm) return LB_EINVAL;
  if (herm && !is_square(n, nullptr)) return LB_EINVAL;
  if (nslices == 0) return LB_OK;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (c->max_squarings < 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      return LB_EUNSUPPORTED;  // the host read of the squaring count cannot be captured
  }
  const long long nn = (long long)n * n;
  for (int s0 = 0; s0 < nslices; s0 += c->max_slices) {
    const int S = (nslices - s0 < c->max_slices) ? nslices - s0 : c->max_slices;
    const z64* Lb = (const z64*)Lbase + (Ldrv == nullptr ? s0 * nn : 0);
    lb_status r = herm ? expm_chunk_herm(c, n, S, Lb, (const z64*)Ldrv, u ? u + s0 : nullptr, dt, prec,
                                         (z64*)P_out + s0 * nn, s_out ? s_out + s0 : nullptr, st)
                       : expm_chunk(c, n, S, Lb, (const z64*)Ldrv, u ? u + s0 : nullptr, dt, prec,
                                    (z64*)P_out + s0 * nn, s_out ? s_out + s0 : nullptr, st);
    if (r != LB_OK) return r;
  }
  return LB_OK;
}

lb_status lb_propagate_batch(lb_ctx* c, int n, int nslices, const lb_c64* P, int steps_per_slice,
                             int B, lb_c64* states, lb_precision prec, int renorm_trace,
                             void* stream) {
  if (c == nullptr || P == nullptr || states == nullptr) return LB_EINVAL;
  int d = 0;
  if (n < 1 || n > c->max_n || !is_square(n, &d)) return LB_EINVAL;
  if (nslices < 0 || steps_per_slice < 0 || B < 1 || B > c->max_batch) return LB_EINVAL;
  if (prec != LB_FP64 && prec != LB_FP32 && prec != LB_BF16X3 && prec != LB_FP64_HERMITIAN &&
      prec != LB_FP32_HERMITIAN && prec != LB_FP64_SLICED)
    return LB_EINVAL;
  if (prec == LB_FP32_HERMITIAN) prec = LB_FP32;  // the propagation of the FP32 forms is the same
  if (nslices == 0 || steps_per_slice == 0) return LB_OK;
  DeviceGuard g(c->device);
  return lb::propagate_impl(c, n, nslices, (const z64*)P, steps_per_slice, B, (z64*)states, prec, renorm_trace,
                            (cudaStream_t)stream);
}

}  // extern "C"

namespace lb {

lb_status propagate_impl(lb_ctx* c, int n, int nslices, const z64* Pz, int steps_per_slice, int B, z64* X,
                         lb_precision prec, int renorm_trace, cudaStream_t st) {
  int d = 0;
  is_square(n, &d);
  const long long nn = (long long)n * n;
  if (prec == LB_FP64_HERMITIAN || prec == LB_FP64_SLICED) {
    int C = 0, K = 0;
    const bool lat = herm_lat_split(n, &C, &K);
    if (lat || herm_resident_fits(n)) {
      // real transfer matrices of a chunk of slices in the build scratch
      double* R = (double*)c->Z1;
      for (int s0 = 0; s0 < nslices; s0 += c->max_slices) {
        const int S = (nslices - s0 < c->max_slices) ? nslices - s0 : c->max_slices;
        LB_CUDA(launch_herm_matrix(n, d, S, Pz + s0 * nn, R, c->sm_count, st));
        if (lat)
          LB_CUDA(launch_prop_herm_lat(n, d, S, R, steps_per_slice, B, X, st));
        else
          LB_CUDA(launch_prop_herm_resident(n, d, S, R, steps_per_slice, B, X, c->sm_count, st));
      }
      return LB_OK;
    }
    return propagate_herm_large(c, n, nslices, Pz, steps_per_slice, B, X, prec == LB_FP64_SLICED, st);
  }
  if (prec == LB_FP64) {
    const bool gemv = gemv_f64_preferred(n, B);
    if (!gemv && resident_f64_fits(n)) {
      LB_CUDA(launch_propagate_resident_f64(n, nslices, Pz, steps_per_slice, B, X, c->sm_count, st));
      return LB_OK;
    }
    z64* cur = X;
    z64* nxt = c->Rtmp;
    for (int s = 0; s < nslices; s++)
      for (int t = 0; t < steps_per_slice; t++) {
        // next[b][i] = sum_j P[i][j] cur[b][j]  ->  C = cur * P^T
        if (gemv) {
          LB_CUDA(launch_zgemv_f64(n, B, Pz + s * nn, n, cur, n, nxt, n, 1.0, nullptr, 0, st));
          z64* tmp = cur;
          cur = nxt;
          nxt = tmp;
          continue;
        }
        ZGemmProblem q;
        q.M = B; q.N = n; q.K = n;
        q.A = cur; q.lda = n;
        q.B = Pz + s * nn; q.ldb = n; q.opB = 1;
        q.C = nxt; q.ldc = n;
        q.batch = 1;
        LB_CUDA(zgemm_f64(&q, 1, c->sm_count, st));
        z64* tmp = cur;
        cur = nxt;
        nxt = tmp;
      }
    if (cur != X)
      LB_CUDA(cudaMemcpyAsync(X, cur, sizeof(z64) * (size_t)B * n, cudaMemcpyDeviceToDevice, st));
    return LB_OK;
  }
  if (prec == LB_BF16X3) {
    // Split BF16 on the tensor cores: next = c (cur + D cur) with D = P - I
    // and c = 1 / Tr(cur) when renormalising (deferred by one step and
    // applied in the epilogue).  The states (A operand, rows = states) are
    // FP32 and enter as two BF16 pieces; D (B operand) keeps three pieces,
    // because its rounding repeats identically at every step and would
    // otherwise add up coherently over long chains; five BF16 products per
    // real product, FP32 accumulation, K split over CTAs when the tiles do
    // not fill the GPU.
    const long long ld = plane_ld(n), dpl = (long long)n * ld, rpl = (long long)B * ld;
    // FP32 states with rows padded to ld (16-byte aligned rows: vector
    // stores in the epilogue), in the FP32 chain's state buffers
    float2* cur = (float2*)c->C32a;
    float2* nxt = (float2*)c->C32b;
    __nv_bfloat16* pc = c->spR[0];
    __nv_bfloat16* pn = c->spR[1];
    LB_CUDA(launch_states_c64_f32(n, B, X, cur, ld, st));
    LB_CUDA(launch_renorm_split(n, d, B, 0, cur, ld, pc, ld, rpl, st));
    for (int s0 = 0; s0 < nslices; s0 += c->max_slices) {
      const int S = (nslices - s0 < c->max_slices) ? nslices - s0 : c->max_slices;
      LB_CUDA(launch_split(n, n, S, Pz + s0 * nn, n, nn, 1.0, 0, c->sp[0], ld, dpl, st, 3));
      for (int s = 0; s < S; s++)
        for (int t = 0; t < steps_per_slice; t++) {
          TcProblem q;
          q.M = B; q.N = n; q.K = n; q.batch = 1;
          q.npa = 2; q.npb = 3;
          q.Aop = pc; q.a_ld = ld; q.a_plane = rpl;
          q.Bop = c->sp[0] + (long long)s * 6 * dpl; q.b_ld = ld; q.b_plane = dpl;
          q.ldc = ld;
          q.nterms = 1; q.X[0] = cur; q.coef[0] = 1.f;
          q.Cf = nxt;
          q.sp = pn; q.sp_ld = ld; q.sp_plane = rpl;
          if (renorm_trace) {
            q.rs_src = cur;
            q.rs_d = d;
          }
          q.part = (float2*)c->part32; q.cnt = c->cnt32; q.max_ctas = c->sm_count;
          q.pdl = (s > 0 || t > 0) ? 1 : 0;  // the first step of a chunk follows the plane split
          q.err = c->err_dev;
          LB_CUDA(zgemm_tc(q, st));
          float2* t1 = cur; cur = nxt; nxt = t1;
          __nv_bfloat16* t2 = pc; pc = pn; pn = t2;
        }
    }
    // the last step's trace factor (the others were applied one step late)
    if (renorm_trace) LB_CUDA(launch_renorm_split(n, d, B, 1, cur, ld, pn, ld, rpl, st));
    LB_CUDA(launch_states_f32_c64(n, B, cur, ld, X, st));
    return LB_OK;
  }
  // FP32: D = P - I in FP32, states in FP32
  if (resident_f32_fits(n)) {
    for (int s0 = 0; s0 < nslices; s0 += c->max_slices) {
      const int S = (nslices - s0 < c->max_slices) ? nslices - s0 : c->max_slices;
      LB_CUDA(launch_make_delta_f32(n, S, Pz + s0 * nn, c->Dr, c->Di, st));
      LB_CUDA(launch_propagate_resident_f32(n, S, c->Dr, c->Di, steps_per_slice, B, X, renorm_trace, c->sm_count,
                                            st));
    }
    return LB_OK;
  }
  // n > 81: one split-K GEMM launch per step on K-major planes, the trace
  // renormalisation deferred into the next step's epilogue
  const size_t dpl = chain32_dplane_floats(n);
  float* cur = c->C32a;
  float* nxt = c->C32b;
  LB_CUDA(launch_chain32_states_in(n, B, X, cur, st));
  for (int s0 = 0; s0 < nslices; s0 += c->max_slices) {
    const int S = (nslices - s0 < c->max_slices) ? nslices - s0 : c->max_slices;
    LB_CUDA(launch_chain32_dplanes(n, S, Pz + s0 * nn, c->Dpl, st));
    // the chunk's steps in one persistent launch where the shape allows
    cudaError_t pe = cudaSuccess;
    if (launch_chain32_persist(n, B, renorm_trace, c->Dpl, (long long)dpl, steps_per_slice, S * steps_per_slice, cur,
                               nxt, c->cnt32 + c->sm_count, c->err_dev, c->sm_count, st, &pe)) {
      LB_CUDA(pe);
      if ((S * steps_per_slice) & 1) {
        float* t1 = cur;
        cur = nxt;
        nxt = t1;
      }
      continue;
    }
    for (int s = 0; s < S; s++)
      for (int t = 0; t < steps_per_slice; t++) {
        const bool pdl = s > 0 || t > 0;  // the first step of a chunk follows the D^T conversion
        LB_CUDA(launch_chain32_step(n, B, renorm_trace, c->Dpl + s * dpl, cur, nxt, c->part32, c->cnt32,
                                    c->sm_count, pdl, st));
        float* t1 = cur;
        cur = nxt;
        nxt = t1;
      }
  }
  LB_CUDA(launch_chain32_states_out(n, B, renorm_trace, cur, X, st));
  return LB_OK;
}

lb_status autotune_impl(lb_ctx* c, int n, int nslices, int B, cudaStream_t st, int* shapes_out) {
  const long long nn = (long long)n * n;
  // zero generators: A = 0, so s = 0 and V - U = I; the values do not matter,
  // only the launch shapes (every tuned launch runs several times)
  LB_CUDA(cudaMemsetAsync(c->Ginst, 0, sizeof(z64) * nn * nslices, st));
  set_tuning(true);
  lb_status r = expm_chunk(c, n, nslices, c->Ginst, nullptr, nullptr, 1.0, LB_FP32, c->Pinst, nullptr, st);
  // the real-coordinate builds: FP32 products with the FP64 LU, then the
  // FP64 products
  const bool square = is_square(n, nullptr);
  if (r == LB_OK && square)
    r = expm_chunk_herm(c, n, nslices, c->Ginst, nullptr, nullptr, 1.0, LB_FP32_HERMITIAN, c->Pinst, nullptr, st);
  if (r == LB_OK && square)
    r = expm_chunk_herm(c, n, nslices, c->Ginst, nullptr, nullptr, 1.0, LB_FP64_HERMITIAN, c->Pinst, nullptr, st);
  if (r == LB_OK && n > 81 && (long long)B * n <= nn * c->max_slices) {
    LB_CUDA(cudaMemsetAsync(c->W, 0, sizeof(z64) * B * n, st));
    r = propagate_impl(c, n, 1, c->Pinst, 1, B, c->W, LB_FP64, 0, st);
    if (r == LB_OK && square) r = propagate_impl(c, n, 1, c->Pinst, 1, B, c->W, LB_FP64_HERMITIAN, 0, st);
  }
  set_tuning(false);
  if (cudaStreamSynchronize(st) != cudaSuccess) return LB_ECUDA;
  LB_CUDA(cudaMemsetAsync(c->err_dev, 0, sizeof(unsigned int), st));
  if (cudaStreamSynchronize(st) != cudaSuccess) return LB_ECUDA;
  if (shapes_out) *shapes_out = tuned_shapes();
  return r;
}

lb_status expm_chunk_public(lb_ctx* c, int n, int S, const z64* Lbase, const z64* Ldrv, const double* u, double dt,
                            lb_precision prec, z64* P, int* s_out, cudaStream_t st) {
  return expm_chunk(c, n, S, Lbase, Ldrv, u, dt, prec, P, s_out, st);
}

}  // namespace lb

