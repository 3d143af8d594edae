// The three GPU timing models of Sec. 3.4 (Eq. 7-9): the device probes that
// supply their constants (Table tab:probes_gpu, Sec. 3.6) and the two
// host-facing propagation calls whose cost they model.
//
//   kernel-only (Eq. 7):  lb_propagate_batch on device-resident P and states;
//   resident P  (Eq. 8):  lb_propagate_resident -- P stays on the device, the
//                         states come from host memory and go back there,
//                         and the call returns after a stream synchronise;
//   host-visible (Eq. 9): lb_propagate_host -- P and states both in host
//                         memory, device buffers allocated and freed inside
//                         the call, as in a caller that keeps nothing on the
//                         device between calls.
//
// The probes: an empty kernel launched back to back (launch cost) or with a
// synchronise after each (launch + sync), synchronous copies of a given size
// in either direction (latency and asymptotic bandwidth of the host link),
// one cudaMalloc + cudaFree pair of a given size (the allocation term of
// Eq. 9, which the paper states rather than measures),
// and two read kernels over a device buffer, a coalesced stream and the
// stride-n gather of Algorithm alg:gpu (consecutive threads read consecutive
// rows of n complex values, so at each inner index the warp's addresses are
// n elements apart).  The read kernels fold the data with integer XOR, which
// costs far less than the memory traffic, and store the result only on an
// impossible match, so the loads cannot be removed.
#include "lb_internal.cuh"

#include <chrono>

namespace lb {
namespace {

__global__ void probe_empty_kernel() {}

constexpr unsigned long long kNever = 0x5a5a5a5a5a5a5a5aULL;

__global__ void __launch_bounds__(256) probe_stream_kernel(const double2* __restrict__ buf, long long count,
                                                           unsigned long long* __restrict__ sink) {
  unsigned long long h = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; e + 3 * stride < count; e += 4 * stride) {
    const double2 a = buf[e], b = buf[e + stride], c = buf[e + 2 * stride], d = buf[e + 3 * stride];
    h ^= __double_as_longlong(a.x) ^ __double_as_longlong(a.y) ^ __double_as_longlong(b.x) ^
         __double_as_longlong(b.y) ^ __double_as_longlong(c.x) ^ __double_as_longlong(c.y) ^
         __double_as_longlong(d.x) ^ __double_as_longlong(d.y);
  }
  for (; e < count; e += stride) {
    const double2 a = buf[e];
    h ^= __double_as_longlong(a.x) ^ __double_as_longlong(a.y);
  }
  if (h == kNever) sink[0] = h;
}

__global__ void __launch_bounds__(256) probe_gather_kernel(const double2* __restrict__ buf, long long rows, int n,
                                                           unsigned long long* __restrict__ sink) {
  const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const double2* row = buf + r * n;
  unsigned long long h = 0;
  for (int j = 0; j < n; j++) {
    const double2 a = row[j];
    h ^= __double_as_longlong(a.x) ^ __double_as_longlong(a.y);
  }
  if (h == kNever) sink[0] = h;
}

bool is_square_n(int n) {
  int d = 1;
  while (d * d < n) d++;
  return d * d == n;
}

double now_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace
}  // namespace lb

using namespace lb;

extern "C" lb_status lb_probe_launch(int reps, int sync_each, double* us_out, void* stream) {
  if (reps < 1 || us_out == nullptr) return LB_EINVAL;
  int dev = 0, sms = 0;
  lb_status s = current_device_sm103(&dev, &sms);
  if (s != LB_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LB_ECUDA;
  const double t0 = now_us();
  for (int r = 0; r < reps; r++) {
    probe_empty_kernel<<<1, 32, 0, st>>>();
    count_launch();
    if (sync_each && cudaStreamSynchronize(st) != cudaSuccess) return LB_ECUDA;
  }
  const double t1 = now_us();
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return LB_ECUDA;
  *us_out = (t1 - t0) / reps;
  return LB_OK;
}

extern "C" lb_status lb_probe_copy(void* host, void* device, long long bytes, int to_device, int reps,
                                   double* us_out, void* stream) {
  if (host == nullptr || device == nullptr || bytes < 1 || reps < 1 || us_out == nullptr) return LB_EINVAL;
  int dev = 0, sms = 0;
  lb_status s = current_device_sm103(&dev, &sms);
  if (s != LB_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LB_ECUDA;
  const cudaMemcpyKind k = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
  const double t0 = now_us();
  for (int r = 0; r < reps; r++) {
    if (cudaMemcpyAsync(to_device ? device : host, to_device ? host : device, (size_t)bytes, k, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return LB_ECUDA;
  }
  *us_out = (now_us() - t0) / reps;
  return LB_OK;
}

extern "C" lb_status lb_probe_alloc(long long bytes, int reps, double* us_out) {
  if (bytes < 1 || reps < 1 || us_out == nullptr) return LB_EINVAL;
  int dev = 0, sms = 0;
  lb_status s = current_device_sm103(&dev, &sms);
  if (s != LB_OK) return s;
  if (cudaDeviceSynchronize() != cudaSuccess) return LB_ECUDA;
  const double t0 = now_us();
  for (int r = 0; r < reps; r++) {
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)bytes) != cudaSuccess) {
      cudaGetLastError();
      return LB_ENOMEM;
    }
    if (cudaFree(p) != cudaSuccess) return LB_ECUDA;
  }
  *us_out = (now_us() - t0) / reps;
  return LB_OK;
}

extern "C" lb_status lb_probe_read(const lb_c64* buf, long long count, int n, unsigned long long* sink,
                                   void* stream) {
  if (buf == nullptr || sink == nullptr || count < 1 || n < 0) return LB_EINVAL;
  int dev = 0, sms = 0;
  lb_status s = current_device_sm103(&dev, &sms);
  if (s != LB_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) {
    long long blocks = (count + 255) / 256;
    if (blocks > 8LL * sms) blocks = 8LL * sms;
    probe_stream_kernel<<<(unsigned)blocks, 256, 0, st>>>((const double2*)buf, count, sink);
  } else {
    const long long rows = count / n;
    if (rows < 1) return LB_EINVAL;
    const long long blocks = (rows + 255) / 256;
    if (blocks > 0x7fffffffLL) return LB_EUNSUPPORTED;
    probe_gather_kernel<<<(unsigned)blocks, 256, 0, st>>>((const double2*)buf, rows, n, sink);
  }
  count_launch();
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

extern "C" lb_status lb_propagate_resident(lb_ctx* c, int n, const lb_c64* P, int B, lb_c64* states_host,
                                           void* stream) {
  if (c == nullptr || P == nullptr || states_host == nullptr) return LB_EINVAL;
  if (n < 1 || n > c->max_n || !is_square_n(n) || B < 1 || B > c->max_batch) return LB_EINVAL;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(z64) * (size_t)B * n;
  if (cudaMemcpyAsync(c->Xh, states_host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return LB_ECUDA;
  lb_status r = propagate_impl(c, n, 1, (const z64*)P, 1, B, c->Xh, LB_FP64, 0, st);
  if (r != LB_OK) return r;
  if (cudaMemcpyAsync(states_host, c->Xh, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LB_ECUDA;
  return LB_OK;
}

extern "C" lb_status lb_propagate_host(lb_ctx* c, int n, const lb_c64* P_host, int B, lb_c64* states_host,
                                       void* stream) {
  if (c == nullptr || P_host == nullptr || states_host == nullptr) return LB_EINVAL;
  if (n < 1 || n > c->max_n || !is_square_n(n) || B < 1 || B > c->max_batch) return LB_EINVAL;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t pbytes = sizeof(z64) * (size_t)n * n, xbytes = sizeof(z64) * (size_t)B * n;
  z64* Pd = nullptr;
  z64* Xd = nullptr;
  lb_status r = LB_OK;
  if (cudaMalloc(&Pd, pbytes) != cudaSuccess || cudaMalloc(&Xd, xbytes) != cudaSuccess) {
    cudaGetLastError();
    r = LB_ENOMEM;
  } else if (cudaMemcpyAsync(Pd, P_host, pbytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
             cudaMemcpyAsync(Xd, states_host, xbytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    r = LB_ECUDA;
  } else {
    r = propagate_impl(c, n, 1, Pd, 1, B, Xd, LB_FP64, 0, st);
    if (r == LB_OK && (cudaMemcpyAsync(states_host, Xd, xbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                       cudaStreamSynchronize(st) != cudaSuccess))
      r = LB_ECUDA;
  }
  if (r != LB_OK) cudaStreamSynchronize(st);  // nothing queued may still use the buffers
  if (Pd) cudaFree(Pd);
  if (Xd) cudaFree(Xd);
  return r;
}
