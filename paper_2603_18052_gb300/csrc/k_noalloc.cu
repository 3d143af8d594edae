// lb_propagate_batch_static: FP64 batched propagation that allocates nothing.
//
// Who needs this: some callers cannot call cudaMalloc at all, or cannot
// afford to.  Examples are a host application whose own caching allocator
// has already reserved the device memory it is allowed to use (a late
// cudaMalloc would fail or fragment that pool), and control loops that must
// not stall, since cudaMalloc may synchronise the device and has no bounded
// latency.  Such callers cannot create an lb_ctx (lb_create allocates the
// scratch arena), so this entry point takes no context.  It runs the same
// chained FP64 step as lb_propagate_batch's large-n path (one grouped GEMM
// launch per step, next = current * P^T), but the ping-pong buffer for the
// states lives in the file-scope array below instead of the context arena.
//
// The array is reserved in device memory on every GPU that loads this
// library's device code and stays there until the process exits.  Every call
// uses the same array and nothing in it needs to start at zero (each step
// writes the whole region it reads next), so the previous call's contents do
// not matter.  Two calls that run on the GPU at the same time, from different
// streams or host threads, share the buffer and race: serialise them.
#include "lb_internal.cuh"

#include <mutex>

namespace {

// Largest B * n accepted: 262144 complex128 values, 4 MiB.
constexpr long long kStaticStateElems = 1LL << 18;

static __device__ __align__(256) double2 g_static_states[kStaticStateElems];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double2* g_static_addr[kMaxDevices] = {};
int g_static_sms[kMaxDevices] = {};

// Per device, once, with that device current: look up the device address of
// the array (the host-side name g_static_states is only a stand-in and must
// never be handed to a kernel) and the SM count used to size the grid.
lb_status static_setup(int dev, double2** addr, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return LB_ENODEV;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_static_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_states) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return LB_ECUDA;
    }
    int s = 0;
    if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s <= 0) {
      cudaGetLastError();
      return LB_ECUDA;
    }
    g_static_sms[dev] = s;
    g_static_addr[dev] = static_cast<double2*>(p);
  }
  *addr = g_static_addr[dev];
  *sms = g_static_sms[dev];
  return LB_OK;
}

}  // namespace

extern "C" lb_status lb_propagate_batch_static(int n, int nslices, const lb_c64* P, int steps_per_slice, int B,
                                               lb_c64* states, void* stream) {
  if (P == nullptr || states == nullptr) return LB_EINVAL;
  int d = 1;
  while (d * d < n) d++;
  if (n < 1 || n > lb::kMaxN || d * d != n) return LB_EINVAL;
  if (nslices < 0 || steps_per_slice < 0 || B < 1) return LB_EINVAL;
  if ((long long)B * n > kStaticStateElems) return LB_EUNSUPPORTED;
  if (nslices == 0 || steps_per_slice == 0) return LB_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LB_ENODEV;
  }
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return LB_ENODEV;
  }
  if (major != 10 || minor != 3) return LB_ENODEV;
  // P and the states must be device memory of the current device (a
  // pointer into another GPU's memory would make the kernels read and write
  // a peer's memory).  cudaPointerGetAttributes allocates nothing.
  for (const void* ptr : {(const void*)P, (const void*)states}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
      cudaGetLastError();
      return LB_EINVAL;
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
      return LB_EINVAL;
  }
  double2* scratch = nullptr;
  int sms = 0;
  lb_status s = static_setup(dev, &scratch, &sms);
  if (s != LB_OK) return s;

  cudaStream_t st = (cudaStream_t)stream;
  const long long nn = (long long)n * n;
  const lb::z64* Pz = (const lb::z64*)P;
  lb::z64* X = (lb::z64*)states;
  lb::z64* cur = X;
  lb::z64* nxt = scratch;
  for (int sl = 0; sl < nslices; sl++)
    for (int t = 0; t < steps_per_slice; t++) {
      lb::ZGemmProblem q;
      q.M = B; q.N = n; q.K = n;
      q.A = cur; q.lda = n;
      q.B = Pz + sl * nn; q.ldb = n; q.opB = 1;
      q.C = nxt; q.ldc = n;
      q.batch = 1;
      if (lb::zgemm_f64(&q, 1, sms, st) != cudaSuccess) return LB_ECUDA;
      lb::z64* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
  if (cur != X &&
      cudaMemcpyAsync(X, cur, sizeof(lb::z64) * (size_t)B * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return LB_ECUDA;
  return LB_OK;
}
