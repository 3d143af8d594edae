// Many independent instances of mixed size in one call: each instance has its
// own Hilbert dimension d, generators (Eq. 5), control slices and batch of
// states, as in a sweep over devices or pulse families.  Instances are
// grouped by n = d*d; within a group, whole instances are packed into chunks
// of at most max_slices slices, the per-slice generators
// G = Lbase_i + u_{i,s} Ldrv_i are gathered by one kernel from a pointer
// table, the chunk's propagators are built by the batched Pade build
// (Algorithm 1), and the states are propagated (Algorithm 2): for n <= 81 by
// one work-list launch in which every CTA takes one (instance, group of
// states) item and runs that instance's whole chain with its propagators in
// shared memory; larger n use the batched GEMM path per instance.
#include "lb_internal.cuh"
#include "res32.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

namespace lb {

namespace {

struct GenEntry {
  const z64* Lb;
  const z64* Ld;
  const double* u;  // points at u_{i,s}
};

struct WorkItem {
  const z64* P;  // first propagator of the instance (slices contiguous)
  z64* X;        // first state of the item
  int nslices, steps, nb;
};

constexpr int kMaxEntries = 1 << 18;  // slices per call
constexpr int kMaxItems = 1 << 18;    // (instance, 8-state group) items per call

__global__ void gather_gen_kernel(int n, long long total, const GenEntry* __restrict__ tab, z64* __restrict__ G) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / nn, o = e - s * nn;
    const GenEntry g = tab[s];
    const z64 a = g.Lb[o], b = g.Ld[o];
    const double u = *g.u;
    G[e] = make_double2(fma(u, b.x, a.x), fma(u, b.y, a.y));
  }
}

// One CTA per work item.  FP64: Gauss three-product form with P planes
// (re, im, re + im).  F32: D = P - I in FP32 (interleaved complex),
// rho <- rho + D rho by the register-blocked step of res32.cuh, optional
// trace renormalisation.
template <bool F32>
__global__ void __launch_bounds__(512)
    worklist_kernel(int n, int d, int chunk, const WorkItem* __restrict__ items, int renorm) {
  extern __shared__ __align__(16) double wsm[];
  const WorkItem it = items[blockIdx.x];
  const int nb = it.nb, tid = threadIdx.x, work = nb * n;
  const long long nn = (long long)n * n;
  if (!F32) {
    double* Pr = wsm;
    double* Pi = Pr + nn;
    double* Ps = Pi + nn;
    double* xr = Ps + nn;
    double* xi = xr + chunk * n;
    double* xs = xi + chunk * n;
    double* yr = xs + chunk * n;
    double* yi = yr + chunk * n;
    for (int e = tid; e < work; e += blockDim.x) {
      const z64 v = it.X[e];
      xr[e] = v.x;
      xi[e] = v.y;
      xs[e] = v.x + v.y;
    }
    for (int s = 0; s < it.nslices; s++) {
      __syncthreads();
      for (int e = tid; e < nn; e += blockDim.x) {
        const z64 v = it.P[s * nn + e];
        Pr[e] = v.x;
        Pi[e] = v.y;
        Ps[e] = v.x + v.y;
      }
      __syncthreads();
      for (int t = 0; t < it.steps; t++) {
        for (int e = tid; e < work; e += blockDim.x) {
          const int q = e / n, i = e - (e / n) * n;
          double a1 = 0.0, a2 = 0.0, a3 = 0.0;
          for (int j = 0; j < n; j++) {
            a1 = fma(Pr[i * n + j], xr[q * n + j], a1);
            a2 = fma(Pi[i * n + j], xi[q * n + j], a2);
            a3 = fma(Ps[i * n + j], xs[q * n + j], a3);
          }
          yr[e] = a1 - a2;
          yi[e] = a3 - a1 - a2;
        }
        __syncthreads();
        for (int e = tid; e < work; e += blockDim.x) {
          xr[e] = yr[e];
          xi[e] = yi[e];
          xs[e] = yr[e] + yi[e];
        }
        __syncthreads();
      }
    }
    for (int e = tid; e < work; e += blockDim.x) it.X[e] = make_double2(xr[e], xi[e]);
  } else {
    float2* D = (float2*)wsm;
    float2* X = D + nn;
    float2* Y = X + chunk * n;
    float2* C = Y + chunk * n;
    const int nt = blockDim.x;
    for (int e = tid; e < work; e += nt) {
      const z64 v = it.X[e];
      X[e] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    if (renorm) res32_traces(n, d, nb, X, C, tid, nt);
    for (int s = 0; s < it.nslices; s++) {
      __syncthreads();
      for (int e = tid; e < nn; e += nt) {
        z64 v = it.P[s * nn + e];
        if (e / n == e % n) v.x -= 1.0;
        D[e] = make_float2((float)v.x, (float)v.y);
      }
      __syncthreads();
      for (int t = 0; t < it.steps; t++) {
        res32_step<2>(n, nb, D, X, Y, tid, nt, renorm ? C : nullptr);  // trace factor of X applied to Y
        __syncthreads();
        if (renorm) {
          res32_traces(n, d, nb, Y, C, tid, nt);
          __syncthreads();
        }
        float2* tmp = X;
        X = Y;
        Y = tmp;
      }
    }
    if (renorm && (long long)it.nslices * it.steps > 0) {  // the last step's trace factor
      res32_renorm(n, d, nb, X, C, tid, nt);
      __syncthreads();
    }
    for (int e = tid; e < work; e += nt) it.X[e] = make_double2((double)X[e].x, (double)X[e].y);
  }
}

size_t worklist_smem(int n, int chunk, bool f32) {
  const size_t nn = (size_t)n * n;
  return f32 ? sizeof(float) * (2 * nn + 4 * (size_t)chunk * n + 2 * (size_t)chunk)
             : sizeof(double) * (3 * nn + 5 * (size_t)chunk * n);
}

}  // namespace

size_t inst_table_bytes() { return (size_t)kMaxEntries * sizeof(GenEntry) + (size_t)kMaxItems * sizeof(WorkItem); }

}  // namespace lb

using namespace lb;

extern "C" lb_status lb_run_instances(lb_ctx* c, const lb_instance* inst, int count, double dt, lb_precision prec,
                                      int renorm_trace, void* stream) {
  if (c == nullptr || (inst == nullptr && count > 0) || count < 0) return LB_EINVAL;
  if (prec != LB_FP64 && prec != LB_FP32 && prec != LB_BF16X3 && prec != LB_FP64_HERMITIAN &&
      prec != LB_FP32_HERMITIAN && prec != LB_FP64_SLICED)
    return LB_EINVAL;
  const bool herm = prec == LB_FP64_HERMITIAN || prec == LB_FP32_HERMITIAN || prec == LB_FP64_SLICED;
  // propagation precision: the FP32 real-coordinate build propagates in FP32
  const lb_precision pprec = prec == LB_FP32_HERMITIAN ? LB_FP32 : prec;
  long long total_slices = 0, total_items = 0;
  for (int i = 0; i < count; i++) {
    const lb_instance& x = inst[i];
    const int n = x.d * x.d;
    if (x.d < 1 || n > c->max_n || x.nslices < 0 || x.steps_per_slice < 0 || x.B < 1) return LB_EINVAL;
    if (x.nslices > 0 && (x.Lbase == nullptr || x.Ldrv == nullptr || x.u == nullptr || x.states == nullptr))
      return LB_EINVAL;
    if (x.nslices > c->max_slices) return LB_EUNSUPPORTED;
    if (n > 81 && x.B > c->max_batch) return LB_EUNSUPPORTED;
    total_slices += x.nslices;
    total_items += (x.B + 7) / 8;
  }
  if (total_slices > kMaxEntries || total_items > kMaxItems) return LB_EUNSUPPORTED;
  if (count == 0 || total_slices == 0) return LB_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != c->device) cudaSetDevice(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  lb_status rs = [&]() -> lb_status {
    // the pinned staging of the previous call must have reached the device
    // (while capturing, the upload is a graph node that reads the staging at
    // replay, and the host may not wait)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
    if (capturing && c->max_squarings < 0) return LB_EUNSUPPORTED;
    if (!capturing) LB_CUDA(cudaEventSynchronize(c->ev_tab));
    GenEntry* htab = (GenEntry*)c->inst_tab_host;
    WorkItem* hitem = (WorkItem*)((char*)c->inst_tab_host + (size_t)kMaxEntries * sizeof(GenEntry));
    GenEntry* dtab = (GenEntry*)c->inst_tab_dev;
    WorkItem* ditem = (WorkItem*)((char*)c->inst_tab_dev + (size_t)kMaxEntries * sizeof(GenEntry));
    // groups by n, chunks of whole instances (<= max_slices slices each)
    std::vector<int> order(count);
    for (int i = 0; i < count; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return inst[a].d < inst[b].d; });
    struct Chunk {
      int n, first, last;  // instances order[first..last)
      long long tab0, item0;
      int S, items;
    };
    std::vector<Chunk> chunks;
    long long te = 0, ti = 0;
    for (int k = 0; k < count;) {
      const int d = inst[order[k]].d, n = d * d;
      Chunk ch{n, k, k, te, ti, 0, 0};
      while (k < count && inst[order[k]].d == d && ch.S + inst[order[k]].nslices <= c->max_slices) {
        const lb_instance& x = inst[order[k]];
        for (int s = 0; s < x.nslices; s++)
          htab[te++] = GenEntry{(const z64*)x.Lbase, (const z64*)x.Ldrv, x.u + s};
        ch.S += x.nslices;
        k++;
      }
      ch.last = k;
      chunks.push_back(ch);
    }
    // work items (n <= 81): groups of up to 8 states of one instance; P
    // points at the instance's first propagator in Pinst (the chunk's slices
    // are built there contiguously, in table order)
    for (Chunk& ch : chunks) {
      ch.item0 = ti;
      if (ch.n <= 81) {
        const long long nn = (long long)ch.n * ch.n;
        long long off = 0;
        for (int k = ch.first; k < ch.last; k++) {
          const lb_instance& x = inst[order[k]];
          for (int b0 = 0; b0 < x.B; b0 += 8)
            hitem[ti++] = WorkItem{c->Pinst + off, (z64*)x.states + (long long)b0 * ch.n, x.nslices,
                                   x.steps_per_slice, std::min(8, x.B - b0)};
          off += (long long)x.nslices * nn;
        }
      }
      ch.items = (int)(ti - ch.item0);
    }
    LB_CUDA(cudaMemcpyAsync(dtab, htab, sizeof(GenEntry) * te, cudaMemcpyHostToDevice, st));
    if (ti > 0) LB_CUDA(cudaMemcpyAsync(ditem, hitem, sizeof(WorkItem) * ti, cudaMemcpyHostToDevice, st));
    if (!capturing) LB_CUDA(cudaEventRecord(c->ev_tab, st));
    for (const Chunk& ch : chunks) {
      if (ch.S == 0) continue;
      const int n = ch.n;
      int d = 1;
      while (d * d < n) d++;
      const long long nn = (long long)n * n;
      const long long total = nn * ch.S;
      long long g = (total + 255) / 256;
      if (g > 152LL * 16) g = 152LL * 16;
      count_launch();
      gather_gen_kernel<<<(unsigned)g, 256, 0, st>>>(n, total, dtab + ch.tab0, c->Ginst);
      LB_CUDA(cudaGetLastError());
      lb_status r = herm ? expm_chunk_herm(c, n, ch.S, c->Ginst, nullptr, nullptr, dt, prec, c->Pinst, nullptr, st)
                         : expm_chunk_public(c, n, ch.S, c->Ginst, nullptr, nullptr, dt, prec, c->Pinst, nullptr, st);
      if (r != LB_OK) return r;
      if (n <= 81) {
        // the FP64 forms: the complex FP64 step (exact for every state)
        const bool f32 = pprec != LB_FP64 && pprec != LB_FP64_HERMITIAN && pprec != LB_FP64_SLICED;
        const size_t smem = worklist_smem(n, 8, f32);
        if (f32) {
          LB_CUDA(set_smem_once((const void*)worklist_kernel<true>, smem));
          const int threads = std::max(64, (n * 4 + 31) / 32 * 32);  // (row, pair of states) units, 8 states
          count_launch();
          worklist_kernel<true><<<ch.items, threads, smem, st>>>(n, d, 8, ditem + ch.item0, renorm_trace);
        } else {
          LB_CUDA(set_smem_once((const void*)worklist_kernel<false>, smem));
          count_launch();
          worklist_kernel<false><<<ch.items, 256, smem, st>>>(n, d, 8, ditem + ch.item0, 0);
        }
        LB_CUDA(cudaGetLastError());
      } else {
        long long off = 0;
        for (int k = ch.first; k < ch.last; k++) {
          const lb_instance& x = inst[order[k]];
          r = propagate_impl(c, n, x.nslices, c->Pinst + off, x.steps_per_slice, x.B, (z64*)x.states, pprec,
                             renorm_trace, st);
          if (r != LB_OK) return r;
          off += (long long)x.nslices * nn;
        }
      }
    }
    return LB_OK;
  }();
  if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
  return rs;
}
