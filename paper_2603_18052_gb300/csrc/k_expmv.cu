// Action of the slice propagators on the states without forming them: the
// route the paper's discussion (Sec. 5) recommends for removing the LU solve,
// after the action-of-the-exponential methods it cites (Al-Mohy and Higham;
// EXPOKIT).  For every control slice the states advance by
//     X <- exp(A_s) X,   A_s = (L_base + u_s L_drv) dt,
// through s sub-steps of the degree-m Taylor series,
//     y <- y + sum_{k=1..m} V_k,   V_k = (A_s / s) V_{k-1} / k,  V_0 = y,
// so each term is one product of the n x n generator with the B states:
// the few-state kernel (k_gemv.cu) for B <= 8, the tiled FP64 GEMM with its
// second output (y += alpha * product) above.  Nothing of size n^2 is formed
// besides the generators themselves, and no factorisation runs.
//
// Parameters (chosen a priori, one pair per call): theta_m is the largest
// theta with theta^(m+1)/(m+1)! e^theta <= 2^-53, the bound on the relative
// remainder of the degree-m Taylor polynomial of exp(X) applied to a vector
// when ||X||_1 <= theta; (m, s) is the pair with the fewest products m * s
// such that a / s <= theta_m, 1 <= m <= 55 (the smaller m on ties), where a
// is the largest ||A_s||_1 of the call.
#include "lb_internal.cuh"

#include <cmath>
#include <cstring>

namespace lb {
namespace {

constexpr int kTaylorMaxM = 55;
constexpr int kTaylorMaxS = 1 << 16;

// A_s = (L_base + u_s L_drv) dt (or L_base[s] dt without a drive), written
// when A is not null; the largest column abs-sum over all slices goes to
// *norm_bits when that is not null (the bit pattern of a non-negative double
// orders like the integer).  A CTA takes 8 columns of one slice (128-byte
// row segments) and 32 row groups (every 32nd row); the 32 partial sums of a
// column meet in shared memory in a fixed order.  Narrow column blocks give
// enough CTAs for all SMs even for one or two slices: the FP64 work here
// (the modulus takes a square root) runs at 1/64 of the FP32 rate.
constexpr int kGenCols = 8, kGenRowGroups = 32;

__global__ void __launch_bounds__(kGenCols * kGenRowGroups)
    expmv_generators_kernel(int n, int S, const z64* __restrict__ Lb, const z64* __restrict__ Ld,
                            const double* __restrict__ u, double dt, z64* __restrict__ A,
                            unsigned long long* __restrict__ norm_bits) {
  __shared__ double part[kGenRowGroups][kGenCols];
  const long long nn = (long long)n * n;
  const int c = threadIdx.x % kGenCols, rg = threadIdx.x / kGenCols;
  const int cblocks = (n + kGenCols - 1) / kGenCols;
  for (long long t = blockIdx.x; t < (long long)S * cblocks; t += gridDim.x) {
    const int s = (int)(t / cblocks), j = (int)(t - (t / cblocks) * cblocks) * kGenCols + c;
    double sum = 0.0;
    if (j < n) {
      const double us = Ld != nullptr ? u[s] : 0.0;
      const z64* base = Ld != nullptr ? Lb : Lb + s * nn;
      for (int i = rg; i < n; i += kGenRowGroups) {
        const long long e = (long long)i * n + j;
        z64 v = base[e];
        if (Ld != nullptr) {  // (L_base + u_s L_drv) dt, products and sums rounded separately
          const z64 w = Ld[e];
          v.x = __dadd_rn(v.x, __dmul_rn(us, w.x));
          v.y = __dadd_rn(v.y, __dmul_rn(us, w.y));
        }
        v.x = __dmul_rn(v.x, dt);
        v.y = __dmul_rn(v.y, dt);
        if (A != nullptr) A[s * nn + e] = v;
        if (norm_bits != nullptr) sum += sqrt(__dadd_rn(__dmul_rn(v.x, v.x), __dmul_rn(v.y, v.y)));
      }
    }
    if (norm_bits != nullptr) {
      part[rg][c] = sum;
      __syncthreads();
      if (rg == 0 && j < n) {
        double col = 0.0;
        for (int r = 0; r < kGenRowGroups; r++) col += part[r][c];
        if (!(col == col)) col = INFINITY;  // a NaN anywhere reports as a non-finite norm
        atomicMax(norm_bits, (unsigned long long)__double_as_longlong(col));
      }
      __syncthreads();
    }
  }
}

// theta_m by bisection on the logarithm of the bound (increasing in theta).
double taylor_theta(int m) {
  const double lg = std::lgamma(m + 2.0), lu = std::log(std::ldexp(1.0, -53));
  double lo = 1e-300, hi = 64.0;
  for (int it = 0; it < 200; it++) {
    const double mid = 0.5 * (lo + hi);
    if ((m + 1) * std::log(mid) + mid - lg - lu <= 0.0)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

const double* theta_table() {
  static const struct T {
    double v[kTaylorMaxM + 1];
    T() {
      v[0] = 0.0;
      for (int m = 1; m <= kTaylorMaxM; m++) v[m] = taylor_theta(m);
    }
  } table;
  return table.v;
}

}  // namespace

bool taylor_parameters(double a, int* m_out, int* s_out) {
  if (!(a >= 0.0) || !std::isfinite(a)) return false;
  const double* th = theta_table();
  long long best_m = 0, best_s = 0;
  for (int m = 1; m <= kTaylorMaxM; m++) {
    const double q = std::ceil(a / th[m]);
    if (q > (double)kTaylorMaxS) continue;
    const long long s = q < 1.0 ? 1 : (long long)q;
    if (best_m == 0 || m * s < best_m * best_s) {
      best_m = m;
      best_s = s;
    }
  }
  if (best_m == 0) return false;
  *m_out = (int)best_m;
  *s_out = (int)best_s;
  return true;
}

}  // namespace lb

using namespace lb;

extern "C" lb_status lb_expmv(lb_ctx* c, int n, int nslices, const lb_c64* Lbase, const lb_c64* Ldrv,
                              const double* u, double dt, int B, lb_c64* states, int* ms_out, void* stream) {
  if (c == nullptr || Lbase == nullptr || states == nullptr) return LB_EINVAL;
  if (n < 1 || n > c->max_n || nslices < 0 || B < 1 || B > c->max_batch) return LB_EINVAL;
  if (Ldrv != nullptr && u == nullptr) return LB_EINVAL;
  if (!std::isfinite(dt)) return LB_EINVAL;
  if (nslices == 0) return LB_OK;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return LB_EUNSUPPORTED;  // the parameter choice reads the norm back to the host
  const long long nn = (long long)n * n;
  const z64* Lb = (const z64*)Lbase;
  const z64* Ld = (const z64*)Ldrv;
  auto grid_for = [&](int S) {
    const long long g = (long long)S * ((n + kGenCols - 1) / kGenCols);
    const long long cap = (long long)c->sm_count * 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
  };
  // when every slice fits in one chunk the generators are formed by the
  // same pass that takes their norms
  const bool one_chunk = nslices <= c->max_slices;

  // 1. the largest ||A_s||_1 over the call, then (m, s)
  unsigned long long* nb = c->norm_bits;
  LB_CUDA(cudaMemsetAsync(nb, 0, sizeof(unsigned long long), st));
  count_launch();
  expmv_generators_kernel<<<grid_for(nslices), kGenCols * kGenRowGroups, 0, st>>>(n, nslices, Lb, Ld, u, dt, one_chunk ? c->A : nullptr,
                                                             nb);
  LB_CUDA(cudaGetLastError());
  unsigned long long bits = 0;
  LB_CUDA(cudaMemcpyAsync(&bits, nb, sizeof(bits), cudaMemcpyDeviceToHost, st));
  LB_CUDA(cudaStreamSynchronize(st));
  double a = 0.0;
  std::memcpy(&a, &bits, sizeof(a));
  if (!std::isfinite(a)) return LB_ENONFINITE;
  int m = 0, s = 0;
  if (!taylor_parameters(a, &m, &s)) return LB_EUNSUPPORTED;
  if (ms_out != nullptr) {
    ms_out[0] = m;
    ms_out[1] = s;
  }

  // 2. per chunk of slices: form the generators, then the Taylor sub-steps
  z64* Y = (z64*)states;
  z64* Va = c->Rtmp;  // two B x n term buffers
  z64* Vb = c->Xh;
  const size_t xbytes = sizeof(z64) * (size_t)B * n;
  const bool small = B <= kGemvMaxB;
  for (int s0 = 0; s0 < nslices; s0 += c->max_slices) {
    const int S = (nslices - s0 < c->max_slices) ? nslices - s0 : c->max_slices;
    if (!one_chunk) {
      count_launch();
      expmv_generators_kernel<<<grid_for(S), kGenCols * kGenRowGroups, 0, st>>>(n, S, Ld != nullptr ? Lb : Lb + s0 * nn, Ld,
                                                           u != nullptr ? u + s0 : nullptr, dt, c->A, nullptr);
      LB_CUDA(cudaGetLastError());
    }
    for (int sl = 0; sl < S; sl++) {
      const z64* A = c->A + sl * nn;
      for (int sub = 0; sub < s; sub++) {
        LB_CUDA(cudaMemcpyAsync(Va, Y, xbytes, cudaMemcpyDeviceToDevice, st));
        z64* prev = Va;
        z64* next = Vb;
        for (int k = 1; k <= m; k++) {
          const double alpha = 1.0 / ((double)s * (double)k);
          if (small) {
            LB_CUDA(launch_zgemv_f64(n, B, A, n, prev, n, next, n, alpha, Y, n, st));
          } else {
            ZGemmProblem q;
            q.M = B; q.N = n; q.K = n;
            q.A = prev; q.lda = n;
            q.B = A; q.ldb = n; q.opB = 1;
            q.C = next; q.ldc = n;
            q.alpha = alpha;
            q.C2 = Y; q.X2 = Y; q.alpha2 = alpha;
            q.batch = 1;
            LB_CUDA(zgemm_f64(&q, 1, c->sm_count, st));
          }
          z64* tmp = prev;
          prev = next;
          next = tmp;
        }
      }
    }
  }
  return LB_OK;
}

// The same route on the real coordinates of Hermitian states (density
// matrices): the generators A_s map Hermitian matrices to Hermitian
// matrices, so on the n real coordinates of a state (diagonal, Re and Im of
// the upper triangle) each A_s is a real n x n matrix G_s (herm_matrix_kernel
// forms it from A_s as it does for a propagator), and every Taylor term is a
// real matrix-vector product: a quarter of the FP64 multiply-adds.  (m, s)
// follows the same rule with a = the largest ||G_s||_1.  Few states only
// (B <= 8, the few-state product); larger batches take lb_expmv.
extern "C" lb_status lb_expmv_hermitian(lb_ctx* c, int n, int nslices, const lb_c64* Lbase, const lb_c64* Ldrv,
                                        const double* u, double dt, int B, lb_c64* states, int* ms_out,
                                        void* stream) {
  if (c == nullptr || Lbase == nullptr || states == nullptr) return LB_EINVAL;
  if (n < 1 || n > c->max_n || nslices < 0 || B < 1 || B > c->max_batch) return LB_EINVAL;
  int d = 1;
  while (d * d < n) d++;
  if (d * d != n) return LB_EINVAL;
  if (Ldrv != nullptr && u == nullptr) return LB_EINVAL;
  if (!std::isfinite(dt)) return LB_EINVAL;
  if (nslices == 0) return LB_OK;
  if (B > kGemvMaxB) return lb_expmv(c, n, nslices, Lbase, Ldrv, u, dt, B, states, ms_out, stream);
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return LB_EUNSUPPORTED;  // the parameter choice reads the norm back to the host
  const long long nn = (long long)n * n;
  const z64* Lb = (const z64*)Lbase;
  const z64* Ld = (const z64*)Ldrv;
  auto grid_for = [&](int S) {
    const long long gr = (long long)S * ((n + kGenCols - 1) / kGenCols);
    const long long cap = (long long)c->sm_count * 8;
    return (unsigned)(gr < 1 ? 1 : (gr > cap ? cap : gr));
  };
  double* G = (double*)c->Z1;  // S real n x n generators
  auto form = [&](int s0, int S, unsigned long long* nb) -> lb_status {
    count_launch();
    expmv_generators_kernel<<<grid_for(S), kGenCols * kGenRowGroups, 0, st>>>(
        n, S, Ld != nullptr ? Lb : Lb + s0 * nn, Ld, u != nullptr ? u + s0 : nullptr, dt, c->A, nullptr);
    LB_CUDA(cudaGetLastError());
    LB_CUDA(launch_herm_matrix(n, d, S, c->A, G, c->sm_count, st));
    if (nb != nullptr) LB_CUDA(launch_real_colnorm(n, S, G, nb, c->sm_count, st));
    return LB_OK;
  };

  // 1. the largest ||G_s||_1 over the call, then (m, s)
  unsigned long long* nb = c->norm_bits;
  LB_CUDA(cudaMemsetAsync(nb, 0, sizeof(unsigned long long), st));
  for (int s0 = 0; s0 < nslices; s0 += c->max_slices) {
    const int S = (nslices - s0 < c->max_slices) ? nslices - s0 : c->max_slices;
    lb_status r = form(s0, S, nb);
    if (r != LB_OK) return r;
  }
  unsigned long long bits = 0;
  LB_CUDA(cudaMemcpyAsync(&bits, nb, sizeof(bits), cudaMemcpyDeviceToHost, st));
  LB_CUDA(cudaStreamSynchronize(st));
  double a = 0.0;
  std::memcpy(&a, &bits, sizeof(a));
  if (!std::isfinite(a)) return LB_ENONFINITE;
  int m = 0, s = 0;
  if (!taylor_parameters(a, &m, &s)) return LB_EUNSUPPORTED;
  if (ms_out != nullptr) {
    ms_out[0] = m;
    ms_out[1] = s;
  }

  // 2. the states' coordinates through the slices
  z64* X = (z64*)states;
  double* Y = (double*)c->Xh;
  double* Va = (double*)c->Rtmp;  // two B x n term buffers
  double* Vb = Va + (size_t)B * n;
  LB_CUDA(launch_herm_coords_in(n, d, B, X, Y, c->sm_count, st));
  const bool one_chunk = nslices <= c->max_slices;
  for (int s0 = 0; s0 < nslices; s0 += c->max_slices) {
    const int S = (nslices - s0 < c->max_slices) ? nslices - s0 : c->max_slices;
    if (!one_chunk) {
      lb_status r = form(s0, S, nullptr);
      if (r != LB_OK) return r;
    }
    for (int sl = 0; sl < S; sl++) {
      const double* Gs = G + sl * nn;
      for (int sub = 0; sub < s; sub++) {
        LB_CUDA(cudaMemcpyAsync(Va, Y, sizeof(double) * (size_t)B * n, cudaMemcpyDeviceToDevice, st));
        double* prev = Va;
        double* next = Vb;
        for (int k = 1; k <= m; k++) {
          LB_CUDA(launch_dgemv_f64(n, B, Gs, n, prev, n, next, n, 1.0 / ((double)s * (double)k), Y, n, st));
          double* tmp = prev;
          prev = next;
          next = tmp;
        }
      }
    }
  }
  LB_CUDA(launch_herm_coords_out(n, d, B, Y, X, c->sm_count, st));
  return LB_OK;
}
