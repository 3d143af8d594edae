// Warm-start network: a small dense MLP (ReLU hidden layers, linear output)
// that proposes control amplitudes for the GRAPE chain of Sec. 2.5.  Weights
// are stored in BF16 (an FP32 master copy lives with the optimiser), every
// product accumulates in FP32.  The shapes are tiny (batch x 4 -> 256 -> 256 ->
// 256 -> 100), so the products are tiled FP32 GEMMs on the CUDA cores; the
// tensor cores would idle on them.
//
// Layout: layer l maps dims[l] -> dims[l+1]; W_l is dims[l+1] x dims[l]
// row-major, packed back to back (BF16); b_l packed likewise (FP32).  acts
// holds the outputs of every layer, batch x dims[l+1] each, back to back
// (hidden layers after the ReLU).
#include "lb_internal.cuh"

#include <cuda_bf16.h>

#include <vector>

namespace lb {

namespace {

// C[M][N] = sum_k A(m, k) B(k, n) (+ bias[n], ReLU) with
//   A(m, k) = TA ? A[k * lda + m] : A[m * lda + k]     (FP32)
//   B(k, n) = TB ? B[n * ldb + k] : B[k * ldb + n]     (BF16 when BB, else FP32)
// mask (optional): C[m][n] = 0 where mask[m * ldc + n] <= 0 (ReLU derivative).
// accumulate: C += result.
template <bool TA, bool TB, bool BB>
__global__ void __launch_bounds__(256)
    sgemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda, const void* __restrict__ Bv, int ldb,
                 float* __restrict__ C, int ldc, const float* __restrict__ bias, int relu,
                 const float* __restrict__ mask, int accumulate) {
  constexpr int BM = 32, BN = 32, BK = 16;
  __shared__ float As[BK][BM + 1], Bs[BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 2 x 2 outputs each
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      const int m = TA ? e % BM : e / BK, k = TA ? e / BM : e % BK;
      const int gm = m0 + m, gk = k0 + k;
      float v = 0.f;
      if (gm < M && gk < K) v = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[k][m] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      const int n = TB ? e / BK : e % BN, k = TB ? e % BK : e / BN;
      const int gn = n0 + n, gk = k0 + k;
      float v = 0.f;
      if (gn < N && gk < K) {
        const long long idx = TB ? (long long)gn * ldb + gk : (long long)gk * ldb + gn;
        v = BB ? __bfloat162float(((const __nv_bfloat16*)Bv)[idx]) : ((const float*)Bv)[idx];
      }
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; k++) {
      const float a0 = As[k][ty * 2], a1 = As[k][ty * 2 + 1];
      const float b0 = Bs[k][tx * 2], b1 = Bs[k][tx * 2 + 1];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const int gm = m0 + ty * 2 + i, gn = n0 + tx * 2 + j;
      if (gm >= M || gn >= N) continue;
      float v = acc[i][j];
      if (bias != nullptr) v += bias[gn];
      if (relu) v = fmaxf(v, 0.f);
      const long long o = (long long)gm * ldc + gn;
      if (mask != nullptr && !(mask[o] > 0.f)) v = 0.f;
      C[o] = accumulate ? C[o] + v : v;
    }
}

// gb[n] = sum_m dZ[m][n] (fixed-order reduction over the batch)
__global__ void colsum_kernel(int M, int N, const float* __restrict__ dZ, float* __restrict__ gb) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; m++) s += dZ[(long long)m * N + n];
  gb[n] = s;
}

// dy = 2 (y - t) / count;  loss = mean (y - t)^2 (one block, fixed order)
__global__ void mse_kernel(long long count, const float* __restrict__ y, const float* __restrict__ t,
                           float* __restrict__ dy, float* __restrict__ loss) {
  __shared__ float red[256];
  float acc = 0.f;
  const float sc = 2.f / (float)count;
  for (long long e = threadIdx.x; e < count; e += blockDim.x) {
    const float r = y[e] - t[e];
    dy[e] = sc * r;
    acc = fmaf(r, r, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss != nullptr) *loss = red[0] / (float)count;
}

// Adam (Kingma and Ba) with bias correction; optional BF16 shadow copy.
template <typename T>
__global__ void adam_kernel(long long count, T* __restrict__ p, const T* __restrict__ g, T* __restrict__ m,
                            T* __restrict__ v, __nv_bfloat16* __restrict__ pb, T lr, T b1, T b2, T eps, T c1, T c2,
                            T sign) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const T gi = sign * g[e];
    const T mi = b1 * m[e] + (T(1) - b1) * gi;
    const T vi = b2 * v[e] + (T(1) - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const T mh = mi / c1, vh = vi / c2;
    const T pi = p[e] - lr * mh / (sqrt(vh) + eps);
    p[e] = pi;
    if (pb != nullptr) pb[e] = __float2bfloat16_rn((float)pi);
  }
}

template <bool TA, bool TB, bool BB>
cudaError_t gemm(int M, int N, int K, const float* A, int lda, const void* B, int ldb, float* C, int ldc,
                 const float* bias, int relu, const float* mask, int accumulate, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + 31) / 32, (M + 31) / 32);
  count_launch();
  sgemm_kernel<TA, TB, BB><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, mask, accumulate);
  return cudaGetLastError();
}

bool check_dims(int nlayers, const int* dims, int batch) {
  if (nlayers < 1 || nlayers > 16 || dims == nullptr || batch < 1) return false;
  for (int l = 0; l <= nlayers; l++)
    if (dims[l] < 1 || dims[l] > 65536) return false;
  return true;
}

}  // namespace

}  // namespace lb

using namespace lb;

extern "C" {

lb_status lb_mlp_forward(int nlayers, const int* dims, int batch, const void* W, const float* b, const float* x,
                         float* acts, void* stream) {
  if (!check_dims(nlayers, dims, batch) || W == nullptr || b == nullptr || x == nullptr || acts == nullptr)
    return LB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const __nv_bfloat16* w = (const __nv_bfloat16*)W;
  const float* in = x;
  float* out = acts;
  for (int l = 0; l < nlayers; l++) {
    const int di = dims[l], dout = dims[l + 1];
    LB_CUDA((gemm<false, true, true>(batch, dout, di, in, di, w, di, out, dout, b, l + 1 < nlayers, nullptr, 0,
                                     st)));
    w += (long long)dout * di;
    b += dout;
    in = out;
    out += (long long)batch * dout;
  }
  return LB_OK;
}

lb_status lb_mlp_backward(int nlayers, const int* dims, int batch, const void* W, const float* x, const float* acts,
                          const float* dy, float* gW, float* gb, float* scratch, void* stream) {
  if (!check_dims(nlayers, dims, batch) || W == nullptr || x == nullptr || acts == nullptr || dy == nullptr ||
      gW == nullptr || gb == nullptr || scratch == nullptr)
    return LB_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<long long> woff(nlayers + 1, 0), boff(nlayers + 1, 0), aoff(nlayers + 1, 0);
  for (int l = 0; l < nlayers; l++) {
    woff[l + 1] = woff[l] + (long long)dims[l + 1] * dims[l];
    boff[l + 1] = boff[l] + dims[l + 1];
    aoff[l + 1] = aoff[l] + (long long)batch * dims[l + 1];
  }
  int maxd = 0;
  for (int l = 0; l <= nlayers; l++) maxd = dims[l] > maxd ? dims[l] : maxd;
  // scratch: two batch x maxd buffers for the layer gradients dZ
  float* dz = scratch;
  float* dprev = scratch + (long long)batch * maxd;
  const __nv_bfloat16* w = (const __nv_bfloat16*)W;
  LB_CUDA(cudaMemcpyAsync(dz, dy, sizeof(float) * batch * dims[nlayers], cudaMemcpyDeviceToDevice, st));
  for (int l = nlayers - 1; l >= 0; l--) {
    const int di = dims[l], dout = dims[l + 1];
    const float* xin = l == 0 ? x : acts + aoff[l - 1];
    // gW_l[o][i] = sum_b dZ[b][o] xin[b][i]
    LB_CUDA((gemm<true, false, false>(dout, di, batch, dz, dout, xin, di, gW + woff[l], di, nullptr, 0, nullptr, 0,
                                      st)));
    count_launch();
    colsum_kernel<<<(dout + 127) / 128, 128, 0, st>>>(batch, dout, dz, gb + boff[l]);
    LB_CUDA(cudaGetLastError());
    if (l > 0) {
      // dZ_{l-1}[b][i] = sum_o dZ[b][o] W_l[o][i], masked by the ReLU of layer l-1
      LB_CUDA((gemm<false, false, true>(batch, di, dout, dz, dout, w + woff[l], di, dprev, di, nullptr, 0,
                                        acts + aoff[l - 1], 0, st)));
      float* t = dz;
      dz = dprev;
      dprev = t;
    }
  }
  return LB_OK;
}

lb_status lb_mse_loss_grad(long long count, const float* y, const float* t, float* dy, float* loss, void* stream) {
  if (count < 1 || y == nullptr || t == nullptr || dy == nullptr) return LB_EINVAL;
  count_launch();
  mse_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(count, y, t, dy, loss);
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

lb_status lb_adam_step(long long count, float* p, const float* g, float* m, float* v, void* p_bf16, float lr,
                       float beta1, float beta2, float eps, int step, void* stream) {
  if (count < 1 || p == nullptr || g == nullptr || m == nullptr || v == nullptr || step < 1) return LB_EINVAL;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  long long grid = (count + 255) / 256;
  if (grid > 152 * 16) grid = 152 * 16;
  count_launch();
  adam_kernel<float><<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(
      count, p, g, m, v, (__nv_bfloat16*)p_bf16, lr, beta1, beta2, eps, c1, c2, 1.f);
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

lb_status lb_adam_step_f64(long long count, double* p, const double* g, double* m, double* v, double lr,
                           double beta1, double beta2, double eps, int step, int ascend, void* stream) {
  if (count < 1 || p == nullptr || g == nullptr || m == nullptr || v == nullptr || step < 1) return LB_EINVAL;
  const double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
  long long grid = (count + 255) / 256;
  if (grid > 152 * 16) grid = 152 * 16;
  count_launch();
  adam_kernel<double><<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(
      count, p, g, m, v, nullptr, lr, beta1, beta2, eps, c1, c2, ascend ? -1.0 : 1.0);
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

}  // extern "C"
