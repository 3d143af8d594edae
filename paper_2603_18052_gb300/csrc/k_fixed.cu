// Fixed-point propagation: the element-serial Q1.15 step of the FPGA design
// (Algorithm alg:fpga, Sec. 3.5), and its 32-bit Q1.31 variant
// (Figure fig:fixed_point_drift), reproduced bit for bit on the GPU.
//
// A Q1.f code c (two's complement, 1 + f bits) stands for c / 2^f.  One step
// forms, for every output row i, the exact complex accumulator
//   acc_i = sum_j P_ij rho_j      (four integer products per term)
// and writes rho_i = sat(floor(acc_i / 2^f)), the clamp being to the code
// range [-2^f, 2^f - 1].  The board's accumulator has 33 + ceil(log2 n)
// bits; here it is 64 bits for Q1.15 (products of 16-bit codes are exact in
// 32 bits, sums of 2n of them stay below 2^40 for n <= 81) and 128 bits for
// Q1.31 (products need 63 bits, sums up to 71), so nothing is ever lost and
// the result is the exact one whatever the summation order.
//
// Parallel form: the FPGA runs one state through k = 1 multiply-accumulate
// per cycle; here many independent states run at once.  A CTA holds P and
// its group of states in shared memory for all steps (n <= 81: P is at most
// 52 KiB in Q1.31); one thread owns one (state, row) output, consecutive
// threads consecutive rows of one state, so the state's codes are broadcast
// and the rows of P are read n words apart (no bank conflicts for odd n).
#include "lb_internal.cuh"

#include <cmath>

namespace lb {
namespace {

template <int F> struct Fx;
template <> struct Fx<15> {
  typedef short code;
  typedef short2 pair;
  typedef long long acc;
};
template <> struct Fx<31> {
  typedef int code;
  typedef int2 pair;
  typedef __int128 acc;
};

__device__ __forceinline__ short2 make_pair_code(short r, short i) { return make_short2(r, i); }
__device__ __forceinline__ int2 make_pair_code(int r, int i) { return make_int2(r, i); }

// acc + a * b exactly, a and b codes: for Q1.15 a 32 x 32 -> 64-bit
// multiply-add (the negated code -a of a subtracted term still fits 32 bits);
// for Q1.31 a 64-bit product added into 128 bits.
__device__ __forceinline__ long long mac(long long acc, short a, short b) {
  return acc + (long long)(int)a * (long long)(int)b;
}
__device__ __forceinline__ long long mac_neg(long long acc, short a, short b) {
  return acc + (long long)(-(int)a) * (long long)(int)b;
}
__device__ __forceinline__ __int128 mac(__int128 acc, int a, int b) {
  return acc + (__int128)((long long)a * (long long)b);
}
__device__ __forceinline__ __int128 mac_neg(__int128 acc, int a, int b) {
  return acc - (__int128)((long long)a * (long long)b);
}

// sat(floor(acc / 2^F)): the arithmetic right shift of a signed integer
// rounds towards minus infinity.
template <int F>
__device__ __forceinline__ typename Fx<F>::code floor_sat(typename Fx<F>::acc a) {
  typedef typename Fx<F>::acc A;
  const A q = a >> F;
  const A lo = -((A)1 << F), hi = ((A)1 << F) - 1;
  return (typename Fx<F>::code)(q < lo ? lo : (q > hi ? hi : q));
}

template <int F>
__global__ void __launch_bounds__(1024) fixed_chain_kernel(int n, int nsteps, int B, int per_cta,
                                                           const typename Fx<F>::pair* __restrict__ P,
                                                           typename Fx<F>::pair* __restrict__ X) {
  typedef typename Fx<F>::pair pair;
  typedef typename Fx<F>::acc acc;
  extern __shared__ __align__(16) unsigned char fixed_smem[];
  pair* Ps = reinterpret_cast<pair*>(fixed_smem);
  pair* S0 = Ps + n * n;
  pair* S1 = S0 + per_cta * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long q0 = (long long)blockIdx.x * per_cta;
  if (q0 >= B) return;
  const int nb = (int)min((long long)per_cta, (long long)B - q0);
  const int m = nb * n;
  for (int e = tid; e < n * n; e += nt) Ps[e] = P[e];
  for (int e = tid; e < m; e += nt) S0[e] = X[q0 * n + e];
  __syncthreads();
  pair* cur = S0;
  pair* nxt = S1;
  for (int t = 0; t < nsteps; t++) {
    for (int u = tid; u < m; u += nt) {
      const int q = u / n, i = u - q * n;
      const pair* prow = Ps + i * n;
      const pair* x = cur + q * n;
      acc ar = 0, ai = 0;
#pragma unroll 9  // measured: 20 % faster than no hint for one state at n = 9, 15 % for batches
      for (int j = 0; j < n; j++) {
        const pair a = prow[j], v = x[j];
        ar = mac_neg(mac(ar, a.x, v.x), a.y, v.y);
        ai = mac(mac(ai, a.x, v.y), a.y, v.x);
      }
      nxt[u] = make_pair_code(floor_sat<F>(ar), floor_sat<F>(ai));
    }
    __syncthreads();
    pair* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  for (int e = tid; e < m; e += nt) X[q0 * n + e] = cur[e];
}

// Nearest code (ties to even), saturated; NaN becomes 0.
template <int F>
__device__ __forceinline__ typename Fx<F>::code to_code(double v) {
  const double lo = -(double)(1LL << F), hi = (double)((1LL << F) - 1);
  double y = rint(v * (double)(1LL << F));
  if (y != y) y = 0.0;
  y = y < lo ? lo : (y > hi ? hi : y);
  return (typename Fx<F>::code)(long long)y;
}

template <int F>
__global__ void quantize_kernel(long long count, const double2* __restrict__ x, typename Fx<F>::pair* __restrict__ q) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x) {
    const double2 v = x[e];
    q[e] = make_pair_code(to_code<F>(v.x), to_code<F>(v.y));
  }
}

template <int F>
__global__ void dequantize_kernel(long long count, const typename Fx<F>::pair* __restrict__ q, double2* __restrict__ x) {
  const double s = 1.0 / (double)(1LL << F);  // a power of two: the division is exact
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x) {
    const typename Fx<F>::pair c = q[e];
    x[e] = make_double2((double)c.x * s, (double)c.y * s);
  }
}

bool square_n(int n) {
  int d = 1;
  while (d * d < n) d++;
  return d * d == n;
}

template <int F>
lb_status run_chain(int n, const void* P, int nsteps, int B, void* X, int sms, cudaStream_t st) {
  typedef typename Fx<F>::pair pair;
  // states per CTA: at most 1024 threads (one per output), and few enough
  // that B states give one CTA per SM when B allows
  const int cap = 1024 / n;
  int per = (int)((B + sms - 1) / sms);
  per = per < 1 ? 1 : (per > cap ? cap : per);
  int threads = ((per * n + 31) / 32) * 32;
  const size_t smem = sizeof(pair) * ((size_t)n * n + 2 * (size_t)per * n);
  const long long grid = ((long long)B + per - 1) / per;
  if (grid > 0x7fffffffLL) return LB_EUNSUPPORTED;
  if (set_smem_once((const void*)fixed_chain_kernel<F>, smem) != cudaSuccess) return LB_ECUDA;
  fixed_chain_kernel<F><<<(unsigned)grid, threads, smem, st>>>(n, nsteps, B, per, (const pair*)P, (pair*)X);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

template <int F>
lb_status run_convert(bool to_fixed, long long count, const void* in, void* out, int sms, cudaStream_t st) {
  typedef typename Fx<F>::pair pair;
  long long blocks = (count + 255) / 256;
  const long long cap = (long long)sms * 8;
  if (blocks > cap) blocks = cap;
  if (to_fixed)
    quantize_kernel<F><<<(unsigned)blocks, 256, 0, st>>>(count, (const double2*)in, (pair*)out);
  else
    dequantize_kernel<F><<<(unsigned)blocks, 256, 0, st>>>(count, (const pair*)in, (double2*)out);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

}  // namespace
}  // namespace lb

using namespace lb;

extern "C" lb_status lb_fixed_quantize(int frac_bits, long long count, const lb_c64* x, void* q, void* stream) {
  if (frac_bits != 15 && frac_bits != 31) return LB_EINVAL;
  if (count < 0 || ((x == nullptr || q == nullptr) && count > 0)) return LB_EINVAL;
  if (count == 0) return LB_OK;
  int dev = 0, sms = 0;
  lb_status s = current_device_sm103(&dev, &sms);
  if (s != LB_OK) return s;
  return frac_bits == 15 ? run_convert<15>(true, count, x, q, sms, (cudaStream_t)stream)
                         : run_convert<31>(true, count, x, q, sms, (cudaStream_t)stream);
}

extern "C" lb_status lb_fixed_dequantize(int frac_bits, long long count, const void* q, lb_c64* x, void* stream) {
  if (frac_bits != 15 && frac_bits != 31) return LB_EINVAL;
  if (count < 0 || ((x == nullptr || q == nullptr) && count > 0)) return LB_EINVAL;
  if (count == 0) return LB_OK;
  int dev = 0, sms = 0;
  lb_status s = current_device_sm103(&dev, &sms);
  if (s != LB_OK) return s;
  return frac_bits == 15 ? run_convert<15>(false, count, q, x, sms, (cudaStream_t)stream)
                         : run_convert<31>(false, count, q, x, sms, (cudaStream_t)stream);
}

extern "C" lb_status lb_propagate_fixed(int frac_bits, int n, const void* P_q, int nsteps, int B, void* states_q,
                                        void* stream) {
  if (frac_bits != 15 && frac_bits != 31) return LB_EINVAL;
  if (P_q == nullptr || states_q == nullptr) return LB_EINVAL;
  if (n < 1 || n > 81 || !square_n(n) || nsteps < 0 || B < 1) return LB_EINVAL;
  if (nsteps == 0) return LB_OK;
  int dev = 0, sms = 0;
  lb_status s = current_device_sm103(&dev, &sms);
  if (s != LB_OK) return s;
  return frac_bits == 15 ? run_chain<15>(n, P_q, nsteps, B, states_q, sms, (cudaStream_t)stream)
                         : run_chain<31>(n, P_q, nsteps, B, states_q, sms, (cudaStream_t)stream);
}
