// Element-wise and small-block kernels of the propagator build:
//   * the vectorised Lindbladian (Eq. 1-3),
//   * per-slice generator, 1-norm, squaring count and scaling (Eq. 5 and the
//     first line of Algorithm 1),
//   * the linear combinations of the Pade step,
//   * the diagonal-block factorisation of the blocked LU (Algorithm 1, the
//     solve line), with explicit inverses of the triangular diagonal blocks so
//     that every O(n^3) part of the factorisation and of the substitutions
//     becomes a GEMM.
#include "lb_internal.cuh"

namespace lb {

namespace {

__device__ __forceinline__ z64 cmul(z64 a, z64 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c - a*b
__device__ __forceinline__ z64 cfms(z64 a, z64 b, z64 c) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ z64 conjz(z64 a) { return make_double2(a.x, -a.y); }

// G = sum_k L_k^+ L_k  (d x d), one block.
__global__ void gram_kernel(int d, int K, const z64* __restrict__ Ls, z64* __restrict__ G) {
  for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
    const int a = e / d, c = e - (e / d) * d;
    double gr = 0.0, gi = 0.0;
    for (int q = 0; q < K; q++) {
      const z64* L = Ls + (long long)q * d * d;
      for (int m = 0; m < d; m++) {
        const z64 x = conjz(L[m * d + a]);
        const z64 y = L[m * d + c];
        gr = fma(x.x, y.x, fma(-x.y, y.y, gr));
        gi = fma(x.x, y.y, fma(x.y, y.x, gi));
      }
    }
    G[e] = make_double2(gr, gi);
  }
}

// L[(i,j),(k,l)] = -i (H[i,k] d_jl - d_ik H[l,j])
//                  + sum_q Lq[i,k] conj(Lq[j,l]) - 1/2 G[i,k] d_jl - 1/2 d_ik G[l,j]
__global__ void assemble_kernel(int d, const z64* __restrict__ H, int K, const z64* __restrict__ Ls,
                                const z64* __restrict__ G, z64* __restrict__ out) {
  const int n = d * d;
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / n), c = (int)(e - (e / n) * n);
    const int i = r / d, j = r - (r / d) * d;
    const int k = c / d, l = c - (c / d) * d;
    double hr = 0.0, hi = 0.0;  // H[i,k] d_jl - d_ik H[l,j]
    double gr = 0.0, gi = 0.0;  // G[i,k] d_jl + d_ik G[l,j]
    if (j == l) {
      hr += H[i * d + k].x;
      hi += H[i * d + k].y;
      if (K > 0) {
        gr += G[i * d + k].x;
        gi += G[i * d + k].y;
      }
    }
    if (i == k) {
      hr -= H[l * d + j].x;
      hi -= H[l * d + j].y;
      if (K > 0) {
        gr += G[l * d + j].x;
        gi += G[l * d + j].y;
      }
    }
    // -i (hr + i hi) = hi - i hr
    double vr = hi - 0.5 * gr, vi = -hr - 0.5 * gi;
    for (int q = 0; q < K; q++) {
      const z64* L = Ls + (long long)q * d * d;
      const z64 a = L[i * d + k];
      const z64 b = conjz(L[j * d + l]);
      vr = fma(a.x, b.x, fma(-a.y, b.y, vr));
      vi = fma(a.x, b.y, fma(a.y, b.x, vi));
    }
    out[e] = make_double2(vr, vi);
  }
}

// Column absolute sums of A_s = (Lbase + u_s Ldrv) dt, max-reduced per slice.
// grid: (ceil(n / blockDim), S).  Threads own columns, loop over rows
// (coalesced: a warp reads 32 consecutive columns of one row).
__global__ void colnorm_kernel(int n, int S, const z64* __restrict__ Lb, const z64* __restrict__ Ld,
                               const double* __restrict__ u, double dt,
                               unsigned long long* __restrict__ norm_bits) {
  // slices s = blockIdx.y, blockIdx.y + gridDim.y, ... (gridDim.y <= 65535)
  for (int s = blockIdx.y; s < S; s += gridDim.y) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double sum = 0.0;
  if (c < n) {
    const long long nn = (long long)n * n;
    const z64* Lbs = (Ld == nullptr) ? Lb + s * nn : Lb;
    const double us = (Ld == nullptr) ? 0.0 : u[s];
    for (int r = 0; r < n; r++) {
      z64 v = Lbs[(long long)r * n + c];
      if (Ld != nullptr) {
        const z64 w = Ld[(long long)r * n + c];
        v.x = fma(us, w.x, v.x);
        v.y = fma(us, w.y, v.y);
      }
      const double ar = v.x * dt, ai = v.y * dt;
      sum += sqrt(fma(ar, ar, ai * ai));
    }
  }
  // block max
  __shared__ double red[32];
  double m = sum;
  if (!(m == m)) m = __longlong_as_double(0x7ff0000000000000LL);  // NaN -> +Inf marker
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    double v = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) atomicMax(norm_bits + s, (unsigned long long)__double_as_longlong(v));
  }
  __syncthreads();  // red[] is reused by the next slice
  }
}

// sc = max(0, ceil(log2(norm / theta))), theta = 0.25.  Non-finite norms
// set the error word and use sc = 0.
__global__ void squaring_count_kernel(int S, const unsigned long long* __restrict__ norm_bits,
                                      int* __restrict__ sc, int* __restrict__ kmix,
                                      int* __restrict__ s_out, int* __restrict__ sc_max,
                                      unsigned int* err) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const double nrm = __longlong_as_double((long long)norm_bits[s]);
  int k = 0;
  if (!isfinite(nrm)) {
    atomicOr(err, ERR_NONFINITE);
  } else if (nrm > 0.25) {
    int e;
    const double m = frexp(nrm * 4.0, &e);  // nrm/theta = m * 2^e, m in [0.5, 1)
    k = (m == 0.5) ? e - 1 : e;
    if (k < 0) k = 0;
    if (k > 1000) k = 1000;
  }
  sc[s] = k;
  if (kmix != nullptr) {
    // squaring j acts on P = exp(A 2^j / 2^k); keep the D-form while
    // ||A||_1 2^(j-k) <= 1, i.e. while ||P - I|| stays of order ||A||
    int m = 0;
    if (isfinite(nrm))
      while (m < k && ldexp(nrm, m - k) <= 1.0) m++;
    kmix[s] = m;
  }
  if (s_out != nullptr) s_out[s] = k;
  atomicMax(sc_max, k);
}

// A_s = (Lbase + u_s Ldrv) * dt / 2^sc[s]
__global__ void scale_kernel(int n, int S, const z64* __restrict__ Lb, const z64* __restrict__ Ld,
                             const double* __restrict__ u, double dt, const int* __restrict__ sc,
                             z64* __restrict__ A) {
  const long long nn = (long long)n * n;
  const long long total = nn * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / nn);
    const long long o = e - s * nn;
    z64 v;
    if (Ld == nullptr) {
      v = Lb[e];
    } else {
      v = Lb[o];
      const z64 w = Ld[o];
      v.x = fma(u[s], w.x, v.x);
      v.y = fma(u[s], w.y, v.y);
    }
    // (v * dt) / 2^sc, with the power-of-two scaling exact
    A[e] = make_double2(ldexp(v.x * dt, -sc[s]), ldexp(v.y * dt, -sc[s]));
  }
}

__global__ void lincomb3_kernel(long long total, const z64* __restrict__ X0, const z64* __restrict__ X1,
                                const z64* __restrict__ X2, double c0, double c1, double c2,
                                z64* __restrict__ Z) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const z64 a = X0[e], b = X1[e], c = X2[e];
    Z[e] = make_double2(fma(c0, a.x, fma(c1, b.x, c2 * c.x)), fma(c0, a.y, fma(c1, b.y, c2 * c.y)));
  }
}

// Z[e] += 2 X[e] (FP64; one add per component, 2 X is exact)
__global__ void add_twice_kernel(long long total, const z64* __restrict__ X, z64* __restrict__ Z) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const z64 a = X[e], z = Z[e];
    Z[e] = make_double2(z.x + 2.0 * a.x, z.y + 2.0 * a.y);
  }
}

__global__ void copy_block_kernel(int S, long long ld, long long stride, int r0, int nr, int c0, int nc,
                                  const z64* __restrict__ src, z64* __restrict__ dst) {
  const long long per = (long long)nr * nc;
  const long long total = per * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / per;
    const long long o = e - s * per;
    const int r = (int)(o / nc), c = (int)(o - (o / nc) * nc);
    const long long idx = s * stride + (long long)(r0 + r) * ld + (c0 + c);
    dst[idx] = src[idx];
  }
}

__global__ void copy_active_kernel(long long nn, int S, const z64* __restrict__ src, z64* __restrict__ dst,
                                   const int* __restrict__ active, int iter) {
  const long long total = nn * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / nn);
    if (active[s] > iter) dst[e] = src[e];
  }
}

__global__ void check_finite_kernel(long long count, const z64* __restrict__ x, unsigned int* err) {
  bool bad = false;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    // exponent field all ones (Inf or NaN), tested on the bits: integer
    // operations only
    const z64 v = x[e];
    const unsigned hx = (unsigned)(__double_as_longlong(v.x) >> 32), hy = (unsigned)(__double_as_longlong(v.y) >> 32);
    if ((hx & 0x7FF00000u) == 0x7FF00000u || (hy & 0x7FF00000u) == 0x7FF00000u) bad = true;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_NONFINITE);
}

// Diagonal block of the blocked LU without pivot search, one CTA per slice.
// Factors the kb x kb block at (k0, k0) of M[s] in shared memory, writes its
// upper factor into Uf[s], and the inverses of the unit-lower and upper
// factors into Linv and Uinv (nb x nb, zero outside kb x kb).
__global__ void __launch_bounds__(256) lu_diag_kernel(int n, int k0, int kb, const z64* __restrict__ M,
                                                      z64* __restrict__ Uf, z64* __restrict__ Linv,
                                                      long long sLinv, z64* __restrict__ Uinv,
                                                      long long sUinv, unsigned int* err) {
  constexpr int NB = kLuNb;
  __shared__ z64 a[NB][NB + 1];
  __shared__ z64 x[NB][NB + 1];
  __shared__ z64 part[8][NB];
  __shared__ z64 rinv_s;
  const int s = blockIdx.x;
  const long long nn = (long long)n * n;
  const z64* Ms = M + s * nn;
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, j = e - (e / NB) * NB;
    a[i][j] = (i < kb && j < kb) ? Ms[(long long)(k0 + i) * n + (k0 + j)] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  // right-looking unblocked LU of the block
  for (int j = 0; j < kb; j++) {
    if (tid == 0) {
      const z64 p = a[j][j];
      const double amax = fmax(fabs(p.x), fabs(p.y));
      if (!(amax >= 1e-300) || !isfinite(amax)) {
        atomicOr(err, isfinite(amax) ? ERR_SINGULAR : ERR_NONFINITE);
        rinv_s = make_double2(1.0, 0.0);
      } else {
        // 1/p = conj(q) / (|q|^2 amax) with q = p / amax, safe from underflow
        const double qx = p.x / amax, qy = p.y / amax;
        const double inv = 1.0 / (fma(qx, qx, qy * qy) * amax);
        rinv_s = make_double2(qx * inv, -qy * inv);
      }
    }
    __syncthreads();
    const z64 rinv = rinv_s;
    for (int i = j + 1 + tid; i < kb; i += blockDim.x) a[i][j] = cmul(a[i][j], rinv);
    __syncthreads();
    const int w = kb - j - 1;
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int i = j + 1 + e / w, c = j + 1 + (e - (e / w) * w);
      a[i][c] = cfms(a[i][j], a[j][c], a[i][c]);
    }
    __syncthreads();
  }
  const int c = tid & 31, p = tid >> 5;  // column, partial-sum group (8 groups)
  // Linv: X = L^{-1}, L unit lower; X[i][c] = d_ic - sum_{j<i} L[i][j] X[j][c]
  for (int e = tid; e < NB * NB; e += blockDim.x) x[e / NB][e % NB] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int i = 0; i < kb; i++) {
    z64 acc = make_double2(0.0, 0.0);
    if (c < kb)
      for (int j = p; j < i; j += 8) acc = cfms(a[i][j], x[j][c], acc);  // acc -= L X
    part[p][c] = acc;
    __syncthreads();
    if (p == 0 && c < kb) {
      z64 v = make_double2(i == c ? 1.0 : 0.0, 0.0);
      for (int q = 0; q < 8; q++) {
        v.x += part[q][c].x;
        v.y += part[q][c].y;
      }
      x[i][c] = v;
    }
    __syncthreads();
  }
  z64* Li = Linv + (long long)s * sLinv;
  for (int e = tid; e < NB * NB; e += blockDim.x) Li[e] = x[e / NB][e % NB];
  __syncthreads();
  // Uinv: X = U^{-1}; X[i][c] = (d_ic - sum_{j>i} U[i][j] X[j][c]) / U[i][i]
  for (int e = tid; e < NB * NB; e += blockDim.x) x[e / NB][e % NB] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int i = kb - 1; i >= 0; i--) {
    z64 acc = make_double2(0.0, 0.0);
    if (c < kb)
      for (int j = i + 1 + p; j < kb; j += 8) acc = cfms(a[i][j], x[j][c], acc);
    part[p][c] = acc;
    __syncthreads();
    if (p == 0 && c < kb) {
      z64 v = make_double2(i == c ? 1.0 : 0.0, 0.0);
      for (int q = 0; q < 8; q++) {
        v.x += part[q][c].x;
        v.y += part[q][c].y;
      }
      const z64 d = a[i][i];
      const double amax = fmax(fabs(d.x), fabs(d.y));
      z64 rd = make_double2(1.0, 0.0);
      if (amax >= 1e-300 && isfinite(amax)) {
        const double qx = d.x / amax, qy = d.y / amax;
        const double inv = 1.0 / (fma(qx, qx, qy * qy) * amax);
        rd = make_double2(qx * inv, -qy * inv);
      }
      x[i][c] = cmul(v, rd);
    }
    __syncthreads();
  }
  z64* Ui = Uinv + (long long)s * sUinv;
  for (int e = tid; e < NB * NB; e += blockDim.x) Ui[e] = x[e / NB][e % NB];
  z64* Ufs = Uf + s * nn;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e - (e / kb) * kb;
    Ufs[(long long)(k0 + i) * n + (k0 + j)] = (j >= i) ? a[i][j] : make_double2(0.0, 0.0);
  }
}

__global__ void check_bound_kernel(const int* __restrict__ sc_max, int bound, unsigned int* err) {
  if (threadIdx.x == 0 && *sc_max > bound) atomicOr(err, ERR_SQUARING_BOUND);
}

inline unsigned grid_for(long long total, int threads, int sm_count) {
  long long g = (total + threads - 1) / threads;
  long long cap = (long long)sm_count * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

cudaError_t launch_assemble(int d, const z64* H, int K, const z64* Ls, z64* L_out, z64* G_scratch,
                            int sm_count, cudaStream_t st) {
  if (K > 0) {
    count_launch();
    gram_kernel<<<1, 256, 0, st>>>(d, K, Ls, G_scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const long long nn = (long long)d * d * d * d;
  count_launch();
  assemble_kernel<<<grid_for(nn, 256, sm_count), 256, 0, st>>>(d, H, K, Ls, G_scratch, L_out);
  return cudaGetLastError();
}

cudaError_t launch_slice_prepare(int n, int S, const z64* Lbase, const z64* Ldrv, const double* u,
                                 double dt, z64* A, unsigned long long* norm_bits, int* sc,
                                 int* kmix, int* s_out, unsigned int* err, int sm_count,
                                 cudaStream_t st) {
  // norm_bits[0..S) and sc_max (stored right after sc[S]) must start at zero
  cudaError_t e = cudaMemsetAsync(norm_bits, 0, sizeof(unsigned long long) * S, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(sc + S, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  dim3 g1((n + 127) / 128, S < 65535 ? S : 65535);
  count_launch();
  colnorm_kernel<<<g1, 128, 0, st>>>(n, S, Lbase, Ldrv, u, dt, norm_bits);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  squaring_count_kernel<<<(S + 127) / 128, 128, 0, st>>>(S, norm_bits, sc, kmix, s_out, sc + S, err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long total = (long long)n * n * S;
  count_launch();
  scale_kernel<<<grid_for(total, 256, sm_count), 256, 0, st>>>(n, S, Lbase, Ldrv, u, dt, sc, A);
  return cudaGetLastError();
}

cudaError_t launch_squaring_count(int S, const unsigned long long* norm_bits, int* sc, int* kmix, int* s_out,
                                  unsigned int* err, cudaStream_t st) {
  count_launch();
  squaring_count_kernel<<<(S + 127) / 128, 128, 0, st>>>(S, norm_bits, sc, kmix, s_out, sc + S, err);
  return cudaGetLastError();
}

cudaError_t launch_lincomb3(int nn, int S, const z64* X0, const z64* X1, const z64* X2, double c0,
                            double c1, double c2, z64* Z, cudaStream_t st) {
  const long long total = (long long)nn * S;
  count_launch();
  lincomb3_kernel<<<grid_for(total, 256, 152), 256, 0, st>>>(total, X0, X1, X2, c0, c1, c2, Z);
  return cudaGetLastError();
}

cudaError_t launch_add_twice(long long nn, int S, const z64* X, z64* Z, cudaStream_t st) {
  const long long total = nn * S;
  long long g = (total + 255) / 256;
  if (g > 152LL * 16) g = 152LL * 16;
  count_launch();
  add_twice_kernel<<<(unsigned)g, 256, 0, st>>>(total, X, Z);
  return cudaGetLastError();
}

cudaError_t launch_lu_diag(int n, int S, int k0, int kb, const z64* M, z64* Uf, z64* Linv,
                           long long sLinv, z64* Uinv, long long sUinv, unsigned int* err,
                           cudaStream_t st) {
  count_launch();
  lu_diag_kernel<<<S, 256, 0, st>>>(n, k0, kb, M, Uf, Linv, sLinv, Uinv, sUinv, err);
  return cudaGetLastError();
}

cudaError_t launch_copy_block(int S, long long ld, long long stride, int r0, int nr, int c0, int nc,
                              const z64* src, z64* dst, cudaStream_t st) {
  const long long total = (long long)nr * nc * S;
  if (total == 0) return cudaSuccess;
  count_launch();
  copy_block_kernel<<<grid_for(total, 256, 152), 256, 0, st>>>(S, ld, stride, r0, nr, c0, nc, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_copy_active(long long nn, int S, const z64* src, z64* dst, const int* active,
                               int iter, cudaStream_t st) {
  const long long total = nn * S;
  count_launch();
  copy_active_kernel<<<grid_for(total, 256, 152), 256, 0, st>>>(nn, S, src, dst, active, iter);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(long long count, const z64* x, unsigned int* err, cudaStream_t st) {
  count_launch();
  check_finite_kernel<<<grid_for(count, 256, 152), 256, 0, st>>>(count, x, err);
  return cudaGetLastError();
}

cudaError_t launch_check_bound(const int* sc_max, int bound, unsigned int* err, cudaStream_t st) {
  count_launch();
  check_bound_kernel<<<1, 32, 0, st>>>(sc_max, bound, err);
  return cudaGetLastError();
}

}  // namespace lb
