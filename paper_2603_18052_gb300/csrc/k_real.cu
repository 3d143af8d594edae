// Element-wise and small-block kernels of the real-coordinate ("Hermitian")
// propagator build (Algorithm 1 on the real coordinates of Hermitian
// matrices; the coordinates and the map of a Hermiticity-preserving
// superoperator onto them are described in k_herm.cu):
//   * the slice generators G_s = (G_base + u_s G_drv) dt on the real
//     coordinates, their 1-norms (maximum absolute column sum), the scaling
//     by 2^-s (Eq. 5 and the scaling line of Algorithm 1),
//   * the linear combinations of the Pade step and the FP64 -> FP32 copies
//     of the reduced-precision form,
//   * the real diagonal-block factorisation of the blocked LU,
//   * the complex propagator P rebuilt from its real-coordinate matrix R.
#include "lb_internal.cuh"

namespace lb {

namespace {

inline unsigned grid_of(long long total, int threads, int sm_count) {
  long long g = (total + threads - 1) / threads;
  const long long cap = (long long)sm_count * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// v = (Gb[o] + u Gd[o]) dt, rounded as the complex path rounds it (product
// and sum in one FMA, then the scaling by dt).
__device__ __forceinline__ double slice_gen(const double* __restrict__ Gb, const double* __restrict__ Gd,
                                            const double* __restrict__ u, int s, long long nn, long long o,
                                            double dt) {
  const double v = Gd == nullptr ? Gb[s * nn + o] : fma(u[s], Gd[o], Gb[o]);
  return v * dt;
}

// Per-slice maximum absolute column sum of G_s (8 columns x 32 row groups
// per CTA, fixed-order sums), max-reduced into norm_bits[s] as the bits of a
// non-negative double (NaN -> +Inf).
__global__ void __launch_bounds__(256) real_gen_norm_kernel(int n, int S, const double* __restrict__ Gb,
                                                           const double* __restrict__ Gd,
                                                           const double* __restrict__ u, double dt,
                                                           unsigned long long* __restrict__ norm_bits) {
  __shared__ double part[32][8];
  const long long nn = (long long)n * n;
  const int c = threadIdx.x % 8, rg = threadIdx.x / 8;
  const int cblocks = (n + 7) / 8;
  for (long long t = blockIdx.x; t < (long long)S * cblocks; t += gridDim.x) {
    const int s = (int)(t / cblocks), j = (int)(t - (t / cblocks) * cblocks) * 8 + c;
    double sum = 0.0;
    if (j < n)
      for (int i = rg; i < n; i += 32) sum += fabs(slice_gen(Gb, Gd, u, s, nn, (long long)i * n + j, dt));
    part[rg][c] = sum;
    __syncthreads();
    if (rg == 0 && j < n) {
      double col = 0.0;
      for (int r = 0; r < 32; r++) col += part[r][c];
      if (!(col == col)) col = INFINITY;
      atomicMax(norm_bits + s, (unsigned long long)__double_as_longlong(col));
    }
    __syncthreads();
  }
}

// A_s = G_s / 2^sc[s] (exact power-of-two scaling); a CTA per row of a
// slice, its threads along the row
__global__ void real_scale_kernel(int n, int S, const double* __restrict__ Gb, const double* __restrict__ Gd,
                                  const double* __restrict__ u, double dt, const int* __restrict__ sc,
                                  double* __restrict__ A) {
  const long long nn = (long long)n * n, rows = (long long)S * n;
  for (long long rw = blockIdx.x; rw < rows; rw += gridDim.x) {
    const int s = (int)(rw / n);
    const long long o0 = (rw - (long long)s * n) * n;
    // (v dt) 2^-sc is exact scaling of the rounded v dt, so one product by
    // dt 2^-sc (exact) rounds the same: two FP64 operations per entry
    const double f = ldexp(dt, -sc[s]);
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const long long o = o0 + c;
      const double v = Gd == nullptr ? Gb[(long long)s * nn + o] : fma(u[s], Gd[o], Gb[o]);
      A[rw * n + c] = v * f;
    }
  }
}

template <typename T>
__global__ void real_lincomb3_kernel(long long total, const T* __restrict__ X0, const T* __restrict__ X1,
                                     const T* __restrict__ X2, T c0, T c1, T c2, T* __restrict__ Z) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    Z[e] = c0 * X0[e] + (c1 * X1[e] + c2 * X2[e]);
}

// A_s^2 of a control-affine slice generator A_s = c_s (G_b + u_s G_d),
// c_s = dt 2^-sc[s], from three slice-independent products:
//   A_s^2 = c_s^2 (P0 + u_s (P1 + u_s P2)),  P0 = G_b^2, P1 = G_b G_d + G_d G_b, P2 = G_d^2;
// a CTA per row of a slice, three FP64 operations per entry.
__global__ void real_affine_square_kernel(int n, int S, const double* __restrict__ P0, const double* __restrict__ P1,
                                          const double* __restrict__ P2, const double* __restrict__ u, double dt,
                                          const int* __restrict__ sc, double* __restrict__ A2) {
  const long long rows = (long long)S * n;
  for (long long rw = blockIdx.x; rw < rows; rw += gridDim.x) {
    const int s = (int)(rw / n);
    const long long o0 = (rw - (long long)s * n) * n;
    const double cs = ldexp(dt, -sc[s]), f = cs * cs, us = u[s];
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const long long o = o0 + c;
      A2[rw * n + c] = fma(us, fma(us, P2[o], P1[o]), P0[o]) * f;
    }
  }
}

// The power terms of the [13/13] approximant's two polynomials in one pass
// over A^6, A^4, A^2 (n x n per slice, FP64), with the A^6 terms of V and W
// moved into the matrices A^6 multiplies (A^6 Z1 = A^6 (Z1 - b6 I) + b6 A^6):
//   Z1 = b12 A^6 + b10 A^4 + b8 A^2 + b6 I,   Z2 = b13 A^6 + b11 A^4 + b9 A^2 + b7 I,
//   V = b4 A^4 + b2 A^2 + b0 I,   W = b5 A^4 + b3 A^2 + b1 I,
// so that V + A^6 Z1 and W + A^6 Z2 are the approximant's polynomials; a
// CTA per row of a slice, its threads along the row.  Ten FP64 operations
// per entry: the FP64 pipe, not the memory, bounds this pass.
__global__ void real_pade_terms_kernel(int n, int S, const double* __restrict__ A6, const double* __restrict__ A4,
                                       const double* __restrict__ A2, PadeCoef cf, double* __restrict__ Z1,
                                       double* __restrict__ Z2, double* __restrict__ V, double* __restrict__ W) {
  const long long rows = (long long)S * n;
  for (long long rw = blockIdx.x; rw < rows; rw += gridDim.x) {
    const int r = (int)(rw % n);
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const long long e = rw * n + c;
      const double p6 = A6[e], p4 = A4[e], p2 = A2[e];
      const double z1 = cf.b[12] * p6 + (cf.b[10] * p4 + cf.b[8] * p2);
      const double z2 = cf.b[13] * p6 + (cf.b[11] * p4 + cf.b[9] * p2);
      const double v = cf.b[4] * p4 + cf.b[2] * p2;
      const double w = cf.b[5] * p4 + cf.b[3] * p2;
      const bool dg = c == r;
      Z1[e] = dg ? z1 + cf.b[6] : z1;
      Z2[e] = dg ? z2 + cf.b[7] : z2;
      V[e] = dg ? v + cf.b[0] : v;
      W[e] = dg ? w + cf.b[1] : w;
    }
  }
}

// dst[s][r][c] = src[s][r][c] for an R x C block of S matrices (leading
// dimensions and batch strides of their own)
__global__ void real_copy_block_kernel(int R, int C, long long total, const double* __restrict__ src, long long sld,
                                       long long ss, double* __restrict__ dst, long long dld, long long ds) {
  const long long rc = (long long)R * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / rc, o = e - s * rc;
    const int r = (int)(o / C), c = (int)(o - (o / C) * C);
    dst[s * ds + r * dld + c] = src[s * ss + r * sld + c];
  }
}

// dst (FP32) = src - shift I  (n x n per slice)
__global__ void real_to_f32_kernel(int n, long long total, const double* __restrict__ src, double shift,
                                   float* __restrict__ dst) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long o = e % nn;
    double v = src[e];
    if (o / n == o % n) v -= shift;
    dst[e] = (float)v;
  }
}

// V, W of the [13/13] approximant as sums of the even powers, for the
// slices with flag[s] != 0:
//   V = b12 A^12 + b10 A^10 + b8 A^8 + b6 A^6 + b4 A^4 + b2 A^2 (+ b0 I)
//   W = b13 A^12 + b11 A^10 + b9 A^8 + b7 A^6 + b5 A^4 + b3 A^2 (+ b1 I)
// (U = A W), the highest powers added first.
template <typename T>
__global__ void real_powsum_kernel(int n, int S, const int* __restrict__ flag, const T* __restrict__ A2,
                                   const T* __restrict__ A4, const T* __restrict__ A6, const T* __restrict__ A8,
                                   const T* __restrict__ A10, const T* __restrict__ A12, PadeCoef c,
                                   int with_identity, T* __restrict__ V, T* __restrict__ W) {
  const long long nn = (long long)n * n, total = nn * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long s = e / nn, o = e - s * nn;
    if (flag[s] == 0) continue;
    const T p12 = A12[e], p10 = A10[e], p8 = A8[e], p6 = A6[e], p4 = A4[e], p2 = A2[e];
    T v = T(c.b[12]) * p12, w = T(c.b[13]) * p12;
    v = v + T(c.b[10]) * p10;
    w = w + T(c.b[11]) * p10;
    v = v + T(c.b[8]) * p8;
    w = w + T(c.b[9]) * p8;
    v = v + T(c.b[6]) * p6;
    w = w + T(c.b[7]) * p6;
    v = v + T(c.b[4]) * p4;
    w = w + T(c.b[5]) * p4;
    v = v + T(c.b[2]) * p2;
    w = w + T(c.b[3]) * p2;
    if (with_identity && o / n == o % n) {
      v += T(c.b[0]);
      w += T(c.b[1]);
    }
    V[e] = v;
    W[e] = w;
  }
}

__global__ void real_copy_active_kernel(long long nn, int S, const double* __restrict__ src, double* __restrict__ dst,
                                        const int* __restrict__ active, int iter) {
  const long long total = nn * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    if (active[e / nn] > iter) dst[e] = src[e];
}

// P[s] from R[s]: the complex superoperator that acts on Hermitian matrices
// as R acts on their real coordinates.  Column (k, l) of P is P(E_kl); with
// Y(r) the Hermitian matrix of coordinate vector r and R_a column a of R,
//   k = l:  P(E_kk) = Y(R_k)
//   k < l:  E_kl = H1 + i H2 with H1 = (E_kl + E_lk)/2 (Re coordinate 1/2)
//           and H2 = -i (E_kl - E_lk)/2 (Im coordinate -1/2), so
//           P(E_kl) = Y(R_re)/2 - i Y(R_im)/2
//   k > l:  E_kl = H1 - i H2 for the pair (l, k): P(E_kl) = Y(R_re)/2 + i Y(R_im)/2
// and entry (i, j) of Y(r) is r_i (i = j), r_re + i r_im (i < j) or
// r_re - i r_im (i > j) for the coordinates of (min, max).
// x / 2: the exponent field lowered by one (no FP64 operation) where x and
// its half are normal; a product otherwise
__device__ __forceinline__ double half_of(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex > 1 && ex < 0x7FF) return __longlong_as_double(b - (1ll << 52));
  return 0.5 * x;
}
__device__ __forceinline__ double neg_of(double x) { return __longlong_as_double(__double_as_longlong(x) ^ (1ll << 63)); }

// a CTA per row (i, j) of P[s], its threads along the row.  With Re / Im
// rows ra, ra + 1 of R for (i, j) (sign sg = +1 for i < j, -1 for i > j) and
// the coordinate pair a, a + 1 of (k, l):
//   k = l:  P = (R[ra][k], sg R[ra+1][k])
//   k < l:  P = ((R[ra][a] + sg R[ra+1][a+1]) / 2, (sg R[ra+1][a] - R[ra][a+1]) / 2)
//   k > l:  P = ((R[ra][a] - sg R[ra+1][a+1]) / 2, (sg R[ra+1][a] + R[ra][a+1]) / 2)
// (for i = j the R[ra+1] terms are absent): at most one FP64 addition per
// real number, the halving and the signs on the bits.
__global__ void herm_to_complex_kernel(int n, int d, int S, const double* __restrict__ R, z64* __restrict__ P) {
  const long long nn = (long long)n * n, rows = (long long)S * n;
  for (long long rw = blockIdx.x; rw < rows; rw += gridDim.x) {
    const long long s = rw / n;
    const int r = (int)(rw - s * n);
    const int i = r / d, j = r - (r / d) * d;
    const bool diag = i == j, up = i < j;
    const int ra = diag ? i : herm_pair_coord(up ? i : j, up ? j : i, d);
    const double* re = R + s * nn + (long long)ra * n;
    const double* im = re + n;  // used only off the diagonal
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int k = c / d, l = c - (c / d) * d;
      z64 v;
      if (k == l) {
        v.x = re[k];
        v.y = diag ? 0.0 : (up ? im[k] : neg_of(im[k]));
      } else {
        const int a = herm_pair_coord(k < l ? k : l, k < l ? l : k, d);
        const double x0 = re[a], x1 = re[a + 1];
        if (diag) {
          v.x = half_of(x0);
          v.y = half_of(k < l ? neg_of(x1) : x1);
        } else {
          double y0 = im[a], y1 = im[a + 1];
          if (!up) {
            y0 = neg_of(y0);
            y1 = neg_of(y1);
          }
          v = k < l ? make_double2(half_of(x0 + y1), half_of(y0 - x1)) : make_double2(half_of(x0 - y1), half_of(y0 + x1));
        }
      }
      P[rw * n + c] = v;
    }
  }
}

// Real diagonal block of the blocked LU without pivot search, one CTA per
// slice: factors the kb x kb block at (k0, k0) of M[s] in shared memory,
// writes its upper factor into Uf[s] and the inverses of the unit-lower and
// upper factors into Linv and Uinv (NB x NB, zero outside kb x kb).  A pivot
// of modulus below 1e-300 (or non-finite) sets the error word.  NB = 32 or
// 64; the triangular inverses sum each entry in 256 / NB partial sums.
template <int NB>
__global__ void __launch_bounds__(256) lu_diag_real_kernel(int n, int k0, int kb, const double* __restrict__ M,
                                                           double* __restrict__ Uf, double* __restrict__ Linv,
                                                           long long sLinv, double* __restrict__ Uinv,
                                                           long long sUinv, unsigned int* err) {
  constexpr int NP = 256 / NB;
  extern __shared__ double lu_smem[];
  double(*a)[NB + 1] = (double(*)[NB + 1])lu_smem;
  double(*xl)[NB + 1] = (double(*)[NB + 1])(lu_smem + NB * (NB + 1));
  double(*xu)[NB + 1] = (double(*)[NB + 1])(lu_smem + 2 * NB * (NB + 1));
  double(*pl)[NB] = (double(*)[NB])(lu_smem + 3 * NB * (NB + 1));
  double(*pu)[NB] = (double(*)[NB])(lu_smem + 3 * NB * (NB + 1) + NP * NB);
  double* rdiag = lu_smem + 3 * NB * (NB + 1) + 2 * NP * NB;  // 1 / U[j][j] (1 where the pivot is unusable)
  const int s = blockIdx.x;
  const long long nn = (long long)n * n;
  const double* Ms = M + s * nn;
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, j = e - (e / NB) * NB;
    a[i][j] = (i < kb && j < kb) ? Ms[(long long)(k0 + i) * n + (k0 + j)] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < kb; j++) {
    if (tid == 0) {
      const double p = a[j][j];
      if (!(fabs(p) >= 1e-300) || !isfinite(p)) {
        atomicOr(err, isfinite(p) ? ERR_SINGULAR : ERR_NONFINITE);
        rdiag[j] = 1.0;
      } else {
        rdiag[j] = 1.0 / p;
      }
    }
    __syncthreads();
    const double rinv = rdiag[j];
    for (int i = j + 1 + tid; i < kb; i += blockDim.x) a[i][j] *= rinv;
    __syncthreads();
    const int w = kb - j - 1;
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int i = j + 1 + e / w, c = j + 1 + (e - (e / w) * w);
      a[i][c] = fma(-a[i][j], a[j][c], a[i][c]);
    }
    __syncthreads();
  }
  // the two triangular inverses row by row, one row of each per round:
  //   L^{-1} (L unit lower), forward:  X[i][c] = d_ic - sum_{j<i} L[i][j] X[j][c]
  //   U^{-1}, backward:  X[i][c] = (d_ic - sum_{j>i} U[i][j] X[j][c]) / U[i][i]
  // (the division as a product with the pivot's reciprocal from the
  // factorisation); each entry's sum in NP partial sums of a fixed order
  const int c = tid % NB, p = tid / NB;  // column, partial-sum group
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    xl[e / NB][e % NB] = 0.0;
    xu[e / NB][e % NB] = 0.0;
  }
  __syncthreads();
  for (int t = 0; t < kb; t++) {
    const int il = t, iu = kb - 1 - t;
    double accl = 0.0, accu = 0.0;
    if (c < kb) {
      for (int j = p; j < il; j += NP) accl = fma(-a[il][j], xl[j][c], accl);
      for (int j = iu + 1 + p; j < kb; j += NP) accu = fma(-a[iu][j], xu[j][c], accu);
    }
    pl[p][c] = accl;
    pu[p][c] = accu;
    __syncthreads();
    if (p == 0 && c < kb) {
      double v = il == c ? 1.0 : 0.0, u = iu == c ? 1.0 : 0.0;
      for (int q = 0; q < NP; q++) {
        v += pl[q][c];
        u += pu[q][c];
      }
      xl[il][c] = v;
      xu[iu][c] = u * rdiag[iu];
    }
    __syncthreads();
  }
  double* Li = Linv + (long long)s * sLinv;
  double* Ui = Uinv + (long long)s * sUinv;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    Li[e] = xl[e / NB][e % NB];
    Ui[e] = xu[e / NB][e % NB];
  }
  double* Ufs = Uf + s * nn;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e / kb, j = e - (e / kb) * kb;
    Ufs[(long long)(k0 + i) * n + (k0 + j)] = (j >= i) ? a[i][j] : 0.0;
  }
}

template <int NB>
constexpr size_t lu_diag_smem() {
  return (size_t)(3 * NB * (NB + 1) + 2 * (256 / NB) * NB + NB) * sizeof(double);
}

}  // namespace

cudaError_t launch_real_slice_prepare(int n, int S, const double* Gb, const double* Gd, const double* u, double dt,
                                      double* A, unsigned long long* norm_bits, int* sc, int* kmix, int* s_out,
                                      unsigned int* err, int sm_count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(norm_bits, 0, sizeof(unsigned long long) * S, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(sc + S, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)S * ((n + 7) / 8);
  count_launch();
  real_gen_norm_kernel<<<grid_of(tiles, 1, sm_count), 256, 0, st>>>(n, S, Gb, Gd, u, dt, norm_bits);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_squaring_count(S, norm_bits, sc, kmix, s_out, err, st);
  if (e != cudaSuccess) return e;
  count_launch();
  real_scale_kernel<<<grid_of((long long)S * n, 1, sm_count), 256, 0, st>>>(n, S, Gb, Gd, u, dt, sc, A);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_real_lincomb3(long long total, const T* X0, const T* X1, const T* X2, double c0, double c1,
                                 double c2, T* Z, int sm_count, cudaStream_t st) {
  count_launch();
  real_lincomb3_kernel<T><<<grid_of(total, 256, sm_count), 256, 0, st>>>(total, X0, X1, X2, T(c0), T(c1), T(c2), Z);
  return cudaGetLastError();
}
template cudaError_t launch_real_lincomb3<double>(long long, const double*, const double*, const double*, double,
                                                  double, double, double*, int, cudaStream_t);

cudaError_t launch_real_copy_block(int R, int C, int S, const double* src, long long sld, long long ss, double* dst,
                                   long long dld, long long ds, int sm_count, cudaStream_t st) {
  const long long total = (long long)R * C * S;
  if (total <= 0) return cudaSuccess;
  count_launch();
  real_copy_block_kernel<<<grid_of(total, 256, sm_count), 256, 0, st>>>(R, C, total, src, sld, ss, dst, dld, ds);
  return cudaGetLastError();
}

cudaError_t launch_real_affine_square(int n, int S, const double* P0, const double* P1, const double* P2,
                                      const double* u, double dt, const int* sc, double* A2, int sm_count,
                                      cudaStream_t st) {
  count_launch();
  real_affine_square_kernel<<<grid_of((long long)S * n, 1, sm_count), 256, 0, st>>>(n, S, P0, P1, P2, u, dt, sc, A2);
  return cudaGetLastError();
}

cudaError_t launch_real_pade_terms(int n, int S, const double* A6, const double* A4, const double* A2,
                                   const double* b, double* Z1, double* Z2, double* V, double* W, int sm_count,
                                   cudaStream_t st) {
  PadeCoef cf;
  for (int j = 0; j < 14; j++) cf.b[j] = b[j];
  count_launch();
  real_pade_terms_kernel<<<grid_of((long long)S * n, 1, sm_count), 256, 0, st>>>(n, S, A6, A4, A2, cf, Z1, Z2, V,
                                                                                  W);
  return cudaGetLastError();
}
template cudaError_t launch_real_lincomb3<float>(long long, const float*, const float*, const float*, double, double,
                                                 double, float*, int, cudaStream_t);

template <typename T>
cudaError_t launch_real_powsum(int n, int S, const int* flag, const T* A2, const T* A4, const T* A6, const T* A8,
                               const T* A10, const T* A12, const double* b, int with_identity, T* V, T* W,
                               int sm_count, cudaStream_t st) {
  PadeCoef c;
  for (int j = 0; j < 14; j++) c.b[j] = b[j];
  const long long total = (long long)n * n * S;
  count_launch();
  real_powsum_kernel<T><<<grid_of(total, 256, sm_count), 256, 0, st>>>(n, S, flag, A2, A4, A6, A8, A10, A12, c,
                                                                       with_identity, V, W);
  return cudaGetLastError();
}
template cudaError_t launch_real_powsum<double>(int, int, const int*, const double*, const double*, const double*,
                                                const double*, const double*, const double*, const double*, int,
                                                double*, double*, int, cudaStream_t);
template cudaError_t launch_real_powsum<float>(int, int, const int*, const float*, const float*, const float*,
                                               const float*, const float*, const float*, const double*, int, float*,
                                               float*, int, cudaStream_t);

cudaError_t launch_real_to_f32(int n, int S, const double* src, double shift, float* dst, int sm_count,
                               cudaStream_t st) {
  const long long total = (long long)n * n * S;
  count_launch();
  real_to_f32_kernel<<<grid_of(total, 256, sm_count), 256, 0, st>>>(n, total, src, shift, dst);
  return cudaGetLastError();
}

cudaError_t launch_real_copy_active(long long nn, int S, const double* src, double* dst, const int* active, int iter,
                                    int sm_count, cudaStream_t st) {
  count_launch();
  real_copy_active_kernel<<<grid_of(nn * S, 256, sm_count), 256, 0, st>>>(nn, S, src, dst, active, iter);
  return cudaGetLastError();
}

cudaError_t launch_herm_to_complex(int n, int d, int S, const double* R, z64* P, int sm_count, cudaStream_t st) {
  count_launch();
  herm_to_complex_kernel<<<grid_of((long long)S * n, 1, sm_count), 256, 0, st>>>(n, d, S, R, P);
  return cudaGetLastError();
}

cudaError_t launch_lu_diag_real(int n, int S, int k0, int kb, const double* M, double* Uf, double* Linv,
                                long long sLinv, double* Uinv, long long sUinv, unsigned int* err, cudaStream_t st,
                                int nb) {
  if (nb == 64) {
    constexpr size_t sm = lu_diag_smem<64>();
    cudaError_t e = set_smem_once((const void*)lu_diag_real_kernel<64>, sm);
    if (e != cudaSuccess) return e;
    count_launch();
    lu_diag_real_kernel<64><<<S, 256, sm, st>>>(n, k0, kb, M, Uf, Linv, sLinv, Uinv, sUinv, err);
    return cudaGetLastError();
  }
  if (nb != kLuNb) return cudaErrorInvalidValue;
  count_launch();
  lu_diag_real_kernel<kLuNb><<<S, 256, lu_diag_smem<kLuNb>(), st>>>(n, k0, kb, M, Uf, Linv, sLinv, Uinv, sUinv, err);
  return cudaGetLastError();
}

}  // namespace lb
