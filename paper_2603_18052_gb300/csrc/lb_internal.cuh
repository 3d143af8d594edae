// Internal declarations shared by the translation units of liblb.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <array>
#include <cstdint>
#include <cstddef>

#include "lb.h"

namespace lb {

// Device error word bits (the context's error word is a uint32).
enum : unsigned int {
  ERR_NONFINITE = 1u,
  ERR_SINGULAR = 2u,
  ERR_TIMEOUT = 4u,
  ERR_SQUARING_BOUND = 8u,  // a slice needed more squarings than the fixed bound
};

constexpr int kMaxN = 729;
constexpr int kLuNb = 32;  // LU block size
constexpr int kLuNbSliced = 128;  // LU block size of the sliced-product schedule (two 64-wide halves)

typedef double2 z64;

// Workspace carve-out.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  void* take(size_t bytes) {
    size_t a = (off + 255) & ~size_t(255);
    if (a + bytes > cap) return nullptr;
    off = a + bytes;
    return base + a;
  }
};

// Process-wide count of kernel launches issued by the library.
void count_launch();

// Return LB_ECUDA from the enclosing lb_status function on a CUDA error.
#define LB_CUDA(call)                       \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) return LB_ECUDA; \
  } while (0)

// For the entry points that take no lb_ctx: the current CUDA device, which
// must be an sm_103 part, and its SM count.  LB_ENODEV otherwise.
lb_status current_device_sm103(int* dev, int* sms);

// Makes `dev` current for the guard's lifetime, then restores the previous
// device.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace lb

struct lb_ctx {
  int device = 0;
  int max_n = 0, max_batch = 0, max_slices = 0;
  int sm_count = 0;
  char* ws = nullptr;  // device scratch (one allocation)
  size_t ws_bytes = 0;
  unsigned int* err_dev = nullptr;  // device error word
  unsigned int* err_host = nullptr; // pinned copy
  int* scmax_host = nullptr;        // pinned: largest squaring count of the last build
  cudaEvent_t ev_scmax = nullptr;
  int max_squarings = -1;  // >= 0: fixed squaring rounds, no host read (graph capture)
  double pade_b[14];
  // --- stage timers of lb_expm_pade (CUDA events in a ring, optional) ---
  int timing = 0;
  static constexpr int kRing = 16;
  cudaEvent_t ev_stage[kRing][6] = {};
  int ring_used[kRing] = {};  // slot holds events not yet accumulated
  int ring_next = 0;
  double stage_ms[5] = {0, 0, 0, 0, 0};
  long long stage_chunks = 0;
  // --- with the stage timers: events around every sliced-product launch
  // without a batch mask (a ring; kern_flops: digit-product FLOPs) ---
  static constexpr int kKRing = 4096;
  cudaEvent_t ev_kern[kKRing][2] = {};
  double kern_flops[kKRing] = {};
  int kern_used[kKRing] = {};
  int kern_next = 0;
  double kern_ms = 0.0, kern_fl = 0.0;
  long long kern_launches = 0;
  // --- propagator build, per slice (stride max_n^2 complex) ---
  lb::z64 *A = nullptr, *A2 = nullptr, *A4 = nullptr, *A6 = nullptr, *Z1 = nullptr, *Z2 = nullptr;
  lb::z64 *V = nullptr, *W = nullptr, *Mx = nullptr;
  lb::z64 *Linv = nullptr;  // per slice nb x nb
  lb::z64 *Uinv = nullptr;  // per slice nblk x nb x nb
  unsigned long long* norm_bits = nullptr;
  int* sc = nullptr;  // max_slices + 1 (last = max)
  int* kmix = nullptr;  // max_slices
  lb::z64* G = nullptr;  // d x d Gram matrix for assembly
  // --- split-BF16 planes for the tensor-core products (per slice 4 x n x ld) ---
  __nv_bfloat16* sp[9] = {};  // split-BF16 planes; all nine share one region, also the sliced-FP64 scratch
  void* oz_scratch = nullptr;
  size_t oz_bytes = 0;
  __nv_bfloat16* spR[2] = {};  // state planes, 4 x max_batch x ld each
  // --- propagation ---
  lb::z64* Rtmp = nullptr;  // max_batch x max_n
  lb::z64* Xh = nullptr;    // max_batch x max_n: device copy of host states (lb_propagate_resident)
  float *Dr = nullptr, *Di = nullptr;  // per slice max_n^2 (n <= 81), inside Dpl
  float* Dpl = nullptr;                // FP32 D^T planes of the chain, per slice chain32_dplane_floats
  float *C32a = nullptr, *C32b = nullptr;  // FP32 state planes, chain32_state_floats(max_n, max_batch)
  float* part32 = nullptr;             // split-K partial tiles, chain32_part_floats(sm_count)
  unsigned* cnt32 = nullptr;           // split-K tickets, sm_count (zero between launches), then a barrier counter
  // --- many-instance batching (lb_run_instances) ---
  lb::z64* Ginst = nullptr;  // per-slice generators, max_slices x max_n^2
  lb::z64* Pinst = nullptr;  // their propagators
  void* inst_tab_dev = nullptr;   // slice and work-item tables
  void* inst_tab_host = nullptr;  // pinned staging of the tables
  size_t inst_tab_bytes = 0;
  cudaEvent_t ev_tab = nullptr;   // the last table upload
  int* spflag = nullptr;  // 2 x max_slices: sparse-operand flags of the real-coordinate build
  int* csr = nullptr;     // a sparse pattern: count (2 ints), row starts, row ends (max_n each), columns (max_n^2)
  // --- GRAPE (contexts with max_n <= 81) ---
  lb::z64* grape = nullptr;
  size_t grape_bytes = 0;
};

namespace lb {

// ---------------------------------------------------------------- GEMM ----
// Grouped, batched complex FP64 GEMM (Gauss three-real-product form):
//   C[b] = alpha * opA(A[b]) opB(B[b]) + beta * C[b] + sum_t coef[t] * X_t[b] + gamma * I
//   C2[b] = X2[b] + alpha2 * opA(A[b]) opB(B[b])          (when C2 != nullptr)
// All matrices row-major complex128.  opB: 0 = B, 1 = B^T, 2 = conj(B), 3 = B^H.
// conjA conjugates A.  A batch element b is skipped when
// active != nullptr and active[b] <= active_iter.
struct ZGemmProblem {
  int M = 0, N = 0, K = 0;
  const z64* A = nullptr; long long lda = 0, sA = 0; int conjA = 0;
  const z64* B = nullptr; long long ldb = 0, sB = 0; int opB = 0;
  z64* C = nullptr; long long ldc = 0, sC = 0;
  double alpha = 1.0, beta = 0.0, gamma = 0.0;
  int nterms = 0;
  const z64* X[4] = {nullptr, nullptr, nullptr, nullptr};
  long long sX[4] = {0, 0, 0, 0};
  double coef[4] = {0, 0, 0, 0};
  z64* C2 = nullptr; const z64* X2 = nullptr; long long sX2 = 0; double alpha2 = 1.0;
  const int* active = nullptr; int active_iter = 0;
  const int* active_lo = nullptr;  // also skip b when active_lo[b] > active_iter
  double shiftA = 0.0, shiftB = 0.0;  // subtracted from the diagonals of A and B as loaded
  int batch = 1;
};

// Launch up to 4 problems in one grouped launch.  Returns a CUDA error code.
cudaError_t zgemm_f64(const ZGemmProblem* probs, int nprob, int sm_count, cudaStream_t st);

// Grouped, batched REAL GEMM (k_rgemm.cu), FP64 (T = double) or FP32
// (T = float: FP32 operands and accumulation), for the real-coordinate forms:
//   r_w  = alpha[w] acc + beta[w] O_w(old) + sum_t coef[w][t] X_t + gamma[w] I   (in T)
//   O_w  = r_w (when O[w] != null);  Od_w = double(r_w) + dcoef[w] Xd + dgamma[w] I (when Od[w] != null)
// acc = (A - shiftA I)(B - shiftB I) or (A - shiftA I)(B - shiftB I)^T (transB),
// row-major; every output and term has leading dimension ldc and batch stride
// sC (sX[t], sXd for the terms).  Batch element b is skipped when
// active[b] <= active_iter or active_lo[b] > active_iter.
template <typename T>
struct RGemmProblem {
  int M = 0, N = 0, K = 0, batch = 1;
  const T* A = nullptr; long long lda = 0, sA = 0;
  const T* B = nullptr; long long ldb = 0, sB = 0; int transB = 0;
  long long ldc = 0, sC = 0;
  T* O[2] = {nullptr, nullptr};
  double* Od[2] = {nullptr, nullptr};
  double alpha[2] = {1.0, 1.0}, beta[2] = {0.0, 0.0}, gamma[2] = {0.0, 0.0};
  int nterms = 0;
  const T* X[3] = {nullptr, nullptr, nullptr};
  long long sX[3] = {0, 0, 0};
  double coef[2][3] = {{0, 0, 0}, {0, 0, 0}};
  const double* Xd = nullptr; long long sXd = 0;
  double dcoef[2] = {0.0, 0.0}, dgamma[2] = {0.0, 0.0};
  const int* active = nullptr; int active_iter = 0;
  const int* active_lo = nullptr;
  const int* pick = nullptr; int pick_val = 0;  // also skip b when pick[b] != pick_val
  double shiftA = 0.0, shiftB = 0.0;
};
cudaError_t rgemm_f64(const RGemmProblem<double>* probs, int nprob, int sm_count, cudaStream_t st);
cudaError_t rgemm_f32(const RGemmProblem<float>* probs, int nprob, int sm_count, cudaStream_t st);
// The same product for a left operand whose rows are mostly zeros (the low
// powers of a local generator): one warp per output row, only the nonzeros
// of A's row multiplied.  Needs transB == 0, shiftB == 0 and N <= 736
// (cudaErrorInvalidValue otherwise).
template <typename T>
cudaError_t rgemm_rowskip(const RGemmProblem<T>& p, int sm_count, cudaStream_t st);
// A nonzero pattern by rows: the columns of row r, increasing, at
// cols[rowbeg[r] .. rowend[r]); total counts them.
struct CsrPattern {
  int* rowbeg = nullptr;
  int* rowend = nullptr;
  int* cols = nullptr;
  unsigned long long* total = nullptr;
};
// The same product with A's nonzero pattern (a superset of every batch
// element's) given by rows; the same terms in the same order as
// rgemm_rowskip.  Needs shiftA == 0 besides rgemm_rowskip's conditions.
template <typename T>
cudaError_t rgemm_csr(const RGemmProblem<T>& p, const int* rowbeg, const int* rowend, const int* cols, int sm_count,
                      cudaStream_t st);
// The union pattern of X0 and X1 (n x n row-major FP64; X1 may be null)
// into pat (row r's columns at cols[r n ..]); flag[0 .. S) = 1 when it has at
// most max_nnz entries, else 0.
cudaError_t launch_csr_union(int n, const double* X0, const double* X1, long long max_nnz, int S, CsrPattern pat,
                             int* flag, cudaStream_t st);
// flag[s] = 1 if M[s] (S row-major n x n matrices) has at most max_nnz
// nonzero entries, else 0.
template <typename T>
cudaError_t launch_sparse_flags(int n, int S, const T* M, long long max_nnz, int* flag, int sm_count,
                                cudaStream_t st);

// Few-state FP64 products (k_gemv.cu), B <= kGemvMaxB:
//   V[b][i] = alpha sum_j A[i][j] X[b][j];  Yacc[b][i] += the same (Yacc may be null)
constexpr int kGemvMaxB = 8;
cudaError_t launch_zgemv_f64(int n, int B, const z64* A, long long lda, const z64* X, long long ldx, z64* V,
                             long long ldv, double alpha, z64* Yacc, long long ldacc, cudaStream_t st);
// The real counterpart (real A and states), B <= kGemvMaxB.
cudaError_t launch_dgemv_f64(int n, int B, const double* A, long long lda, const double* X, long long ldx, double* V,
                             long long ldv, double alpha, double* Yacc, long long ldacc, cudaStream_t st);
// Whether a B-state FP64 propagation step at size n goes to launch_zgemv_f64.
bool gemv_f64_preferred(int n, int B);

// Real coordinates of a d x d Hermitian matrix (n = d^2 of them): the
// diagonal entries, then Re and Im of the upper-triangle entries (k < l) in
// row-major order.  Coordinate a -> (k, l, part): part 0 = rho_kk (k = l),
// 1 = Re rho_kl, 2 = Im rho_kl.
// Coordinates of the upper-triangle rows before row k: sum_{r < k} (d - 1 - r).
__host__ __device__ inline int herm_row_base(int k, int d) { return k * (2 * d - k - 1) / 2; }
__host__ __device__ inline void herm_coord(int a, int d, int* k, int* l, int* part) {
  if (a < d) {
    *k = a;
    *l = a;
    *part = 0;
    return;
  }
  const int q = (a - d) >> 1;
  *part = 1 + ((a - d) & 1);
  // the row r with herm_row_base(r) <= q < herm_row_base(r + 1): the root of
  // the quadratic, then corrected by whole steps
  const float t = (float)(2 * d - 1);
  int r = (int)(0.5f * (t - sqrtf(fmaxf(t * t - 8.0f * (float)q, 0.0f))));
  if (r < 0) r = 0;
  if (r > d - 2) r = d - 2;
  while (r > 0 && herm_row_base(r, d) > q) r--;
  while (r < d - 2 && herm_row_base(r + 1, d) <= q) r++;
  *k = r;
  *l = r + 1 + q - herm_row_base(r, d);
}
// Index of the Re coordinate of the upper-triangle entry (k, l), k < l.
__host__ __device__ inline int herm_pair_coord(int k, int l, int d) { return d + 2 * (herm_row_base(k, d) + l - k - 1); }

// Hermitian (real-coordinate) FP64 propagation, k_herm.cu: the lane split of
// the one-warp latency form (false: n above 9), the real transfer matrices of
// S propagators (S x n x n doubles), and the propagation of B states.
bool herm_lat_split(int n, int* C, int* K);
cudaError_t launch_herm_matrix(int n, int d, int S, const z64* P, double* R, int sm_count, cudaStream_t st);
cudaError_t launch_prop_herm_lat(int n, int d, int nslices, const double* R, int steps_per_slice, int B, z64* X,
                                 cudaStream_t st);
bool herm_resident_fits(int n);
cudaError_t launch_herm_coords_in(int n, int d, int B, const z64* X, double* Y, int sm_count, cudaStream_t st);
cudaError_t launch_herm_coords_out(int n, int d, int B, const double* Y, z64* X, int sm_count, cudaStream_t st);
cudaError_t launch_real_colnorm(int n, int S, const double* G, unsigned long long* norm_bits, int sm_count,
                                cudaStream_t st);
cudaError_t launch_prop_herm_resident(int n, int d, int nslices, const double* R, int steps_per_slice, int B,
                                      z64* X, int sm_count, cudaStream_t st);

// (m, s) of the truncated Taylor series for ||A||_1 = a (k_expmv.cu); false
// for a non-finite a or more than 65536 sub-steps.
bool taylor_parameters(double a, int* m_out, int* s_out);

// Autotuner shared by the GEMM families (k_gemm.cu).  A launch shape key
// (family, precision, every problem's sizes and flags) and a launcher of
// candidate tile configuration `cand`.  In tuning mode, which set_tuning
// switches for the CALLING HOST THREAD only, a launch runs and times every
// candidate and records the fastest for its shape; otherwise a recorded shape
// uses its record and other shapes the caller's heuristic.
typedef std::array<long long, 24> TuneKey;
typedef cudaError_t (*TuneCand)(int cand, const void* args, cudaStream_t st);
cudaError_t tuned_launch(const TuneKey& key, int ncand, int heuristic, TuneCand run, const void* args,
                         cudaStream_t st);
void set_tuning(bool on);
int tuned_shapes();

// FP32 variant (operands rounded to FP32, FP32 accumulation, FP64 epilogue).
cudaError_t zgemm_f32(const ZGemmProblem* probs, int nprob, int sm_count, cudaStream_t st);

// ------------------------------------------------------------ assembly ----
cudaError_t launch_assemble(int d, const z64* H, int K, const z64* Ls, z64* L_out, z64* G_scratch,
                            int sm_count, cudaStream_t st);

// A_s = (Lbase + u_s Ldrv) dt (or Lbase[s] dt); column abs-sums -> norm1[s]
// (as uint64 bit patterns of non-negative doubles, max-reduced), then
// sc[s] and A_s /= 2^sc[s].
// kmix[s] (may be null) receives how many of the leading squarings of slice s
// keep ||P - I|| small enough for the mixed D-form (scaled norm * 2^k <= 1).
cudaError_t launch_slice_prepare(int n, int S, const z64* Lbase, const z64* Ldrv, const double* u,
                                 double dt, z64* A, unsigned long long* norm_bits, int* sc,
                                 int* kmix, int* s_out, unsigned int* err, int sm_count,
                                 cudaStream_t st);

// sc[s] = max(0, ceil(log2(norm_s / theta))) from norm_bits[s] (and kmix, s_out,
// the maximum into sc[S], as launch_slice_prepare does).
cudaError_t launch_squaring_count(int S, const unsigned long long* norm_bits, int* sc, int* kmix, int* s_out,
                                  unsigned int* err, cudaStream_t st);

// ------------------------------------------- real-coordinate build (k_real.cu)
// A_s = (Gb + u_s Gd) dt / 2^sc[s] on the real coordinates (Gd == null: Gb
// holds S generators); per-slice 1-norms, squaring counts as above.
cudaError_t launch_real_slice_prepare(int n, int S, const double* Gb, const double* Gd, const double* u, double dt,
                                      double* A, unsigned long long* norm_bits, int* sc, int* kmix, int* s_out,
                                      unsigned int* err, int sm_count, cudaStream_t st);
template <typename T>
cudaError_t launch_real_lincomb3(long long total, const T* X0, const T* X1, const T* X2, double c0, double c1,
                                 double c2, T* Z, int sm_count, cudaStream_t st);
// an R x C block of S real matrices (leading dimension, batch stride each)
cudaError_t launch_real_copy_block(int R, int C, int S, const double* src, long long sld, long long ss, double* dst,
                                   long long dld, long long ds, int sm_count, cudaStream_t st);
// A_s^2 = (dt 2^-sc[s])^2 (P0 + u_s (P1 + u_s P2)) for S slices (P0, P1, P2: n x n)
cudaError_t launch_real_affine_square(int n, int S, const double* P0, const double* P1, const double* P2,
                                      const double* u, double dt, const int* sc, double* A2, int sm_count,
                                      cudaStream_t st);
// Z1, Z2, V, W of the [13/13] approximant from A^6, A^4, A^2 (b: the 14 coefficients)
cudaError_t launch_real_pade_terms(int n, int S, const double* A6, const double* A4, const double* A2,
                                   const double* b, double* Z1, double* Z2, double* V, double* W, int sm_count,
                                   cudaStream_t st);
// The Pade coefficients b_0 .. b_13 by value.
struct PadeCoef {
  double b[14];
};
// V, W of the approximant as sums of the even powers A^2 .. A^12 (slices
// with flag[s] != 0), the identity terms b0, b1 added when with_identity.
template <typename T>
cudaError_t launch_real_powsum(int n, int S, const int* flag, const T* A2, const T* A4, const T* A6, const T* A8,
                               const T* A10, const T* A12, const double* b, int with_identity, T* V, T* W,
                               int sm_count, cudaStream_t st);
// dst = float(src - shift I), S n x n matrices
cudaError_t launch_real_to_f32(int n, int S, const double* src, double shift, float* dst, int sm_count,
                               cudaStream_t st);
cudaError_t launch_real_copy_active(long long nn, int S, const double* src, double* dst, const int* active, int iter,
                                    int sm_count, cudaStream_t st);
// P[s] (complex superoperator) from R[s] (its real-coordinate matrix)
cudaError_t launch_herm_to_complex(int n, int d, int S, const double* R, z64* P, int sm_count, cudaStream_t st);
// nb: the block size, 32 (kLuNb) or 64
cudaError_t launch_lu_diag_real(int n, int S, int k0, int kb, const double* M, double* Uf, double* Linv,
                                long long sLinv, double* Uinv, long long sUinv, unsigned int* err, cudaStream_t st,
                                int nb = kLuNb);
// The real-coordinate propagator build (lb_expm_pade with a Hermitian
// precision) and the real-coordinate propagation for n > 81 (lb_real.cu).
lb_status expm_chunk_herm(lb_ctx* c, int n, int S, const z64* Lbase, const z64* Ldrv, const double* u, double dt,
                          lb_precision prec, z64* P, int* s_out, cudaStream_t st);
lb_status propagate_herm_large(lb_ctx* c, int n, int nslices, const z64* P, int steps_per_slice, int B, z64* X,
                               bool sliced, cudaStream_t st);
// Stage-timer events of one build chunk (null when timing is off).
lb_status stage_events_begin(lb_ctx* c, cudaStream_t st, cudaEvent_t** ev_out);

// Elementwise linear combinations used by the Pade step.
// Z[b] = c0*X0[b] + c1*X1[b] + c2*X2[b]  (n x n each, batch strides = n*n)
cudaError_t launch_lincomb3(int nn, int S, const z64* X0, const z64* X1, const z64* X2, double c0,
                            double c1, double c2, z64* Z, cudaStream_t st);
// Z[b] += 2 X[b] (nn elements per batch element)
cudaError_t launch_add_twice(long long nn, int S, const z64* X, z64* Z, cudaStream_t st);

// --------------------------------------------------------------- LU -------
// Factor the kb x kb diagonal block at (k0, k0) of M[b] (no pivot search),
// write Linv and Uinv (nb x nb each, per batch) and the U11 factor into Uf.
cudaError_t launch_lu_diag(int n, int S, int k0, int kb, const z64* M, z64* Uf, z64* Linv,
                           long long sLinv, z64* Uinv, long long sUinv, unsigned int* err,
                           cudaStream_t st);

// Copy rows/cols helper: dst[b][r][c] = src[b][r][c] for r in [r0,r0+nr), c in [c0,c0+nc)
cudaError_t launch_copy_block(int S, long long ld, long long stride, int r0, int nr, int c0, int nc,
                              const z64* src, z64* dst, cudaStream_t st);

// ------------------------------------------------------------ misc --------
cudaError_t launch_copy_active(long long nn, int S, const z64* src, z64* dst, const int* active,
                               int iter, cudaStream_t st);
cudaError_t launch_check_finite(long long count, const z64* x, unsigned int* err, cudaStream_t st);

// ----------------------------------------------------------- propagation --
// Resident FP64 propagation for small n (P in shared memory): every step of
// the chain in one launch, states split across CTAs.
cudaError_t launch_propagate_resident_f64(int n, int nslices, const z64* P, int steps_per_slice,
                                          int B, z64* states, int sm_count, cudaStream_t st);
bool resident_f64_fits(int n);

// FP32 propagation with D = P - I stored in FP32 planes.
cudaError_t launch_make_delta_f32(int n, int S, const z64* P, float* Dr, float* Di, cudaStream_t st);
cudaError_t launch_propagate_resident_f32(int n, int nslices, const float* Dr, const float* Di,
                                          int steps_per_slice, int B, z64* states, int renorm,
                                          int sm_count, cudaStream_t st);
bool resident_f32_fits(int n);
// Large-n FP32 step: Rout = Rin + Rin * D^T (planar FP32 states), optional renorm.
// FP32 chain for n > 81 (k_chain32.cu)
size_t chain32_dplane_floats(int n);
size_t chain32_state_floats(int n, int B);
size_t chain32_part_floats(int sm_count);
cudaError_t launch_chain32_dplanes(int n, int S, const z64* P, float* Dt, cudaStream_t st);
cudaError_t launch_chain32_states_in(int n, int B, const z64* X, float* Rt, cudaStream_t st);
cudaError_t launch_chain32_states_out(int n, int B, int renorm, const float* Rt, z64* X, cudaStream_t st);
// The whole chain in one persistent launch (nsteps steps, slice t /
// steps_per_slice of the D^T planes at Dt + slice * dstride; states ping-pong
// between Ra and Rb, the result in Ra if nsteps is even, else in Rb; bar: a
// scratch counter).  false: not possible for this shape (nothing queued), use
// per-step launches.  *status: a CUDA error met after the decision.
bool launch_chain32_persist(int n, int B, int renorm, const float* Dt, long long dstride, int steps_per_slice,
                            int nsteps, float* Ra, float* Rb, unsigned* bar, unsigned int* err, int sm_count,
                            cudaStream_t st, cudaError_t* status);
// pdl: launch with programmatic stream serialisation (only when the
// previous launch on the stream is another step of the same chain)
cudaError_t launch_chain32_step(int n, int B, int renorm, const float* Dt, const float* Rt, float* Ot, float* part,
                                unsigned* cnt, int sm_count, bool pdl, cudaStream_t st);

// n x n square problem, batch S, slice stride n*n (helper for the build).
ZGemmProblem sq(int n, int S, const z64* A, const z64* B, z64* C);

// Blocked LU (no pivot search) of Mx[s] and solve for the nrhs columns of N[s].
lb_status lu_solve_blocked(lb_ctx* c, int n, int S, z64* Mx, z64* N, int nrhs, long long ldN, long long sN,
                           z64* Uf, z64* Y, z64* Lp, cudaStream_t st);

// GRAPE scratch (bytes) for a context of these limits; 0 when max_n > 81.
size_t grape_ws_bytes(int max_n, int max_batch, int max_slices);
constexpr int kGrapeMaxN = 81;
constexpr int kGrapeMaxB = 64;
constexpr int kGrapeMaxStepsPerSlice = 20;

// Resident FP64 chain with optional history and adjoint (conjugate transpose,
// slices in reverse order).  hist (may be null) receives the states before the
// first step and after every step: forward index t = 0..T, adjoint index T - k
// after k steps (T = nslices * steps_per_slice).
cudaError_t launch_propagate_resident_f64_hist(int n, int nslices, const z64* P, int steps_per_slice, int B,
                                               z64* states, int adjoint, z64* hist, int sm_count,
                                               cudaStream_t st);

// The same chain for K independent problems in one launch (problem k: its
// nslices propagators at P + k nslices n^2, its B states at states + k B n),
// with the compact history (T = nslices * steps_per_slice entries per
// problem at hist + k T B n: forward X_0 .. X_{T-1}, adjoint Lam_1 .. Lam_T).
cudaError_t launch_propagate_resident_f64_multi(int n, int K, int nslices, const z64* P, int steps_per_slice, int B,
                                                z64* states, int adjoint, z64* hist, int sm_count, cudaStream_t st);

// dst[s](ld_d, col off_d) = c0 X0[s](ld_0, off_0) + c1 X1[s](ld_1, off_1), n x n blocks.
cudaError_t launch_combine(int n, int S, double c0, const z64* X0, long long ld0, long long s0, double c1,
                           const z64* X1, long long ld1, long long s1, z64* dst, long long ldd, long long sd,
                           cudaStream_t st);
// E[s] = Ldrv * dt / 2^sc[s]
cudaError_t launch_scale_bcast(int n, int S, const z64* Ldrv, double dt, const int* sc, z64* E, cudaStream_t st);
// out[s] = scale * Re sum_e conj(L[s][e]) Y[s][e], e < len, slice strides sL, sY (deterministic).
cudaError_t launch_redot(int S, long long len, const z64* L, long long sL, const z64* Y, long long sY,
                         double scale, double* out, cudaStream_t st);

// ------------------------------------------------------ tensor cores ----
// Complex GEMM in split-BF16 x3 on tcgen05 (see k_tc.cu).  Operands are plane
// tensors bf16 [batch][4][rows][ld] (re_hi, re_lo, im_hi, im_lo), K-major:
// A operand = X (M x K), B operand = Y^T (N x K) for C = X Y.
struct TcProblem {
  int M = 0, N = 0, K = 0, batch = 1;
  int npa = 2, npb = 2;  // BF16 pieces per value of A / B: (2, 2) or (2, 3); planes = 2 * pieces
  const __nv_bfloat16* Aop = nullptr; long long a_ld = 0, a_plane = 0;
  const __nv_bfloat16* Bop = nullptr; long long b_ld = 0, b_plane = 0;
  // every output and X term is row-major [row][col] with leading dimension
  // ldc and batch stride sC (sX for the X terms)
  long long ldc = 0, sC = 0;
  // r = alpha acc + sum_t coef_t X_t,  r2 = alpha2 acc + sum_t coef2_t X_t  (FP32)
  float alpha = 1.f, alpha2 = 0.f;
  int nterms = 0;
  const float2* X[4] = {nullptr, nullptr, nullptr, nullptr};
  long long sX[4] = {0, 0, 0, 0};
  float coef[4] = {0, 0, 0, 0}, coef2[4] = {0, 0, 0, 0};
  float2* Cf = nullptr;                  // r in FP32
  z64* Cd = nullptr; double gamma = 0;   // r widened to FP64, + gamma on the diagonal
  z64* C2d = nullptr; double gamma2 = 0; // r2 widened to FP64, + gamma2 on the diagonal
  __nv_bfloat16* sp = nullptr; long long sp_ld = 0, sp_plane = 0; float sp_shift = 0.f;    // planes of r
  __nv_bfloat16* spT = nullptr; long long spT_ld = 0, spT_plane = 0; float spT_shift = 0.f;  // of r^T
  // optional per-row factor 1 / Tr(row of rs_src) (a row read as a d x d
  // matrix, leading dimension ldc) applied to r before it is written
  const float2* rs_src = nullptr; int rs_d = 0;
  // optional split of K over up to max_ctas / tiles CTAs: FP32 partial tiles
  // in part (max_ctas x 128 x 64 float2), one ticket per tile in cnt
  // (zero between launches); the last CTA of a tile sums them in split order
  float2* part = nullptr; unsigned* cnt = nullptr; int max_ctas = 0;
  // optional batch mask: batch element b is skipped when active[b] <= active_iter
  const int* active = nullptr; int active_iter = 0;
  // launch with programmatic stream serialisation: only when the previous
  // launch on the stream is a step of the same chain (it writes the A
  // operand and the X terms, never the B operand)
  int pdl = 0;
  unsigned int* err = nullptr;
};
cudaError_t zgemm_tc(const TcProblem& p, cudaStream_t st);

// FP64 product C = alpha A B + beta C through exact BF16 slices on the
// tensor cores (k_ozaki.cu).  A(m, k) of batch element b at
// A[b sA + m a_sm + k a_sk], B(k, n) at B[b sB + k b_sk + n b_sn], C
// row-major with leading dimension ldc.  C may alias A or B (both are
// consumed into slices before C is written).  K <= kOzMaxK.
constexpr int kOzSlices = 9;    // base-64 digits per operand row / column (54 bits)
constexpr int kOzMaxK = 1488;   // every group sum exact in FP32 up to this K
constexpr int kOzPairs = kOzSlices * (kOzSlices + 1) / 2;  // digit products per multiply-add (45)
// Further outputs of a sliced product, formed in its epilogue from the
// product's element out (after alpha and beta) and two matrices T1, T2 laid
// out like C (row-major, C's ldc and sC; T1 or T2 may be null, read as 0):
//   X_w[e] = c[w][0] out + (c[w][1] T1[e] + c[w][2] T2[e]) (+ g[w] where row == column)
// for w < nx (at most 4); or, with pm set (and nx = 2), X_0 = T1 - out and
// X_1 = T1 + out (one FP64 operation each).  Not with transC.
struct OzExtra {
  int nx = 0;
  int pm = 0;
  const double* T1 = nullptr;
  const double* T2 = nullptr;
  double* X[4] = {nullptr, nullptr, nullptr, nullptr};
  double c[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double g[4] = {0, 0, 0, 0};
};
struct OzGemm {
  int M = 0, N = 0, K = 0, batch = 1;
  const double* A = nullptr; long long a_sm = 0, a_sk = 1, sA = 0;
  const double* B = nullptr; long long b_sk = 0, b_sn = 1, sB = 0;
  double* C = nullptr; long long ldc = 0, sC = 0;
  int transC = 0;  // C element (m, n) at C[b sC + n ldc + m] instead of C[b sC + m ldc + n]
  double alpha = 1.0, beta = 0.0;
  // optional batch mask: batch element b is skipped when active[b] <= active_iter
  const int* active = nullptr; int active_iter = 0;
  const int* EA = nullptr; const int* EB = nullptr;  // row / column exponents (set by ozgemm_f64)
  unsigned int* err = nullptr;
  OzExtra x;  // C may be null when x.nx > 0 (the product itself not stored)
};
constexpr int kOzBN = 48;       // columns of C per CTA (B tile rows)
constexpr int kOzBNSmall = 16;  // the narrow tile, for products with few output tiles
constexpr int kOzBNMid = 32;    // for products with 64 columns
constexpr int kOzTileM = 128;   // rows of C per CTA (A tile rows)
// An operand in slices: digit planes in the tile-blocked layout of
// k_ozaki.cu (tile_rows = 128 for A, kOzBN for B) and one exponent per row.
struct OzSliced {
  __nv_bfloat16* Q = nullptr;
  int* E = nullptr;
  int rows = 0, K = 0, batch = 0, tile_rows = 0;
};
size_t oz_sliced_bytes(int rows, int K, int batch, int tile_rows);
OzSliced oz_carve(void* base, int rows, int K, int batch, int tile_rows);
OzSliced oz_view(const OzSliced& o, int b);  // batch element b alone
// rows r of X (element (r, k) of batch element b at X[b sb + r sr + k sk]) in slices
cudaError_t oz_slice(const double* X, long long sr, long long sk, long long sb, const OzSliced& o, const int* active,
                     int active_iter, cudaStream_t st);
// C = alpha A B + beta C from sliced A (M rows) and sliced B^T (N rows); p's
// A, B pointers are not used
cudaError_t oz_multiply(const OzSliced& A, const OzSliced& B, const OzGemm& p, int sm_count, cudaStream_t st,
                        cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
// scratch for one call of ozgemm_f64: the slices of both operands
size_t oz_scratch_bytes(int M, int N, int K, int batch);
int oz_bn_for(int N);  // the column tile ozgemm_f64 takes for N columns
cudaError_t ozgemm_f64(const OzGemm& p, void* scratch, size_t scratch_bytes, int sm_count, cudaStream_t st,
                       cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
// events to bracket one sliced-product launch of `flops` digit-product FLOPs
// (both null unless the context's stage timers are on)
cudaError_t kernel_events(lb_ctx* c, double flops, cudaEvent_t* ev0, cudaEvent_t* ev1);
// Z = c0 X0 + c1 X1 + c2 X2 (FP32) written as the two-piece planes of Z^T
cudaError_t launch_lincomb_splitT(int n, int S, const float2* X0, const float2* X1, const float2* X2, float c0,
                                  float c1, float c2, __nv_bfloat16* dst, long long ldd, long long plane,
                                  cudaStream_t st);
// per FP32 state: optional division by the trace, then the row's two-piece planes
cudaError_t launch_renorm_split(int n, int d, int B, int renorm, float2* X, long long xld, __nv_bfloat16* planes,
                                long long ld, long long plane, cudaStream_t st);
cudaError_t launch_states_c64_f32(int n, int B, const z64* a, float2* b, long long ld, cudaStream_t st);
cudaError_t launch_states_f32_c64(int n, int B, const float2* a, long long ld, z64* b, cudaStream_t st);
long long plane_ld(int K);
// planes of src (R x Kc per slice) or of its transpose, diagonal shifted
// np BF16 pieces per value: planes [S][2 np][..] (re pieces, then im pieces)
// (f32, optional: FP32 copy of the shifted source, row-major R x Kc per slice)
cudaError_t launch_split(int R, int Kc, int S, const z64* src, long long lds, long long ss, double shift, int trans,
                         __nv_bfloat16* dst, long long ldd, long long plane, cudaStream_t st, int np = 2,
                         float2* f32 = nullptr);

// Internal entry points shared by the C ABI functions.
lb_status propagate_impl(lb_ctx* c, int n, int nslices, const z64* P, int steps_per_slice, int B, z64* X,
                         lb_precision prec, int renorm_trace, cudaStream_t st);
size_t inst_table_bytes();
lb_status autotune_impl(lb_ctx* c, int n, int nslices, int B, cudaStream_t st, int* shapes_out);
lb_status expm_chunk_public(lb_ctx* c, int n, int S, const z64* Lbase, const z64* Ldrv, const double* u, double dt,
                            lb_precision prec, z64* P, int* s_out, cudaStream_t st);

// err |= ERR_SQUARING_BOUND when *sc_max > bound
cudaError_t launch_check_bound(const int* sc_max, int bound, unsigned int* err, cudaStream_t st);

// Raise a kernel's dynamic shared-memory limit only when a larger size is
// needed (no host API call on repeated launches, e.g. during graph capture).
cudaError_t set_smem_once(const void* kernel, size_t bytes);

}  // namespace lb


