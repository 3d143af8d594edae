// Host orchestration of the real-coordinate ("Hermitian") forms: the
// propagator build of Algorithm 1 and, for n > 81, the propagation chain of
// Algorithm 2 on the n = d^2 real coordinates of Hermitian matrices.
//
// Every Lindbladian maps Hermitian matrices to Hermitian matrices, and so do
// its exponential and every polynomial in it.  On the real coordinates
// c = (rho_kk; Re rho_kl, Im rho_kl for k < l) a Hermiticity-preserving
// superoperator is a real n x n matrix (k_herm.cu builds it from the complex
// one), and because that correspondence is an algebra map (it takes sums to
// sums, products to products and I to I) Algorithm 1 run on G = the real form
// of L dt gives the real form of exp(L dt).  The build here therefore forms
// the real generators, runs the scaling, the six Pade products, the LU
// factorisation and solve of (V - U) R = (V + U) and the squarings on real
// matrices, and rebuilds the complex P from R at the end.  A real
// multiply-add is one FMA instead of four (three in the Gauss form of the
// complex GEMM), which is what bounds the build on GB300's FP64 pipe.
// The scaling parameter s is taken from ||G||_1 on these coordinates.
// Four of the six Pade products have A or A^2 as their left operand (A^6 is
// formed as A^2 A^4); where that operand is sparse, as for a local
// Lindbladian, they skip its zeros as the paper's products do (Sec. 3.1),
// chosen per slice on the device from the operand's nonzero count.  Where
// A^2 is sparse, the two dense products A^6 Z1 and A^6 Z2 are replaced too:
// A^8, A^10 and A^12 come from three more zero-skipping products with A^2 and
// V, W are summed term by term from the powers (the same [13/13]
// approximant), so every product of the build skips zeros.
#include "lb_internal.cuh"

namespace lb {

namespace {

int nblocks_r(int n) { return (n + kLuNb - 1) / kLuNb; }

RGemmProblem<double> rsq(int n, int S, const double* A, const double* B, double* C) {
  RGemmProblem<double> p;
  const long long nn = (long long)n * n;
  p.M = p.N = p.K = n;
  p.batch = S;
  p.A = A; p.lda = n; p.sA = nn;
  p.B = B; p.ldb = n; p.sB = nn;
  p.ldc = n; p.sC = nn;
  p.O[0] = C;
  return p;
}

RGemmProblem<float> fsq(int n, int S, const float* A, const float* B, float* C) {
  RGemmProblem<float> p;
  const long long nn = (long long)n * n;
  p.M = p.N = p.K = n;
  p.batch = S;
  p.A = A; p.lda = n; p.sA = nn;
  p.B = B; p.ldb = n; p.sB = nn;
  p.ldc = n; p.sC = nn;
  p.O[0] = C;
  return p;
}

// C -= L_panel U_panel style update: C(M x N, ldc) += alpha A(M x K) B(K x N)
RGemmProblem<double> rupd(int M, int N, int K, const double* A, long long lda, long long sA, const double* B,
                          long long ldb, long long sB, double* C, long long ldc, long long sC, double alpha,
                          double beta, int S) {
  RGemmProblem<double> p;
  p.M = M; p.N = N; p.K = K; p.batch = S;
  p.A = A; p.lda = lda; p.sA = sA;
  p.B = B; p.ldb = ldb; p.sB = sB;
  p.ldc = ldc; p.sC = sC;
  p.O[0] = C;
  p.alpha[0] = alpha;
  p.beta[0] = beta;
  return p;
}

// Blocked LU (no pivot search, left-looking) of the real Mx[s] and solve for
// the n columns of N[s]:  N <- Mx^{-1} N.  Uf (U), Lp (L) and Y are n x n
// per-slice scratch.  The same schedule as the complex form: at block step
// k one grouped GEMM brings block row k, block column k and the right-hand
// sides' block row up to date with all previous blocks (K = 32 k), the
// diagonal block is factored and inverted in shared memory, and the panels
// follow from the block inverses; the back substitution is left-looking too.
lb_status lu_solve_blocked_real(lb_ctx* c, int n, int S, double* Mx, double* N, double* Uf, double* Y, double* Lp,
                                cudaStream_t st) {
  const long long nn = (long long)n * n;
  const int nb = kLuNb, nbk = nblocks_r(n);
  const long long sLinv = (long long)nb * nb, sUinv = (long long)nbk * nb * nb;
  double* Linv = (double*)c->Linv;
  double* Uinv = (double*)c->Uinv;
  for (int k = 0; k < nbk; k++) {
    const int k0 = k * nb, kb = (n - k0 < nb) ? n - k0 : nb, rest = n - k0 - kb;
    double* Uinv_k = Uinv + (long long)k * nb * nb;
    if (k0 > 0) {
      RGemmProblem<double> pr[3];
      int np = 0;
      // block row k:  Mx[k0:k0+kb, k0:] -= L[k0:k0+kb, :k0] U[:k0, k0:]
      pr[np++] = rupd(kb, n - k0, k0, Lp + (long long)k0 * n, n, nn, Uf + k0, n, nn, Mx + (long long)k0 * n + k0, n,
                      nn, -1.0, 1.0, S);
      // block column k below the diagonal
      if (rest > 0)
        pr[np++] = rupd(rest, kb, k0, Lp + (long long)(k0 + kb) * n, n, nn, Uf + k0, n, nn,
                        Mx + (long long)(k0 + kb) * n + k0, n, nn, -1.0, 1.0, S);
      // right-hand sides, block row k:  N[k0:k0+kb, :] -= L[k0:k0+kb, :k0] Y[:k0, :]
      pr[np++] = rupd(kb, n, k0, Lp + (long long)k0 * n, n, nn, Y, n, nn, N + (long long)k0 * n, n, nn, -1.0, 1.0, S);
      LB_CUDA(rgemm_f64(pr, np, c->sm_count, st));
    }
    LB_CUDA(launch_lu_diag_real(n, S, k0, kb, Mx, Uf, Linv, sLinv, Uinv_k, sUinv, c->err_dev, st));
    RGemmProblem<double> pr[3];
    int np = 0;
    if (rest > 0) {
      // U[k0:k0+kb, k0+kb:] = Linv_k Mx[k0:k0+kb, k0+kb:]
      pr[np++] = rupd(kb, rest, kb, Linv, nb, sLinv, Mx + (long long)k0 * n + k0 + kb, n, nn,
                      Uf + (long long)k0 * n + k0 + kb, n, nn, 1.0, 0.0, S);
      // L[k0+kb:, k0:k0+kb] = Mx[k0+kb:, k0:k0+kb] Uinv_k
      pr[np++] = rupd(rest, kb, kb, Mx + (long long)(k0 + kb) * n + k0, n, nn, Uinv_k, nb, sUinv,
                      Lp + (long long)(k0 + kb) * n + k0, n, nn, 1.0, 0.0, S);
    }
    // Y[k0:k0+kb, :] = Linv_k N[k0:k0+kb, :]
    pr[np++] = rupd(kb, n, kb, Linv, nb, sLinv, N + (long long)k0 * n, n, nn, Y + (long long)k0 * n, n, nn, 1.0, 0.0,
                    S);
    LB_CUDA(rgemm_f64(pr, np, c->sm_count, st));
  }
  // back substitution: X_k = Uinv_k (Y_k - U[k0:k0+kb, k0+kb:] X[k0+kb:]), X into N
  for (int k = nbk - 1; k >= 0; k--) {
    const int k0 = k * nb, kb = (n - k0 < nb) ? n - k0 : nb, rest = n - k0 - kb;
    double* Uinv_k = Uinv + (long long)k * nb * nb;
    if (rest > 0) {
      RGemmProblem<double> g = rupd(kb, n, rest, Uf + (long long)k0 * n + k0 + kb, n, nn, N + (long long)(k0 + kb) * n,
                                    n, nn, Y + (long long)k0 * n, n, nn, -1.0, 1.0, S);
      LB_CUDA(rgemm_f64(&g, 1, c->sm_count, st));
    }
    RGemmProblem<double> f =
        rupd(kb, n, kb, Uinv_k, nb, sUinv, Y + (long long)k0 * n, n, nn, N + (long long)k0 * n, n, nn, 1.0, 0.0, S);
    LB_CUDA(rgemm_f64(&f, 1, c->sm_count, st));
  }
  return LB_OK;
}

// C = alpha A B + beta C through the sliced FP64 product, in chunks of
// batch elements that fit the context's scratch (defined below).
lb_status oz_product(lb_ctx* c, const OzGemm& p, cudaStream_t st);

// C_j = A B_j + beta_j C_j (j = 0, 1; n x n, S slices, row-major) with A
// sliced once, where both products' slices fit the scratch (else two
// oz_product calls).  B_1 is sliced after the first product is written, so
// it may be C_0.  x1 (may be null): further outputs of the second product.
lb_status oz_product_shared_a(lb_ctx* c, int n, int S, const double* A, const double* B0, double* C0, double beta0,
                              const double* B1, double* C1, double beta1, const OzExtra* x1, cudaStream_t st);

#define LB_TRY(x)                     \
  do {                                \
    lb_status r_ = (x);               \
    if (r_ != LB_OK) return r_;       \
  } while (0)

// C = alpha A B + beta C of a small real product (no transposed B, one
// output) as a sliced FP64 product
lb_status oz_small(lb_ctx* c, const RGemmProblem<double>& r, cudaStream_t st) {
  OzGemm q;
  q.M = r.M; q.N = r.N; q.K = r.K; q.batch = r.batch;
  q.A = r.A; q.a_sm = r.lda; q.a_sk = 1; q.sA = r.sA;
  q.B = r.B; q.b_sk = r.ldb; q.b_sn = 1; q.sB = r.sB;
  q.C = r.O[0]; q.ldc = r.ldc; q.sC = r.sC;
  q.alpha = r.alpha[0];
  q.beta = r.beta[0];
  return oz_product(c, q, st);
}

// The diagonal block of the two-level schedule: the kb x kb block (kb <= 128)
// at (k0, k0) of Mx, up to date with all earlier blocks, factored from two
// 64-wide halves (the first by lu_diag_real_kernel<64>, the off-diagonal
// blocks of U and L from its inverses, the second half's Schur complement
// and its factorisation), and the inverses of its unit-lower and upper
// factors assembled by the 2 x 2 block formulas
//   L^{-1} = [[L1^{-1}, 0], [-L2^{-1} L21 L1^{-1}, L2^{-1}]],
//   U^{-1} = [[U1^{-1}, -U1^{-1} U12 U2^{-1}], [0, U2^{-1}]]
// into Linv (128 x 128, zeroed here) and Uinv_k (128 x 128, zero on entry).  U's blocks go
// to Uf, L21 to Lp.  The seven 64 x 64 x 64 products are sliced FP64
// products too; `tmp` holds 6 S 64 x 64 doubles.
lb_status diag_block128(lb_ctx* c, int n, int S, double* Mx, double* Uf, double* Lp, int k0, int kb, double* Linv,
                        long long sLinv, double* Uinv_k, long long sUinv, double* tmp, cudaStream_t st) {
  constexpr int H = 64, NB = 128;
  const long long nn = (long long)n * n, hh = (long long)H * H;
  const int h0 = kb < H ? kb : H, h1 = kb - h0, k1 = k0 + h0;
  double *Li1 = tmp, *Ui1 = tmp + S * hh, *Li2 = tmp + 2 * S * hh, *Ui2 = tmp + 3 * S * hh, *T = tmp + 4 * S * hh,
         *T2 = tmp + 5 * S * hh;
  LB_CUDA(cudaMemsetAsync(Linv, 0, sizeof(double) * NB * NB * S, st));  // Uinv_k: zeroed by the caller
  LB_CUDA(launch_lu_diag_real(n, S, k0, h0, Mx, Uf, Li1, hh, Ui1, hh, c->err_dev, st, H));
  LB_CUDA(launch_real_copy_block(h0, h0, S, Li1, H, hh, Linv, NB, sLinv, c->sm_count, st));
  LB_CUDA(launch_real_copy_block(h0, h0, S, Ui1, H, hh, Uinv_k, NB, sUinv, c->sm_count, st));
  if (h1 == 0) return LB_OK;
  double* U12 = Uf + (long long)k0 * n + k1;
  double* L21 = Lp + (long long)k1 * n + k0;
  RGemmProblem<double> pr[2];
  // U12 = L1^{-1} Mx[k0:k1, k1:k1+h1];  L21 = Mx[k1:k1+h1, k0:k1] U1^{-1}
  pr[0] = rupd(h0, h1, h0, Li1, H, hh, Mx + (long long)k0 * n + k1, n, nn, U12, n, nn, 1.0, 0.0, S);
  pr[1] = rupd(h1, h0, h0, Mx + (long long)k1 * n + k0, n, nn, Ui1, H, hh, L21, n, nn, 1.0, 0.0, S);
  LB_TRY(oz_small(c, pr[0], st));
  LB_TRY(oz_small(c, pr[1], st));
  // the Schur complement of the second half, then its factorisation
  RGemmProblem<double> q = rupd(h1, h1, h0, L21, n, nn, U12, n, nn, Mx + (long long)k1 * n + k1, n, nn, -1.0, 1.0, S);
  LB_TRY(oz_small(c, q, st));
  LB_CUDA(launch_lu_diag_real(n, S, k1, h1, Mx, Uf, Li2, hh, Ui2, hh, c->err_dev, st, H));
  LB_CUDA(launch_real_copy_block(h1, h1, S, Li2, H, hh, Linv + (long long)h0 * NB + h0, NB, sLinv, c->sm_count, st));
  LB_CUDA(launch_real_copy_block(h1, h1, S, Ui2, H, hh, Uinv_k + (long long)h0 * NB + h0, NB, sUinv, c->sm_count, st));
  // T = L21 L1^{-1}, T2 = U12 U2^{-1}; then the off-diagonal blocks
  pr[0] = rupd(h1, h0, h0, L21, n, nn, Li1, H, hh, T, H, hh, 1.0, 0.0, S);
  pr[1] = rupd(h0, h1, h1, U12, n, nn, Ui2, H, hh, T2, H, hh, 1.0, 0.0, S);
  LB_TRY(oz_small(c, pr[0], st));
  LB_TRY(oz_small(c, pr[1], st));
  pr[0] = rupd(h1, h0, h1, Li2, H, hh, T, H, hh, Linv + (long long)h0 * NB, NB, sLinv, -1.0, 0.0, S);
  pr[1] = rupd(h0, h1, h0, Ui1, H, hh, T2, H, hh, Uinv_k + h0, NB, sUinv, -1.0, 0.0, S);
  LB_TRY(oz_small(c, pr[0], st));
  LB_TRY(oz_small(c, pr[1], st));
  return LB_OK;
}

// The same factorisation and solve with every product sliced (the
// LB_FP64_SLICED form), on a left-looking schedule: at block step k, block
// row k of the matrix (from the diagonal on), block column k below the
// diagonal and block row k of the right-hand sides are brought up to date
// with all earlier blocks in one product each (K = k0), so every entry is
// updated once, by one long product; the diagonal block is factored and
// inverted and the block row of U, the block column of L and block row k of
// Y = L^{-1} N follow from the block inverses.  The back substitution is
// left-looking too: block row k of Y takes U[k, k+1:] X[k+1:] in one
// product, then X_k = Uinv_k Y_k.  Every product has the columns of one
// block (128, or 32 below n = 256) on its short side; the products whose natural form has the
// block's rows run transposed (the long operand as the 128-row side, C
// written transposed).  Every product is one sliced launch over all slices.
// (A right-looking schedule with the same blocks slices each panel once but
// rewrites the trailing matrix at every step; measured at n = 729, 200
// slices: 35.3 ms against 31.0 ms for this one.)
lb_status lu_solve_sliced_ll(lb_ctx* c, int n, int S, double* Mx, double* N, double* Uf, double* Y, double* Lp,
                             double* inv, cudaStream_t st) {
  const long long nn = (long long)n * n;
  // 128-wide blocks (two 64-wide halves) from n = 256, their inverses and
  // the halves' scratch in `inv` (which holds 2 n^2 S doubles); else the
  // 32-wide blocks of the context's buffers
  const bool two = n >= 256;
  const int nb = two ? kLuNbSliced : kLuNb, nbk = (n + nb - 1) / nb;
  const long long sLinv = (long long)nb * nb, sUinv = (long long)nbk * nb * nb;
  double* Linv = two ? inv : (double*)c->Linv;                            // S x nb x nb
  double* Uinv = two ? inv + (long long)S * sLinv : (double*)c->Uinv;    // S x nbk x nb x nb
  double* tmp = inv + (long long)S * (sLinv + sUinv);                     // 6 S 64 x 64 (two-level only)
  if (two) LB_CUDA(cudaMemsetAsync(Uinv, 0, sizeof(double) * S * sUinv, st));
  // C = alpha A B + beta C (one per slice): A(m, k) at A + m a_sm + k a_sk,
  // B(k, j) at B + k b_sk + j b_sn, C(m, j) at C + m n + j or, transposed,
  // at C + j n + m
  auto prod = [&](int M, int Ncol, int K, const double* A, long long a_sm, long long a_sk, long long sA,
                  const double* B, long long b_sk, long long b_sn, long long sB, double* C, int trans, double alpha,
                  double beta) -> lb_status {
    OzGemm q;
    q.M = M; q.N = Ncol; q.K = K; q.batch = S;
    q.A = A; q.a_sm = a_sm; q.a_sk = a_sk; q.sA = sA;
    q.B = B; q.b_sk = b_sk; q.b_sn = b_sn; q.sB = sB;
    q.C = C; q.ldc = n; q.sC = nn; q.transC = trans;
    q.alpha = alpha;
    q.beta = beta;
    return oz_product(c, q, st);
  };
  for (int k = 0; k < nbk; k++) {
    const int k0 = k * nb, kb = (n - k0 < nb) ? n - k0 : nb, r0 = k0 + kb, rest = n - r0;
    double* Uinv_k = Uinv + (long long)k * nb * nb;
    lb_status r = LB_OK;
    if (k0 > 0) {
      // Mx[k0:r0, k0:] -= L[k0:r0, :k0] U[:k0, k0:], as its transpose (rows: the n - k0 columns)
      r = prod(n - k0, kb, k0, Uf + k0, 1, n, nn, Lp + (long long)k0 * n, 1, n, nn, Mx + (long long)k0 * n + k0, 1,
               -1.0, 1.0);
      // Mx[r0:, k0:r0] -= L[r0:, :k0] U[:k0, k0:r0]
      if (r == LB_OK && rest > 0)
        r = prod(rest, kb, k0, Lp + (long long)r0 * n, n, 1, nn, Uf + k0, n, 1, nn, Mx + (long long)r0 * n + k0, 0,
                 -1.0, 1.0);
      // N[k0:r0, :] -= L[k0:r0, :k0] Y[:k0, :], transposed
      if (r == LB_OK)
        r = prod(n, kb, k0, Y, 1, n, nn, Lp + (long long)k0 * n, 1, n, nn, N + (long long)k0 * n, 1, -1.0, 1.0);
    }
    if (r != LB_OK) return r;
    if (two)
      LB_TRY(diag_block128(c, n, S, Mx, Uf, Lp, k0, kb, Linv, sLinv, Uinv_k, sUinv, tmp, st));
    else
      LB_CUDA(launch_lu_diag_real(n, S, k0, kb, Mx, Uf, Linv, sLinv, Uinv_k, sUinv, c->err_dev, st, nb));
    if (rest > 0) {
      // U[k0:r0, r0:] = Linv_k Mx[k0:r0, r0:], transposed
      r = prod(rest, kb, kb, Mx + (long long)k0 * n + r0, 1, n, nn, Linv, 1, nb, sLinv, Uf + (long long)k0 * n + r0,
               1, 1.0, 0.0);
      // L[r0:, k0:r0] = Mx[r0:, k0:r0] Uinv_k
      if (r == LB_OK)
        r = prod(rest, kb, kb, Mx + (long long)r0 * n + k0, n, 1, nn, Uinv_k, nb, 1, sUinv,
                 Lp + (long long)r0 * n + k0, 0, 1.0, 0.0);
    }
    // Y[k0:r0, :] = Linv_k N[k0:r0, :], transposed
    if (r == LB_OK)
      r = prod(n, kb, kb, N + (long long)k0 * n, 1, n, nn, Linv, 1, nb, sLinv, Y + (long long)k0 * n, 1, 1.0, 0.0);
    if (r != LB_OK) return r;
  }
  for (int k = nbk - 1; k >= 0; k--) {
    const int k0 = k * nb, kb = (n - k0 < nb) ? n - k0 : nb, r0 = k0 + kb, rest = n - r0;
    double* Uinv_k = Uinv + (long long)k * nb * nb;
    lb_status r = LB_OK;
    // Y[k0:r0, :] -= U[k0:r0, r0:] X[r0:, :] (X in N's rows below), transposed
    if (rest > 0)
      r = prod(n, kb, rest, N + (long long)r0 * n, 1, n, nn, Uf + (long long)k0 * n + r0, 1, n, nn,
               Y + (long long)k0 * n, 1, -1.0, 1.0);
    // X[k0:r0, :] = Uinv_k Y[k0:r0, :] into N, transposed
    if (r == LB_OK)
      r = prod(n, kb, kb, Y + (long long)k0 * n, 1, n, nn, Uinv_k, 1, nb, sUinv, N + (long long)k0 * n, 1, 1.0, 0.0);
    if (r != LB_OK) return r;
  }
  return LB_OK;
}

// Density below which a power of A is multiplied as a row-sparse left
// operand (the zero-skip of the paper's Pade products, Sec. 3.1): the low
// powers of a local Lindbladian's real form have a few percent of nonzeros
// (A 1.2 %, A^2 5.6 % for the d = 27 transmon chain), where the row-sparse
// product is several times cheaper than the dense one.
constexpr double kSparseDensity = 0.15;

cudaError_t dense_gemm(const RGemmProblem<double>& p, int sms, cudaStream_t st) { return rgemm_f64(&p, 1, sms, st); }
cudaError_t dense_gemm(const RGemmProblem<float>& p, int sms, cudaStream_t st) { return rgemm_f32(&p, 1, sms, st); }

// C = A B for the S slices, A row-sparse where flag[s] = 1: the row-sparse
// product for those slices and the dense GEMM for the others (each launch
// skips the slices that are not its own).
template <typename T>
lb_status skip_product(lb_ctx* c, RGemmProblem<T> p, const int* flag, cudaStream_t st) {
  RGemmProblem<T> q = p;
  q.pick = flag;
  q.pick_val = 1;
  LB_CUDA(rgemm_rowskip(q, c->sm_count, st));
  p.pick = flag;
  p.pick_val = 0;
  LB_CUDA(dense_gemm(p, c->sm_count, st));
  return LB_OK;
}

// The same with A's nonzero pattern given by rows (flag[s] = 1: the pattern
// is sparse, the same for every slice).
lb_status csr_product(lb_ctx* c, RGemmProblem<double> p, const int* flag, const CsrPattern& pat, cudaStream_t st) {
  RGemmProblem<double> q = p;
  q.pick = flag;
  q.pick_val = 1;
  LB_CUDA(rgemm_csr(q, pat.rowbeg, pat.rowend, pat.cols, c->sm_count, st));
  p.pick = flag;
  p.pick_val = 0;
  LB_CUDA(dense_gemm(p, c->sm_count, st));
  return LB_OK;
}

// C = alpha A B + beta C through the sliced FP64 product, in chunks of
// batch elements that fit the context's scratch.
lb_status oz_product_shared_a(lb_ctx* c, int n, int S, const double* A, const double* B0, double* C0, double beta0,
                              const double* B1, double* C1, double beta1, const OzExtra* x1, cudaStream_t st) {
  const long long nn = (long long)n * n;
  OzGemm q;
  q.M = q.N = q.K = n;
  q.batch = S;
  q.A = A; q.a_sm = n; q.a_sk = 1; q.sA = nn;
  q.ldc = n; q.sC = nn;
  q.err = c->err_dev;
  const double* Bs[2] = {B0, B1};
  double* Cs[2] = {C0, C1};
  const double betas[2] = {beta0, beta1};
  if (oz_scratch_bytes(n, n, n, S) > c->oz_bytes) {
    for (int j = 0; j < 2; j++) {
      OzGemm p = q;
      p.B = Bs[j]; p.b_sk = n; p.b_sn = 1; p.sB = nn;
      p.C = Cs[j];
      p.beta = betas[j];
      if (j == 1 && x1 != nullptr) p.x = *x1;
      LB_TRY(oz_product(c, p, st));
    }
    return LB_OK;
  }
  const OzSliced As = oz_carve(c->oz_scratch, n, n, S, kOzTileM);
  const OzSliced Bsl = oz_carve((uint8_t*)c->oz_scratch + oz_sliced_bytes(n, n, S, kOzTileM), n, n, S, oz_bn_for(n));
  LB_CUDA(oz_slice(A, n, 1, nn, As, nullptr, 0, st));
  for (int j = 0; j < 2; j++) {
    LB_CUDA(oz_slice(Bs[j], 1, n, nn, Bsl, nullptr, 0, st));  // B(k, c) is row c, position k of B^T
    OzGemm p = q;
    p.C = Cs[j];
    p.beta = betas[j];
    if (j == 1 && x1 != nullptr) p.x = *x1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LB_CUDA(kernel_events(c, 2.0 * kOzPairs * (double)n * n * n * S, &e0, &e1));
    LB_CUDA(oz_multiply(As, Bsl, p, c->sm_count, st, e0, e1));
  }
  return LB_OK;
}

// p.C and the further outputs' matrices advanced by off elements
OzGemm oz_shift_out(const OzGemm& p, long long off) {
  OzGemm q = p;
  if (p.C != nullptr) q.C = p.C + off;
  if (p.x.T1 != nullptr) q.x.T1 = p.x.T1 + off;
  if (p.x.T2 != nullptr) q.x.T2 = p.x.T2 + off;
  for (int w = 0; w < p.x.nx; w++) q.x.X[w] = p.x.X[w] + off;
  return q;
}

lb_status oz_product(lb_ctx* c, const OzGemm& p, cudaStream_t st) {
  int chunk = p.batch;
  while (chunk > 1 && oz_scratch_bytes(p.M, p.N, p.K, chunk) > c->oz_bytes) chunk = (chunk + 1) / 2;
  if (oz_scratch_bytes(p.M, p.N, p.K, chunk) > c->oz_bytes) {
    // one batch element does not fit: blocks of rows of A and C (multiples
    // of the 128-row tile), each batch element in turn
    int rows = (p.M + 127) / 128 * 128;
    while (rows > 128 && oz_scratch_bytes(rows, p.N, p.K, 1) > c->oz_bytes) rows = (rows / 2 + 127) / 128 * 128;
    if (oz_scratch_bytes(rows, p.N, p.K, 1) > c->oz_bytes) return LB_EINVAL;
    for (int b0 = 0; b0 < p.batch; b0++)
      for (int m0 = 0; m0 < p.M; m0 += rows) {
        OzGemm q = oz_shift_out(p, (long long)b0 * p.sC + (p.transC ? (long long)m0 : (long long)m0 * p.ldc));
        q.batch = 1;
        q.M = std::min(rows, p.M - m0);
        q.A = p.A + (long long)b0 * p.sA + (long long)m0 * p.a_sm;
        q.B = p.B + (long long)b0 * p.sB;
        if (p.active != nullptr) q.active = p.active + b0;
        q.err = c->err_dev;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (p.active == nullptr)
          LB_CUDA(kernel_events(c, 2.0 * kOzPairs * q.M * (double)q.N * q.K, &e0, &e1));
        LB_CUDA(ozgemm_f64(q, c->oz_scratch, c->oz_bytes, c->sm_count, st, e0, e1));
      }
    return LB_OK;
  }
  for (int b0 = 0; b0 < p.batch; b0 += chunk) {
    OzGemm q = oz_shift_out(p, (long long)b0 * p.sC);
    q.batch = std::min(chunk, p.batch - b0);
    q.A = p.A + (long long)b0 * p.sA;
    q.B = p.B + (long long)b0 * p.sB;
    if (p.active != nullptr) q.active = p.active + b0;
    q.err = c->err_dev;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (p.active == nullptr)
      LB_CUDA(kernel_events(c, 2.0 * kOzPairs * q.M * (double)q.N * q.K * q.batch, &e0, &e1));
    LB_CUDA(ozgemm_f64(q, c->oz_scratch, c->oz_bytes, c->sm_count, st, e0, e1));
  }
  return LB_OK;
}


}  // namespace

lb_status expm_chunk_herm(lb_ctx* c, int n, int S, const z64* Lbase, const z64* Ldrv, const double* u, double dt,
                          lb_precision prec, z64* P, int* s_out, cudaStream_t st) {
  int d = 1;
  while (d * d < n) d++;
  const long long nn = (long long)n * n;
  const double* b = c->pade_b;
  cudaEvent_t* ev = nullptr;
  {
    lb_status r = stage_events_begin(c, st, &ev);
    if (r != LB_OK) return r;
  }
  double* Ar = (double*)c->A;
  double* Mx = (double*)c->Mx;
  double* N = (double*)c->Z1;  // right-hand sides, then the solution R, then the squarings
  double* T2 = (double*)c->Z2; // squaring products (FP64)
  // the real generators: G_base, G_drv (or the S generators) in V's buffer
  double* Gb = (double*)c->V;
  double* Gd = nullptr;
  if (Ldrv != nullptr) {
    Gd = Gb + nn;
    LB_CUDA(launch_herm_matrix(n, d, 1, Lbase, Gb, c->sm_count, st));
    LB_CUDA(launch_herm_matrix(n, d, 1, Ldrv, Gd, c->sm_count, st));
  } else {
    LB_CUDA(launch_herm_matrix(n, d, S, Lbase, Gb, c->sm_count, st));
  }
  LB_CUDA(launch_real_slice_prepare(n, S, Gb, Gd, u, dt, Ar, c->norm_bits, c->sc, c->kmix, s_out, c->err_dev,
                                    c->sm_count, st));
  if (c->max_squarings < 0) {
    LB_CUDA(cudaMemcpyAsync(c->scmax_host, c->sc + S, sizeof(int), cudaMemcpyDeviceToHost, st));
    LB_CUDA(cudaEventRecord(c->ev_scmax, st));
  } else {
    LB_CUDA(launch_check_bound(c->sc + S, c->max_squarings, c->err_dev, st));
  }
  if (ev) LB_CUDA(cudaEventRecord(ev[1], st));
  const long long max_nnz = (long long)(kSparseDensity * (double)nn);
  int* flagA = c->spflag;                     // A row-sparse
  int* flagA2 = c->spflag + c->max_slices;    // A^2 row-sparse
  if (prec == LB_FP64_SLICED) {
    // the sliced form: A^2 skips A's zeros (a local generator's A is about
    // 1 % nonzero); A^4, A^6 and the two products with A^6 are dense sliced
    // products (V and W start from their power terms and take A^6 Z1,
    // A^6 Z2 with beta = 1); U = A W is a dense sliced product.  With a
    // drive generator, A_s = c_s (G_base + u_s G_drv) and A_s^2 comes from
    // the three slice-independent products G_base^2, G_base G_drv + G_drv
    // G_base and G_drv^2 (zero-skipping, on the pattern of G_base and G_drv
    // together, found once by rows) and one pass over the slices.
    double *A2 = (double*)c->A2, *A4 = (double*)c->A4, *A6 = (double*)c->A6, *Z1 = (double*)c->Z1,
           *Z2 = (double*)c->Z2, *V = (double*)c->V, *W = (double*)c->W;
    const bool csr = Gd != nullptr;
    CsrPattern pat;
    pat.total = (unsigned long long*)c->csr;
    pat.rowbeg = c->csr + 2;
    pat.rowend = pat.rowbeg + c->max_n;
    pat.cols = pat.rowend + c->max_n;
    if (csr)
      LB_CUDA(launch_csr_union(n, Gb, Gd, max_nnz, S, pat, flagA, st));
    else
      LB_CUDA(launch_sparse_flags<double>(n, S, Ar, max_nnz, flagA, c->sm_count, st));
    auto sparse_left = [&](const RGemmProblem<double>& q) {
      return csr ? csr_product(c, q, flagA, pat, st) : skip_product(c, q, flagA, st);
    };
    if (csr) {
      double *P0 = Z1, *P1 = Z1 + nn, *P2 = Z2;  // free until the power terms
      LB_TRY(sparse_left(rsq(n, 1, Gb, Gb, P0)));
      LB_TRY(sparse_left(rsq(n, 1, Gb, Gd, P1)));
      RGemmProblem<double> p1 = rsq(n, 1, Gd, Gb, P1);
      p1.beta[0] = 1.0;
      LB_TRY(sparse_left(p1));
      LB_TRY(sparse_left(rsq(n, 1, Gd, Gd, P2)));
      LB_CUDA(launch_real_affine_square(n, S, P0, P1, P2, u, dt, c->sc, A2, c->sm_count, st));
    } else {
      LB_TRY(sparse_left(rsq(n, S, Ar, Ar, A2)));
    }
    // A^4 = A^2 A^2 then A^6 = A^2 A^4 (A^2 sliced once; A^4 is complete
    // before it is sliced as the second product's operand)
    LB_TRY(oz_product_shared_a(c, n, S, A2, A2, A4, 0.0, A4, A6, 0.0, nullptr, st));
    LB_CUDA(launch_real_pade_terms(n, S, A6, A4, A2, b, Z1, Z2, V, W, c->sm_count, st));
    // V += A^6 Z1, W += A^6 Z2 with A^6 sliced once
    LB_TRY(oz_product_shared_a(c, n, S, A6, Z1, V, 1.0, Z2, W, 1.0, nullptr, st));
    // U = A W as a sliced product (A W is dense), its epilogue forming
    // Mx = V - U and N = V + U (U itself not stored)
    OzGemm q;
    q.M = q.N = q.K = n;
    q.batch = S;
    q.A = Ar; q.a_sm = n; q.a_sk = 1; q.sA = nn;
    q.B = W; q.b_sk = n; q.b_sn = 1; q.sB = nn;
    q.C = nullptr; q.ldc = n; q.sC = nn;
    q.x.nx = 2;
    q.x.pm = 1;
    q.x.T1 = V;
    q.x.X[0] = Mx;
    q.x.X[1] = N;
    LB_TRY(oz_product(c, q, st));
  } else if (prec == LB_FP64_HERMITIAN) {
    double *A2 = (double*)c->A2, *A4 = (double*)c->A4, *A6 = (double*)c->A6, *Z1 = (double*)c->Z1,
           *Z2 = (double*)c->Z2, *V = (double*)c->V, *W = (double*)c->W;
    LB_CUDA(launch_sparse_flags<double>(n, S, Ar, max_nnz, flagA, c->sm_count, st));
    RGemmProblem<double> p = rsq(n, S, Ar, Ar, A2);
    LB_TRY(skip_product(c, p, flagA, st));
    LB_CUDA(launch_sparse_flags<double>(n, S, A2, max_nnz, flagA2, c->sm_count, st));
    p = rsq(n, S, A2, A2, A4);
    LB_TRY(skip_product(c, p, flagA2, st));
    // A6 = A2 A4 (powers of A commute: A2 is the sparser left operand), and
    // Z1 = b12 A6 + b10 A4 + b8 A2 from the same accumulators
    p = rsq(n, S, A2, A4, A6);
    p.O[1] = Z1;
    p.alpha[1] = b[12];
    p.nterms = 2;
    p.X[0] = A4; p.X[1] = A2;
    p.sX[0] = p.sX[1] = nn;
    p.coef[1][0] = b[10]; p.coef[1][1] = b[8];
    LB_TRY(skip_product(c, p, flagA2, st));
    LB_CUDA(launch_real_lincomb3<double>(nn * S, A6, A4, A2, b[13], b[11], b[9], Z2, c->sm_count, st));
    // slices with a sparse A^2: A^8, A^10, A^12 by three more zero-skipping
    // products with A^2 and V, W summed from the powers (the same
    // approximant, its polynomials summed term by term instead of through
    // the two dense products A^6 Z1, A^6 Z2); in the second halves of the
    // A^2 .. A^6 buffers
    {
      const size_t half = (size_t)c->max_slices * c->max_n * c->max_n;
      double *A8 = (double*)c->A2 + half, *A10 = (double*)c->A4 + half, *A12 = (double*)c->A6 + half;
      const double* lo[3] = {A6, A8, A10};
      double* hi[3] = {A8, A10, A12};
      for (int i = 0; i < 3; i++) {
        RGemmProblem<double> h = rsq(n, S, A2, lo[i], hi[i]);
        h.pick = flagA2;
        h.pick_val = 1;
        LB_CUDA(rgemm_rowskip(h, c->sm_count, st));
      }
      LB_CUDA(launch_real_powsum<double>(n, S, flagA2, A2, A4, A6, A8, A10, A12, b, 1, V, W, c->sm_count, st));
    }
    // other slices: V = A6 Z1 + b6 A6 + b4 A4 + b2 A2 + b0 I;  W = A6 Z2 + b7 A6 + b5 A4 + b3 A2 + b1 I
    RGemmProblem<double> vw[2];
    for (int i = 0; i < 2; i++) {
      vw[i] = rsq(n, S, A6, i == 0 ? Z1 : Z2, i == 0 ? V : W);
      vw[i].nterms = 3;
      vw[i].X[0] = A6; vw[i].X[1] = A4; vw[i].X[2] = A2;
      vw[i].sX[0] = vw[i].sX[1] = vw[i].sX[2] = nn;
      vw[i].pick = flagA2;
      vw[i].pick_val = 0;
    }
    vw[0].coef[0][0] = b[6]; vw[0].coef[0][1] = b[4]; vw[0].coef[0][2] = b[2]; vw[0].gamma[0] = b[0];
    vw[1].coef[0][0] = b[7]; vw[1].coef[0][1] = b[5]; vw[1].coef[0][2] = b[3]; vw[1].gamma[0] = b[1];
    LB_CUDA(rgemm_f64(vw, 2, c->sm_count, st));
    // U = A W:  Mx = V - U, N = V + U
    p = rsq(n, S, Ar, W, Mx);
    p.alpha[0] = -1.0;
    p.O[1] = N;
    p.nterms = 1;
    p.X[0] = V; p.sX[0] = nn;
    p.coef[0][0] = 1.0; p.coef[1][0] = 1.0;
    LB_TRY(skip_product(c, p, flagA, st));
  } else {
    // FP32 products (operands and accumulation in FP32), every intermediate
    // kept in FP32; the FP64 LU inputs V - U and V + U are widened with the
    // identity and b1 A added in FP64, so the FP32 rounding touches only the
    // O(A^2) parts.
    const long long fl = nn * S;
    float* f0 = (float*)c->Z2;
    float *Af = f0, *A2f = f0 + fl, *A4f = f0 + 2 * fl, *A6f = f0 + 3 * fl;
    float* f1 = (float*)c->W;
    float *Z1f = f1, *Z2f = f1 + fl, *Vsf = f1 + 2 * fl, *Wsf = f1 + 3 * fl;
    LB_CUDA(launch_real_to_f32(n, S, Ar, 0.0, Af, c->sm_count, st));
    LB_CUDA(launch_sparse_flags<float>(n, S, Af, max_nnz, flagA, c->sm_count, st));
    RGemmProblem<float> p = fsq(n, S, Af, Af, A2f);
    LB_TRY(skip_product(c, p, flagA, st));
    LB_CUDA(launch_sparse_flags<float>(n, S, A2f, max_nnz, flagA2, c->sm_count, st));
    p = fsq(n, S, A2f, A2f, A4f);
    LB_TRY(skip_product(c, p, flagA2, st));
    p = fsq(n, S, A2f, A4f, A6f);
    p.O[1] = Z1f;
    p.alpha[1] = b[12];
    p.nterms = 2;
    p.X[0] = A4f; p.X[1] = A2f;
    p.sX[0] = p.sX[1] = nn;
    p.coef[1][0] = b[10]; p.coef[1][1] = b[8];
    LB_TRY(skip_product(c, p, flagA2, st));
    LB_CUDA(launch_real_lincomb3<float>(fl, A6f, A4f, A2f, b[13], b[11], b[9], Z2f, c->sm_count, st));
    {  // sparse A^2: the higher powers and the power sums, as in the FP64 form (in V's buffer)
      float* f2 = (float*)c->V;
      float *A8f = f2, *A10f = f2 + fl, *A12f = f2 + 2 * fl;
      const float* lo[3] = {A6f, A8f, A10f};
      float* hi[3] = {A8f, A10f, A12f};
      for (int i = 0; i < 3; i++) {
        RGemmProblem<float> h = fsq(n, S, A2f, lo[i], hi[i]);
        h.pick = flagA2;
        h.pick_val = 1;
        LB_CUDA(rgemm_rowskip(h, c->sm_count, st));
      }
      LB_CUDA(launch_real_powsum<float>(n, S, flagA2, A2f, A4f, A6f, A8f, A10f, A12f, b, 0, Vsf, Wsf, c->sm_count,
                                        st));
    }
    RGemmProblem<float> vw[2];
    for (int i = 0; i < 2; i++) {
      vw[i] = fsq(n, S, A6f, i == 0 ? Z1f : Z2f, i == 0 ? Vsf : Wsf);
      vw[i].nterms = 3;
      vw[i].X[0] = A6f; vw[i].X[1] = A4f; vw[i].X[2] = A2f;
      vw[i].sX[0] = vw[i].sX[1] = vw[i].sX[2] = nn;
      vw[i].pick = flagA2;
      vw[i].pick_val = 0;
    }
    vw[0].coef[0][0] = b[6]; vw[0].coef[0][1] = b[4]; vw[0].coef[0][2] = b[2];
    vw[1].coef[0][0] = b[7]; vw[1].coef[0][1] = b[5]; vw[1].coef[0][2] = b[3];
    LB_CUDA(rgemm_f32(vw, 2, c->sm_count, st));
    // acc = A Ws:  V - U = b0 I + Vs - b1 A - acc,  V + U = b0 I + Vs + b1 A + acc
    p = fsq(n, S, Af, Wsf, nullptr);
    p.O[0] = nullptr;
    p.Od[0] = Mx; p.Od[1] = N;
    p.alpha[0] = -1.0; p.alpha[1] = 1.0;
    p.nterms = 1;
    p.X[0] = Vsf; p.sX[0] = nn;
    p.coef[0][0] = 1.0; p.coef[1][0] = 1.0;
    p.Xd = Ar; p.sXd = nn;
    p.dcoef[0] = -b[1]; p.dcoef[1] = b[1];
    p.dgamma[0] = b[0]; p.dgamma[1] = b[0];
    LB_TRY(skip_product(c, p, flagA, st));
  }
  if (ev) LB_CUDA(cudaEventRecord(ev[2], st));
  // (V - U) R = (V + U), FP64.  U, Y, L reuse A2, A4, A6.
  {
    lb_status r = prec == LB_FP64_SLICED
                      ? lu_solve_sliced_ll(c, n, S, Mx, N, (double*)c->A2, (double*)c->A4, (double*)c->A6,
                                           (double*)c->Z2, st)
                      : lu_solve_blocked_real(c, n, S, Mx, N, (double*)c->A2, (double*)c->A4, (double*)c->A6, st);
    if (r != LB_OK) return r;
  }
  if (ev) LB_CUDA(cudaEventRecord(ev[3], st));
  int smax = c->max_squarings;
  if (smax < 0) {
    LB_CUDA(cudaEventSynchronize(c->ev_scmax));
    smax = *c->scmax_host;
  }
  // squarings; in the FP32 form the leading ones, whose operand is still
  // near I (kmix[s] of them), run as R^2 = 2R - I + D D with D = R - I and
  // only D D in FP32; the rest are FP64
  for (int it = 0; it < smax && prec == LB_FP64_SLICED; it++) {
    // in place: both operands are sliced before R is overwritten, and the
    // slices whose squarings are done are skipped whole
    OzGemm q;
    q.M = q.N = q.K = n;
    q.batch = S;
    q.A = N; q.a_sm = n; q.a_sk = 1; q.sA = nn;
    q.B = N; q.b_sk = n; q.b_sn = 1; q.sB = nn;
    q.C = N; q.ldc = n; q.sC = nn;
    q.active = c->sc;
    q.active_iter = it;
    LB_TRY(oz_product(c, q, st));
  }
  for (int it = 0; it < smax && prec != LB_FP64_SLICED; it++) {
    RGemmProblem<double> q = rsq(n, S, N, N, T2);
    q.active = c->sc;
    q.active_iter = it;
    if (prec == LB_FP32_HERMITIAN) {
      float* Df = (float*)c->V;
      LB_CUDA(launch_real_to_f32(n, S, N, 1.0, Df, c->sm_count, st));
      RGemmProblem<float> m = fsq(n, S, Df, Df, nullptr);
      m.O[0] = nullptr;
      m.Od[0] = T2;
      m.Xd = N; m.sXd = nn;
      m.dcoef[0] = 2.0;
      m.dgamma[0] = -1.0;
      m.active = c->kmix;
      m.active_iter = it;
      LB_CUDA(rgemm_f32(&m, 1, c->sm_count, st));
      q.active_lo = c->kmix;
    }
    LB_CUDA(rgemm_f64(&q, 1, c->sm_count, st));
    LB_CUDA(launch_real_copy_active(nn, S, T2, N, c->sc, it, c->sm_count, st));
  }
  if (ev) LB_CUDA(cudaEventRecord(ev[4], st));
  LB_CUDA(launch_herm_to_complex(n, d, S, N, P, c->sm_count, st));
  LB_CUDA(launch_check_finite(nn * S, P, c->err_dev, st));
  if (ev) LB_CUDA(cudaEventRecord(ev[5], st));
  return LB_OK;
}

// FP64 propagation on the real coordinates for n > 81: the real matrices R_s
// of a chunk of slices (built from P), the states' coordinates in two
// ping-pong buffers, one real product per step (a few-state product for
// B <= 8), and the states written back exactly Hermitian.
lb_status propagate_herm_large(lb_ctx* c, int n, int nslices, const z64* P, int steps_per_slice, int B, z64* X,
                               bool sliced, cudaStream_t st) {
  int d = 1;
  while (d * d < n) d++;
  const long long nn = (long long)n * n;
  double* R = (double*)c->Z1;
  double* cur = (double*)c->Rtmp;
  double* nxt = cur + (long long)B * n;
  LB_CUDA(launch_herm_coords_in(n, d, B, X, cur, c->sm_count, st));
  sliced = sliced && B > kGemvMaxB;
  // sliced products: the slices of the chunk's R_s (B operands, narrow
  // tiles: a product has few output tiles) and of the states in the
  // context's scratch; chunks of at most max_slices slices that fit there
  const size_t xs_bytes = oz_sliced_bytes(B, n, 1, kOzTileM);
  int chunk = c->max_slices;
  while (sliced && chunk > 1 && xs_bytes + oz_sliced_bytes(n, n, chunk, kOzBNSmall) > c->oz_bytes) chunk = (chunk + 1) / 2;
  if (sliced && xs_bytes + oz_sliced_bytes(n, n, chunk, kOzBNSmall) > c->oz_bytes) return LB_EINVAL;
  for (int s0 = 0; s0 < nslices; s0 += chunk) {
    const int S = (nslices - s0 < chunk) ? nslices - s0 : chunk;
    LB_CUDA(launch_herm_matrix(n, d, S, P + s0 * nn, R, c->sm_count, st));
    OzSliced Rs, Xs;
    if (sliced) {
      Rs = oz_carve(c->oz_scratch, n, n, S, kOzBNSmall);
      Xs = oz_carve((uint8_t*)c->oz_scratch + oz_sliced_bytes(n, n, S, kOzBNSmall), B, n, 1, kOzTileM);
      LB_CUDA(oz_slice(R, n, 1, nn, Rs, nullptr, 0, st));  // row c of R_s = column c of R_s^T
    }
    for (int s = 0; s < S; s++)
      for (int t = 0; t < steps_per_slice; t++) {
        if (B <= kGemvMaxB) {
          LB_CUDA(launch_dgemv_f64(n, B, R + s * nn, n, cur, n, nxt, n, 1.0, nullptr, 0, st));
        } else if (sliced) {
          // next = cur R_s^T: the states in slices, then the product with the
          // slices of R_s made once for the chunk
          LB_CUDA(oz_slice(cur, n, 1, 0, Xs, nullptr, 0, st));
          OzGemm q;
          q.M = B; q.N = n; q.K = n;
          q.C = nxt; q.ldc = n;
          q.err = c->err_dev;
          cudaEvent_t e0 = nullptr, e1 = nullptr;
          LB_CUDA(kernel_events(c, 2.0 * kOzPairs * B * (double)n * n, &e0, &e1));
          LB_CUDA(oz_multiply(Xs, oz_view(Rs, s), q, c->sm_count, st, e0, e1));
        } else {
          // next[b][a] = sum_k R_s[a][k] cur[b][k]  ->  next = cur R_s^T
          RGemmProblem<double> q;
          q.M = B; q.N = n; q.K = n;
          q.A = cur; q.lda = n;
          q.B = R + s * nn; q.ldb = n; q.transB = 1;
          q.ldc = n;
          q.O[0] = nxt;
          LB_CUDA(rgemm_f64(&q, 1, c->sm_count, st));
        }
        double* tmp = cur;
        cur = nxt;
        nxt = tmp;
      }
  }
  LB_CUDA(launch_herm_coords_out(n, d, B, cur, X, c->sm_count, st));
  return LB_OK;
}

}  // namespace lb

extern "C" lb_status lb_gemm_f64_sliced(lb_ctx* c, int M, int N, int K, int batch, const double* A, long long lda,
                                        long long sA, const double* B, long long ldb, long long sB, double* C,
                                        long long ldc, long long sC, double alpha, double beta, void* stream) {
  using namespace lb;
  if (c == nullptr || A == nullptr || B == nullptr || C == nullptr) return LB_EINVAL;
  if (M < 0 || N < 0 || batch < 0 || K < 1 || K > kOzMaxK) return LB_EINVAL;
  if (lda < K || ldb < N || ldc < N) return LB_EINVAL;
  if (M == 0 || N == 0 || batch == 0) return LB_OK;
  DeviceGuard g(c->device);
  OzGemm q;
  q.M = M; q.N = N; q.K = K; q.batch = batch;
  q.A = A; q.a_sm = lda; q.a_sk = 1; q.sA = sA;
  q.B = B; q.b_sk = ldb; q.b_sn = 1; q.sB = sB;
  q.C = C; q.ldc = ldc; q.sC = sC;
  q.alpha = alpha;
  q.beta = beta;
  return oz_product(c, q, (cudaStream_t)stream);
}
