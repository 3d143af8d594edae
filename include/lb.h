/*
 * lb.h -- C ABI of the GB300 (sm_103a) library for dense small-d Lindblad
 * propagation.
 *
 * The operations follow arXiv 2603.18052 ("Hardware-Aware Performance
 * Characterization of Small Dense Lindblad Propagation for Near-Term Quantum
 * Control"): the vectorised Lindbladian of Eq. 1-3, the segment generator of
 * Eq. 5, the Pade [13/13] scaling-and-squaring propagator build of
 * Algorithm 1 and the propagation step of Algorithm 2, batched over states as
 * in Algorithm 3, plus the gradient of a piecewise-constant control
 * (Sec. 2.5).
 *
 * Conventions shared by every call
 *  - Complex numbers are interleaved (re, im) doubles, the layout of
 *    torch.complex128 and of C99 double complex.
 *  - Matrices are dense and row-major.  A d x d density matrix is stored as
 *    its row-major n-vector, n = d*d (Sec. 3.2: the d x d array is the
 *    vector), so a batch of B states is a B x n row-major array.
 *  - Every array argument is DEVICE memory owned by the caller, on the device
 *    the context was created for, unless stated otherwise.  The library never
 *    frees or keeps caller pointers after a call returns.
 *  - All scratch memory is owned by the context and allocated in lb_create
 *    only; the compute calls allocate nothing.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream).  Argument errors are detected on the host and returned
 *    before anything is launched.  Numerical faults found on the device
 *    (non-finite values, a zero pivot) are recorded in the context's error
 *    word; lb_sync_status synchronises the stream and reports them.
 *  - Calls on one context must not run concurrently (they share scratch).
 */
#ifndef LB_H
#define LB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LB_OK = 0,
  LB_EINVAL = 1,        /* bad argument (null pointer, size out of range) */
  LB_ENODEV = 2,        /* no CUDA device, or the device is not sm_103 */
  LB_ENOMEM = 3,        /* device allocation failed in lb_create */
  LB_ECUDA = 4,         /* a CUDA runtime call or launch failed */
  LB_ENONFINITE = 5,    /* NaN or Inf met on the device */
  LB_ESINGULAR = 6,     /* zero pivot in the LU factorisation */
  LB_ETIMEOUT = 7,      /* a bounded device-side wait gave up */
  LB_EUNSUPPORTED = 8   /* valid request outside what this build supports */
} lb_status;

typedef enum {
  LB_FP64 = 0,    /* every product in FP64 */
  LB_FP32 = 1,    /* products in FP32 with FP32 accumulation */
  LB_BF16X3 = 2,  /* products as split-BF16 x3 on the tensor cores, FP32 accumulation */
  LB_FP64_HERMITIAN = 3, /* FP64 on the n real coordinates of Hermitian matrices: for
                            Hermiticity-preserving generators and propagators (every
                            Lindbladian and its exponential are); see lb_expm_pade and
                            lb_propagate_batch */
  LB_FP32_HERMITIAN = 4, /* lb_expm_pade: the real-coordinate build with FP32 Pade
                            products; lb_propagate_batch: the same as LB_FP32 */
  LB_FP64_SLICED = 5     /* LB_FP64_HERMITIAN with the dense FP64 products (squarings,
                            propagation steps) on the BF16 tensor cores through exact
                            slices (Ozaki scheme, see lb_gemm_f64_sliced): FP64
                            operands and results, error of the size of an FP64
                            product's rounding */
} lb_precision;

typedef struct lb_ctx lb_ctx;

typedef struct {
  double re, im;
} lb_c64;

/* Library version (major*10000 + minor*100 + patch). */
int lb_version(void);

/* Human-readable name of a status code.  Never NULL. */
const char* lb_status_str(int status);

/*
 * lb_create: bind a context to CUDA device `device` and allocate its scratch
 * for problems up to n = max_n (at most 729), max_batch states and
 * max_slices propagators per call.  Larger slice counts are processed in
 * chunks of max_slices.  *ctx receives the context (NULL on error).
 * Returns LB_ENODEV without a usable sm_103 device, LB_ENOMEM if the scratch
 * does not fit.
 */
lb_status lb_create(lb_ctx** ctx, int device, int max_n, int max_batch, int max_slices);

/* Release the context and its scratch.  NULL is accepted. */
lb_status lb_destroy(lb_ctx* ctx);

/*
 * Synchronise `stream`, then report (and clear) the device error word:
 * LB_ENONFINITE, LB_ESINGULAR, LB_ETIMEOUT, or LB_EUNSUPPORTED (a squaring
 * count above the bound of lb_set_max_squarings), else LB_OK.  A CUDA error met
 * while synchronising gives LB_ECUDA.
 */
lb_status lb_sync_status(lb_ctx* ctx, void* stream);

/*
 * lb_set_max_squarings: with bound >= 0, every later lb_expm_pade and
 * lb_run_instances runs exactly `bound` masked squaring rounds (slices that
 * need fewer skip the extra ones on the device) instead of reading the
 * largest squaring count back to the host.  This makes those calls free of
 * host waits, so they can be captured in a CUDA graph.  A slice that needs
 * more than `bound` squarings sets the error word: lb_sync_status then
 * returns LB_EUNSUPPORTED (and that slice's P is not valid).  bound < 0
 * restores the default.  Without a bound, lb_expm_pade and
 * lb_run_instances return LB_EUNSUPPORTED when the stream is capturing.
 * While capturing lb_run_instances, its tables are uploaded from the
 * context's pinned staging buffer when the graph runs: do not replay such a
 * graph after another lb_run_instances call on the same context.  Limits:
 * bound <= 64.
 */
lb_status lb_set_max_squarings(lb_ctx* ctx, int bound);

/*
 * lb_autotune: choose the GEMM tile configuration for every launch shape of
 * an n-sized propagator build over nslices slices (its LU updates, back
 * substitution and FP32 products) and of a B-state FP64 propagation step:
 * each such launch is run once per candidate configuration on the context's
 * scratch, timed with CUDA events, and the fastest is recorded in a
 * process-wide table that later calls of the same shape use (other shapes
 * keep the tile-count rule).  Synchronises `stream`; takes a few seconds for
 * n = 729 and 200 slices; must not be called while capturing.
 * *shapes_out (may be NULL) receives the number of recorded shapes.
 */
lb_status lb_autotune(lb_ctx* ctx, int n, int nslices, int B, int* shapes_out, void* stream);

/* Bytes of device scratch owned by the context. */
unsigned long long lb_workspace_bytes(const lb_ctx* ctx);

/* Number of kernel launches the library has issued in this process (all
 * contexts).  For accounting in benchmarks. */
unsigned long long lb_launch_count(void);

/*
 * Stage timers of lb_expm_pade, following the stages of Algorithm 1 (the
 * paper's build-time breakdown).  lb_set_stage_timing(ctx, 1) clears the
 * totals and makes every later lb_expm_pade record CUDA events on its stream
 * around each stage, without synchronising (a ring of 16 event sets; the
 * host waits only when more than 16 chunks of slices are in flight).
 * lb_stage_times waits for the recorded events and returns in ms_out (host,
 * 5 doubles) the totals since the last lb_set_stage_timing call:
 *   ms_out[0] generator, 1-norm, squaring count and scaling
 *   ms_out[1] the six Pade products (three powers, V, W, U)
 *   ms_out[2] LU factorisation and solve of (V - U) P = (V + U)
 *   ms_out[3] squarings
 *   ms_out[4] final non-finite check
 * and in *chunks_out (may be NULL) the number of slice chunks timed.
 */
lb_status lb_set_stage_timing(lb_ctx* ctx, int enable);
lb_status lb_stage_times(lb_ctx* ctx, double* ms_out, long long* chunks_out);

/*
 * lb_kernel_times -- with the stage timers on (lb_set_stage_timing), every
 * launch of the sliced FP64 product kernel (LB_FP64_SLICED; launches with a
 * per-slice mask, the squarings, excepted) is bracketed by CUDA events on
 * its stream.  Waits for them and returns since the last
 * lb_set_stage_timing: *ms_out the summed kernel time (ms), *flops_out its
 * digit-product FLOPs (45 BF16 products per multiply-add: 90 M N K per
 * product; may be NULL), *launches_out the launches (may be NULL).
 */
lb_status lb_kernel_times(lb_ctx* ctx, double* ms_out, double* flops_out, long long* launches_out);

/*
 * lb_assemble -- the vectorised Lindbladian of Eq. 1 under row-major vec
 * (Eq. 2-3):
 *   L = -i (H (x) I - I (x) H^T)
 *       + sum_k [ L_k (x) conj(L_k) - 1/2 (L_k^+ L_k) (x) I - 1/2 I (x) (L_k^+ L_k)^T ]
 *   H      : d x d (Hermitian in physical use; not checked)
 *   Ls     : K x d x d jump operators, contiguous; may be NULL when K == 0
 *   L_out  : n x n, n = d*d, fully overwritten
 * The drive generator of Eq. 5 is lb_assemble(X, K = 0).
 * Limits: 1 <= d, d*d <= max_n; 0 <= K <= 64.
 */
lb_status lb_assemble(lb_ctx* ctx, int d, const lb_c64* H, int K, const lb_c64* Ls,
                      lb_c64* L_out, void* stream);

/*
 * lb_expm_pade -- P[s] = exp(A_s), A_s = (Lbase + u[s] * Ldrv) * dt, for
 * s < nslices (Eq. 5 and Algorithm 1 with theta = 0.25):
 *   sc = max(0, ceil(log2(||A_s||_1 / theta))), ||.||_1 the maximum absolute
 *   column sum; A = A_s / 2^sc; the three power products and three U/V
 *   products of the [13/13] approximant; P from (V - U) P = (V + U) by an
 *   FP64 LU factorisation and forward/back substitution; sc FP64 squarings.
 *   Lbase : n x n; if Ldrv == NULL, Lbase holds nslices generators
 *           (nslices x n x n) and u is ignored (may be NULL)
 *   Ldrv  : n x n or NULL
 *   u     : nslices doubles (device)
 *   prec  : precision of the six Pade products; LU, solve and squarings are
 *           always FP64 (in the reduced forms a leading squaring whose operand
 *           is still near I runs as P^2 = 2P - I + D D, D = P - I, with only
 *           D D in the reduced precision)
 *           LB_FP64_HERMITIAN / LB_FP32_HERMITIAN: the whole of Algorithm 1
 *           on the n = d^2 real coordinates of Hermitian matrices (diagonal,
 *           then Re and Im of the upper triangle, row-major), where L dt and
 *           exp(L dt) are real n x n matrices G and R: the generators must
 *           map Hermitian matrices to Hermitian matrices (every Lindbladian
 *           and every drive term -i[X, .] with X Hermitian does; for others
 *           the result is not exp(A)); sc is taken from ||G||_1; every
 *           product, the LU and the solve are real (one FMA per multiply-
 *           add instead of four); P is rebuilt from R at the end.  The FP32
 *           variant runs the six Pade products and the near-I squarings in
 *           FP32; LU, solve and the other squarings stay FP64.  n must be a
 *           square (else LB_EINVAL).
 *           LB_FP64_SLICED: LB_FP64_HERMITIAN with the squarings as sliced
 *           FP64 products (lb_gemm_f64_sliced) for n > 81.
 *   P_out : nslices x n x n
 *   s_out : nslices ints (device) receiving sc, or NULL
 * The LU takes no pivots: at theta = 0.25 the matrix V - U is strictly
 * column diagonally dominant, for which partial pivoting selects the
 * diagonal at every step.  A pivot of modulus below 1e-300 sets
 * LB_ESINGULAR in the error word.
 */
lb_status lb_expm_pade(lb_ctx* ctx, int n, int nslices, const lb_c64* Lbase, const lb_c64* Ldrv,
                       const double* u, double dt, lb_precision prec, lb_c64* P_out, int* s_out,
                       void* stream);

/*
 * lb_propagate_batch -- chained propagation steps rho <- P rho (Algorithm 2)
 * for B states sharing the propagators (Algorithm 3's batch):
 *   step t = 0 .. nslices*steps_per_slice - 1 uses P[t / steps_per_slice].
 *   P      : nslices x n x n (FP64, as written by lb_expm_pade)
 *   states : B x n, read as the initial states and overwritten with the
 *            final ones
 *   prec   : LB_FP64 computes in FP64.  LB_FP32 and LB_BF16X3 store
 *            D = P - I in the lower precision, keep the states in FP32,
 *            and apply rho + D rho with FP32 accumulation; the result is
 *            written back as complex128.
 *   renorm_trace : if nonzero and prec != LB_FP64, divide every state by
 *            its trace (sum of entries i*d + i) after each step.
 * Limits: n a perfect square, n <= max_n; 1 <= B <= max_batch.
  *   prec = LB_FP64_HERMITIAN: the states must be Hermitian (each read from
 *   its diagonal real parts and upper triangle) and P must map Hermitian
 *   matrices to Hermitian matrices; the step then runs on the n real
 *   coordinates of each state (n^2 real multiply-adds instead of 4 n^2) and
 *   the states come back exactly Hermitian.  Same result as LB_FP64 up to
 *   rounding for such inputs.  n <= 9: one warp per state, the state
 *   exchanged by shuffles; 9 < n <= 81: the real transfer matrix and each
 *   CTA's states in shared memory; n > 81: one real product per step over
 *   all states (a few-state product for B <= 8) with the real transfer
 *   matrices of up to max_slices slices in the context's scratch.
 *   renorm_trace is ignored, as for LB_FP64.
 *   prec = LB_FP32_HERMITIAN runs the LB_FP32 form.
 *   prec = LB_FP64_SLICED: LB_FP64_HERMITIAN with the per-step real product
 *   for n > 81 and B > 8 as a sliced FP64 product (lb_gemm_f64_sliced).
 */
lb_status lb_propagate_batch(lb_ctx* ctx, int n, int nslices, const lb_c64* P, int steps_per_slice,
                             int B, lb_c64* states, lb_precision prec, int renorm_trace,
                             void* stream);

/*
 * lb_gemm_f64_sliced -- C = alpha A B + beta C for a batch of real FP64
 * matrices, computed on the BF16 tensor cores through exact slices (the
 * Ozaki scheme: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012).  The
 * building block of the LB_FP64_SLICED form (the dense products of Algorithm
 * 1's squarings and Algorithm 2's steps on the real coordinates); the paper
 * computes these products in FP64, which this reproduces to the size of an
 * FP64 product's rounding.  Each row of A and each column of B is written as
 * nine signed base-64 digits against its own power-of-two exponent; the
 * digit products of equal weight are summed exactly in FP32 on the tensor
 * cores and combined in integer arithmetic; the one rounding is to FP64.
 * Error: |C - A B| <= K 2^(e_r + f_c) 2^-54 (13/4) for row r, column c,
 * where 2^e_r > max_k |A[r][k]| and 2^f_c > max_k |B[k][c]|.
 *   A : batch x M x K, row-major, leading dimension lda, batch stride sA
 *   B : batch x K x N, row-major, ldb, sB
 *   C : batch x M x N, row-major, ldc, sC (may alias A or B: both are
 *       consumed before C is written)
 * All pointers device memory owned by the caller; 1 <= K <= 1488 (else
 * LB_EINVAL); the batch is processed in chunks that fit the context's
 * scratch.  Non-finite inputs give unspecified results.
 */
lb_status lb_gemm_f64_sliced(lb_ctx* ctx, int M, int N, int K, int batch, const double* A, long long lda,
                             long long sA, const double* B, long long ldb, long long sB, double* C, long long ldc,
                             long long sC, double alpha, double beta, void* stream);

/*
 * lb_grape_grad -- fidelity of a piecewise-constant control and its gradient
 * (Sec. 2.5 landscape point, Eq. 5 segment generator):
 *   P_s = exp((Lbase + u[s] Ldrv) dt), applied steps_per_slice times per
 *   slice; X_T = chain applied to each of the B rows of X0;
 *   F = Re sum_b <Xt_b, X_T,b> / B, <a, b> = sum_i conj(a_i) b_i;
 *   grad[s] = dF/du[s] = sum over the steps t of slice s of
 *             Re <Lam_t, dP_s X_{t-1}> / B,
 *   with the adjoint chain Lam_T = Xt, Lam_{t-1} = P^+ Lam_t and dP_s the
 *   Frechet derivative of exp at (Lbase + u[s] Ldrv) dt in the direction
 *   Ldrv dt, obtained by differentiating the Pade approximant and the
 *   squarings.  All FP64.
 *   X0, Xtarget : B x n
 *   fidelity_out: 1 double (device); grad_out: nslices doubles (device)
 * Limits: the context must have been created with max_n <= 81 (its GRAPE
 * scratch is sized then); n <= max_n; B <= min(max_batch, 64);
 * nslices <= max_slices; steps_per_slice <= 20.  Other sizes return
 * LB_EUNSUPPORTED.  The call waits on the host for the small copy of the
 * largest squaring count (made right after the norm kernel).
 */
lb_status lb_grape_grad(lb_ctx* ctx, int n, int nslices, const lb_c64* Lbase, const lb_c64* Ldrv,
                        const double* u, double dt, int steps_per_slice, int B, const lb_c64* X0,
                        const lb_c64* Xtarget, double* fidelity_out, double* grad_out,
                        void* stream);

/*
 * lb_grape_grad_batch -- lb_grape_grad for K independent problems in one
 * call (the many GRAPE optimisations of a training set for the warm-start
 * network, Sec. 2.5):
 *   problem k has the base generator Lbase + k * lbase_stride (n x n;
 *   lbase_stride = 0 shares one, else lbase_stride >= n*n), the shared
 *   drive generator Ldrv, the controls u[k * nslices + s], the start and
 *   target operators X0[k], Xtarget[k] (B x n each, stored one problem after
 *   another); fidelity_out[k] and grad_out[k * nslices + s] are that
 *   problem's F and dF/du[s] as lb_grape_grad defines them.
 *   prec = LB_FP64: exactly the arithmetic of lb_grape_grad.  LB_FP32: the
 *   Pade products and their derivatives in FP32 (FP32 operands and
 *   accumulation); LU, solve, squarings, chains and reductions FP64.
 * Limits: as lb_grape_grad, and K * nslices <= max_slices,
 * K * B <= max_batch, K <= 65535 (LB_EUNSUPPORTED beyond).  Reads the largest
 * squaring count back to the host (not capturable).
 */
lb_status lb_grape_grad_batch(lb_ctx* ctx, int n, int K, int nslices, const lb_c64* Lbase, long long lbase_stride,
                              const lb_c64* Ldrv, const double* u, double dt, int steps_per_slice, int B,
                              const lb_c64* X0, const lb_c64* Xtarget, lb_precision prec, double* fidelity_out,
                              double* grad_out, void* stream);

/*
 * lb_run_instances -- many independent problems of mixed size in one call:
 * for every instance i, its slice propagators
 *   P_{i,s} = exp((Lbase_i + u_i[s] Ldrv_i) dt)      (Eq. 5, Algorithm 1)
 * are built and its B_i states are propagated through its slices, each slice
 * applied steps_per_slice times (Algorithm 2); states are overwritten.
 * Instances are grouped by n = d*d and packed into chunks of whole instances
 * of at most max_slices slices; each chunk's propagators are built in one
 * batched pass, and for n <= 81 one launch propagates every instance of the
 * chunk (one CTA per instance and group of up to 8 states).
 *   inst  : HOST array of count descriptors; the pointers in it are device
 *           memory (n x n generators, nslices controls, B x n states)
 *   prec  : precision of the Pade products and of the propagation, as in
 *           lb_expm_pade and lb_propagate_batch (for n <= 81 the reduced
 *           forms propagate in FP32 with D = P - I; the Hermitian forms build
 *           on the real coordinates, LB_FP64_HERMITIAN and LB_FP64_SLICED
 *           propagate n <= 81 in complex FP64 and n > 81 on the real
 *           coordinates (LB_FP64_SLICED with sliced products),
 *           LB_FP32_HERMITIAN propagates in FP32)
 *   renorm_trace : as in lb_propagate_batch (reduced forms only)
 * Limits: n <= max_n; nslices <= max_slices per instance; for n > 81,
 * B <= max_batch; at most 262144 slices and 262144 state groups per call
 * (LB_EUNSUPPORTED beyond).  The host waits on the upload of the previous
 * call's tables and on the squaring count of each chunk.
 */
typedef struct {
  int d, nslices, steps_per_slice, B;
  const lb_c64* Lbase;
  const lb_c64* Ldrv;
  const double* u;
  lb_c64* states;
} lb_instance;

lb_status lb_run_instances(lb_ctx* ctx, const lb_instance* inst, int count, double dt, lb_precision prec,
                           int renorm_trace, void* stream);

/*
 * Warm-start network (GRAPE application of Sec. 2.5): a dense MLP with ReLU
 * hidden layers and a linear output layer, BF16 weights and FP32
 * accumulation.  Layer l maps dims[l] -> dims[l+1] (dims: HOST array of
 * nlayers + 1 ints); its weights W_l (dims[l+1] x dims[l], row-major, BF16)
 * and biases b_l (FP32) are packed back to back in W and b.  All arrays are
 * device memory, row-major, batch rows.
 *   lb_mlp_forward : acts (batch x sum_{l>=1} dims[l]) receives every layer's
 *                    output, hidden layers after the ReLU; the last block is
 *                    the network output.
 *   lb_mlp_backward: from dy = dLoss/doutput (batch x dims[nlayers]) writes
 *                    gW (FP32, packed like W) and gb; scratch holds
 *                    2 * batch * max(dims) floats.
 *   lb_mse_loss_grad: dy = 2 (y - t) / count and *loss = mean (y - t)^2
 *                    (loss may be NULL).
 *   lb_adam_step   : Adam with bias correction on FP32 parameters; p_bf16
 *                    (optional) receives the BF16 copy used by the forward.
 *   lb_adam_step_f64: the same on FP64 parameters; ascend != 0 maximises.
 * These allocate nothing and return LB_EINVAL for bad sizes or pointers.
 */
lb_status lb_mlp_forward(int nlayers, const int* dims, int batch, const void* W, const float* b, const float* x,
                         float* acts, void* stream);
lb_status lb_mlp_backward(int nlayers, const int* dims, int batch, const void* W, const float* x, const float* acts,
                          const float* dy, float* gW, float* gb, float* scratch, void* stream);
lb_status lb_mse_loss_grad(long long count, const float* y, const float* t, float* dy, float* loss, void* stream);
lb_status lb_adam_step(long long count, float* p, const float* g, float* m, float* v, void* p_bf16, float lr,
                       float beta1, float beta2, float eps, int step, void* stream);
lb_status lb_adam_step_f64(long long count, double* p, const double* g, double* m, double* v, double lr,
                           double beta1, double beta2, double eps, int step, int ascend, void* stream);

/*
 * lb_expm_frechet -- slice propagators and their control derivatives (the
 * reuse of P for nearby controls recommended in the paper's discussion, Sec.
 * 5, built on the differentiated Pade build of lb_grape_grad, Sec. 2.5):
 *   P_out[s]  = exp(A_s),  A_s = (Lbase + u[s] Ldrv) dt             (Alg. 1)
 *   dP_out[s] = d/du exp((Lbase + u Ldrv) dt) at u = u[s], the Frechet
 *               derivative of exp at A_s in the direction Ldrv dt.
 *   FP64.  Lbase, Ldrv: n x n; u: nslices doubles; P_out, dP_out:
 *   nslices x n x n complex128, row-major, caller-owned device memory.
 *   Contexts with max_n <= 81 (the GRAPE workspace); nslices <= max_slices.
 *   Reads the largest squaring count back to the host, so it cannot be
 *   captured in a CUDA graph (LB_EUNSUPPORTED while capturing).
 *   Errors: LB_EINVAL (null pointer, bad size, non-finite dt),
 *   LB_EUNSUPPORTED (context too large, too many slices, capture).
 */
lb_status lb_expm_frechet(lb_ctx* ctx, int n, int nslices, const lb_c64* Lbase, const lb_c64* Ldrv,
                          const double* u, double dt, lb_c64* P_out, lb_c64* dP_out, void* stream);

/*
 * lb_control_update -- first-order update of slice propagators for changed
 * controls, P_out[s] = P[s] + delta[s] dP[s] (FP64), with dP from
 * lb_expm_frechet; its error against a rebuild at u + delta is second order
 * in delta.  n x n x nslices complex128 arrays, delta: nslices doubles, all
 * device memory on the current device; P_out may alias P.  No context.
 *   Errors: LB_EINVAL (null pointer, n < 1); LB_ECUDA (launch failure).
 */
lb_status lb_control_update(int n, int nslices, const lb_c64* P, const lb_c64* dP, const double* delta,
                            lb_c64* P_out, void* stream);

/*
 * lb_propagate_batch_static -- the FP64 form of lb_propagate_batch for
 * callers that cannot allocate device memory.  The paper has no counterpart;
 * this exists for applications whose device memory is already owned by their
 * own allocator, and for loops that must not risk the device-wide
 * synchronisation and unbounded latency of cudaMalloc.  It needs no lb_ctx,
 * allocates nothing (no cudaMalloc, cudaFree or allocating library call),
 * and runs on the CURRENT CUDA device, which must hold P and states.
 *   Same arguments and results as lb_propagate_batch with prec = LB_FP64:
 *   step t uses P[t / steps_per_slice]; states (B x n) are overwritten.
 *   Limit: B * n <= 262144 (4 MiB of complex128); larger requests return
 *   LB_EUNSUPPORTED before any work is queued.
 *   The intermediate states live in one 4 MiB array in device memory that
 *   the library reserves on every GPU where its device code is loaded, kept
 *   until the process exits.  All calls share it: two calls running on the
 *   GPU at the same time (different streams or threads) race and must be
 *   serialised by the caller.  Nothing in it needs clearing between calls.
 *   The first call on each device looks up the array's device address (which
 *   can load the library's device code on that device); make that first call
 *   before any stream capture.  The address is kept for the life of the
 *   process: do not use this entry point after a cudaDeviceReset of that
 *   device.  P and states must be device (or managed) memory of the current
 *   device, else LB_EINVAL.
 */
lb_status lb_propagate_batch_static(int n, int nslices, const lb_c64* P, int steps_per_slice, int B,
                                    lb_c64* states, void* stream);

/*
 * lb_selftest_wait_timeout -- failure-detection self test (the paper has no
 * counterpart).  Queues one CTA on `stream` whose thread waits on a
 * shared-memory mbarrier that nothing ever completes, the same bounded wait
 * the tensor-core kernels use, for at most `cycles` SM clock cycles
 * (clamped to [1e3, 4e9]; 2e6 is about 1 ms).  The wait gives up, sets the
 * timeout bit of the context's device error word and the kernel returns;
 * nothing faults or hangs.  The next lb_sync_status returns LB_ETIMEOUT and
 * clears the word, after which the context is usable as before.
 *   Errors: LB_EINVAL for a null ctx; LB_ECUDA if the launch fails.
 */
lb_status lb_selftest_wait_timeout(lb_ctx* ctx, long long cycles, void* stream);

/*
 * lb_expmv -- the states through the control slices WITHOUT forming the
 * propagators (the action-of-the-exponential route that the paper's
 * discussion, Sec. 5, names for removing the LU solve; Al-Mohy and Higham's
 * truncated Taylor series with scaling):
 *     for s = 0 .. nslices-1:  X <- exp(A_s) X,  A_s = (Lbase + u[s] Ldrv) dt
 * with each state a row of X (as in lb_propagate_batch).  exp(A_s) x is the
 * sum of s_sub sub-steps of the degree-m Taylor series; one pair (m, s_sub)
 * serves the whole call, the one with the fewest products m * s_sub such
 * that a / s_sub <= theta_m, where a is the largest ||A_s||_1 (maximum
 * absolute column sum) of the call and theta_m the largest theta with
 * theta^(m+1)/(m+1)! e^theta <= 2^-53 (1 <= m <= 55).  FP64 throughout.
 *   n:       <= ctx max_n (any n; not only squares).
 *   Lbase, Ldrv, u: as lb_expm_pade (device): Ldrv = NULL means Lbase holds
 *            nslices generators and u is ignored.
 *   dt:      finite slice length.
 *   B:       1 .. ctx max_batch states in `states` (B x n complex128,
 *            device), overwritten.
 *   ms_out:  NULL or host int[2] receiving (m, s_sub).
 *   Reads the largest norm back to the host (the stream is synchronised
 *   once), so it cannot be captured in a CUDA graph (LB_EUNSUPPORTED when
 *   the stream is capturing).  Uses the context's build and state scratch.
 *   Errors: LB_EINVAL for bad arguments; LB_ENONFINITE for a NaN or Inf in
 *   a generator; LB_EUNSUPPORTED if more than 65536 sub-steps would be
 *   needed; LB_ECUDA for a failed launch.
 */
lb_status lb_expmv(lb_ctx* ctx, int n, int nslices, const lb_c64* Lbase, const lb_c64* Ldrv, const double* u,
                   double dt, int B, lb_c64* states, int* ms_out, void* stream);

/*
 * lb_expmv_hermitian -- lb_expmv for density matrices: the same route on the
 * n = d^2 real coordinates of Hermitian states (diagonal, Re and Im of the
 * upper triangle), where each generator A_s is a real n x n matrix G_s and
 * every Taylor term a real product (a quarter of the FP64 multiply-adds).
 * (m, s_sub) follows lb_expmv's rule with a = the largest ||G_s||_1.
 *   Same arguments as lb_expmv; n must be a square.  The states must be
 *   Hermitian (each is read from its diagonal real parts and upper
 *   triangle) and come back exactly Hermitian.  B <= 8 (the few-state
 *   product); larger B run lb_expmv.  Same errors as lb_expmv.
 */
lb_status lb_expmv_hermitian(lb_ctx* ctx, int n, int nslices, const lb_c64* Lbase, const lb_c64* Ldrv,
                             const double* u, double dt, int B, lb_c64* states, int* ms_out, void* stream);

/* ------------------------------------------------------------------------
 * Fixed-point propagation: the element-serial Q1.15 step of the FPGA design
 * (Algorithm alg:fpga, Sec. 3.5; formats Sec. 2.2) and its Q1.31 variant
 * (Figure fig:fixed_point_drift), bit-exact.  No lb_ctx: these run on the
 * CURRENT CUDA device (sm_103 only, else LB_ENODEV), which must hold every
 * pointer passed.  Asynchronous on `stream`; they allocate nothing.
 *
 * Codes: frac_bits = 15 or 31 (else LB_EINVAL).  A Q1.f complex value is a
 * pair (re, im) of two's-complement codes standing for code / 2^f: two
 * int16 (4 bytes per complex value) for f = 15, two int32 (8 bytes) for
 * f = 31, re first.  A state is the row-major vectorisation of rho
 * (n = d^2 values); B states are stored one after another.
 * ------------------------------------------------------------------------ */

/*
 * lb_fixed_quantize -- q[e] = nearest code of x[e] (x * 2^f rounded to the
 * nearest integer, ties to even), saturated to [-2^f, 2^f - 1], real and
 * imaginary parts separately; so 1.0 becomes 2^f - 1.  NaN becomes 0.
 *   count complex128 values in x (device), count code pairs out in q
 *   (device).  count = 0 does nothing.  LB_EINVAL for count < 0 or a null
 *   pointer with count > 0.
 */
lb_status lb_fixed_quantize(int frac_bits, long long count, const lb_c64* x, void* q, void* stream);

/*
 * lb_fixed_dequantize -- x[e] = q[e] / 2^f (exact in double).  Same
 * argument rules as lb_fixed_quantize.
 */
lb_status lb_fixed_dequantize(int frac_bits, long long count, const void* q, lb_c64* x, void* stream);

/*
 * lb_propagate_fixed -- nsteps chained steps of Algorithm alg:fpga on each
 * of B states with one propagator:
 *     acc_i = sum_j P[i][j] rho_j            (exact: four integer products
 *                                             per term, 64-bit sums for
 *                                             Q1.15, 128-bit for Q1.31)
 *     rho_i <- sat(floor(acc_i / 2^f))       (floor = towards -infinity,
 *                                             sat = clamp to the code range)
 *   n:        d^2 with 1 <= n <= 81 (P is held in shared memory).
 *   P_q:      n x n code pairs, row-major, row i produces output i (device).
 *   nsteps:   >= 0; 0 does nothing.
 *   B:        >= 1 states in states_q (B x n code pairs, device), overwritten
 *             with the states after nsteps steps.
 *   Errors: LB_EINVAL for an unsupported frac_bits, n, nsteps < 0, B < 1 or
 *   a null pointer; LB_ECUDA if the launch fails.
 */
lb_status lb_propagate_fixed(int frac_bits, int n, const void* P_q, int nsteps, int B, void* states_q,
                             void* stream);

/* ------------------------------------------------------------------------
 * The three GPU timing models of Sec. 3.4 (Eq. 7-9) and the device probes
 * behind their constants (Table tab:probes_gpu).  Kernel-only timing is
 * lb_propagate_batch with one step; the two calls below add what Eq. 8 and
 * Eq. 9 add to it.
 * ------------------------------------------------------------------------ */

/*
 * lb_propagate_resident -- resident-P timing model (Eq. 8): one FP64
 * propagation step (P = one n x n propagator, device) of B states that live
 * in HOST memory (B x n complex128, pageable or pinned): copies them to the
 * context's device buffer, runs the same step as lb_propagate_batch with
 * prec = LB_FP64, copies the result back into states_host and synchronises
 * `stream` before returning.
 *   Errors: LB_EINVAL for a null argument, n not a square in [1, max_n] or
 *   B outside [1, max_batch]; LB_ECUDA for a failed copy or launch.
 */
lb_status lb_propagate_resident(lb_ctx* ctx, int n, const lb_c64* P, int B, lb_c64* states_host, void* stream);

/*
 * lb_propagate_host -- host-visible timing model (Eq. 9): as
 * lb_propagate_resident, but P is in HOST memory too and the device buffers
 * for P and the states are allocated (cudaMalloc) and freed (cudaFree)
 * inside every call, as by a caller that keeps nothing on the device.
 *   Errors: as lb_propagate_resident; LB_ENOMEM if an allocation fails.
 *   Buffers are freed on every path.
 */
lb_status lb_propagate_host(lb_ctx* ctx, int n, const lb_c64* P_host, int B, lb_c64* states_host, void* stream);

/*
 * lb_probe_launch -- host time per launch of an empty kernel on `stream`,
 * in microseconds (*us_out), over `reps` >= 1 launches: back to back
 * (sync_each = 0: the launch cost t_launch) or each followed by a stream
 * synchronise (sync_each = 1: launch + sync).  Waits for the stream first.
 */
lb_status lb_probe_launch(int reps, int sync_each, double* us_out, void* stream);

/*
 * lb_probe_copy -- host time per synchronous copy of `bytes` bytes between
 * `host` (pageable or pinned) and `device` (to_device = 1: host to device,
 * 0: device to host), in microseconds, over `reps` >= 1 copies, each
 * followed by a synchronise of `stream`.
 */
lb_status lb_probe_copy(void* host, void* device, long long bytes, int to_device, int reps, double* us_out,
                        void* stream);

/*
 * lb_probe_alloc -- host time of one cudaMalloc of `bytes` bytes followed
 * by its cudaFree on the CURRENT device, in microseconds, averaged over
 * `reps` >= 1 pairs (the allocation term of Eq. 9).  Synchronises the
 * device first.  LB_ENOMEM if an allocation fails.
 */
lb_status lb_probe_alloc(long long bytes, int reps, double* us_out);

/*
 * lb_probe_read -- one read pass over `count` complex128 values of `buf`
 * (device): n = 0 is a coalesced stream (consecutive threads read
 * consecutive values); n >= 1 is the stride-n gather of Algorithm alg:gpu
 * (one thread per row of n values, consecutive threads consecutive rows;
 * the count % n trailing values are not read).  `sink` (device, 8 bytes)
 * is written only on an impossible match.  Time it with events on `stream`.
 */
lb_status lb_probe_read(const lb_c64* buf, long long count, int n, unsigned long long* sink, void* stream);

/* ------------------------------------------------------------------------
 * Arithmetic peak probes (the measured ceilings of Sec. 3.6, Table
 * tab:probes_gpu, for the FP64 / FP32 / tensor-core rooflines): each runs
 * one untimed and five timed launches of a kernel that keeps one unit busy
 * with independent work and no memory traffic, timed with CUDA events on
 * `stream` (synchronised), and writes the best rate in TFLOP/s (2 FLOPs per
 * multiply-add) to *tflops_out (host).  On the CURRENT device (sm_103 only,
 * else LB_ENODEV); no device memory is allocated.
 *   lb_probe_dfma     FP64 FMA on the CUDA cores
 *   lb_probe_ffma     FP32 FMA on the CUDA cores
 *   lb_probe_dmma     FP64 tensor-core MMA (mma.sync m8n8k4 f64)
 *   lb_probe_bf16_tc  BF16 tcgen05 MMA, M = 128, N = 256, K = 16, FP32
 *                     accumulation in TMEM; its wait for the MMAs is
 *                     bounded (about 2 s), LB_ETIMEOUT if it gives up
 *   Errors: LB_EINVAL (null pointer), LB_ENODEV, LB_ECUDA, LB_ETIMEOUT.
 * ------------------------------------------------------------------------ */
lb_status lb_probe_dfma(double* tflops_out, void* stream);
lb_status lb_probe_ffma(double* tflops_out, void* stream);
lb_status lb_probe_dmma(double* tflops_out, void* stream);
lb_status lb_probe_bf16_tc(double* tflops_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
