/*
 * gp.h -- C ABI of libgp: exact Gaussian-process inference by blackbox
 * kernel-matrix products on one NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2109.09817 ("Molecular energy learning using alternative
 * blackbox matrix-matrix multiplication algorithm for exact Gaussian
 * process").  Problem statement (Sec. 2.2): data X in R^{N x d}, targets
 * y in R^N, Gaussian noise sigma^2, kernel K : R^d x R^d -> R,
 *   K-hat = K(X, X) + sigma^2 I,
 *   E[f(X')]   = K(X', X) K-hat^{-1} y                        (Eq. pred)
 *   L          = -1/2 y^T K-hat^{-1} y - 1/2 log|K-hat| - N/2 log 2 pi (Eq. ll)
 * Kernel (Sec. 4): Matern 5/2, read with one lengthscale per feature (ARD):
 *   r^2 = sum_j ((x_j - x'_j) / l_j)^2,
 *   k(x, x') = s (1 + sqrt5 r + 5 r^2 / 3) exp(-sqrt5 r).
 *
 * CONVENTIONS (all entry points)
 *  - Every array argument is DEVICE memory on the context's device unless
 *    the argument says "host".  The caller owns every array; the library
 *    never frees or keeps caller pointers past the call.
 *  - Feature matrices (X, X') are float32, row-major: point a's features at
 *    X + a*d.
 *  - A "block of t vectors of length n" is float32 COLUMN-MAJOR: vector c at
 *    V + c*n, element a of it at V[c*n + a].
 *  - Work is queued on the context's CUDA stream.  Calls that return host
 *    values (ranks, iteration counts, scalars) synchronise that stream
 *    before returning; the others are asynchronous.
 *  - Return value: GP_OK or a negative-free error code below; the message
 *    of the last error is gp_last_error(ctx).  Invalid sizes/pointers give
 *    GP_EINVAL before any work is queued.
 *  - Hyperparameters are natural positive values (l_j, s, sigma^2 > 0).
 */
#ifndef GP_H_
#define GP_H_

#include <stdint.h>

#if defined(__GNUC__)
#define GP_API __attribute__((visibility("default")))
#else
#define GP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes -------------------------------------------------------- */
enum {
  GP_OK = 0,
  GP_EINVAL = 1,      /* bad argument (size, null pointer, value range)      */
  GP_ENOMEM = 2,      /* device workspace allocation failed                  */
  GP_ENOTCONV = 3,    /* CG hit max_iter before every column met tol; the
                         outputs hold the last iterate and its residuals    */
  GP_EBREAKDOWN = 4,  /* CG lost definiteness: d^T K-hat d <= 0 or r^T z <= 0 */
  GP_ENONPD = 5,      /* pivoted Cholesky met a residual diagonal <= 0 before
                         the requested rank (rank_out holds the rank reached) */
  GP_ETIMEOUT = 6,    /* a bounded device-side wait gave up                  */
  GP_ECUDA = 7        /* a CUDA runtime/driver call failed                   */
};

/* ---- arithmetic of the K-hat product ------------------------------------ */
enum {
  GP_FP32_PLAIN = 0,      /* FP32 FFMA on the CUDA cores only               */
  GP_FP32_SPLIT_TF32 = 1, /* tcgen05 kind::tf32, hi+lo split operands
                             (3 products) for both the cross term X X^T and
                             the contraction K V: FP32-class accuracy       */
  GP_FP32_SPLIT_F16 = 2,  /* tcgen05 kind::f16 with FP16 hi+lo split operands
                             (3 products) for both contractions.  Operands
                             are scaled by powers of two (features: one
                             factor for the whole matrix; vectors: one per
                             vector; K: 2^14) so that FP16's range holds
                             them; the split then keeps 22 significant bits
                             as the TF32 split does, at twice the reduction
                             depth per MMA.  Needs d <= 64.                 */
  GP_TF32 = 3             /* tcgen05 kind::tf32, single-pass operands       */
};
/* No BF16 forms: a BF16 hi + lo split keeps 16 significant bits of every
 * operand where the FP16 and TF32 splits keep 22, at the same tensor rate as
 * FP16; an operand-rounding emulation on the 2048-row workload gives K-hat V
 * errors of 1.3e-5 (split BF16) against 2.4e-7 (split FP16), which leaves no
 * margin under the 2e-5 split tolerance once the tensor core's FP32
 * accumulation (about 1e-5 at N = 2^20) is added.  Split FP16 takes the slot
 * of split BF16, and single TF32 that of single BF16. */

/* GP_HOST, OR-ed into the `precision` argument of gp_kmatmul,
 * gp_kcross_matmul and gp_logml_and_grad: their feature, vector and output
 * arrays (X, Xp, V, out, y) are HOST memory.  The library copies the inputs
 * into its device workspace on the context's stream (pinned memory copies
 * asynchronously, pageable memory through the runtime's staging), runs the
 * device path and copies out back; such a call synchronises.  The other
 * arguments keep their meaning. */
#define GP_HOST 0x100

/* preconditioner forms (P = L L^T + D, L from the rank-k pivoted Cholesky) */
enum {
  GP_PC_SIGMA = 0,  /* D = sigma^2 I: the form of Sec. 3.2                   */
  GP_PC_RESID = 1   /* D = diag(K - L L^T) + sigma^2 I: the residual diagonal
                       of the same factorisation is kept (reduces to the first
                       form when K is close to rank k; stays well conditioned
                       when K is close to diagonal)                          */
};

/* stop rules of the CG solves (gp_mbcg, gp_logml_and_grad, gp_model_fit) */
enum {
  GP_STOP_RECURRENCE = 0, /* a column stops when its CG recurrence residual
                             ||r_c|| / ||b_c|| is below tol (Sec. 4)        */
  GP_STOP_TRUE = 1        /* as GP_STOP_RECURRENCE, then the solution
                             columns are verified: one K-hat product of the
                             iterate measures ||b_c - K-hat w_c|| / ||b_c||,
                             and a column not below 0.8 tol continues its own
                             recurrence to a proportionally lower target (its
                             CG coefficients stay one unbroken Lanczos
                             sequence); at most 4 verifications, after which
                             a column still above 0.8 tol gives GP_ENOTCONV.
                             In FP32 storage the attainable true residual is
                             bounded below by rounding (about 1e-6 to 1e-5 on
                             ill-conditioned K-hat), so tight tolerances need
                             GP_STOP_RECURRENCE.                             */
};

/* posterior variance modes of gp_predict / gp_predict_sum */
enum {
  GP_VAR_NONE = 0,
  GP_VAR_EXACT = 1,   /* K-hat^{-1} by preconditioned CG solves              */
  GP_VAR_CACHED = 2   /* K-hat^{-1} ~ R R^T from the model's Lanczos cache
                         (gp_model_variance_cache)                          */
};
#define GP_VAR_CACHE_MAX_RANK 128

typedef struct gp_ctx gp_ctx;
typedef struct gp_model gp_model;

/* Hyperparameters theta = (l, s, sigma^2).  lengthscale: HOST pointer to d
 * doubles, read during the call only. */
typedef struct {
  const double* lengthscale;
  double outputscale;
  double sigma2;
} gp_theta;

/* Solver diagnostics (host struct, filled when a pointer is passed). */
typedef struct {
  int iters_max;        /* CG steps taken (max over columns)                */
  int iters_y;          /* steps taken by column 0 (the y column)           */
  int rank;             /* preconditioner rank reached                      */
  int n_kmatmul;        /* K-hat products issued                            */
  double relres_y;      /* CG recurrence residual ||r||/||b|| of column 0   */
  double relres_max;    /* max over columns                                  */
  double logdet_P;      /* log|P|, P = L L^T + sigma^2 I                    */
  double yKinvy;        /* y^T K-hat^{-1} y                                  */
  double true_relres_y; /* ||y - K-hat a|| / ||y|| measured by one product of
                           the final iterate (-1 if not measured)           */
  int true_checks;      /* products spent on those measurements             */
} gp_stats;

/* ---- context -------------------------------------------------------------
 * gp_create: bind a context to CUDA device `device` and stream `stream`
 * (a cudaStream_t; NULL = legacy default stream).  The context owns a
 * device workspace that grows on demand and is freed by gp_destroy.  One
 * context per stream; a context is not thread-safe. */
GP_API int gp_create(gp_ctx** out, int device, void* stream);
GP_API void gp_destroy(gp_ctx* ctx);
GP_API int gp_set_stream(gp_ctx* ctx, void* stream);
GP_API int gp_sync(gp_ctx* ctx);
GP_API const char* gp_last_error(const gp_ctx* ctx);
/* Number of kernels this context has launched (diagnostics). */
GP_API int64_t gp_launch_count(const gp_ctx* ctx);
/* Context options.  GP_OPT_SYMMETRIC_KMV (default 1): K-hat V products in
 * GP_FP32_SPLIT_F16 use K's symmetry, forming only the tiles at and right of
 * the diagonal blocks and contracting each twice (K_IJ V_J and K_IJ^T V_I);
 * 0 selects the full-grid kernel (every tile formed once), for comparisons.
 * GP_EINVAL for an unknown option or value. */
enum { GP_OPT_SYMMETRIC_KMV = 1 };
GP_API int gp_set_option(gp_ctx* ctx, int option, int value);
/* K-hat V timing: gp_profile(ctx, 1) resets the counters and records a CUDA
 * event pair on the context's stream around every K-hat V product issued
 * from then on (gp_profile(ctx, 0) stops recording).  gp_profile_read
 * synchronises and returns (HOST outputs) the number of products, their
 * summed device time in ms, their GEMM-equivalent flops 2 m n (d + t) and
 * the kernel entries they evaluated: m n (m, n = rows and columns of the
 * product), or, for the symmetric split-FP16 product, the entries of the
 * tiles at and right of the diagonal blocks (about n^2 / 2). */
GP_API int gp_profile(gp_ctx* ctx, int enable);
GP_API int gp_profile_read(gp_ctx* ctx, int64_t* products, double* ms,
                           double* flops, double* entries);

/* ---- K-hat V (Sec. 3.1 "only the matrix-vector multiplications"; Sec. 3.2
 * "O(N) memory"; Sec. 4 kernel tiles) --------------------------------------
 * out = (K(X, X) + sigma^2 I) V, with K formed tile by tile from X and
 * never stored.  X: N x d row-major.  V, out: t vectors of length N,
 * column-major.  1 <= t <= 512.  `precision` is one of GP_FP32_PLAIN ...
 * GP_TF32; the tensor-core forms need d <= 64 (GP_EINVAL otherwise).  out
 * must not alias V. */
GP_API int gp_kmatmul(gp_ctx* ctx, const float* X, int64_t N, int d,
               const gp_theta* theta, const float* V, int t, float* out,
               int precision);

/* out = K(X', X) V (the cross covariance of Eq. pred).  X': M x d, X: N x d,
 * V: t vectors of length N, out: t vectors of length M. */
GP_API int gp_kcross_matmul(gp_ctx* ctx, const float* Xp, int64_t M, const float* X,
                     int64_t N, int d, const gp_theta* theta, const float* V,
                     int t, float* out, int precision);

/* ---- pivoted Cholesky preconditioner (Sec. 3.2, rank-k greedy factor) ----
 * Greedy rank-k factor K ~ L L^T in FP64: at step j the pivot is the row
 * with the largest residual diagonal (lowest index on ties), the column is
 * (K(X, x_p) - L_{:,<j} L_{p,<j}^T) / sqrt(d_p), and the pivot's residual
 * is set to zero.  Stops early when the largest residual diagonal is
 * <= 1e-12 s.  L: N x k FP64 column-major (column j at L + j*N); columns
 * past the rank reached are zero.  piv: k int64 (past the rank: -1).
 * rank_out: HOST int.  resid_diag (nullable, N doubles, device): the
 * residual diagonal diag(K - L L^T) after the last step, zero at the pivots.
 * Synchronises. */
GP_API int gp_pivchol(gp_ctx* ctx, const float* X, int64_t N, int d,
               const gp_theta* theta, int k, double* L, int64_t* piv,
               int* rank_out, double* resid_diag);

/* ---- mBCG (Sec. 3.2; CG of Sec. 3.1 with preconditioner P) ----------------
 * Solves K-hat Omega = B for t right-hand sides at once with preconditioned
 * CG, P = L L^T + D applied by the Woodbury identity (L from gp_pivchol,
 * rank k; D = sigma^2 I, or diag(resid_diag) + sigma^2 I when resid_diag
 * (device, N doubles, from gp_pivchol) is given; k = 0 and no resid_diag
 * means P = sigma^2 I, i.e. plain CG).  Every
 * column shares each K-hat product.  Column c stops (is frozen) once
 * ||r_c|| / ||b_c|| < tol (Sec. 4 stop rule); the solve stops when all
 * columns stopped or after max_iter steps (then GP_ENOTCONV).
 * B, Omega: t vectors of length N (column-major).  alpha_hist, beta_hist:
 * nullable device FP64 arrays of max_iter*t, entry [j*t + c] = the CG
 * coefficient of column c at step j (0 after the column stopped); the
 * Lanczos tridiagonal of column c follows from its first iters[c] entries
 * (entries are indexed by the column's own steps).  stop_rule: GP_STOP_
 * RECURRENCE, or GP_STOP_TRUE to verify every column's true residual (one
 * extra product per verification).  iters, rel_resid: nullable HOST arrays
 * of t; rel_resid holds the measured true residuals under GP_STOP_TRUE, the
 * recurrence residuals otherwise.  Synchronises. */
GP_API int gp_mbcg(gp_ctx* ctx, const float* X, int64_t N, int d,
            const gp_theta* theta, const double* L, int k,
            const double* resid_diag, const float* B,
            int t, double tol, int max_iter, int stop_rule, int precision, float* Omega,
            double* alpha_hist, double* beta_hist, int* iters,
            double* rel_resid);

/* Lanczos quadrature of mBCG's coefficients (Sec. 3.2: the log-determinant
 * term of Eq. ll).  For each column c, T_c is the iters[c] x iters[c]
 * tridiagonal of the PCG/Lanczos relation, T_jj = 1/alpha_j +
 * beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j, and
 * quad[c] = e1^T log(T_c) e1 (0 when iters[c] = 0); the log-determinant
 * estimate is log|P| + (1/t) sum_c ||z_c||^2_{P^{-1}} quad[c] over the probe
 * columns.  alpha_hist, beta_hist: device FP64, max_iter*t, entry [j*t + c]
 * (the layout gp_mbcg writes); iters: HOST, t ints in [0, max_iter];
 * quad: HOST, t doubles.  1 <= t <= 256.  Computed on the device to about
 * 1e-13 absolute (a trapezoid rule on an integral representation, no
 * eigendecomposition).  GP_EBREAKDOWN if some T_c is not positive definite
 * (its quad[c] is 0).  Synchronises. */
GP_API int gp_lanczos_logquad(gp_ctx* ctx, const double* alpha_hist, const double* beta_hist, int t,
                              int max_iter, const int* iters, double* quad);

/* AltBBMM solve (Sec. 3.2): block CG (Sec. 3.1, BCG) on the symmetrically
 * preconditioned system S^T K-hat S W = S^T B, Omega = S W, with S S^T =
 * P^{-1}, P = L L^T + D the Nystrom preconditioner whose landmarks are the
 * pivots of gp_pivchol (L, rank k; D = sigma^2 I, or diag(resid_diag) +
 * sigma^2 I when resid_diag is given; k = 0: S = D^{-1/2}).  All t columns
 * share one block Krylov space; the solve stops when every relative residual
 * ||B_c - K-hat Omega_c|| / ||B_c|| (by its recurrence) is below tol.
 * B, Omega: device, N x t column-major (ld N), 1 <= t <= 32, no zero column
 * (GP_EINVAL).  iters (host int, nullable): block steps taken; rel_resid
 * (host t doubles, nullable).  The s x s systems are solved by pseudo-inverse
 * (directions below 1e-10 of the largest eigenvalue are dropped), so columns
 * that converge or become dependent get zero steps.  In FP32 storage the
 * block recurrence can stall a little above a tight tol (for example at
 * 1.1e-5 on 2048 points with D = sigma^2 I); when the largest residual is
 * within 4 tol and has not fallen by 10 % over 3 steps, the residual is
 * recomputed as B - K-hat Omega (one more product) and the recurrence
 * restarts from the current iterate, at most twice.  GP_ENOTCONV after
 * max_iter steps (Omega holds the last iterate); GP_EBREAKDOWN if a block
 * Gram matrix vanishes.
 * Synchronises every step. */
GP_API int gp_bcg(gp_ctx* ctx, const float* X, int64_t N, int d,
                  const gp_theta* theta, const double* L, int k,
                  const double* resid_diag, const float* B, int t, double tol,
                  int max_iter, int precision, float* Omega, int* iters,
                  double* rel_resid);

/* Mixed-precision iterative refinement of K-hat Omega = B (the solve of
 * Sec. 3.1; the refinement loop itself is not in the paper).  Starting from
 * Omega = 0: solve K-hat delta = R with preconditioned mBCG whose products use
 * `inner_precision` (e.g. GP_TF32), to relative residual `inner_tol`; then
 * Omega += delta and R = B - K-hat Omega with products in `outer_precision`
 * (GP_FP32_SPLIT_TF32, GP_FP32_SPLIT_F16 or GP_FP32_PLAIN).  A column stops once
 * ||R_c|| / ||B_c|| < 0.8 tol (the margin of GP_STOP_TRUE for the measuring
 * product's own error; its R is zeroed, so later inner solves skip it);
 * the loop ends when every column has stopped or after max_outer rounds.
 * Preconditioner as in gp_mbcg (L, k, resid_diag).  B, Omega: device, N x t
 * column-major (ld N).  outer_steps, inner_steps (total inner CG steps over
 * all rounds, max over columns per round), rel_resid (t, the last true
 * relative residuals in the outer precision): nullable HOST outputs.
 * Returns GP_ENOTCONV (Omega holds the last iterate) when a column has not
 * reached tol after max_outer rounds.  If an inner solve breaks down (the
 * inner operator is too inexact to stay positive definite, e.g. single TF32
 * on near-duplicate rows) its partial iterate is used; a round that breaks
 * down and reduces no residual by 10 % returns GP_EBREAKDOWN.  Synchronises
 * once per round. */
GP_API int gp_mbcg_refine(gp_ctx* ctx, const float* X, int64_t N, int d,
                   const gp_theta* theta, const double* L, int k,
                   const double* resid_diag, const float* B, int t, double tol,
                   double inner_tol, int max_outer, int max_iter,
                   int inner_precision, int outer_precision, float* Omega,
                   int* outer_steps, int* inner_steps, double* rel_resid);

/* ---- log marginal likelihood and gradient (Eq. ll; Sec. 3.2) -------------
 * One pass of the whole training path: rank-k pivoted Cholesky and the
 * preconditioner P = L L^T + D of form `precond` (GP_PC_SIGMA or
 * GP_PC_RESID); probes z_c = L e1_c + D^{1/2} e2_c (c < n_probes), so that
 * Cov(z) = P, with Rademacher signs from the
 * SplitMix64 sequence seeded by `seed`; mBCG on [y | z_1..z_t]; Lanczos
 * quadrature of log|K-hat|; and the gradient
 *   dL/dtheta = 1/2 a^T dK a - 1/(2t) sum_c (K-hat^{-1} z_c)^T dK (P^{-1} z_c)
 * with a = K-hat^{-1} y.  y: N floats (device).  Outputs are HOST:
 * logml, logdet, logdet_stderr (standard error over probes, nullable),
 * grad (d + 2 doubles: dL/dl_1..dL/dl_d, dL/ds, dL/dsigma^2; nullable to
 * skip the gradient pass), stats (nullable).  1 <= n_probes <= 255.
 * `precision` is the arithmetic of the K-hat products; with either split
 * form the gradient pass runs on the tensor cores in split TF32 (the split
 * FP16 form prepares the TF32 split features as well).  stop_rule
 * (GP_STOP_RECURRENCE or GP_STOP_TRUE) applies to y's column, the solve
 * a = K-hat^{-1} y; the probe columns stop by their recurrences.
 * Synchronises. */
GP_API int gp_logml_and_grad(gp_ctx* ctx, const float* X, int64_t N, int d,
                      const gp_theta* theta, const float* y, int n_probes,
                      uint64_t seed, int k, int precond, double tol, int max_iter,
                      int stop_rule, int precision, double* logml, double* logdet,
                      double* grad, double* logdet_stderr, gp_stats* stats);

/* ---- K-hat V without any allocation ---------------------------------------
 * For callers that cannot allocate device memory (a process whose memory is
 * reserved by another framework's pool, a real-time loop where cudaMalloc /
 * cudaFree and the synchronisation they imply are not allowed).  The paper
 * has no counterpart: this is a deployment variant of gp_kmatmul with
 * GP_FP32_PLAIN arithmetic.  It calls no cudaMalloc, cudaFree,
 * cudaMallocHost or other allocating routine and needs no context: its
 * scratch (column means, prepared features, row norms) is one fixed
 * file-scope device array of about 4.4 MiB, which every GPU that loads the
 * library holds until the process exits.
 *  - X, V, out: as in gp_kmatmul (device; V and out t x N column-major;
 *    out must not alias V).  stream: a cudaStream_t (NULL = default).
 *  - Limits: N <= GP_NOALLOC_MAX_ROWS, d <= GP_NOALLOC_MAX_D,
 *    round_up(N, 64) * round_up(d, 32) <= GP_NOALLOC_MAX_FEATURES,
 *    1 <= t <= 512; larger sizes return GP_EINVAL before any work.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents:
 *    calls that overlap on the GPU (other streams, other host threads) race
 *    and must be serialised by the caller.
 *  - Asynchronous on `stream`; errors: GP_EINVAL (sizes, pointers,
 *    hyperparameters), GP_ECUDA (a launch failed). */
#define GP_NOALLOC_MAX_ROWS 65536
#define GP_NOALLOC_MAX_D 256
#define GP_NOALLOC_MAX_FEATURES (1 << 20)
GP_API int gp_kmatmul_noalloc(const float* X, int64_t N, int d,
                              const gp_theta* theta, const float* V, int t,
                              float* out, void* stream);

/* ---- hyperparameter optimisation (Sec. 4, computational details) ---------
 * gp_subset_indices: M distinct row indices of 0..N-1 drawn by a seeded
 * partial Fisher-Yates shuffle (SplitMix64 stream from `seed`), sorted, into
 * idx (HOST, M int64).  Runs on the host; GP_EINVAL for M > N or M < 1.
 *
 * gp_hyperopt: the paper optimises the hyperparameters on a random subset of
 * the training data and does not name the optimiser; here `steps` steps of
 * Adam (beta1 0.9, beta2 0.999, step `lr`) on log theta ascend the log
 * marginal likelihood of Eq. (ll) on the `subset` rows chosen by
 * gp_subset_indices(N, subset, seed), with the value and gradient of
 * gp_logml_and_grad (n_probes trace probes from one fixed seed, so the
 * objective is the same function of theta at every step; rank-k
 * preconditioner of form `precond`, tol, max_iter, precision as there; a
 * solve that reaches max_iter is used as it stands).  X: N x d, y: N
 * (device).  lengthscale (d), outputscale, sigma2: HOST, the starting point
 * on entry, the optimised values on return.  logml_hist (HOST, steps + 1,
 * nullable): the objective at each visited theta, the last one at the
 * returned theta; grad_out (HOST, d + 2, nullable): the gradient there.
 * Synchronises.
 *
 * gp_train: gp_hyperopt, then gp_model_fit on all N rows with sigma^2 +
 * sigma2_add (Sec. 4 adds sigma^2_add to the optimised noise before the
 * full fit; block = 1, GP_STOP_RECURRENCE); the hyperparameters returned
 * are the optimised ones, without sigma2_add. */
GP_API int gp_subset_indices(int64_t N, int64_t M, uint64_t seed, int64_t* idx);
GP_API int gp_hyperopt(gp_ctx* ctx, const float* X, int64_t N, int d, const float* y,
                       int64_t subset, uint64_t seed, int steps, double lr, int n_probes,
                       int k, int precond, double tol, int max_iter, int precision,
                       double* lengthscale, double* outputscale, double* sigma2,
                       double* logml_hist, double* grad_out);
GP_API int gp_train(gp_ctx* ctx, const float* X, int64_t N, int d, const float* y,
                    int64_t subset, uint64_t seed, int steps, double lr, int n_probes, int k,
                    int precond, double tol, int max_iter, int precision, double sigma2_add,
                    double* lengthscale, double* outputscale, double* sigma2,
                    double* logml_hist, gp_model** out);

/* ---- trained model and prediction (Eq. pred) ------------------------------
 * gp_model_fit keeps, on the device, the prepared features, a = K-hat^{-1} y,
 * the preconditioner factor and the hyperparameters.  block = 1: a by
 * preconditioned CG on y alone (mBCG to `tol`); 2 <= block <= 32: AltBBMM
 * (Sec. 3.1-3.2), block CG on [y | block - 1 random right-hand sides] with
 * the symmetric Nystrom preconditioner (as gp_bcg), stopping when y's
 * residual is below tol; a = column 0 (the block Krylov space contains y's
 * own, so y converges in fewer steps; a product costs the same for up to 16
 * vectors).  stop_rule (block = 1 only; block CG stops by its recurrence):
 * GP_STOP_RECURRENCE or GP_STOP_TRUE for the solve of y.  X and y are copied; the caller may free them afterwards.
 * GP_ENOTCONV / GP_EBREAKDOWN: no model is returned.  Synchronises. */
GP_API int gp_model_fit(gp_ctx* ctx, const float* X, int64_t N, int d,
                 const gp_theta* theta, const float* y, int k, int precond, int block,
                 double tol, int max_iter, int stop_rule, int precision, gp_model** out,
                 gp_stats* stats);
GP_API void gp_model_free(gp_model* model);

/* mean = K(X', X) a.  var (nullable): var_mode GP_VAR_EXACT gives the latent
 * posterior variance k(x', x') - k*^T K-hat^{-1} k* (Eq. pred read as the
 * standard posterior variance) by an mBCG solve with the M columns k* as
 * right-hand sides (to the model's tol); GP_VAR_CACHED reads it from the
 * model's variance cache (GP_EINVAL without one) with one cross product.
 * Xp: M x d row-major; mean, var: M floats.  Synchronises when var is
 * requested with GP_VAR_EXACT. */
GP_API int gp_predict(gp_ctx* ctx, const gp_model* model, const float* Xp, int64_t M,
               float* mean, float* var, int var_mode);

/* ---- variance cache (Eq. pred at sizes where one solve per test row is
 * out of reach) --------------------------------------------------------------
 * The paper does not say how it serves variances; this is the low-rank
 * Lanczos cache of Pleiss et al. (2018).  `rank` (1 <= rank <=
 * GP_VAR_CACHE_MAX_RANK) steps of Lanczos on K-hat from the start vector b
 * (device, N floats; NULL = K-hat a, which is y up to the fit's tolerance),
 * with full reorthogonalisation (FP32 vectors, FP64 coefficients and dot
 * products), give K-hat Q ~ Q T; the model keeps R = Q C^{-T}, T = C C^T,
 * so that K-hat^{-1} ~ R R^T and the latent variance is read as
 * k(x',x') - |R^T k*|^2 (an upper bound of the exact variance that tightens
 * as the rank grows; exact with a full Krylov basis).  Costs `rank` K-hat
 * products; the cache takes rank x N floats of device memory, owned by the
 * model (freed by gp_model_free).  *rank_out: the steps taken (fewer when
 * b's Krylov space is exhausted).  GP_EBREAKDOWN if T is not positive
 * definite.  Synchronises. */
GP_API int gp_model_variance_cache(gp_ctx* ctx, gp_model* model, const float* b, int rank,
                                   int* rank_out);

/* Per-molecule prediction (Sec. 2.1: a molecule's correlation energy is the
 * sum of its pair energies): over the M rows of Xp (device, M x d), the
 * HOST outputs mean_sum = sum_i E[f(x'_i)] and var_sum (nullable) =
 * Var[sum_i f(x'_i)] = 1^T K(X',X') 1 - c^T K-hat^{-1} c with c = K(X,X') 1,
 * every cross-covariance between the molecule's rows included.  var_mode
 * GP_VAR_EXACT solves for K-hat^{-1} c (one CG solve to the model's tol);
 * GP_VAR_CACHED uses the model's cache (|R^T c|^2).  1^T K(X',X') 1 is summed
 * in FP64 from kernel entries formed by direct differences.  A diagonal and
 * an off-diagonal model are independent GPs: their sums and variances add.
 * Synchronises. */
GP_API int gp_predict_sum(gp_ctx* ctx, const gp_model* model, const float* Xp, int64_t M,
                          double* mean_sum, double* var_sum, int var_mode);

/* ---- serving: continuous batching over resident models (Eq. pred) --------
 * A gp_server holds trained models on one device and serves two request
 * kinds from host memory:
 *  - predict: the mean K(X', X) a (and, from the model's variance cache, the
 *    latent variances) of one request's M feature rows against a resident
 *    model; a molecule request sums the predictions of its diagonal and
 *    off-diagonal pair rows over two models, with the variance of the sum.  Each model has its own stream and batching thread:
 *    every request queued when a batch starts (up to max_batch_rows rows) is
 *    packed into ONE fused K(X', X) a launch; requests arriving meanwhile join
 *    the next batch.  Batches of different models overlap on the device.
 *  - solve: a new model's a = K-hat^{-1} y (split-TF32 mBCG, rank-k
 *    residual-diagonal preconditioner), on its own stream, overlapping the
 *    predict batches; admitted when the device's free memory covers the
 *    solve's estimated footprint plus reserve_bytes (waits up to ~60 s, then
 *    the request fails with GP_ENOMEM).
 * Host arrays passed to gp_server_predict / gp_server_solve must stay valid
 * until gp_server_wait for that ticket has returned.  The server object is
 * thread-safe: requests may be submitted and waited for from any thread. */
typedef struct gp_server gp_server;

/* device: CUDA device index; max_batch_rows >= 1: row budget of one predict
 * batch (a single request may not exceed it); reserve_bytes >= 0: device
 * memory kept free when admitting a solve.  GP_ECUDA if the device or its
 * streams cannot be set up. */
GP_API int gp_server_create(gp_server** out, int device, int64_t max_batch_rows,
                            double reserve_bytes);
/* Fit a model from DEVICE arrays X (N x d) and y (N) as gp_model_fit does
 * (block = 1, GP_STOP_RECURRENCE), build its variance cache of rank var_rank
 * (0 = none; 1 <= var_rank <= GP_VAR_CACHE_MAX_RANK, started at K-hat a),
 * keep it resident and start its batching thread; *model_id is its index.
 * Synchronises; errors as gp_model_fit and gp_model_variance_cache (message
 * in gp_server_last_error). */
GP_API int gp_server_add_model(gp_server* srv, const float* X, int64_t N, int d,
                               const gp_theta* theta, const float* y, int k, int precond,
                               double tol, int max_iter, int precision, int var_rank,
                               int* model_id);
/* Queue a predict request: Xp HOST M x d row-major, mean HOST M floats, var
 * HOST M floats or NULL (the latent variances from the model's variance
 * cache), both written before the request completes.  GP_EINVAL for an
 * unknown model, M < 1, M > max_batch_rows, or var without a cache. */
GP_API int gp_server_predict(gp_server* srv, int model_id, const float* Xp, int64_t M,
                             float* mean, float* var, uint64_t* ticket);
/* Queue a molecule request (Sec. 2.1: the correlation energy is the sum of
 * the pair energies): Xd HOST Md x d, the molecule's diagonal pair rows for
 * model diag_model; Xo HOST Mo x d (Mo >= 0), its off-diagonal pair rows for
 * model off_model.  energy HOST 2 doubles, written before completion:
 * [0] = the sum of the predictive means over all Md + Mo rows, [1] = the
 * variance of that sum (cross-covariances within each model's rows from the
 * models' variance caches; the two models are independent GPs).  Both parts
 * join their models' batches.  GP_EINVAL for unknown models, sizes out of
 * range, or a model without a variance cache. */
GP_API int gp_server_molecule(gp_server* srv, int diag_model, const float* Xd, int64_t Md,
                              int off_model, const float* Xo, int64_t Mo, double* energy,
                              uint64_t* ticket);
/* Queue a solve request: X HOST N x d, y HOST N, alpha HOST N (out). */
GP_API int gp_server_solve(gp_server* srv, const float* X, int64_t N, int d,
                           const gp_theta* theta, const float* y, int k, double tol,
                           int max_iter, float* alpha, uint64_t* ticket);
/* Wait up to timeout_s seconds for a request; returns its status (GP_OK or
 * the error it failed with), GP_ETIMEOUT if it has not completed (the ticket
 * stays valid), GP_EINVAL for an unknown ticket.  latency_ms (nullable HOST):
 * submit-to-completion time.  A completed ticket is released. */
GP_API int gp_server_wait(gp_server* srv, uint64_t ticket, double timeout_s,
                          double* latency_ms);
/* Predict batches launched and predict requests served so far. */
GP_API int gp_server_stats(gp_server* srv, int64_t* batches, int64_t* predicted);
GP_API const char* gp_server_last_error(gp_server* srv);
/* Finishes every queued request, then frees models, streams and buffers. */
GP_API void gp_server_destroy(gp_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* GP_H_ */
