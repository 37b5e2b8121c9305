// Internal declarations shared by the libgp translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "../../include/gp.h"

namespace gp {

// ---------------------------------------------------------------------------
// Feature scaling.  Prepared features are x~ = c (x - mu) / l with
// c = sqrt(5) * log2(e), so that for two prepared rows
//   u^2 = |x~_a|^2 + |x~_b|^2 - 2 x~_a . x~_b = (sqrt5 r log2 e)^2
// and the Matern-5/2 kernel (Sec. 4) becomes
//   k / s = (1 + ln2 u + (ln2)^2 u^2 / 3) 2^{-u},
// one square root and one base-2 exponential per entry.
// ---------------------------------------------------------------------------
constexpr double kSqrt5 = 2.23606797749978969640917366873;
constexpr double kLog2e = 1.44269504088896340735992468100;
constexpr double kLn2 = 0.69314718055994530941723212146;
constexpr double kFeatScale = kSqrt5 * kLog2e;
constexpr float kC1 = 0.69314718055994530942f;   // ln 2
constexpr float kC2 = 0.16014921423310860f;      // (ln 2)^2 / 3

constexpr int kRowPad = 256;   // rows of prepared arrays are padded to this
constexpr int kColPad = 32;    // features are padded to this (zeros)
constexpr int kHalfCols = 64;  // width of the FP16 split feature arrays (zeros)
constexpr int kHalfTop = 15;   // FP16 operands are scaled into [2^14, 2^15)
constexpr int kKExp = 14;      // K entries (<= 1) are held as 2^14 K in FP16
// the Matern polynomial's coefficients times 2^14 (exact powers of two), so
// that 2^14 k/s = (2^14 + 2^14 ln2 u + 2^14 (ln2)^2 u^2 / 3) 2^-u
constexpr float kP0s = 16384.f;
constexpr float kC1s = kC1 * 16384.f;
constexpr float kC2s = kC2 * 16384.f;
constexpr int kMaxT = 512;

// Workspace slots owned by a context.  Each grows on demand.
enum WsSlot {
  WS_MU = 0, WS_SCALE, WS_PART,
  // two families of prepared features with the same layout (rows, cross rows)
  WS_XT, WS_NORM, WS_XT_HI, WS_XT_LO, WS_XH_HI, WS_XH_LO, WS_NORMH, WS_XH_SC,
  WS_XT2, WS_NORM2, WS_XT2_HI, WS_XT2_LO, WS_XH2_HI, WS_XH2_LO, WS_NORMH2, WS_XH2_SC,
  WS_VHI, WS_VLO, WS_VBHI, WS_VBLO, WS_VPAD, WS_VMAX,
  WS_CG_U, WS_CG_R, WS_CG_Z, WS_CG_D, WS_CG_W, WS_CG_Z0, WS_CG_B,
  WS_CG_SCAL, WS_CG_PART, WS_CG_AH, WS_CG_BH, WS_CG_G,
  WS_PC_L, WS_PC_L32, WS_PC_D, WS_PC_PIV, WS_PC_STATE, WS_PC_GRAM, WS_PC_CF,
  WS_LZ_SCR, WS_LZ_OUT,
  WS_GR_U, WS_GR_W, WS_GR_ACC,
  WS_PR_K, WS_PR_O, WS_STATUS, WS_PC_DG, WS_PC_DH, WS_PC_RES,
  WS_RF_R, WS_RF_D, WS_RF_W, WS_RF_S, WS_GT_P, WS_GT_T,
  WS_BC_C, WS_BC_P, WS_BC_W, WS_BC_S, WS_BC_R, WS_BC_RH, WS_BC_D, WS_BC_D2, WS_BC_DT,
  WS_BC_WK, WS_BC_Q, WS_BC_OM, WS_BC_M, WS_BC_DH, WS_PC_D2FF, WS_PC_LFF, WS_CG_W64,
  WS_LV_W, WS_LV_P, WS_LV_T, WS_LV_K, WS_LV_M, WS_LV_C,
  WS_HO_IDX, WS_HO_X, WS_HO_Y,
  WS_HS_X, WS_HS_XP, WS_HS_V, WS_HS_O,
  WS_COUNT
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace gp

// A fitted model resident on the device (gp_model_fit / gp_predict).
struct gp_model {
  int device = 0;
  int64_t n = 0, n_pad = 0;
  int d = 0, d_pad = 0;
  int precision = GP_FP32_PLAIN;
  std::vector<double> ell;
  double s = 1.0, sigma2 = 1e-4, tol = 1e-6;
  int max_iter = 1000;
  double* mu = nullptr;
  float* xt = nullptr;
  float* norm = nullptr;
  float* xt_hi = nullptr;
  float* xt_lo = nullptr;
  __half* xh_hi = nullptr;
  __half* xh_lo = nullptr;
  float* norm_h = nullptr;
  float* xh_scale = nullptr;
  float* alpha = nullptr;      // n_pad, zero padded
  double* L = nullptr;         // n x k
  int k = 0;
  float* L32 = nullptr;
  double* cfac = nullptr;
  float* dh = nullptr;         // D^{-1/2}, n_pad
  double pc_logdet = 0.0;
  float* love_R = nullptr;     // variance cache R = Q C^{-T}: love_m vectors, ld n_pad
  int love_m = 0;
};

struct gp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 148;
  std::string err;
  int64_t launches = 0;
  gp::DevBuf ws[gp::WS_COUNT];
  void* pinned = nullptr;        // small pinned host staging area
  size_t pinned_bytes = 0;
  // K-hat V launch timing (gp_profile): one event pair per product
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  size_t ev_used = 0;
  double prof_flops = 0.0, prof_elems = 0.0;
  bool status_init = false;      // device status word (bounded-wait timeouts)
  bool sym_kmv = true;           // symmetric split-FP16 K-hat V (gp_set_option)
  int* status_host = nullptr;    // its own pinned word (never the staging area)
};

namespace gp {

// ---- error helpers --------------------------------------------------------
int set_err(gp_ctx* ctx, int code, const char* fmt, ...);
int check_cuda(gp_ctx* ctx, cudaError_t e, const char* what);
#define GP_CUDA(ctx, call)                                        \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return ::gp::check_cuda(ctx, e_, #call); \
  } while (0)
#define GP_LAUNCHED(ctx)                                          \
  do {                                                            \
    (ctx)->launches++;                                            \
    cudaError_t e_ = cudaGetLastError();                          \
    if (e_ != cudaSuccess) return ::gp::check_cuda(ctx, e_, "kernel launch"); \
  } while (0)
#define GP_TRY(expr)                 \
  do {                               \
    int rc_ = (expr);                \
    if (rc_ != GP_OK) return rc_;    \
  } while (0)

// Workspace: returns a device buffer of at least `bytes` for `slot`
// (grown with cudaMalloc when needed; contents are not preserved).
void* ws_get(gp_ctx* ctx, int slot, size_t bytes);
template <class T>
T* ws(gp_ctx* ctx, int slot, size_t count) {
  return static_cast<T*>(ws_get(ctx, slot, count * sizeof(T)));
}
void* pinned_get(gp_ctx* ctx, size_t bytes);

// Raises a kernel's dynamic shared-memory limit once per device: the
// attribute belongs to the device that is current, so a process driving
// several devices (or several threads driving one) needs a per-device,
// thread-safe record.  `done` is one static mask per kernel instance.
template <class Kernel>
int smem_attr_once(gp_ctx* ctx, Kernel* kernel, size_t smem, std::atomic<uint64_t>& done) {
  const uint64_t bit = 1ull << (ctx->device & 63);
  if (done.load(std::memory_order_acquire) & bit) return GP_OK;
  GP_CUDA(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  done.fetch_or(bit, std::memory_order_release);
  return GP_OK;
}

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---- prepared features ------------------------------------------------------
struct Prep {
  int64_t n = 0, n_pad = 0;
  int d = 0, d_pad = 0;
  const float* xt = nullptr;      // n_pad x d_pad, row-major, FP32
  const float* norm = nullptr;    // n_pad
  const float* xt_hi = nullptr;   // TF32-representable hi part (FP32 storage)
  const float* xt_lo = nullptr;   // TF32 lo part
  // FP16 split (GP_FP32_SPLIT_F16): hi + lo = 2^e x~ to 22 bits, n_pad x 64
  // halves; norm_h = |hi + lo|^2 / 2^2e; xh_scale (device, 1 float) = 2^-e
  const __half* xh_hi = nullptr;
  const __half* xh_lo = nullptr;
  const float* norm_h = nullptr;
  const float* xh_scale = nullptr;
};

// mu (d doubles, device) = column means of X.
int feature_mean(gp_ctx* ctx, const float* X, int64_t n, int d, double* mu);
// Prepared features of X (n x d) with the given mu and l into the workspace
// slots starting at `slot_xt` (WS_XT or WS_XT2).  `precision` decides which
// split copies are built.
int prepare_features(gp_ctx* ctx, const float* X, int64_t n, int d,
                     const double* mu_dev, const double* lengthscale_host,
                     int precision, int slot_xt, Prep* out);

// ---- K-hat V ----------------------------------------------------------------
// out(t vectors, ld ldo) = s K(rows, cols) V + (sym ? sigma2 V : 0).
// V: t vectors of length cols.n with leading dimension ldv.
// sym: rows and cols are the same point set (diagonal entries exact).
int kmv(gp_ctx* ctx, const Prep& rows, const Prep& cols, const float* V,
        int64_t ldv, int t, float* out, int64_t ldo, double s, double sigma2,
        bool sym, int precision);
int kmv_plain(gp_ctx* ctx, const Prep& rows, const Prep& cols, const float* V,
              int64_t ldv, int t, float* out, int64_t ldo, float s, bool sym);
int kmv_tc(gp_ctx* ctx, const Prep& rows, const Prep& cols, const float* V,
           int64_t ldv, int t, float* out, int64_t ldo, float s, bool sym,
           int precision);
bool kmv_tc_supported(const Prep& rows, int t, int precision);
// Symmetric split-FP16 product (kmv_sym.cu): rows and columns are the same
// point set; V already split into FP16 hi/lo parts (T = 16 or 32 padded
// vectors of length n_pad, leading dimension vld) with per-vector factors vsc.
int kmv_sym_f16(gp_ctx* ctx, const Prep& p, const __half* vhi, const __half* vlo, const float* vsc,
                int64_t vld, int t, int T, float* out, int64_t ldo, float s, int* status);
// kernel entries the symmetric product forms for n points (whole tiles)
double kmv_sym_entries(int64_t n);
// whether kmv() takes the symmetric kernel for these arguments
bool kmv_uses_sym(const gp_ctx* ctx, const Prep& rows, const Prep& cols, bool sym, int precision);
// Device status word written by kernels whose waits are bounded (0 = ok,
// GP_ETIMEOUT = a wait gave up).  check_status synchronises, returns the
// recorded code as a gp error and clears it.
int* device_status(gp_ctx* ctx);
int check_status(gp_ctx* ctx);
// out = sigma2 * V (sym) or 0, rows of length n
int kmv_init_out(gp_ctx* ctx, const float* V, int64_t ldv, int t, int64_t n,
                 float* out, int64_t ldo, float sigma2);

// ---- pivoted Cholesky (FP64) -------------------------------------------------
// P = L L^T + D, D = sigma2 I or diag(resid) + sigma2 I
struct Precond {
  int k = 0;               // rank reached
  int64_t n = 0;
  const double* L = nullptr;     // n x k_alloc FP64 column-major (ld n)
  const double* resid = nullptr; // residual diagonal (device, nullable)
  const float* L32 = nullptr;    // L~ = D^{-1/2} L in FP32, ld n_pad
  const float* dh = nullptr;     // D^{-1/2}, n_pad floats (0 on padding)
  const float* Lff = nullptr;    // the FP64 L as FP32 pairs: hi rows (rank x ld32), then lo rows
  const float* d2ff = nullptr;   // D^{-1} as FP32 pairs: hi (ld32), then lo (ld32); 0 on padding
  int64_t ld32 = 0;
  const double* cfac = nullptr;  // k x k lower Cholesky of I + L~^T L~
  const double* cinv = nullptr;  // (I + L~^T L~)^{-1}, k x k, FP64
  double logdet = 0.0;           // log|P|
  double sigma2 = 0.0;
};
int pivchol_run(gp_ctx* ctx, const float* X, int64_t n, int d,
                const double* lengthscale_host, double s, int k, double* L,
                int64_t* piv, int* rank_out, double* resid_out);
int precond_setup(gp_ctx* ctx, const double* L, int64_t n, int k_alloc,
                  int rank, double sigma2, const double* resid, Precond* out);

// ---- mBCG --------------------------------------------------------------------
struct CgResult {
  int iters_max = 0;
  int n_kmv = 0;
  bool converged = false;
  bool breakdown = false;
  int true_checks = 0;   // K-hat products spent verifying true residuals
  bool true_ok = false;  // every verified column passed
};
struct CgArgs {
  const Prep* prep = nullptr;
  double s = 1.0, sigma2 = 1e-4;
  const Precond* pc = nullptr;   // null: P = sigma2 I
  const float* B = nullptr;      // t vectors, ld ldb
  int64_t ldb = 0;
  int t = 0;
  double tol = 1e-6;
  int max_iter = 1000;
  int precision = GP_FP32_PLAIN;
  float* U = nullptr;            // solution, t vectors, ld ldu
  int64_t ldu = 0;
  double* alpha_hist = nullptr;  // max_iter*t (device, required)
  double* beta_hist = nullptr;
  float* Z0 = nullptr;           // optional: P^{-1} B out (ld n_pad)
  double* rz0 = nullptr;         // optional device t: r0^T z0
  int* iters_dev = nullptr;      // device t
  double* relres_dev = nullptr;  // device t (true residual for the verified columns)
  // the first true_cols columns must meet tol by their true relative
  // residual ||B_c - K-hat U_c|| / ||B_c||, measured with one product of the
  // iterate once the recurrence has converged (0: recurrence only)
  int true_cols = 0;
  double* true_dev = nullptr;    // optional device true_cols: last measured true residuals
};
int mbcg_run(gp_ctx* ctx, const CgArgs& a, CgResult* res);
// Block CG on S^T K-hat S (AltBBMM, bcg.cu): B, Omega t <= 32 vectors (ld
// ldb / ldo); iters_out, relres_out host; stop_col < 0: stop when every
// column is below tol, else when column stop_col is.
int bcg_run(gp_ctx* ctx, const Prep& p, double s_out, double sigma2, const Precond& pc, const float* B,
            int64_t ldb, int t, double tol, int max_iter, int precision, float* Omega, int64_t ldo,
            int* iters_out, double* relres_out, int stop_col);
// Z = P^{-1} R for t vectors (ld ld), optional rz[c] += R_c . Z_c partials
int precond_apply(gp_ctx* ctx, const Precond* pc, int64_t n, const float* R,
                  float* Z, int64_t ld, int t, const int* active,
                  double* rz_out);

// ---- Lanczos quadrature ---------------------------------------------------------
// quad[c] = e1^T log(T_c) e1 for columns c0..c0+nc-1 of the histories.
int lanczos_quadrature(gp_ctx* ctx, const double* alpha_hist,
                       const double* beta_hist, int t, int c0, int nc,
                       const int* iters_dev, int max_iter, double* quad_dev,
                       int* bad_dev);

// ---- gradient -----------------------------------------------------------------
// G[j] (d_pad doubles) and gs (1 double) accumulated by the backward kernel
// for M_sym = 1/2 (U W^T + W U^T), U, W: T1 vectors of length n (ld n_pad).
// precision GP_FP32_SPLIT_TF32 with d_pad 32/64 and 2 T1 <= 64 runs the
// tensor-core backward (grad_tc.cu), otherwise the CUDA-core one.
int grad_tiles(gp_ctx* ctx, const Prep& p, const float* U, const float* W,
               int T1, double* G, double* gs, int precision);
bool grad_tc_supported(const Prep& p, int T1);
int grad_tc(gp_ctx* ctx, const Prep& p, const float* U, const float* W, int T1, double* G);

// ---- serving variances (love.cu) ---------------------------------------------------
int lanczos_cache_build(gp_ctx* ctx, const Prep& p, double s, double sigma2, int precision, const float* b,
                        int m, float* Q, int* m_out);
int cached_variance(gp_ctx* ctx, const gp_model* m, const Prep& mp, const Prep& q, float* var);
int block_ksum(gp_ctx* ctx, const Prep& q, double s, double* sums);
int row_sums(gp_ctx* ctx, const float* A, int64_t lda, int k, int64_t M, double* sums);
Prep model_prep_of(const gp_model* m);
int serve_batch(gp_ctx* ctx, const gp_model* m, const float* Xp, int64_t rows, float* mean, float* var, int nseg,
                const int64_t* seg, double* sums, int64_t max_part_rows);

// ---- small helpers (cg.cu) ------------------------------------------------------
// out[c] = sum_a A[c*ld + a] * B[c*ld + a] in FP64, c < t (device doubles)
int dot_columns(gp_ctx* ctx, const float* A, const float* B, int64_t ld,
                int64_t n, int t, double* out);
int probe_vectors(gp_ctx* ctx, const double* L, int64_t n, int k, double sigma2,
                  const double* resid, uint64_t seed, int n_probes, float* Z, int64_t ldz);
int copy_vectors(gp_ctx* ctx, const float* src, int64_t lds, float* dst,
                 int64_t ldd, int64_t n, int t, float scale);
// out = a X + b Y for t vectors of length n (common leading dimension ld);
// out may alias X or Y
int axpby_vectors(gp_ctx* ctx, float a, const float* X, float b, const float* Y, float* out,
                  int64_t ld, int64_t n, int t);

}  // namespace gp
