// kernels.h -- host launchers of the GB300 UoI kernels (internal interface).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

#include <nvtx3/nvToolsExt.h>

#include <optional>

#include <string>

namespace uoi {

// Detail text of the last error on this thread (uoi_get_last_error_detail).
extern thread_local std::string g_last_error;

// Checked build: throws UOI_ERR_BOUNDS if an index check fired (api.cu).
void check_bounds_status(cudaStream_t s);

// ---- per-kernel timing --------------------------------------------------------
// CUDA events recorded on the launch stream around the launches of the kernels
// that bound a fit (the tensor-core Gram and the ADMM x-update), with their
// algorithmic work.  Resolved after the fit's final synchronisation.
enum TimedKernel { TK_GRAM_TC = 0, TK_XUPDATE = 1, TK_COUNT = 2 };
struct KernelTotals { float ms = 0.f; int64_t launches = 0; double flops = 0.0; double bytes = 0.0; };
// A named range on the host timeline (NVTX), from construction to destruction: the
// stages of a fit, for profilers that group or filter kernels by range.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

void ktimer_reset();
void ktimer_begin(TimedKernel k, cudaStream_t s);
void ktimer_end(TimedKernel k, cudaStream_t s, double flops, double bytes);
void ktimer_credit(TimedKernel k, double ms, int64_t launches);   // work timed on another thread
void ktimer_add_work(TimedKernel k, double flops, double bytes);
KernelTotals ktimer_total(TimedKernel k);   // synchronises on the recorded events

// ---- memory ------------------------------------------------------------------
// Stream-ordered device buffer from the device's default memory pool.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    DevBuf() = default;
    DevBuf(size_t n, cudaStream_t s) { alloc(n, s); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
    DevBuf& operator=(DevBuf&& o) noexcept
    {
        release();
        ptr = o.ptr; bytes = o.bytes; stream = o.stream;
        o.ptr = nullptr; o.bytes = 0;
        return *this;
    }
    void alloc(size_t n, cudaStream_t s);
    void release();
    ~DevBuf() { release(); }
    template <typename T> T* as() const { return reinterpret_cast<T*>(ptr); }
};

// Allow `kern` the largest dynamic shared memory the current device opts in to (its
// static shared memory deducted).  Kernels launched with a size that varies by call
// use this, so that every caller sets the same value and concurrent callers on
// other streams cannot undercut each other.
void allow_max_dynamic_smem(const void* kern);
// A small pinned host buffer owned by the calling thread (allocated on first use,
// kept until exit): device-to-host polling without a pinned allocation and free
// (and their synchronisation) per call.
int32_t* pinned_scratch_i32();

// ---- G0: bootstrap indices (bootstrap.cu) -----------------------------------
// w[k*m + row] = multiplicity of the row in selection bootstrap k, k < B.
// block_mode 1: moving blocks (starts uniform on 0..m-L) instead of non-overlapping.
void selection_weights(int64_t m, int64_t block_len, PhiloxKey key, int32_t B, uint32_t* w,
                       cudaStream_t s, int32_t block_mode = 0);
// Training multiplicities and evaluation masks of estimation bootstraps k < B.
void estimation_weights(int64_t m, int64_t block_len, double train_frac, int split_fixed,
                        PhiloxKey key, int32_t B, uint32_t* w_train, uint8_t* eval,
                        cudaStream_t s);
// nk[k] = sum_t w[k*m + t] (as double), and eval counts when w is a mask.
void weight_sums(const uint32_t* w, const uint8_t* mask, int64_t m, int32_t B, double* nk,
                 cudaStream_t s);

// ---- G1: moments (gram.cu) ------------------------------------------------------
// For every k < B: G_k = X^T diag(w_k) X (p x p, full) and Bm_k = X^T diag(w_k) Y
// (p x r).  Exactly one of w (counts) and mask (0/1) may be non-null; both null
// means unweighted.  b_only = 1 skips G.  FP64 CUDA-core form.
void moments_fp64(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m,
                  int64_t p, int64_t r, const uint32_t* w, const uint8_t* mask, int32_t B,
                  double* G, double* Bm, int b_only, cudaStream_t s);
// moments_fp64 restricted to the nu X columns listed in cols, written into the
// p_out x p_out / p_out x r outputs at the original feature indices (other
// entries untouched).
void moments_fp64_cols(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t p_out,
                       int64_t r, int64_t nu, const int32_t* cols, const uint32_t* w, const uint8_t* mask,
                       int32_t B, double* G, double* Bm, cudaStream_t s);
// yy[k*r + e] = sum_t mask_k[t] Y[t,e]^2.
void masked_sumsq(const double* Y, int64_t ldy, int64_t m, int64_t r, const uint8_t* mask,
                  int32_t B, double* yy, cudaStream_t s);
// lambda_max = max |Bm| / m, then the descending log grid (Eq. 2 scaling).
void lambda_grid(const double* XtY, int64_t count, int64_t m, int32_t q, double ratio,
                 double* lambdas, cudaStream_t s);
// Device check: every value finite; flag[0] = 1 on the first non-finite.
void check_finite(const double* X, int64_t ldx, int64_t m, int64_t cols, int32_t* flag,
                  cudaStream_t s);

// Mixed form: split-bf16 tensor-core Gram (gram_tc.cu).
bool gram_tc_available();
// X32: optional FP32 copy of X (same leading dimension), read instead of X.
// lower_only: G's upper triangle is left unwritten (for a caller that reads the
// lower triangle alone, build_system_lower).
void moments_tc(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t p,
                int64_t r, const uint32_t* w, const uint8_t* mask, int32_t B, double* G,
                double* Bm, cudaStream_t s, const float* X32 = nullptr, bool lower_only = false);
// out[i*ldx + j] = X[i*ldx + j] rounded to FP32, i < m, j < p; with a flag, also
// *flag = 1 if any of those X entries is NaN or Inf (the same test as check_finite).
void to_f32(const double* X, int64_t ldx, int64_t m, int64_t p, float* out, cudaStream_t s,
            int32_t* flag = nullptr);

// Tensor-core moments restricted to the pz_x X columns listed in colmap (written
// into p_out x p_out / p_out x r outputs at the original feature indices).
void moments_tc_cols(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m,
                     int64_t p_out, int64_t r, int32_t pz_x, const int32_t* colmap,
                     const uint32_t* w, const uint8_t* mask, int32_t B, double* G, double* Bm,
                     cudaStream_t s, const float* X32 = nullptr, int64_t ld32 = 0,
                     bool x32_compact = false, bool lower_only = false);
// out[i*nu + t] = X32[i*ld + cols[t]]: the FP32 design restricted to the listed columns
// (X32_compact form for moments_tc_cols: column t of the copy is colmap[t] of X).
void gather_cols_f32(const float* X32, int64_t ld, int64_t m, const int32_t* cols, int64_t nu, float* out,
                     cudaStream_t s);

// ---- G3: factor (factor.cu) -------------------------------------------------------
// A_k = G_k / nk[k] + rho I in T, lower Cholesky in place.  status->code set to
// UOI_ERR_NOT_PD (where = k) on a non-positive pivot.
template <typename T>
void build_and_factor(const double* G, const double* nk, double rho, int64_t p, int32_t B,
                      T* A, DevStatus* status, cudaStream_t s);
// A_k = G_k / nk[k] + rho I in FP32 from the lower triangle of G_k alone (the
// upper triangle is not read); equal to build_system<float> on the mirrored G.
void build_system_lower(const double* G, const double* nk, double rho, int64_t p, int32_t B, float* A,
                        cudaStream_t s);
// The two halves of build_and_factor.
template <typename T>
void build_system(const double* G, const double* nk, double rho, int64_t p, int32_t B, T* A,
                  cudaStream_t s);
template <typename T>
void cholesky_inplace(T* A, int64_t p, int32_t B, DevStatus* status, cudaStream_t s);
// M_k = A_k^{-1} from the factor in the lower triangle of A (Linv: p x p scratch).
template <typename T>
void spd_inverse_from_factor(const T* L, int64_t p, int32_t B, T* Linv, T* M, cudaStream_t s);
// c_k[e][i] = (M_k Bm_k)[i][e] / nk[k].  rhs_scratch: B*p elements of T used for
// r == 1 (nullptr = a buffer from the device's memory pool).
template <typename T>
void rhs_from_inverse(const T* M, const double* Bm, const double* nk, int64_t p, int64_t r, int32_t B,
                      T* c, cudaStream_t s, T* rhs_scratch = nullptr);
// M_k = A_k^{-1} for SPD A_k (FP32, p x p each) by block Schur-complement recursion
// with FP32-accurate tensor-core GEMMs (gemm_tc.cu); A is left unchanged.  A batch
// of 8 or more runs as two halves side by side, on s and on the calling thread's
// side stream (the second half enqueued by a helper thread; not on the workers of
// a batch of fits); s waits for both.
bool inverse_tc_available();
void spd_inverse_tc(const float* A, int64_t p, int32_t G, float* M, DevStatus* status, cudaStream_t s);
// The calling host thread's second stream (estimate.cu).
cudaStream_t side_stream();
// M_k = A_k^{-1} from the factor L (lower triangle of A), then
// c_k[e][i] = (M_k Bm_k)[i][e] / nk[k].
template <typename T>
void inverse_and_rhs(const T* L, const double* Bm, const double* nk, int64_t p, int64_t r,
                     int32_t B, T* Linv, T* M, T* c, cudaStream_t s, T* rhs_scratch = nullptr);
// XtY[j*r + e] = sum_t X[t,j] Y[t,e] for few responses (split over rows, fixed order).
void xty_small(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t p,
               int64_t r, double* XtY, cudaStream_t s);

// ---- G4: ADMM (admm.cu) -------------------------------------------------------------
template <typename T>
struct AdmmProblem {
    int32_t G = 0;            // groups (bootstraps) sharing p
    int64_t p = 0, r = 0;     // features, response columns per group
    int32_t q = 0;            // lambdas
    const T* M = nullptr;     // G x p x p   (A_g^{-1}, symmetric)
    const T* c = nullptr;     // G x r x p   (A_g^{-1} b_ge / n_g)
    const double* lambdas = nullptr;   // q (device)
    double rho = 1.0, abs_tol = 1e-6, rel_tol = 1e-6;
    int32_t max_iter = 1000;
    int32_t warm = 1;         // 0 cold, 1 path
    // outputs, columns indexed ((g*q + j)*r + e)
    double* beta = nullptr;   // G x q x r x p (nullable)
    int32_t* iters = nullptr; // G x q x r     (nullable)
    uint8_t* conv = nullptr;  // G x q x r     (nullable)
    uint64_t* family = nullptr;   // q x r x W, AND of the supports (nullable, preset to ~0)
    double* u_out = nullptr;  // G x q x r x p final scaled dual (nullable)
    const float* z0 = nullptr;    // G x q x r x p initial z, cold schedule only (nullable)
    const float* u0 = nullptr;    // initial u, same layout
    // count of near-threshold features over all finished columns (nullable): the
    // margin |v_i| - lambda/rho of the final iterate (|z_i| where z_i != 0, |u_i| -
    // lambda/rho where z_i = 0, since v = z + u) lies within kNearThreshold of zero
    unsigned long long* near_count = nullptr;
};
// Half-width of the near-threshold band counted at column completion.
constexpr double kNearThreshold = 1e-6;
template <typename T>
void admm_solve(const AdmmProblem<T>& P, cudaStream_t s);
// Streaming schedule with the tensor-core x-update (FP32 state, p > resident limit).
bool admm_tc_available();
void admm_solve_tc(const AdmmProblem<float>& P, cudaStream_t s);
// Grouped solve of a batch of problems.  Each batch worker thread enters the batch
// before a fit and leaves it after; the fit's first tensor-core ADMM solve
// (admm_solve<float> past the resident schedule) joins the batch instead of
// running alone: its state is prepared on the worker's stream, a solver thread
// iterates it together with the other members (grouped launches replayed as CUDA
// graphs, tiles chosen by timing) and releases the worker once its columns have
// finished.  Each problem's iterates are those of its own solve.
struct AdmmBatch;
AdmmBatch* admm_batch_create(int32_t expected);
void admm_batch_destroy(AdmmBatch* b);
void admm_batch_enter(AdmmBatch* b);
void admm_batch_leave();
bool admm_batch_try_join(const AdmmProblem<float>& P, cudaStream_t s);
// Resident schedule only, with the caller's zeroed per-group chain counters
// (G int32).  Returns false (launching nothing) when p is too large for it.
template <typename T>
bool admm_solve_resident_with(const AdmmProblem<T>& P, int32_t* chain_next, cudaStream_t s);

// ---- G8: the warm-start network's hidden layers on tensor cores (mlp_tc.cu) --------
// C = A B^T over bf16 row-major operands (K contiguous), FP32 accumulation, fused
// epilogues.  width = 512 (a multiple of 256), rows of the batch M arbitrary.
bool mlp_tc_available();
// Hn = gelu(H W^T + b) (bf16, M x width), pre = H W^T + b (FP32, nullable), HnT (bf16,
// width x ldT, nullable) the transpose.
void mlp_forward_tc(const __nv_bfloat16* H, int64_t M, const __nv_bfloat16* W, int32_t width,
                    const float* bias, float* pre, __nv_bfloat16* Hn, __nv_bfloat16* HnT, int64_t ldT,
                    int32_t* err, cudaStream_t s);
// Inference through the last hidden layer and the head: h = gelu(H W^T + b) rounded
// to bf16, head_part[slot][m][j] = sum over the slot's 128 columns c of h[m][c] w4[j][c]
// (width / 128 slots, 3 outputs j; w4 is 3 x width bf16).  h is not stored.
void mlp_forward_head_tc(const __nv_bfloat16* H, int64_t M, const __nv_bfloat16* W, int32_t width,
                         const float* bias, const __nv_bfloat16* w4, float* head_part, int32_t* err, cudaStream_t s);
// dAp = (dA W) * gelu'(pre_prev) (bf16) with WT = W^T, dApT its transpose (nullable).
void mlp_backward_tc(const __nv_bfloat16* dA, int64_t M, const __nv_bfloat16* WT, int32_t width,
                     const float* pre_prev, __nv_bfloat16* dAp, __nv_bfloat16* dApT, int64_t ldT, int32_t* err,
                     cudaStream_t s);
// part[z] (width x width, FP32) = dA^T H over slice z of the rows, from the transposes
// dAT, HT (width x ld bf16, rows past `rows` zero).
void mlp_weight_grad_tc(const __nv_bfloat16* dAT, const __nv_bfloat16* HT, int64_t ld, int64_t rows, int32_t width,
                        int32_t slices, float* part, int32_t* err, cudaStream_t s);

// ---- G8: learned warm start (mlp.cu) ------------------------------------------------
struct WsModel;
WsModel* ws_create(uint64_t seed, cudaStream_t s);
void ws_destroy(WsModel* M);
int64_t ws_param_count();
void ws_set_params(WsModel* M, const float* params, cudaStream_t s);
void ws_get_params(WsModel* M, float* params, cudaStream_t s);
void ws_forward(WsModel* M, const float* X, int64_t N, float* out, cudaStream_t s);
double ws_loss_grad(WsModel* M, const float* X, const float* T, int64_t N, float* g, cudaStream_t s);
double ws_train(WsModel* M, const float* X, const float* T, int64_t N, int32_t epochs, int32_t batch,
                float lr, uint64_t seed, cudaStream_t s);
template <typename TC>
void ws_build_features(const double* G, const double* Bm, const double* nk, const TC* x0,
                       const double* lam, int32_t q, int64_t p, int64_t r, int32_t B, double rho,
                       const double* zt, const double* ut, float* F, float* T, cudaStream_t s);
void ws_start_state(const float* out, const float* F, const double* lam, int32_t q, int64_t p,
                    int64_t r, int64_t total, double rho, float* z0, float* u0, cudaStream_t s);
// u0 = (b/n_k - (G/n_k) z0) / rho for every column (the dual consistent with z0).
void ws_consistent_dual(const double* G, const double* Bm, const double* nk, const float* z0,
                        int64_t p, int64_t r, int32_t q, int32_t B, double rho, float* u0,
                        cudaStream_t s);
void ws_save(WsModel* M, const char* path);
WsModel* ws_load(const char* path, cudaStream_t s);

// ---- VAR(d) lagged design and the intercept (design.cu) ------------------------------
// Rows t - d, t = d..N-1, of Eq. 7-8 from the series S (N x p, time ascending):
// Y[i, :] = X_t, X[i, (j-1)p .. jp-1] = X_{t-j}, j = 1..d.
void lagged_design(const double* S, int64_t N, int64_t p, int32_t d, double* X, int64_t ldx,
                   double* Y, int64_t ldy, cudaStream_t s);
// xbar, ybar = unweighted column means of X (m x p) and Y (m x r); Xa (m x (p+1),
// contiguous) = [X - xbar, 1], Ya (m x r, contiguous) = Y - ybar.
void center_with_ones(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t p,
                      int64_t r, double* Xa, double* Ya, double* xbar, double* ybar, cudaStream_t s);
// Eliminates the ones coordinate (index p) from the (p+1)-column moments Ga, Ba of
// each of the B items: G = Ga[:p,:p] - g g^T / n_k, Bm = Ba[:p,:] - g Ba[p,:] / n_k,
// g = Ga[:p, p].  nk holds nk_count values (1 = shared by all items).
void schur_intercept(const double* Ga, const double* Ba, const double* nk, int nk_count, int64_t p,
                     int64_t r, int32_t B, double* G, double* Bm, cudaStream_t s);
// out (count x Wa words) = fam (count x W words) with bit `bit` set in every member.
void family_add_bit(const uint64_t* fam, int64_t count, int64_t W, int64_t Wa, int64_t bit,
                    uint64_t* out, cudaStream_t s);
// chosen: count rows of p + 1 (coefficients, then the intercept of the centred
// data); row c's intercept becomes ybar[c % r] + mu~ - xbar^T b.
void intercept_to_original(double* chosen, int64_t count, int64_t r, int64_t p, const double* xbar,
                           const double* ybar, cudaStream_t s);
// A (d x p x p), mu (p, nullable) from beta (p rows of d p + icpt): Alg. 2's partition.
void partition_var(const double* beta, int64_t p, int32_t d, int icpt, double* A, double* mu,
                   cudaStream_t s);

// ---- G5/G6/G7: supports, OLS, loss, bagging (estimate.cu) -----------------------------
void family_init(uint64_t* fam, int64_t words, cudaStream_t s);
// Union of all family supports as an increasing column list; returns its size.
int32_t union_columns(const uint64_t* family, int64_t count, int64_t p, int32_t* cols,
                      cudaStream_t s);
void family_mask_tail(uint64_t* fam, int64_t count, int64_t p, cudaStream_t s);
// losses[(k*q + j)*r + e] = held-out squared error sum of the OLS fit on support
// S_{j,e} from training moments (Gt, Bt) and evaluation moments (Ge, Be, yye);
// singular[...] = 1 where the fallback ran.  Solves use an FP32 factor with FP64
// iterative refinement (FP64-accurate), an FP64 factor for those it rejects
// (their number is returned).
int64_t ols_losses(const double* Gt, const double* Bt, const double* Ge, const double* Be,
                const double* yye, const uint64_t* family, int64_t p, int64_t r, int32_t q,
                int32_t B2, double* losses, int32_t* singular, cudaStream_t s);
// jstar[k] = argmin_j sum_e losses[k][j][e] (ties -> smallest j).
void loss_argmin(const double* losses, int32_t B2, int32_t q, int64_t r, int32_t* jstar,
                 cudaStream_t s);
// chosen[k][e][:] = OLS on S_{jstar[k], e} from (Gt_k, Bt_k), zero-filled.
int64_t ols_chosen(const double* Gt, const double* Bt, const uint64_t* family, const int32_t* jstar,
                int64_t p, int64_t r, int32_t q, int32_t B2, double* chosen, cudaStream_t s);
// beta_out[e][i] = median (bagging 0) or mean (1) over k of chosen[k][e][i].
void bagging(const double* chosen, int32_t B2, int64_t count, int32_t mode, double* out,
             cudaStream_t s);

}  // namespace uoi
