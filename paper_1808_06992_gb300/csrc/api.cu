// api.cu -- the C ABI (include/uoi.h) and the host orchestration of one fit.
//
// uoi_fit_traced runs Alg. 1 (r = 1) / Alg. 2 with order 1 (r = p) on one GPU:
//   lambda grid -> selection bootstraps (G0) -> moments (G1) -> factor (G3)
//   -> ADMM over all (bootstrap, equation, lambda) columns with the support
//   intersection fused into column completion (G4/G5) -> estimation bootstraps
//   -> training/evaluation moments -> OLS + held-out loss per (k, j, e) (G6)
//   -> argmin per bootstrap, chosen OLS, bagging (G7).
// Inputs may live on the host or the device; host data is copied in once.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"

namespace uoi {

thread_local int64_t g_launches = 0;
thread_local bool g_fit_in_batch = false;

void DevBuf::alloc(size_t n, cudaStream_t s)
{
    release();
    if (n == 0) n = 16;
    UOI_CUDA(cudaMallocAsync(&ptr, n, s));
    bytes = n;
    stream = s;
}

void DevBuf::release()
{
    if (ptr) cudaFreeAsync(ptr, stream);
    ptr = nullptr;
    bytes = 0;
}

thread_local std::string g_last_error;

namespace {
std::vector<DevStatus (*)()>& bounds_readers()
{
    static std::vector<DevStatus (*)()> readers;    // filled while the library loads
    return readers;
}
}  // namespace

void register_bounds_reader(DevStatus (*reader)()) { bounds_readers().push_back(reader); }

// Checked build: fail if an index check of any translation unit fired since the
// last call (the words are cleared as they are read).  Release build: nothing.
void check_bounds_status(cudaStream_t s)
{
#if defined(UOI_BOUNDS_CHECK) && UOI_BOUNDS_CHECK
    UOI_CUDA(cudaStreamSynchronize(s));
    for (auto rd : bounds_readers()) {
        const DevStatus h = rd();
        if (h.code != 0)
            throw Error(UOI_ERR_BOUNDS, "index check failed at site " + std::to_string(h.where) +
                                            " (checked build)");
    }
#else
    (void)s;
#endif
}

int32_t* pinned_scratch_i32()
{
    thread_local int32_t* buf = nullptr;
    if (!buf) UOI_CUDA(cudaMallocHost(&buf, 64 * sizeof(int32_t)));
    return buf;
}

void allow_max_dynamic_smem(const void* kern)
{
    int dev = 0, optin = 0;
    UOI_CUDA(cudaGetDevice(&dev));
    UOI_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    UOI_CUDA(cudaFuncGetAttributes(&fa, kern));
    UOI_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - (int)fa.sharedSizeBytes));
}

namespace {
struct PendingTimes {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    KernelTotals tot;
    cudaEvent_t open = nullptr;
    double extra_ms = 0.0;          // time measured elsewhere and credited to this thread
};
thread_local PendingTimes g_kt[TK_COUNT];   // per host thread, like the fit using it
}  // namespace

void ktimer_reset()
{
    for (auto& k : g_kt) {
        for (auto& e : k.ev) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
        k.ev.clear();
        k.tot = KernelTotals{};
        k.extra_ms = 0.0;
        if (k.open) { cudaEventDestroy(k.open); k.open = nullptr; }
    }
}

void ktimer_begin(TimedKernel k, cudaStream_t s)
{
    cudaEvent_t e;
    UOI_CUDA(cudaEventCreate(&e));
    UOI_CUDA(cudaEventRecord(e, s));
    g_kt[k].open = e;
}

void ktimer_end(TimedKernel k, cudaStream_t s, double flops, double bytes)
{
    cudaEvent_t e;
    UOI_CUDA(cudaEventCreate(&e));
    UOI_CUDA(cudaEventRecord(e, s));
    g_kt[k].ev.push_back({ g_kt[k].open, e });
    g_kt[k].open = nullptr;
    g_kt[k].tot.launches += 1;
    g_kt[k].tot.flops += flops;
    g_kt[k].tot.bytes += bytes;
}

void ktimer_credit(TimedKernel k, double ms, int64_t launches)
{
    g_kt[k].extra_ms += ms;
    g_kt[k].tot.launches += launches;
}

void ktimer_add_work(TimedKernel k, double flops, double bytes)
{
    g_kt[k].tot.flops += flops;
    g_kt[k].tot.bytes += bytes;
}

KernelTotals ktimer_total(TimedKernel k)
{
    KernelTotals t = g_kt[k].tot;
    t.ms = (float)g_kt[k].extra_ms;
    for (auto& e : g_kt[k].ev) {
        cudaEventSynchronize(e.second);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) t.ms += ms;
    }
    return t;
}

namespace {

void ensure_pool()
{
    int dev = 0;
    UOI_CUDA(cudaGetDevice(&dev));
    static bool done[64] = {};
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 64 && !done[dev]) {
        cudaMemPool_t pool;
        UOI_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
        uint64_t thr = UINT64_MAX;
        UOI_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
        done[dev] = true;
    }
}

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device view of a caller input: the pointer itself, or a copy of host data.
template <typename T>
const T* dev_in(const T* p, size_t count, DevBuf& hold, cudaStream_t s)
{
    if (!p) return nullptr;
    if (is_device_ptr(p)) return p;
    hold.alloc(sizeof(T) * count, s);
    UOI_CUDA(cudaMemcpyAsync(hold.ptr, p, sizeof(T) * count, cudaMemcpyHostToDevice, s));
    return hold.as<T>();
}

// Device destination for a caller output; finish() copies back host outputs.
template <typename T>
struct DevOut {
    T* user = nullptr;
    T* dev = nullptr;
    size_t count = 0;
    DevBuf hold;
    void init(T* p, size_t n, cudaStream_t s)
    {
        user = p;
        count = n;
        if (!p) { dev = nullptr; return; }
        if (is_device_ptr(p)) { dev = p; return; }
        hold.alloc(sizeof(T) * n, s);
        dev = hold.as<T>();
    }
    void finish(cudaStream_t s)
    {
        if (user && dev && dev != user)
            UOI_CUDA(cudaMemcpyAsync(user, dev, sizeof(T) * count, cudaMemcpyDeviceToHost, s));
    }
};

struct StageTimer {
    cudaStream_t s;
    std::vector<cudaEvent_t> ev;
    explicit StageTimer(cudaStream_t st) : s(st) {}
    int mark()
    {
        cudaEvent_t e;
        UOI_CUDA(cudaEventCreate(&e));
        UOI_CUDA(cudaEventRecord(e, s));
        ev.push_back(e);
        return (int)ev.size() - 1;
    }
    float ms(int a, int b)
    {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
    ~StageTimer()
    {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

void check_status(DevStatus* st, cudaStream_t s, const char* what)
{
    DevStatus h{};
    UOI_CUDA(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    if (h.code != 0)
        throw Error(h.code, std::string(what) + " failed on batch item " + std::to_string(h.where));
}

// prm->intercept, or 0 for a caller whose struct ends before that field.
int32_t param_intercept(const uoi_params* prm)
{
    if (prm->struct_size != 0 && prm->struct_size < offsetof(uoi_params, intercept) + sizeof(int32_t))
        return 0;
    return prm->intercept;
}

// prm->block_mode, or 0 for a caller whose struct ends before that field.
int32_t param_block_mode(const uoi_params* prm)
{
    if (prm->struct_size != 0 && prm->struct_size < offsetof(uoi_params, block_mode) + sizeof(int32_t))
        return 0;
    return prm->block_mode;
}

void validate(const uoi_params* prm)
{
    if (!prm) throw Error(UOI_ERR_INVALID_ARG, "params is NULL");
    if (prm->struct_size != 0 && prm->struct_size < offsetof(uoi_params, intercept))
        throw Error(UOI_ERR_INVALID_ARG, "uoi_params.struct_size too small");
    if (param_intercept(prm) != 0 && param_intercept(prm) != 1)
        throw Error(UOI_ERR_INVALID_ARG, "intercept must be 0 or 1");
    if (param_block_mode(prm) != UOI_BLOCKS_FIXED && param_block_mode(prm) != UOI_BLOCKS_MOVING)
        throw Error(UOI_ERR_INVALID_ARG, "unknown block mode");
    if (prm->B1 <= 0 || prm->B2 <= 0 || prm->q <= 0)
        throw Error(UOI_ERR_INVALID_ARG, "B1, B2 and q must be positive");
    if (!(prm->rho > 0.0)) throw Error(UOI_ERR_INVALID_ARG, "rho must be positive");
    if (prm->max_iter <= 0) throw Error(UOI_ERR_INVALID_ARG, "max_iter must be positive");
    if (!(prm->train_frac > 0.0 && prm->train_frac < 1.0))
        throw Error(UOI_ERR_INVALID_ARG, "train_frac must lie in (0, 1)");
    if (!(prm->abs_tol >= 0.0) || !(prm->rel_tol >= 0.0))
        throw Error(UOI_ERR_INVALID_ARG, "tolerances must be non-negative");
    if (prm->bagging != UOI_BAG_MEDIAN && prm->bagging != UOI_BAG_MEAN)
        throw Error(UOI_ERR_INVALID_ARG, "unknown bagging mode");
    if (prm->bagging == UOI_BAG_MEDIAN && prm->B2 > 128)
        throw Error(UOI_ERR_UNSUPPORTED, "median bagging supports B2 <= 128");
    if (prm->precision != UOI_PREC_FP64 && prm->precision != UOI_PREC_MIXED)
        throw Error(UOI_ERR_INVALID_ARG, "unknown precision");
    if (prm->warm_start != UOI_WARM_NONE && prm->warm_start != UOI_WARM_PATH &&
        prm->warm_start != UOI_WARM_LEARNED)
        throw Error(UOI_ERR_INVALID_ARG, "unknown warm start mode");
    if (prm->lambda_min_ratio <= 0.0 && !prm->lambdas)
        throw Error(UOI_ERR_INVALID_ARG, "lambda_min_ratio must be positive");
}

// Moments for B weight vectors in the precision of the fit.
// lower_only (tensor-core form): G's upper triangle may be left unwritten.
void moments(int precision, const double* X, int64_t ldx, const double* Y, int64_t ldy,
             int64_t m, int64_t p, int64_t r, const uint32_t* w, const uint8_t* mask, int32_t B,
             double* G, double* Bm, cudaStream_t s, const float* X32 = nullptr, bool lower_only = false)
{
    if (precision == UOI_PREC_MIXED && gram_tc_available())
        moments_tc(X, ldx, Y, ldy, m, p, r, w, mask, B, G, Bm, s, X32, lower_only);
    else
        moments_fp64(X, ldx, Y, ldy, m, p, r, w, mask, B, G, Bm, 0, s);
}

template <typename T>
void selection_admm(int precision, const double* Xd, int64_t ldx, const double* Yd, int64_t ldy,
                    int64_t m, int64_t p, int64_t r, const uint32_t* w, int32_t B,
                    const double* lam, int32_t q, double rho, double abs_tol, double rel_tol,
                    int32_t max_iter, int32_t warm, double* beta, int32_t* iters, uint8_t* conv,
                    uint64_t* family, cudaStream_t s, StageTimer* tm, int* marks, bool icpt,
                    WsModel* ws = nullptr, const float* X32 = nullptr,
                    unsigned long long* near_count = nullptr)
{
    int t0 = tm ? tm->mark() : 0;
    std::optional<NvtxRange> stage;
    stage.emplace("uoi:selection:moments");
    // mixed form, large p: the block inverse on tensor cores; when nothing but the
    // FP32 system reads G (no intercept elimination, no learned start), the Gram's
    // lower triangle is enough and the system is built from it
    bool tc_inverse = false;
    if constexpr (sizeof(T) == 4) tc_inverse = p >= 512 && inverse_tc_available();
    const bool lower_only = tc_inverse && !icpt && !ws && precision == UOI_PREC_MIXED && gram_tc_available();
    DevBuf G(sizeof(double) * (size_t)(B * p * p), s), Bm(sizeof(double) * (size_t)(B * p * r), s);
    DevBuf nk(sizeof(double) * B, s);
    if (w) {
        weight_sums(w, nullptr, m, B, nk.as<double>(), s);
    } else {
        const double mm = (double)m;
        UOI_CUDA(cudaMemcpyAsync(nk.ptr, &mm, sizeof(double), cudaMemcpyHostToDevice, s));
    }
    if (icpt) {
        // moments of [X~ 1] (column p = ones), then the ones coordinate eliminated:
        // the moments of the bootstrap-weighted centred data
        const int64_t pa = p + 1;
        DevBuf Ga(sizeof(double) * (size_t)(B * pa * pa), s), Ba(sizeof(double) * (size_t)(B * pa * r), s);
        moments(precision, Xd, ldx, Yd, ldy, m, pa, r, w, nullptr, B, Ga.as<double>(), Ba.as<double>(), s,
                X32);
        schur_intercept(Ga.as<double>(), Ba.as<double>(), nk.as<double>(), w ? B : 1, p, r, B, G.as<double>(),
                        Bm.as<double>(), s);
    } else {
        moments(precision, Xd, ldx, Yd, ldy, m, p, r, w, nullptr, B, G.as<double>(), Bm.as<double>(), s, X32,
                lower_only);
    }
    int t1 = tm ? tm->mark() : 0;
    stage.reset();
    stage.emplace("uoi:selection:factor");
    DevBuf st(sizeof(DevStatus), s);
    UOI_CUDA(cudaMemsetAsync(st.ptr, 0, st.bytes, s));
    DevBuf A(sizeof(T) * (size_t)(B * p * p), s);
    DevBuf M(sizeof(T) * (size_t)(B * p * p), s);
    DevBuf c(sizeof(T) * (size_t)(B * p * r), s);
    if constexpr (sizeof(T) == 4) {
        // mixed form, large p: block inverse with tensor-core GEMMs
        if (tc_inverse) {
            if (lower_only)
                build_system_lower(G.as<double>(), nk.as<double>(), rho, p, B, A.as<float>(), s);
            else
                build_system<float>(G.as<double>(), nk.as<double>(), rho, p, B, A.as<float>(), s);
            if (!ws) G.release();
            spd_inverse_tc(A.as<float>(), p, B, M.as<float>(), st.as<DevStatus>(), s);
            check_status(st.as<DevStatus>(), s, "inverse of G/n + rho I");
            rhs_from_inverse<float>(M.as<float>(), Bm.as<double>(), nk.as<double>(), p, r, B, c.as<float>(), s);
        }
    }
    if (!tc_inverse) {
        build_and_factor<T>(G.as<double>(), nk.as<double>(), rho, p, B, A.as<T>(), st.as<DevStatus>(), s);
        if (!ws) G.release();
        check_status(st.as<DevStatus>(), s, "Cholesky of G/n + rho I");
        DevBuf Linv(sizeof(T) * (size_t)(B * p * p), s);
        inverse_and_rhs<T>(A.as<T>(), Bm.as<double>(), nk.as<double>(), p, r, B, Linv.as<T>(),
                           M.as<T>(), c.as<T>(), s);
    }
    A.release();
    // learned warm start: predicted z for every column, the dual consistent with
    // it, then the cold schedule from that state
    DevBuf z0, u0;
    if (ws) {
        const int64_t rows = (int64_t)B * q * r * p;
        DevBuf F(sizeof(float) * (size_t)rows * 8, s), out(sizeof(float) * (size_t)rows * 3, s);
        ws_build_features<T>(G.as<double>(), Bm.as<double>(), nk.as<double>(), c.as<T>(), lam, q, p,
                             r, B, rho, nullptr, nullptr, F.as<float>(), nullptr, s);
        ws_forward(ws, F.as<float>(), rows, out.as<float>(), s);
        z0.alloc(sizeof(float) * (size_t)rows, s);
        u0.alloc(sizeof(float) * (size_t)rows, s);
        ws_start_state(out.as<float>(), F.as<float>(), lam, q, p, r, rows, rho, z0.as<float>(),
                       u0.as<float>(), s);
        ws_consistent_dual(G.as<double>(), Bm.as<double>(), nk.as<double>(), z0.as<float>(), p, r, q,
                           B, rho, u0.as<float>(), s);
        G.release();
    }
    int t2 = tm ? tm->mark() : 0;
    stage.reset();
    stage.emplace("uoi:selection:admm");
    AdmmProblem<T> P;
    P.G = B; P.p = p; P.r = r; P.q = q;
    P.M = M.as<T>(); P.c = c.as<T>(); P.lambdas = lam;
    P.rho = rho; P.abs_tol = abs_tol; P.rel_tol = rel_tol; P.max_iter = max_iter;
    P.warm = ws ? 0 : (warm == UOI_WARM_LEARNED ? 1 : warm);
    P.beta = beta; P.iters = iters; P.conv = conv; P.family = family;
    P.near_count = near_count;
    if (ws) { P.z0 = z0.as<float>(); P.u0 = u0.as<float>(); }
    admm_solve<T>(P, s);
    int t3 = tm ? tm->mark() : 0;
    if (marks) { marks[0] = t0; marks[1] = t1; marks[2] = t2; marks[3] = t3; }
}

struct IterStats {
    int64_t cols = 0, noncon = 0, iters = 0, group_iters = 0;
    int32_t maxit = 0;
    int64_t hist[8] = { 0, 0, 0, 0, 0, 0, 0, 0 };   // uoi_diag.admm_iter_hist
};

// Column statistics; group_iters = sum over groups of the iterations during which
// the group had an active column (a path chain runs its lambdas back to back).
IterStats iteration_stats(const int32_t* iters_d, const uint8_t* conv_d, int64_t n, cudaStream_t s,
                          int32_t G = 0, int32_t q = 0, int64_t r = 0, int32_t warm = 0)
{
    std::vector<int32_t> it((size_t)n);
    std::vector<uint8_t> cv((size_t)n);
    UOI_CUDA(cudaMemcpyAsync(it.data(), iters_d, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaMemcpyAsync(cv.data(), conv_d, n, cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    IterStats st;
    st.cols = n;
    for (int64_t i = 0; i < n; ++i) {
        st.iters += it[i];
        st.maxit = std::max(st.maxit, it[i]);
        st.noncon += cv[i] ? 0 : 1;
        int b = 7;                                  // stopped at max_iter without converging
        if (cv[i]) {
            b = 0;
            while (b < 6 && it[i] > (16 << b)) ++b;  // <= 16, <= 32, ..., <= 512, > 512
        }
        st.hist[b] += 1;
    }
    if (G > 0 && (int64_t)G * q * r == n) {
        for (int32_t g = 0; g < G; ++g) {
            int64_t longest = 0;
            if (warm) {
                for (int64_t e = 0; e < r; ++e) {
                    int64_t chain = 0;
                    for (int32_t j = 0; j < q; ++j) chain += it[((int64_t)g * q + j) * r + e];
                    longest = std::max(longest, chain);
                }
            } else {
                for (int64_t c = 0; c < (int64_t)q * r; ++c)
                    longest = std::max<int64_t>(longest, it[(int64_t)g * q * r + c]);
            }
            st.group_iters += longest;
        }
    }
    return st;
}

// Warm-start weights loaded from a file, cached by path for the process.
struct WsCache {
    std::string path;
    WsModel* model = nullptr;
};
thread_local WsCache g_ws_cache;          // per host thread (batch workers load their own)

WsModel* ws_for_path(const char* path, cudaStream_t s)
{
    if (!path || !*path) return nullptr;
    if (g_ws_cache.model && g_ws_cache.path == path) return g_ws_cache.model;
    WsModel* m = nullptr;
    try {
        m = ws_load(path, s);
    } catch (const Error&) {
        return nullptr;                        // unusable weights: path warm start instead
    }
    if (g_ws_cache.model) ws_destroy(g_ws_cache.model);
    g_ws_cache.model = m;
    g_ws_cache.path = path;
    return m;
}

int fit_core(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t p,
             int64_t r, const uoi_params* prm, double* beta_out, uoi_trace* tr, uoi_diag* diag,
             const double* shared_series = nullptr, int64_t series_count = 0)
{
    validate(prm);
    if (!X || !Y || !beta_out) throw Error(UOI_ERR_INVALID_ARG, "NULL data pointer");
    if (m <= 0 || p <= 0 || r <= 0) throw Error(UOI_ERR_INVALID_ARG, "sizes must be positive");
    if (prm->block_len > m) throw Error(UOI_ERR_INVALID_ARG, "block_len exceeds the number of rows");
    ensure_pool();
    cudaStream_t s = (cudaStream_t)prm->stream;
    const int64_t launches0 = g_launches;
    ktimer_reset();
    StageTimer tm(s);
    NvtxRange fit_range("uoi:fit");
    const int tstart = tm.mark();
    const int32_t B1 = prm->B1, B2 = prm->B2, q = prm->q;
    const int64_t W = (p + 63) / 64;
    const bool mixed = prm->precision == UOI_PREC_MIXED;
    const bool tc_moments = mixed && gram_tc_available();   // one decision for the whole fit

    // inputs (the VAR series is copied once; X and Y are views into it)
    DevBuf hx, hy;
    const double* Xd;
    const double* Yd;
    if (shared_series) {
        const double* sd = dev_in(shared_series, (size_t)series_count, hx, s);
        Xd = sd + (X - shared_series);
        Yd = sd + (Y - shared_series);
    } else {
        Xd = dev_in(X, (size_t)((m - 1) * ldx + p), hx, s);
        Yd = dev_in(Y, (size_t)((m - 1) * ldy + r), hy, s);
    }
    // mixed form: one FP32 copy of X feeds every tensor-core moment pass; without an
    // intercept (X used as given) it is made here, in the same pass as X's check
    DevBuf X32;
    {
        DevBuf flag(sizeof(int32_t), s);
        UOI_CUDA(cudaMemsetAsync(flag.ptr, 0, sizeof(int32_t), s));
        if (tc_moments && param_intercept(prm) == 0) {
            X32.alloc(sizeof(float) * (size_t)(m * ldx), s);
            to_f32(Xd, ldx, m, p, X32.as<float>(), s, flag.as<int32_t>());
        } else {
            check_finite(Xd, ldx, m, p, flag.as<int32_t>(), s);
        }
        check_finite(Yd, ldy, m, r, flag.as<int32_t>(), s);
        int32_t h = 0;
        UOI_CUDA(cudaMemcpyAsync(&h, flag.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        UOI_CUDA(cudaStreamSynchronize(s));
        if (h) throw Error(UOI_ERR_NONFINITE, "X or Y holds NaN or Inf");
    }
    const PhiloxKey key{ prm->seed, prm->problem_id };

    // intercept: the design centred by its column means with a ones column
    // appended (index p), the responses centred; xbar, ybar map mu back
    const bool icpt = param_intercept(prm) != 0;
    const int64_t pe = p + (icpt ? 1 : 0);            // estimation coordinates
    DevBuf xa, ya, xbar, ybar;
    if (icpt) {
        xa.alloc(sizeof(double) * (size_t)(m * pe), s);
        ya.alloc(sizeof(double) * (size_t)(m * r), s);
        xbar.alloc(sizeof(double) * (size_t)p, s);
        ybar.alloc(sizeof(double) * (size_t)r, s);
        center_with_ones(Xd, ldx, Yd, ldy, m, p, r, xa.as<double>(), ya.as<double>(), xbar.as<double>(),
                         ybar.as<double>(), s);
        Xd = xa.as<double>();
        ldx = pe;
        Yd = ya.as<double>();
        ldy = r;
    }

    // lambda grid
    DevBuf lam(sizeof(double) * q, s), lam_hold;
    if (prm->lambdas) {
        const double* ld = dev_in(prm->lambdas, (size_t)q, lam_hold, s);
        UOI_CUDA(cudaMemcpyAsync(lam.ptr, ld, sizeof(double) * q, cudaMemcpyDeviceToDevice, s));
    } else {
        DevBuf xty(sizeof(double) * (size_t)(p * r), s);
        if (r <= 4)
            xty_small(Xd, ldx, Yd, ldy, m, p, r, xty.as<double>(), s);
        else
            moments_fp64(Xd, ldx, Yd, ldy, m, p, r, nullptr, nullptr, 1, nullptr, xty.as<double>(), 1, s);
        lambda_grid(xty.as<double>(), p * r, m, q, prm->lambda_min_ratio, lam.as<double>(), s);
    }

    // ---- selection ----
    const int t_sel0 = tm.mark();
    std::optional<NvtxRange> phase;
    phase.emplace("uoi:selection");
    DevBuf wsel(sizeof(uint32_t) * (size_t)(B1 * m), s);
    selection_weights(m, prm->block_len, key, B1, wsel.as<uint32_t>(), s, param_block_mode(prm));
    const int t_sel1 = tm.mark();
    const int64_t ncol = (int64_t)B1 * q * r;
    DevOut<double> sel_beta;
    sel_beta.init(tr ? tr->sel_beta : nullptr, (size_t)(ncol * p), s);
    DevBuf iters_b(sizeof(int32_t) * ncol, s), conv_b(ncol, s);
    DevBuf fam(sizeof(uint64_t) * (size_t)(q * r * W), s);
    family_init(fam.as<uint64_t>(), q * r * W, s);
    DevBuf near_b(sizeof(unsigned long long), s);
    UOI_CUDA(cudaMemsetAsync(near_b.ptr, 0, near_b.bytes, s));
    int marks[4] = { 0, 0, 0, 0 };
    WsModel* ws = prm->warm_start == UOI_WARM_LEARNED ? ws_for_path(prm->mlp_weights_path, s) : nullptr;
    const int32_t warm_used = prm->warm_start == UOI_WARM_LEARNED ? (ws ? UOI_WARM_LEARNED : UOI_WARM_PATH)
                                                                  : prm->warm_start;
    if (tc_moments && !X32.ptr) {                   // with an intercept: the centred design
        X32.alloc(sizeof(float) * (size_t)(m * ldx), s);
        to_f32(Xd, ldx, m, pe, X32.as<float>(), s);
    }
    if (mixed)
        selection_admm<float>(prm->precision, Xd, ldx, Yd, ldy, m, p, r, wsel.as<uint32_t>(), B1,
                              lam.as<double>(), q, prm->rho, prm->abs_tol, prm->rel_tol,
                              prm->max_iter, prm->warm_start, sel_beta.dev, iters_b.as<int32_t>(),
                              conv_b.as<uint8_t>(), fam.as<uint64_t>(), s, &tm, marks, icpt, ws,
                              X32.ptr ? X32.as<float>() : nullptr, near_b.as<unsigned long long>());
    else
        selection_admm<double>(prm->precision, Xd, ldx, Yd, ldy, m, p, r, wsel.as<uint32_t>(), B1,
                               lam.as<double>(), q, prm->rho, prm->abs_tol, prm->rel_tol,
                               prm->max_iter, prm->warm_start, sel_beta.dev, iters_b.as<int32_t>(),
                               conv_b.as<uint8_t>(), fam.as<uint64_t>(), s, &tm, marks, icpt, ws,
                               nullptr, near_b.as<unsigned long long>());
    family_mask_tail(fam.as<uint64_t>(), q * r, p, s);
    const int t_sel2 = tm.mark();
    phase.reset();
    phase.emplace("uoi:estimation");

    // ---- estimation ----
    // with an intercept every support also holds the ones column (index p)
    DevBuf fam_e;
    const uint64_t* fe = fam.as<uint64_t>();
    if (icpt) {
        const int64_t We = (pe + 63) / 64;
        fam_e.alloc(sizeof(uint64_t) * (size_t)(q * r * We), s);
        family_add_bit(fam.as<uint64_t>(), q * r, W, We, p, fam_e.as<uint64_t>(), s);
        fe = fam_e.as<uint64_t>();
    }
    DevBuf west(sizeof(uint32_t) * (size_t)(B2 * m), s), evm((size_t)(B2 * m), s);
    estimation_weights(m, prm->block_len, prm->train_frac, prm->split_mode, key, B2,
                       west.as<uint32_t>(), evm.as<uint8_t>(), s);
    DevBuf Gt(sizeof(double) * (size_t)(B2 * pe * pe), s), Bt(sizeof(double) * (size_t)(B2 * pe * r), s);
    DevBuf Ge(sizeof(double) * (size_t)(B2 * pe * pe), s), Be(sizeof(double) * (size_t)(B2 * pe * r), s);
    DevBuf yye(sizeof(double) * (size_t)(B2 * r), s);
    if (tc_moments) {
        // OLS on S_j only touches features in the union U of the family, so the
        // estimation moments are formed on U alone.
        DevBuf ucols(sizeof(int32_t) * (size_t)pe, s);
        const int32_t nu = union_columns(fe, q * r, pe, ucols.as<int32_t>(), s);
        if (nu > 0) {
            // the design restricted to U once, so both passes read contiguous rows
            DevBuf Xu(sizeof(float) * (size_t)(m * nu), s);
            gather_cols_f32(X32.as<float>(), ldx, m, ucols.as<int32_t>(), nu, Xu.as<float>(), s);
            moments_tc_cols(Xd, ldx, Yd, ldy, m, pe, r, nu, ucols.as<int32_t>(), west.as<uint32_t>(),
                            nullptr, B2, Gt.as<double>(), Bt.as<double>(), s, Xu.as<float>(), nu, true);
            moments_tc_cols(Xd, ldx, Yd, ldy, m, pe, r, nu, ucols.as<int32_t>(), nullptr,
                            evm.as<uint8_t>(), B2, Ge.as<double>(), Be.as<double>(), s, Xu.as<float>(), nu,
                            true);
        }
    } else {
        // FP64 form: the same restriction to U, on the CUDA cores
        DevBuf ucols(sizeof(int32_t) * (size_t)pe, s);
        const int32_t nu = union_columns(fe, q * r, pe, ucols.as<int32_t>(), s);
        moments_fp64_cols(Xd, ldx, Yd, ldy, m, pe, r, nu, ucols.as<int32_t>(), west.as<uint32_t>(), nullptr, B2,
                          Gt.as<double>(), Bt.as<double>(), s);
        moments_fp64_cols(Xd, ldx, Yd, ldy, m, pe, r, nu, ucols.as<int32_t>(), nullptr, evm.as<uint8_t>(), B2,
                          Ge.as<double>(), Be.as<double>(), s);
    }
    masked_sumsq(Yd, ldy, m, r, evm.as<uint8_t>(), B2, yye.as<double>(), s);
    const int t_est1 = tm.mark();
    DevOut<double> loss_o;
    DevBuf loss_b;
    loss_o.init(tr ? tr->est_loss : nullptr, (size_t)(B2 * q * r), s);
    double* losses = loss_o.dev;
    if (!losses) { loss_b.alloc(sizeof(double) * (size_t)(B2 * q * r), s); losses = loss_b.as<double>(); }
    DevBuf sing(sizeof(int32_t) * (size_t)(B2 * q * r), s);
    int64_t n_ols64 = ols_losses(Gt.as<double>(), Bt.as<double>(), Ge.as<double>(), Be.as<double>(), yye.as<double>(),
               fe, pe, r, q, B2, losses, sing.as<int32_t>(), s);
    DevBuf jst(sizeof(int32_t) * B2, s);
    loss_argmin(losses, B2, q, r, jst.as<int32_t>(), s);
    DevBuf chosen(sizeof(double) * (size_t)(B2 * r * pe), s);
    n_ols64 += ols_chosen(Gt.as<double>(), Bt.as<double>(), fe, jst.as<int32_t>(), pe, r, q, B2,
               chosen.as<double>(), s);
    if (icpt)
        intercept_to_original(chosen.as<double>(), (int64_t)B2 * r, r, p, xbar.as<double>(), ybar.as<double>(),
                              s);
    DevOut<double> bo;
    bo.init(beta_out, (size_t)(r * pe), s);
    bagging(chosen.as<double>(), B2, r * pe, prm->bagging, bo.dev, s);
    const int t_end = tm.mark();
    phase.reset();

    // ---- outputs ----
    bo.finish(s);
    if (tr) {
        auto copy_out = [&](void* dst, const void* src, size_t bytes) {
            if (!dst) return;
            UOI_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
        };
        copy_out(tr->lambdas, lam.ptr, sizeof(double) * q);
        copy_out(tr->sel_weights, wsel.ptr, sizeof(uint32_t) * (size_t)(B1 * m));
        copy_out(tr->est_weights, west.ptr, sizeof(uint32_t) * (size_t)(B2 * m));
        copy_out(tr->est_eval, evm.ptr, (size_t)(B2 * m));
        copy_out(tr->sel_iters, iters_b.ptr, sizeof(int32_t) * ncol);
        copy_out(tr->sel_conv, conv_b.ptr, (size_t)ncol);
        copy_out(tr->family, fam.ptr, sizeof(uint64_t) * (size_t)(q * r * W));
        copy_out(tr->est_jstar, jst.ptr, sizeof(int32_t) * B2);
        copy_out(tr->est_beta, chosen.ptr, sizeof(double) * (size_t)(B2 * r * pe));
        copy_out(tr->est_singular, sing.ptr, sizeof(int32_t) * (size_t)(B2 * q * r));
        sel_beta.finish(s);
        loss_o.finish(s);
    }
    UOI_CUDA(cudaStreamSynchronize(s));
    IterStats its = iteration_stats(iters_b.as<int32_t>(), conv_b.as<uint8_t>(), ncol, s, B1, q, r,
                                    warm_used == UOI_WARM_PATH ? 1 : 0);
    {
        // algorithmic work of the streaming x-update: 2 p^2 flops per active
        // column-iteration; M once per group-iteration plus the c, z, u, V reads
        // and z, u, V writes of each active column-iteration
        const double tsz = mixed ? 4.0 : 8.0;
        ktimer_add_work(TK_XUPDATE, 2.0 * (double)p * p * (double)its.iters,
                        (double)its.group_iters * p * p * tsz + 7.0 * p * tsz * (double)its.iters);
    }
    std::vector<int32_t> sg((size_t)(B2 * q * r));
    UOI_CUDA(cudaMemcpyAsync(sg.data(), sing.ptr, sizeof(int32_t) * sg.size(), cudaMemcpyDeviceToHost, s));
    unsigned long long near_h = 0;
    UOI_CUDA(cudaMemcpyAsync(&near_h, near_b.ptr, sizeof(near_h), cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    int64_t nsing = 0;
    for (auto v : sg) nsing += v;
    if (diag) {
        diag->ms_total = tm.ms(tstart, t_end);
        diag->ms_bootstrap = tm.ms(t_sel0, t_sel1);
        diag->ms_gram = tm.ms(marks[0], marks[1]);
        diag->ms_factor = tm.ms(marks[1], marks[2]);
        diag->ms_admm = tm.ms(marks[2], marks[3]);
        // supports are taken at ADMM column completion (ballot bitsets ANDed into the
        // family); what remains after the ADMM launches is the family's tail mask
        diag->ms_support = tm.ms(marks[3], t_sel2);
        diag->ms_estimation = tm.ms(t_sel2, t_end);
        (void)t_est1;
        diag->admm_columns = its.cols;
        diag->admm_nonconverged = its.noncon;
        diag->admm_iterations = its.iters;
        diag->admm_max_iterations = its.maxit;
        diag->ols_singular = nsing;
        diag->gpu_launches = g_launches - launches0;
        if (diag->struct_size == 0 || diag->struct_size >= offsetof(uoi_diag, ols_fp64) + sizeof(int64_t)) {
            const KernelTotals g = ktimer_total(TK_GRAM_TC), x = ktimer_total(TK_XUPDATE);
            diag->ms_gram_tc = g.ms;
            diag->n_gram_tc = g.launches;
            diag->flops_gram_tc = g.flops;
            diag->ms_xupdate = x.ms;
            diag->n_xupdate = x.launches;
            diag->flops_xupdate = x.flops;
            diag->bytes_xupdate = x.bytes;
            diag->warm_start_used = warm_used;
            diag->ols_fp64 = n_ols64;
        }
        if (diag->struct_size == 0 || diag->struct_size >= offsetof(uoi_diag, admm_iter_hist) + sizeof(diag->admm_iter_hist)) {
            diag->admm_near_threshold = (int64_t)near_h;
            for (int b = 0; b < 8; ++b) diag->admm_iter_hist[b] = its.hist[b];
        }
    }
    check_bounds_status(s);
    return (its.noncon > 0 || nsing > 0) ? UOI_OK_WITH_WARNINGS : UOI_OK;
}

template <typename F>
int guarded(F&& f)
{
    try {
        g_last_error.clear();
        return f();
    } catch (const Error& e) {
        g_last_error = e.what();
        return e.status;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return UOI_ERR_OOM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return UOI_ERR_CUDA;
    } catch (...) {
        g_last_error = "unknown error";
        return UOI_ERR_CUDA;
    }
}

}  // namespace
}  // namespace uoi

using namespace uoi;

extern "C" {

void uoi_params_default(uoi_params* prm)
{
    if (!prm) return;
    std::memset(prm, 0, sizeof(*prm));
    prm->struct_size = sizeof(uoi_params);
    prm->B1 = 20; prm->B2 = 20; prm->q = 16;
    prm->lambda_min_ratio = 1e-3;
    prm->rho = 1.0; prm->abs_tol = 1e-6; prm->rel_tol = 1e-6; prm->max_iter = 1000;
    prm->train_frac = 0.8;
    prm->bagging = UOI_BAG_MEDIAN;
    prm->split_mode = UOI_SPLIT_PER_BOOTSTRAP;
    prm->precision = UOI_PREC_FP64;
    prm->warm_start = UOI_WARM_PATH;
}

int uoi_fit_traced(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m,
                   int64_t p, int64_t r, const uoi_params* prm, double* beta_out, uoi_trace* trace,
                   uoi_diag* diag)
{
    return guarded([&] { return fit_core(X, ldx, Y, ldy, m, p, r, prm, beta_out, trace, diag); });
}

int uoi_lasso_fit(const double* X, const double* y, int64_t n, int64_t p, const uoi_params* prm,
                  double* beta_out, uint64_t* family_out, uoi_diag* diag)
{
    return guarded([&] {
        if (prm && param_intercept(prm))
            throw Error(UOI_ERR_UNSUPPORTED, "uoi_lasso_fit has no output for an intercept (use uoi_fit_traced)");
        uoi_trace tr;
        std::memset(&tr, 0, sizeof(tr));
        tr.family = family_out;
        return fit_core(X, p, y, 1, n, p, 1, prm, beta_out, family_out ? &tr : nullptr, diag);
    });
}

int uoi_lasso_fit_batch(int32_t count, const double* const* X, const double* const* y, const int64_t* n,
                        const int64_t* p, const uoi_params* prm, double* const* beta_out, int32_t* status_out,
                        uoi_diag* diags, int32_t streams)
{
    return guarded([&] {
        if (count < 0) throw uoi::Error(UOI_ERR_INVALID_ARG, "count must be >= 0");
        if (count == 0) return (int)UOI_OK;
        if (!X || !y || !n || !p || !prm || !beta_out)
            throw uoi::Error(UOI_ERR_INVALID_ARG, "NULL array argument");
        if (prm->lambdas) throw uoi::Error(UOI_ERR_INVALID_ARG, "a batch takes each problem's own lambda grid");
        if (uoi::param_intercept(prm))
            throw uoi::Error(UOI_ERR_UNSUPPORTED, "the batch has no output for an intercept");
        uoi::validate(prm);
        int dev = 0;
        UOI_CUDA(cudaGetDevice(&dev));
        // largest problems first (n p^2 orders the Gram and the inverse)
        std::vector<int32_t> order((size_t)count);
        for (int32_t i = 0; i < count; ++i) order[(size_t)i] = i;
        std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            return (double)n[a] * p[a] * p[a] > (double)n[b] * p[b] * p[b];
        });
        // streams > 0: that many workers, each fitting one problem at a time.
        // streams == 0 (grouped): one worker per problem, in waves of at most kWave
        // problems, and the selection solves of the problems that reach the
        // tensor-core ADMM iterate together (AdmmBatch).
        constexpr int32_t kWave = 128;
        const bool grouped = streams == 0;
        std::vector<int32_t> st((size_t)count, UOI_OK);
        std::vector<std::string> detail((size_t)count);
        std::atomic<int32_t> next(0);
        int32_t wave_end = count;
        uoi::AdmmBatch* batch = nullptr;
        auto worker = [&]() {
            cudaSetDevice(dev);
            uoi::g_fit_in_batch = true;
            cudaStream_t ws = nullptr;
            if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
                for (int32_t t; (t = next.fetch_add(1)) < wave_end;) {
                    st[(size_t)order[(size_t)t]] = UOI_ERR_CUDA;
                    if (batch) {                  // the batch counts every problem once
                        uoi::admm_batch_enter(batch);
                        uoi::admm_batch_leave();
                    }
                }
                return;
            }
            for (int32_t t; (t = next.fetch_add(1)) < wave_end;) {
                const int32_t i = order[(size_t)t];
                uoi_params q = *prm;
                q.stream = ws;
                q.problem_id = prm->problem_id + (uint64_t)i;
                if (batch) uoi::admm_batch_enter(batch);
                st[(size_t)i] = uoi::guarded([&] {
                    return uoi::fit_core(X[i], p[i], y[i], 1, n[i], p[i], 1, &q, beta_out[i], nullptr,
                                         diags ? &diags[i] : nullptr);
                });
                if (st[(size_t)i] < 0) detail[(size_t)i] = uoi::g_last_error;
                if (batch) uoi::admm_batch_leave();     // counts a problem that never joined
            }
            cudaStreamSynchronize(ws);
            cudaStreamDestroy(ws);
        };
        for (int32_t w0 = 0; w0 < count;) {
            const int32_t w1 = grouped ? std::min(count, w0 + kWave) : count;
            const int nw = grouped ? w1 - w0 : std::max(1, std::min<int32_t>(streams, count));
            next = w0;
            wave_end = w1;
            batch = grouped ? uoi::admm_batch_create(w1 - w0) : nullptr;
            std::vector<std::thread> pool;
            for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
            for (auto& th : pool) th.join();
            if (batch) uoi::admm_batch_destroy(batch);
            w0 = w1;
        }
        int ret = UOI_OK;
        int32_t first_bad = -1;
        for (int32_t i = 0; i < count; ++i) {
            if (status_out) status_out[i] = st[(size_t)i];
            if (st[(size_t)i] < 0 && ret >= 0) { ret = st[(size_t)i]; first_bad = i; }
            else if (st[(size_t)i] == UOI_OK_WITH_WARNINGS && ret == UOI_OK) ret = UOI_OK_WITH_WARNINGS;
        }
        if (ret < 0)
            throw uoi::Error(ret, "problem " + std::to_string(first_bad) + " of the batch failed: " +
                                      detail[(size_t)first_bad]);
        return ret;
    });
}

int uoi_var_fit(const double* series, int64_t N, int64_t p, int32_t order, const uoi_params* prm,
                double* A_out, double* mu_out, uoi_diag* diag)
{
    return guarded([&] {
        if (!series || !A_out || !prm) throw Error(UOI_ERR_INVALID_ARG, "NULL data pointer");
        if (order < 1) throw Error(UOI_ERR_INVALID_ARG, "VAR order must be >= 1");
        if (p <= 0 || N - order < 2) throw Error(UOI_ERR_INVALID_ARG, "need N - order >= 2 and p > 0");
        validate(prm);
        cudaStream_t s = (cudaStream_t)prm->stream;
        const bool icpt = param_intercept(prm) != 0;
        if (order == 1 && !icpt) {
            // Eq. 7-8 with d = 1, ascending time: row t regresses X_{t+1} on X_t; the
            // design and the responses are views of one device copy of the series.
            const int st = fit_core(series, p, series + p, p, N - 1, p, p, prm, A_out, nullptr, diag,
                                    series, N * p);
            if (mu_out) {
                if (is_device_ptr(mu_out)) UOI_CUDA(cudaMemsetAsync(mu_out, 0, sizeof(double) * p, s));
                else std::memset(mu_out, 0, sizeof(double) * p);
                UOI_CUDA(cudaStreamSynchronize(s));
            }
            return st;
        }
        ensure_pool();
        // Eq. 7-8: rows t = order..N-1 of (X_t ; X_{t-1} .. X_{t-order}) built on the device
        const int64_t m = N - order, P = (int64_t)order * p, pe = P + (icpt ? 1 : 0);
        DevBuf hs;
        const double* sd = dev_in(series, (size_t)(N * p), hs, s);
        DevBuf X(sizeof(double) * (size_t)(m * P), s), Y(sizeof(double) * (size_t)(m * p), s);
        lagged_design(sd, N, p, order, X.as<double>(), P, Y.as<double>(), p, s);
        DevBuf beta(sizeof(double) * (size_t)(p * pe), s);
        const int st = fit_core(X.as<double>(), P, Y.as<double>(), p, m, P, p, prm, beta.as<double>(), nullptr,
                                diag);
        DevOut<double> ao, mo;
        ao.init(A_out, (size_t)(order * p * p), s);
        mo.init(mu_out, (size_t)p, s);
        partition_var(beta.as<double>(), p, order, icpt ? 1 : 0, ao.dev, mo.dev, s);
        ao.finish(s);
        mo.finish(s);
        UOI_CUDA(cudaStreamSynchronize(s));
        return st;
    });
}

int lasso_admm_batch(const double* X, const double* Y, int64_t n, int64_t p, int64_t r,
                     const uint32_t* weights, int32_t B, const double* lambdas, int32_t q,
                     double rho, double abs_tol, double rel_tol, int32_t max_iter,
                     int32_t precision, int32_t warm_start, double* beta_out, int32_t* iters_out,
                     uint8_t* converged_out, void* stream)
{
    return guarded([&] {
        if (!X || !Y || !lambdas || !beta_out) throw Error(UOI_ERR_INVALID_ARG, "NULL pointer");
        if (n <= 0 || p <= 0 || r <= 0 || q <= 0 || B <= 0 || max_iter <= 0)
            throw Error(UOI_ERR_INVALID_ARG, "sizes must be positive");
        if (!weights && B != 1) throw Error(UOI_ERR_INVALID_ARG, "unweighted call needs B == 1");
        if (!(rho > 0.0)) throw Error(UOI_ERR_INVALID_ARG, "rho must be positive");
        if (precision != UOI_PREC_FP64 && precision != UOI_PREC_MIXED)
            throw Error(UOI_ERR_INVALID_ARG, "unknown precision");
        if (warm_start != UOI_WARM_NONE && warm_start != UOI_WARM_PATH)
            throw Error(warm_start == UOI_WARM_LEARNED ? UOI_ERR_UNSUPPORTED : UOI_ERR_INVALID_ARG,
                        "lasso_admm_batch supports warm_start NONE or PATH");
        ensure_pool();
        cudaStream_t s = (cudaStream_t)stream;
        DevBuf hx, hy, hw, hl;
        const double* Xd = dev_in(X, (size_t)(n * p), hx, s);
        const double* Yd = dev_in(Y, (size_t)(n * r), hy, s);
        const uint32_t* wd = dev_in(weights, (size_t)(B * n), hw, s);
        const double* ld = dev_in(lambdas, (size_t)q, hl, s);
        const int64_t ncol = (int64_t)B * q * r;
        DevOut<double> bo;
        bo.init(beta_out, (size_t)(ncol * p), s);
        DevOut<int32_t> io;
        io.init(iters_out, (size_t)ncol, s);
        DevOut<uint8_t> co;
        co.init(converged_out, (size_t)ncol, s);
        DevBuf ib, cb;
        int32_t* it_d = io.dev;
        uint8_t* cv_d = co.dev;
        if (!it_d) { ib.alloc(sizeof(int32_t) * ncol, s); it_d = ib.as<int32_t>(); }
        if (!cv_d) { cb.alloc(ncol, s); cv_d = cb.as<uint8_t>(); }
        if (precision == UOI_PREC_MIXED)
            selection_admm<float>(precision, Xd, p, Yd, r, n, p, r, wd, B, ld, q, rho, abs_tol,
                                  rel_tol, max_iter, warm_start, bo.dev, it_d, cv_d, nullptr, s,
                                  nullptr, nullptr, false);
        else
            selection_admm<double>(precision, Xd, p, Yd, r, n, p, r, wd, B, ld, q, rho, abs_tol,
                                   rel_tol, max_iter, warm_start, bo.dev, it_d, cv_d, nullptr, s,
                                   nullptr, nullptr, false);
        bo.finish(s);
        io.finish(s);
        co.finish(s);
        UOI_CUDA(cudaStreamSynchronize(s));
        IterStats its = iteration_stats(it_d, cv_d, ncol, s);
        check_bounds_status(s);
        return its.noncon > 0 ? UOI_OK_WITH_WARNINGS : UOI_OK;
    });
}

int uoi_weighted_moments(const double* X, const double* Y, int64_t n, int64_t p, int64_t r,
                         const uint32_t* weights, int32_t B, int32_t precision, double* G_out,
                         double* B_out, void* stream)
{
    return guarded([&] {
        if (!X || !Y || !weights || !G_out || !B_out)
            throw Error(UOI_ERR_INVALID_ARG, "NULL pointer");
        if (n <= 0 || p <= 0 || r <= 0 || B <= 0) throw Error(UOI_ERR_INVALID_ARG, "sizes must be positive");
        if (precision != UOI_PREC_FP64 && precision != UOI_PREC_MIXED)
            throw Error(UOI_ERR_INVALID_ARG, "unknown precision");
        if (precision == UOI_PREC_MIXED && !gram_tc_available())
            throw Error(UOI_ERR_UNSUPPORTED, "tensor-core Gram needs an sm_103 device");
        ensure_pool();
        cudaStream_t s = (cudaStream_t)stream;
        DevBuf hx, hy, hw;
        const double* Xd = dev_in(X, (size_t)(n * p), hx, s);
        const double* Yd = dev_in(Y, (size_t)(n * r), hy, s);
        const uint32_t* wd = dev_in(weights, (size_t)(B * n), hw, s);
        DevOut<double> go, bo;
        go.init(G_out, (size_t)(B * p * p), s);
        bo.init(B_out, (size_t)(B * p * r), s);
        moments(precision, Xd, p, Yd, r, n, p, r, wd, nullptr, B, go.dev, bo.dev, s);
        go.finish(s);
        bo.finish(s);
        UOI_CUDA(cudaStreamSynchronize(s));
        check_bounds_status(s);
        return UOI_OK;
    });
}

struct uoi_ws_model {
    WsModel* m;
};

int64_t uoi_ws_param_count(void) { return ws_param_count(); }

int uoi_ws_create(uint64_t seed, uoi_ws_model** out)
{
    return guarded([&] {
        if (!out) throw Error(UOI_ERR_INVALID_ARG, "NULL handle pointer");
        WsModel* m = ws_create(seed, nullptr);
        UOI_CUDA(cudaStreamSynchronize(nullptr));
        *out = new uoi_ws_model{ m };
        return UOI_OK;
    });
}

int uoi_ws_load(const char* path, uoi_ws_model** out)
{
    return guarded([&] {
        if (!out || !path) throw Error(UOI_ERR_INVALID_ARG, "NULL argument");
        *out = new uoi_ws_model{ ws_load(path, nullptr) };
        return UOI_OK;
    });
}

int uoi_ws_save(uoi_ws_model* model, const char* path)
{
    return guarded([&] {
        if (!model || !path) throw Error(UOI_ERR_INVALID_ARG, "NULL argument");
        ws_save(model->m, path);
        return UOI_OK;
    });
}

void uoi_ws_free(uoi_ws_model* model)
{
    if (!model) return;
    ws_destroy(model->m);
    delete model;
}

int uoi_ws_set_params(uoi_ws_model* model, const float* params)
{
    return guarded([&] {
        if (!model || !params) throw Error(UOI_ERR_INVALID_ARG, "NULL argument");
        ws_set_params(model->m, params, nullptr);
        UOI_CUDA(cudaStreamSynchronize(nullptr));
        return UOI_OK;
    });
}

int uoi_ws_get_params(uoi_ws_model* model, float* params)
{
    return guarded([&] {
        if (!model || !params) throw Error(UOI_ERR_INVALID_ARG, "NULL argument");
        ws_get_params(model->m, params, nullptr);
        return UOI_OK;
    });
}

int uoi_ws_forward(uoi_ws_model* model, const float* X, int64_t N, float* out)
{
    return guarded([&] {
        if (!model || !X || !out || N <= 0) throw Error(UOI_ERR_INVALID_ARG, "bad argument");
        ensure_pool();
        DevBuf hx;
        const float* Xd = dev_in(X, (size_t)(N * 8), hx, nullptr);
        DevOut<float> o;
        o.init(out, (size_t)(N * 3), nullptr);
        ws_forward(model->m, Xd, N, o.dev, nullptr);
        o.finish(nullptr);
        UOI_CUDA(cudaStreamSynchronize(nullptr));
        return UOI_OK;
    });
}

int uoi_ws_loss_grad(uoi_ws_model* model, const float* X, const float* T, int64_t N, double* loss,
                     float* grad)
{
    return guarded([&] {
        if (!model || !X || !T || !grad || N <= 0) throw Error(UOI_ERR_INVALID_ARG, "bad argument");
        ensure_pool();
        DevBuf hx, ht;
        const float* Xd = dev_in(X, (size_t)(N * 8), hx, nullptr);
        const float* Td = dev_in(T, (size_t)(N * 3), ht, nullptr);
        DevOut<float> g;
        g.init(grad, (size_t)ws_param_count(), nullptr);
        const double L = ws_loss_grad(model->m, Xd, Td, N, g.dev, nullptr);
        g.finish(nullptr);
        UOI_CUDA(cudaStreamSynchronize(nullptr));
        if (loss) *loss = L;
        return UOI_OK;
    });
}

int uoi_ws_train(uoi_ws_model* model, const float* X, const float* T, int64_t N, int32_t epochs,
                 int32_t batch, float lr, uint64_t seed, double* final_loss)
{
    return guarded([&] {
        if (!model || !X || !T || N <= 0 || epochs <= 0 || batch <= 0 || batch > N)
            throw Error(UOI_ERR_INVALID_ARG, "bad argument");
        ensure_pool();
        const double L = ws_train(model->m, X, T, N, epochs, batch, lr, seed, nullptr);
        if (final_loss) *final_loss = L;
        return UOI_OK;
    });
}

int uoi_ws_dataset(const double* X, const double* Y, int64_t n, int64_t p, int64_t r,
                   const uint32_t* weights, int32_t B, const double* lambdas, int32_t q, double rho,
                   double abs_tol, double rel_tol, int32_t max_iter, float* features_out,
                   float* targets_out, void* stream)
{
    return guarded([&] {
        if (!X || !Y || !weights || !lambdas || !features_out || !targets_out)
            throw Error(UOI_ERR_INVALID_ARG, "NULL pointer");
        if (n <= 0 || p <= 0 || r <= 0 || q <= 0 || B <= 0 || max_iter <= 0 || !(rho > 0.0))
            throw Error(UOI_ERR_INVALID_ARG, "bad size or parameter");
        ensure_pool();
        cudaStream_t s = (cudaStream_t)stream;
        DevBuf hx, hy, hw, hl;
        const double* Xd = dev_in(X, (size_t)(n * p), hx, s);
        const double* Yd = dev_in(Y, (size_t)(n * r), hy, s);
        const uint32_t* wd = dev_in(weights, (size_t)(B * n), hw, s);
        const double* ld = dev_in(lambdas, (size_t)q, hl, s);
        const int64_t rows = (int64_t)B * q * r * p;
        DevBuf G(sizeof(double) * (size_t)(B * p * p), s), Bm(sizeof(double) * (size_t)(B * p * r), s);
        DevBuf nk(sizeof(double) * B, s), A(sizeof(double) * (size_t)(B * p * p), s);
        moments_fp64(Xd, p, Yd, r, n, p, r, wd, nullptr, B, G.as<double>(), Bm.as<double>(), 0, s);
        weight_sums(wd, nullptr, n, B, nk.as<double>(), s);
        DevBuf st(sizeof(DevStatus), s);
        UOI_CUDA(cudaMemsetAsync(st.ptr, 0, st.bytes, s));
        build_and_factor<double>(G.as<double>(), nk.as<double>(), rho, p, B, A.as<double>(),
                                 st.as<DevStatus>(), s);
        check_status(st.as<DevStatus>(), s, "Cholesky of G/n + rho I");
        DevBuf Linv(sizeof(double) * (size_t)(B * p * p), s), M(sizeof(double) * (size_t)(B * p * p), s);
        DevBuf c(sizeof(double) * (size_t)(B * p * r), s);
        inverse_and_rhs<double>(A.as<double>(), Bm.as<double>(), nk.as<double>(), p, r, B,
                                Linv.as<double>(), M.as<double>(), c.as<double>(), s);
        DevBuf zs(sizeof(double) * (size_t)rows, s), us(sizeof(double) * (size_t)rows, s);
        AdmmProblem<double> P;
        P.G = B; P.p = p; P.r = r; P.q = q;
        P.M = M.as<double>(); P.c = c.as<double>(); P.lambdas = ld;
        P.rho = rho; P.abs_tol = abs_tol; P.rel_tol = rel_tol; P.max_iter = max_iter; P.warm = 1;
        P.beta = zs.as<double>(); P.u_out = us.as<double>();
        admm_solve<double>(P, s);
        DevOut<float> fo, to;
        fo.init(features_out, (size_t)rows * 8, s);
        to.init(targets_out, (size_t)rows * 3, s);
        ws_build_features<double>(G.as<double>(), Bm.as<double>(), nk.as<double>(), c.as<double>(),
                                  ld, q, p, r, B, rho, zs.as<double>(), us.as<double>(), fo.dev,
                                  to.dev, s);
        fo.finish(s);
        to.finish(s);
        UOI_CUDA(cudaStreamSynchronize(s));
        return UOI_OK;
    });
}

const char* uoi_status_string(int status)
{
    switch (status) {
    case UOI_OK: return "ok";
    case UOI_OK_WITH_WARNINGS: return "ok with warnings (non-converged columns or singular supports)";
    case UOI_ERR_INVALID_ARG: return "invalid argument";
    case UOI_ERR_NONFINITE: return "non-finite input";
    case UOI_ERR_NOT_PD: return "matrix not positive definite";
    case UOI_ERR_CUDA: return "CUDA error";
    case UOI_ERR_OOM: return "out of device memory";
    case UOI_ERR_TIMEOUT: return "bounded device loop ran out of iterations";
    case UOI_ERR_BOUNDS: return "an index check of the checked build failed";
    case UOI_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
    }
}

int uoi_get_last_error_detail(char* buf, size_t len)
{
    const int n = (int)g_last_error.size();
    if (buf && len > 0) {
        std::snprintf(buf, len, "%s", g_last_error.c_str());
    }
    return n;
}

void uoi_shutdown(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaDeviceSynchronize();
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
}

}  // extern "C"
