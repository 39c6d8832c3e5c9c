// mlp.cu -- G8: the learned warm start of the ADMM selection step.
//
// A per-feature network predicts, for every (bootstrap k, lambda_j, equation e,
// feature i), the converged scaled ADMM state of column (k, j, e): z_i in units
// of the ridge proxy's scale, rho u_i / lambda_j, and whether z_i != 0.  Inputs
// (8 per row, listed at k_ws_features) are lambda and statistics that exist
// before any iteration: the marginal correlation, the Gram diagonal, and the
// ridge solution (G/n + rho I)^{-1} b/n -- the first x-update from zero --
// scaled by lambda_j and by the previous lambda_{j-1}.
// Network: 8 -> 512 -> 512 -> 512 -> 3 with GELU (Phi to 7e-8, gelu.cuh), BF16
// weights and BF16 hidden activations in every product (FP32 master copy in the
// optimizer), FP32 accumulation and FP32 pre-activations.  The two 512 x 512
// layers, their backward products and their weight gradients run on the tensor
// cores (mlp_tc.cu); the 8-input layer stays on CUDA cores, and so does the
// 3-output head in training (in inference it is folded into the last hidden
// layer's epilogue).  Loss
// per row: squared errors of the two state outputs plus the logistic loss of the
// active logit, averaged over rows.
//
// The network only chooses where ADMM starts: its z is used, and the dual is
// set consistent with it (rho u = b/n - (G/n) z, the fixed point of the
// x-update with x = z), so an exact z starts ADMM at its fixed point.  The
// converged answer is the same convex minimiser, which path-warm ADMM checks
// (tests) and falls back to.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gelu.cuh"
#include "kernels.h"

namespace uoi {

constexpr int WS_IN = 8, WS_H = 512, WS_OUT = 3;

namespace {

// parameter offsets in the flat layout W1 b1 W2 b2 W3 b3 W4 b4 (matrices [out][in])
constexpr int64_t OFF_W1 = 0;
constexpr int64_t OFF_B1 = OFF_W1 + (int64_t)WS_H * WS_IN;
constexpr int64_t OFF_W2 = OFF_B1 + WS_H;
constexpr int64_t OFF_B2 = OFF_W2 + (int64_t)WS_H * WS_H;
constexpr int64_t OFF_W3 = OFF_B2 + WS_H;
constexpr int64_t OFF_B3 = OFF_W3 + (int64_t)WS_H * WS_H;
constexpr int64_t OFF_W4 = OFF_B3 + WS_H;
constexpr int64_t OFF_B4 = OFF_W4 + (int64_t)WS_OUT * WS_H;
constexpr int64_t N_PARAMS = OFF_B4 + WS_OUT;

// dst[i] = sum over slices (fixed order) of part[s][i]
__global__ void k_sum_slices(const float* part, int slices, int64_t count, float* dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < slices; ++z) s += part[(int64_t)z * count + i];
        dst[i] = s;
    }
}

// column sums of an N x C matrix in a fixed order: dst[c] = sum_n A[n*C + c]
template <typename TA>
__global__ void k_col_sums(const TA* A, int64_t N, int C, float* dst)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int64_t n = 0; n < N; ++n) s += (float)A[n * C + c];
    dst[c] = s;
}

// layer 1 (K = 8): a1 = X W1^T + b1, h1 = gelu(a1) stored in BF16 (and transposed,
// h1t[o * ldt + n], for the weight gradient of layer 2).  W1 and b1 are staged in
// shared memory; a warp takes one group of 64 outputs for 32 consecutive rows
// (lane = row: the weights it reads are the same for every lane), reads each row's
// 8 inputs once and writes 64 consecutive BF16 outputs as 16-byte vectors.
constexpr int LIN_GROUP = 64;
__global__ void __launch_bounds__(256)
k_layer_in(const float* X, int64_t N, const __nv_bfloat16* w, const float* master, float* pre,
           __nv_bfloat16* h, __nv_bfloat16* ht, int64_t ldt)
{
    __shared__ float sw[WS_H * WS_IN];
    __shared__ float sb[WS_H];
    for (int i = threadIdx.x; i < WS_H * WS_IN; i += blockDim.x) sw[i] = __bfloat162float(w[OFF_W1 + i]);
    for (int i = threadIdx.x; i < WS_H; i += blockDim.x) sb[i] = master[OFF_B1 + i];
    __syncthreads();
    constexpr int groups = WS_H / LIN_GROUP;                   // 8 per row
    const int64_t items = ((N + 31) / 32) * 32 * groups;       // (32-row tile, group, lane)
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < items;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = (t / (32 * groups)) * 32 + (t & 31);
        const int o0 = (int)((t >> 5) % groups) * LIN_GROUP;
        if (n >= N) continue;
        const float4 x0 = *reinterpret_cast<const float4*>(X + n * WS_IN);
        const float4 x1 = *reinterpret_cast<const float4*>(X + n * WS_IN + 4);
        const float xv[WS_IN] = { x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w };
#pragma unroll 2
        for (int v = 0; v < LIN_GROUP; v += 8) {
            uint32_t packed[4];
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                float r2[2];
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int o = o0 + v + u + h2;
                    float acc = sb[o];
#pragma unroll
                    for (int k = 0; k < WS_IN; ++k) acc = fmaf(xv[k], sw[o * WS_IN + k], acc);
                    if (pre) pre[n * WS_H + o] = acc;
                    r2[h2] = gelu_f(acc);
                    if (ht) ht[(int64_t)o * ldt + n] = __float2bfloat16_rn(r2[h2]);
                }
                const __nv_bfloat162 hb = __floats2bfloat162_rn(r2[0], r2[1]);
                packed[u / 2] = *reinterpret_cast<const uint32_t*>(&hb);
            }
            *reinterpret_cast<uint4*>(h + n * WS_H + o0 + v) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        }
    }
}

// head of the inference forward: out[n][j] = b4[j] + the partial products of the
// last hidden layer's epilogue, summed over its slots in a fixed order.
constexpr int HEAD_SLOTS = WS_H / 128;
__global__ void k_head_sum(const float* part, int64_t N, const float* master, float* out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N * WS_OUT;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % WS_OUT);
        float v = part[i];
#pragma unroll
        for (int sl = 1; sl < HEAD_SLOTS; ++sl) v += part[(int64_t)sl * N * WS_OUT + i];
        out[i] = v + master[OFF_B4 + j];
    }
}

// head: out[n][j] = h3[n] . W4[j] + b4[j]   (one warp per row)
__global__ void k_head(const __nv_bfloat16* h3, int64_t N, const __nv_bfloat16* w, const float* master,
                       float* out)
{
    const int64_t n = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (n >= N) return;
    float s[WS_OUT] = {};
    for (int k = lane; k < WS_H; k += 32) {
        const float hv = __bfloat162float(h3[n * WS_H + k]);
#pragma unroll
        for (int j = 0; j < WS_OUT; ++j)
            s[j] = fmaf(hv, __bfloat162float(w[OFF_W4 + j * WS_H + k]), s[j]);
    }
#pragma unroll
    for (int j = 0; j < WS_OUT; ++j) {
        const float v = warp_sum(s[j]);
        if (lane == 0) out[n * WS_OUT + j] = v + master[OFF_B4 + j];
    }
}

// dOut and per-block loss partials
__global__ void k_loss_grad(const float* out, const float* T, int64_t N, float* dout, double* loss_part)
{
    double local = 0.0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
         n += (int64_t)gridDim.x * blockDim.x) {
        const float o0 = out[n * 3], o1 = out[n * 3 + 1], o2 = out[n * 3 + 2];
        const float t0 = T[n * 3], t1 = T[n * 3 + 1], t2 = T[n * 3 + 2];
        const float d0 = o0 - t0, d1 = o1 - t1;
        const float sp = o2 > 0.f ? o2 + log1pf(expf(-o2)) : log1pf(expf(o2));
        local += (double)(d0 * d0 + d1 * d1 + sp - t2 * o2);
        const float inv = 1.0f / (float)N;
        dout[n * 3] = 2.f * d0 * inv;
        dout[n * 3 + 1] = 2.f * d1 * inv;
        dout[n * 3 + 2] = (1.f / (1.f + expf(-o2)) - t2) * inv;
    }
    __shared__ double red[256];
    red[threadIdx.x] = local;
    __syncthreads();
    for (int sft = blockDim.x / 2; sft > 0; sft >>= 1) {
        if (threadIdx.x < sft) red[threadIdx.x] += red[threadIdx.x + sft];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// da3 = (dOut W4) * gelu'(a3), stored in BF16 and transposed (da3t[k * ldt + n])
__global__ void k_head_back(const float* dout, int64_t N, const __nv_bfloat16* w, const float* pre3,
                            __nv_bfloat16* da3, __nv_bfloat16* da3t, int64_t ldt)
{
    const int64_t total = N * WS_H;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = t / WS_H;
        const int k = (int)(t % WS_H);
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < WS_OUT; ++j)
            s = fmaf(dout[n * 3 + j], __bfloat162float(w[OFF_W4 + j * WS_H + k]), s);
        const __nv_bfloat16 d = __float2bfloat16_rn(s * gelu_grad_f(pre3[t]));
        da3[t] = d;
        da3t[(int64_t)k * ldt + n] = d;
    }
}

// gradient of W1 (K over rows, 8 inputs): g[o][k] = sum_n da1[n][o] X[n][k]
__global__ void k_grad_w1(const __nv_bfloat16* da1, const float* X, int64_t N, float* g)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= WS_H) return;
    float s[WS_IN] = {};
    for (int64_t n = 0; n < N; ++n) {
        const float d = __bfloat162float(da1[n * WS_H + o]);
#pragma unroll
        for (int k = 0; k < WS_IN; ++k) s[k] = fmaf(d, X[n * WS_IN + k], s[k]);
    }
#pragma unroll
    for (int k = 0; k < WS_IN; ++k) g[OFF_W1 + o * WS_IN + k] = s[k];
}

// gradient of W4: g[j][k] = sum_n dout[n][j] h3[n][k]
__global__ void k_grad_w4(const float* dout, const __nv_bfloat16* h3, int64_t N, float* g)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= WS_H) return;
    float s[WS_OUT] = {};
    for (int64_t n = 0; n < N; ++n) {
        const float hv = __bfloat162float(h3[n * WS_H + k]);
#pragma unroll
        for (int j = 0; j < WS_OUT; ++j) s[j] = fmaf(dout[n * 3 + j], hv, s[j]);
    }
#pragma unroll
    for (int j = 0; j < WS_OUT; ++j) g[OFF_W4 + j * WS_H + k] = s[j];
}

__global__ void k_transpose_bf16(const __nv_bfloat16* src, __nv_bfloat16* dst, int rows, int cols)
{
    __shared__ __nv_bfloat16 t[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[i][threadIdx.x] = src[(int64_t)r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(int64_t)c * rows + r] = t[threadIdx.x][i];
    }
}

__global__ void k_to_bf16(const float* src, int64_t n, __nv_bfloat16* dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void k_adam(float* master, float* m, float* v, const float* g, int64_t n, float lr,
                       float b1, float b2, float eps, float wd, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        master[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * master[i]);
    }
}

// Kaiming-uniform initialisation from Philox draws: U(-a, a), a = sqrt(6 / fan_in)
// for matrices, zero biases.
__global__ void k_init_params(float* master, uint64_t seed)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N_PARAMS;
         i += (int64_t)gridDim.x * blockDim.x) {
        int fan_in = 0;
        if (i < OFF_B1) fan_in = WS_IN;
        else if (i >= OFF_W2 && i < OFF_B2) fan_in = WS_H;
        else if (i >= OFF_W3 && i < OFF_B3) fan_in = WS_H;
        else if (i >= OFF_W4 && i < OFF_B4) fan_in = WS_H;
        if (fan_in == 0) { master[i] = 0.f; continue; }
        const uint64_t r = philox_draw(PhiloxKey{ seed, 0x4D4C50ull }, 0, 7, (uint64_t)i);
        const float u = (float)(r >> 40) * (1.0f / 16777216.0f);          // [0, 1)
        master[i] = (2.f * u - 1.f) * sqrtf(6.f / (float)fan_in);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Model
// ---------------------------------------------------------------------------
struct WsModel {
    float* master = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    __nv_bfloat16* w = nullptr;       // bf16 copy of every parameter
    __nv_bfloat16* w2t = nullptr;     // W2^T, W3^T (bf16) for the backward products
    __nv_bfloat16* w3t = nullptr;
    int64_t step = 0;
};

namespace {

void sync_weights(WsModel* M, cudaStream_t s)
{
    k_to_bf16<<<256, 256, 0, s>>>(M->master, N_PARAMS, M->w);
    UOI_CHECK_LAUNCH();
    dim3 g(WS_H / 32, WS_H / 32), b(32, 8);
    k_transpose_bf16<<<g, b, 0, s>>>(M->w + OFF_W2, M->w2t, WS_H, WS_H);
    UOI_CHECK_LAUNCH();
    k_transpose_bf16<<<g, b, 0, s>>>(M->w + OFF_W3, M->w3t, WS_H, WS_H);
    UOI_CHECK_LAUNCH();
    count_launch(3);
}

unsigned blocks_for(int64_t work) { return (unsigned)std::min<int64_t>(ceil_div(work, 256), 152 * 16); }

struct Acts {
    DevBuf a1, a2, a3;        // FP32 pre-activations (training)
    DevBuf h1, h2, h3;        // BF16 hidden activations, N x 512
    DevBuf h1t, h2t;          // BF16 512 x ldt transposes (training: the weight gradients' B)
    DevBuf head;              // inference: the head's partial sums, HEAD_SLOTS x N x 3
    DevBuf out;
    int64_t ldt = 0;
};

// Rows of the batch padded for the weight gradients' K extent (transposed copies).
int64_t padded_rows(int64_t N) { return ceil_div(N, 32) * 32; }

void check_err(const DevBuf& err, cudaStream_t s)
{
    int32_t h = 0;
    UOI_CUDA(cudaMemcpyAsync(&h, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    if (h) throw Error(h, "tensor-core MLP product: a bounded pipeline wait expired");
}

// Forward over N rows; keeps pre-activations and transposed activations when
// train is set.
void forward(WsModel* M, const float* X, int64_t N, Acts& A, bool train, int32_t* err, cudaStream_t s)
{
    if (!mlp_tc_available()) throw Error(UOI_ERR_UNSUPPORTED, "the warm-start network needs sm_103a tensor cores");
    const size_t hsz = sizeof(float) * (size_t)N * WS_H, hb = sizeof(__nv_bfloat16) * (size_t)N * WS_H;
    A.ldt = padded_rows(N);
    if (train) {
        A.a1.alloc(hsz, s); A.a2.alloc(hsz, s); A.a3.alloc(hsz, s);
        const size_t tb = sizeof(__nv_bfloat16) * (size_t)WS_H * A.ldt;
        A.h1t.alloc(tb, s); A.h2t.alloc(tb, s);
        UOI_CUDA(cudaMemsetAsync(A.h1t.ptr, 0, tb, s));      // padding rows of the K extent
        UOI_CUDA(cudaMemsetAsync(A.h2t.ptr, 0, tb, s));
    }
    A.h1.alloc(hb, s); A.h2.alloc(hb, s);
    if (train) A.h3.alloc(hb, s);
    else A.head.alloc(sizeof(float) * (size_t)HEAD_SLOTS * N * WS_OUT, s);
    A.out.alloc(sizeof(float) * (size_t)N * WS_OUT, s);
    k_layer_in<<<blocks_for(N * (WS_H / LIN_GROUP)), 256, 0, s>>>(X, N, M->w, M->master, train ? A.a1.as<float>() : nullptr,
                                                   A.h1.as<__nv_bfloat16>(),
                                                   train ? A.h1t.as<__nv_bfloat16>() : nullptr, A.ldt);
    UOI_CHECK_LAUNCH();
    mlp_forward_tc(A.h1.as<__nv_bfloat16>(), N, M->w + OFF_W2, WS_H, M->master + OFF_B2,
                   train ? A.a2.as<float>() : nullptr, A.h2.as<__nv_bfloat16>(),
                   train ? A.h2t.as<__nv_bfloat16>() : nullptr, A.ldt, err, s);
    if (!train) {
        // inference: the head is fused into the last hidden layer's epilogue
        mlp_forward_head_tc(A.h2.as<__nv_bfloat16>(), N, M->w + OFF_W3, WS_H, M->master + OFF_B3,
                            M->w + OFF_W4, A.head.as<float>(), err, s);
        k_head_sum<<<blocks_for(N * WS_OUT), 256, 0, s>>>(A.head.as<float>(), N, M->master, A.out.as<float>());
        UOI_CHECK_LAUNCH();
        count_launch(2);
        return;
    }
    mlp_forward_tc(A.h2.as<__nv_bfloat16>(), N, M->w + OFF_W3, WS_H, M->master + OFF_B3,
                   train ? A.a3.as<float>() : nullptr, A.h3.as<__nv_bfloat16>(), nullptr, 0, err, s);
    k_head<<<(unsigned)ceil_div(N * 32, 256), 256, 0, s>>>(A.h3.as<__nv_bfloat16>(), N, M->w, M->master,
                                                           A.out.as<float>());
    UOI_CHECK_LAUNCH();
    count_launch(2);
}

// Weight gradient g[o][k] = sum_n dA[n][o] H[n][k] (512 x 512) on the tensor cores
// from the transposed BF16 copies, in slices of the batch rows reduced in a fixed order.
void grad_square(const __nv_bfloat16* dAt, const __nv_bfloat16* Ht, int64_t ldt, int64_t N, float* g,
                 int32_t* err, cudaStream_t s)
{
    const int64_t kst = ceil_div(N, 32);
    const int slices = (int)std::max<int64_t>(1, std::min<int64_t>(32, kst / 8));
    DevBuf part(sizeof(float) * (size_t)slices * WS_H * WS_H, s);
    mlp_weight_grad_tc(dAt, Ht, ldt, N, WS_H, slices, part.as<float>(), err, s);
    k_sum_slices<<<blocks_for((int64_t)WS_H * WS_H), 256, 0, s>>>(part.as<float>(), slices,
                                                                   (int64_t)WS_H * WS_H, g);
    UOI_CHECK_LAUNCH();
    count_launch();
}

// Full gradient into g (N_PARAMS floats); returns the mean loss.
double loss_grad(WsModel* M, const float* X, const float* T, int64_t N, float* g, cudaStream_t s)
{
    DevBuf err(sizeof(int32_t), s);
    UOI_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), s));
    Acts A;
    forward(M, X, N, A, true, err.as<int32_t>(), s);
    DevBuf dout(sizeof(float) * (size_t)N * 3, s);
    const int lb = 256;
    DevBuf lp(sizeof(double) * lb, s);
    k_loss_grad<<<lb, 256, 0, s>>>(A.out.as<float>(), T, N, dout.as<float>(), lp.as<double>());
    UOI_CHECK_LAUNCH();
    const size_t hb = sizeof(__nv_bfloat16) * (size_t)N * WS_H;
    const size_t tb = sizeof(__nv_bfloat16) * (size_t)WS_H * A.ldt;
    DevBuf da3(hb, s), da2(hb, s), da3t(tb, s), da2t(tb, s);
    UOI_CUDA(cudaMemsetAsync(da3t.ptr, 0, tb, s));
    UOI_CUDA(cudaMemsetAsync(da2t.ptr, 0, tb, s));
    k_grad_w4<<<WS_H / 128, 128, 0, s>>>(dout.as<float>(), A.h3.as<__nv_bfloat16>(), N, g);
    UOI_CHECK_LAUNCH();
    k_col_sums<float><<<1, 32, 0, s>>>(dout.as<float>(), N, WS_OUT, g + OFF_B4);
    UOI_CHECK_LAUNCH();
    k_head_back<<<blocks_for(N * WS_H), 256, 0, s>>>(dout.as<float>(), N, M->w, A.a3.as<float>(),
                                                     da3.as<__nv_bfloat16>(), da3t.as<__nv_bfloat16>(), A.ldt);
    UOI_CHECK_LAUNCH();
    // layer 3
    grad_square(da3t.as<__nv_bfloat16>(), A.h2t.as<__nv_bfloat16>(), A.ldt, N, g + OFF_W3, err.as<int32_t>(), s);
    k_col_sums<__nv_bfloat16><<<WS_H / 128, 128, 0, s>>>(da3.as<__nv_bfloat16>(), N, WS_H, g + OFF_B3);
    UOI_CHECK_LAUNCH();
    mlp_backward_tc(da3.as<__nv_bfloat16>(), N, M->w3t, WS_H, A.a2.as<float>(), da2.as<__nv_bfloat16>(),
                    da2t.as<__nv_bfloat16>(), A.ldt, err.as<int32_t>(), s);                  // da2
    // layer 2
    grad_square(da2t.as<__nv_bfloat16>(), A.h1t.as<__nv_bfloat16>(), A.ldt, N, g + OFF_W2, err.as<int32_t>(), s);
    k_col_sums<__nv_bfloat16><<<WS_H / 128, 128, 0, s>>>(da2.as<__nv_bfloat16>(), N, WS_H, g + OFF_B2);
    UOI_CHECK_LAUNCH();
    mlp_backward_tc(da2.as<__nv_bfloat16>(), N, M->w2t, WS_H, A.a1.as<float>(), da3.as<__nv_bfloat16>(),
                    nullptr, 0, err.as<int32_t>(), s);                                       // da1 (in da3)
    // layer 1
    k_grad_w1<<<WS_H / 128, 128, 0, s>>>(da3.as<__nv_bfloat16>(), X, N, g);
    UOI_CHECK_LAUNCH();
    k_col_sums<__nv_bfloat16><<<WS_H / 128, 128, 0, s>>>(da3.as<__nv_bfloat16>(), N, WS_H, g + OFF_B1);
    UOI_CHECK_LAUNCH();
    count_launch(8);
    check_err(err, s);
    std::vector<double> h(lb);
    UOI_CUDA(cudaMemcpyAsync(h.data(), lp.ptr, sizeof(double) * lb, cudaMemcpyDeviceToHost, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    double L = 0.0;
    for (double v : h) L += v;
    return L / (double)N;
}

// Features of row (k, j, e, i) and, when z/u are given, the targets.  x0 is the
// ridge solution (G/n_k + rho I)^{-1} b/n_k (the first x-update from zero), c the
// marginal correlation b/n_k, d = G_ii/n_k.  With a_j = x0 d / lambda_j:
//   f0 lambda_j/lambda_0, f1 log(lambda_j/lambda_0)/log(lambda_{q-1}/lambda_0),
//   f2 c/lambda_j, f3 d, f4 a_j, f5 |a_j|, f6 c/lambda_{j-1}, f7 a_{j-1}
// (ratios clipped to [-50, 50]).  Targets: z / s with s = (lambda_j/d) max(1, |f4|)
// clipped to [-4, 4], rho u / lambda_j, [z != 0].
template <typename TC>
__global__ void k_ws_features(const double* gdiag, const double* Bm, const double* nk,
                              const TC* x0, const double* lam, int32_t q, int64_t p, int64_t r,
                              int32_t B, double rho, const double* zt, const double* ut, float* F,
                              float* T)
{
    const int64_t total = (int64_t)B * q * r * p;
    const double l0 = lam[0], lmin = lam[q - 1];
    const double span = (q > 1 && lmin > 0.0 && lmin < l0) ? log(lmin / l0) : -1.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % p;
        const int64_t col = t / p;                        // (k*q + j)*r + e
        const int64_t e = col % r;
        const int64_t j = (col / r) % q;
        const int64_t k = col / (r * q);
        const double lj = lam[j], lp = lam[j > 0 ? j - 1 : 0];
        const double c = Bm[(k * p + i) * r + e] / nk[k];
        const double d = gdiag[k * p + i] / nk[k];
        const double xr = (double)x0[(k * r + e) * p + i];
        auto clip = [](double v) { return fmax(-50.0, fmin(50.0, v)); };
        const double aj = clip(xr * d / lj), ap = clip(xr * d / lp);
        float* f = F + t * WS_IN;
        f[0] = (float)(lj / l0);
        f[1] = (float)(log(lj / l0) / span);
        f[2] = (float)clip(c / lj);
        f[3] = (float)d;
        f[4] = (float)aj;
        f[5] = (float)fabs(aj);
        f[6] = (float)clip(c / lp);
        f[7] = (float)ap;
        if (T) {
            const double scale = (lj / d) * fmax(1.0, fabs((double)(float)aj));
            T[t * 3] = (float)fmax(-4.0, fmin(4.0, zt[t] / scale));
            T[t * 3 + 1] = (float)(rho * ut[t] / lj);
            T[t * 3 + 2] = zt[t] != 0.0 ? 1.f : 0.f;
        }
    }
}

// Predicted start: z0 = o0 (lambda_j / d) max(1, |f4|) where the active logit is
// positive, else 0; u0 = (lambda_j / rho) clamp(o1, -1.5, 1.5) (replaced by the
// consistent dual in the fit).
__global__ void k_ws_start(const float* out, const float* F, const double* lam, int32_t q, int64_t p,
                           int64_t r, int64_t total, double rho, float* z0, float* u0)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = (t / (p * r)) % q;
        const float lj = (float)lam[j];
        const float scale = (lj / F[t * WS_IN + 3]) * fmaxf(1.f, fabsf(F[t * WS_IN + 4]));
        const float o0 = out[t * 3], o1 = out[t * 3 + 1], o2 = out[t * 3 + 2];
        z0[t] = o2 > 0.f ? o0 * scale : 0.f;
        u0[t] = (lj / (float)rho) * fminf(1.5f, fmaxf(-1.5f, o1));
    }
}

// Dual consistent with a start z0 at the x-update's fixed point (x = z):
// rho u0 = b/n_k - (G/n_k) z0, for every column of every group.  One thread per
// (feature i, 8 columns); G is symmetric, so G[k][i] is read along k with
// consecutive i across threads.  FP32 arithmetic (G taken to FP32 with integer
// operations); the start only decides how many iterations ADMM needs.
__global__ void __launch_bounds__(128)
k_ws_dual(const double* G, const double* Bm, const double* nk, const float* z0, int64_t p, int64_t r,
          int32_t q, double rho, float* u0)
{
    const int g = blockIdx.z;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t cols = (int64_t)q * r;
    const int64_t c0 = (int64_t)blockIdx.y * 8;
    const double* Gg = G + (size_t)g * p * p;
    const float inv_n = (float)(1.0 / nk[g]);
    float acc[8] = {};
    if (i < p) {
        for (int64_t k = 0; k < p; ++k) {
            const float gik = f64_to_f32_int(Gg[k * p + i]);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int64_t col = c0 + c;
                if (col < cols) acc[c] = fmaf(gik, z0[((int64_t)g * cols + col) * p + k], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int64_t col = c0 + c;
            if (col >= cols) continue;
            const int64_t e = col % r;
            const float b = f64_to_f32_int(Bm[((int64_t)g * p + i) * r + e]) * inv_n;
            u0[((int64_t)g * cols + col) * p + i] = (b - acc[c] * inv_n) / (float)rho;
        }
    }
}

__global__ void k_gdiag(const double* G, int64_t p, int32_t B, double* out)
{
    const int64_t total = (int64_t)B * p;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / p, i = t % p;
        out[t] = G[(k * p + i) * p + i];
    }
}

}  // namespace

WsModel* ws_create(uint64_t seed, cudaStream_t s)
{
    WsModel* M = new WsModel();
    try {
        UOI_CUDA(cudaMalloc(&M->master, sizeof(float) * N_PARAMS));
        UOI_CUDA(cudaMalloc(&M->m, sizeof(float) * N_PARAMS));
        UOI_CUDA(cudaMalloc(&M->v, sizeof(float) * N_PARAMS));
        UOI_CUDA(cudaMalloc(&M->w, sizeof(__nv_bfloat16) * N_PARAMS));
        UOI_CUDA(cudaMalloc(&M->w2t, sizeof(__nv_bfloat16) * WS_H * WS_H));
        UOI_CUDA(cudaMalloc(&M->w3t, sizeof(__nv_bfloat16) * WS_H * WS_H));
        UOI_CUDA(cudaMemsetAsync(M->m, 0, sizeof(float) * N_PARAMS, s));
        UOI_CUDA(cudaMemsetAsync(M->v, 0, sizeof(float) * N_PARAMS, s));
        k_init_params<<<256, 256, 0, s>>>(M->master, seed);
        UOI_CHECK_LAUNCH();
        count_launch();
        sync_weights(M, s);
    } catch (...) {
        ws_destroy(M);
        throw;
    }
    return M;
}

void ws_destroy(WsModel* M)
{
    if (!M) return;
    cudaFree(M->master); cudaFree(M->m); cudaFree(M->v);
    cudaFree(M->w); cudaFree(M->w2t); cudaFree(M->w3t);
    delete M;
}

int64_t ws_param_count() { return N_PARAMS; }

void ws_set_params(WsModel* M, const float* host_or_dev, cudaStream_t s)
{
    UOI_CUDA(cudaMemcpyAsync(M->master, host_or_dev, sizeof(float) * N_PARAMS, cudaMemcpyDefault, s));
    UOI_CUDA(cudaMemsetAsync(M->m, 0, sizeof(float) * N_PARAMS, s));
    UOI_CUDA(cudaMemsetAsync(M->v, 0, sizeof(float) * N_PARAMS, s));
    M->step = 0;
    sync_weights(M, s);
}

void ws_get_params(WsModel* M, float* host_or_dev, cudaStream_t s)
{
    UOI_CUDA(cudaMemcpyAsync(host_or_dev, M->master, sizeof(float) * N_PARAMS, cudaMemcpyDefault, s));
    UOI_CUDA(cudaStreamSynchronize(s));
}

void ws_forward(WsModel* M, const float* X, int64_t N, float* out, cudaStream_t s)
{
    DevBuf err(sizeof(int32_t), s);
    UOI_CUDA(cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), s));
    const int64_t chunk = 1 << 20;
    for (int64_t n0 = 0; n0 < N; n0 += chunk) {
        const int64_t nn = std::min(chunk, N - n0);
        Acts A;
        forward(M, X + n0 * WS_IN, nn, A, false, err.as<int32_t>(), s);
        UOI_CUDA(cudaMemcpyAsync(out + n0 * WS_OUT, A.out.ptr, sizeof(float) * nn * WS_OUT,
                                 cudaMemcpyDeviceToDevice, s));
    }
    check_err(err, s);
}

double ws_loss_grad(WsModel* M, const float* X, const float* T, int64_t N, float* g, cudaStream_t s)
{
    return loss_grad(M, X, T, N, g, s);
}

// Adam over shuffled mini-batches (Philox permutation of the rows per epoch).
double ws_train(WsModel* M, const float* X, const float* T, int64_t N, int32_t epochs, int32_t batch,
                float lr, uint64_t seed, cudaStream_t s)
{
    DevBuf g(sizeof(float) * N_PARAMS, s);
    DevBuf xb(sizeof(float) * (size_t)batch * WS_IN, s), tb(sizeof(float) * (size_t)batch * 3, s);
    std::vector<int64_t> order((size_t)N);
    double last = 0.0;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f, wd = 1e-5f;
    std::vector<float> hx((size_t)batch * WS_IN), ht((size_t)batch * 3);
    std::vector<float> allx((size_t)N * WS_IN), allt((size_t)N * 3);
    UOI_CUDA(cudaMemcpyAsync(allx.data(), X, sizeof(float) * allx.size(), cudaMemcpyDefault, s));
    UOI_CUDA(cudaMemcpyAsync(allt.data(), T, sizeof(float) * allt.size(), cudaMemcpyDefault, s));
    UOI_CUDA(cudaStreamSynchronize(s));
    for (int32_t ep = 0; ep < epochs; ++ep) {
        // deterministic shuffle: sort rows by a splitmix of (seed, epoch, row)
        for (int64_t i = 0; i < N; ++i) order[(size_t)i] = i;
        uint64_t st = seed * 0x9E3779B97F4A7C15ull + (uint64_t)ep + 1;
        for (int64_t i = N - 1; i > 0; --i) {
            st += 0x9E3779B97F4A7C15ull;
            uint64_t zz = st;
            zz = (zz ^ (zz >> 30)) * 0xBF58476D1CE4E5B9ull;
            zz = (zz ^ (zz >> 27)) * 0x94D049BB133111EBull;
            zz ^= zz >> 31;
            const int64_t jdx = (int64_t)(zz % (uint64_t)(i + 1));
            std::swap(order[(size_t)i], order[(size_t)jdx]);
        }
        double ep_loss = 0.0;
        int64_t nb = 0;
        for (int64_t b0 = 0; b0 + batch <= N; b0 += batch) {
            for (int32_t t = 0; t < batch; ++t) {
                const int64_t src = order[(size_t)(b0 + t)];
                std::memcpy(&hx[(size_t)t * WS_IN], &allx[(size_t)src * WS_IN], sizeof(float) * WS_IN);
                std::memcpy(&ht[(size_t)t * 3], &allt[(size_t)src * 3], sizeof(float) * 3);
            }
            UOI_CUDA(cudaMemcpyAsync(xb.ptr, hx.data(), xb.bytes, cudaMemcpyHostToDevice, s));
            UOI_CUDA(cudaMemcpyAsync(tb.ptr, ht.data(), tb.bytes, cudaMemcpyHostToDevice, s));
            ep_loss += loss_grad(M, xb.as<float>(), tb.as<float>(), batch, g.as<float>(), s);
            ++nb;
            M->step += 1;
            const float c1 = 1.f - powf(b1, (float)M->step), c2 = 1.f - powf(b2, (float)M->step);
            k_adam<<<256, 256, 0, s>>>(M->master, M->m, M->v, g.as<float>(), N_PARAMS, lr, b1, b2, eps,
                                       wd, c1, c2);
            UOI_CHECK_LAUNCH();
            count_launch();
            sync_weights(M, s);
        }
        last = nb ? ep_loss / (double)nb : 0.0;
    }
    UOI_CUDA(cudaStreamSynchronize(s));
    return last;
}

// Features (and targets) for all rows of B groups from moments and the ridge
// solution x0 (B x r x p, the ADMM right-hand side c_k) already on the device.
template <typename TC>
void ws_build_features(const double* G, const double* Bm, const double* nk, const TC* x0,
                       const double* lam, int32_t q, int64_t p, int64_t r, int32_t B, double rho,
                       const double* zt, const double* ut, float* F, float* T, cudaStream_t s)
{
    DevBuf gd(sizeof(double) * (size_t)(B * p), s);
    k_gdiag<<<blocks_for(B * p), 256, 0, s>>>(G, p, B, gd.as<double>());
    UOI_CHECK_LAUNCH();
    k_ws_features<TC><<<blocks_for((int64_t)B * q * r * p), 256, 0, s>>>(gd.as<double>(), Bm, nk, x0,
                                                                       lam, q, p, r, B, rho, zt, ut,
                                                                       F, T);
    UOI_CHECK_LAUNCH();
    count_launch(2);
}

template void ws_build_features<double>(const double*, const double*, const double*, const double*,
                                        const double*, int32_t, int64_t, int64_t, int32_t, double,
                                        const double*, const double*, float*, float*, cudaStream_t);
template void ws_build_features<float>(const double*, const double*, const double*, const float*,
                                       const double*, int32_t, int64_t, int64_t, int32_t, double,
                                       const double*, const double*, float*, float*, cudaStream_t);

void ws_start_state(const float* out, const float* F, const double* lam, int32_t q, int64_t p,
                    int64_t r, int64_t total, double rho, float* z0, float* u0, cudaStream_t s)
{
    k_ws_start<<<blocks_for(total), 256, 0, s>>>(out, F, lam, q, p, r, total, rho, z0, u0);
    UOI_CHECK_LAUNCH();
    count_launch();
}

void ws_consistent_dual(const double* G, const double* Bm, const double* nk, const float* z0,
                        int64_t p, int64_t r, int32_t q, int32_t B, double rho, float* u0,
                        cudaStream_t s)
{
    dim3 g((unsigned)ceil_div(p, 128), (unsigned)ceil_div((int64_t)q * r, 8), (unsigned)B);
    k_ws_dual<<<g, 128, 0, s>>>(G, Bm, nk, z0, p, r, q, rho, u0);
    UOI_CHECK_LAUNCH();
    count_launch();
}

// Weights file: "UOIMLP01", int32 in, hidden, out, layers, then the FP32 parameters.
void ws_save(WsModel* M, const char* path)
{
    std::vector<float> h((size_t)N_PARAMS);
    ws_get_params(M, h.data(), nullptr);
    FILE* f = std::fopen(path, "wb");
    if (!f) throw Error(UOI_ERR_INVALID_ARG, std::string("cannot write ") + path);
    const char magic[8] = { 'U', 'O', 'I', 'M', 'L', 'P', '0', '1' };
    const int32_t hdr[4] = { WS_IN, WS_H, WS_OUT, 3 };
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int32_t), 4, f) == 4 &&
              std::fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
    std::fclose(f);
    if (!ok) throw Error(UOI_ERR_INVALID_ARG, std::string("short write to ") + path);
}

WsModel* ws_load(const char* path, cudaStream_t s)
{
    FILE* f = std::fopen(path, "rb");
    if (!f) throw Error(UOI_ERR_INVALID_ARG, std::string("cannot open ") + path);
    char magic[8];
    int32_t hdr[4];
    std::vector<float> h((size_t)N_PARAMS);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "UOIMLP01", 8) == 0 &&
              std::fread(hdr, sizeof(int32_t), 4, f) == 4 && hdr[0] == WS_IN && hdr[1] == WS_H &&
              hdr[2] == WS_OUT && hdr[3] == 3 &&
              std::fread(h.data(), sizeof(float), h.size(), f) == h.size();
    std::fclose(f);
    if (!ok) throw Error(UOI_ERR_INVALID_ARG, std::string("not a warm-start weights file: ") + path);
    WsModel* M = ws_create(0, s);
    ws_set_params(M, h.data(), s);
    UOI_CUDA(cudaStreamSynchronize(s));
    return M;
}

}  // namespace uoi
