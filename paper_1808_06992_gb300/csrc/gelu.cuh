// gelu.cuh -- the warm-start network's activation, GELU(x) = x Phi(x), and its
// derivative Phi(x) + x phi(x), for the forward and backward kernels.
//
// Phi(x) = (1 + erf(x / sqrt 2)) / 2 is evaluated with the approximation of
// Abramowitz & Stegun, Handbook of Mathematical Functions, formula 7.1.26
// (Hastings): for z >= 0, erfc(z) ~ (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) e^(-z^2)
// with t = 1 / (1 + p z), absolute error of erf at most 1.5e-7.  The exponential
// e^(-z^2) = e^(-x^2 / 2) is shared with the density phi(x) = e^(-x^2 / 2) / sqrt(2 pi).
// At the network's BF16 activations (relative step 2^-8) the approximation is
// invisible; it costs two fast special-function evaluations and a degree-5
// polynomial per element, where the epilogues of the 512-wide layers spend most
// of their time.
#pragma once

namespace uoi {

struct NormalCdfPdf {
    float cdf;      // Phi(x)
    float pdf;      // phi(x)
};

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float exp2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// With z = |x| / sqrt 2: t = 1 / (1 + (p / sqrt 2) |x|), e^(-z^2) = 2^(x * x * (-log2(e) / 2)),
// and the coefficients halved, so the polynomial times e is Phi(-|x|) directly.
__device__ __forceinline__ NormalCdfPdf normal_cdf_pdf(float x)
{
    constexpr float p_s = 0.3275911f * 0.70710678118654752f;
    constexpr float h1 = 0.5f * 0.254829592f, h2 = 0.5f * -0.284496736f, h3 = 0.5f * 1.421413741f,
                    h4 = 0.5f * -1.453152027f, h5 = 0.5f * 1.061405429f;
    constexpr float c = -0.72134752044448170f;               // -log2(e) / 2
    const float t = rcp_approx(fmaf(p_s, fabsf(x), 1.0f));
    const float e = exp2_approx(x * (x * c));                 // e^(-x^2 / 2)
    const float tail = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, h5, h4), h3), h2), h1) * e;   // Phi(-|x|)
    NormalCdfPdf r;
    r.cdf = x >= 0.0f ? 1.0f - tail : tail;
    r.pdf = e * 0.39894228040143268f;
    return r;
}

__device__ __forceinline__ float gelu_f(float x) { return x * normal_cdf_pdf(x).cdf; }

__device__ __forceinline__ float gelu_grad_f(float x)
{
    const NormalCdfPdf v = normal_cdf_pdf(x);
    return fmaf(x, v.pdf, v.cdf);
}

}  // namespace uoi
