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

__device__ __forceinline__ NormalCdfPdf normal_cdf_pdf(float x)
{
    constexpr float p = 0.3275911f;
    constexpr float a1 = 0.254829592f, a2 = -0.284496736f, a3 = 1.421413741f, a4 = -1.453152027f,
                    a5 = 1.061405429f;
    const float z = fabsf(x) * 0.70710678118654752f;
    const float t = __fdividef(1.0f, fmaf(p, z, 1.0f));
    const float e = __expf(-z * z);
    const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, a5, a4), a3), a2), a1);
    const float half_erfc = 0.5f * poly * e;                 // Phi(-|x|)
    NormalCdfPdf r;
    r.cdf = x >= 0.0f ? 1.0f - half_erfc : half_erfc;
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
