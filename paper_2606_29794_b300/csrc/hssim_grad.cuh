// Per-pixel gradient of the L1 + HSSIM loss (Sec. 4.1; Eq. supp_hssim_eval), shared
// by the HSSIM backward kernel and the backward blend that consumes it in place of a
// dL/dI map (hpxgs_backward_hssim): both produce the same value with the same
// operations in the same order.
#pragma once
#include <cstdint>

namespace hpxgs {

// Window-table gradient at in-mask pixel p of a map with npix pixels:
//   g_c = cf(p) + sum_s e_s(p) cf(idx_s(p)),  cf(q) = alpha_c(q) + beta_c(q) x_c(p) + gamma_c(q) y_c(p)
// (coefficients of the forward per window, divided by its weight sum), then
//   dL/dI_c(p) = scale ((1 - lambda) sign(x_c - y_c) - lambda g_c),  scale = dL/dloss / (3 |M|).
// idx/e are the table's slot arrays [8][npix] (unused slots: idx = p, e = 0).
__device__ __forceinline__ void hssim_pixel_grad(uint32_t p, uint32_t npix, const float* __restrict__ I,
                                                 const float* __restrict__ Gt, const uint32_t* __restrict__ idx,
                                                 const float* __restrict__ e, const float* __restrict__ coef,
                                                 float scale, float lambda, float out[3]) {
  float x[3], y[3], g[3];
  for (int ch = 0; ch < 3; ++ch) {
    x[ch] = I[3 * (size_t)p + ch]; y[ch] = Gt[3 * (size_t)p + ch];
    const float cf0 = coef[9 * (size_t)p + 3 * ch], cf1 = coef[9 * (size_t)p + 3 * ch + 1],
                cf2 = coef[9 * (size_t)p + 3 * ch + 2];
    g[ch] = cf0 + cf1 * x[ch] + cf2 * y[ch];
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t q = idx[(size_t)j * npix + p];
    const float ej = e[(size_t)j * npix + p];
    const float* cf = coef + 9 * (size_t)q;
    for (int ch = 0; ch < 3; ++ch) g[ch] += ej * (cf[3 * ch] + cf[3 * ch + 1] * x[ch] + cf[3 * ch + 2] * y[ch]);
  }
  for (int ch = 0; ch < 3; ++ch) {
    const float d = x[ch] - y[ch];
    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    out[ch] = scale * ((1.f - lambda) * sgn - lambda * g[ch]);
  }
}

}  // namespace hpxgs
