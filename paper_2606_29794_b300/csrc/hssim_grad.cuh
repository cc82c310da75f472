// Per-pixel gradient of the L1 + HSSIM loss (Sec. 4.1; Eq. supp_hssim_eval), shared
// by the HSSIM backward kernel and the backward blend that consumes it in place of a
// dL/dI map (hpxgs_backward_hssim): both produce the same value with the same
// operations in the same order.
#pragma once
#include <cstdint>

namespace hpxgs {

// Window directions (dx, dy) in the order of the neighbour walk (dx = -1, 0, 1, then dy):
// slot s of the window table belongs to direction s.
__host__ __device__ __forceinline__ int window_dx(int s) { return s < 3 ? -1 : (s < 5 ? 0 : 1); }
__host__ __device__ __forceinline__ int window_dy(int s) { return (s == 0 || s == 3 || s == 5) ? -1 : ((s == 1 || s == 6) ? 0 : 1); }

// Neighbours of a pixel away from its face's edges, on the interleaved bits of the NESTED
// index (x in the even bits, y in the odd ones): with MX the x bits and MY the y bits,
// x + 1 = ((q | MY) + 1) & MX (the carry runs through the y gaps) and x - 1 = ((q & MX) - 1) & MX.
// `interior` is false on the face's edges, where the table's ids are used instead
// (the HSSIM forward takes this step; the backward gathers read the ids).
struct WinStep {
  uint32_t MX, MY, qx, qy, face;
  bool interior;
  __device__ __forceinline__ WinStep(int k, uint32_t p) {
    const uint32_t fm = (1u << (2 * k)) - 1u;
    MX = 0x55555555u & fm;
    MY = MX << 1;
    qx = p & MX;
    qy = p & MY;
    face = p & ~fm;
    interior = qx != 0u && qx != MX && qy != 0u && qy != MY;
  }
  __device__ __forceinline__ uint32_t at(int s) const {
    const int dx = window_dx(s), dy = window_dy(s);
    const uint32_t nx = dx > 0 ? (((qx | MY) + 1u) & MX) : (dx < 0 ? ((qx - 1u) & MX) : qx);
    const uint32_t ny = dy > 0 ? (((qy | MX) + 1u) & MY) : (dy < 0 ? ((qy - 1u) & MY) : qy);
    return face | nx | ny;
  }
};

// Window-table gradient at in-mask pixel p of an order-k map with npix pixels:
//   g_c = cf(p) + sum_s e_s(p) cf(n_s(p)),  cf(q) = alpha_c(q) + beta_c(q) x_c(p) + gamma_c(q) y_c(p)
// (coefficients of the forward per window, divided by its weight sum), then
//   dL/dI_c(p) = scale ((1 - lambda) sign(x_c - y_c) - lambda g_c),  scale = dL/dloss / (3 |M|).
// idx/e are the table's arrays [8][npix] by walk direction; where that neighbour is missing
// or outside the mask, e = 0 and idx = p, so the term adds an exact zero.
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
