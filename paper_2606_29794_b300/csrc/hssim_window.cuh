// Per-pixel HEALPix-SSIM window and SSIM value (Sec. 4.1; Eq. supp_hssim_eval), shared by
// the HSSIM kernels that use a workspace (hssim.cu) and the workspace-free loss value
// (hssim_noalloc.cu), so that every entry point evaluates the window weights, the local
// statistics, h_q and |I - G| with the same operations in the same order.
//
// Window of an in-mask pixel q: q and its in-mask 8- (or 7-) neighbours in the order of
// the neighbour walk (dx = -1, 0, 1, then dy); weights exp(-theta^2 / (2 sigma^2)) of the
// angle between pixel centres, sigma = 1.5 sqrt(Omega_pix), normalised over the window;
// SSIM constants C1 = 0.01^2, C2 = 0.03^2.
#pragma once
#include <cstdint>

#include "hpx_math.cuh"

namespace hpxgs {

constexpr float kSsimC1 = 1e-4f, kSsimC2 = 9e-4f;

__device__ __forceinline__ bool mask_bit(const uint32_t* m, uint32_t p) { return (m[p >> 5] >> (p & 31)) & 1u; }

// 1 / (2 sigma^2) at order k: sigma^2 = 2.25 Omega_pix, Omega_pix = 4 pi / Npix.
__device__ __forceinline__ float window_inv2sig2(uint32_t npix) {
  const float omega = 4.f * (float)hpx::kPi / (float)npix;
  return 1.f / (2.f * 2.25f * omega);
}

// Weight of a neighbour at unit direction b seen from the window centre a.
__device__ __forceinline__ float window_pair_weight(float3 a, float3 b, float inv2sig2) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float ch = sqrtf(dx * dx + dy * dy + dz * dz);
  const float th = 2.f * asinf(fminf(1.f, 0.5f * ch));
  return __expf(-th * th * inv2sig2);
}

// The window of in-mask pixel p: slot 0 is p itself (weight 1), then the in-mask
// neighbours in walk order; iZ = 1 / (sum of the weights).
struct HWindow {
  uint32_t idx[9];
  float w[9];
  int n;
  float iZ;
};

__device__ __forceinline__ void hssim_window(int k, uint32_t p, const uint32_t* __restrict__ mask, HWindow& W) {
  const uint32_t npix = 12u << (2 * k);
  const float inv2sig2 = window_inv2sig2(npix);
  const float3 cq = hpx::pix2vec_f32(k, p);
  const hpx::FaceXY c = hpx::nest_to_fxy(k, p);
  W.n = 0;
  W.idx[W.n] = p; W.w[W.n] = 1.f; ++W.n;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy) {
      if (dx == 0 && dy == 0) continue;
      const int64_t nb = hpx::neighbour_nest(k, c.f, c.x, c.y, dx, dy);
      if (nb < 0 || !mask_bit(mask, (uint32_t)nb)) continue;
      W.idx[W.n] = (uint32_t)nb;
      W.w[W.n] = window_pair_weight(cq, hpx::pix2vec_f32(k, (uint32_t)nb), inv2sig2);
      ++W.n;
    }
  float Z = 0.f;
  for (int j = 0; j < W.n; ++j) Z += W.w[j];
  W.iZ = 1.f / Z;
}

// Weighted local statistics of one channel: running sums, one window slot at a time.
struct WinStats {
  float mx, my, xx, yy, xy;
  __device__ __forceinline__ WinStats() : mx(0.f), my(0.f), xx(0.f), yy(0.f), xy(0.f) {}
  __device__ __forceinline__ void add(float wj, float x, float y) {
    mx += wj * x; my += wj * y; xx += wj * x * x; yy += wj * y * y; xy += wj * x * y;
  }
};

// SSIM of the statistics and the pieces its gradient coefficients reuse. The reciprocals
// run on the MUFU unit (rcp.approx, about one unit in the last place), against
// the loss's FP64 reference tolerance of 2e-6.
struct SsimTerms {
  float ssim, A1, A2, B2, iB, iB2;
};

__device__ __forceinline__ float rcp_mufu(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ SsimTerms ssim_terms(const WinStats& s) {
  SsimTerms t;
  const float vx = s.xx - s.mx * s.mx, vy = s.yy - s.my * s.my, cxy = s.xy - s.mx * s.my;
  t.A1 = 2.f * s.mx * s.my + kSsimC1;
  t.A2 = 2.f * cxy + kSsimC2;
  const float B1 = s.mx * s.mx + s.my * s.my + kSsimC1;
  t.B2 = vx + vy + kSsimC2;
  t.iB2 = rcp_mufu(t.B2);
  t.iB = rcp_mufu(B1) * t.iB2;
  t.ssim = t.A1 * t.A2 * t.iB;
  return t;
}

// Gradient coefficients of one channel: d ssim_q / d x_p = w_qp (alpha + beta x_p + gamma y_p)
// for every p in the window, stored as (alpha, beta, gamma) / (window weight sum), from the
// partials of ssim with respect to (mu_x, var_x, cov_xy).
__device__ __forceinline__ void ssim_coefs(const WinStats& s, const SsimTerms& t, float iZ, float* __restrict__ cf) {
  const float dmu = (2.f * s.my * t.A2 - t.ssim * t.B2 * 2.f * s.mx) * t.iB;
  const float dvar = -t.ssim * t.iB2;
  const float dcov = 2.f * t.A1 * t.iB;
  cf[0] = (dmu - 2.f * s.mx * dvar - s.my * dcov) * iZ;
  cf[1] = 2.f * dvar * iZ;
  cf[2] = dcov * iZ;
}

// h_q (mean SSIM over the three channels) and sum_c |I_c - G_c| at in-mask pixel p.
__device__ __forceinline__ void hssim_pixel_value(const HWindow& W, uint32_t p, const float* __restrict__ I,
                                                  const float* __restrict__ Gt, float& h, float& l1) {
  float hs = 0.f;
  l1 = 0.f;
  for (int ch = 0; ch < 3; ++ch) {
    WinStats st;
    for (int j = 0; j < W.n; ++j)
      st.add(W.w[j] * W.iZ, I[3 * (size_t)W.idx[j] + ch], Gt[3 * (size_t)W.idx[j] + ch]);
    hs += ssim_terms(st).ssim;
    l1 += fabsf(I[3 * (size_t)p + ch] - Gt[3 * (size_t)p + ch]);
  }
  h = hs * (1.f / 3.f);
}

}  // namespace hpxgs
