// HEALPix-SSIM and the L1 + HSSIM training loss (Sec. 4.1; Eq. supp_hssim_eval).
//
// Window of an in-mask pixel q: q and its in-mask 8- (or 7-) neighbours, found
// with the face-edge neighbour walk; weights exp(-theta^2 / (2 sigma^2)) of the
// angle between pixel centres (sigma = 1.5 sqrt(Omega_pix)), normalised over the
// window. Using the true angle gives isotropic kernels near the equator and the
// anisotropic, renormalised ones at the poles and the 24 seven-neighbour pixels.
//
// k_hssim_fwd: per pixel, local statistics, SSIM per channel, block partial sums
//   of h_q, |I - G| and the mask count, and the per-pixel coefficients of the
//   gradient (alpha + beta x_p + gamma y_p per channel, divided by the window sum).
// k_hssim_reduce: fixed-order sum of the block partials -> {loss, HSSIM, L1}.
// k_hssim_bwd: per pixel, gather over the windows that contain it.
#include "hpx_math.cuh"
#include "hssim_grad.cuh"
#include "hssim_window.cuh"
#include "internal.cuh"

using namespace hpx;

namespace hpxgs {

constexpr int kHThreads = 256;

// Block partials of the loss: sum of h_q and of |I - G| in FP32 (8 warp sums of at
// most 32 terms, added in a fixed order) and the exact in-mask count. FP64 work is
// kept out of the per-pixel kernels (the FP64 pipe is slow on this part).
struct HPart { float h, l1; uint32_t cnt, pad; };

struct HSSIMWs {
  size_t coef, part, nmask, total;
};
static HSSIMWs hssim_layout(int k) {
  const size_t npix = 12ull << (2 * k);
  const size_t nblocks = (npix + kHThreads - 1) / kHThreads;
  HSSIMWs L;
  L.coef = 0;
  L.part = (sizeof(float) * 9 * npix + 255) / 256 * 256;
  L.nmask = L.part + (sizeof(HPart) * nblocks + 255) / 256 * 256;   // double count, then its float copy
  L.total = L.nmask + 256;
  return L;
}

__device__ __forceinline__ void block_partials(float h, float l1, uint32_t cnt, HPart* __restrict__ part,
                                               uint32_t slot) {
  for (int o = 16; o > 0; o >>= 1) {
    h += __shfl_xor_sync(0xffffffffu, h, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  __shared__ float sh[2][kHThreads / 32];
  __shared__ uint32_t sc[kHThreads / 32];
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[0][warp] = h; sh[1][warp] = l1; sc[warp] = cnt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f, b = 0.f;
    uint32_t c = 0;
    for (int w2 = 0; w2 < kHThreads / 32; ++w2) { a += sh[0][w2]; b += sh[1][w2]; c += sc[w2]; }
    part[slot] = HPart{a, b, c, 0u};
  }
}

__global__ void __launch_bounds__(kHThreads) k_hssim_fwd(int k, const float* __restrict__ I, const float* __restrict__ Gt,
                                                         const uint32_t* __restrict__ mask, float* __restrict__ coef,
                                                         HPart* __restrict__ part) {
  const uint32_t npix = 12u << (2 * k);
  const uint32_t p = blockIdx.x * kHThreads + threadIdx.x;
  float h = 0.f, l1 = 0.f;
  uint32_t cnt = 0;
  if (p < npix && mask_bit(mask, p)) {
    HWindow W;
    hssim_window(k, p, mask, W);
    float hs = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
      WinStats st;
      for (int j = 0; j < W.n; ++j)
        st.add(W.w[j] * W.iZ, I[3 * (size_t)W.idx[j] + ch], Gt[3 * (size_t)W.idx[j] + ch]);
      const SsimTerms t = ssim_terms(st);
      hs += t.ssim;
      ssim_coefs(st, t, W.iZ, coef + 9 * (size_t)p + 3 * ch);
      l1 += fabsf(I[3 * (size_t)p + ch] - Gt[3 * (size_t)p + ch]);
    }
    h = hs * (1.f / 3.f);
    cnt = 1u;
  }
  block_partials(h, l1, cnt, part, blockIdx.x);
}

// Fixed-order sum of the block partials: per thread compensated (Kahan) FP32 sums of a
// strided subset, then a double tree over the block's threads; the count in integers.
constexpr int kRedThreads = 1024;
__global__ void __launch_bounds__(kRedThreads) k_hssim_reduce(const HPart* __restrict__ part, int nblocks, float lambda,
                                                              float* out3, double* nmask) {
  __shared__ double s[2][kRedThreads];
  __shared__ unsigned long long sc[kRedThreads];
  float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
  unsigned long long cnt = 0;
  for (int i = threadIdx.x; i < nblocks; i += kRedThreads) {
    const HPart q = part[i];
    const float ya = q.h - ca, ta = sa + ya; ca = (ta - sa) - ya; sa = ta;
    const float yb = q.l1 - cb, tb = sb + yb; cb = (tb - sb) - yb; sb = tb;
    cnt += q.cnt;
  }
  s[0][threadIdx.x] = (double)sa - (double)ca;
  s[1][threadIdx.x] = (double)sb - (double)cb;
  sc[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s[0][threadIdx.x] += s[0][threadIdx.x + o];
      s[1][threadIdx.x] += s[1][threadIdx.x + o];
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nm = (double)sc[0];
    const double hssim = nm > 0 ? s[0][0] / nm : 0.0;
    const double l1 = nm > 0 ? s[1][0] / (3.0 * nm) : 0.0;
    out3[0] = (float)((1.0 - lambda) * l1 + lambda * (1.0 - hssim));
    out3[1] = (float)hssim;
    out3[2] = (float)l1;
    nmask[0] = nm;
    reinterpret_cast<float*>(nmask + 1)[0] = (float)nm;   // for the backward, without an FP64 conversion
  }
}

__global__ void __launch_bounds__(kHThreads) k_hssim_bwd(int k, const float* __restrict__ I, const float* __restrict__ Gt,
                                                         const uint32_t* __restrict__ mask, const float* __restrict__ coef,
                                                         const double* __restrict__ nmask, float lambda,
                                                         const float* __restrict__ dloss, float* __restrict__ dI) {
  const uint32_t npix = 12u << (2 * k);
  const uint32_t p = blockIdx.x * kHThreads + threadIdx.x;
  if (p >= npix) return;
  if (!mask_bit(mask, p)) { dI[3 * (size_t)p] = 0.f; dI[3 * (size_t)p + 1] = 0.f; dI[3 * (size_t)p + 2] = 0.f; return; }
  const float nm = reinterpret_cast<const float*>(nmask + 1)[0];
  const float scale = (dloss ? *dloss : 1.f) / (3.f * nm);
  const float inv2sig2 = window_inv2sig2(npix);
  const float3 cp = pix2vec_f32(k, p);
  const FaceXY c = nest_to_fxy(k, p);
  float x[3], y[3], g[3];
  for (int ch = 0; ch < 3; ++ch) {
    x[ch] = I[3 * (size_t)p + ch]; y[ch] = Gt[3 * (size_t)p + ch];
    const float cf0 = coef[9 * (size_t)p + 3 * ch], cf1 = coef[9 * (size_t)p + 3 * ch + 1], cf2 = coef[9 * (size_t)p + 3 * ch + 2];
    g[ch] = cf0 + cf1 * x[ch] + cf2 * y[ch];                 // q = p, e_pp = 1
  }
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy) {
      if (dx == 0 && dy == 0) continue;
      const int64_t nb = neighbour_nest(k, c.f, c.x, c.y, dx, dy);
      if (nb < 0 || !mask_bit(mask, (uint32_t)nb)) continue;
      const float e = window_pair_weight(cp, pix2vec_f32(k, (uint32_t)nb), inv2sig2);
      const float* cf = coef + 9 * (size_t)nb;
      for (int ch = 0; ch < 3; ++ch) g[ch] += e * (cf[3 * ch] + cf[3 * ch + 1] * x[ch] + cf[3 * ch + 2] * y[ch]);
    }
  for (int ch = 0; ch < 3; ++ch) {
    const float d = x[ch] - y[ch];
    const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    dI[3 * (size_t)p + ch] = scale * ((1.f - lambda) * sgn - lambda * g[ch]);
  }
}

// ----------------------------------------------------------------------------
// Window table: the window of a pixel depends only on the grid and the mask, not
// on the maps, so it can be built once per (order, mask) and reused by every
// forward and backward that uses that mask. Per pixel p, structure of arrays:
// e[s][p], the weight towards walk direction s (window_dx/dy), 0 where that
// neighbour is missing or outside the mask; idx[s][p], that neighbour (p where the
// weight is 0), which the forward reads only on a face's edges (elsewhere the
// interleaved-bit step gives it) and the gradient gathers read everywhere; and
// iZ[p] = 1 / (1 + sum e). A zero-weight slot adds an exact zero. The weights come from the same
// window_pair_weight calls in the same order and a zero weight is skipped, so the table
// kernels give the results of k_hssim_fwd / k_hssim_bwd bit for bit while skipping
// the neighbour walk, the pixel centres and the transcendental weights.
// ----------------------------------------------------------------------------
struct HTable {
  uint32_t* idx;   // [8][npix]
  float* e;        // [8][npix]
  float* iZ;       // [npix]
};
static size_t htable_bytes(int k) { return (size_t)17 * 4 * (12ull << (2 * k)); }
static HTable htable(void* t, int k) {
  const size_t npix = 12ull << (2 * k);
  char* b = static_cast<char*>(t);
  return HTable{reinterpret_cast<uint32_t*>(b), reinterpret_cast<float*>(b + 32 * npix),
                reinterpret_cast<float*>(b + 64 * npix)};
}

__global__ void __launch_bounds__(kHThreads) k_hssim_table(int k, const uint32_t* __restrict__ mask, HTable T) {
  const uint32_t npix = 12u << (2 * k);
  const uint32_t p = blockIdx.x * kHThreads + threadIdx.x;
  if (p >= npix) return;
  float Z = 1.f;                               // the pixel itself, e_pp = 1
  const bool in = mask_bit(mask, p);
  const FaceXY c = nest_to_fxy(k, p);
  const float inv2sig2 = window_inv2sig2(npix);
  const float3 cq = pix2vec_f32(k, p);
  for (int s = 0; s < 8; ++s) {                // the walk order: dx = -1, 0, 1, then dy
    const int64_t nb = neighbour_nest(k, c.f, c.x, c.y, window_dx(s), window_dy(s));
    float w = 0.f;
    if (in && nb >= 0 && mask_bit(mask, (uint32_t)nb)) {
      w = window_pair_weight(cq, pix2vec_f32(k, (uint32_t)nb), inv2sig2);
      Z += w;
    }
    T.idx[(size_t)s * npix + p] = w != 0.f ? (uint32_t)nb : p;
    T.e[(size_t)s * npix + p] = w;
  }
  T.iZ[p] = in ? 1.f / Z : 0.f;
}

__global__ void __launch_bounds__(kHThreads) k_hssim_fwd_t(int k, const float* __restrict__ I, const float* __restrict__ Gt,
                                                           const uint32_t* __restrict__ mask, HTable T,
                                                           float* __restrict__ coef, HPart* __restrict__ part) {
  const uint32_t npix = 12u << (2 * k);
  // pixel ranges in decreasing order: the backward blend that follows walks its units upwards
  // from pixel 0, so the table rows, maps and coefficients it gathers first are the ones this
  // kernel touched last (still in L2). Each range keeps its own partial slot (same loss bits).
  const uint32_t blk = gridDim.x - 1u - blockIdx.x;
  const uint32_t p = blk * kHThreads + threadIdx.x;
  float h = 0.f, l1 = 0.f;
  uint32_t cnt = 0;
  if (p < npix && mask_bit(mask, p)) {
    const float iZ = T.iZ[p];
    const WinStep wst(k, p);
    uint32_t q[8];
    float e[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      e[j] = T.e[(size_t)j * npix + p];
      q[j] = wst.interior ? wst.at(j) : T.idx[(size_t)j * npix + p];
    }
    float hs = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
      WinStats st;
      st.add(1.f * iZ, I[3 * (size_t)p + ch], Gt[3 * (size_t)p + ch]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (e[j] == 0.f) continue;
        st.add(e[j] * iZ, I[3 * (size_t)q[j] + ch], Gt[3 * (size_t)q[j] + ch]);
      }
      const SsimTerms t = ssim_terms(st);
      hs += t.ssim;
      ssim_coefs(st, t, iZ, coef + 9 * (size_t)p + 3 * ch);
      l1 += fabsf(I[3 * (size_t)p + ch] - Gt[3 * (size_t)p + ch]);
    }
    h = hs * (1.f / 3.f);
    cnt = 1u;
  }
  block_partials(h, l1, cnt, part, blk);
}

__global__ void __launch_bounds__(kHThreads) k_hssim_bwd_t(int k, const float* __restrict__ I, const float* __restrict__ Gt,
                                                           const uint32_t* __restrict__ mask, HTable T,
                                                           const float* __restrict__ coef,
                                                           const double* __restrict__ nmask, float lambda,
                                                           const float* __restrict__ dloss, float* __restrict__ dI) {
  const uint32_t npix = 12u << (2 * k);
  const uint32_t p = blockIdx.x * kHThreads + threadIdx.x;
  if (p >= npix) return;
  if (!mask_bit(mask, p)) { dI[3 * (size_t)p] = 0.f; dI[3 * (size_t)p + 1] = 0.f; dI[3 * (size_t)p + 2] = 0.f; return; }
  const float nm = reinterpret_cast<const float*>(nmask + 1)[0];
  const float scale = (dloss ? *dloss : 1.f) / (3.f * nm);
  float g[3];
  hssim_pixel_grad(p, npix, I, Gt, T.idx, T.e, coef, scale, lambda, g);
  for (int ch = 0; ch < 3; ++ch) dI[3 * (size_t)p + ch] = g[ch];
}

// The buffers the per-pixel gradient of one view reads: the window table's slot
// arrays and, in the HSSIM workspace the forward wrote, the coefficients and the
// float copy of the in-mask count.
void hssim_bind(int k, const void* table, const void* ws, LossView* out) {
  const HTable T = htable(const_cast<void*>(table), k);
  const HSSIMWs L = hssim_layout(k);
  const char* w = static_cast<const char*>(ws);
  out->idx = T.idx;
  out->e = T.e;
  out->coef = reinterpret_cast<const float*>(w + L.coef);
  out->nm = reinterpret_cast<const float*>(w + L.nmask + sizeof(double));
  out->npix = (uint32_t)(12u << (2 * k));
}

}  // namespace hpxgs

using namespace hpxgs;

extern "C" {

int hpxgs_hssim_workspace_size(int k, size_t* bytes) {
  if (k < 3 || k > 13 || !bytes) return HPXGS_E_INVALID_ARG;
  *bytes = hssim_layout(k).total;
  return HPXGS_OK;
}

int hpxgs_hssim_forward(const float* I, const float* G, const uint32_t* mask, int k, float lambda, void* ws,
                        size_t ws_bytes, float* out3, hpxgs_stream_t stream) {
  if (k < 3 || k > 13 || !I || !G || !mask || !ws || !out3 || !(lambda >= 0.f && lambda <= 1.f))
    return HPXGS_E_INVALID_ARG;
  HSSIMWs L = hssim_layout(k);
  if (ws_bytes < L.total) return HPXGS_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t npix = 12u << (2 * k);
  const int nblocks = (int)((npix + kHThreads - 1) / kHThreads);
  char* w = static_cast<char*>(ws);
  prof_begin(HPXGS_STAGE_HSSIM_FWD, s);
  k_hssim_fwd<<<nblocks, kHThreads, 0, s>>>(k, I, G, mask, reinterpret_cast<float*>(w + L.coef),
                                            reinterpret_cast<HPart*>(w + L.part));
  k_hssim_reduce<<<1, kRedThreads, 0, s>>>(reinterpret_cast<const HPart*>(w + L.part), nblocks, lambda, out3,
                                   reinterpret_cast<double*>(w + L.nmask));
  note_launches(2);
  HPXGS_LAUNCH_CHECK();
  prof_end(HPXGS_STAGE_HSSIM_FWD, s);
  return HPXGS_OK;
}

int hpxgs_hssim_backward(const float* I, const float* G, const uint32_t* mask, int k, float lambda, const void* ws,
                         size_t ws_bytes, const float* dloss, float* dI, hpxgs_stream_t stream) {
  if (k < 3 || k > 13 || !I || !G || !mask || !ws || !dI || !(lambda >= 0.f && lambda <= 1.f))
    return HPXGS_E_INVALID_ARG;
  HSSIMWs L = hssim_layout(k);
  if (ws_bytes < L.total) return HPXGS_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t npix = 12u << (2 * k);
  const int nblocks = (int)((npix + kHThreads - 1) / kHThreads);
  const char* w = static_cast<const char*>(ws);
  prof_begin(HPXGS_STAGE_HSSIM_BWD, s);
  k_hssim_bwd<<<nblocks, kHThreads, 0, s>>>(k, I, G, mask, reinterpret_cast<const float*>(w + L.coef),
                                            reinterpret_cast<const double*>(w + L.nmask), lambda, dloss, dI);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  prof_end(HPXGS_STAGE_HSSIM_BWD, s);
  return HPXGS_OK;
}


int hpxgs_hssim_table_size(int k, size_t* bytes) {
  if (k < 3 || k > 13 || !bytes) return HPXGS_E_INVALID_ARG;
  *bytes = htable_bytes(k);
  return HPXGS_OK;
}

int hpxgs_hssim_table_build(const uint32_t* mask, int k, void* table, size_t table_bytes, hpxgs_stream_t stream) {
  if (k < 3 || k > 13 || !mask || !table) return HPXGS_E_INVALID_ARG;
  if (table_bytes < htable_bytes(k)) return HPXGS_E_WORKSPACE;
  const uint32_t npix = 12u << (2 * k);
  k_hssim_table<<<(npix + kHThreads - 1) / kHThreads, kHThreads, 0, (cudaStream_t)stream>>>(k, mask, htable(table, k));
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

int hpxgs_hssim_forward_table(const float* I, const float* G, const uint32_t* mask, int k, float lambda,
                              const void* table, void* ws, size_t ws_bytes, float* out3, hpxgs_stream_t stream) {
  if (k < 3 || k > 13 || !I || !G || !mask || !table || !ws || !out3 || !(lambda >= 0.f && lambda <= 1.f))
    return HPXGS_E_INVALID_ARG;
  HSSIMWs L = hssim_layout(k);
  if (ws_bytes < L.total) return HPXGS_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t npix = 12u << (2 * k);
  const int nblocks = (int)((npix + kHThreads - 1) / kHThreads);
  char* w = static_cast<char*>(ws);
  prof_begin(HPXGS_STAGE_HSSIM_FWD, s);
  k_hssim_fwd_t<<<nblocks, kHThreads, 0, s>>>(k, I, G, mask, htable(const_cast<void*>(table), k),
                                              reinterpret_cast<float*>(w + L.coef), reinterpret_cast<HPart*>(w + L.part));
  k_hssim_reduce<<<1, kRedThreads, 0, s>>>(reinterpret_cast<const HPart*>(w + L.part), nblocks, lambda, out3,
                                   reinterpret_cast<double*>(w + L.nmask));
  note_launches(2);
  HPXGS_LAUNCH_CHECK();
  prof_end(HPXGS_STAGE_HSSIM_FWD, s);
  return HPXGS_OK;
}

int hpxgs_hssim_backward_table(const float* I, const float* G, const uint32_t* mask, int k, float lambda,
                               const void* table, const void* ws, size_t ws_bytes, const float* dloss, float* dI,
                               hpxgs_stream_t stream) {
  if (k < 3 || k > 13 || !I || !G || !mask || !table || !ws || !dI || !(lambda >= 0.f && lambda <= 1.f))
    return HPXGS_E_INVALID_ARG;
  HSSIMWs L = hssim_layout(k);
  if (ws_bytes < L.total) return HPXGS_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t npix = 12u << (2 * k);
  const int nblocks = (int)((npix + kHThreads - 1) / kHThreads);
  const char* w = static_cast<const char*>(ws);
  prof_begin(HPXGS_STAGE_HSSIM_BWD, s);
  k_hssim_bwd_t<<<nblocks, kHThreads, 0, s>>>(k, I, G, mask, htable(const_cast<void*>(table), k),
                                              reinterpret_cast<const float*>(w + L.coef),
                                              reinterpret_cast<const double*>(w + L.nmask), lambda, dloss, dI);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  prof_end(HPXGS_STAGE_HSSIM_BWD, s);
  return HPXGS_OK;
}

}  // extern "C"
