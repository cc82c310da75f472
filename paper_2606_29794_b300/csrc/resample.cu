// Sphere <-> image resampling: the rendered HEALPix map to a camera image
// (Eq. camera_synthesis) and a camera image to the HEALPix grid
// (Eqs. supp_image_to_healpix, supp_hssim_mask), with the camera models of
// Sec. D.1 (Eq. persp_sphere; Eqs. fish_weff, fish_sphere, imaging_region,
// semi_axes; the omnidirectional mapping).
//
// The paper names the operations, not the schemes; the readings:
//  - image samples sit at pixel centres (i + 1/2, j + 1/2);
//  - Interp_H is HEALPix ring-bilinear interpolation: along each of the two
//    rings that bracket the colatitude, linear in longitude between the two
//    pixel centres that bracket it; between the rings, linear in colatitude;
//    above the first ring (below the last) linear in colatitude to a pole
//    value, the mean of that ring's 4 pixels;
//  - the image is sampled bilinearly between pixel centres, clamped at the
//    edges and, for the panorama, wrapped in longitude.
// The map lives in the camera frame: HEALPix (X, Y, Z) = camera (d_z, d_x, d_y).
// All three kernels are gathers or scatters bound by memory traffic: one thread
// per output pixel, grid-stride over a grid of a few waves of the SM count.
#include <algorithm>
#include <cmath>

#include "camera.cuh"
#include "hpx_math.cuh"
#include "internal.cuh"

using namespace hpx;

namespace hpxgs {
namespace {

constexpr int kRsThreads = 256;

struct ImgCam {
  int kind, W, H;
  float fx, fy;      // pinhole: W / (2 tan(FoV_x / 2)), H / (2 tan(FoV_y / 2)); fisheye: W / pi, H / pi
  float cx, cy;      // principal point: pinhole (W/2)(1 + ppx), (H/2)(1 + ppy); fisheye and panorama W/2, H/2
  float wx, wy;      // fisheye FoV / 180 deg
};

// P_C: image point (u, v) -> unit camera direction; false outside D_C.
__device__ __forceinline__ bool img_to_dir(const ImgCam& c, float u, float v, float3& d) {
  if (c.kind == HPXGS_CAM_FULL) {
    float so, co, sp, cp;                         // angles in units of pi: no wide range reduction
    sincospif(2.f * u / (float)c.W - 1.f, &so, &co);
    sincospif(0.5f - v / (float)c.H, &sp, &cp);
    d = make_float3(cp * so, sp, cp * co);
    return true;
  }
  const float mx = (u - c.cx) / c.fx, my = (v - c.cy) / c.fy;
  if (c.kind == HPXGS_CAM_PINHOLE) {
    const float inv = rsqrtf(mx * mx + my * my + 1.f);
    d = make_float3(mx * inv, my * inv, inv);
    return true;                                  // pixel centres lie inside [0, W] x [0, H]
  }
  const float rm2 = mx * mx + my * my;
  if (rm2 > 0.25f * (float)kPi * (float)kPi) return false;   // outside the ellipse a = f_x pi/2, b = f_y pi/2
  const float rm = sqrtf(rm2);
  if (rm == 0.f) { d = make_float3(0.f, 0.f, 1.f); return true; }
  const float cg = mx / rm, sg = my / rm;
  const float weff = sqrtf(c.wx * c.wx * cg * cg + c.wy * c.wy * sg * sg);
  float sp, cp;
  sincospif(rm * weff * (1.f / (float)kPi), &sp, &cp);
  d = make_float3(sp * cg, sp * sg, cp);
  return true;
}

// Pi_C^{-1} for a direction inside the camera's region: image point (u, v).
__device__ __forceinline__ float2 dir_to_img(const ImgCam& c, float3 d) {
  if (c.kind == HPXGS_CAM_FULL) {
    const float om = atan2f(d.x, d.z), ph = asinf(fminf(1.f, fmaxf(-1.f, d.y)));
    return make_float2((float)c.W * (om + (float)kPi) / (2.f * (float)kPi),
                       (float)c.H * (0.5f * (float)kPi - ph) / (float)kPi);
  }
  if (c.kind == HPXGS_CAM_PINHOLE)
    return make_float2(c.cx + c.fx * d.x / d.z, c.cy + c.fy * d.y / d.z);
  const float rxy = sqrtf(d.x * d.x + d.y * d.y);
  if (rxy == 0.f) return make_float2(c.cx, c.cy);
  const float cg = d.x / rxy, sg = d.y / rxy;
  const float weff = sqrtf(c.wx * c.wx * cg * cg + c.wy * c.wy * sg * sg);
  const float rm = atan2f(rxy, d.z) / weff;
  return make_float2(c.cx + c.fx * rm * cg, c.cy + c.fy * rm * sg);
}

__device__ __forceinline__ float ring_theta(int k, int i) {
  const RingF R = ring_f32(k, i);
  return atan2f(R.sth, R.z);
}

// Ring i in [0, 4N - 1] with theta_i <= theta < theta_{i+1} (ring 0: the north pole),
// from the ring's closed form in z (1 -+ z taken from sin^2 near the poles), then
// corrected against the ring colatitudes.
__device__ __forceinline__ int ring_above(int k, float z, float s2, float theta) {
  const int N = 1 << k, nr = 4 * N - 1;
  float rf;
  if (z > 2.f / 3.f) rf = (float)N * sqrtf(3.f * s2 / (1.f + z));
  else if (z < -2.f / 3.f) rf = 4.f * (float)N - (float)N * sqrtf(3.f * s2 / (1.f - z));
  else rf = (float)N * (2.f - 1.5f * z);
  int i = min(nr, max(0, (int)floorf(rf)));
  if (i >= 1 && ring_theta(k, i) > theta) --i;
  else if (i < nr && ring_theta(k, i + 1) <= theta) ++i;
  return i;
}

__device__ __forceinline__ uint32_t ring_pixel_nest(int k, int i, int j, int npix) {
  j %= npix;
  if (j < 0) j += npix;
  const FaceXY f = ring_to_fxy(k, i, j);
  return fxy_to_nest(k, f.f, f.x, f.y);
}

// Interp_H weights at (theta, phi): 4 NESTED pixels (one may repeat) summing to 1.
__device__ __forceinline__ void interp_weights(int k, float theta, float phi, float z, float s2, uint32_t pix[4],
                                               float w[4]) {
  const int N = 1 << k, nr = 4 * N - 1;
  const int ir = ring_above(k, z, s2, theta);
  struct Br { uint32_t p0, p1; float f; };
  auto bracket = [&](int i) {
    const RingF R = ring_f32(k, i);
    const float t = (phi - R.phi0) * (float)R.npix * (0.5f / (float)kPi);
    const float j0 = floorf(t);
    return Br{ring_pixel_nest(k, i, (int)j0, R.npix), ring_pixel_nest(k, i, (int)j0 + 1, R.npix), t - j0};
  };
  if (ir >= 1 && ir < nr) {
    const float t0 = ring_theta(k, ir), t1 = ring_theta(k, ir + 1);
    const float wt = fminf(1.f, fmaxf(0.f, (theta - t0) / (t1 - t0)));
    const Br a = bracket(ir), b = bracket(ir + 1);
    pix[0] = a.p0; pix[1] = a.p1; pix[2] = b.p0; pix[3] = b.p1;
    w[0] = (1.f - wt) * (1.f - a.f); w[1] = (1.f - wt) * a.f; w[2] = wt * (1.f - b.f); w[3] = wt * b.f;
    return;
  }
  const int ring = ir == 0 ? 1 : nr;
  const float tr = ring_theta(k, ring);
  const float wr = fminf(1.f, fmaxf(0.f, ir == 0 ? theta / tr : ((float)kPi - theta) / ((float)kPi - tr)));
  const Br a = bracket(ring);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    pix[j] = ring_pixel_nest(k, ring, j, 4);
    w[j] = 0.25f * (1.f - wr) + (pix[j] == a.p0 ? wr * (1.f - a.f) : 0.f) + (pix[j] == a.p1 ? wr * a.f : 0.f);
  }
}

// HEALPix angles of a camera direction: theta from atan2 (accurate at the poles).
__device__ __forceinline__ void healpix_angles(float3 d, float& theta, float& phi, float& z, float& s2) {
  const float X = d.z, Y = d.x;
  z = d.y;
  s2 = X * X + Y * Y;
  theta = atan2f(sqrtf(s2), z);
  phi = atan2f(Y, X);
  if (phi < 0.f) phi += 2.f * (float)kPi;
}

// The Interp_H taps of image pixel p: 4 NESTED map pixels and weights, false outside D_C
// (then no taps). Shared by the direct kernels and the resampling plan.
__device__ __forceinline__ bool s2i_taps(int k, const ImgCam& c, int64_t p, uint32_t pix[4], float w[4]) {
  const int row = (int)(p / c.W), col = (int)(p - (int64_t)row * c.W);
  float3 d;
  if (!img_to_dir(c, (float)col + 0.5f, (float)row + 0.5f, d)) return false;
  float th, ph, z, s2;
  healpix_angles(d, th, ph, z, s2);
  interp_weights(k, th, ph, z, s2, pix, w);
  return true;
}

// sum_q w_q map[pix_q] per channel, q in order
__device__ __forceinline__ void s2i_gather(const float* __restrict__ map, const uint32_t pix[4], const float w[4],
                                           float o[3]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) o[ch] += w[q] * __ldg(map + 3 * (size_t)pix[q] + ch);
}

__global__ void __launch_bounds__(kRsThreads) k_sphere_to_image(const float* __restrict__ map, int k, ImgCam c,
                                                                 float* __restrict__ img, uint8_t* __restrict__ valid) {
  const int64_t n = (int64_t)c.W * c.H;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    uint32_t pix[4];
    float w[4];
    const bool ok = s2i_taps(k, c, p, pix, w);
    float o[3] = {0.f, 0.f, 0.f};
    if (ok) s2i_gather(map, pix, w, o);
    img[3 * p + 0] = o[0]; img[3 * p + 1] = o[1]; img[3 * p + 2] = o[2];
    if (valid) valid[p] = ok;
  }
}

// dmap[pix_q] += w_q g per channel by atomics (several image pixels share a map pixel)
__device__ __forceinline__ void s2i_scatter(float* __restrict__ dmap, const uint32_t pix[4], const float w[4],
                                            const float g[3]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (w[q] != 0.f)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) atomicAdd(dmap + 3 * (size_t)pix[q] + ch, w[q] * g[ch]);
}

// dmap += A^T dimg, by atomics (several image pixels share a HEALPix pixel).
__global__ void __launch_bounds__(kRsThreads) k_sphere_to_image_bwd(const float* __restrict__ dimg, int k, ImgCam c,
                                                                     float* __restrict__ dmap) {
  const int64_t n = (int64_t)c.W * c.H;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float g[3] = {dimg[3 * p], dimg[3 * p + 1], dimg[3 * p + 2]};
    if (g[0] == 0.f && g[1] == 0.f && g[2] == 0.f) continue;
    uint32_t pix[4];
    float w[4];
    if (!s2i_taps(k, c, p, pix, w)) continue;
    s2i_scatter(dmap, pix, w, g);
  }
}

// I_H(q) = I_C(Pi_C^{-1}(s_q)) and M_C(q) for every NESTED pixel q (0 outside M_C).
// A sample of the image as a value in [0, 1]: float images as they are, 8-bit codes v as
// v / 255 (IEEE division, the value a float image holding v / 255 would give).
__device__ __forceinline__ float image_value(const float* px) { return __ldg(px); }
__device__ __forceinline__ float image_value(const uint8_t* px) { return __fdiv_rn((float)__ldg(px), 255.f); }

// The bilinear image taps of in-mask map pixel q: image pixel indices row * W + col and
// weights, in the order (row 0, col 0), (0, 1), (1, 0), (1, 1). Shared by the direct kernel
// and the resampling plan.
__device__ __forceinline__ void i2s_taps(const ImgCam& c, int k, uint32_t q, uint32_t idx[4], float w[4]) {
  const float3 h = pix2vec_f32(k, q);
  const float2 uv = dir_to_img(c, make_float3(h.y, h.z, h.x));
  const float x = uv.x - 0.5f, y = uv.y - 0.5f;
  const float x0 = floorf(x), y0 = floorf(y), fx = x - x0, fy = y - y0;
  int xs[2] = {(int)x0, (int)x0 + 1}, ys[2] = {(int)y0, (int)y0 + 1};
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    if (c.kind == HPXGS_CAM_FULL) { xs[t] %= c.W; if (xs[t] < 0) xs[t] += c.W; }
    else xs[t] = min(c.W - 1, max(0, xs[t]));
    ys[t] = min(c.H - 1, max(0, ys[t]));
  }
  const float wx[2] = {1.f - fx, fx}, wy[2] = {1.f - fy, fy};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      idx[2 * a + b] = (uint32_t)ys[a] * (uint32_t)c.W + (uint32_t)xs[b];
      w[2 * a + b] = wy[a] * wx[b];
    }
}

// sum_t w_t image[idx_t] per channel, t in order
template <typename T>
__device__ __forceinline__ void i2s_gather(const T* __restrict__ img, const uint32_t idx[4], const float w[4],
                                           float o[3]) {
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const T* px = img + 3 * (size_t)idx[t];
    o[0] += w[t] * image_value(px); o[1] += w[t] * image_value(px + 1); o[2] += w[t] * image_value(px + 2);
  }
}

template <typename T>
__global__ void __launch_bounds__(kRsThreads) k_image_to_sphere(const T* __restrict__ img, ImgCam c, ViewParams vp,
                                                                 float* __restrict__ map, uint32_t* __restrict__ words) {
  const uint32_t npix = 12u << (2 * vp.k);                   // a multiple of 32 for k >= 2
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < npix; base += stride) {
    const uint32_t q = base + threadIdx.x;
    const bool inr = q < npix;
    const bool in = inr && pixel_in_mask(vp, q);
    float o[3] = {0.f, 0.f, 0.f};
    if (in) {
      uint32_t idx[4];
      float w[4];
      i2s_taps(c, vp.k, q, idx, w);
      i2s_gather(img, idx, w, o);
    }
    if (inr) { map[3 * (size_t)q] = o[0]; map[3 * (size_t)q + 1] = o[1]; map[3 * (size_t)q + 2] = o[2]; }
    const uint32_t bits = __ballot_sync(0xffffffffu, in);
    if (words && inr && (threadIdx.x & 31) == 0) words[q >> 5] = bits;
  }
}

// ----------------------------------------------------------------------------
// Resampling plans: the taps of every output pixel, computed once for a camera (its
// intrinsics, image size and HEALPix order) and applied to any number of maps or
// images. Layout (structure of arrays, each part 256-byte aligned), n output pixels:
//   sphere -> image (n = W H):     pix [4][n] u32, w [4][n] f32, valid [n] u8
//   image -> sphere (n = 12 4^k):  idx [4][n] u32, w [4][n] f32, mask words [n / 32] u32
// Applying a plan runs the direct kernel's accumulation over the same taps in the same
// order, so it gives the direct kernel's results bit for bit.
// ----------------------------------------------------------------------------
struct PlanLayout {
  size_t taps, w, extra, total;
  int64_t n;
};

PlanLayout plan_layout(int dir, int k, int W, int H) {
  PlanLayout L;
  L.n = dir == HPXGS_PLAN_SPHERE_TO_IMAGE ? (int64_t)W * H : (12LL << (2 * k));
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  L.taps = 0;
  L.w = al(sizeof(uint32_t) * 4 * (size_t)L.n);
  L.extra = L.w + al(sizeof(float) * 4 * (size_t)L.n);
  L.total = L.extra + al(dir == HPXGS_PLAN_SPHERE_TO_IMAGE ? (size_t)L.n : sizeof(uint32_t) * (size_t)(L.n / 32));
  return L;
}

__global__ void __launch_bounds__(kRsThreads) k_plan_s2i(int k, ImgCam c, uint32_t* __restrict__ pix,
                                                          float* __restrict__ wt, uint8_t* __restrict__ valid) {
  const int64_t n = (int64_t)c.W * c.H;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    uint32_t px[4] = {0u, 0u, 0u, 0u};
    float w[4] = {0.f, 0.f, 0.f, 0.f};
    const bool ok = s2i_taps(k, c, p, px, w);
#pragma unroll
    for (int q = 0; q < 4; ++q) { pix[q * n + p] = ok ? px[q] : 0u; wt[q * n + p] = ok ? w[q] : 0.f; }
    valid[p] = ok;
  }
}

__global__ void __launch_bounds__(kRsThreads) k_plan_s2i_apply(const float* __restrict__ map, int64_t n,
                                                                const uint32_t* __restrict__ pix,
                                                                const float* __restrict__ wt,
                                                                const uint8_t* __restrict__ pvalid,
                                                                float* __restrict__ img, uint8_t* __restrict__ valid) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const bool ok = pvalid[p];
    float o[3] = {0.f, 0.f, 0.f};
    if (ok) {
      uint32_t px[4];
      float w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { px[q] = pix[q * n + p]; w[q] = wt[q * n + p]; }
      s2i_gather(map, px, w, o);
    }
    img[3 * p + 0] = o[0]; img[3 * p + 1] = o[1]; img[3 * p + 2] = o[2];
    if (valid) valid[p] = ok;
  }
}

__global__ void __launch_bounds__(kRsThreads) k_plan_s2i_adjoint(const float* __restrict__ dimg, int64_t n,
                                                                  const uint32_t* __restrict__ pix,
                                                                  const float* __restrict__ wt,
                                                                  const uint8_t* __restrict__ pvalid,
                                                                  float* __restrict__ dmap) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const float g[3] = {dimg[3 * p], dimg[3 * p + 1], dimg[3 * p + 2]};
    if (g[0] == 0.f && g[1] == 0.f && g[2] == 0.f) continue;
    if (!pvalid[p]) continue;
    uint32_t px[4];
    float w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { px[q] = pix[q * n + p]; w[q] = wt[q * n + p]; }
    s2i_scatter(dmap, px, w, g);
  }
}

__global__ void __launch_bounds__(kRsThreads) k_plan_i2s(ImgCam c, ViewParams vp, uint32_t* __restrict__ idx,
                                                          float* __restrict__ wt, uint32_t* __restrict__ words) {
  const uint32_t npix = 12u << (2 * vp.k);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < npix; base += stride) {
    const uint32_t q = base + threadIdx.x;
    const bool inr = q < npix;
    const bool in = inr && pixel_in_mask(vp, q);
    uint32_t ix[4] = {0u, 0u, 0u, 0u};
    float w[4] = {0.f, 0.f, 0.f, 0.f};
    if (in) i2s_taps(c, vp.k, q, ix, w);
    if (inr)
#pragma unroll
      for (int t = 0; t < 4; ++t) { idx[(size_t)t * npix + q] = ix[t]; wt[(size_t)t * npix + q] = w[t]; }
    const uint32_t bits = __ballot_sync(0xffffffffu, in);
    if (inr && (threadIdx.x & 31) == 0) words[q >> 5] = bits;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRsThreads) k_plan_i2s_apply(const T* __restrict__ img, uint32_t npix,
                                                                const uint32_t* __restrict__ idx,
                                                                const float* __restrict__ wt,
                                                                const uint32_t* __restrict__ pwords,
                                                                float* __restrict__ map, uint32_t* __restrict__ words) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < npix; base += stride) {
    const uint32_t q = base + threadIdx.x;
    const bool inr = q < npix;
    const bool in = inr && ((pwords[q >> 5] >> (q & 31)) & 1u);
    float o[3] = {0.f, 0.f, 0.f};
    if (in) {
      uint32_t ix[4];
      float w[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) { ix[t] = idx[(size_t)t * npix + q]; w[t] = wt[(size_t)t * npix + q]; }
      i2s_gather(img, ix, w, o);
    }
    if (inr) { map[3 * (size_t)q] = o[0]; map[3 * (size_t)q + 1] = o[1]; map[3 * (size_t)q + 2] = o[2]; }
    if (words && inr && (threadIdx.x & 31) == 0) words[q >> 5] = pwords[q >> 5];
  }
}

bool make_cam(const hpxgs_camera* cam, int W, int H, ImgCam& c) {
  if (!cam || W < 1 || H < 1 || W > 65536 || H > 65536) return false;
  if ((int64_t)W * H > 0xFFFFFFFFLL) return false;            // image pixel indices fit 32 bits
  c.kind = cam->kind; c.W = W; c.H = H; c.fx = c.fy = 1.f; c.wx = c.wy = 1.f;
  c.cx = (float)(0.5 * W); c.cy = (float)(0.5 * H);
  if (!valid_camera(*cam)) return false;
  if (cam->kind == HPXGS_CAM_PINHOLE) {
    c.fx = (float)(W / (2.0 * std::tan(0.5 * cam->fov_x_deg * kPi / 180.0)));
    c.fy = (float)(H / (2.0 * std::tan(0.5 * cam->fov_y_deg * kPi / 180.0)));
    c.cx = (float)(0.5 * W * (1.0 + (double)cam->ppx)); c.cy = (float)(0.5 * H * (1.0 + (double)cam->ppy));
  } else if (cam->kind == HPXGS_CAM_FISHEYE) {
    if (!(cam->fov_x_deg > 0 && cam->fov_x_deg <= 360 && cam->fov_y_deg > 0 && cam->fov_y_deg <= 360)) return false;
    c.fx = (float)(W / kPi); c.fy = (float)(H / kPi);
    c.wx = (float)(cam->fov_x_deg / 180.0); c.wy = (float)(cam->fov_y_deg / 180.0);
  } else if (cam->kind != HPXGS_CAM_FULL) {
    return false;
  }
  return true;
}

int grid_for(int64_t n) {
  const int64_t want = (n + kRsThreads - 1) / kRsThreads, cap = 8LL * num_sms();
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

}  // namespace
}  // namespace hpxgs

using namespace hpxgs;

extern "C" int hpxgs_sphere_to_image(const float* map, int nside_log2, const hpxgs_camera* cam, int width, int height,
                                     float* image, uint8_t* valid, hpxgs_stream_t stream) {
  ImgCam c;
  if (!map || !image || nside_log2 < 1 || nside_log2 > 13 || !make_cam(cam, width, height, c)) return HPXGS_E_INVALID_ARG;
  const int64_t n = (int64_t)width * height;
  k_sphere_to_image<<<grid_for(n), kRsThreads, 0, (cudaStream_t)stream>>>(map, nside_log2, c, image, valid);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

extern "C" int hpxgs_sphere_to_image_backward(const float* dimage, int nside_log2, const hpxgs_camera* cam, int width,
                                              int height, float* dmap, hpxgs_stream_t stream) {
  ImgCam c;
  if (!dimage || !dmap || nside_log2 < 1 || nside_log2 > 13 || !make_cam(cam, width, height, c))
    return HPXGS_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  HPXGS_CUDA_CHECK(cudaMemsetAsync(dmap, 0, sizeof(float) * 3 * (size_t)(12LL << (2 * nside_log2)), s));
  const int64_t n = (int64_t)width * height;
  k_sphere_to_image_bwd<<<grid_for(n), kRsThreads, 0, s>>>(dimage, nside_log2, c, dmap);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

template <typename T>
static int image_to_sphere(const T* image, int width, int height, const hpxgs_camera* cam, int nside_log2, float* map,
                           uint32_t* mask_bits, hpxgs_stream_t stream) {
  ImgCam c;
  if (!image || !map || nside_log2 < 2 || nside_log2 > 13 || !make_cam(cam, width, height, c)) return HPXGS_E_INVALID_ARG;
  ViewParams vp{};
  camera_params(*cam, nside_log2, vp);
  const int64_t npix = 12LL << (2 * nside_log2);
  // the grid-stride loop keeps whole warps together: blocks of 256 over a multiple of 32 pixels
  k_image_to_sphere<T><<<grid_for(npix), kRsThreads, 0, (cudaStream_t)stream>>>(image, c, vp, map, mask_bits);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

extern "C" int hpxgs_image_to_sphere(const float* image, int width, int height, const hpxgs_camera* cam, int nside_log2,
                                     float* map, uint32_t* mask_bits, hpxgs_stream_t stream) {
  return image_to_sphere(image, width, height, cam, nside_log2, map, mask_bits, stream);
}

extern "C" int hpxgs_image_to_sphere_u8(const uint8_t* image, int width, int height, const hpxgs_camera* cam,
                                        int nside_log2, float* map, uint32_t* mask_bits, hpxgs_stream_t stream) {
  return image_to_sphere(image, width, height, cam, nside_log2, map, mask_bits, stream);
}

// ---- resampling plans ----
static bool plan_args(int dir, int k, int W, int H) {
  if (dir != HPXGS_PLAN_SPHERE_TO_IMAGE && dir != HPXGS_PLAN_IMAGE_TO_SPHERE) return false;
  if (k < (dir == HPXGS_PLAN_SPHERE_TO_IMAGE ? 1 : 2) || k > 13) return false;
  return W >= 1 && H >= 1 && W <= 65536 && H <= 65536 && (int64_t)W * H <= 0xFFFFFFFFLL;
}

extern "C" int hpxgs_resample_plan_size(int direction, int nside_log2, int width, int height, size_t* bytes) {
  if (!bytes || !plan_args(direction, nside_log2, width, height)) return HPXGS_E_INVALID_ARG;
  *bytes = plan_layout(direction, nside_log2, width, height).total;
  return HPXGS_OK;
}

extern "C" int hpxgs_resample_plan_build(int direction, int nside_log2, const hpxgs_camera* cam, int width, int height,
                                         void* plan, size_t plan_bytes, hpxgs_stream_t stream) {
  ImgCam c;
  if (!plan || !plan_args(direction, nside_log2, width, height) || !make_cam(cam, width, height, c))
    return HPXGS_E_INVALID_ARG;
  const PlanLayout L = plan_layout(direction, nside_log2, width, height);
  if (plan_bytes < L.total) return HPXGS_E_WORKSPACE;
  char* b = static_cast<char*>(plan);
  cudaStream_t s = (cudaStream_t)stream;
  if (direction == HPXGS_PLAN_SPHERE_TO_IMAGE) {
    k_plan_s2i<<<grid_for(L.n), kRsThreads, 0, s>>>(nside_log2, c, reinterpret_cast<uint32_t*>(b + L.taps),
                                                    reinterpret_cast<float*>(b + L.w),
                                                    reinterpret_cast<uint8_t*>(b + L.extra));
  } else {
    ViewParams vp{};
    camera_params(*cam, nside_log2, vp);
    k_plan_i2s<<<grid_for(L.n), kRsThreads, 0, s>>>(c, vp, reinterpret_cast<uint32_t*>(b + L.taps),
                                                    reinterpret_cast<float*>(b + L.w),
                                                    reinterpret_cast<uint32_t*>(b + L.extra));
  }
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

extern "C" int hpxgs_sphere_to_image_planned(const float* map, int nside_log2, int width, int height, const void* plan,
                                             size_t plan_bytes, float* image, uint8_t* valid, hpxgs_stream_t stream) {
  if (!map || !image || !plan || !plan_args(HPXGS_PLAN_SPHERE_TO_IMAGE, nside_log2, width, height))
    return HPXGS_E_INVALID_ARG;
  const PlanLayout L = plan_layout(HPXGS_PLAN_SPHERE_TO_IMAGE, nside_log2, width, height);
  if (plan_bytes < L.total) return HPXGS_E_WORKSPACE;
  const char* b = static_cast<const char*>(plan);
  k_plan_s2i_apply<<<grid_for(L.n), kRsThreads, 0, (cudaStream_t)stream>>>(
      map, L.n, reinterpret_cast<const uint32_t*>(b + L.taps), reinterpret_cast<const float*>(b + L.w),
      reinterpret_cast<const uint8_t*>(b + L.extra), image, valid);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

extern "C" int hpxgs_sphere_to_image_backward_planned(const float* dimage, int nside_log2, int width, int height,
                                                      const void* plan, size_t plan_bytes, float* dmap,
                                                      hpxgs_stream_t stream) {
  if (!dimage || !dmap || !plan || !plan_args(HPXGS_PLAN_SPHERE_TO_IMAGE, nside_log2, width, height))
    return HPXGS_E_INVALID_ARG;
  const PlanLayout L = plan_layout(HPXGS_PLAN_SPHERE_TO_IMAGE, nside_log2, width, height);
  if (plan_bytes < L.total) return HPXGS_E_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  HPXGS_CUDA_CHECK(cudaMemsetAsync(dmap, 0, sizeof(float) * 3 * (size_t)(12LL << (2 * nside_log2)), s));
  const char* b = static_cast<const char*>(plan);
  k_plan_s2i_adjoint<<<grid_for(L.n), kRsThreads, 0, s>>>(dimage, L.n, reinterpret_cast<const uint32_t*>(b + L.taps),
                                                          reinterpret_cast<const float*>(b + L.w),
                                                          reinterpret_cast<const uint8_t*>(b + L.extra), dmap);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

template <typename T>
static int image_to_sphere_planned(const T* image, int width, int height, int nside_log2, const void* plan,
                                   size_t plan_bytes, float* map, uint32_t* mask_bits, hpxgs_stream_t stream) {
  if (!image || !map || !plan || !plan_args(HPXGS_PLAN_IMAGE_TO_SPHERE, nside_log2, width, height))
    return HPXGS_E_INVALID_ARG;
  const PlanLayout L = plan_layout(HPXGS_PLAN_IMAGE_TO_SPHERE, nside_log2, width, height);
  if (plan_bytes < L.total) return HPXGS_E_WORKSPACE;
  const char* b = static_cast<const char*>(plan);
  k_plan_i2s_apply<T><<<grid_for(L.n), kRsThreads, 0, (cudaStream_t)stream>>>(
      image, (uint32_t)L.n, reinterpret_cast<const uint32_t*>(b + L.taps), reinterpret_cast<const float*>(b + L.w),
      reinterpret_cast<const uint32_t*>(b + L.extra), map, mask_bits);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

extern "C" int hpxgs_image_to_sphere_planned(const float* image, int width, int height, int nside_log2,
                                             const void* plan, size_t plan_bytes, float* map, uint32_t* mask_bits,
                                             hpxgs_stream_t stream) {
  return image_to_sphere_planned(image, width, height, nside_log2, plan, plan_bytes, map, mask_bits, stream);
}

extern "C" int hpxgs_image_to_sphere_u8_planned(const uint8_t* image, int width, int height, int nside_log2,
                                                const void* plan, size_t plan_bytes, float* map, uint32_t* mask_bits,
                                                hpxgs_stream_t stream) {
  return image_to_sphere_planned(image, width, height, nside_log2, plan, plan_bytes, map, mask_bits, stream);
}
