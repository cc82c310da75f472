// The FoV test of a camera (Sec. 3.1; Sec. D.1), shared by the mask kernel and
// the image -> sphere resampling so that both give the same mask M_C.
#pragma once
#include "hpx_math.cuh"
#include "internal.cuh"

namespace hpxgs {

// Signed margin of camera direction d against the camera's valid region (>= 0
// inside). Pinhole (Eq. persp_sphere on [0,W] x [0,H], principal point anywhere
// inside): per axis the smaller of hi d_z - d and d - lo d_z, with [lo, hi] the
// frustum's range of d / d_z (for a centred camera: d_z tan(FoV/2) - |d|). Anisotropic equidistant fisheye (Eqs. fish_weff, imaging_region,
// semi_axes): psi <= (pi/2) w_eff(gamma), w_eff = sqrt((wx cos g)^2 + (wy sin g)^2)
// with cos g = dx / rxy, sin g = dy / rxy.
template <typename T>
__device__ __forceinline__ T camera_margin(int kind, T dx, T dy, T dz, T xlo, T xhi, T ylo, T yhi, T wx, T wy) {
  if (kind == HPXGS_CAM_PINHOLE) {
    const T ax = xhi * dz - dx, bx = dx - xlo * dz, ay = yhi * dz - dy, by = dy - ylo * dz;
    const T mx = ax < bx ? ax : bx, my = ay < by ? ay : by;
    return mx < my ? mx : my;
  }
  T rxy = sqrt(dx * dx + dy * dy);
  T psi = atan2(rxy, dz);
  T weff = rxy > T(0) ? sqrt(wx * wx * dx * dx + wy * wy * dy * dy) / rxy : wx;
  return T(0.5 * hpx::kPi) * weff - psi;
}

// M_C(p): the FP32 decision, taken again in FP64 when the FP32 margin is within
// 1e-4 of the boundary.
__device__ __forceinline__ bool pixel_in_mask(const ViewParams& vp, uint32_t p) {
  if (vp.kind == HPXGS_CAM_FULL) return true;
  float3 h = hpx::pix2vec_f32(vp.k, p);
  // camera direction (d_x, d_y, d_z) = HEALPix (Y, Z, X)
  float m = camera_margin<float>(vp.kind, h.y, h.z, h.x, vp.xlo, vp.xhi, vp.ylo, vp.yhi, vp.wx, vp.wy);
  if (fabsf(m) > 1e-4f) return m >= 0.0f;
  double3 hd = hpx::pix2vec_f64(vp.k, p);
  double md = camera_margin<double>(vp.kind, hd.y, hd.z, hd.x, vp.xlo64, vp.xhi64, vp.ylo64, vp.yhi64, vp.wx64,
                                           vp.wy64);
  return md >= 0.0;
}

}  // namespace hpxgs
