// HEALPix Gaussian rasterizer: forward (Algorithm 1) and backward (Sec. 3.2).
//
// Forward pipeline of hpxgs_forward, on the caller's stream and two helper streams:
//   k_mask            FoV masks and tile flags (helper stream, beside the preprocess)
//   k_preprocess      per (view, Gaussian): record (64 B), depth key, r_s
//   radix sort        Gaussians by float32 bits of the radial depth r (stable; high-
//                     priority helper stream, beside the count pass)
//   k_tiles<count>    per Gaussian: RING query + exact membership (after the masks)
//   scan              exclusive scan of the counts in depth order -> pair offsets, total
//   k_tiles<emit>     write (global tile, Gaussian id) pairs in depth order
//   radix sort        pairs by tile id only (stable: depth order is kept)
//   k_ranges          per-tile [start, end)
//   k_unit_*          longest-first order of the blend units
//   k_blend_fwd       persistent: blocks take units (tiles or tile quarters), one thread per pixel
// Backward (hpxgs_backward): k_unit_* (the backward's order, from the forward's unit
// times), k_blend_bwd (reverse walk, per-Gaussian partials, warp shuffles + one atomic
// per block and entry), k_preprocess_bwd.
//
// Geometry in the tangent-frame form: with g the unit direction of t = W mu + b
// and (e1, e2) the east/north tangents at g, S_phi J = [e1; e2] / r exactly
// (Eqs. 1-2), so Sigma_arc = (E W) Sigma3D (E W)^T / r^2. The pixel offset d is
// the azimuthal-equidistant coordinate of the pixel direction about g, which
// equals the haversine distance split by the bearing (Sec. 3.4).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "hpx_math.cuh"
#include "hssim_grad.cuh"
#include "internal.cuh"

using namespace hpx;

namespace hpxgs {

int launch_mask(const ViewParams& vp, int b, uint32_t* words, uint32_t* tile_flags, cudaStream_t s);

// Real SH normalisation constants sqrt((2l+1)/(4pi) (l-|m|)!/(l+|m|)!) (times sqrt2 for m != 0),
// folded into the Cartesian polynomials of degree <= 3 (3DGS order and signs).
__constant__ float kSH[10] = {0.28209479177387814f, 0.4886025119029199f, 1.0925484305920792f,
                              0.31539156525252005f, 0.5462742152960396f, 0.5900435899266435f,
                              2.890611442640554f,   0.4570457994644658f, 0.3731763325901154f,
                              1.445305721320277f};

// Basis Y_k(d), k < (deg+1)^2, and (optionally) its gradient in Cartesian coordinates.
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y, float3* dY) {
  const float C0 = kSH[0], C1 = kSH[1], C2a = kSH[2], C2b = kSH[3], C2c = kSH[4];
  const float C3a = kSH[5], C3b = kSH[6], C3c = kSH[7], C3d = kSH[8], C3e = kSH[9];
  Y[0] = C0;
  if (dY) dY[0] = make_float3(0.f, 0.f, 0.f);
  if (deg < 1) return;
  Y[1] = -C1 * y; Y[2] = C1 * z; Y[3] = -C1 * x;
  if (dY) { dY[1] = make_float3(0, -C1, 0); dY[2] = make_float3(0, 0, C1); dY[3] = make_float3(-C1, 0, 0); }
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = C2a * x * y; Y[5] = -C2a * y * z; Y[6] = C2b * (2.f * zz - xx - yy); Y[7] = -C2a * x * z;
  Y[8] = C2c * (xx - yy);
  if (dY) {
    dY[4] = make_float3(C2a * y, C2a * x, 0.f);
    dY[5] = make_float3(0.f, -C2a * z, -C2a * y);
    dY[6] = make_float3(-2.f * C2b * x, -2.f * C2b * y, 4.f * C2b * z);
    dY[7] = make_float3(-C2a * z, 0.f, -C2a * x);
    dY[8] = make_float3(2.f * C2c * x, -2.f * C2c * y, 0.f);
  }
  if (deg < 3) return;
  Y[9] = -C3a * y * (3.f * xx - yy);
  Y[10] = C3b * x * y * z;
  Y[11] = -C3c * y * (4.f * zz - xx - yy);
  Y[12] = C3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -C3c * x * (4.f * zz - xx - yy);
  Y[14] = C3e * z * (xx - yy);
  Y[15] = -C3a * x * (xx - 3.f * yy);
  if (dY) {
    dY[9] = make_float3(-6.f * C3a * x * y, -C3a * (3.f * xx - 3.f * yy), 0.f);
    dY[10] = make_float3(C3b * y * z, C3b * x * z, C3b * x * y);
    dY[11] = make_float3(2.f * C3c * x * y, -C3c * (4.f * zz - xx - 3.f * yy), -8.f * C3c * y * z);
    dY[12] = make_float3(-6.f * C3d * x * z, -6.f * C3d * y * z, C3d * (6.f * zz - 3.f * xx - 3.f * yy));
    dY[13] = make_float3(-C3c * (4.f * zz - 3.f * xx - yy), 2.f * C3c * x * y, -8.f * C3c * x * z);
    dY[14] = make_float3(2.f * C3e * x * z, -2.f * C3e * y * z, C3e * (xx - yy));
    dY[15] = make_float3(-C3a * (3.f * xx - 3.f * yy), 6.f * C3a * x * y, 0.f);
  }
}

// sum_k w_k grad Y_k(d) (the gradient formulas of sh_basis contracted with w), so
// that no per-k gradient has to be kept.
__device__ __forceinline__ float3 sh_grad_dot(int deg, float x, float y, float z, const float* w) {
  float3 g = make_float3(0.f, 0.f, 0.f);
  if (deg < 1) return g;
  const float C1 = kSH[1], C2a = kSH[2], C2b = kSH[3], C2c = kSH[4];
  const float C3a = kSH[5], C3b = kSH[6], C3c = kSH[7], C3d = kSH[8], C3e = kSH[9];
  g.x = -C1 * w[3]; g.y = -C1 * w[1]; g.z = C1 * w[2];
  if (deg < 2) return g;
  const float xx = x * x, yy = y * y, zz = z * z;
  g.x += C2a * (y * w[4] - z * w[7]) - 2.f * C2b * x * w[6] + 2.f * C2c * x * w[8];
  g.y += C2a * (x * w[4] - z * w[5]) - 2.f * C2b * y * w[6] - 2.f * C2c * y * w[8];
  g.z += -C2a * (y * w[5] + x * w[7]) + 4.f * C2b * z * w[6];
  if (deg < 3) return g;
  g.x += -6.f * C3a * x * y * w[9] + C3b * y * z * w[10] + 2.f * C3c * x * y * w[11] - 6.f * C3d * x * z * w[12]
         - C3c * (4.f * zz - 3.f * xx - yy) * w[13] + 2.f * C3e * x * z * w[14] - C3a * (3.f * xx - 3.f * yy) * w[15];
  g.y += -C3a * (3.f * xx - 3.f * yy) * w[9] + C3b * x * z * w[10] - C3c * (4.f * zz - xx - 3.f * yy) * w[11]
         - 6.f * C3d * y * z * w[12] + 2.f * C3c * x * y * w[13] - 2.f * C3e * y * z * w[14] + 6.f * C3a * x * y * w[15];
  g.z += C3b * x * y * w[10] - 8.f * C3c * y * z * w[11] + C3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12]
         - 8.f * C3c * x * z * w[13] + C3e * (xx - yy) * w[14];
  return g;
}

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

// Everything preprocess computes for one (view, Gaussian); shared by forward and backward.
struct Geo {
  bool valid;
  float3 t;          // camera frame
  float r;
  float3 g;          // HEALPix frame unit direction
  float3 e1, e2;     // HEALPix frame east / north
  float3 gc, e1c, e2c;  // same in the camera frame
  float a1[3], a2[3];   // rows of S_phi J W = W^T e_c / r (world frame)
  float R[9], s[3], qn[4], qnorm;
  float u1[3], u2[3];   // M^T a_i, M = R diag(s)
  float A, B, C;        // Sigma_arc (with blur)
  float qa, qb, qc;     // conic
  float rs;
};

// EXACT (the forward's preprocess): t = W mu + b and the radial depth r = |t| in FP64,
// each product and sum rounded once in a fixed order (the _rn intrinsics are never
// contracted into FMAs), so that float32(r) -- the sort key, the recorded depth and the
// near-plane test -- is the value any IEEE FP64 evaluation in this order gives; the FP32
// geometry starts from float32(t). Otherwise (the backward, which takes validity from
// the forward's radii) t and r in FP32, within rounding of the same values.
template <bool EXACT>
__device__ __forceinline__ void geo_compute(const ViewParams& vp, float near_plane, const float* __restrict__ mu,
                                            const float* __restrict__ sc, const float* __restrict__ q, Geo& G) {
  if constexpr (EXACT) {
    const double m0 = mu[0], m1 = mu[1], m2 = mu[2];
    double t64[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      t64[i] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn((double)vp.W[3 * i], m0), __dmul_rn((double)vp.W[3 * i + 1], m1)),
                                   __dmul_rn((double)vp.W[3 * i + 2], m2)),
                         (double)vp.b[i]);
    const double r64 = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(t64[0], t64[0]), __dmul_rn(t64[2], t64[2])),
                                            __dmul_rn(t64[1], t64[1])));
    G.t = make_float3(__double2float_rn(t64[0]), __double2float_rn(t64[1]), __double2float_rn(t64[2]));
    G.r = __double2float_rn(r64);
    G.valid = r64 > (double)near_plane;
  } else {
    const float m0 = mu[0], m1 = mu[1], m2 = mu[2];
    G.t.x = vp.W[0] * m0 + vp.W[1] * m1 + vp.W[2] * m2 + vp.b[0];
    G.t.y = vp.W[3] * m0 + vp.W[4] * m1 + vp.W[5] * m2 + vp.b[1];
    G.t.z = vp.W[6] * m0 + vp.W[7] * m1 + vp.W[8] * m2 + vp.b[2];
    G.r = sqrtf(G.t.x * G.t.x + G.t.y * G.t.y + G.t.z * G.t.z);
    G.valid = G.r > 0.f;
  }
  if (!G.valid) return;
  const float ir = 1.0f / G.r;
  G.gc = make_float3(G.t.x * ir, G.t.y * ir, G.t.z * ir);
  G.g = make_float3(G.gc.z, G.gc.x, G.gc.y);              // HEALPix (X, Y, Z) = camera (z, x, y)
  const float rho = sqrtf(G.g.x * G.g.x + G.g.y * G.g.y);
  if (rho > 1e-12f) {
    const float irho = 1.0f / rho;
    G.e1 = make_float3(-G.g.y * irho, G.g.x * irho, 0.f);
    G.e2 = make_float3(-G.g.x * G.g.z * irho, -G.g.y * G.g.z * irho, rho);
  } else {  // at the pole any tangent frame gives the same alpha; take a fixed one
    G.e1 = make_float3(0.f, 1.f, 0.f);
    G.e2 = make_float3(G.g.z > 0 ? -1.f : 1.f, 0.f, 0.f);
  }
  G.e1c = make_float3(G.e1.y, G.e1.z, G.e1.x);
  G.e2c = make_float3(G.e2.y, G.e2.z, G.e2.x);
  for (int j = 0; j < 3; ++j) {
    G.a1[j] = (vp.W[j] * G.e1c.x + vp.W[3 + j] * G.e1c.y + vp.W[6 + j] * G.e1c.z) * ir;
    G.a2[j] = (vp.W[j] * G.e2c.x + vp.W[3 + j] * G.e2c.y + vp.W[6 + j] * G.e2c.z) * ir;
  }
  G.qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const float iq = 1.0f / G.qnorm;
  for (int j = 0; j < 4; ++j) G.qn[j] = q[j] * iq;
  quat_rot(G.qn[0], G.qn[1], G.qn[2], G.qn[3], G.R);
  for (int j = 0; j < 3; ++j) G.s[j] = sc[j];
  for (int kk = 0; kk < 3; ++kk) {
    G.u1[kk] = G.s[kk] * (G.R[kk] * G.a1[0] + G.R[3 + kk] * G.a1[1] + G.R[6 + kk] * G.a1[2]);
    G.u2[kk] = G.s[kk] * (G.R[kk] * G.a2[0] + G.R[3 + kk] * G.a2[1] + G.R[6 + kk] * G.a2[2]);
  }
  G.A = G.u1[0] * G.u1[0] + G.u1[1] * G.u1[1] + G.u1[2] * G.u1[2] + vp.blur;
  G.B = G.u1[0] * G.u2[0] + G.u1[1] * G.u2[1] + G.u1[2] * G.u2[2];
  G.C = G.u2[0] * G.u2[0] + G.u2[1] * G.u2[1] + G.u2[2] * G.u2[2] + vp.blur;
  const float det = G.A * G.C - G.B * G.B;
  if (!(det > 0.f)) { G.valid = false; return; }
  const float idet = 1.0f / det;
  G.qa = G.C * idet; G.qb = -G.B * idet; G.qc = G.A * idet;
  const float hm = 0.5f * (G.A + G.C), hd = 0.5f * (G.A - G.C);
  const float lmax = hm + sqrtf(hd * hd + G.B * G.B);
  G.rs = 3.0f * sqrtf(lmax);
}

// ----------------------------------------------------------------------------
// k_preprocess: one thread per (view, Gaussian) id gid = v * P + i.
// ----------------------------------------------------------------------------
// Grid (P / kPreThreads, views): a block's SH rows are one contiguous span, loaded
// coalesced into shared memory (rows padded to 3K + 1 floats).
constexpr int kPreThreads = 128;
template <int DEG>
__global__ void __launch_bounds__(kPreThreads) k_preprocess(const __grid_constant__ ViewTable vt, hpxgs_gaussians gs,
                                                    float4* __restrict__ rec, float* __restrict__ radii,
                                                    float* __restrict__ depth, uint32_t* __restrict__ keys,
                                                    uint32_t* __restrict__ vals) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int RW = 3 * K + 1;
  __shared__ float s_sh[kPreThreads * RW];
  const int v = blockIdx.y;
  const int i0 = blockIdx.x * kPreThreads;
  const int nrow = min(kPreThreads, vt.P - i0);
  for (int t = threadIdx.x; t < nrow * 3 * K; t += kPreThreads) {
    const int r = t / (3 * K), c = t - r * (3 * K);
    s_sh[r * RW + c] = gs.sh[(int64_t)i0 * 3 * K + t];
  }
  __syncthreads();
  const int i = i0 + threadIdx.x;
  if (i >= vt.P) return;
  const int64_t gid = (int64_t)v * vt.P + i;
  const ViewParams& vp = vt.v[v];
  Geo G;
  geo_compute<true>(vp, vt.near_plane, gs.means + 3 * (int64_t)i, gs.scales + 3 * (int64_t)i, gs.rotations + 4 * (int64_t)i, G);
  vals[gid] = (uint32_t)gid;
  depth[gid] = G.r;
  // exact FoV-cap cull (the camera axis is the HEALPix X axis): no tile of the view can list it
  if (G.valid && vp.fov_cull >= 0.f && G.g.x < cosf(fminf((float)kPi, vp.fov_cull + G.rs))) G.valid = false;
  if (!G.valid) {
    keys[gid] = 0xffffffffu;
    radii[gid] = 0.f;
    rec[4 * gid + 0] = make_float4(0.f, 0.f, 1.f, 0.f);
    rec[4 * gid + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    rec[4 * gid + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
    rec[4 * gid + 3] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  // colour: SH at the world direction from the camera centre
  float dx = gs.means[3 * i] - vp.cam[0], dy = gs.means[3 * i + 1] - vp.cam[1], dz = gs.means[3 * i + 2] - vp.cam[2];
  const float idist = rsqrtf(dx * dx + dy * dy + dz * dz);
  dx *= idist; dy *= idist; dz *= idist;
  float Y[K];
  sh_basis(DEG, dx, dy, dz, Y, nullptr);
  const float* sh = s_sh + threadIdx.x * RW;
  float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
  for (int kk = 0; kk < K; ++kk)
#pragma unroll
    for (int c = 0; c < 3; ++c) col[c] += sh[3 * kk + c] * Y[kk];
#pragma unroll
  for (int c = 0; c < 3; ++c) col[c] = fmaxf(col[c], 0.f);
  rec[4 * gid + 0] = make_float4(G.g.x, G.g.y, G.g.z, gs.opacities[i]);
  rec[4 * gid + 1] = make_float4(G.e1.x, G.e1.y, G.e1.z, G.qa);
  rec[4 * gid + 2] = make_float4(G.e2.x, G.e2.y, G.e2.z, G.qb);
  rec[4 * gid + 3] = make_float4(col[0], col[1], col[2], G.qc);
  radii[gid] = G.rs;
  keys[gid] = __float_as_uint(G.r);     // r > 0: the bit pattern orders like the value
}

// ----------------------------------------------------------------------------
// Stable LSD radix sort of (u32 key, u32 value) pairs with a fixed grid of G
// blocks; each block owns a contiguous chunk, so no block waits on another.
// The element count is read on the device (min(*n, n_max)).
// ----------------------------------------------------------------------------
__device__ __forceinline__ void chunk_of(uint32_t n, int G, int b, uint32_t& begin, uint32_t& end) {
  uint32_t chunk = (n + G - 1) / G;
  chunk = (chunk + kSortTile - 1) / kSortTile * kSortTile;
  uint64_t bb = (uint64_t)chunk * b, ee = bb + chunk;
  begin = (uint32_t)(bb < n ? bb : n);
  end = (uint32_t)(ee < n ? ee : n);
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys, const uint32_t* n_ptr,
                                                            uint32_t n_max, int shift, int nbits,
                                                            uint32_t* __restrict__ hist, int G) {
  __shared__ uint32_t cnt[256];
  const uint32_t n = n_ptr ? min(*n_ptr, n_max) : n_max;
  uint32_t begin, end;
  chunk_of(n, G, blockIdx.x, begin, end);
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t mask = (1u << nbits) - 1u;
  for (uint32_t i = begin + threadIdx.x; i < end; i += kSortThreads) atomicAdd(&cnt[(keys[i] >> shift) & mask], 1u);
  __syncthreads();
  hist[threadIdx.x * G + blockIdx.x] = cnt[threadIdx.x];
}

// Digit-major exclusive scan of the per-block histograms hist[d * G + b], the order
// a stable LSD pass needs, in one launch of one block per digit row: each block scans
// its row in place and posts the row total; the block that finishes last (an atomic
// ticket, nothing waits) turns the totals into digit bases in place and resets the
// ticket. The scatter adds base[d] to the row prefix it reads.
__global__ void __launch_bounds__(256) k_scan_digit_rows(uint32_t* __restrict__ hist, int G,
                                                         uint32_t* __restrict__ base, uint32_t* ticket) {
  __shared__ uint32_t wsum[8];
  __shared__ bool s_last;
  const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* row = hist + (size_t)d * G;
  // each thread owns up to 4 consecutive entries of the row (G <= 1024)
  uint32_t v[4], t = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) { const int b = 4 * tid + q; v[q] = b < G ? row[b] : 0u; t += v[q]; }
  uint32_t x = t;
  for (int o = 1; o < 32; o <<= 1) { const uint32_t y = __shfl_up_sync(0xffffffffu, x, o); if (lane >= o) x += y; }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < 8 ? wsum[lane] : 0u;
    for (int o = 1; o < 8; o <<= 1) { const uint32_t y = __shfl_up_sync(0xffffffffu, w, o); if (lane >= o) w += y; }
    if (lane < 8) wsum[lane] = w;
  }
  __syncthreads();
  uint32_t run = x - t + (warp > 0 ? wsum[warp - 1] : 0u);
#pragma unroll
  for (int q = 0; q < 4; ++q) { const int b = 4 * tid + q; if (b < G) row[b] = run; run += v[q]; }
  if (tid == 0) {
    base[d] = wsum[7];                          // row total for now
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const uint32_t tot = tid < (int)gridDim.x ? *(volatile uint32_t*)&base[tid] : 0u;
  x = tot;
  for (int o = 1; o < 32; o <<= 1) { const uint32_t y = __shfl_up_sync(0xffffffffu, x, o); if (lane >= o) x += y; }
  __syncthreads();
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < 8 ? wsum[lane] : 0u;
    for (int o = 1; o < 8; o <<= 1) { const uint32_t y = __shfl_up_sync(0xffffffffu, w, o); if (lane >= o) w += y; }
    if (lane < 8) wsum[lane] = w;
  }
  __syncthreads();
  if (tid < (int)gridDim.x) base[tid] = x - tot + (warp > 0 ? wsum[warp - 1] : 0u);
  if (tid == 0) *ticket = 0u;
}

// Stable scatter of one pass over the block's chunk, one 4096-element tile at a
// time: warp w ranks the contiguous elements [w * 512, (w + 1) * 512) of the tile
// (16 rounds of 32, ranks from __match_any_sync plus a per-warp running count
// per digit); a digit-major scan over the warps gives each element its place in
// the tile sorted by digit; the tile is reordered in shared memory and written
// out so that elements of one digit go to consecutive addresses (full sectors).
#ifndef HPXGS_SCATTER_MINB
#define HPXGS_SCATTER_MINB 3
#endif
constexpr int kWarpSeg = kSortTile / (kSortThreads / 32);   // 512 elements per warp
constexpr int kSegRounds = kWarpSeg / 32;                   // 16
__global__ void __launch_bounds__(kSortThreads, HPXGS_SCATTER_MINB) k_sort_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                               uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                               const uint32_t* n_ptr, uint32_t n_max, int shift, int nbits,
                                                               const uint32_t* __restrict__ hist,
                                                               const uint32_t* __restrict__ dbase, int G) {
  constexpr int NW = kSortThreads / 32;
  __shared__ uint32_t s_key[kSortTile];        // 16 KB, tile in digit order
  __shared__ uint32_t s_val[kSortTile];        // 16 KB
  __shared__ uint32_t wcnt[NW][256];           // 8 KB: per-warp digit counts, then bases
  __shared__ uint32_t dstart[257];             // tile-local start of each digit
  __shared__ uint32_t gbase[256];              // next global position of each digit for this block
  __shared__ uint32_t wsum[NW];
  const uint32_t n = n_ptr ? min(*n_ptr, n_max) : n_max;
  uint32_t begin, end;
  chunk_of(n, G, blockIdx.x, begin, end);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t mask = (1u << nbits) - 1u;
  const uint32_t lt = (1u << lane) - 1u;
  gbase[tid] = tid <= (int)mask ? hist[tid * G + blockIdx.x] + dbase[tid] : 0u;
  for (uint32_t t0 = begin; t0 < end; t0 += kSortTile) {
    // ---- phase 1: per-warp ranks
    for (int d = lane; d < 256; d += 32) wcnt[warp][d] = 0;
    __syncwarp();
    uint32_t key[kSegRounds], val[kSegRounds], dr[kSegRounds];   // dr = digit << 16 | rank in warp segment
#pragma unroll
    for (int r = 0; r < kSegRounds; ++r) {
      const uint32_t idx = t0 + warp * kWarpSeg + r * 32 + lane;
      const bool valid = idx < end;
      key[r] = valid ? kin[idx] : 0u;
      val[r] = valid ? vin[idx] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kSegRounds; ++r) {
      const uint32_t idx = t0 + warp * kWarpSeg + r * 32 + lane;
      const bool valid = idx < end;
      const uint32_t digit = valid ? ((key[r] >> shift) & mask) : 0xffffu;
      const uint32_t peers = __match_any_sync(0xffffffffu, digit);
      const uint32_t before = valid ? wcnt[warp][digit] : 0u;
      __syncwarp();
      const uint32_t rk = __popc(peers & lt);
      if (valid && rk == 0) wcnt[warp][digit] = before + __popc(peers);
      __syncwarp();
      dr[r] = (digit << 16) | (before + rk);
    }
    __syncthreads();
    // ---- phase 2: digit-major scan over warps, then over digits
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) { const uint32_t c = wcnt[w][tid]; wcnt[w][tid] = tot; tot += c; }
    uint32_t inc = tot;
    for (int o = 1; o < 32; o <<= 1) { const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o); if (lane >= o) inc += y; }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += wsum[w];
    dstart[tid] = wpre + inc - tot;
    if (tid == kSortThreads - 1) dstart[256] = wpre + inc;
    __syncthreads();
    // ---- phase 3: reorder the tile in shared memory
#pragma unroll
    for (int r = 0; r < kSegRounds; ++r) {
      const uint32_t digit = dr[r] >> 16;
      if (digit != 0xffffu) {
        const uint32_t p = dstart[digit] + wcnt[warp][digit] + (dr[r] & 0xffffu);
        s_key[p] = key[r];
        s_val[p] = val[r];
      }
    }
    __syncthreads();
    // ---- phase 4: write runs of equal digits to consecutive global positions
    const uint32_t m = dstart[256];
    for (uint32_t i = tid; i < m; i += kSortThreads) {
      const uint32_t k = s_key[i];
      const uint32_t d = (k >> shift) & mask;
      const uint32_t pos = gbase[d] + (i - dstart[d]);
      kout[pos] = k;
      vout[pos] = s_val[i];
    }
    __syncthreads();
    gbase[tid] += dstart[tid + 1] - dstart[tid];
    __syncthreads();
  }
}

// Sorts n (device count, capped at n_max) pairs by bits [0, bits) of the key.
// Returns 0 if the result is in (k0, v0), 1 if in (k1, v1).
// hist holds 256 * G per-block counts followed by 256 digit bases; ticket is a
// zeroed counter (reset by every pass).
static int radix_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const uint32_t* n_dev, uint32_t n_max,
                      int bits, uint32_t* hist, int G, uint32_t* ticket, cudaStream_t s, int* which) {
  int cur = 0;
  if (n_max == 0) { *which = 0; return HPXGS_OK; }
  for (int shift = 0; shift < bits; shift += 8) {
    const int nb = min(8, bits - shift);
    uint32_t* kin = cur ? k1 : k0; uint32_t* vin = cur ? v1 : v0;
    uint32_t* kout = cur ? k0 : k1; uint32_t* vout = cur ? v0 : v1;
    k_sort_hist<<<G, kSortThreads, 0, s>>>(kin, n_dev, n_max, shift, nb, hist, G);
    k_scan_digit_rows<<<1 << nb, 256, 0, s>>>(hist, G, hist + 256 * (size_t)G, ticket);
    k_sort_scatter<<<G, kSortThreads, 0, s>>>(kin, vin, kout, vout, n_dev, n_max, shift, nb, hist,
                                              hist + 256 * (size_t)G, G);
    note_launches(3);
    HPXGS_LAUNCH_CHECK();
    cur ^= 1;
  }
  *which = cur;
  return HPXGS_OK;
}

// Blocks of kernel fn (threads per block) that can be resident at once: the largest
// grid of a cooperative launch (0 where the device has none).
static int coop_capacity(const void* fn, int threads) {
  int dev = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * num_sms();
}
template <typename... KArgs, typename... Args>
static cudaError_t launch_cooperative(void (*fn)(KArgs...), unsigned grid, unsigned threads, cudaStream_t s,
                                      Args... args) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(threads);
  lc.dynamicSmemBytes = 0;
  lc.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, fn, args...);
}
// Wait limit of a grid barrier in these launches.
constexpr uint64_t kGridWaitNs = 1000000000ull;   // 1 s

// ----------------------------------------------------------------------------
// Tile query (Algorithm 3 at the tile order) and exact membership:
// tile t is listed for Gaussian g iff t has an in-mask pixel and
// c_t . g >= cos(min(pi, r_s + rho + 1e-7)), decided in FP32 when the margin
// exceeds the FP32 error bound and in FP64 otherwise.
// ----------------------------------------------------------------------------
__device__ __forceinline__ float ring_of_z(float z, int Nt) {
  if (z > 2.0f / 3.0f) return Nt * sqrtf(3.0f * (1.0f - z));
  if (z < -2.0f / 3.0f) return 4.0f * Nt - Nt * sqrtf(3.0f * (1.0f + z));
  return Nt * (2.0f - 1.5f * z);
}

// phi / pi of ring pixel (i, j) as num / den (exact integers)
__device__ __forceinline__ void ring_phi_frac(int k, int i, int j, int& num, int& den) {
  const int N = 1 << k;
  if (i < N) { num = 2 * j + 1; den = 4 * i; }
  else if (i > 3 * N) { num = 2 * j + 1; den = 4 * (4 * N - i); }
  else { num = 2 * j + 2 - ((i - N + 1) & 1); den = 4 * N; }
}

// One warp per Gaussian: the rings of the disc are set up in parallel (one ring
// per lane), their candidate intervals are flattened with a warp scan, and the
// candidates are then evaluated 32 at a time, so a Gaussian that covers
// thousands of tiles does not stall its warp-mates. Members are compacted with
// a ballot, which keeps the emission order deterministic.
struct DiscQ {
  float zc, sc, omc, zmin, zmax, cosRe;
  float cosRm32, cosRa32, cosRq32;   // RING x f only: candidate, quick-accept and query-pixel thresholds
  float tin, tout;          // RING: chord-form thresholds of the membership test (see chord_bounds)
  int ilo, ihi;
};

// |g|^2 - 1 of an FP32 direction of unit length to FP32 rounding, to about 1e-13: each
// square is split exactly into its rounded product and the FMA remainder, the products
// are summed with Knuth's TwoSum, and the sum (within a few ulps of 1) minus 1 is exact
// (Sterbenz). The _rn intrinsics keep the compiler from contracting the products.
__device__ __forceinline__ float norm2_minus_1(float3 g) {
  const float px = __fmul_rn(g.x, g.x), py = __fmul_rn(g.y, g.y), pz = __fmul_rn(g.z, g.z);
  const float ex = fmaf(g.x, g.x, -px), ey = fmaf(g.y, g.y, -py), ez = fmaf(g.z, g.z, -pz);
  const float s1 = __fadd_rn(px, py);
  const float b1 = __fsub_rn(s1, px);
  const float e1 = __fadd_rn(__fsub_rn(px, __fsub_rn(s1, b1)), __fsub_rn(py, b1));
  const float s2 = __fadd_rn(s1, pz);
  const float b2 = __fsub_rn(s2, s1);
  const float e2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, b2)), __fsub_rn(pz, b2));
  return __fadd_rn(__fsub_rn(s2, 1.f), __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(ex, ey), ez)));
}

// Error bound of an FP32 ring-pixel centre (sth cos(phi), sth sin(phi), z) against the
// exact centre, as a vector norm: longitude (j + off) inv folded to (-1, 1] pi with two
// roundings (3.8e-7 rad), sincospif (5.3e-8 per component, the largest error over every
// float in [-1, 1]), sin(theta) (3.0e-7 in the belt near |z| = 2/3, 1.9e-7 in the caps)
// and z (8.3e-8): 9.2e-7 in all, taken with a margin of 2.
constexpr float kCentreErr32 = 2e-6f;
constexpr float kU32 = 5.9604645e-8f;     // 2^-24, the unit roundoff of FP32

// Chord form of the RING membership test. For the exact unit centre c and the FP32
// direction g, c . g = (1 + |g|^2 - |c - g|^2) / 2, so c . g >= cos R iff
// D = |c - g|^2 <= T = (|g|^2 - 1) + 4 sin^2(R / 2). The FP32 value d2 of D from the
// FP32 centre (within E = kCentreErr32) satisfies (sqrt(D) - E)^2 (1 - 6u) <= d2 <=
// (sqrt(D) + E)^2 (1 + 6u); bounding 2 sqrt(D) E by D E / s + s E with s = R gives
// linear bounds, so that d2 <= tin proves membership and d2 > tout proves the
// opposite; d2 in between takes the FP64 test. T is known to eT: sin(R / 2) from the
// FP32 R (3 roundings) and sinf (2 ulp), its square, |g|^2 - 1 (2e-13) and the FP64
// test's own rounding (1e-15); 16u in place of 6u covers the roundings of tin and tout.
__device__ __forceinline__ void chord_bounds(float3 g, float R, float sh, DiscQ& Q) {
  const float n2m1 = norm2_minus_1(g);
  const float T4 = 4.f * sh * sh;
  const float T = n2m1 + T4;
  const float eT = 32.f * kU32 * (T4 + fabsf(n2m1)) + 3e-13f;
  const float E = kCentreErr32, es = E / R;
  Q.tin = (T - eT - E * R - E * E) * (1.f - 16.f * kU32) / (1.f + es);
  Q.tout = (T + eT + E * R) * (1.f + 16.f * kU32) / (1.f - es);
}

// The exact membership test of ring pixel (i, j) at order kt, as the rule states it, in
// FP64. Out of line: inlined, the compiler issued parts of it (FP64 on this part issues at
// 1/64 the FP32 rate) on every candidate, not only on the few in the band.
__device__ __noinline__ bool ring_member_f64(int kt, int i, int j, float3 g, float rs, double rho) {
  const double cosR = cos(fmin(kPi, (double)rs + rho + 1e-7));
  const double3 c = ringpix_vec_f64(kt, i, j);
  return c.x * (double)g.x + c.y * (double)g.y + c.z * (double)g.z >= cosR;
}
// The same for query pixel p at order kq against r_s + rho_q (the RING x f query).
__device__ __noinline__ bool query_member_f64(int kq, uint32_t p, float3 g, float rs, double rhoq) {
  const double cosR = cos(fmin(kPi, (double)rs + rhoq + 1e-7));
  const double3 c = pix2vec_f64(kq, p);
  return c.x * (double)g.x + c.y * (double)g.y + c.z * (double)g.z >= cosR;
}

// RF: the RING query at search order k_t + log2f. Candidate tiles are the tiles whose
// centre lies within r_s + rho_q + rho_c (+1e-7) of the Gaussian, enumerated by
// Algorithm 3 at the tile order; each is then tested on its query pixels.
template <bool RF>
__device__ __forceinline__ void disc_setup(const ViewParams& vp, int kt, float3 g, float rs, int lane, DiscQ& Q) {
  (void)lane;
  const float rho_e = RF ? vp.rhoq32 + vp.rhoc32 : vp.rho32;
  // RF: FP32 thresholds of the candidate test at the tile centre and of the query-pixel
  // test (the RING query's own test takes the chord form, set up below)
  if (RF) {
    Q.cosRm32 = cosf(fminf((float)kPi, rs + rho_e + 1e-7f));
    const float Rq = fminf((float)kPi, rs + vp.rhoq32 + 1e-7f);
    Q.cosRq32 = cosf(Rq);
    Q.cosRa32 = cosf(fmaxf(0.f, Rq - vp.rhoc32));   // tile centre this close: all its query pixels pass
  }
  // Enumeration radius with slack. The stored centre g is unit length only to FP32 rounding,
  // and the membership test c . g >= cos(R) holds for directions within acos(cos R / |g|) of
  // g / |g|, a little more than R when |g| > 1 (by about (|g| - 1) / tan R, which matters for
  // small R): that angle is 2 asin sqrt(h), h = (|g| - 1 + 2 sin^2(R / 2)) / (2 |g|), taken
  // here with |g| - 1 at its largest (the FP32 error of g . g included). The rings and the
  // longitude intervals are then laid out about the normalised centre.
  const float R = fminf((float)kPi, rs + rho_e + 1e-7f);
  const float n2 = g.x * g.x + g.y * g.y + g.z * g.z;
  const float dg = 0.5f * fabsf(n2 - 1.f) + 1e-6f;
  const float sh = sinf(0.5f * R);
  if (!RF) chord_bounds(g, R, sh, Q);
  const float h = (dg + 2.f * sh * sh) / (2.f * (1.f - dg));
  const float Reff = h >= 1.f ? (float)kPi : 2.f * asinf(sqrtf(h));
  const float Re = fminf((float)kPi, fmaxf(R, Reff) + 1e-5f);
  float sRe, cRe;
  sincosf(Re, &sRe, &cRe);
  Q.cosRe = cRe;
  const int Nt = 1 << kt;
  const float ig = rsqrtf(n2);
  Q.zc = g.z * ig;
  Q.sc = sqrtf(fmaxf(0.f, g.x * g.x + g.y * g.y)) * ig;
  Q.omc = atan2f(g.y, g.x);
  // z range sin(phi_c -+ Re) = z_c cos Re -+ s_c sin Re; it reaches the north pole once
  // Re >= the centre's colatitude (cos Re <= z_c) and the south pole once cos Re <= -z_c
  Q.zmin = (cRe <= -Q.zc ? -1.f : Q.zc * cRe - Q.sc * sRe) - 1e-6f;
  Q.zmax = (cRe <= Q.zc ? 1.f : Q.zc * cRe + Q.sc * sRe) + 1e-6f;
  Q.ilo = max(1, (int)floorf(ring_of_z(fminf(Q.zmax, 1.f), Nt)) - 1);
  Q.ihi = min(4 * Nt - 1, (int)ceilf(ring_of_z(fmaxf(Q.zmin, -1.f), Nt)) + 1);
}

// Candidate positions [jlo, jlo + n) of ring i (Algorithm 3 with Eq. ring_phi_range).
// Also returns the ring's longitude as (j + off) * inv in units of pi.
__device__ __forceinline__ int ring_interval(int kt, int i, const DiscQ& Q, RingF& rg, int& jlo, float& off, float& inv) {
  rg = ring_f32(kt, i);
  const int N = 1 << kt;
  if (i < N) { off = 0.5f; inv = 1.f / (float)(2 * i); }
  else if (i > 3 * N) { off = 0.5f; inv = 1.f / (float)(2 * (4 * N - i)); }
  else { off = 1.f - 0.5f * (float)((i - N + 1) & 1); inv = 1.f / (float)(2 * N); }
  jlo = 0;
  if (rg.z < Q.zmin || rg.z > Q.zmax) return 0;
  const float delta = Q.sc * rg.sth;
  if (delta < 1e-6f) return (Q.zc * rg.z >= Q.cosRe - 1e-5f) ? rg.npix : 0;
  const float cw = (Q.cosRe - Q.zc * rg.z) / delta;
  if (cw <= -1.f) return rg.npix;
  if (cw > 1.f) return 0;
  const float dw = acosf(fminf(1.f, fmaxf(-1.f, cw)));
  const float sc2 = rg.npix / (2.0f * (float)kPi);
  // floor/ceil already take in every centre of the (slack-widened) interval
  jlo = (int)floorf((Q.omc - dw - rg.phi0) * sc2);
  const int jhi = (int)ceilf((Q.omc + dw - rg.phi0) * sc2);
  if (jhi - jlo + 1 >= rg.npix) { jlo = 0; return rg.npix; }
  return jhi - jlo + 1;
}

// Half-width of the band around the FP32 threshold of the RING x f candidate test
// (the tile-centre pre-test and the quick accept). The FP32 dot and threshold are within 1.6e-6 of their exact
// values: longitude folded to (-1, 1] pi (3.8e-7), sincospif's 1 ulp (0.9e-7), the
// dot's four roundings (2.4e-7), the ring's z and sin(theta) (2.4e-7), and the
// threshold's argument (up to 4.8e-7 at r_s + rho near pi) and cosf's 2 ulp
// (1.2e-7). An FP32 emulation at Nside 512 with 300k Gaussians stays within 2e-7.
constexpr float kBand32 = 3e-6f;
// Band of the RING x f query-pixel test, whose centres come from pix2vec_f32 (the
// NESTED query's band).
constexpr float kBandQ32 = 1e-5f;

// Count pass (EMIT = false), over the Gaussians in index order: counts members
// (counts[gid]) and stages up to kStage member tiles per Gaussian in shared memory,
// then copies them to a scratch list at a slot taken from an atomic counter
// (stage[gid] = slot, or ~0 when the Gaussian has more members or the scratch is
// full). Emit pass (EMIT = true), over the depth-sorted positions j: staged Gaussians
// copy their list to offsets[j]; the others run the query again and write directly.
constexpr int kStage = 256;
// RING band candidates a warp queues per Gaussian for the FP64 test (more: the Gaussian's
// candidates are scanned again, testing the band in place). The band is about 4e-6 rad wide,
// so a Gaussian of radius R at tile spacing s has about 2 pi sin(R) 4e-6 / s^2 of them: 25 for
// a hemisphere at the finest tile order (10), well under one at the training workload's.
#ifndef HPXGS_BAND_QUEUE
#define HPXGS_BAND_QUEUE 32
#endif
constexpr int kBandQueue = HPXGS_BAND_QUEUE;
// Gaussians a warp sets up together (one per lane) before running their queries.
#ifndef HPXGS_TILES_BATCH
#define HPXGS_TILES_BATCH 16
#endif
constexpr int kTilesBatch = HPXGS_TILES_BATCH;
// A Gaussian's query setup as one lane leaves it for its warp.
struct TileSet {
  DiscQ Q;
  float3 g;
  float rs;
  uint32_t gid, slot, n;
  uint64_t base;
};

template <bool EMIT, bool RF>
__global__ void __launch_bounds__(256, 4) k_tiles(const __grid_constant__ ViewTable vt, const float4* __restrict__ rec,
                                               const float* __restrict__ radii, const uint32_t* __restrict__ skeys,
                                               const uint32_t* __restrict__ svals, const uint32_t* __restrict__ flags,
                                               uint32_t* __restrict__ counts, const uint64_t* __restrict__ offsets,
                                               uint32_t* __restrict__ out_tile, uint32_t* __restrict__ out_id, uint64_t cap,
                                               int32_t* status, uint32_t* __restrict__ stage,
                                               uint32_t* __restrict__ scratch, uint32_t* scratch_top) {
  __shared__ uint32_t s_stage[8][kStage];
  __shared__ TileSet s_set[8][kTilesBatch];
  __shared__ uint32_t s_band[8][kBandQueue];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t PV = (int64_t)vt.P * vt.nviews;
  const int64_t wpb = blockDim.x >> 5;
  // A warp takes kTilesBatch consecutive Gaussians: lane t loads and sets up Gaussian
  // jb + t into the warp's slot table (FoV-invisible ones are dropped here), then the
  // warp runs the query of each in turn.
  const int64_t nwarps = (int64_t)gridDim.x * wpb;
  for (int64_t jb = (blockIdx.x * wpb + wib) * (int64_t)kTilesBatch; jb < PV; jb += nwarps * kTilesBatch) {
    bool vl = false;
    if (lane < kTilesBatch && jb + lane < PV) {
      // count pass: jl is the Gaussian itself (no depth order needed: it runs beside the depth
      // sort); emit pass: its depth-sorted position
      const int64_t jl = jb + lane;
      const bool listed = EMIT ? skeys[jl] != 0xffffffffu : radii[jl] > 0.f;
      if (!listed) {
        if (!EMIT) counts[jl] = 0;
      } else {
        vl = true;
        TileSet& ts = s_set[wib][lane];
        ts.gid = EMIT ? svals[jl] : (uint32_t)jl;
        ts.slot = EMIT ? stage[ts.gid] : 0xffffffffu;
        if (EMIT) { ts.n = counts[ts.gid]; ts.base = offsets[jl]; }
        if (!EMIT || ts.slot == 0xffffffffu) {
          const ViewParams& vpl = vt.v[ts.gid / (uint32_t)vt.P];
          const float4 r0 = rec[4 * (int64_t)ts.gid];
          const float3 gl = make_float3(r0.x, r0.y, r0.z);
          const float rsl = radii[ts.gid];
          DiscQ Ql;
          disc_setup<RF>(vpl, vpl.k - vt.b, gl, rsl, lane, Ql);
          ts.g = gl; ts.rs = rsl; ts.Q = Ql;
        }
      }
    }
    const uint32_t todo0 = __ballot_sync(FULL, vl);
    __syncwarp();
    for (uint32_t todo = todo0; todo; todo &= todo - 1u) {
    const int t = __ffs(todo) - 1;
    const int64_t j = jb + t;
    const TileSet& ts = s_set[wib][t];
    const uint32_t gid = ts.gid;
    if (EMIT) {
      const uint32_t slot = ts.slot;
      if (slot != 0xffffffffu) {                     // staged by the count pass: copy
        const uint32_t n = ts.n;
        const uint64_t base = ts.base;
        for (uint32_t e = lane; e < n; e += 32) {
          const uint64_t p = base + e;
          if (p < cap) { out_tile[p] = scratch[slot + e]; out_id[p] = gid; }
        }
        if (lane == 0 && base + n > cap && status) atomicOr(status, HPXGS_F_CAPACITY);
        continue;
      }
    }
    const int v = (int)(gid / (uint32_t)vt.P);
    const ViewParams& vp = vt.v[v];
    const int kt = vp.k - vt.b;
    const float3 g = ts.g;
    const DiscQ Q = ts.Q;
    const float rs = ts.rs;
    const uint64_t base = EMIT ? ts.base : 0;
    uint32_t cnt = 0;
    // appends this step's members (lane order) to the Gaussian's list
    auto append = [&](bool member, uint32_t gt) {
      const uint32_t bal = __ballot_sync(FULL, member);
      if (member) {
        const uint32_t r = cnt + __popc(bal & lt);
        if (EMIT) {
          const uint64_t p = base + r;
          if (p < cap) { out_tile[p] = gt; out_id[p] = gid; }
        } else if (r < kStage) {
          s_stage[wib][r] = gt;
        }
      }
      cnt += __popc(bal);
    };
    // RING: the exact FP64 test of a band candidate, then the tile's flag
    auto band_member = [&](int ii, int jj, uint32_t& gt) -> bool {
      if (!ring_member_f64(kt, ii, jj, g, rs, vp.rho)) return false;
      const FaceXY fx = ring_to_fxy(kt, ii, jj);
      gt = (uint32_t)vp.tile_base + fxy_to_nest(kt, fx.f, fx.x, fx.y);
      return flags[gt] & 1u;
    };
    uint32_t nq = 0;                           // RING: band candidates, queued in s_band
    // The candidates of the Gaussian. BAND = false: each is decided in FP32 and the few in the
    // RING band are queued, to take the FP64 test after the loop, so that the loop itself makes
    // no call. BAND = true (a Gaussian whose band overflowed the queue): only the band
    // candidates, each tested in place.
    auto scan = [&](auto band_pass) {
      constexpr bool BAND = decltype(band_pass)::value;
      for (int r0i = Q.ilo; r0i <= Q.ihi; r0i += 32) {
        const int i = r0i + lane;
        RingF rg; rg.z = 0.f; rg.sth = 0.f; rg.phi0 = 0.f; rg.npix = 1;
        int jlo = 0, nc = 0;
        float off = 0.f, inv = 0.f;
        if (i <= Q.ihi) nc = ring_interval(kt, i, Q, rg, jlo, off, inv);
        int inc = nc;
        for (int o = 1; o < 32; o <<= 1) { const int y = __shfl_up_sync(FULL, inc, o); if (lane >= o) inc += y; }
        const int total = __shfl_sync(FULL, inc, 31);
        const int exc = inc - nc;
        for (int q0 = 0; q0 < total; q0 += 32) {
          const int q = q0 + lane;
          // owner ring of candidate q: the number of leading lanes whose inclusive count is <= q
          int pos = 0;
          for (int step = 16; step > 0; step >>= 1) {
            const int val = __shfl_sync(FULL, inc, pos + step - 1);
            if (val <= q) pos += step;
          }
          const int o_exc = __shfl_sync(FULL, exc, pos);
          const int o_jlo = __shfl_sync(FULL, jlo, pos);
          const float o_z = __shfl_sync(FULL, rg.z, pos);
          const float o_sth = __shfl_sync(FULL, rg.sth, pos);
          const int o_np = __shfl_sync(FULL, rg.npix, pos);
          const float o_off = __shfl_sync(FULL, off, pos);
          const float o_inv = __shfl_sync(FULL, inv, pos);
          bool member = false, band = false;
          uint32_t gt = 0;
          const int ii = r0i + pos;
          int jj = o_jlo + (q - o_exc);          // within (-np, 2 np)
          if (q < total) {
            if (jj < 0) jj += o_np;
            if (jj >= o_np) jj -= o_np;
            // longitude / pi = (jj + off) inv = n / d with n = 2 (jj + off) and d = 4 / (2 inv), the
            // ring's pixel count; folded exactly to (-1, 1] so that its FP32 rounding is at most
            // 2^-23 in units of pi (0.5 inv = fl(1 / d))
            int n = 2 * jj + (int)(2.f * o_off);
            if (n > o_np) n -= 2 * o_np;
            float sp, cp;
            sincospif((float)n * (0.5f * o_inv), &sp, &cp);
            if (!RF) {
              // squared chord to the candidate's centre against the Gaussian's bounds; the
              // few candidates between them take the exact test in FP64
              const float dx = fmaf(o_sth, cp, -g.x), dy = fmaf(o_sth, sp, -g.y), dz = __fsub_rn(o_z, g.z);
              const float d2 = fmaf(dx, dx, fmaf(dy, dy, __fmul_rn(dz, dz)));
              if (BAND) {
                if (d2 > Q.tin && d2 <= Q.tout) member = band_member(ii, jj, gt);
              } else if (d2 <= Q.tin) {
                const FaceXY fx = ring_to_fxy(kt, ii, jj);
                gt = (uint32_t)vp.tile_base + fxy_to_nest(kt, fx.f, fx.x, fx.y);
                member = flags[gt] & 1u;
              } else if (d2 <= Q.tout) {
                band = true;
              }
            } else if (const float dot = o_sth * (cp * g.x + sp * g.y) + o_z * g.z; dot >= Q.cosRm32 - kBand32) {
              // a candidate tile: listed when one of its 4^log2f query pixels has its centre
              // within r_s + rho_q (+1e-7) of g, decided in FP32 and, within kBandQ32 of the
              // threshold, in FP64 as the membership rule states it
              const FaceXY fx = ring_to_fxy(kt, ii, jj);
              const uint32_t tn = fxy_to_nest(kt, fx.f, fx.x, fx.y);
              gt = (uint32_t)vp.tile_base + tn;
              if (flags[gt] & 1u) {
                if (dot > Q.cosRa32 + kBand32) {
                  member = true;
                } else {
                  const int L = vt.log2f, kq = kt + L;
                  for (uint32_t c = 0; c < (1u << (2 * L)) && !member; ++c) {
                    const uint32_t qp = (tn << (2 * L)) | c;
                    const float3 cq = pix2vec_f32(kq, qp);
                    const float dq = cq.x * g.x + cq.y * g.y + cq.z * g.z;
                    if (dq > Q.cosRq32 + kBandQ32) member = true;
                    else if (dq >= Q.cosRq32 - kBandQ32) member = query_member_f64(kq, qp, g, rs, vp.rhoq);
                  }
                }
              }
            }
          }
          append(member, gt);
          if (!RF && !BAND) {
            const uint32_t bb = __ballot_sync(FULL, band);
            if (bb) {
              if (band) {
                const uint32_t r = nq + __popc(bb & lt);
                if (r < kBandQueue) s_band[wib][r] = ((uint32_t)ii << 16) | (uint32_t)jj;   // ii, jj < 2^15
              }
              nq += __popc(bb);
            }
          }
        }
      }
    };
    scan(std::false_type{});
    if constexpr (!RF) {
      if (nq > kBandQueue) {
        scan(std::true_type{});
      } else if (nq > 0) {
        __syncwarp();
        for (uint32_t e0 = 0; e0 < nq; e0 += 32) {
          const uint32_t e = e0 + lane;
          bool member = false;
          uint32_t gt = 0;
          if (e < nq) {
            const uint32_t w = s_band[wib][e];
            member = band_member((int)(w >> 16), (int)(w & 0xffffu), gt);
          }
          append(member, gt);
        }
        __syncwarp();                              // the queue is refilled by the next Gaussian
      }
    }
    if (EMIT) {
      if (lane == 0 && base + cnt > cap && status) atomicOr(status, HPXGS_F_CAPACITY);
    } else {
      uint32_t slot = 0xffffffffu;
      if (cnt <= kStage && cnt > 0) {
        if (lane == 0) slot = atomicAdd(scratch_top, cnt);
        slot = __shfl_sync(FULL, slot, 0);
        if ((uint64_t)slot + cnt > cap) slot = 0xffffffffu;     // scratch full: emit runs the query again
        else for (uint32_t e = lane; e < cnt; e += 32) scratch[slot + e] = s_stage[wib][e];
      } else if (cnt == 0) {
        slot = 0u;
      }
      __syncwarp();
      if (lane == 0) { counts[gid] = cnt; stage[gid] = slot; }
    }
    }
    __syncwarp();                                    // the table is refilled by the next batch
  }
}

// ----------------------------------------------------------------------------
// Exclusive scan of u32 counts into u64 offsets (fixed grid, no inter-block waits).
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint64_t block_exclusive_scan_u64(uint64_t x, uint64_t* total) {
  __shared__ uint64_t ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint64_t inc = x;
  for (int o = 1; o < 32; o <<= 1) { uint64_t y = __shfl_up_sync(0xffffffffu, inc, o); if (lane >= o) inc += y; }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < nw ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) { uint64_t y = __shfl_up_sync(0xffffffffu, w, o); if (lane >= o) w += y; }
    ws[lane] = w;
  }
  __syncthreads();
  const uint64_t res = inc - x + (warp > 0 ? ws[warp - 1] : 0);
  *total = ws[nw - 1];
  __syncthreads();
  return res;
}

// The counts are per Gaussian; the scan takes them in depth order, c[perm[i]].
__global__ void __launch_bounds__(256) k_scan_part(const uint32_t* __restrict__ c, const uint32_t* __restrict__ perm,
                                                   int64_t n, int G, uint64_t* part) {
  const int64_t chunk = (n + G - 1) / G;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  uint64_t s = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += c[perm[i]];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ uint64_t ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    part[blockIdx.x] = t;
  }
}

// One block of kMaxSortBlocks threads: exclusive scan of the G <= kMaxSortBlocks partials.
__global__ void __launch_bounds__(kMaxSortBlocks) k_scan_top(uint64_t* part, int G, uint32_t* counters,
                                                           uint64_t* total_out) {
  const int t = threadIdx.x;
  const uint64_t v = t < G ? part[t] : 0;
  uint64_t run;
  const uint64_t ex = block_exclusive_scan_u64(v, &run);
  if (t < G) part[t] = ex;
  if (t == 0) {
    part[G] = run;
    counters[C_NPAIRS] = (uint32_t)(run > 0xffffffffull ? 0xffffffffull : run);
    counters[C_NPAIRS_HI] = (uint32_t)(run >> 32);
    if (total_out) *total_out = run;
  }
}

__global__ void __launch_bounds__(256) k_scan_apply(const uint32_t* __restrict__ c, const uint32_t* __restrict__ perm,
                                                    int64_t n, int G, const uint64_t* __restrict__ part,
                                                    uint64_t* __restrict__ off) {
  const int64_t chunk = (n + G - 1) / G;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  uint64_t run = part[blockIdx.x];
  for (int64_t t0 = lo; t0 < hi; t0 += blockDim.x) {
    const int64_t i = t0 + threadIdx.x;
    const uint64_t x = i < hi ? c[perm[i]] : 0;
    uint64_t tot;
    const uint64_t ex = block_exclusive_scan_u64(x, &tot);
    if (i < hi) off[i] = run + ex;
    run += tot;
  }
}

// The three phases above as one cooperative launch of G resident blocks, a grid
// barrier (on *bar, zero before the launch) between the chunk sums and their use.
__global__ void __launch_bounds__(256) k_scan_coop(const uint32_t* __restrict__ c, const uint32_t* __restrict__ perm,
                                                   int64_t n, uint64_t* part,
                                                   uint64_t* __restrict__ off, uint32_t* counters,
                                                   uint64_t* total_out, uint32_t* bar, int32_t* status) {
  const int G = gridDim.x, b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t chunk = (n + G - 1) / G;
  const int64_t lo = b * chunk, hi = min(n, lo + chunk);
  __shared__ uint64_t ws[2][8];
  uint64_t s = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += c[perm[i]];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) ws[0][warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < 8; ++w) t += ws[0][w];
    part[b] = t;
  }
  if (!grid_barrier(bar, (uint32_t)G, kGridWaitNs, status)) return;
  // this block's prefix and the total, from every block's chunk sum
  uint64_t pre = 0, tot = 0;
  for (int q = threadIdx.x; q < G; q += blockDim.x) {
    const uint64_t x = __ldcg(reinterpret_cast<const unsigned long long*>(part) + q);
    tot += x;
    if (q < b) pre += x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    pre += __shfl_xor_sync(0xffffffffu, pre, o);
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
  }
  if (lane == 0) { ws[0][warp] = pre; ws[1][warp] = tot; }
  __syncthreads();
  uint64_t run = 0, total = 0;
  for (int w = 0; w < 8; ++w) { run += ws[0][w]; total += ws[1][w]; }
  if (b == 0 && threadIdx.x == 0) {
    part[G] = total;
    counters[C_NPAIRS] = (uint32_t)(total > 0xffffffffull ? 0xffffffffull : total);
    counters[C_NPAIRS_HI] = (uint32_t)(total >> 32);
    if (total_out) *total_out = total;
  }
  for (int64_t t0 = lo; t0 < hi; t0 += blockDim.x) {
    const int64_t i = t0 + threadIdx.x;
    const uint64_t x = i < hi ? c[perm[i]] : 0;
    uint64_t t;
    const uint64_t ex = block_exclusive_scan_u64(x, &t);
    if (i < hi) off[i] = run + ex;
    run += t;
  }
}

// ----------------------------------------------------------------------------
// Per-tile ranges over the sorted tile ids (Algorithm 1: [start_t, end_t)).
// ----------------------------------------------------------------------------
// Each thread takes 4 consecutive ids in one 16-byte load; the neighbours across threads
// come by shuffles, across warps by one load at each end.
__global__ void k_ranges(const uint32_t* __restrict__ tiles, const uint32_t* n_ptr, uint32_t n_max, uint2* ranges) {
  const uint32_t n = min(*n_ptr, n_max);
  const int lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x * 4u;
  for (uint32_t i0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4u; i0 - 4u * (uint32_t)lane < n; i0 += stride) {
    uint32_t t[4];
    if (i0 + 3u < n) {
      const uint4 v = *reinterpret_cast<const uint4*>(tiles + i0);
      t[0] = v.x; t[1] = v.y; t[2] = v.z; t[3] = v.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) t[k] = i0 + k < n ? tiles[i0 + k] : 0xffffffffu;
    }
    uint32_t prev = __shfl_up_sync(0xffffffffu, t[3], 1);
    uint32_t next = __shfl_down_sync(0xffffffffu, t[0], 1);
    if (lane == 0) prev = (i0 > 0u && i0 <= n) ? tiles[i0 - 1] : 0xffffffffu;
    if (lane == 31) next = i0 + 4u < n ? tiles[i0 + 4] : 0xffffffffu;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t i = i0 + k;
      if (i >= n) break;
      const uint32_t left = k ? t[k - 1] : prev, right = k < 3 ? t[k + 1] : next;
      if (i == 0 || left != t[k]) ranges[t[k]].x = i;
      if (i == n - 1 || right != t[k]) ranges[t[k]].y = i + 1;
    }
  }
}

// ----------------------------------------------------------------------------
// NESTED quadtree query (Algorithm 2): one thread per Gaussian (count pass: in index order; emit: in depth order),
// an explicit stack of (pixel, order) nodes from the 12 base pixels down to the
// tile order + log2 f. A node is pruned when the angle d from the Gaussian
// centre to the node centre exceeds r_s + PixRad(o) (zone 0); a node with
// d <= r_s (zones 2, 3) at or below the tile order adds its tile; other nodes
// are refined, and a node left at the deepest order adds its tile (zone 1).
// Each test is decided in FP32 and again in FP64 within 1e-5 of its threshold.
// The nodes inside a tile are visited consecutively, so a tile added twice is
// added twice in a row: one comparison removes repeats. The stack never holds
// more than 12 + 3 (deepest order) <= 45 entries.
// ----------------------------------------------------------------------------
constexpr int kNestStack = 48;

// d(node, g) <= ang, i.e. node . g >= cos(min(pi, ang)) for the unit vector g, as FP64
// decides it. The stored centre is unit length only to FP32 rounding, and near small
// angles that rounding moves the angle by cot(d) times as much, so both paths normalise:
// `gn` in FP32; `graw` again in FP64 for a decision within 1e-5 of the threshold. (Kept
// inline: out of line, as the RING query's FP64 test is, this query ran slower.)
__device__ __forceinline__ bool node_within(float dot, float ang32, double ang, int o, uint32_t p, float3 graw) {
  const float c32 = cosf(fminf((float)kPi, ang32));
  if (dot > c32 + 1e-5f) return true;
  if (dot < c32 - 1e-5f) return false;
  const double3 c = pix2vec_f64(o, p);
  const double gx = graw.x, gy = graw.y, gz = graw.z;
  const double inv = 1.0 / sqrt(gx * gx + gy * gy + gz * gz);
  return (c.x * gx + c.y * gy + c.z * gz) * inv >= cos(fmin(kPi, ang));
}

template <bool EMIT>
__global__ void __launch_bounds__(256) k_tiles_nested(const __grid_constant__ ViewTable vt, const float4* __restrict__ rec,
                                                      const float* __restrict__ radii, const uint32_t* __restrict__ skeys,
                                                      const uint32_t* __restrict__ svals, const uint32_t* __restrict__ flags,
                                                      uint32_t* __restrict__ counts, const uint64_t* __restrict__ offsets,
                                                      uint32_t* __restrict__ out_tile, uint32_t* __restrict__ out_id,
                                                      uint64_t cap, int32_t* status) {
  const int64_t PV = (int64_t)vt.P * vt.nviews;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < PV; j += (int64_t)gridDim.x * blockDim.x) {
    // count pass: j is the Gaussian itself; emit pass: its depth-sorted position
    const bool listed = EMIT ? skeys[j] != 0xffffffffu : radii[j] > 0.f;
    if (!listed) { if (!EMIT) counts[j] = 0; continue; }
    const uint32_t gid = EMIT ? svals[j] : (uint32_t)j;
    const ViewParams& vp = vt.v[gid / (uint32_t)vt.P];
    const int kt = vp.k - vt.b, kmax = kt + vt.log2f;
    const float4 r0 = rec[4 * (int64_t)gid];
    const float3 g = make_float3(r0.x, r0.y, r0.z);
    const float ig = rsqrtf(g.x * g.x + g.y * g.y + g.z * g.z);
    const float3 gn = make_float3(g.x * ig, g.y * ig, g.z * ig);
    const float rs = radii[gid];
    const uint64_t base = EMIT ? offsets[j] : 0;
    uint32_t stack[kNestStack];                 // (p << 4) | o; p < 12 * 4^11 < 2^26
    int sp = 0;
    for (int f = 11; f >= 0; --f) stack[sp++] = (uint32_t)f << 4;
    uint32_t cnt = 0, last = 0xffffffffu;
    while (sp > 0) {
      const uint32_t e = stack[--sp];
      const int o = (int)(e & 15u);
      const uint32_t p = e >> 4;
      const float3 c = pix2vec_f32(o, p);
      const float dot = c.x * gn.x + c.y * gn.y + c.z * gn.z;
      const float pr32 = vt.pixrad32[o];
      const double pr = vt.pixrad64[o];
      if (!node_within(dot, rs + pr32, (double)rs + pr, o, p, g)) continue;          // zone 0
      const bool centre_in = node_within(dot, rs, (double)rs, o, p, g);            // zones 2 and 3
      bool add = false;
      if (centre_in && o >= kt) add = true;
      else if (o < kmax) {
        if (sp + 4 > kNestStack) break;       // cannot happen (see above); keeps the array in bounds
        for (int ch = 3; ch >= 0; --ch) stack[sp++] = ((4u * p + (uint32_t)ch) << 4) | (uint32_t)(o + 1);
      } else add = true;
      if (!add) continue;
      const uint32_t t = p >> (2 * (o - kt));
      if (t == last) continue;
      last = t;
      const uint32_t gt = (uint32_t)vp.tile_base + t;
      if (!(flags[gt] & 1u)) continue;
      if (EMIT) {
        const uint64_t q = base + cnt;
        if (q < cap) { out_tile[q] = gt; out_id[q] = gid; }
      }
      ++cnt;
    }
    if (!EMIT) counts[gid] = cnt;
    else if (base + cnt > cap && status) atomicOr(status, HPXGS_F_CAPACITY);
  }
}

// ----------------------------------------------------------------------------
// Per-pixel weight. m = d^T conic d with d = (theta / s) u, u = (delta.e1, delta.e2),
// delta = p - g, s = |u| = sin(theta), cos(theta) = 1 - |delta|^2 / 2.
// (theta/s)^2 = asin(s)^2 / s^2 by its Taylor series near the centre
// (1 + s^2/3 + 8 s^4/45 + 4 s^6/35 + 128 s^8/1575), atan2 further out.
// ----------------------------------------------------------------------------
// Lanes of a warp whose backward partials are summed by shuffles before they go
// to shared memory (a power of two, 1 .. 32).
#ifndef HPXGS_BWD_RED_LANES
#define HPXGS_BWD_RED_LANES 8
#endif
constexpr float kSeriesN2 = 0.04f;      // |delta|^2 below which the series is used (theta < 0.2)

struct Pix {
  float u1, u2, n2, s2, q, ser, m, Qu1, Qu2;   // Qu = conic u, q = u . Qu
  bool series;
};

// m of pixel p for the entry (r0, r1, r2, r3): tangent offset u, q(u), (theta/s)^2.
// (A pixel past the Gaussian's reach gets m > cutoff; the blends' cull skips most of
// them by groups of 32, so no per-pixel early exit is taken.)
// exp(-m / 2) of a reaching entry (m <= cutoff) as 2^(m * (-log2(e) / 2)) on the MUFU ex2
// unit: one multiply and one ex2. Both blends take their Gaussian factor from this one
// function, so the backward's alpha is the forward's bit for bit.
__device__ __forceinline__ float exp_neg_half(float m) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(m * -0.72134752044448170368f));
  return y;
}

// (pixel_offsets, then pixel_series or pixel_atan by P.series: the backward takes the branch
// once for both the weight and its partials)
__device__ __forceinline__ void pixel_offsets(const float3 p, const float4 r0, const float4 r1, const float4 r2,
                                              const float4 r3, Pix& P) {
  // every rounding written out (fmaf, __fmul_rn), so that all launch shapes give the same bits
  const float dx = p.x - r0.x, dy = p.y - r0.y, dz = p.z - r0.z;
  P.n2 = fmaf(dz, dz, fmaf(dy, dy, __fmul_rn(dx, dx)));
  P.u1 = fmaf(dz, r1.z, fmaf(dy, r1.y, __fmul_rn(dx, r1.x)));
  P.u2 = fmaf(dz, r2.z, fmaf(dy, r2.y, __fmul_rn(dx, r2.x)));
  P.s2 = fmaf(P.u2, P.u2, __fmul_rn(P.u1, P.u1));
  P.Qu1 = fmaf(r2.w, P.u2, __fmul_rn(r1.w, P.u1));
  P.Qu2 = fmaf(r3.w, P.u2, __fmul_rn(r2.w, P.u1));
  P.q = fmaf(P.u2, P.Qu2, __fmul_rn(P.u1, P.Qu1));
  P.series = P.n2 < kSeriesN2;
}
__device__ __forceinline__ void pixel_series(Pix& P) {
  const float s2 = P.s2;
  P.ser = fmaf(s2, fmaf(s2, fmaf(s2, fmaf(s2, 128.f / 1575.f, 4.f / 35.f), 8.f / 45.f), 1.f / 3.f), 1.f);
  P.m = __fmul_rn(P.q, P.ser);
}
__device__ __forceinline__ void pixel_atan(Pix& P) {
  const float c = fmaf(-0.5f, P.n2, 1.f);
  if (P.s2 < 1e-24f) { P.ser = 0.f; P.m = (c < 0.f) ? 3.0e38f : 0.f; return; }
  const float s = sqrtf(P.s2);
  const float ratio = atan2f(s, c) / s;
  P.ser = __fmul_rn(ratio, ratio);
  P.m = __fmul_rn(P.q, P.ser);
}
__device__ __forceinline__ void pixel_weight(const float3 p, const float4 r0, const float4 r1, const float4 r2,
                                             const float4 r3, Pix& P) {
  pixel_offsets(p, r0, r1, r2, r3, P);
  if (P.series) pixel_series(P);
  else pixel_atan(P);
}

// Cull of (entry, 32-pixel group) pairs, taken once per staged entry. A tile's
// pixels split into 16-pixel sub-tiles (the order-(k-2) pixels inside it) whose
// pixel centres lie within rho_sub of the sub-tile centre p_c. For a pixel with
// FP32 offset U that contributes (m <= cutoff), m = q(U) (theta/s)^2 with
// (theta/s)^2 >= 1 (the series is 1 + positive terms; the atan form runs at
// theta >= 0.2, where theta/s - 1 >= theta^2/6 dwarfs FP32 error), so the exact
// form satisfies q(U) <= cutoff (1 + 1e-5) + g M |U|^2, with g M |U|^2 bounding
// the FP32 rounding of q (g = 2e-6 is ~30 units of 2^-24, M = max(A, C) + |B|).
// sqrt(q) is a norm and |U - u_c| <= rho' (rho_sub plus FP32 slack of the
// directions and projections), so
//   sqrt(q(u_c)) <= sqrt(cut + 2 g M (|u_c|^2 + rho'^2)) + sqrt(lambda_max) rho'
//                <= c0 + c1 |u_c|^2   (sqrt(a^2 + x) <= a + x / (2a)).
// A sub-tile whose centre violates that bound (with q(u_c) lowered by its own
// rounding bound and the right side raised by 1e-5) holds no contributing pixel
// in this kernel's own arithmetic, so skipping it leaves every output bit-identical.
// Returns bit g set when sub-tile 2g or 2g+1 may hold a contributing pixel. The two
// sub-tiles of a group are tested side by side on the packed FP32 pipe (FFMA2 and FMUL2,
// each half rounded like the scalar operation): sub holds their centres as pairs,
// sub[3 g + {0, 1, 2}] = (x, y, z) of sub-tiles (2g, 2g + 1).
template <int NS>
__device__ __forceinline__ uint32_t live_groups(const float4 r0, const float4 r1, const float4 r2, const float4 r3,
                                               const float2* __restrict__ sub, float rho_p, float sqrt_cut) {
  const float A = r1.w, B = r2.w, C = r3.w;
  const float h = 0.5f * (A - C);
  const float lmax = (0.5f * (A + C) + sqrtf(h * h + B * B)) * (1.f + 1e-5f);
  const float gM = 2e-6f * (fmaxf(A, C) + fabsf(B));
  const float c1 = gM / sqrt_cut;
  const float c0 = sqrt_cut + c1 * rho_p * rho_p + sqrtf(lmax) * rho_p;
  // u_c = p_c . e - g . e (g . e ~ 0): three FMAs per component, within 4e-7 of (p_c - g) . e
  const float gE1 = r0.x * r1.x + r0.y * r1.y + r0.z * r1.z;
  const float gE2 = r0.x * r2.x + r0.y * r2.y + r0.z * r2.z;
  const float2 e1x = make_float2(r1.x, r1.x), e1y = make_float2(r1.y, r1.y), e1z = make_float2(r1.z, r1.z);
  const float2 e2x = make_float2(r2.x, r2.x), e2y = make_float2(r2.y, r2.y), e2z = make_float2(r2.z, r2.z);
  const float2 m1 = make_float2(-gE1, -gE1), m2 = make_float2(-gE2, -gE2);
  const float2 AA = make_float2(A, A), B2 = make_float2(2.f * B, 2.f * B), CC = make_float2(C, C);
  const float2 C0 = make_float2(c0, c0), C1 = make_float2(c1, c1), NG = make_float2(-gM, -gM);
  const float2 K = make_float2(1.f + 1e-5f, 1.f + 1e-5f);
  uint32_t live = 0;
#pragma unroll
  for (int g = 0; g < NS / 2; ++g) {
    const float2 x = sub[3 * g], y = sub[3 * g + 1], z = sub[3 * g + 2];
    const float2 u1 = __ffma2_rn(z, e1z, __ffma2_rn(y, e1y, __ffma2_rn(x, e1x, m1)));
    const float2 u2 = __ffma2_rn(z, e2z, __ffma2_rn(y, e2y, __ffma2_rn(x, e2x, m2)));
    const float2 s2 = __ffma2_rn(u2, u2, __fmul2_rn(u1, u1));
    const float2 t = __ffma2_rn(B2, u2, __fmul2_rn(AA, u1));
    const float2 q = __ffma2_rn(__fmul2_rn(CC, u2), u2, __fmul2_rn(u1, t));
    const float2 rhs = __ffma2_rn(C1, s2, C0);
    const float2 lhs = __ffma2_rn(NG, s2, q);       // q - gM |u|^2
    const float2 rr = __fmul2_rn(__fmul2_rn(rhs, rhs), K);
    const bool cull = lhs.x > rr.x && lhs.y > rr.y; // false for NaN: kept
    live |= (cull ? 0u : 1u) << g;
  }
  return live;
}

// Resident blocks per SM the blend kernels ask of the register allocator: the
// group guards of the cull would otherwise grow the one- and four-pixel shapes
// and cost them resident warps (forward 48 registers, 5 blocks of 256 threads, measured
// faster than 40 with its spills; backward 96, 10 blocks of 64 threads).
#ifndef HPXGS_FWD_REGS
#define HPXGS_FWD_REGS 48
#endif
constexpr int fwd_min_blocks(int nt, int ppt, bool depth) { return (ppt == 1 && nt >= 128 && !depth) ? 65536 / (nt * HPXGS_FWD_REGS) : 1; }
#ifndef HPXGS_BWD_REGS
#define HPXGS_BWD_REGS 96
#endif
constexpr int bwd_min_blocks(int nt, int ppt, bool depth) { return (ppt <= 4 && !depth) ? 65536 / (nt * HPXGS_BWD_REGS) : 1; }

// Sub-tile centres of a tile (order k - 2 pixels) and the cull's per-view constants.
template <int NS>
__device__ __forceinline__ void sub_centres(const ViewParams& vp, uint32_t lt, int b, float2* sub, int tid, int nt) {
  // pairs of sub-tiles (2g, 2g + 1) as sub[3 g + {0, 1, 2}] = their x, y, z
  for (int t = tid; t < NS; t += nt) {
    const float3 c = pix2vec_f32(vp.k - 2, (lt << (2 * (b - 2))) + (uint32_t)t);
    float* f = reinterpret_cast<float*>(sub + 3 * (t >> 1)) + (t & 1);
    f[0] = c.x; f[2] = c.y; f[4] = c.z;
  }
}
__device__ __forceinline__ float cull_rho(const ViewParams& vp) { return vp.rho_sub32 * (1.f + 1e-5f) + 4e-6f; }
__device__ __forceinline__ float cull_sqrt_cut(float cutoff) { return sqrtf(cutoff * (1.f + 1e-5f)) * (1.f + 1e-6f); }

// ----------------------------------------------------------------------------
// Longest-first order of the persistent blends' units. A blend block takes its next
// unit from a counter; taken in index order, units with long lists that come late
// keep a few blocks busy after the others have run out of work. Each unit gets an
// estimate w of its work (MODE 0, the forward: its tile's list length, 0 for a tile
// without an in-mask pixel; MODE 1, the backward: the time the forward blend spent on
// the unit, in units of 256 SM clocks, which follows the pairs, cull and termination
// that the backward's work follows too), a class by w (four per
// octave, the largest first, w = 0 last), and the blend takes units class by class.
// Inside a class the order is that of the atomics: the blends' outputs do not depend
// on which block takes which unit.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int unit_class(uint32_t w) {
  if (w == 0) return kUnitClasses - 1;
  const int lg = 31 - __clz(w);
  const uint32_t sub = lg >= 2 ? (w >> (lg - 2)) & 3u : (w << (2 - lg)) & 3u;
  return 127 - (4 * lg + (int)sub);
}

template <int MODE>
__device__ __forceinline__ uint32_t unit_estimate(int u, int shift, const uint2* __restrict__ ranges,
                                                  const uint32_t* __restrict__ flags, const uint32_t* __restrict__ work) {
  if (MODE == 1) return work[u];
  const int tile = u >> shift;
  if (!(flags[tile] & 1u)) return 0u;
  const uint2 r = ranges[tile];
  return r.y > r.x ? r.y - r.x : 0u;
}

// cls[0 .. kUnitClasses): units per class (zero before the launch).
template <int MODE>
__global__ void __launch_bounds__(256) k_unit_count(int nunits, int shift, const uint2* __restrict__ ranges,
                                                    const uint32_t* __restrict__ flags,
                                                    const uint32_t* __restrict__ work, uint32_t* cls) {
  __shared__ uint32_t h[kUnitClasses];
  for (int i = threadIdx.x; i < kUnitClasses; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < nunits) atomicAdd(&h[unit_class(unit_estimate<MODE>(u, shift, ranges, flags, work))], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kUnitClasses; i += blockDim.x)
    if (h[i]) atomicAdd(&cls[i], h[i]);
}

// order[base(c) + k] = the k-th unit placed in class c; cls[kUnitClasses + c] is class c's
// cursor (zero before the launch), base(c) the units of the classes before c.
template <int MODE>
__global__ void __launch_bounds__(256) k_unit_place(int nunits, int shift, const uint2* __restrict__ ranges,
                                                    const uint32_t* __restrict__ flags,
                                                    const uint32_t* __restrict__ work, uint32_t* cls,
                                                    uint32_t* __restrict__ order) {
  __shared__ uint32_t base[kUnitClasses];
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {                          // exclusive scan of the class counts, 5 per lane
    constexpr int PER = (kUnitClasses + 31) / 32;
    uint32_t v[PER], t = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) { const int c = PER * lane + q; v[q] = c < kUnitClasses ? cls[c] : 0u; t += v[q]; }
    uint32_t inc = t;
    for (int o = 1; o < 32; o <<= 1) { const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o); if (lane >= o) inc += y; }
    uint32_t run = inc - t;
#pragma unroll
    for (int q = 0; q < PER; ++q) { const int c = PER * lane + q; if (c < kUnitClasses) base[c] = run; run += v[q]; }
  }
  __syncthreads();
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = u < nunits;
  const int c = ok ? unit_class(unit_estimate<MODE>(u, shift, ranges, flags, work)) : -1;
  const uint32_t peers = __match_any_sync(0xffffffffu, c);
  const int leader = __ffs(peers) - 1;
  uint32_t first = 0;
  if (ok && lane == leader) first = atomicAdd(&cls[kUnitClasses + c], (uint32_t)__popc(peers));
  first = __shfl_sync(0xffffffffu, first, leader);
  if (ok) order[base[c] + first + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)u;
}

static int launch_unit_order(int mode, int nunits, int shift, const uint2* ranges, const uint32_t* flags,
                             const uint32_t* work, uint32_t* cls, uint32_t* order, cudaStream_t s) {
  if (nunits <= 0) return HPXGS_OK;
  const unsigned nb = (unsigned)((nunits + 255) / 256);
  if (mode == 0) {
    k_unit_count<0><<<nb, 256, 0, s>>>(nunits, shift, ranges, flags, work, cls);
    k_unit_place<0><<<nb, 256, 0, s>>>(nunits, shift, ranges, flags, work, cls, order);
  } else {
    k_unit_count<1><<<nb, 256, 0, s>>>(nunits, shift, ranges, flags, work, cls);
    k_unit_place<1><<<nb, 256, 0, s>>>(nunits, shift, ranges, flags, work, cls, order);
  }
  note_launches(2);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

// ----------------------------------------------------------------------------
// Forward compositing: persistent blocks take tiles from a counter; one thread
// per pixel (PPT pixels per thread for 1024-pixel tiles); Gaussian records of the
// tile's list are staged through shared memory in batches of BATCH.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int view_of_tile(const ViewTable& vt, int tile) {
  int v = 0;
  while (v + 1 < vt.nviews && tile >= vt.v[v + 1].tile_base) ++v;
  return v;
}

// DEPTH adds the inverse-depth channel D = sum_i T_i alpha_i / r_i (Sec. 3.2, depth
// supervision by 1/r): rdepth holds r per (view, Gaussian), dmap receives D per pixel.
template <int NT, int PPT, int BATCH, bool DEPTH = false, bool SPLIT = false>
__global__ void __launch_bounds__(NT, fwd_min_blocks(NT, PPT, DEPTH)) k_blend_fwd(const __grid_constant__ ViewTable vt, const float4* __restrict__ rec,
                                                  const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids,
                                                  const uint32_t* __restrict__ flags, const uint32_t* __restrict__ mask,
                                                  float* __restrict__ maps, float* __restrict__ Tout,
                                                  uint32_t* __restrict__ lastout, uint32_t* work,
                                                  unsigned long long* __restrict__ evals, uint32_t* __restrict__ gmask,
                                                  const uint32_t* __restrict__ order, uint32_t* __restrict__ unit_work,
                                                  const float* __restrict__ rdepth = nullptr,
                                                  float* __restrict__ dmap = nullptr) {
  constexpr int NW = NT / 32;
  constexpr int NS = NT * PPT / 16;                 // 16-pixel sub-tiles per tile
  __shared__ float4 s_rec[BATCH][4];
  __shared__ float s_invr[DEPTH ? BATCH : 1];
  constexpr int NG = NS / 2;                        // 32-pixel groups per tile
  constexpr int BW = BATCH / 32;                    // bitmap words per batch
  __shared__ uint32_t s_live[NG][BW];               // per group: the staged entries it may take
  __shared__ float2 s_sub[3 * (NS / 2)];
  __shared__ int s_tile;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int b = SPLIT ? vt.b - 1 : vt.b;            // order of a blend unit below k
  const int nunits = SPLIT ? 4 * vt.total_tiles : vt.total_tiles;
  const float sqrt_cut = cull_sqrt_cut(vt.cutoff);
  int prev = -1;
  long long t_unit = 0;                             // thread 0: SM clock when the current unit was taken
  for (;;) {
    if (tid == 0) {                                  // the next unit, longest-first when an order is given
      const uint32_t t = atomicAdd(work, 1u);
      s_tile = (order && t < (uint32_t)nunits) ? (int)order[t] : (int)t;
    }
    __syncthreads();
    const int unit = s_tile;
    if (tid == 0 && unit_work) {                     // the previous unit's time, for the backward's order
      const long long tn = clock64();
      if (prev >= 0) unit_work[prev] = (uint32_t)max(1ll, (tn - t_unit) >> 8);
      t_unit = tn;
    }
    prev = unit;
    __syncthreads();
    if (unit >= nunits) break;
    const int tile = SPLIT ? unit >> 2 : unit;       // SPLIT: unit = one quarter of a listed tile
    const int v = view_of_tile(vt, tile);
    const ViewParams& vp = vt.v[v];
    const uint32_t lt = SPLIT ? (((uint32_t)(tile - vp.tile_base) << 2) | (uint32_t)(unit & 3))
                              : (uint32_t)(tile - vp.tile_base);
    const bool active = flags[tile] & 1u;
    if (!active && !vt.write_outside) continue;
    const uint32_t* vmask = mask + (vp.pix_base >> 5);
    const float rho_p = cull_rho(vp);
    sub_centres<NS>(vp, lt, b, s_sub, tid, NT);
    float3 pv[PPT];
    float C[PPT][3], T[PPT];
    float D[DEPTH ? PPT : 1];
    uint32_t last[PPT];
    bool done[PPT], inm[PPT];
    uint32_t lp[PPT];
    uint32_t ncontrib = 0, neval = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      lp[q] = (lt << (2 * b)) + q * NT + tid;
      inm[q] = active && ((vmask[lp[q] >> 5] >> (lp[q] & 31)) & 1u);
      done[q] = !inm[q];
      pv[q] = inm[q] ? pix2vec_f32(vp.k, lp[q]) : make_float3(0.f, 0.f, 1.f);
      C[q][0] = C[q][1] = C[q][2] = 0.f;
      if (DEPTH) D[DEPTH ? q : 0] = 0.f;
      T[q] = 1.f;
      last[q] = 0;
    }
    bool unit_active = active;
    if (SPLIT) {                                     // a quarter with no in-mask pixel stages nothing
      int any = 0;
#pragma unroll
      for (int q = 0; q < PPT; ++q) any |= inm[q];
      unit_active = __syncthreads_or(any) != 0;
    }
    const uint2 rg = unit_active ? ranges[tile] : make_uint2(0, 0);
    for (uint32_t bs = rg.x; bs < rg.y; bs += BATCH) {
      const int n = (int)min((uint32_t)BATCH, rg.y - bs);
      // the staging below reuses the batch buffers and reads the sub-tile centres: after the first
      // batch the previous batch's closing count barrier orders it, and with SPLIT the unit's
      // __syncthreads_or does for the first
      if (!SPLIT && bs == rg.x) __syncthreads();
      for (int e0 = 0; e0 < n; e0 += NT) {
        const int e = e0 + tid;
        uint32_t gm = 0;
        if (e < n) {
          const uint32_t id = ids[bs + e];
          const float4* src = rec + 4 * (int64_t)id;
          const float4 a0 = src[0], a1 = src[1], a2 = src[2], a3 = src[3];
          s_rec[e][0] = a0; s_rec[e][1] = a1; s_rec[e][2] = a2; s_rec[e][3] = a3;
          if (DEPTH) s_invr[e] = 1.f / rdepth[id];
          gm = vt.cull ? live_groups<NS>(a0, a1, a2, a3, s_sub, rho_p, sqrt_cut) : (NG == 32 ? ~0u : (1u << NG) - 1u);
          // for the backward pass over the same entries (SPLIT: one byte of the entry's word per quarter)
          if (SPLIT) reinterpret_cast<uint8_t*>(gmask)[4 * (size_t)(bs + e) + (unit & 3)] = (uint8_t)gm;
          else gmask[bs + e] = gm;
        }
        if (e0 + (warp << 5) < n) {                  // this warp staged entries: one bitmap word per group
#pragma unroll
          for (int g = 0; g < NG; ++g) {
            const uint32_t bl = __ballot_sync(0xffffffffu, (gm >> g) & 1u);
            if ((tid & 31) == 0) s_live[g][(e0 >> 5) + warp] = bl;
          }
        }
      }
      __syncthreads();
      const int nwords = (n + 31) >> 5;
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int gq = q * NW + warp;
        // only the entries that may reach a pixel of this warp's group, in list order
        for (int wj = 0; wj < nwords && !done[q]; ++wj) {
          uint32_t bits = s_live[gq][wj];
          while (bits) {
            const int e = (wj << 5) + __ffs(bits) - 1;
            bits &= bits - 1u;
            const float4 r0 = s_rec[e][0], r1 = s_rec[e][1], r2 = s_rec[e][2], r3 = s_rec[e][3];
            Pix P;
            pixel_offsets(pv[q], r0, r1, r2, r3, P);
            // compositing of a reaching entry; true when the pixel terminates
            auto composite = [&]() -> bool {
              if (!(P.m <= vt.cutoff)) return false;
              ++ncontrib;
              const float a = fminf(vt.alpha_max, __fmul_rn(r0.w, exp_neg_half(P.m)));
              const float w = __fmul_rn(a, T[q]);
              C[q][0] = fmaf(w, r3.x, C[q][0]); C[q][1] = fmaf(w, r3.y, C[q][1]); C[q][2] = fmaf(w, r3.z, C[q][2]);
              if (DEPTH) D[DEPTH ? q : 0] = fmaf(w, s_invr[e], D[DEPTH ? q : 0]);
              T[q] = __fmul_rn(T[q], 1.f - a);
              if (T[q] < vt.eps_T) { done[q] = true; last[q] = bs + e + 1 - rg.x; return true; }
              return false;
            };
            // one branch on the arc-length form, taken for the weight and the compositing together
            bool term;
            if (P.series) { pixel_series(P); term = composite(); }
            else { pixel_atan(P); term = composite(); }
            if (term) break;
          }
        }
      }
      int alive = 0;
#pragma unroll
      for (int q = 0; q < PPT; ++q) alive |= !done[q];
      if (__syncthreads_count(alive) == 0) break;
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int64_t pg = vp.pix_base + lp[q];
      if (inm[q]) {
        if (T[q] >= vt.eps_T) last[q] = rg.y - rg.x;     // ran through the whole list
        neval += last[q];
        maps[3 * pg + 0] = fmaf(T[q], vt.bg[0], C[q][0]);
        maps[3 * pg + 1] = fmaf(T[q], vt.bg[1], C[q][1]);
        maps[3 * pg + 2] = fmaf(T[q], vt.bg[2], C[q][2]);
        Tout[pg] = T[q];
        lastout[pg] = last[q];
        if (DEPTH) dmap[pg] = D[DEPTH ? q : 0];
      } else if (vt.write_outside) {
        maps[3 * pg + 0] = vt.bg[0]; maps[3 * pg + 1] = vt.bg[1]; maps[3 * pg + 2] = vt.bg[2];
        Tout[pg] = 1.f;
        lastout[pg] = 0;
        if (DEPTH) dmap[pg] = 0.f;
      }
    }
    // per-warp totals of evaluated and contributing (pixel, entry) pairs
    unsigned long long e64 = neval, c64 = ncontrib;
    for (int o = 16; o > 0; o >>= 1) {
      e64 += __shfl_xor_sync(0xffffffffu, e64, o);
      c64 += __shfl_xor_sync(0xffffffffu, c64, o);
    }
    if ((tid & 31) == 0 && e64) { atomicAdd(&evals[0], e64); atomicAdd(&evals[1], c64); }
  }
}

// Backward of one (pixel, entry) on the scalar path. From m (P) and the pixel's running
// transmittance T behind the entry: alpha, T in front of it (T_j = T / (1 - a)), the
// entry's partials added to acc, and the pixel's running T and B moved in front of the
// entry. acc[4 .. 8] hold their partials times -2 / dL/dm's -1/2 left out, and acc[5],
// acc[7], acc[8] at half weight on top: kPartScale applies both once per entry after the
// reduction. dD and invr: the depth channel's dL/dD and 1/r (DEPTH only).
// Returns false when the entry does not reach the pixel (m > cutoff).
// Per-entry factor of each backward partial (see bwd_pixel): 1 for the colour, opacity
// and depth partials, -1/2 for acc[4], acc[6], and -1 (-1/2 times 2) for acc[5], acc[7], acc[8].
__host__ __device__ constexpr float kPartScale(int c) {
  return (c == 4 || c == 6) ? -0.5f : ((c == 5 || c == 7 || c == 8) ? -1.f : 1.f);
}

template <bool DEPTH, int NA, bool SERIES>
__device__ __forceinline__ bool bwd_pixel(const ViewTable& vt, const Pix& P, float4 r0, float4 r1, float4 r2,
                                          float4 r3, const float* dI, float dD, float invr, float& T, float& B,
                                          float* acc) {
  if (!(P.m <= vt.cutoff)) return false;
  const float G = exp_neg_half(P.m);
  const float og = r0.w * G;
  const float a = fminf(vt.alpha_max, og);
  float inv1ma;                                     // 1 / (1 - a) on the MUFU reciprocal
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv1ma) : "f"(1.f - a));
  const float Tj = T * inv1ma;
  const float wj = Tj * a;
  // A = dL/dI . colour (+ dL/dD / r); dL/da = T_j A - B / (1 - a); then B takes this entry
  float A = dI[0] * r3.x + dI[1] * r3.y + dI[2] * r3.z;
#pragma unroll
  for (int c = 0; c < 3; ++c) acc[c] += wj * dI[c];
  if (DEPTH) {
    acc[NA - 1] += wj * dD;
    A += dD * invr;
  }
  const float dLda = Tj * A - B * inv1ma;
  B += wj * A;
  T = Tj;
  if (og >= vt.alpha_max) return true;          // clamped: no gradient to o, m
  acc[3] += dLda * G;
  // dL/dm = -Lm / 2 with Lm = dLda o G (the -1/2 goes with kPartScale); m = q(u) ser, ser = (theta/s)^2
  const float Lm = dLda * og;
  const float u1 = P.u1, u2 = P.u2;
  const float Ws = Lm * P.ser;
  const float t1 = Ws * u1;
  acc[4] += t1 * u1;
  acc[5] += t1 * u2;
  acc[6] += Ws * u2 * u2;
  const float Qu1 = P.Qu1, Qu2 = P.Qu2;
  const float c = 1.f - 0.5f * P.n2;
  // dm/du_j / 2 = ser Qu_j + q (d ser / d u_j) / 2 = ser Qu_j + K u_j (K per branch below);
  // dm/dc / 2 = Lc per unit Lm (atan form only)
  // moving g by a tangent step delta: du_i = -c delta_i, dc = u . delta
  if constexpr (SERIES) {
    const float s2 = P.s2;
    const float dser = 1.f / 3.f + s2 * (16.f / 45.f + s2 * (12.f / 35.f + s2 * (512.f / 1575.f)));
    const float K = Lm * P.q * dser;
    const float h1 = Ws * Qu1 + K * u1, h2 = Ws * Qu2 + K * u2;
    acc[7] += -c * h1;
    acc[8] += -c * h2;
  } else {
    const float s = sqrtf(P.s2);
    const float ratio = sqrtf(P.ser);
    const float th = ratio * s;
    const float kf = (c * s - th) / (P.s2 * s);     // d(theta/s)/du_j = kf u_j
    const float K = Lm * P.q * ratio * kf;
    const float Lc = -Lm * P.q * ratio;              // d(theta/s)/dc = -1/s^2... times s: -1
    const float h1 = Ws * Qu1 + K * u1, h2 = Ws * Qu2 + K * u2;
    acc[7] += -c * h1 + Lc * u1;
    acc[8] += -c * h2 + Lc * u2;
  }
  return true;
}

// ----------------------------------------------------------------------------
// Backward compositing: reverse walk of each pixel's processed prefix.
// Per (pixel, entry): T_j = T_{j+1} / (1 - a); dL/dc = T_j a dI;
// dL/da = dI . (T_j c - S / (1 - a)), S = colour behind entry j incl. background;
// then through a = o exp(-m/2) and m = q(u) (theta/s)^2 to the conic and to a
// tangent displacement of the centre g (parallel-transported frame).
// Accumulators per (view, Gaussian): [dcol(3), dopacity, dconic_a, dconic_b (unique
// off-diagonal), dconic_c, d_east, d_north].
// ----------------------------------------------------------------------------
// DEPTH adds the inverse-depth channel: ddepth is dL/dD per pixel, and the tenth
// partial dL/d(1/r) per (view, Gaussian) goes to accum_d.
// LOSS takes dL/dI of each pixel from the L1 + HSSIM gradient of its view
// (hssim_pixel_grad over the view's window table and the HSSIM forward's
// coefficients) instead of a dL/dI map: the HSSIM backward runs in this prologue.
template <int NT, int PPT, int BATCH, bool DEPTH = false, bool SPLIT = false, bool LOSS = false>
__global__ void __launch_bounds__(NT, bwd_min_blocks(NT, PPT, DEPTH)) k_blend_bwd(const __grid_constant__ ViewTable vt, const float4* __restrict__ rec,
                                                  const uint2* __restrict__ ranges, const uint32_t* __restrict__ ids,
                                                  const uint32_t* __restrict__ flags, const uint32_t* __restrict__ mask,
                                                  const float* __restrict__ dmaps, const float* __restrict__ Tin,
                                                  const uint32_t* __restrict__ lastin, float* __restrict__ accum,
                                                  uint32_t* work, const uint32_t* __restrict__ gmask,
                                                  const uint32_t* __restrict__ order,
                                                  const float* __restrict__ rdepth,
                                                  const float* __restrict__ ddepth,
                                                  float* __restrict__ accum_d,
                                                  const __grid_constant__ std::conditional_t<LOSS, LossViews, NoLossViews> lv) {
  constexpr int NW = NT / 32;
  constexpr int NA = HPXGS_NACC + (DEPTH ? 1 : 0);
  __shared__ float4 s_rec[BATCH][4];
  __shared__ float s_invr[DEPTH ? BATCH : 1];
  __shared__ uint32_t s_id[BATCH];
  constexpr int RL = HPXGS_BWD_RED_LANES;            // lanes summed by shuffles; RL-lane partials go to shared memory
  constexpr int NR = 32 / RL;
  __shared__ float s_part[BATCH][NW][NR][NA];
  constexpr int BW = (BATCH + 31) / 32;             // bitmap words per batch
  __shared__ uint32_t s_gm[BATCH];                  // live 32-pixel groups per staged entry
  __shared__ uint32_t s_wlive[NW][BW];              // per warp: staged entries live in one of its groups
  __shared__ int s_tile;
  __shared__ uint32_t s_maxlast;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = SPLIT ? vt.b - 1 : vt.b;            // order of a blend unit below k
  const int nunits = SPLIT ? 4 * vt.total_tiles : vt.total_tiles;
  for (;;) {
    if (tid == 0) {                                  // the next unit, longest-first when an order is given
      const uint32_t t = atomicAdd(work, 1u);
      s_tile = (order && t < (uint32_t)nunits) ? (int)order[t] : (int)t;
      s_maxlast = 0;
    }
    __syncthreads();
    const int unit = s_tile;
    if (unit >= nunits) break;
    const int tile = SPLIT ? unit >> 2 : unit;       // SPLIT: unit = one quarter of a listed tile
    const bool active = flags[tile] & 1u;
    if (!active) { __syncthreads(); continue; }
    const int v = view_of_tile(vt, tile);
    const ViewParams& vp = vt.v[v];
    const uint32_t lt = SPLIT ? (((uint32_t)(tile - vp.tile_base) << 2) | (uint32_t)(unit & 3))
                              : (uint32_t)(tile - vp.tile_base);
    const uint2 rg = ranges[tile];
    const uint32_t* vmask = mask + (vp.pix_base >> 5);
    float3 pv[PPT];
    // B = dL/dI . (colour behind the entry, background included) (+ dL/dD x depth behind it), the
    // only form in which the colour behind enters dL/dalpha, kept as one scalar per pixel
    float dI[PPT][3], B[PPT], T[PPT];
    float dDp[DEPTH ? PPT : 1];                         // dL/dD
    uint32_t lastp[PPT];
    uint32_t mylast = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const uint32_t lp = (lt << (2 * b)) + q * NT + tid;
      const bool inm = (vmask[lp >> 5] >> (lp & 31)) & 1u;
      const int64_t pg = vp.pix_base + lp;
      lastp[q] = inm ? lastin[pg] : 0u;
      T[q] = inm ? Tin[pg] : 1.f;
      pv[q] = inm ? pix2vec_f32(vp.k, lp) : make_float3(0.f, 0.f, 1.f);
      if constexpr (LOSS) {
        if (inm) {
          const LossView& lw = lv.v[v];
          const float scale = (lw.dloss ? *lw.dloss : 1.f) / (3.f * *lw.nm);
          hssim_pixel_grad(lp, lw.npix, lw.I, lw.G, lw.idx, lw.e, lw.coef, scale, lv.lambda, dI[q]);
        } else {
          dI[q][0] = 0.f; dI[q][1] = 0.f; dI[q][2] = 0.f;
        }
      } else {
        for (int c = 0; c < 3; ++c) dI[q][c] = inm ? dmaps[3 * pg + c] : 0.f;
      }
      B[q] = T[q] * (dI[q][0] * vt.bg[0] + dI[q][1] * vt.bg[1] + dI[q][2] * vt.bg[2]);
      if (DEPTH) dDp[DEPTH ? q : 0] = inm ? ddepth[pg] : 0.f;
      mylast = max(mylast, lastp[q]);
    }
    if (mylast) atomicMax(&s_maxlast, mylast);
    __syncthreads();
    const uint32_t hi = rg.x + s_maxlast;
    for (uint32_t be = hi; be > rg.x;) {
      const uint32_t bs = (be - rg.x > (uint32_t)BATCH) ? be - BATCH : rg.x;
      const int n = (int)(be - bs);
      __syncthreads();
      for (int e0 = 0; e0 < n; e0 += NT) {
        const int e = e0 + tid;
        uint32_t gmv = 0;
        if (e < n) {
          const uint32_t id = ids[bs + e];
          s_id[e] = id;
          const float4* src = rec + 4 * (int64_t)id;
          s_rec[e][0] = src[0]; s_rec[e][1] = src[1]; s_rec[e][2] = src[2]; s_rec[e][3] = src[3];
          if (DEPTH) s_invr[e] = 1.f / rdepth[id];
          gmv = SPLIT ? (uint32_t)reinterpret_cast<const uint8_t*>(gmask)[4 * (size_t)(bs + e) + (unit & 3)]
                      : gmask[bs + e];             // the forward's cull of this entry
          s_gm[e] = gmv;
        }
        if (e0 + (warp << 5) < n) {                // this warp staged entries: one bitmap word per warp
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            uint32_t wg = 0;
#pragma unroll
            for (int q = 0; q < PPT; ++q) wg |= 1u << (q * NW + w);
            const uint32_t bl = __ballot_sync(0xffffffffu, (gmv & wg) != 0u);
            if (lane == 0) s_wlive[w][(e0 >> 5) + warp] = bl;
          }
        }
      }
      __syncthreads();
      // only the entries live in one of this warp's groups, in reverse list order (warp-uniform)
      for (int wj = (n - 1) >> 5; wj >= 0; --wj) {
        for (uint32_t bits = s_wlive[warp][wj]; bits;) {
          const int i = 31 - __clz(bits);
          bits ^= 1u << i;
          const int e = (wj << 5) + i;
          const uint32_t gm = s_gm[e];
          const uint32_t j = bs + e - rg.x;          // position in the tile list
          float acc[NA];
#pragma unroll
          for (int c = 0; c < NA; ++c) acc[c] = 0.f;
          bool any = false;
          const float4 r0 = s_rec[e][0], r1 = s_rec[e][1], r2 = s_rec[e][2], r3 = s_rec[e][3];
#pragma unroll
          for (int q = 0; q < PPT; ++q) {
            if (j >= lastp[q] || !((gm >> (q * NW + warp)) & 1u)) continue;
            Pix P;
            pixel_offsets(pv[q], r0, r1, r2, r3, P);
            const float dDq = DEPTH ? dDp[DEPTH ? q : 0] : 0.f, invr = DEPTH ? s_invr[e] : 0.f;
            bool hit;
            if (P.series) {
              pixel_series(P);
              hit = bwd_pixel<DEPTH, NA, true>(vt, P, r0, r1, r2, r3, dI[q], dDq, invr, T[q], B[q], acc);
            } else {
              pixel_atan(P);
              hit = bwd_pixel<DEPTH, NA, false>(vt, P, r0, r1, r2, r3, dI[q], dDq, invr, T[q], B[q], acc);
            }
            if (hit) any = true;
          }
          // reduction of the 9 partials over groups of RL lanes, then one shared-memory
          // slot per group (the block-level pass below adds the slots)
          const unsigned ball = __ballot_sync(0xffffffffu, any);
          if (ball) {                                 // pairs of partials added on FADD2
#pragma unroll
            for (int c = 0; c + 1 < NA; c += 2) {
              float2 x = make_float2(acc[c], acc[c + 1]);
#pragma unroll
              for (int o = RL / 2; o > 0; o >>= 1) {
                const float2 y = make_float2(__shfl_xor_sync(0xffffffffu, x.x, o), __shfl_xor_sync(0xffffffffu, x.y, o));
                x = __fadd2_rn(x, y);
              }
              acc[c] = x.x;
              acc[c + 1] = x.y;
            }
            if (NA & 1) {
              float x = acc[NA - 1];
#pragma unroll
              for (int o = RL / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
              acc[NA - 1] = x;
            }
          }
          if ((lane & (RL - 1)) == 0) {
#pragma unroll
            for (int c = 0; c < NA; ++c) s_part[e][warp][lane / RL][c] = ball ? kPartScale(c) * acc[c] : 0.f;
          }
        }
      }
      __syncthreads();
      for (int t = tid; t < n * NA; t += NT) {
        const int e = t / NA, c = t - e * NA;
        const uint32_t gm = s_gm[e];
        float sum = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          uint32_t wg = 0;
#pragma unroll
          for (int q = 0; q < PPT; ++q) wg |= 1u << (q * NW + w);
          if (gm & wg) {                            // warps with no live group wrote no partials
#pragma unroll
            for (int r = 0; r < NR; ++r) sum += s_part[e][w][r][c];
          }
        }
        if (sum == 0.f) continue;
        if (!DEPTH || c < HPXGS_NACC) atomicAdd(&accum[(int64_t)s_id[e] * HPXGS_NACC + c], sum);
        else atomicAdd(&accum_d[s_id[e]], sum);
      }
      be = bs;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// Preprocess backward: one thread per Gaussian, summing over views.
// conic -> Sigma_arc: G_S = -Q G_Q Q; Sigma_arc = U U^T + blur I with rows
// u_i = M^T a_i, a_i = W^T e_i / r (S_phi J W); the frame (e_i, g) is moved by
// parallel transport under a change of t (the loss is invariant under a rotation
// of the tangent frame, so this gives the exact derivative):
//   d(e_i / r) = -(g (e_i . dt) + e_i (g . dt)) / r^2,  dg = (I - g g^T) dt / r.
// ----------------------------------------------------------------------------
// DEG is the SH degree as a compile-time constant. A block's SH rows are staged
// through shared memory (coalesced in and out; rows padded to 3K + 1 floats so that
// the per-thread rows fall in distinct banks), and the per-Gaussian SH gradient
// accumulates there over the views.
constexpr int kPreBwdThreads = 64;
#ifndef HPXGS_PREBWD_MINB
#define HPXGS_PREBWD_MINB 8
#endif
template <int DEG>
__global__ void __launch_bounds__(kPreBwdThreads, HPXGS_PREBWD_MINB) k_preprocess_bwd(const __grid_constant__ ViewTable vt, hpxgs_gaussians gs,
                                                        const float* __restrict__ radii, const float* __restrict__ accum,
                                                        float* __restrict__ dmeans, float* __restrict__ dscales,
                                                        float* __restrict__ drot, float* __restrict__ dopac,
                                                        float* __restrict__ dsh,
                                                        const float* __restrict__ accum_d) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int RW = 3 * K + 1;                       // padded row
  __shared__ float s_sh[kPreBwdThreads * RW];
  __shared__ float s_dsh[kPreBwdThreads * RW];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * kPreBwdThreads;
  const int nrow = min(kPreBwdThreads, vt.P - i0);
  const int i = i0 + tid;
  const bool own = i < vt.P;
  // this thread's parameters and its first view's radius and partials, issued before the
  // block's SH rows so that their latencies overlap
  float mu[3] = {0.f, 0.f, 0.f}, scl[3] = {1.f, 1.f, 1.f}, rq[4] = {1.f, 0.f, 0.f, 0.f};
  float rad = 0.f, A[HPXGS_NACC];
  for (int c = 0; c < HPXGS_NACC; ++c) A[c] = 0.f;
  if (own) {
    for (int c = 0; c < 3; ++c) { mu[c] = gs.means[3 * (int64_t)i + c]; scl[c] = gs.scales[3 * (int64_t)i + c]; }
    for (int c = 0; c < 4; ++c) rq[c] = gs.rotations[4 * (int64_t)i + c];
    rad = radii[i];
    for (int c = 0; c < HPXGS_NACC; ++c) A[c] = accum[(int64_t)i * HPXGS_NACC + c];
  }
  for (int t = tid; t < nrow * 3 * K; t += kPreBwdThreads) {
    const int r = t / (3 * K), c = t - r * (3 * K);
    s_sh[r * RW + c] = gs.sh[(int64_t)i0 * 3 * K + t];
    s_dsh[r * RW + c] = 0.f;
  }
  __syncthreads();
  if (own) {
  float dmu[3] = {0.f, 0.f, 0.f}, ds[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f}, dop = 0.f;
  const float* sh = s_sh + tid * RW;
  float* dshl = s_dsh + tid * RW;
  for (int v = 0; v < vt.nviews; ++v) {
    const int64_t gid = (int64_t)v * vt.P + i;
    if (v > 0) {                                   // the view's radius and partials together
      rad = radii[gid];
      for (int c = 0; c < HPXGS_NACC; ++c) A[c] = accum[gid * HPXGS_NACC + c];
    }
    if (!(rad > 0.f)) continue;
    const ViewParams& vp = vt.v[v];
    Geo G;
    geo_compute<false>(vp, vt.near_plane, mu, scl, rq, G);     // valid: the forward listed it (rad > 0)
    if (!G.valid) continue;
    // colour -> SH and the viewing direction
    float dx = mu[0] - vp.cam[0], dy = mu[1] - vp.cam[1], dz = mu[2] - vp.cam[2];
    const float dist = sqrtf(dx * dx + dy * dy + dz * dz), idist = 1.f / dist;
    dx *= idist; dy *= idist; dz *= idist;
    float Y[K];
    sh_basis(DEG, dx, dy, dz, Y, nullptr);
    float Lcr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float raw = 0.5f;
#pragma unroll
      for (int kk = 0; kk < K; ++kk) raw += sh[3 * kk + c] * Y[kk];
      Lcr[c] = raw > 0.f ? A[c] : 0.f;
    }
    // dL/dsh_kc = Y_k Lcr_c; the direction gets sum_k w_k grad Y_k with w_k = sum_c Lcr_c sh_kc
    // (Y_k is replaced by w_k in place)
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
      float w = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) { dshl[3 * kk + c] += Y[kk] * Lcr[c]; w += Lcr[c] * sh[3 * kk + c]; }
      Y[kk] = w;
    }
    const float3 Ld = sh_grad_dot(DEG, dx, dy, dz, Y);
    const float pd = Ld.x * dx + Ld.y * dy + Ld.z * dz;
    dmu[0] += (Ld.x - dx * pd) * idist;
    dmu[1] += (Ld.y - dy * pd) * idist;
    dmu[2] += (Ld.z - dz * pd) * idist;
    dop += A[3];
    // conic -> Sigma_arc
    const float GQa = A[4], GQb = 0.5f * A[5], GQc = A[6];
    // T1 = Q GQ
    const float t00 = G.qa * GQa + G.qb * GQb, t01 = G.qa * GQb + G.qb * GQc;
    const float t10 = G.qb * GQa + G.qc * GQb, t11 = G.qb * GQb + G.qc * GQc;
    const float GS00 = -(t00 * G.qa + t01 * G.qb);
    const float GS01 = -(t00 * G.qb + t01 * G.qc);
    const float GS11 = -(t10 * G.qb + t11 * G.qc);
    // Sigma = U U^T: G_u1 = 2 (GS00 u1 + GS01 u2), G_u2 = 2 (GS01 u1 + GS11 u2)
    float Gu1[3], Gu2[3];
    for (int kk = 0; kk < 3; ++kk) {
      Gu1[kk] = 2.f * (GS00 * G.u1[kk] + GS01 * G.u2[kk]);
      Gu2[kk] = 2.f * (GS01 * G.u1[kk] + GS11 * G.u2[kk]);
    }
    // u_i[k] = s_k sum_j R[j][k] a_i[j]:  G_a_i[j] = sum_k R[j][k] s_k G_u_i[k];
    // G_R[j][k] = s_k (a1[j] Gu1[k] + a2[j] Gu2[k]);  G_s[k] = sum_j R[j][k] (a1[j] Gu1[k] + a2[j] Gu2[k])
    float Ga1[3], Ga2[3], GR[9];
    for (int jj = 0; jj < 3; ++jj) {
      Ga1[jj] = 0.f; Ga2[jj] = 0.f;
      for (int kk = 0; kk < 3; ++kk) {
        const float Rjk = G.R[3 * jj + kk];
        Ga1[jj] += Rjk * G.s[kk] * Gu1[kk];
        Ga2[jj] += Rjk * G.s[kk] * Gu2[kk];
        const float gm = G.a1[jj] * Gu1[kk] + G.a2[jj] * Gu2[kk];
        GR[3 * jj + kk] = G.s[kk] * gm;
        ds[kk] += Rjk * gm;
      }
    }
    // a_i = W^T e_ic / r -> gradient w.r.t. (e_ic / r) in the camera frame: W G_a_i
    float Gc1[3], Gc2[3];
    for (int r = 0; r < 3; ++r) {
      Gc1[r] = vp.W[3 * r] * Ga1[0] + vp.W[3 * r + 1] * Ga1[1] + vp.W[3 * r + 2] * Ga1[2];
      Gc2[r] = vp.W[3 * r] * Ga2[0] + vp.W[3 * r + 1] * Ga2[1] + vp.W[3 * r + 2] * Ga2[2];
    }
    const float ir = 1.f / G.r, ir2 = ir * ir;
    const float g1 = Gc1[0] * G.gc.x + Gc1[1] * G.gc.y + Gc1[2] * G.gc.z;
    const float g2 = Gc2[0] * G.gc.x + Gc2[1] * G.gc.y + Gc2[2] * G.gc.z;
    const float h1 = Gc1[0] * G.e1c.x + Gc1[1] * G.e1c.y + Gc1[2] * G.e1c.z;
    const float h2 = Gc2[0] * G.e2c.x + Gc2[1] * G.e2c.y + Gc2[2] * G.e2c.z;
    float Lt[3];
    Lt[0] = -ir2 * (g1 * G.e1c.x + g2 * G.e2c.x + (h1 + h2) * G.gc.x) + ir * (A[7] * G.e1c.x + A[8] * G.e2c.x);
    Lt[1] = -ir2 * (g1 * G.e1c.y + g2 * G.e2c.y + (h1 + h2) * G.gc.y) + ir * (A[7] * G.e1c.y + A[8] * G.e2c.y);
    Lt[2] = -ir2 * (g1 * G.e1c.z + g2 * G.e2c.z + (h1 + h2) * G.gc.z) + ir * (A[7] * G.e1c.z + A[8] * G.e2c.z);
    if (accum_d) {                                 // inverse-depth channel: d(1/r)/dt = -t / r^3 = -g_c / r^2
      const float ad = accum_d[gid] * ir2;
      Lt[0] -= ad * G.gc.x; Lt[1] -= ad * G.gc.y; Lt[2] -= ad * G.gc.z;
    }
    for (int e = 0; e < 3; ++e) dmu[e] += vp.W[e] * Lt[0] + vp.W[3 + e] * Lt[1] + vp.W[6 + e] * Lt[2];
    // R(q_hat) -> q_hat -> q
    const float w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
    const float Lw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
    const float Lx = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] - 2.f * x * GR[8]);
    const float Ly = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] - 2.f * y * GR[8]);
    const float Lz = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] + x * GR[6] + y * GR[7]);
    const float qd = Lw * w + Lx * x + Ly * y + Lz * z;
    const float iq = 1.f / G.qnorm;
    dq[0] += (Lw - w * qd) * iq;
    dq[1] += (Lx - x * qd) * iq;
    dq[2] += (Ly - y * qd) * iq;
    dq[3] += (Lz - z * qd) * iq;
  }
  for (int c = 0; c < 3; ++c) { dmeans[3 * (int64_t)i + c] = dmu[c]; dscales[3 * (int64_t)i + c] = ds[c]; }
  for (int c = 0; c < 4; ++c) drot[4 * (int64_t)i + c] = dq[c];
  dopac[i] = dop;
  }
  __syncthreads();
  for (int t = tid; t < nrow * 3 * K; t += kPreBwdThreads) {
    const int r = t / (3 * K), c = t - r * (3 * K);
    dsh[(int64_t)i0 * 3 * K + t] = s_dsh[r * RW + c];
  }
}

// ----------------------------------------------------------------------------
// Radian-space density statistics (Sec. 4.2): one thread per (view, Gaussian).
// The blend backward's partials hold dL/d(east, north displacement) with the conic
// held in the parallel-transported frame (accum 7, 8) and dL/d(conic a, b, c)
// (accum 4-6). Moving the centre east by d omega turns the local (east, north)
// frame against the transported one by sin(phi) d omega, so with the conic held in
// the local frame dL/domega = cos(phi) L_E + sin(phi) (2 b (L_c - L_a) + (a - c) L_b)
// and dL/dphi = L_N.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_density_stats(int64_t PV, int P, const uint32_t* __restrict__ skeys,
                                                       const uint32_t* __restrict__ svals, const uint32_t* __restrict__ counts,
                                                       const float4* __restrict__ rec,
                                                       const float* __restrict__ radii, const float* __restrict__ accum,
                                                       float* __restrict__ rs_max, float* __restrict__ grad_accum,
                                                       uint32_t* __restrict__ vis_count, float* __restrict__ angular) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // depth-sorted position
  if (j >= PV) return;
  const uint32_t gid = svals[j];
  // visible: listed for at least one active tile of its view
  const bool vis = skeys[j] != 0xffffffffu && counts[gid] > 0u;
  float dw = 0.f, dp = 0.f;
  if (vis) {
    const float rs = radii[gid];
    const float4 r0 = rec[4 * (int64_t)gid], r1 = rec[4 * (int64_t)gid + 1], r2 = rec[4 * (int64_t)gid + 2],
                 r3 = rec[4 * (int64_t)gid + 3];
    const float* A = accum + (int64_t)gid * HPXGS_NACC;
    const float a = r1.w, b = r2.w, c = r3.w;
    const float sphi = r0.z, cphi = sqrtf(r0.x * r0.x + r0.y * r0.y);
    const float La = 2.f * b * (A[6] - A[4]) + (a - c) * A[5];
    dw = cphi * A[7] + sphi * La;
    dp = A[8];
    const uint32_t i = gid % (uint32_t)P;
    atomicMax(reinterpret_cast<int*>(rs_max) + i, __float_as_int(rs));   // rs > 0: int order = float order
    atomicAdd(grad_accum + i, sqrtf(dw * dw + dp * dp));
    atomicAdd(vis_count + i, 1u);
  }
  if (angular) { angular[2 * (int64_t)gid] = dw; angular[2 * (int64_t)gid + 1] = dp; }
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
template <typename T>
static T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

static int blend_blocks(const void* fn, int nt, int want_per_sm) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, 0) != cudaSuccess || occ < 1) occ = 1;
  if (want_per_sm > 0 && want_per_sm < occ) occ = want_per_sm;
  return occ * num_sms();
}

// Entries staged per batch by the forward blend (a multiple of 32).
#ifndef HPXGS_FWD_BATCH
#define HPXGS_FWD_BATCH 128
#endif
// Launch of a blend kernel with NT threads x PPT pixels per thread = the tile's pixels.
template <int NT, int PPT, bool DEPTH = false, bool SPLIT = false, typename... Args>
static void launch_fwd(int bps, cudaStream_t s, Args... args) {
  auto fn = k_blend_fwd<NT, PPT, HPXGS_FWD_BATCH, DEPTH, SPLIT>;
  fn<<<blend_blocks((const void*)fn, NT, bps), NT, 0, s>>>(args...);
}
template <int NT, int PPT, bool DEPTH = false, bool SPLIT = false, bool LOSS = false, typename... Args>
static void launch_bwd(int bps, cudaStream_t s, Args... args) {
  auto fn = k_blend_bwd<NT, PPT, 32, DEPTH, SPLIT, LOSS>;
  fn<<<blend_blocks((const void*)fn, NT, bps), NT, 0, s>>>(args...);
}

// Pixels per thread of each kernel by tile level (the first entry is the default).
static int pick_ppt(int b, int want, bool fwd) {
  static const int f3[] = {1, 2}, f4[] = {1, 2, 4}, f5[] = {4, 8};
  static const int g3[] = {2, 1}, g4[] = {4, 2, 8}, g5[] = {4, 8};
  const int* opts; int n;
  if (b == 3) { opts = fwd ? f3 : g3; n = 2; }
  else if (b == 4) { opts = fwd ? f4 : g4; n = 3; }
  else { opts = fwd ? f5 : g5; n = 2; }
  for (int i = 0; i < n; ++i) if (opts[i] == want) return want;
  return opts[0];
}

constexpr int kBatchFwd = 128;
constexpr int kBatchBwd = 32;

static bool check_gaussians(const hpxgs_gaussians* g) {
  if (!g || g->P < 0 || g->sh_degree < 0 || g->sh_degree > 3) return false;
  if (g->P > 0 && (!g->means || !g->scales || !g->rotations || !g->opacities || !g->sh)) return false;
  return true;
}

// Steps shared by forward and count: table, mask/flags, preprocess, depth sort,
// counts, scan. On return `which` tells where the depth-sorted keys/values are.
static int front_half(const hpxgs_gaussians* g, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                      void* ws, const Layout& L, ViewTable* vt, uint32_t* mask_out, int32_t* status,
                      uint64_t* total_out, cudaStream_t s, int* which_depth) {
  int rc = make_table(g, g->P, views, nviews, cfg, s, true, vt);
  if (rc != HPXGS_OK) return rc;
  uint32_t* flags = at<uint32_t>(ws, L.tile_flags);
  uint32_t* counters = at<uint32_t>(ws, L.counters);
  HPXGS_CUDA_CHECK(cudaMemsetAsync(counters, 0, sizeof(uint32_t) * C_COUNT, s));
  // Three chains meet at the scan: the FoV masks and tile flags (kept in the workspace: the
  // backward reads them) depend only on the cameras; the depth sort only on the preprocess;
  // the tile count pass on the preprocess and the flags, not on the depth order (it counts
  // per Gaussian). The masks run on a helper stream and the depth sort on a high-priority
  // one (its short kernels would otherwise wait behind the count pass's blocks); the count
  // pass waits for the masks, the scan for the sort.
  const Fork* fk = fork_of(s);
  cudaStream_t ms = s;
  if (fk) {
    HPXGS_CUDA_CHECK(cudaEventRecord(fk->fork, s));
    HPXGS_CUDA_CHECK(cudaStreamWaitEvent(fk->side, fk->fork, 0));
    ms = fk->side;
  }
  HPXGS_CUDA_CHECK(cudaMemsetAsync(flags, 0, sizeof(uint32_t) * L.total_tiles, ms));
  prof_begin(HPXGS_STAGE_MASK, ms);
  for (int v = 0; v < nviews && rc == HPXGS_OK; ++v)
    rc = launch_mask(vt->v[v], cfg->tile_level, mask_out + (vt->v[v].pix_base >> 5), flags + vt->v[v].tile_base, ms);
  prof_end(HPXGS_STAGE_MASK, ms);
  if (fk) HPXGS_CUDA_CHECK(cudaEventRecord(fk->mid[0], fk->side));    // masks and flags done
  bool sorting = false;                            // the depth sort was enqueued on side_hi
  auto join = [&]() -> int {                      // s waits for all the helper streams hold
    if (fk) {
      HPXGS_CUDA_CHECK(cudaEventRecord(fk->join, fk->side));
      HPXGS_CUDA_CHECK(cudaStreamWaitEvent(s, fk->join, 0));
      if (sorting) {
        HPXGS_CUDA_CHECK(cudaEventRecord(fk->join_hi, fk->side_hi));
        HPXGS_CUDA_CHECK(cudaStreamWaitEvent(s, fk->join_hi, 0));
      }
      fk = nullptr;
    }
    return HPXGS_OK;
  };
  if (rc != HPXGS_OK) { join(); return rc; }
  const int64_t PV = L.PV;
  *which_depth = 0;
  if (PV == 0) return join();
  float4* rec = at<float4>(ws, L.records);
  float* radii = at<float>(ws, L.radii);
  float* depth = at<float>(ws, L.depth);
  uint32_t* ka = at<uint32_t>(ws, L.key_a); uint32_t* kb = at<uint32_t>(ws, L.key_b);
  uint32_t* va = at<uint32_t>(ws, L.val_a); uint32_t* vb = at<uint32_t>(ws, L.val_b);
  prof_begin(HPXGS_STAGE_PREPROCESS, s);
  {
    const dim3 nb((unsigned)((g->P + kPreThreads - 1) / kPreThreads), (unsigned)nviews);
    switch (g->sh_degree) {
      case 0: k_preprocess<0><<<nb, kPreThreads, 0, s>>>(*vt, *g, rec, radii, depth, ka, va); break;
      case 1: k_preprocess<1><<<nb, kPreThreads, 0, s>>>(*vt, *g, rec, radii, depth, ka, va); break;
      case 2: k_preprocess<2><<<nb, kPreThreads, 0, s>>>(*vt, *g, rec, radii, depth, ka, va); break;
      default: k_preprocess<3><<<nb, kPreThreads, 0, s>>>(*vt, *g, rec, radii, depth, ka, va); break;
    }
  }
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  prof_end(HPXGS_STAGE_PREPROCESS, s);
  cudaStream_t ss = s;                             // the depth sort's stream
  if (fk) {                                        // the depth sort follows the preprocess on side_hi
    HPXGS_CUDA_CHECK(cudaEventRecord(fk->mid[1], s));
    HPXGS_CUDA_CHECK(cudaStreamWaitEvent(fk->side_hi, fk->mid[1], 0));
    ss = fk->side_hi;
    sorting = true;
  }
  prof_begin(HPXGS_STAGE_DEPTH_SORT, ss);
  // a grid sized to the element count (HPXGS_DSORT_TPB tiles of 4096 per block, at most kMaxSortBlocks)
  const int Gd = (int)std::max<int64_t>(1, std::min<int64_t>(kMaxSortBlocks, (PV + HPXGS_DSORT_TPB * kSortTile - 1) / (HPXGS_DSORT_TPB * kSortTile)));
  rc = radix_sort(ka, va, kb, vb, nullptr, (uint32_t)PV, 32, at<uint32_t>(ws, L.hist), Gd, counters + C_SORT_TICKET, ss,
                  which_depth);
  if (rc != HPXGS_OK) { join(); return rc; }
  prof_end(HPXGS_STAGE_DEPTH_SORT, ss);
  if (fk) HPXGS_CUDA_CHECK(cudaStreamWaitEvent(s, fk->mid[0], 0));      // the count pass reads the tile flags
  const uint32_t* sk = *which_depth ? kb : ka;
  const uint32_t* sv = *which_depth ? vb : va;
  uint32_t* counts = at<uint32_t>(ws, L.counts);
  uint64_t* offsets = at<uint64_t>(ws, L.offsets);
  uint64_t* part = at<uint64_t>(ws, L.scan_part);
  prof_begin(HPXGS_STAGE_TILE_COUNT, s);
  const unsigned tblocks = (unsigned)std::min<int64_t>((PV + 8 * kTilesBatch - 1) / (8 * kTilesBatch), 32LL * num_sms());
  if (vt->query == HPXGS_QUERY_NESTED) {
    const unsigned nblocks = (unsigned)std::min<int64_t>((PV + 255) / 256, 32LL * num_sms());
    k_tiles_nested<false><<<nblocks, 256, 0, s>>>(*vt, rec, radii, sk, sv, flags, counts, nullptr, nullptr, nullptr,
                                                  (uint64_t)L.cap, status);
  } else {
    // the count pass stages member lists in the second pair buffers (unused until the pair sort)
    if (vt->log2f > 0)                             // RING x f: search at order k_t + log2f
      k_tiles<false, true><<<tblocks, 256, 0, s>>>(*vt, rec, radii, sk, sv, flags, counts, nullptr, nullptr, nullptr,
                                                   (uint64_t)L.cap, status, at<uint32_t>(ws, L.stage),
                                                   at<uint32_t>(ws, L.pair_key_b), counters + C_STAGE);
    else
      k_tiles<false, false><<<tblocks, 256, 0, s>>>(*vt, rec, radii, sk, sv, flags, counts, nullptr, nullptr, nullptr,
                                                    (uint64_t)L.cap, status, at<uint32_t>(ws, L.stage),
                                                    at<uint32_t>(ws, L.pair_key_b), counters + C_STAGE);
  }
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  prof_end(HPXGS_STAGE_TILE_COUNT, s);
  rc = join();                                     // the scan takes the counts in depth order
  if (rc != HPXGS_OK) return rc;
  const int G = L.sort_blocks;
  prof_begin(HPXGS_STAGE_SCAN, s);
  static int scan_cap = -1;
  if (scan_cap < 0) scan_cap = coop_capacity((const void*)k_scan_coop, 256);
  if (G <= scan_cap) {
    HPXGS_CUDA_CHECK(launch_cooperative(k_scan_coop, (unsigned)G, 256, s, (const uint32_t*)counts, sv, (int64_t)PV,
                                        part, offsets, counters, total_out, counters + C_GRID_BAR_SCAN, status));
    note_launches(1);
  } else {
    k_scan_part<<<G, 256, 0, s>>>(counts, sv, PV, G, part);
    k_scan_top<<<1, kMaxSortBlocks, 0, s>>>(part, G, counters, total_out);
    k_scan_apply<<<G, 256, 0, s>>>(counts, sv, PV, G, part, offsets);
    note_launches(3);
  }
  HPXGS_LAUNCH_CHECK();
  prof_end(HPXGS_STAGE_SCAN, s);
  return HPXGS_OK;
}

}  // namespace hpxgs

using namespace hpxgs;

extern "C" {

int hpxgs_forward_workspace_size(int32_t P, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                                 int64_t cap, size_t* bytes) {
  if (!bytes) return HPXGS_E_INVALID_ARG;
  Layout L;
  int rc = make_layout(P, views, nviews, cfg, cap, &L);
  if (rc != HPXGS_OK) return rc;
  // the mask area used when the caller passes no mask buffer
  int64_t pix = L.total_pix;
  *bytes = L.total + ((size_t)(pix / 32) * 4 + 255) / 256 * 256;
  return HPXGS_OK;
}

static uint32_t* internal_mask(void* ws, const Layout& L) { return at<uint32_t>(ws, L.total); }

int hpxgs_workspace_inspect(int32_t P, const hpxgs_view* views, int nviews, const hpxgs_config* cfg, int64_t cap,
                            const void* ws, hpxgs_workspace_view* out) {
  if (!ws || !out) return HPXGS_E_INVALID_ARG;
  Layout L;
  int rc = make_layout(P, views, nviews, cfg, cap, &L);
  if (rc != HPXGS_OK) return rc;
  void* w = const_cast<void*>(ws);
  int pbits = L.pair_bits, passes = (pbits + 7) / 8;
  out->records = at<float>(w, L.records);
  out->radii = at<float>(w, L.radii);
  out->depth = at<float>(w, L.depth);
  out->pair_tiles = (passes & 1) ? at<uint32_t>(w, L.pair_key_b) : at<uint32_t>(w, L.pair_key_a);
  out->pair_ids = (passes & 1) ? at<uint32_t>(w, L.pair_val_b) : at<uint32_t>(w, L.pair_val_a);
  out->ranges = at<uint32_t>(w, L.ranges);
  out->n_pairs = at<uint32_t>(w, L.counters) + C_NPAIRS;
  out->accum = at<float>(w, L.accum);
  out->n_eval = reinterpret_cast<const uint64_t*>(at<uint32_t>(w, L.counters) + C_NEVAL);
  out->n_contrib = reinterpret_cast<const uint64_t*>(at<uint32_t>(w, L.counters) + C_NCONTRIB);
  out->cull_masks = (passes & 1) ? at<uint32_t>(w, L.pair_key_a) : at<uint32_t>(w, L.pair_key_b);
  out->total_tiles = L.total_tiles;
  return HPXGS_OK;
}

int hpxgs_count_pairs(const hpxgs_gaussians* g, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                      void* ws, size_t ws_bytes, uint64_t* count, int32_t* status, hpxgs_stream_t stream) {
  if (!check_gaussians(g) || !ws || !count) return HPXGS_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Layout L;
  int rc = make_layout(g->P, views, nviews, cfg, 0, &L);
  if (rc != HPXGS_OK) return rc;
  size_t need = 0;
  hpxgs_forward_workspace_size(g->P, views, nviews, cfg, 0, &need);
  if (ws_bytes < need) return HPXGS_E_WORKSPACE;
  ViewTable* vt = new ViewTable;
  int which = 0;
  HPXGS_CUDA_CHECK(cudaMemsetAsync(count, 0, sizeof(uint64_t), s));
  rc = front_half(g, views, nviews, cfg, ws, L, vt, internal_mask(ws, L), status, count, s, &which);
  delete vt;
  return rc;
}

int hpxgs_forward(const hpxgs_gaussians* g, const hpxgs_view* views, int nviews, const hpxgs_config* cfg, void* ws,
                  size_t ws_bytes, int64_t cap, float* maps, float* T_final, uint32_t* last, uint32_t* mask_bits,
                  float* radii_out, float* depth_map, int32_t* status, hpxgs_stream_t stream) {
  if (!check_gaussians(g) || !ws || !maps || !T_final || !last) return HPXGS_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Layout L;
  int rc = make_layout(g->P, views, nviews, cfg, cap, &L);
  if (rc != HPXGS_OK) return rc;
  size_t need = 0;
  hpxgs_forward_workspace_size(g->P, views, nviews, cfg, cap, &need);
  if (ws_bytes < need) return HPXGS_E_WORKSPACE;
  ViewTable* vt = new ViewTable;
  int which = 0;
  uint32_t* mask = internal_mask(ws, L);
  rc = front_half(g, views, nviews, cfg, ws, L, vt, mask, status, nullptr, s, &which);
  if (rc != HPXGS_OK) { delete vt; return rc; }
  uint32_t* counters = at<uint32_t>(ws, L.counters);
  uint32_t* flags = at<uint32_t>(ws, L.tile_flags);
  uint2* ranges = at<uint2>(ws, L.ranges);
  float4* rec = at<float4>(ws, L.records);
  uint32_t* pka = at<uint32_t>(ws, L.pair_key_a); uint32_t* pkb = at<uint32_t>(ws, L.pair_key_b);
  uint32_t* pva = at<uint32_t>(ws, L.pair_val_a); uint32_t* pvb = at<uint32_t>(ws, L.pair_val_b);
  const int64_t PV = L.PV;
  if (PV > 0 && cap > 0) {
    const uint32_t* sk = which ? at<uint32_t>(ws, L.key_b) : at<uint32_t>(ws, L.key_a);
    const uint32_t* sv = which ? at<uint32_t>(ws, L.val_b) : at<uint32_t>(ws, L.val_a);
    prof_begin(HPXGS_STAGE_TILE_EMIT, s);
    const unsigned tblocks = (unsigned)std::min<int64_t>((PV + 8 * kTilesBatch - 1) / (8 * kTilesBatch), 32LL * num_sms());
    if (vt->query == HPXGS_QUERY_NESTED) {
      const unsigned nblocks = (unsigned)std::min<int64_t>((PV + 255) / 256, 32LL * num_sms());
      k_tiles_nested<true><<<nblocks, 256, 0, s>>>(*vt, rec, at<float>(ws, L.radii), sk, sv, flags,
                                                   at<uint32_t>(ws, L.counts), at<uint64_t>(ws, L.offsets), pka, pva,
                                                   (uint64_t)cap, status);
    } else {
      if (vt->log2f > 0)
        k_tiles<true, true><<<tblocks, 256, 0, s>>>(*vt, rec, at<float>(ws, L.radii), sk, sv, flags,
                                                    at<uint32_t>(ws, L.counts), at<uint64_t>(ws, L.offsets), pka, pva,
                                                    (uint64_t)cap, status, at<uint32_t>(ws, L.stage), pkb,
                                                    counters + C_STAGE);
      else
        k_tiles<true, false><<<tblocks, 256, 0, s>>>(*vt, rec, at<float>(ws, L.radii), sk, sv, flags,
                                                     at<uint32_t>(ws, L.counts), at<uint64_t>(ws, L.offsets), pka, pva,
                                                     (uint64_t)cap, status, at<uint32_t>(ws, L.stage), pkb,
                                                     counters + C_STAGE);
    }
    note_launches(1);
    HPXGS_LAUNCH_CHECK();
    prof_end(HPXGS_STAGE_TILE_EMIT, s);
    int wp = 0;
    prof_begin(HPXGS_STAGE_PAIR_SORT, s);
    rc = radix_sort(pka, pva, pkb, pvb, counters + C_NPAIRS, (uint32_t)cap, L.pair_bits, at<uint32_t>(ws, L.hist),
                    L.pair_sort_blocks, counters + C_SORT_TICKET, s, &wp);
    if (rc != HPXGS_OK) { delete vt; return rc; }
    prof_end(HPXGS_STAGE_PAIR_SORT, s);
    const uint32_t* sorted_tiles = wp ? pkb : pka;
    prof_begin(HPXGS_STAGE_RANGES, s);
    HPXGS_CUDA_CHECK(cudaMemsetAsync(ranges, 0, sizeof(uint2) * L.total_tiles, s));
    const int64_t rblocks = std::min<int64_t>((cap + 1023) / 1024, 16LL * num_sms());
    k_ranges<<<(unsigned)rblocks, 256, 0, s>>>(sorted_tiles, counters + C_NPAIRS, (uint32_t)cap, ranges);
    note_launches(1);
    HPXGS_LAUNCH_CHECK();
    prof_end(HPXGS_STAGE_RANGES, s);
  } else {
    HPXGS_CUDA_CHECK(cudaMemsetAsync(ranges, 0, sizeof(uint2) * L.total_tiles, s));
  }
  const int passes = (L.pair_bits + 7) / 8;
  const uint32_t* ids = (passes & 1) ? pvb : pva;
  uint32_t* gmask = (passes & 1) ? pka : pkb;        // the sort's free key buffer: per-entry cull masks
  uint32_t* work = counters + C_WORK_FWD;
  unsigned long long* evals = reinterpret_cast<unsigned long long*>(counters + C_NEVAL);
  const int b = cfg->tile_level;
  const bool split = b == 5 && cfg->blend_split;   // quarters of order-5 tiles as blend units
  const int bps = cfg->blocks_per_sm;
  // blend units: [forward order | backward order | forward evaluations per unit], 4 x tiles each
  uint32_t* uorder = at<uint32_t>(ws, L.unit_order);
  const int64_t ustride = 4 * L.total_tiles;
  prof_begin(HPXGS_STAGE_BLEND_FWD, s);
  rc = launch_unit_order(0, (int)(split ? 4 * L.total_tiles : L.total_tiles), split ? 2 : 0, ranges, flags, nullptr,
                         counters + C_UNITS_FWD, uorder, s);
  if (rc != HPXGS_OK) { delete vt; return rc; }
  {
    const int ppt = pick_ppt(b, cfg->fwd_ppt, true);
#define FWD_BASE bps, s, *vt, (const float4*)rec, (const uint2*)ranges, ids, (const uint32_t*)flags, (const uint32_t*)mask, maps, T_final, last, work, evals, gmask, (const uint32_t*)uorder, uorder + 2 * ustride
#define FWD_ARGS FWD_BASE, (const float*)nullptr, (float*)nullptr
#define FWD_DEPTH_ARGS FWD_BASE, (const float*)at<float>(ws, L.depth), depth_map
    if (split) {                                   // order-5 lists, quarters blended in the order-4 shapes
      if (depth_map) launch_fwd<256, 1, true, true>(FWD_DEPTH_ARGS);
      else if (pick_ppt(4, cfg->fwd_ppt, true) == 2) launch_fwd<128, 2, false, true>(FWD_ARGS);
      else if (pick_ppt(4, cfg->fwd_ppt, true) == 4) launch_fwd<64, 4, false, true>(FWD_ARGS);
      else launch_fwd<256, 1, false, true>(FWD_ARGS);
    } else if (depth_map) {                        // the depth channel runs in each level's default shape
      if (b == 3) launch_fwd<64, 1, true>(FWD_DEPTH_ARGS);
      else if (b == 4) launch_fwd<256, 1, true>(FWD_DEPTH_ARGS);
      else launch_fwd<256, 4, true>(FWD_DEPTH_ARGS);
    } else if (b == 3) { if (ppt == 2) launch_fwd<32, 2>(FWD_ARGS); else launch_fwd<64, 1>(FWD_ARGS); }
    else if (b == 4) {
      if (ppt == 2) launch_fwd<128, 2>(FWD_ARGS);
      else if (ppt == 4) launch_fwd<64, 4>(FWD_ARGS);
      else launch_fwd<256, 1>(FWD_ARGS);
    } else { if (ppt == 8) launch_fwd<128, 8>(FWD_ARGS); else launch_fwd<256, 4>(FWD_ARGS); }
#undef FWD_DEPTH_ARGS
#undef FWD_ARGS
#undef FWD_BASE
  }
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  prof_end(HPXGS_STAGE_BLEND_FWD, s);
  if (mask_bits)
    HPXGS_CUDA_CHECK(cudaMemcpyAsync(mask_bits, mask, sizeof(uint32_t) * (L.total_pix / 32), cudaMemcpyDeviceToDevice, s));
  if (radii_out && PV > 0)
    HPXGS_CUDA_CHECK(cudaMemcpyAsync(radii_out, at<float>(ws, L.radii), sizeof(float) * PV, cudaMemcpyDeviceToDevice, s));
  delete vt;
  return HPXGS_OK;
}

}  // extern "C"

// hpxgs_backward with dL/dI from a map (dmaps) or, with lv, from the views' L1 + HSSIM gradient.
static int backward_impl(const hpxgs_gaussians* g, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                         void* ws, size_t ws_bytes, int64_t cap, const float* dmaps, const LossViews* lv,
                         const float* T_final, const uint32_t* last, const float* ddepth, float* dmeans,
                         float* dscales, float* drot, float* dopac, float* dsh, hpxgs_stream_t stream) {
  if (!check_gaussians(g) || !ws || !(dmaps || lv) || !T_final || !last) return HPXGS_E_INVALID_ARG;
  if (g->P > 0 && (!dmeans || !dscales || !drot || !dopac || !dsh)) return HPXGS_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Layout L;
  int rc = make_layout(g->P, views, nviews, cfg, cap, &L);
  if (rc != HPXGS_OK) return rc;
  size_t need = 0;
  hpxgs_forward_workspace_size(g->P, views, nviews, cfg, cap, &need);
  if (ws_bytes < need) return HPXGS_E_WORKSPACE;
  ViewTable* vt = new ViewTable;
  rc = make_table(g, g->P, views, nviews, cfg, s, true, vt);
  if (rc != HPXGS_OK) { delete vt; return rc; }
  const int64_t PV = L.PV;
  if (PV == 0) { delete vt; return HPXGS_OK; }
  uint32_t* counters = at<uint32_t>(ws, L.counters);
  float* accum = at<float>(ws, L.accum);
  HPXGS_CUDA_CHECK(cudaMemsetAsync(accum, 0, sizeof(float) * HPXGS_NACC * PV, s));
  float* accum_d = at<float>(ws, L.accum_d);
  if (ddepth) HPXGS_CUDA_CHECK(cudaMemsetAsync(accum_d, 0, sizeof(float) * PV, s));
  const float* rdepth = at<float>(ws, L.depth);
  HPXGS_CUDA_CHECK(cudaMemsetAsync(counters + C_WORK_BWD, 0, sizeof(uint32_t) * (1 + 2 * kUnitClasses), s));
  const int passes = (L.pair_bits + 7) / 8;
  const uint32_t* ids = (passes & 1) ? at<uint32_t>(ws, L.pair_val_b) : at<uint32_t>(ws, L.pair_val_a);
  const uint32_t* gmask = (passes & 1) ? at<uint32_t>(ws, L.pair_key_a) : at<uint32_t>(ws, L.pair_key_b);
  const float4* rec = at<float4>(ws, L.records);
  const uint2* ranges = at<uint2>(ws, L.ranges);
  const uint32_t* flags = at<uint32_t>(ws, L.tile_flags);
  const uint32_t* mask = internal_mask(ws, L);      // written by the forward
  uint32_t* work = counters + C_WORK_BWD;
  const int b = cfg->tile_level;
  const bool split = b == 5 && cfg->blend_split;   // quarters of order-5 tiles as blend units
  const int bps = cfg->blocks_per_sm;
  uint32_t* uorder = at<uint32_t>(ws, L.unit_order);
  const int64_t ustride = 4 * L.total_tiles;
  prof_begin(HPXGS_STAGE_BLEND_BWD, s);
  rc = launch_unit_order(1, (int)(split ? 4 * L.total_tiles : L.total_tiles), 0, ranges, flags, uorder + 2 * ustride,
                         counters + C_UNITS_BWD, uorder + ustride, s);
  if (rc != HPXGS_OK) { delete vt; return rc; }
  {
    // several pixels per thread: the per-entry warp reduction then covers 32 * PPT pixels
    const int ppt = pick_ppt(b, cfg->bwd_ppt, false);
#define BWD_BASE bps, s, *vt, rec, ranges, ids, flags, mask, dmaps, T_final, last, accum, work, gmask, (const uint32_t*)(uorder + ustride)
#define BWD_ARGS BWD_BASE, (const float*)nullptr, (const float*)nullptr, (float*)nullptr, NoLossViews{0.f}
#define BWD_DEPTH_ARGS BWD_BASE, rdepth, ddepth, accum_d, NoLossViews{0.f}
#define BWD_LOSS_ARGS BWD_BASE, (const float*)nullptr, (const float*)nullptr, (float*)nullptr, *lv
    if (lv) {                                      // each level's default shape
      if (split) launch_bwd<64, 4, false, true, true>(BWD_LOSS_ARGS);
      else if (b == 3) launch_bwd<32, 2, false, false, true>(BWD_LOSS_ARGS);
      else if (b == 4) launch_bwd<64, 4, false, false, true>(BWD_LOSS_ARGS);
      else launch_bwd<256, 4, false, false, true>(BWD_LOSS_ARGS);
    } else if (split) {                                   // order-5 lists, quarters blended in the order-4 shapes
      if (ddepth) launch_bwd<64, 4, true, true>(BWD_DEPTH_ARGS);
      else if (pick_ppt(4, cfg->bwd_ppt, false) == 2) launch_bwd<128, 2, false, true>(BWD_ARGS);
      else if (pick_ppt(4, cfg->bwd_ppt, false) == 8) launch_bwd<32, 8, false, true>(BWD_ARGS);
      else launch_bwd<64, 4, false, true>(BWD_ARGS);
    } else if (ddepth) {                           // the depth channel runs in each level's default shape
      if (b == 3) launch_bwd<32, 2, true>(BWD_DEPTH_ARGS);
      else if (b == 4) launch_bwd<64, 4, true>(BWD_DEPTH_ARGS);
      else launch_bwd<256, 4, true>(BWD_DEPTH_ARGS);
    } else if (b == 3) { if (ppt == 1) launch_bwd<64, 1>(BWD_ARGS); else launch_bwd<32, 2>(BWD_ARGS); }
    else if (b == 4) {
      if (ppt == 2) launch_bwd<128, 2>(BWD_ARGS);
      else if (ppt == 8) launch_bwd<32, 8>(BWD_ARGS);
      else launch_bwd<64, 4>(BWD_ARGS);
    } else { if (ppt == 8) launch_bwd<128, 8>(BWD_ARGS); else launch_bwd<256, 4>(BWD_ARGS); }
#undef BWD_LOSS_ARGS
#undef BWD_DEPTH_ARGS
#undef BWD_ARGS
#undef BWD_BASE
  }
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  prof_end(HPXGS_STAGE_BLEND_BWD, s);
  prof_begin(HPXGS_STAGE_PREPROCESS_BWD, s);
  {
    const int nb = (int)((g->P + kPreBwdThreads - 1) / kPreBwdThreads);
    const float* rad = at<float>(ws, L.radii);
    const float* acd = ddepth ? at<float>(ws, L.accum_d) : nullptr;
    switch (g->sh_degree) {
      case 0: k_preprocess_bwd<0><<<nb, kPreBwdThreads, 0, s>>>(*vt, *g, rad, accum, dmeans, dscales, drot, dopac, dsh, acd); break;
      case 1: k_preprocess_bwd<1><<<nb, kPreBwdThreads, 0, s>>>(*vt, *g, rad, accum, dmeans, dscales, drot, dopac, dsh, acd); break;
      case 2: k_preprocess_bwd<2><<<nb, kPreBwdThreads, 0, s>>>(*vt, *g, rad, accum, dmeans, dscales, drot, dopac, dsh, acd); break;
      default: k_preprocess_bwd<3><<<nb, kPreBwdThreads, 0, s>>>(*vt, *g, rad, accum, dmeans, dscales, drot, dopac, dsh, acd); break;
    }
  }
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  prof_end(HPXGS_STAGE_PREPROCESS_BWD, s);
  delete vt;
  return HPXGS_OK;
}

extern "C" {

int hpxgs_backward(const hpxgs_gaussians* g, const hpxgs_view* views, int nviews, const hpxgs_config* cfg, void* ws,
                   size_t ws_bytes, int64_t cap, const float* dmaps, const float* T_final, const uint32_t* last,
                   const float* ddepth, float* dmeans, float* dscales, float* drot, float* dopac, float* dsh,
                   int32_t* status, hpxgs_stream_t stream) {
  (void)status;
  if (!dmaps) return HPXGS_E_INVALID_ARG;
  return backward_impl(g, views, nviews, cfg, ws, ws_bytes, cap, dmaps, nullptr, T_final, last, ddepth, dmeans,
                       dscales, drot, dopac, dsh, stream);
}

int hpxgs_backward_hssim(const hpxgs_gaussians* g, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                         void* ws, size_t ws_bytes, int64_t cap, const hpxgs_loss_view* loss_views, float lambda,
                         const float* T_final, const uint32_t* last, float* dmeans, float* dscales, float* drot,
                         float* dopac, float* dsh, int32_t* status, hpxgs_stream_t stream) {
  (void)status;
  if (!loss_views || !views || nviews < 1 || nviews > HPXGS_MAX_VIEWS || !(lambda >= 0.f && lambda <= 1.f))
    return HPXGS_E_INVALID_ARG;
  LossViews* lv = new LossViews;
  std::memset(lv, 0, sizeof(*lv));
  lv->lambda = lambda;
  for (int v = 0; v < nviews; ++v) {
    const hpxgs_loss_view& l = loss_views[v];
    const int k = views[v].nside_log2;
    if (!l.maps || !l.targets || !l.table || !l.hssim_ws || k < 3 || k > 13) { delete lv; return HPXGS_E_INVALID_ARG; }
    hssim_bind(k, l.table, l.hssim_ws, &lv->v[v]);
    lv->v[v].I = l.maps;
    lv->v[v].G = l.targets;
    lv->v[v].dloss = l.dloss;
  }
  const int rc = backward_impl(g, views, nviews, cfg, ws, ws_bytes, cap, nullptr, lv, T_final, last, nullptr, dmeans,
                               dscales, drot, dopac, dsh, stream);
  delete lv;
  return rc;
}

int hpxgs_density_stats(int32_t P, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                        const void* ws, size_t ws_bytes, int64_t cap, float* rs_max, float* grad_accum,
                        uint32_t* vis_count, float* angular, hpxgs_stream_t stream) {
  if (!ws || !rs_max || !grad_accum || !vis_count || P < 0) return HPXGS_E_INVALID_ARG;
  Layout L;
  int rc = make_layout(P, views, nviews, cfg, cap, &L);
  if (rc != HPXGS_OK) return rc;
  size_t need = 0;
  hpxgs_forward_workspace_size(P, views, nviews, cfg, cap, &need);
  if (ws_bytes < need) return HPXGS_E_WORKSPACE;
  if (L.PV == 0) return HPXGS_OK;
  void* w = const_cast<void*>(ws);
  cudaStream_t s = (cudaStream_t)stream;
  // the 32-bit depth sort takes an even number of passes: its result is in the first key/value buffers
  k_density_stats<<<(unsigned)((L.PV + 255) / 256), 256, 0, s>>>(L.PV, P, at<uint32_t>(w, L.key_a), at<uint32_t>(w, L.val_a),
                                                               at<uint32_t>(w, L.counts), at<float4>(w, L.records),
                                                               at<float>(w, L.radii), at<float>(w, L.accum), rs_max,
                                                               grad_accum, vis_count, angular);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

}  // extern "C"
