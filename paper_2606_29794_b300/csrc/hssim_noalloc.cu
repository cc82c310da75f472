// HEALPix-SSIM + L1 loss value without a caller workspace.
//
// Some callers cannot hand the library device memory: a plugin running inside a
// host application that owns the whole GPU memory budget, or a real-time loop
// that forbids allocation once it has started. hpxgs_hssim_loss_noalloc serves
// them. It computes the same {loss, HSSIM, L1} as hpxgs_hssim_forward, but only
// the value (no gradient coefficients), and keeps its per-block partial sums in
// a fixed array that lives in this library's device image instead of in a
// workspace.
//
//  - Limit: HEALPix order k <= 10 (Nside <= 1024). The array holds one partial
//    triple per 256-pixel block at that size: 49,152 x 3 doubles = 1.18 MB, and
//    every GPU that loads the library keeps it until the process exits.
//  - The array's address is looked up once per device (cudaGetSymbolAddress,
//    with that device current) on the first call made on that device; make that
//    first call before capturing a stream into a CUDA graph.
//  - Every call writes all the partials it later reads, so nothing needs
//    clearing, but all calls share the one array: calls that overlap on the GPU
//    (different streams without ordering between them) race and give wrong values.
#include <mutex>

#include "hpx_math.cuh"
#include "internal.cuh"

using namespace hpx;

namespace hpxgs {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxOrder = 10;
constexpr int kNaMaxBlocks = (12 << (2 * kNaMaxOrder)) / kNaThreads;   // 49,152
constexpr float kNaC1 = 1e-4f, kNaC2 = 9e-4f;

static __device__ __align__(256) double g_partials[3 * kNaMaxBlocks];

__device__ __forceinline__ bool bit_of(const uint32_t* m, uint32_t p) { return (m[p >> 5] >> (p & 31)) & 1u; }

__device__ __forceinline__ float neighbour_weight(float3 a, float3 b, float inv2sig2) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float th = 2.f * asinf(fminf(1.f, 0.5f * sqrtf(dx * dx + dy * dy + dz * dz)));
  return __expf(-th * th * inv2sig2);
}

// Per 256-pixel block: sum of h_q, sum of |I - G| and the number of in-mask pixels.
__global__ void __launch_bounds__(kNaThreads) k_value_partials(int k, const float* __restrict__ I,
                                                               const float* __restrict__ Gt,
                                                               const uint32_t* __restrict__ mask,
                                                               double* __restrict__ part) {
  const uint32_t npix = 12u << (2 * k);
  const uint32_t p = blockIdx.x * kNaThreads + threadIdx.x;
  double h = 0.0, l1 = 0.0, cnt = 0.0;
  if (p < npix && bit_of(mask, p)) {
    const float inv2sig2 = 1.f / (2.f * 2.25f * (4.f * (float)kPi / (float)npix));
    const float3 cq = pix2vec_f32(k, p);
    const FaceXY c = nest_to_fxy(k, p);
    uint32_t idx[9];
    float w[9];
    int n = 0;
    idx[n] = p; w[n] = 1.f; ++n;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy) {
        if (dx == 0 && dy == 0) continue;
        const int64_t nb = neighbour_nest(k, c.f, c.x, c.y, dx, dy);
        if (nb < 0 || !bit_of(mask, (uint32_t)nb)) continue;
        idx[n] = (uint32_t)nb;
        w[n] = neighbour_weight(cq, pix2vec_f32(k, (uint32_t)nb), inv2sig2);
        ++n;
      }
    float Z = 0.f;
    for (int j = 0; j < n; ++j) Z += w[j];
    const float iZ = 1.f / Z;
    float hs = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
      float mx = 0.f, my = 0.f, xx = 0.f, yy = 0.f, xy = 0.f;
      for (int j = 0; j < n; ++j) {
        const float wj = w[j] * iZ;
        const float x = I[3 * (size_t)idx[j] + ch], y = Gt[3 * (size_t)idx[j] + ch];
        mx += wj * x; my += wj * y; xx += wj * x * x; yy += wj * y * y; xy += wj * x * y;
      }
      const float vx = xx - mx * mx, vy = yy - my * my, cxy = xy - mx * my;
      hs += ((2.f * mx * my + kNaC1) * (2.f * cxy + kNaC2)) / ((mx * mx + my * my + kNaC1) * (vx + vy + kNaC2));
      l1 += fabsf(I[3 * (size_t)p + ch] - Gt[3 * (size_t)p + ch]);
    }
    h = hs / 3.f;
    cnt = 1.0;
  }
  __shared__ double sh[3][kNaThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    h += __shfl_xor_sync(0xffffffffu, h, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[0][warp] = h; sh[1][warp] = l1; sh[2][warp] = cnt; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, cc = 0;
    for (int w2 = 0; w2 < kNaThreads / 32; ++w2) { a += sh[0][w2]; b += sh[1][w2]; cc += sh[2][w2]; }
    part[3 * blockIdx.x + 0] = a; part[3 * blockIdx.x + 1] = b; part[3 * blockIdx.x + 2] = cc;
  }
}

__global__ void k_value_reduce(const double* __restrict__ part, int nblocks, float lambda, float* out3) {
  __shared__ double s[3][256];
  double a = 0, b = 0, c = 0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) { a += part[3 * i]; b += part[3 * i + 1]; c += part[3 * i + 2]; }
  s[0][threadIdx.x] = a; s[1][threadIdx.x] = b; s[2][threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) for (int r = 0; r < 3; ++r) s[r][threadIdx.x] += s[r][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nm = s[2][0];
    const double hssim = nm > 0 ? s[0][0] / nm : 0.0;
    const double l1 = nm > 0 ? s[1][0] / (3.0 * nm) : 0.0;
    out3[0] = (float)((1.0 - lambda) * l1 + lambda * (1.0 - hssim));
    out3[1] = (float)hssim;
    out3[2] = (float)l1;
  }
}

std::mutex g_addr_mu;
double* g_addr[256];          // device address of g_partials, per device ordinal

int partials_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return HPXGS_E_CUDA;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return HPXGS_E_CUDA;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return HPXGS_OK;
}

}  // namespace
}  // namespace hpxgs

using namespace hpxgs;

extern "C" int hpxgs_hssim_loss_noalloc(const float* I, const float* G, const uint32_t* mask_bits, int k, float lambda,
                                        float* out3, hpxgs_stream_t stream) {
  if (k < 3 || k > kNaMaxOrder || !I || !G || !mask_bits || !out3 || !(lambda >= 0.f && lambda <= 1.f))
    return HPXGS_E_INVALID_ARG;
  double* part = nullptr;
  int rc = partials_address(&part);
  if (rc != HPXGS_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t npix = 12u << (2 * k);
  const int nblocks = (int)(npix / kNaThreads);
  k_value_partials<<<nblocks, kNaThreads, 0, s>>>(k, I, G, mask_bits, part);
  k_value_reduce<<<1, 256, 0, s>>>(part, nblocks, lambda, out3);
  note_launches(2);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}
