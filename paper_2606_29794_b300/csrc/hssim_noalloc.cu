// HEALPix-SSIM + L1 loss value without a caller workspace.
//
// Some callers cannot hand the library device memory: a plugin running inside a
// host application that owns the whole GPU memory budget, or a real-time loop
// that forbids allocation once it has started. hpxgs_hssim_loss_noalloc serves
// them. It returns the {loss, HSSIM, L1} value (no gradient coefficients) and
// keeps its per-block partial sums in a fixed array that lives in this library's
// device image instead of in a workspace.
//
//  - Per pixel it evaluates h_q and |I - G| with the functions the workspace
//    kernels use (hssim_window.cuh); only the block sums differ (FP64 here,
//    compensated FP32 there), so the two entry points agree within 2e-6.
//  - Limit: HEALPix order k <= 10 (Nside <= 1024). The array holds one partial
//    triple per 256-pixel block at that size: 49,152 x 3 doubles = 1.18 MB, and
//    every GPU that loads the library keeps it until the process exits.
//  - Host code cannot use the array's name as a device address. The first call on
//    a device looks the address up (cudaGetSymbolAddress, with that device
//    current); that first call, and the first after a cudaDeviceReset (which
//    discards the module), must come before any stream capture. Calls outside
//    capture look it up again and refresh a per-device cache; a capturing stream
//    on a device without a cached address gets HPXGS_E_CAPTURE.
//  - Every call writes all the partials it later reads, so nothing needs
//    clearing, but all calls share the one array: calls that overlap on the GPU
//    (different streams without ordering between them) race and give wrong values.
#include <mutex>

#include "hpx_math.cuh"
#include "hssim_window.cuh"
#include "internal.cuh"

using namespace hpx;

namespace hpxgs {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxOrder = 10;
constexpr int kNaMaxBlocks = (12 << (2 * kNaMaxOrder)) / kNaThreads;   // 49,152
static __device__ __align__(256) double g_partials[3 * kNaMaxBlocks];

// Per 256-pixel block: sum of h_q, sum of |I - G| and the number of in-mask pixels.
__global__ void __launch_bounds__(kNaThreads) k_value_partials(int k, const float* __restrict__ I,
                                                               const float* __restrict__ Gt,
                                                               const uint32_t* __restrict__ mask,
                                                               double* __restrict__ part) {
  const uint32_t npix = 12u << (2 * k);
  const uint32_t p = blockIdx.x * kNaThreads + threadIdx.x;
  double h = 0.0, l1 = 0.0, cnt = 0.0;
  if (p < npix && mask_bit(mask, p)) {
    HWindow W;
    hssim_window(k, p, mask, W);
    float hq, l1q;
    hssim_pixel_value(W, p, I, Gt, hq, l1q);
    h = hq;
    l1 = l1q;
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

// Address of g_partials on the current device. Outside stream capture it is looked up
// on every call (so a module reloaded after cudaDeviceReset is seen) and cached; while
// `s` is capturing only the cache is used, and a device with no cached address fails.
int partials_address(cudaStream_t s, double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return HPXGS_E_CUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return HPXGS_E_CUDA;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return HPXGS_E_CUDA;
    g_addr[dev] = static_cast<double*>(p);
  } else if (!g_addr[dev]) {
    return HPXGS_E_CAPTURE;
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
  cudaStream_t s = (cudaStream_t)stream;
  double* part = nullptr;
  int rc = partials_address(s, &part);
  if (rc != HPXGS_OK) return rc;
  const uint32_t npix = 12u << (2 * k);
  const int nblocks = (int)(npix / kNaThreads);
  k_value_partials<<<nblocks, kNaThreads, 0, s>>>(k, I, G, mask_bits, part);
  k_value_reduce<<<1, 256, 0, s>>>(part, nblocks, lambda, out3);
  note_launches(2);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}
