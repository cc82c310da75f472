// Host API basics, FoV masks (Sec. 3.1, Sec. D.1), HEALPix batch utilities,
// the tile radius rho(k, b) and the workspace layout of the rasterizer.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "hpx_math.cuh"
#include "internal.cuh"
#include "camera.cuh"

using namespace hpx;

namespace hpxgs {

// ----------------------------------------------------------------------------
// Instrumentation: one-shot stage timing with caller events; launch counter.
// ----------------------------------------------------------------------------
static std::mutex g_prof_mu;
static cudaEvent_t g_prof[HPXGS_NUM_STAGES][2];
static std::atomic<uint64_t> g_launches{0};

void note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// In stream capture a plain record only marks a dependency; the external flag
// makes it an event-record node that the graph performs at every replay.
static void prof_record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

void prof_begin(int stage, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof[stage][0]) prof_record(g_prof[stage][0], s);
}
void prof_end(int stage, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof[stage][1]) prof_record(g_prof[stage][1], s);
  g_prof[stage][0] = nullptr;
  g_prof[stage][1] = nullptr;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

// Helper streams, one per (device, caller stream), created on first use and kept for
// the life of the process. Creation switches this thread to the relaxed capture mode
// for its few calls, so that a first use inside a stream capture is allowed too.
namespace {
constexpr int kMaxForks = 32;
std::mutex g_fork_mu;
Fork g_forks[kMaxForks];
int g_fork_dev[kMaxForks];
int g_nforks = 0;
}  // namespace

const Fork* fork_of(cudaStream_t s) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_fork_mu);
  for (int i = 0; i < g_nforks; ++i)
    if (g_forks[i].origin == s && g_fork_dev[i] == dev) return &g_forks[i];
  if (g_nforks == kMaxForks) return nullptr;
  Fork f{s, nullptr, nullptr, nullptr, nullptr, nullptr, {nullptr, nullptr}};
  cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
  if (cudaThreadExchangeStreamCaptureMode(&mode) != cudaSuccess) return nullptr;
  int prio = 0, least = 0, greatest = 0;
  bool ok = cudaStreamGetPriority(s, &prio) == cudaSuccess &&
            cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&f.side, cudaStreamNonBlocking, prio) == cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&f.side_hi, cudaStreamNonBlocking, greatest) == cudaSuccess;
  cudaEvent_t* evs[5] = {&f.fork, &f.join, &f.join_hi, &f.mid[0], &f.mid[1]};
  for (cudaEvent_t* e : evs) ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    for (cudaEvent_t* e : evs)
      if (*e) cudaEventDestroy(*e);
    if (f.side_hi) cudaStreamDestroy(f.side_hi);
    if (f.side) cudaStreamDestroy(f.side);
  }
  cudaThreadExchangeStreamCaptureMode(&mode);
  if (!ok) { cudaGetLastError(); return nullptr; }
  g_forks[g_nforks] = f;
  g_fork_dev[g_nforks] = dev;
  return &g_forks[g_nforks++];
}

// FoV mask: camera_margin and pixel_in_mask live in camera.cuh.
// One thread per pixel; a warp's 32 consecutive NESTED pixels form one mask word.
// tile_flags (optional) gets bit 0 set for every tile with an in-mask pixel.
__global__ void k_mask(ViewParams vp, int b, uint32_t* __restrict__ words, uint32_t* __restrict__ tile_flags) {
  const uint32_t npix = 12u << (2 * vp.k);
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;   // npix is a multiple of 32
  if (p >= npix) return;
  bool in = pixel_in_mask(vp, p);
  uint32_t bits = __ballot_sync(0xffffffffu, in);
  if ((threadIdx.x & 31) == 0) {
    words[p >> 5] = bits;
    if (tile_flags && bits) atomicOr(&tile_flags[p >> (2 * b)], 1u);
  }
}

int launch_mask(const ViewParams& vp, int b, uint32_t* words, uint32_t* tile_flags, cudaStream_t s) {
  const uint32_t npix = 12u << (2 * vp.k);
  k_mask<<<(npix + 255) / 256, 256, 0, s>>>(vp, b, words, tile_flags);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

// ----------------------------------------------------------------------------
// rho(k, b): per tile, the smallest dot between the tile centre and its pixel
// centres (FP64), minimised over tiles with an atomic on the double's bits
// (all dots are positive, so the bit patterns order like the values).
// ----------------------------------------------------------------------------
__global__ void k_tile_mindot(int k, int b, unsigned long long* out) {
  const int kt = k - b;
  const uint32_t tile = blockIdx.x;
  const uint32_t per = 1u << (2 * b);
  double3 c = pix2vec_f64(kt, tile);
  double best = 2.0;
  for (uint32_t j = threadIdx.x; j < per; j += blockDim.x) {
    double3 p = pix2vec_f64(k, tile * per + j);
    double d = c.x * p.x + c.y * p.y + c.z * p.z;
    best = fmin(best, d);
  }
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  __shared__ double wmin[32];
  if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 2.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) m = fmin(m, wmin[w]);
    atomicMin(out, (unsigned long long)__double_as_longlong(m));
  }
}

static std::mutex g_rho_mu;
static std::map<std::pair<int, int>, double> g_rho;

static bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
  return st != cudaStreamCaptureStatusNone;
}

// Result word of k_tile_mindot. The computation runs once per (k, b) under
// g_rho_mu, so no two calls use the word at the same time.
static __device__ unsigned long long d_mindot;

// PixRad(o): per node, the largest angle from its centre to 36 boundary points (9 per
// edge, corners included), maximised over nodes with an atomic on the double's bits.
static std::mutex g_pixrad_mu;
static std::map<int, double> g_pixrad;
static __device__ unsigned long long d_maxang;

__global__ void k_pixrad_max(int o, unsigned long long* out) {
  const uint32_t nside = 1u << o, npix = 12u * nside * nside;
  const double iN = 1.0 / (double)nside;
  double mx = 0.0;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    const FaceXY c = nest_to_fxy(o, p);
    const double3 a = pix2vec_f64(o, p);
    for (int t = 0; t <= 8; ++t) {
      const double sft = t / 8.0;
      const double uu[4] = {c.x + sft, c.x + sft, (double)c.x, c.x + 1.0};
      const double vv[4] = {(double)c.y, c.y + 1.0, c.y + sft, c.y + sft};
      for (int e = 0; e < 4; ++e) {
        const double3 q = face_uv_vec_f64(c.f, uu[e] * iN, vv[e] * iN);
        const double cx = a.y * q.z - a.z * q.y, cy = a.z * q.x - a.x * q.z, cz = a.x * q.y - a.y * q.x;
        mx = fmax(mx, atan2(sqrt(cx * cx + cy * cy + cz * cz), a.x * q.x + a.y * q.y + a.z * q.z));
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

int pixrad(int o, double* out, cudaStream_t s) {
  if (o < 0 || o > 15) return HPXGS_E_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_pixrad_mu);
  auto it = g_pixrad.find(o);
  if (it != g_pixrad.end()) { *out = it->second; return HPXGS_OK; }
  if (stream_capturing(s)) return HPXGS_E_CAPTURE;
  unsigned long long* dptr = nullptr;
  HPXGS_CUDA_CHECK(cudaGetSymbolAddress((void**)&dptr, d_maxang));
  HPXGS_CUDA_CHECK(cudaMemsetAsync(dptr, 0, sizeof(unsigned long long), s));
  const long long npix = 12LL << (2 * o);
  const int grid = (int)std::min<long long>((npix + 255) / 256, 8LL * num_sms());
  k_pixrad_max<<<grid, 256, 0, s>>>(o, dptr);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  unsigned long long res = 0;
  HPXGS_CUDA_CHECK(cudaMemcpyAsync(&res, dptr, sizeof(res), cudaMemcpyDeviceToHost, s));
  HPXGS_CUDA_CHECK(cudaStreamSynchronize(s));
  double mx = 0;
  std::memcpy(&mx, &res, sizeof(mx));
  const double r = std::ceil(mx * 1048576.0) / 1048576.0;
  g_pixrad[o] = r;
  *out = r;
  return HPXGS_OK;
}

int tile_rho(int k, int b, double* rho, cudaStream_t s) {
  if (k < b || b < 0 || k > 13) return HPXGS_E_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_rho_mu);
  auto it = g_rho.find({k, b});
  if (it != g_rho.end()) { *rho = it->second; return HPXGS_OK; }
  if (stream_capturing(s)) return HPXGS_E_CAPTURE;
  const double two = 2.0;
  unsigned long long init = 0;
  std::memcpy(&init, &two, sizeof(init));
  unsigned long long* dptr = nullptr;
  HPXGS_CUDA_CHECK(cudaGetSymbolAddress((void**)&dptr, d_mindot));
  HPXGS_CUDA_CHECK(cudaMemcpyAsync(dptr, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  const int ntile = 12 << (2 * (k - b));
  const int per = 1 << (2 * b);
  k_tile_mindot<<<ntile, per < 256 ? (per < 32 ? 32 : per) : 256, 0, s>>>(k, b, dptr);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  unsigned long long res = 0;
  HPXGS_CUDA_CHECK(cudaMemcpyAsync(&res, dptr, sizeof(res), cudaMemcpyDeviceToHost, s));
  HPXGS_CUDA_CHECK(cudaStreamSynchronize(s));
  double mindot = 0;
  std::memcpy(&mindot, &res, sizeof(mindot));
  double r = std::acos(std::fmin(1.0, mindot));
  r = std::ceil(r * 1048576.0) / 1048576.0;
  g_rho[{k, b}] = r;
  *rho = r;
  return HPXGS_OK;
}

// ----------------------------------------------------------------------------
// View table and workspace layout
// ----------------------------------------------------------------------------
// Pinhole: FoV in (0, 180) and the principal point strictly inside the image; the
// other cameras have a centred principal point.
bool valid_camera(const hpxgs_camera& c) {
  const bool pp_in = std::fabs(c.ppx) < 1.f && std::fabs(c.ppy) < 1.f;   // false for NaN
  if (c.kind == HPXGS_CAM_PINHOLE)
    return c.fov_x_deg > 0 && c.fov_x_deg < 180 && c.fov_y_deg > 0 && c.fov_y_deg < 180 && pp_in;
  return c.ppx == 0.f && c.ppy == 0.f;
}

static bool valid_view(const hpxgs_view& v, int b) {
  if (v.nside_log2 < b || v.nside_log2 > 13) return false;
  if (v.cam.kind < 0 || v.cam.kind > 2) return false;
  if (!valid_camera(v.cam)) return false;
  if (v.cam.kind == HPXGS_CAM_FISHEYE &&
      !(v.cam.fov_x_deg > 0 && v.cam.fov_x_deg <= 360 && v.cam.fov_y_deg > 0 && v.cam.fov_y_deg <= 360))
    return false;
  for (int i = 0; i < 9; ++i) if (!std::isfinite(v.W[i])) return false;
  for (int i = 0; i < 3; ++i) if (!std::isfinite(v.b[i])) return false;
  return true;
}

static bool valid_ppt(int v) { return v == 0 || v == 1 || v == 2 || v == 4 || v == 8; }

static bool valid_cfg(const hpxgs_config* c) {
  return c && c->tile_level >= 3 && c->tile_level <= 5 && c->eps_T >= 0 && c->eps_T < 1 &&
         c->alpha_max > 0 && c->alpha_max < 1 && c->cutoff_m > 0 && c->near_plane >= 0 &&
         valid_ppt(c->fwd_ppt) && valid_ppt(c->bwd_ppt) && c->blocks_per_sm >= 0 && c->blocks_per_sm <= 64 &&
         (c->query == HPXGS_QUERY_RING || c->query == HPXGS_QUERY_NESTED) && c->query_log2f >= 0 &&
         c->query_log2f <= 3 && (c->blend_cull == 0 || c->blend_cull == 1) &&
         (c->blend_split == 0 || c->blend_split == 1);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int make_layout(int32_t P, const hpxgs_view* views, int nviews, const hpxgs_config* cfg, int64_t cap, Layout* L) {
  if (!valid_cfg(cfg) || !views || nviews < 1 || nviews > HPXGS_MAX_VIEWS || P < 0 || cap < 0 ||
      cap > 0xffffffffLL)
    return HPXGS_E_INVALID_ARG;
  const int b = cfg->tile_level;
  int64_t tiles = 0, pix = 0;
  for (int v = 0; v < nviews; ++v) {
    if (!valid_view(views[v], b)) return HPXGS_E_INVALID_ARG;
    tiles += 12LL << (2 * (views[v].nside_log2 - b));
    pix += 12LL << (2 * views[v].nside_log2);
  }
  const int64_t PV = (int64_t)P * nviews;
  if (PV >= 0xffffffffLL || tiles >= 0x7fffffffLL) return HPXGS_E_INVALID_ARG;
  L->P = P; L->PV = PV; L->cap = cap; L->total_tiles = tiles; L->total_pix = pix;
  const int G = std::min(2 * num_sms(), kMaxSortBlocks);
  L->sort_blocks = G;
  L->pair_sort_blocks = std::min(HPXGS_SORT_BPS * num_sms(), kMaxSortBlocks);
  int bits = 1;
  while ((1LL << bits) < tiles) ++bits;
  L->pair_bits = bits;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
  const size_t pv = (size_t)(PV > 0 ? PV : 1);
  const size_t cp = (size_t)(cap > 0 ? cap : 1);
  L->tile_flags = take(sizeof(uint32_t) * tiles);
  L->records = take(64 * pv);
  L->radii = take(4 * pv);
  L->stage = take(4 * pv);
  L->depth = take(4 * pv);
  L->key_a = take(4 * pv);
  L->key_b = take(4 * pv);
  L->val_a = take(4 * pv);
  L->val_b = take(4 * pv);
  L->counts = take(4 * pv);
  L->offsets = take(8 * (pv + 1));
  L->scan_part = take(8 * (G + 1));
  L->pair_key_a = take(4 * cp);
  L->pair_key_b = take(4 * cp);
  L->pair_val_a = take(4 * cp);
  L->pair_val_b = take(4 * cp);
  L->hist = take(4 * (256 * (size_t)kMaxSortBlocks + 256));   // per-block digit counts, then the digit bases
  L->ranges = take(8 * tiles);
  L->counters = take(4 * C_COUNT);
  L->accum = take(4 * HPXGS_NACC * pv);
  L->accum_d = take(4 * pv);                     // dL/d(1/r) of the inverse-depth channel
  L->unit_order = take(4 * 3 * 4 * (size_t)tiles);   // blend units: forward order, backward order, forward work
  L->total = o;
  return HPXGS_OK;
}

void camera_params(const hpxgs_camera& cam, int k, ViewParams& p) {
  p.k = k;
  p.kind = cam.kind;
  // u in [0, W] with x = (u - c_x) / f_x, c_x = (W/2)(1 + ppx), W / (2 f_x) = tan(fov_x / 2)
  const double tx = std::tan(0.5 * cam.fov_x_deg * kPi / 180.0), ty = std::tan(0.5 * cam.fov_y_deg * kPi / 180.0);
  p.xlo64 = -tx * (1.0 + (double)cam.ppx); p.xhi64 = tx * (1.0 - (double)cam.ppx);
  p.ylo64 = -ty * (1.0 + (double)cam.ppy); p.yhi64 = ty * (1.0 - (double)cam.ppy);
  p.wx64 = cam.fov_x_deg / 180.0;
  p.wy64 = cam.fov_y_deg / 180.0;
  p.xlo = (float)p.xlo64; p.xhi = (float)p.xhi64; p.ylo = (float)p.ylo64; p.yhi = (float)p.yhi64;
  p.wx = (float)p.wx64; p.wy = (float)p.wy64;
}

int make_table(const hpxgs_gaussians* g, int P, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
               cudaStream_t stream, bool need_rho, ViewTable* vt) {
  if (!valid_cfg(cfg) || !views || nviews < 1 || nviews > HPXGS_MAX_VIEWS) return HPXGS_E_INVALID_ARG;
  if (g && (g->sh_degree < 0 || g->sh_degree > 3 || g->P != P)) return HPXGS_E_INVALID_ARG;
  std::memset(vt, 0, sizeof(*vt));
  vt->nviews = nviews; vt->P = P; vt->b = cfg->tile_level;
  vt->sh_degree = g ? g->sh_degree : 0;
  vt->eps_T = cfg->eps_T; vt->alpha_max = cfg->alpha_max; vt->cutoff = cfg->cutoff_m;
  vt->near_plane = cfg->near_plane;
  for (int c = 0; c < 3; ++c) vt->bg[c] = cfg->bg[c];
  vt->write_outside = cfg->write_outside;
  int64_t tile_base = 0, pix_base = 0;
  for (int v = 0; v < nviews; ++v) {
    const hpxgs_view& hv = views[v];
    if (!valid_view(hv, cfg->tile_level)) return HPXGS_E_INVALID_ARG;
    ViewParams& p = vt->v[v];
    for (int i = 0; i < 9; ++i) p.W[i] = hv.W[i];
    for (int i = 0; i < 3; ++i) p.b[i] = hv.b[i];
    for (int j = 0; j < 3; ++j) p.cam[j] = -(hv.W[j] * hv.b[0] + hv.W[3 + j] * hv.b[1] + hv.W[6 + j] * hv.b[2]);
    camera_params(hv.cam, hv.nside_log2, p);
    const double omega_pix = 4.0 * kPi / (12.0 * std::ldexp(1.0, 2 * p.k));
    p.blur = cfg->blur_rad2 < 0 ? (float)(0.3 * omega_pix) : cfg->blur_rad2;
    p.ntiles = 12 << (2 * (p.k - cfg->tile_level));
    p.tile_base = (int)tile_base;
    p.pix_base = pix_base;
    p.rho = 0;
    p.rho32 = 0.f;
    p.rho_sub32 = 0.f;
    if (need_rho) {
      int rc = tile_rho(p.k, cfg->tile_level, &p.rho, stream);
      double rs = 0;
      if (rc == HPXGS_OK) rc = tile_rho(p.k, 2, &rs, stream);
      if (rc != HPXGS_OK) return rc;
      p.rho_sub32 = (float)rs;
    }
    // FoV cap: every in-mask pixel lies within psi_max of the optical axis (camera +z), an
    // active tile's centre within rho of one of them, and a listed tile's centre within
    // r_s + rho of the Gaussian, so a Gaussian farther than psi_max + 2 rho + r_s from
    // the axis has no listed tile and can be culled before sorting.
    double psi_max = -1.0;
    if (hv.cam.kind == HPXGS_CAM_PINHOLE) {
      const double ex = std::fmax(-p.xlo64, p.xhi64), ey = std::fmax(-p.ylo64, p.yhi64);   // farthest frustum corner
      psi_max = std::atan(std::sqrt(ex * ex + ey * ey));
    }
    else if (hv.cam.kind == HPXGS_CAM_FISHEYE) psi_max = 0.5 * kPi * std::fmax(p.wx64, p.wy64);
    p.rho32 = (float)p.rho;
    // the NESTED query lists a tile from a node within r_s + PixRad(k_max) of the
    // Gaussian, the node lies within PixRad(k_t) of the tile centre, and an in-mask
    // pixel within rho of it: the cap grows by those radii instead of 2 rho
    double reach = 2.0 * p.rho;
    p.rhoq = 0.0; p.rhoq32 = 0.f; p.rhoc32 = 0.f;
    if (need_rho && cfg->query == HPXGS_QUERY_RING && cfg->query_log2f > 0) {
      // a tile is listed from a query pixel within r_s + rho_q of the Gaussian whose centre
      // lies within rho_c of the tile centre (at log2f = b the query pixels are the render
      // pixels, rho_q = 0 exactly)
      const int L = cfg->query_log2f, kt = p.k - cfg->tile_level;
      double rc = 0;
      int rc2 = L == cfg->tile_level ? HPXGS_OK : tile_rho(p.k, cfg->tile_level - L, &p.rhoq, stream);
      if (rc2 == HPXGS_OK) rc2 = tile_rho(kt + L, L, &rc, stream);
      if (rc2 != HPXGS_OK) return rc2;
      p.rhoq32 = (float)p.rhoq;
      p.rhoc32 = (float)rc;
      reach = p.rho + rc + p.rhoq;
    }
    if (need_rho && cfg->query == HPXGS_QUERY_NESTED) {
      double a = 0, c = 0;
      const int kt = p.k - cfg->tile_level;
      int rc2 = pixrad(kt, &a, stream);
      if (rc2 == HPXGS_OK) rc2 = pixrad(kt + cfg->query_log2f, &c, stream);
      if (rc2 != HPXGS_OK) return rc2;
      reach = p.rho + a + c;
    }
    const double cull = psi_max + reach + 1e-5;
    p.fov_cull = (need_rho && psi_max >= 0.0 && cull < kPi) ? (float)cull : -1.0f;
    tile_base += p.ntiles;
    pix_base += 12LL << (2 * p.k);
  }
  vt->total_tiles = (int)tile_base;
  vt->total_pix = pix_base;
  vt->query = cfg->query;
  vt->log2f = cfg->query_log2f;
  vt->cull = cfg->blend_cull;
  for (int o = 0; o < 16; ++o) { vt->pixrad32[o] = 0.f; vt->pixrad64[o] = 0.0; }
  if (need_rho && cfg->query == HPXGS_QUERY_NESTED) {
    int omax = 0;
    for (int v = 0; v < nviews; ++v) omax = std::max(omax, views[v].nside_log2 - cfg->tile_level + cfg->query_log2f);
    if (omax > 11) return HPXGS_E_INVALID_ARG;              // the quadtree search stops at order 11
    for (int o = 0; o <= omax; ++o) {
      int rc2 = pixrad(o, &vt->pixrad64[o], stream);
      if (rc2 != HPXGS_OK) return rc2;
      vt->pixrad32[o] = (float)vt->pixrad64[o];
    }
  }
  return HPXGS_OK;
}

// ----------------------------------------------------------------------------
// HEALPix batch utilities
// ----------------------------------------------------------------------------
__global__ void k_pix2vec(int k, const int64_t* pix, int64_t n, float* v32, double* v64) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t p = (uint32_t)pix[i];
  if (v32) { float3 a = pix2vec_f32(k, p); v32[3 * i] = a.x; v32[3 * i + 1] = a.y; v32[3 * i + 2] = a.z; }
  if (v64) { double3 a = pix2vec_f64(k, p); v64[3 * i] = a.x; v64[3 * i + 1] = a.y; v64[3 * i + 2] = a.z; }
}
__global__ void k_vec2pix(int k, const double* v, int64_t n, int64_t* pix) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  pix[i] = vec2pix_f64(k, make_double3(v[3 * i], v[3 * i + 1], v[3 * i + 2]));
}
// Angles of a direction: colatitude theta = atan2(sqrt(x^2 + y^2), z), longitude
// phi = atan2(y, x) in [0, 2 pi) (HEALPix frame).
__global__ void k_pix2ang(int k, const int64_t* pix, int64_t n, double* theta, double* phi) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double3 a = pix2vec_f64(k, (uint32_t)pix[i]);
  theta[i] = atan2(sqrt(a.x * a.x + a.y * a.y), a.z);
  double ph = atan2(a.y, a.x);
  phi[i] = ph < 0.0 ? ph + 2.0 * kPi : ph;
}
__global__ void k_ang2pix(int k, const double* theta, const double* phi, int64_t n, int64_t* pix) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double st, ct, sp, cp;
  sincos(theta[i], &st, &ct);
  sincos(phi[i], &sp, &cp);
  pix[i] = vec2pix_f64(k, make_double3(st * cp, st * sp, ct));
}
__global__ void k_nest2ring(int k, const int64_t* in, int64_t n, int64_t* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = nest2ring(k, (uint32_t)in[i]);
}
__global__ void k_ring2nest(int k, const int64_t* in, int64_t n, int64_t* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = ring2nest(k, in[i]);
}
__global__ void k_neighbours(int k, const int64_t* in, int64_t n, int64_t* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  FaceXY c = nest_to_fxy(k, (uint32_t)in[i]);
  int s = 0;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy) {
      if (dx == 0 && dy == 0) continue;
      out[8 * i + (s++)] = neighbour_nest(k, c.f, c.x, c.y, dx, dy);
    }
}

static int grid_for(int64_t n) { return (int)((n + 255) / 256); }

}  // namespace hpxgs

using namespace hpxgs;

extern "C" {

const char* hpxgs_strerror(int code) {
  switch (code) {
    case HPXGS_OK: return "ok";
    case HPXGS_E_INVALID_ARG: return "invalid argument";
    case HPXGS_E_CAPACITY: return "pair capacity exceeded";
    case HPXGS_E_TIMEOUT: return "bounded device wait timed out";
    case HPXGS_E_CUDA: return "CUDA error";
    case HPXGS_E_UNIMPLEMENTED: return "not implemented";
    case HPXGS_E_WORKSPACE: return "workspace too small";
    case HPXGS_E_CAPTURE: return "call needs a host synchronisation inside stream capture";
    default: return "unknown status";
  }
}

int hpxgs_status_error(int32_t flags) {
  if (flags & HPXGS_F_CAPACITY) return HPXGS_E_CAPACITY;
  if (flags & HPXGS_F_TIMEOUT) return HPXGS_E_TIMEOUT;
  return HPXGS_OK;
}

void hpxgs_config_default(hpxgs_config* c) {
  if (!c) return;
  c->tile_level = 4;
  c->eps_T = 1e-4f;
  c->alpha_max = 0.99f;
  c->cutoff_m = 9.0f;
  c->blur_rad2 = -1.0f;
  c->near_plane = 0.2f;
  c->bg[0] = c->bg[1] = c->bg[2] = 0.0f;
  c->lambda_ssim = 0.2f;
  c->write_outside = 1;
  c->fwd_ppt = 0;
  c->bwd_ppt = 0;
  c->blocks_per_sm = 0;
  c->query = HPXGS_QUERY_RING;
  c->query_log2f = 0;
  c->blend_cull = 1;
  c->blend_split = 1;
}

int hpxgs_nside_for_image(int kind, double W, double H, double fovx, double fovy, double* nstar, int* k,
                          int* kL, int* kH) {
  if (!(W > 0 && H > 0)) return HPXGS_E_INVALID_ARG;
  const double hx = 0.5 * fovx * kPi / 180.0, hy = 0.5 * fovy * kPi / 180.0;
  double om;
  if (kind == HPXGS_CAM_FULL) om = 4.0 * kPi;
  else if (kind == HPXGS_CAM_FISHEYE) om = 2.0 * kPi * (1.0 - std::cos(hx));
  else if (kind == HPXGS_CAM_PINHOLE) om = 4.0 * std::asin(std::sin(hx) * std::sin(hy));
  else return HPXGS_E_INVALID_ARG;
  if (!(om > 0)) return HPXGS_E_INVALID_ARG;
  const double ns = std::sqrt(4.0 * kPi * W * H / (12.0 * om));
  const double l2 = std::log2(ns);
  if (nstar) *nstar = ns;
  if (k) *k = (int)std::lround(l2);
  if (kL) *kL = (int)std::floor(l2);
  if (kH) *kH = (int)std::ceil(l2);
  return HPXGS_OK;
}

int hpxgs_profile_arm(int stage, void* start_event, void* stop_event) {
  if (stage < 0 || stage >= HPXGS_NUM_STAGES) return HPXGS_E_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof[stage][0] = (cudaEvent_t)start_event;
  g_prof[stage][1] = (cudaEvent_t)stop_event;
  return HPXGS_OK;
}

int hpxgs_profile_armed(int stage) {
  if (stage < 0 || stage >= HPXGS_NUM_STAGES) return HPXGS_E_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return (g_prof[stage][0] || g_prof[stage][1]) ? 1 : 0;
}

uint64_t hpxgs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int hpxgs_pixrad(int o, double* out, hpxgs_stream_t stream) {
  if (!out) return HPXGS_E_INVALID_ARG;
  return pixrad(o, out, (cudaStream_t)stream);
}

int hpxgs_tile_rho(int k, int b, double* rho, hpxgs_stream_t stream) {
  if (!rho) return HPXGS_E_INVALID_ARG;
  return tile_rho(k, b, rho, (cudaStream_t)stream);
}

int hpxgs_prepare(const hpxgs_view* views, int nviews, const hpxgs_config* cfg, hpxgs_stream_t stream) {
  ViewTable* vt = new ViewTable;
  int rc = make_table(nullptr, 0, views, nviews, cfg, (cudaStream_t)stream, true, vt);
  delete vt;
  return rc;
}

int hpxgs_mask_build(const hpxgs_view* view, const hpxgs_config* cfg, uint32_t* mask_bits, hpxgs_stream_t stream) {
  if (!view || !mask_bits) return HPXGS_E_INVALID_ARG;
  ViewTable* vt = new ViewTable;
  int rc = make_table(nullptr, 0, view, 1, cfg, (cudaStream_t)stream, false, vt);
  if (rc == HPXGS_OK) rc = launch_mask(vt->v[0], cfg->tile_level, mask_bits, nullptr, (cudaStream_t)stream);
  delete vt;
  return rc;
}

int hpxgs_pix2vec_nest(int k, const int64_t* pix, int64_t n, float* v32, double* v64, hpxgs_stream_t s) {
  if (k < 0 || k > 13 || n < 0 || (n > 0 && !pix)) return HPXGS_E_INVALID_ARG;
  if (n == 0) return HPXGS_OK;
  k_pix2vec<<<grid_for(n), 256, 0, (cudaStream_t)s>>>(k, pix, n, v32, v64);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}
int hpxgs_vec2pix_nest(int k, const double* v, int64_t n, int64_t* pix, hpxgs_stream_t s) {
  if (k < 0 || k > 13 || n < 0 || (n > 0 && (!v || !pix))) return HPXGS_E_INVALID_ARG;
  if (n == 0) return HPXGS_OK;
  k_vec2pix<<<grid_for(n), 256, 0, (cudaStream_t)s>>>(k, v, n, pix);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}
int hpxgs_pix2ang_nest(int k, const int64_t* pix, int64_t n, double* theta, double* phi, hpxgs_stream_t s) {
  if (k < 0 || k > 13 || n < 0 || (n > 0 && (!pix || !theta || !phi))) return HPXGS_E_INVALID_ARG;
  if (n == 0) return HPXGS_OK;
  k_pix2ang<<<grid_for(n), 256, 0, (cudaStream_t)s>>>(k, pix, n, theta, phi);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}
int hpxgs_ang2pix_nest(int k, const double* theta, const double* phi, int64_t n, int64_t* pix, hpxgs_stream_t s) {
  if (k < 0 || k > 13 || n < 0 || (n > 0 && (!theta || !phi || !pix))) return HPXGS_E_INVALID_ARG;
  if (n == 0) return HPXGS_OK;
  k_ang2pix<<<grid_for(n), 256, 0, (cudaStream_t)s>>>(k, theta, phi, n, pix);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}
int hpxgs_nest2ring(int k, const int64_t* in, int64_t n, int64_t* out, hpxgs_stream_t s) {
  if (k < 0 || k > 13 || n < 0 || (n > 0 && (!in || !out))) return HPXGS_E_INVALID_ARG;
  if (n == 0) return HPXGS_OK;
  k_nest2ring<<<grid_for(n), 256, 0, (cudaStream_t)s>>>(k, in, n, out);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}
int hpxgs_ring2nest(int k, const int64_t* in, int64_t n, int64_t* out, hpxgs_stream_t s) {
  if (k < 0 || k > 13 || n < 0 || (n > 0 && (!in || !out))) return HPXGS_E_INVALID_ARG;
  if (n == 0) return HPXGS_OK;
  k_ring2nest<<<grid_for(n), 256, 0, (cudaStream_t)s>>>(k, in, n, out);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}
int hpxgs_neighbours_nest(int k, const int64_t* in, int64_t n, int64_t* out, hpxgs_stream_t s) {
  if (k < 1 || k > 13 || n < 0 || (n > 0 && (!in || !out))) return HPXGS_E_INVALID_ARG;
  if (n == 0) return HPXGS_OK;
  k_neighbours<<<grid_for(n), 256, 0, (cudaStream_t)s>>>(k, in, n, out);
  note_launches(1);
  HPXGS_LAUNCH_CHECK();
  return HPXGS_OK;
}

}  // extern "C"
