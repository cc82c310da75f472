// Shared host/device definitions of the rasterizer library (not part of the ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hpxgs.h"

namespace hpxgs {

// Per-view constants, passed to kernels by value (kernel parameter space).
struct ViewParams {
  float W[9];          // world -> camera rotation
  float b[3];
  float cam[3];        // camera centre -W^T b (world)
  int k;               // HEALPix order of the view
  int kind;            // HPXGS_CAM_*
  float xlo, xhi, ylo, yhi;   // pinhole frustum: xlo <= d_x / d_z <= xhi, ylo <= d_y / d_z <= yhi
  float wx, wy;        // fisheye fov / 180 deg
  double xlo64, xhi64, ylo64, yhi64, wx64, wy64;
  double rho;          // tile rho(k, b)
  float rho32;         // (float) rho, so kernels need no FP64 conversion
  float fov_cull;      // Gaussians farther than fov_cull + r_s from the optical axis have no listed tile (< 0: none)
  float blur;          // isotropic Sigma_arc term
  int ntiles;          // 12 * 4^(k-b)
  int64_t pix_base;    // first pixel of this view in packed outputs
  int tile_base;       // first global tile id of this view
  float rho_sub32;     // rho(k, 2): 4 x 4 sub-tile centre to pixel bound (the blend's cull)
  // RING query at search order k_t + log2f (log2f > 0): rho_q = rho(k, b - log2f), the
  // query-pixel centre to render-pixel bound of the membership test, and rho_c =
  // rho(k_t + log2f, log2f), the tile centre to query-pixel centre bound
  double rhoq;
  float rhoq32, rhoc32;
};

struct ViewTable {
  int nviews;
  int P;
  int b;               // tile level
  int sh_degree;
  float eps_T, alpha_max, cutoff, near_plane;
  float bg[3];
  int write_outside;
  int total_tiles;
  int query;           // HPXGS_QUERY_*
  int log2f;           // refinement of the tile query below the tile order (RING: search order k_t + log2f)
  int cull;            // 1: the blends' per-(entry, 32-pixel group) cull is on
  float pixrad32[16];  // NESTED query: PixRad(o), o = 0 .. deepest order used
  double pixrad64[16];
  int64_t total_pix;
  ViewParams v[HPXGS_MAX_VIEWS];
};

// Inputs of the per-pixel L1 + HSSIM gradient of each view, read by the backward
// blend of hpxgs_backward_hssim in place of a dL/dI map (kernel parameter space).
struct LossView {
  const float* I;          // rendered maps of the view [npix, 3]
  const float* G;          // targets [npix, 3]
  const uint32_t* idx;     // window table neighbours [8][npix] by walk direction
  const float* e;          // window table weights [8][npix] by walk direction
  const float* coef;       // per-window gradient coefficients [npix, 9] (HSSIM forward)
  const float* nm;         // float in-mask count (HSSIM forward)
  const float* dloss;      // dL/dloss of the view, or null for 1
  uint32_t npix;
};
struct LossViews {
  float lambda;
  LossView v[HPXGS_MAX_VIEWS];
};
struct NoLossViews { float lambda; };

// One record per (view, Gaussian): 4 x float4 = 64 bytes.
//   r0 = (g.x, g.y, g.z, opacity)     g: unit direction of the centre, HEALPix frame
//   r1 = (e1.x, e1.y, e1.z, conic_a)  e1: east tangent (increasing longitude)
//   r2 = (e2.x, e2.y, e2.z, conic_b)  e2: north tangent
//   r3 = (col.r, col.g, col.b, conic_c)
// m = conic_a d1^2 + 2 conic_b d1 d2 + conic_c d2^2 in the (e1, e2) frame.
constexpr int kRecFloat4 = 4;

// Workspace layout of hpxgs_forward / hpxgs_backward. All offsets 256-aligned.
struct Layout {
  size_t tile_flags, records, radii, stage, depth, key_a, key_b, val_a, val_b, counts, offsets, scan_part,
         pair_key_a, pair_key_b, pair_val_a, pair_val_b, hist, ranges, counters, accum, accum_d, unit_order,
         total;
  int64_t P, PV, cap, total_tiles, total_pix;
  int sort_blocks;        // grid of the count scan
  int pair_sort_blocks;   // grid of the pair sort
  int pair_bits;
};

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                     // items per thread per tile
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kMaxSortBlocks = 1024;
// Blocks per SM of the pair sort's fixed grid, and 4096-element tiles per block of
// the depth sort's grid (build-time tunables; both grids stay within kMaxSortBlocks).
#ifndef HPXGS_SORT_BPS
#define HPXGS_SORT_BPS 3
#endif
#ifndef HPXGS_DSORT_TPB
#define HPXGS_DSORT_TPB 1
#endif

// counters block (u32 each)
// (u64 counters live at u32 index 8 (n_eval) and 10 (n_contrib), 8-byte aligned)
// C_GRID_BAR_SCAN: arrivals at the grid barrier of the count scan's cooperative launch.
// C_WORK_BWD, then C_UNITS_BWD: the backward blend's unit counter and its longest-first
// order's class counts and cursors (zeroed together by the backward); C_UNITS_FWD: the
// same for the forward blend (zeroed with the rest by the forward).
constexpr int kUnitClasses = 129;
enum Counter { C_NPAIRS = 0, C_WORK_FWD = 1, C_NSORT = 3, C_NPAIRS_HI = 4, C_STAGE = 5, C_NEVAL = 8, C_NCONTRIB = 10, C_SORT_TICKET = 12,
               C_GRID_BAR_SCAN = 13, C_WORK_BWD = 16, C_UNITS_BWD = 17, C_UNITS_FWD = C_UNITS_BWD + 2 * kUnitClasses,
               C_COUNT = C_UNITS_FWD + 2 * kUnitClasses };

#ifdef __CUDACC__
// Grid-wide barrier of a cooperative launch (every block resident at once). Each block
// adds one arrival to *count (zero before the launch) and waits until the count reaches
// `target`, the barrier's number (1, 2, ...) times the grid size. Writes before the
// barrier are released by a fence, reads after it acquire. The wait is bounded: a block
// that waited limit_ns sets HPXGS_F_TIMEOUT in *status (when given) and gets false; the
// kernel must then return. A block that gave up arrives at no later barrier, so the
// other blocks give up too, each within its own limit.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool grid_barrier(uint32_t* count, uint32_t target, uint64_t limit_ns, int32_t* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    const uint64_t t0 = global_ns();
    int ok = 1;
    for (;;) {
      uint32_t c;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(count) : "memory");
      if (c >= target) break;
      if (global_ns() - t0 > limit_ns) {
        ok = 0;
        if (status) atomicOr(status, HPXGS_F_TIMEOUT);
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}
#endif

// instrumentation (geometry.cu)
void prof_begin(int stage, cudaStream_t s);
void prof_end(int stage, cudaStream_t s);
void note_launches(int n);

int make_layout(int32_t P, const hpxgs_view* views, int nviews, const hpxgs_config* cfg, int64_t cap, Layout* L);
// PixRad(o) of the NESTED query: the largest angle from a node centre to its
// boundary at order o (9 samples per edge), rounded up to 2^-20; cached per order.
// The first call for an order synchronises the stream (HPXGS_E_CAPTURE in capture).
int pixrad(int o, double* out, cudaStream_t s);
// Camera fields of a view (k, kind, tan(FoV/2) and FoV/180 deg in FP32 and FP64).
void camera_params(const hpxgs_camera& cam, int k, ViewParams& p);
bool valid_camera(const hpxgs_camera& cam);
int make_table(const hpxgs_gaussians* g, int P, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
               cudaStream_t stream, bool need_rho, ViewTable* vt);
int num_sms();
void hssim_bind(int k, const void* table, const void* ws, LossView* out);
// Helper streams for work that does not depend on what precedes it on `origin`:
// record `fork` on origin, make a helper wait for it, launch there, record an event
// on the helper and make origin wait for it (in stream capture this forks and joins
// the graph). `side` has origin's priority, `side_hi` the device's highest, for short
// latency-bound chains that must not wait behind a grid filling the GPU. Null when
// none can be made; the caller then runs that work on origin.
struct Fork {
  cudaStream_t origin, side, side_hi;
  cudaEvent_t fork, join, join_hi, mid[2];   // mid: two more events for a caller's intermediate joins
};
const Fork* fork_of(cudaStream_t origin);

}  // namespace hpxgs

#define HPXGS_CUDA_CHECK(expr)                                   \
  do {                                                           \
    cudaError_t err__ = (expr);                                  \
    if (err__ != cudaSuccess) return HPXGS_E_CUDA;               \
  } while (0)

#define HPXGS_LAUNCH_CHECK()                                     \
  do {                                                           \
    cudaError_t err__ = cudaGetLastError();                      \
    if (err__ != cudaSuccess) return HPXGS_E_CUDA;               \
  } while (0)
