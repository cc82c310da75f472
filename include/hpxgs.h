/*
 * hpxgs.h -- C ABI of the B300 HEALPix spherical Gaussian rasterizer
 * (UniTriSplat, arXiv 2606.29794).
 *
 * The library splats 3D Gaussians onto a NESTED HEALPix grid attached to a
 * camera (Sec. 3.1), composites them front to back per pixel (Sec. 3.4,
 * Algorithm 1), differentiates the result (Sec. 3.2) and evaluates the
 * HEALPix-SSIM + L1 training loss (Sec. 4.1).
 *
 * Conventions shared by every call
 *  - Device pointers are owned by the caller. The library never allocates
 *    device memory: callers size a workspace with the *_workspace_size query
 *    and pass it in. All calls are asynchronous on the given CUDA stream,
 *    except where a comment says the call synchronises.
 *  - Every call returns an int status (HPXGS_OK or a negative HPXGS_E_*).
 *    Argument errors are detected on the host before anything is launched.
 *    Conditions that only the device can see (pair-buffer overflow, a
 *    bounded wait that ran out) are OR-ed as HPXGS_F_* flags into the
 *    caller's device int32 `status`; read it after synchronising the stream
 *    and map it with hpxgs_status_error(). No call synchronises in secret.
 *  - Maps are float32 [Npix, 3] in NESTED order, Npix = 12 * 4^k for
 *    nside_log2 = k. Several views are packed back to back in one buffer,
 *    view v starting at pixel sum_{u<v} Npix(u) ("pixel base").
 *  - Camera frame: t = W mu + b (Sec. 3.2); camera direction d maps to the
 *    HEALPix unit vector (X, Y, Z) = (d_z, d_x, d_y), i.e. HEALPix longitude
 *    = omega = atan2(t_x, t_z) and colatitude = pi/2 - phi (Eq. 1).
 *  - C linkage, POD structs, no exceptions across the ABI.
 */
#ifndef HPXGS_H_
#define HPXGS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* hpxgs_stream_t; /* a cudaStream_t (0 = legacy default stream) */

/* ---- status codes (return values) ---- */
#define HPXGS_OK 0
#define HPXGS_E_INVALID_ARG -1   /* bad pointer, size, order, camera or config */
#define HPXGS_E_CAPACITY -2      /* pair buffer too small (see HPXGS_F_CAPACITY) */
#define HPXGS_E_TIMEOUT -3       /* a bounded device wait ran out */
#define HPXGS_E_CUDA -4          /* a CUDA runtime call or launch failed */
#define HPXGS_E_UNIMPLEMENTED -5 /* feature not built */
#define HPXGS_E_WORKSPACE -6     /* workspace smaller than the size query returned */
#define HPXGS_E_CAPTURE -7       /* call needs a host synchronisation inside stream capture */

/* ---- device status flags (OR-ed into the caller's int32 status word) ---- */
#define HPXGS_F_CAPACITY 1       /* more (Gaussian, tile) pairs than capacity_pairs */
#define HPXGS_F_TIMEOUT 2        /* a bounded wait gave up */

/* ---- cameras (Sec. 3.1, Sec. D.1) ---- */
#define HPXGS_CAM_FULL 0     /* omnidirectional: every pixel is valid */
#define HPXGS_CAM_PINHOLE 1  /* Eq. persp_sphere; valid iff -t_x (1 + ppx) <= d_x/d_z <= t_x (1 - ppx), likewise y, t = tan(fov/2) */
#define HPXGS_CAM_FISHEYE 2  /* anisotropic equidistant, Eqs. fish_weff..semi_axes; valid iff psi <= (pi/2) w_eff(gamma), w = fov/180 deg */

#define HPXGS_MAX_VIEWS 64
#define HPXGS_NACC 9         /* per-(view, Gaussian) backward accumulators */

/* Scene (Algorithm 1, Require): P Gaussians, float32, row-major, device memory. */
typedef struct {
  const float* means;      /* [P,3] world positions mu */
  const float* scales;     /* [P,3] linear scales s (caller applies exp) */
  const float* rotations;  /* [P,4] quaternions (w,x,y,z), need not be normalised */
  const float* opacities;  /* [P]   o in (0,1) (caller applies sigmoid) */
  const float* sh;         /* [P,K,3] real SH coefficients, K = (sh_degree+1)^2, 3DGS order/sign convention */
  int32_t P;
  int32_t sh_degree;       /* 0..3 */
} hpxgs_gaussians;

typedef struct {
  int32_t kind;            /* HPXGS_CAM_* */
  float fov_x_deg;         /* full horizontal FoV, degrees (pinhole: of the centred frustum, 2 atan(W / 2 f_x)) */
  float fov_y_deg;         /* full vertical FoV, degrees */
  /* Pinhole principal point (Eq. persp_sphere) as an offset from the image centre in
   * half-image units: c_x = (W/2)(1 + ppx), c_y = (H/2)(1 + ppy), |ppx|, |ppy| < 1, so the
   * frustum is asymmetric: d_x/d_z in [-tan(fov_x/2)(1 + ppx), tan(fov_x/2)(1 - ppx)].
   * Must be 0 for the fisheye (the paper fixes its principal point at the centre) and
   * the full sphere. Zero-initialised structs give the centred camera. */
  float ppx, ppy;
} hpxgs_camera;

/* One view V = [W | b] (Sec. 3.2) rendered at HEALPix order nside_log2. */
typedef struct {
  float W[9];              /* world-to-camera rotation, row-major */
  float b[3];              /* translation */
  int32_t nside_log2;      /* k: Nside = 2^k, Npix = 12 * 4^k; tile_level + 0 <= k <= 13 */
  hpxgs_camera cam;
} hpxgs_view;

/* Rasterizer settings. The paper fixes B = 16 (Table "resolution") and eps
 * (Algorithm 1); the others are readings where the paper is silent. */
typedef struct {
  int32_t tile_level;      /* b: tiles are NESTED blocks of 4^b pixels (B = 2^b); 3..5, default 4 */
  float eps_T;             /* early termination T < eps_T (Algorithm 1), default 1e-4 */
  float alpha_max;         /* alpha clamp, default 0.99 */
  float cutoff_m;          /* alpha = 0 where d^T conic d > cutoff_m (3-sigma ellipse), default 9.
                            * INFINITY gives the literal tile semantics of the paper's ablation
                            * (Sec. 3.3): every listed Gaussian contributes at every pixel of its
                            * listed tiles (the lists keep their 3-sigma radius r_s), so the image
                            * depends on the tile query. */
  float blur_rad2;         /* isotropic term added to Sigma_arc; < 0 selects 0.3 * Omega_pix (default) */
  float near_plane;        /* Gaussians with radial depth r <= near_plane are culled, default 0.2 */
  float bg[3];             /* background seen through T_final, default 0 */
  float lambda_ssim;       /* loss weight lambda (Sec. 4.1), default 0.2 */
  int32_t write_outside;   /* 1: pixels outside the FoV mask get bg, T=1, last=0; 0: inactive tiles untouched */
  /* launch shape of the blend kernels (0 = built-in default; results do not depend on them):
   * pixels per thread of the forward (1, 2, 4 or 8) and of the backward (1, 2, 4 or 8), and
   * resident blocks per SM of the persistent grids (capped by occupancy). */
  int32_t fwd_ppt;
  int32_t bwd_ppt;
  int32_t blocks_per_sm;
  /* tile query (Sec. 3.3): HPXGS_QUERY_RING (default; Algorithm 3 with the exact
   * membership test) or HPXGS_QUERY_NESTED (Algorithm 2, the quadtree search refined
   * down to tile order + query_log2f). query_log2f (0..3, at most tile_level, default 0)
   * is the search refinement f = 2^query_log2f of either query: RING x f runs Algorithm 3
   * at order k_t + query_log2f (Sec. D.2) and lists a tile once when one of its query
   * pixels has its centre within r_s + rho(k, tile_level - query_log2f) + 1e-7 of the
   * Gaussian. Every choice lists every tile the cutoff ellipse can reach, so with the
   * default cutoff the maps do not depend on it; under cutoff_m = INFINITY they do. */
  int32_t query;
  int32_t query_log2f;
  /* 1 (default): the blends skip a list entry for each group of 32 pixels that a
   * conservative bound on its conic shows it cannot reach (m > cutoff in the
   * kernels' own arithmetic); 0: every entry is evaluated at every pixel. The
   * results are the same bit for bit either way. */
  int32_t blend_cull;
  /* 1 (default): with tile_level 5 the blends take the four order-4 quarters of each
   * listed tile as separate units (the lists stay at order 5, about half the pairs of
   * order 4; the blend runs in the order-4 launch shapes). 0: whole tiles. Results are
   * the same bit for bit either way (gradients up to the order of atomic sums). */
  int32_t blend_split;
} hpxgs_config;

#define HPXGS_QUERY_RING 0
#define HPXGS_QUERY_NESTED 1

/* Human-readable name of a status code. */
const char* hpxgs_strerror(int code);
/* Map a device status word (HPXGS_F_* flags) to a return code. */
int hpxgs_status_error(int32_t flags);
/* Fill *cfg with the defaults listed above. */
void hpxgs_config_default(hpxgs_config* cfg);

/* Adaptive resolution (Sec. 3.1, Table "resolution"):
 * N* = sqrt(4 pi W H / (12 Omega_in)), Omega_in = 4 pi (full), 2 pi (1 - cos(fov/2))
 * (fisheye), 4 asin(sin(fov_x/2) sin(fov_y/2)) (pinhole); k = round(log2 N*),
 * kL = floor, kH = ceil. Host only; any output pointer may be NULL. */
int hpxgs_nside_for_image(int kind, double W, double H, double fov_x_deg, double fov_y_deg,
                          double* nstar, int* k, int* kL, int* kH);

/* rho(k, b): the largest angle between a tile centre (order k - b) and a pixel
 * centre (order k) of that tile, rounded up to a multiple of 2^-20 rad. It
 * widens the tile-membership test (tile t is listed for Gaussian i iff t has
 * an in-mask pixel and c_t . g_i >= cos(min(pi, r_s + rho + 1e-7))).
 * Computed once per (k, b) on the device and cached for the process.
 * SYNCHRONISES `stream` the first time a pair (k, b) is seen; returns
 * HPXGS_E_CAPTURE if that first time happens inside stream capture. */
int hpxgs_tile_rho(int k, int b, double* rho, hpxgs_stream_t stream);
/* PixRad(o) of the NESTED tile query (Algorithm 2), 0 <= o <= 15: the largest angle from a
 * node centre to its boundary at order o (9 samples per edge, corners included),
 * rounded up to 2^-20 rad. Cached per order; the first call for an order
 * synchronises the stream and returns HPXGS_E_CAPTURE inside stream capture. */
int hpxgs_pixrad(int o, double* out, hpxgs_stream_t stream);

/* Fill the rho cache for every (view order, tile_level) pair of `views`.
 * Call once before capturing forward/backward calls into a CUDA graph. */
int hpxgs_prepare(const hpxgs_view* views, int nviews, const hpxgs_config* cfg, hpxgs_stream_t stream);

/* FoV mask M_C(p) (Sec. 3.1) of one view as bits: bit (p & 31) of word p >> 5.
 * mask_bits: device uint32 [Npix/32]. Decided in FP32 with an FP64 re-check
 * within 1e-4 of the boundary. */
int hpxgs_mask_build(const hpxgs_view* view, const hpxgs_config* cfg, uint32_t* mask_bits,
                     hpxgs_stream_t stream);

/* ---- HEALPix batch utilities (device arrays of n entries) ---- */
/* Pixel centre unit vectors of NESTED pixels (HEALPix frame), FP32 and/or FP64 (either may be NULL). */
int hpxgs_pix2vec_nest(int k, const int64_t* pix, int64_t n, float* vec32, double* vec64, hpxgs_stream_t stream);
/* NESTED pixel containing each direction (FP64 input, need not be normalised). */
int hpxgs_vec2pix_nest(int k, const double* vec, int64_t n, int64_t* pix, hpxgs_stream_t stream);
/* Pixel centre angles of NESTED pixels (Sec. 3.1): colatitude theta in [0, pi] and longitude
 * phi in [0, 2 pi) of the HEALPix frame, FP64. */
int hpxgs_pix2ang_nest(int k, const int64_t* pix, int64_t n, double* theta, double* phi, hpxgs_stream_t stream);
/* NESTED pixel containing the direction (theta, phi) (FP64; the vec2pix construction of
 * the unit vector (sin theta cos phi, sin theta sin phi, cos theta)). */
int hpxgs_ang2pix_nest(int k, const double* theta, const double* phi, int64_t n, int64_t* pix, hpxgs_stream_t stream);
/* NESTED <-> RING index conversion. */
int hpxgs_nest2ring(int k, const int64_t* in, int64_t n, int64_t* out, hpxgs_stream_t stream);
int hpxgs_ring2nest(int k, const int64_t* in, int64_t n, int64_t* out, hpxgs_stream_t stream);
/* 8-neighbourhood (pixels sharing a vertex), out [n,8], -1 where the pixel
 * has only 7 neighbours; order: (dx,dy) = (-1,-1),(-1,0),(-1,1),(0,-1),(0,1),(1,-1),(1,0),(1,1)
 * in the face's (x, y) frame. Requires k >= 1. */
int hpxgs_neighbours_nest(int k, const int64_t* pix, int64_t n, int64_t* out, hpxgs_stream_t stream);

/* ---- rasterizer (Algorithm 1 forward; Sec. 3.2 backward) ---- */

/* Bytes of workspace for hpxgs_forward/hpxgs_backward/hpxgs_count_pairs with
 * P Gaussians, these views, and room for capacity_pairs (Gaussian, tile) pairs. */
int hpxgs_forward_workspace_size(int32_t P, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                                 int64_t capacity_pairs, size_t* bytes);

/* Forward render of nviews views in one batch (Algorithm 1):
 *  1. preprocess per (view, Gaussian): t, r, Sigma_arc (Eqs. 1-2), conic,
 *     r_s = 3 sqrt(lambda_max), SH colour;
 *  2. stable radix sort of the Gaussians by radial depth r;
 *  3. per Gaussian: RING query (Algorithm 3) + exact tile membership -> counts
 *     (beside the depth sort), exclusive scan of the counts in depth order,
 *     emission of (tile, Gaussian) pairs in depth order;
 *  4. stable radix sort of the pairs by global tile id, per-tile ranges;
 *  5. per tile, per pixel: front-to-back compositing with early exit at
 *     T < eps_T (Eq. unified_rendering).
 * Outputs (packed over views, see "pixel base"): maps [sum Npix, 3],
 * T_final [sum Npix], last [sum Npix] (number of list entries processed),
 * mask_bits [sum Npix / 32] (may be NULL), radii [nviews * P] (r_s in rad,
 * 0 when culled; may be NULL), depth_map [sum Npix] (may be NULL: the
 * inverse-depth channel D = sum_i T_i alpha_i / r_i of Sec. 3.2's depth
 * supervision, 0 outside the mask; it runs each tile level's default blend
 * shape). The workspace keeps what hpxgs_backward needs;
 * do not modify it in between. If more than capacity_pairs pairs are needed,
 * HPXGS_F_CAPACITY is set in *status, the extra pairs are dropped and the
 * outputs are incomplete: grow the capacity and call again. */
int hpxgs_forward(const hpxgs_gaussians* g, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                  void* workspace, size_t workspace_bytes, int64_t capacity_pairs,
                  float* maps, float* T_final, uint32_t* last, uint32_t* mask_bits, float* radii,
                  float* depth_map, int32_t* status, hpxgs_stream_t stream);

/* Backward (Sec. 3.2, Eqs. backward_lat_scale, grad_via_J_S): from dL/dmaps
 * (packed like maps) and the forward's T_final/last, walk each tile list in
 * reverse recovering T by division, accumulate per-(view, Gaussian) partials
 * (warp shuffles, then one global atomic per block and entry), then chain
 * them to the parameters. Gradients are written (not accumulated): dmeans
 * [P,3], dscales [P,3], drotations [P,4] (w.r.t. the unnormalised q),
 * dopacities [P], dsh [P,K,3], summed over the views. The cull, cutoff, clamp
 * and termination sets of the forward are held fixed. dL_ddepth [sum Npix]
 * (may be NULL) is the gradient of the inverse-depth channel; it enters through
 * dL/dalpha and through d(1/r)/dt = -t / r^3. */
int hpxgs_backward(const hpxgs_gaussians* g, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                   void* workspace, size_t workspace_bytes, int64_t capacity_pairs,
                   const float* dL_dmaps, const float* T_final, const uint32_t* last, const float* dL_ddepth,
                   float* dmeans, float* dscales, float* drotations, float* dopacities, float* dsh,
                   int32_t* status, hpxgs_stream_t stream);

/* The L1 + HSSIM loss gradient of one view, for hpxgs_backward_hssim. All device memory. */
typedef struct {
  const float* maps;       /* I: the view's rendered maps [Npix, 3] (its slice of hpxgs_forward's maps) */
  const float* targets;    /* G: the view's targets [Npix, 3] */
  const void* table;       /* window table of the view's order and mask (hpxgs_hssim_table_build) */
  const void* hssim_ws;    /* HSSIM workspace that hpxgs_hssim_forward_table filled for I, G this step */
  const float* dloss;      /* dL/dloss of the view (one float), or NULL for 1 */
} hpxgs_loss_view;

/* hpxgs_backward for the training loss of Sec. 4.1 (Eq. supp_hssim_eval), with the HSSIM
 * backward folded into the backward blend: each pixel's dL/dI is formed where the blend
 * reads it, from the view's window table and the coefficients its HSSIM forward stored,
 * instead of being written to and read from a dL/dmaps buffer. The result equals
 * hpxgs_hssim_backward_table per view (same lambda, dloss) followed by hpxgs_backward
 * with the packed dL/dmaps, up to the order of the atomic sums. Preconditions: the
 * forward on the same workspace, then hpxgs_hssim_forward_table for every view, on the
 * same stream. No inverse-depth channel (use hpxgs_backward with dL_ddepth); each tile
 * level runs its default blend shape (cfg->bwd_ppt is not used). loss_views [nviews];
 * lambda in [0, 1]; views need nside_log2 >= 3. Errors: HPXGS_E_INVALID_ARG for null or
 * out-of-range arguments, HPXGS_E_WORKSPACE for a workspace smaller than the layout. */
int hpxgs_backward_hssim(const hpxgs_gaussians* g, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                         void* workspace, size_t workspace_bytes, int64_t capacity_pairs,
                         const hpxgs_loss_view* loss_views, float lambda, const float* T_final,
                         const uint32_t* last, float* dmeans, float* dscales, float* drotations,
                         float* dopacities, float* dsh, int32_t* status, hpxgs_stream_t stream);

/* Radian-space density-control statistics (Sec. 4.2), after hpxgs_backward on the same
 * workspace (same g->P, views, cfg, capacity). For every (view, Gaussian) the Gaussian is
 * visible in (listed for at least one active tile of the view), updates the caller's
 * per-Gaussian buffers [P] in place:
 *   rs_max[i]      <- max(rs_max[i], r_s)                       (angular radius, rad)
 *   grad_accum[i]  += |(dL/domega, dL/dphi)|                     (rad^-1 units of the loss)
 *   vis_count[i]   += 1
 * dL/domega, dL/dphi: the gradient of the loss with respect to the centre's longitude and
 * latitude through the pixel offsets, with the conic held in the local (east, north) frame
 * (the radian-space counterpart of the screen-space mean gradient; a reading: the paper
 * does not spell out the angular gradient). From the backward's partials: dL/dphi is the
 * north partial; dL/domega = cos(phi) (east partial) + sin(phi) (2 b (L_c - L_a) + (a - c) L_b),
 * the second term the turn of the local frame against the transported one. angular (may
 * be NULL) receives (dL/domega, dL/dphi) per (view, Gaussian), [nviews * P, 2], 0 where
 * not visible. rs_max entries must be non-negative (zero-initialised by the caller: the
 * maximum compares float bit patterns). All buffers device memory; asynchronous on the
 * stream. Errors: HPXGS_E_INVALID_ARG for null buffers, HPXGS_E_WORKSPACE for a workspace
 * smaller than the layout. */
int hpxgs_density_stats(int32_t P, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                        const void* workspace, size_t workspace_bytes, int64_t capacity_pairs,
                        float* rs_max, float* grad_accum, uint32_t* vis_count, float* angular,
                        hpxgs_stream_t stream);

/* Steps 1-3 of hpxgs_forward without emission: writes the total number of
 * (Gaussian, tile) pairs the views need to *count (device uint64). Used to
 * size capacity and for memory-based admission. */
int hpxgs_count_pairs(const hpxgs_gaussians* g, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                      void* workspace, size_t workspace_bytes, uint64_t* count, int32_t* status,
                      hpxgs_stream_t stream);

/* ---- sphere <-> image resampling (Eq. camera_synthesis; Eqs. supp_image_to_healpix,
 *      supp_hssim_mask; camera models of Sec. D.1) ----
 * Images are row-major [height, width, 3] FP32 with pixel centres at (i + 1/2, j + 1/2).
 * HEALPix maps are NESTED [12 * 4^k, 3] FP32 in the camera frame: HEALPix (X, Y, Z)
 * is the camera direction (d_z, d_x, d_y). Camera kinds: pinhole (FoV_x, FoV_y in
 * (0, 180)), anisotropic equidistant fisheye (f = W / pi, H / pi, w = FoV / 180 deg,
 * FoV in (0, 360]), panorama (HPXGS_CAM_FULL: omega = 2 pi u / W - pi, phi = pi/2 - pi v / H).
 * The paper names the operations, not the schemes: Interp_H is HEALPix
 * ring-bilinear interpolation (linear in longitude along the two rings that
 * bracket the colatitude, linear in colatitude between them, and towards the
 * mean of the first/last ring's 4 pixels above/below it); images are sampled
 * bilinearly between pixel centres, clamped at the edges (wrapped in longitude
 * for the panorama). Asynchronous on `stream`; HPXGS_E_INVALID_ARG for a null
 * pointer, an order outside the stated range, a size outside [1, 65536] or a bad
 * camera. All buffers are device memory owned by the caller. */

/* I_C(u, v) = Interp_H(map, P_C(u, v)) at every pixel centre (Eq. camera_synthesis),
 * 1 <= nside_log2 <= 13. Pixels outside the valid domain D_C get 0; `valid`
 * ([height * width] bytes, may be NULL) gets 1 inside D_C, 0 outside. */
int hpxgs_sphere_to_image(const float* map, int nside_log2, const hpxgs_camera* cam, int width, int height,
                          float* image, uint8_t* valid, hpxgs_stream_t stream);
/* The adjoint of hpxgs_sphere_to_image: dmap = A^T dimage. dmap [12 * 4^k, 3] is
 * overwritten (zeroed, then accumulated with atomics, so the summation order varies). */
int hpxgs_sphere_to_image_backward(const float* dimage, int nside_log2, const hpxgs_camera* cam, int width,
                                   int height, float* dmap, hpxgs_stream_t stream);
/* I_H(q) = I_C(Pi_C^{-1}(s_q)) for every NESTED pixel q with M_C(q) = 1, 0 elsewhere
 * (Eq. supp_image_to_healpix), 2 <= nside_log2 <= 13; mask_bits ([12 * 4^k / 32]
 * words, may be NULL) gets M_C (Eq. supp_hssim_mask), the same mask as hpxgs_mask_build. */
int hpxgs_image_to_sphere(const float* image, int width, int height, const hpxgs_camera* cam, int nside_log2,
                          float* map, uint32_t* mask_bits, hpxgs_stream_t stream);
/* The same for an 8-bit camera image ([height, width, 3] bytes, the form a camera delivers):
 * code v is the value v / 255 (IEEE division), so the map equals hpxgs_image_to_sphere's on
 * the float image holding v / 255, bit for bit. A training step can take its target as the
 * camera image itself, a quarter of the bytes of a float image. */
int hpxgs_image_to_sphere_u8(const uint8_t* image, int width, int height, const hpxgs_camera* cam, int nside_log2,
                             float* map, uint32_t* mask_bits, hpxgs_stream_t stream);

/* ---- resampling plans (Eq. camera_synthesis; Eq. supp_image_to_healpix) ----
 * The taps of every output pixel of a resampling, computed once for a camera (kind, FoV,
 * principal point), an image size and a HEALPix order, then applied to any number of maps
 * or images (a training loop or a renderer with fixed intrinsics): an application is a
 * pure gather (its adjoint a scatter) and gives the direct call's result bit for bit.
 * HPXGS_PLAN_SPHERE_TO_IMAGE serves hpxgs_sphere_to_image and its adjoint (taps of the
 * width x height image pixels: 4 map pixels and weights, 33 bytes per image pixel);
 * HPXGS_PLAN_IMAGE_TO_SPHERE serves hpxgs_image_to_sphere(_u8) (taps of the 12 * 4^k map
 * pixels: 4 image pixels and weights, and M_C; 32 bytes per map pixel). The plan is device
 * memory owned by the caller, at least hpxgs_resample_plan_size bytes; building it launches
 * one kernel on the stream. An application must pass the order and image size the plan was
 * built for (else HPXGS_E_INVALID_ARG or HPXGS_E_WORKSPACE when the sizes disagree; a plan
 * of another camera of the same sizes is not detected). Image sizes are limited to
 * width * height < 2^32 (also for the direct calls). */
#define HPXGS_PLAN_SPHERE_TO_IMAGE 0
#define HPXGS_PLAN_IMAGE_TO_SPHERE 1
int hpxgs_resample_plan_size(int direction, int nside_log2, int width, int height, size_t* bytes);
int hpxgs_resample_plan_build(int direction, int nside_log2, const hpxgs_camera* cam, int width, int height,
                              void* plan, size_t plan_bytes, hpxgs_stream_t stream);
int hpxgs_sphere_to_image_planned(const float* map, int nside_log2, int width, int height, const void* plan,
                                  size_t plan_bytes, float* image, uint8_t* valid, hpxgs_stream_t stream);
int hpxgs_sphere_to_image_backward_planned(const float* dimage, int nside_log2, int width, int height,
                                           const void* plan, size_t plan_bytes, float* dmap, hpxgs_stream_t stream);
int hpxgs_image_to_sphere_planned(const float* image, int width, int height, int nside_log2, const void* plan,
                                  size_t plan_bytes, float* map, uint32_t* mask_bits, hpxgs_stream_t stream);
int hpxgs_image_to_sphere_u8_planned(const uint8_t* image, int width, int height, int nside_log2, const void* plan,
                                     size_t plan_bytes, float* map, uint32_t* mask_bits, hpxgs_stream_t stream);

/* ---- instrumentation ---- */
/* Stages that hpxgs_profile_arm can time. */
#define HPXGS_STAGE_MASK 0
#define HPXGS_STAGE_PREPROCESS 1
#define HPXGS_STAGE_DEPTH_SORT 2
#define HPXGS_STAGE_TILE_COUNT 3
#define HPXGS_STAGE_SCAN 4
#define HPXGS_STAGE_TILE_EMIT 5
#define HPXGS_STAGE_PAIR_SORT 6
#define HPXGS_STAGE_RANGES 7
#define HPXGS_STAGE_BLEND_FWD 8
#define HPXGS_STAGE_BLEND_BWD 9
#define HPXGS_STAGE_PREPROCESS_BWD 10
#define HPXGS_STAGE_HSSIM_FWD 11
#define HPXGS_STAGE_HSSIM_BWD 12
#define HPXGS_NUM_STAGES 13
/* Arm a one-shot timing of `stage`: the next call that runs the stage records
 * start_event (a cudaEvent_t) on its stream right before the stage's first
 * kernel and stop_event right after its last one, then disarms. Pass NULL
 * events to disarm. Host only; the events belong to the caller. When the stream
 * is being captured, the records become event-record nodes of the graph, so
 * every replay records both events again. */
int hpxgs_profile_arm(int stage, void* start_event, void* stop_event);
/* 1 if `stage` is still armed (no call has run it since hpxgs_profile_arm), 0 if not,
 * HPXGS_E_INVALID_ARG for an unknown stage. After a captured step, the stages still
 * armed are the ones the graph does not record. */
int hpxgs_profile_armed(int stage);
/* Number of kernels this library has launched in this process. */
uint64_t hpxgs_launch_count(void);
/* Measured FP32 throughput of this GPU at its current clocks, the denominators
 * of the blend kernels' roofline: dependency-free FMA chains over every SM
 * (fma_tflops, 2 flops per FMA) and MUFU ex2 chains (ex2_tops, 1e12 ops/s).
 * Synchronises the stream (about 20 ms of GPU time); HPXGS_E_CAPTURE inside
 * stream capture. */
int hpxgs_probe_alu_peak(double* fma_tflops, double* ex2_tops, hpxgs_stream_t stream);
/* Check of the bounded grid barrier that the count scan uses in its cooperative
 * launch: `blocks` resident blocks meet at one barrier that waits
 * for blocks + `missing` arrivals, at most limit_ns each. `counter` (device u32) is
 * zeroed by this call; passed[b] (device u32 [blocks]) becomes 1 where block b got
 * through, 0 where it gave up. With missing = 0 every block passes; with missing > 0
 * every block gives up after limit_ns and HPXGS_F_TIMEOUT is OR-ed into *status (a
 * device int32). Asynchronous on `stream`. HPXGS_E_INVALID_ARG for null buffers,
 * blocks < 1, missing < 0, limit_ns > 2 s or more blocks than fit at once. */
int hpxgs_probe_grid_barrier(int blocks, int missing, uint64_t limit_ns, uint32_t* counter, uint32_t* passed,
                             int32_t* status, hpxgs_stream_t stream);

/* FP32 work of the blend kernels, counted from their inner loops (an FMA is 2
 * flops, a MUFU op is counted apart): per evaluated (pixel, entry) pair, the
 * offset and m = d^T conic d (offset and its squared chord, tangent components, quadratic form,
 * arc-length series); per contributing pair (m <= cutoff, before termination),
 * alpha and compositing in the forward, and T recovery, dL/dalpha and the
 * conic and position partials in the backward. */
#define HPXGS_FLOPS_EVAL 40
#define HPXGS_FLOPS_FWD_CONTRIB 13
#define HPXGS_FLOPS_BWD_CONTRIB 83
#define HPXGS_MUFU_FWD_CONTRIB 1   /* ex2 */
#define HPXGS_MUFU_BWD_CONTRIB 2   /* ex2, reciprocal */

/* Device pointers into a forward workspace (for inspection and tests). */
typedef struct {
  const float* records;        /* [nviews*P, 16]: g(3), o, e_east(3), conic_a, e_north(3), conic_b, colour(3), conic_c */
  const float* radii;          /* [nviews*P] r_s */
  const float* depth;          /* [nviews*P] radial depth r */
  const uint32_t* pair_tiles;  /* [n_pairs] sorted global tile ids (after hpxgs_forward) */
  const uint32_t* pair_ids;    /* [n_pairs] Gaussian ids v*P + i in list order */
  const uint32_t* ranges;      /* [total_tiles, 2] start/end into pair_ids */
  const uint32_t* n_pairs;     /* device scalar: pairs needed (may exceed capacity) */
  const float* accum;          /* [nviews*P, HPXGS_NACC] backward partials (after hpxgs_backward) */
  const uint64_t* n_eval;      /* device scalar: (pixel, list entry) pairs up to each pixel's termination in the
                                  last forward blend (the blend cull skips most of those that cannot contribute) */
  const uint64_t* n_contrib;   /* device scalar: of those, entries with alpha > 0 */
  int64_t total_tiles;
  /* [n_pairs] blend cull per list entry (aligned with pair_ids): bit g set unless
   * no pixel of the entry's tile at in-tile NESTED offsets 32g .. 32g+31 can reach
   * m <= cutoff. Written by the forward blend for every entry it staged (at least
   * the first max(last) entries of each active tile); read by the backward. */
  const uint32_t* cull_masks;
} hpxgs_workspace_view;
int hpxgs_workspace_inspect(int32_t P, const hpxgs_view* views, int nviews, const hpxgs_config* cfg,
                            int64_t capacity_pairs, const void* workspace, hpxgs_workspace_view* out);

/* ---- HEALPix-SSIM and training loss (Sec. 4.1; Eq. supp_hssim_eval) ----
 * Window of pixel q: q and its in-mask 8- (7-) neighbours, weights
 * exp(-theta^2 / (2 sigma^2)) of the centre-to-centre angle, sigma =
 * 1.5 sqrt(Omega_pix), normalised per window; SSIM constants C1 = 0.01^2,
 * C2 = 0.03^2; h_q = mean over RGB; HSSIM = masked mean of h_q;
 * loss = (1 - lambda) mean_mask |I - G| + lambda (1 - HSSIM). */
int hpxgs_hssim_workspace_size(int k, size_t* bytes);
/* out3 (device float[3]) = {loss, HSSIM, L1}. I, G: [Npix,3]; mask_bits as hpxgs_mask_build. */
int hpxgs_hssim_forward(const float* I, const float* G, const uint32_t* mask_bits, int k, float lambda,
                        void* workspace, size_t workspace_bytes, float* out3, hpxgs_stream_t stream);
/* dI = dloss * dL/dI (written, zero outside the mask); dloss is a device scalar
 * (may be NULL for 1). Needs the workspace of the matching hpxgs_hssim_forward. */
int hpxgs_hssim_backward(const float* I, const float* G, const uint32_t* mask_bits, int k, float lambda,
                         const void* workspace, size_t workspace_bytes, const float* dloss, float* dI,
                         hpxgs_stream_t stream);
/* Window table of (order k, mask): the neighbour walk and the window weights of
 * every pixel (Sec. 4.1), which depend on the grid and the mask only, stored so
 * that forward and backward skip them: [8][Npix] neighbour ids and [8][Npix]
 * weights by neighbour direction (weight 0 and the pixel's own id where that
 * neighbour is missing or outside the mask), [Npix] 1 / window sum (68 bytes per
 * pixel, caller-owned device
 * memory of at least hpxgs_hssim_table_size bytes). Build it once per mask; the
 * *_table calls give the results of hpxgs_hssim_forward / _backward bit for bit
 * when given the same mask. A mask depends on the camera's intrinsics only, so
 * one table serves every pose of a camera. */
int hpxgs_hssim_table_size(int k, size_t* bytes);
int hpxgs_hssim_table_build(const uint32_t* mask_bits, int k, void* table, size_t table_bytes,
                            hpxgs_stream_t stream);
int hpxgs_hssim_forward_table(const float* I, const float* G, const uint32_t* mask_bits, int k, float lambda,
                              const void* table, void* ws, size_t ws_bytes, float* out3, hpxgs_stream_t stream);
int hpxgs_hssim_backward_table(const float* I, const float* G, const uint32_t* mask_bits, int k, float lambda,
                               const void* table, const void* ws, size_t ws_bytes, const float* dloss, float* dI,
                               hpxgs_stream_t stream);

/* ---- loss value without a workspace ----
 * No counterpart in the paper. For callers that cannot give the library device
 * memory (a plugin inside a host application that owns the GPU memory budget,
 * a real-time loop that must not allocate after start-up): out3 = {loss, HSSIM,
 * L1}, value only (no gradient). Per pixel it runs the same window and SSIM
 * arithmetic as hpxgs_hssim_forward; only the block sums are added differently,
 * and the two agree within 2e-6. The per-block partial sums live in a fixed
 * 1.18 MB array inside the library's device image, which every GPU that loads
 * the library holds until exit; the call allocates nothing. Limit: k <= 10
 * (Nside <= 1024); larger k returns HPXGS_E_INVALID_ARG. The first call on each
 * device looks up the array's device address (with that device current); make
 * that first call, and the first call after a cudaDeviceReset, before any stream
 * capture. Calls outside capture look the address up again (so a module reloaded
 * after a reset is found); a capturing stream on a device that has made no call
 * yet gets HPXGS_E_CAPTURE. All calls share the array: calls that overlap on the
 * GPU race. */
int hpxgs_hssim_loss_noalloc(const float* I, const float* G, const uint32_t* mask_bits, int k, float lambda,
                             float* out3, hpxgs_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* HPXGS_H_ */
