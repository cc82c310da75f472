// FP64 CPU oracle for the HEALPix spherical Gaussian rasterizer (UniTriSplat,
// arXiv 2606.29794).
//
// TEST INFRASTRUCTURE. Only the test suite, the smoke check and the bench's
// CPU-baseline leg may load this library. The product path (the CUDA library
// under paper_2606_29794_b300/) shares no code with it and never calls it.
//
// Everything here is plain, slow and double precision. Each function follows
// one passage of the paper in the paper's order and notation:
//   Sec. 3.1            HEALPix grid, NESTED (x, y, f), tiles, FoV mask, adaptive Nside
//   Sec. 3.2, Eq. 1-2   spherical projection Pi, Sigma_arc = S_phi J W Sigma3D W^T J^T S_phi
//   Sec. 3.2, Eq. 3-4   backward: latitude term and position paths
//   Sec. 3.3, Eq. 5     RING query (Algorithm 3) for candidate tiles
//   Sec. 3.4, Eq. 6     haversine + bearing offset, front-to-back compositing (Algorithm 1)
//   Sec. 4.1            HEALPix-SSIM and the L1 + HSSIM training loss
//   Sec. D.1            camera models (pinhole, equidistant fisheye, ERP), Table "resolution"
// Where the paper is silent, the reading taken is stated next to the code that
// takes it.
//
// HEALPix geometry follows the published equations of Gorski et al. (2005,
// ApJ 622:759) for ring latitudes/longitudes and the planar HEALPix projection
// of Calabretta & Roukema (2007, MNRAS 381:865) for the inverse map.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;
typedef uint32_t u32;
typedef uint8_t u8;

static const double kPi = 3.14159265358979323846;

// ===========================================================================
// HEALPix indexing (Sec. 3.1)
// ===========================================================================

// Put bit k of v at bit 2k (NESTED index = interleave of x (even bits) and y (odd bits)).
static i64 spread_bits(i64 v) {
  i64 r = 0;
  for (int k = 0; k < 31; ++k) r |= ((v >> k) & 1LL) << (2 * k);
  return r;
}
static i64 compact_bits(i64 v) {
  i64 r = 0;
  for (int k = 0; k < 31; ++k) r |= ((v >> (2 * k)) & 1LL) << k;
  return r;
}

struct XYF { i64 x, y, f; };

static XYF nest2xyf(i64 nside, i64 p) {
  i64 npface = nside * nside;
  XYF r;
  r.f = p / npface;
  i64 q = p % npface;
  r.x = compact_bits(q);
  r.y = compact_bits(q >> 1);
  return r;
}
static i64 xyf2nest(i64 nside, i64 x, i64 y, i64 f) {
  return f * nside * nside + spread_bits(x) + (spread_bits(y) << 1);
}
static i64 pmod(i64 a, i64 m) { i64 r = a % m; return r < 0 ? r + m : r; }

// Face row (0 north, 1 equatorial, 2 south) and the face centre longitude in units of pi/4.
static i64 face_row(i64 f) { return f / 4; }
static i64 face_jpll(i64 f) { return face_row(f) == 1 ? 2 * (f % 4) : 2 * (f % 4) + 1; }

// Ring geometry (Gorski et al. 2005): ring i = 1..4N-1 counted from the north pole.
struct Ring { double z, sth; i64 npix; double phi0; };
static Ring ring_info(i64 nside, i64 i) {
  Ring R;
  double N = (double)nside;
  if (i < nside) {                      // north polar cap: 4i pixels
    double t = (double)i * i / (3.0 * N * N);
    R.z = 1.0 - t; R.sth = std::sqrt(t * (2.0 - t));
    R.npix = 4 * i; R.phi0 = kPi / (4.0 * i);
  } else if (i > 3 * nside) {           // south polar cap
    i64 ii = 4 * nside - i;
    double t = (double)ii * ii / (3.0 * N * N);
    R.z = t - 1.0; R.sth = std::sqrt(t * (2.0 - t));
    R.npix = 4 * ii; R.phi0 = kPi / (4.0 * ii);
  } else {                              // equatorial belt: 4N pixels, alternating shift
    R.z = (2.0 * N - (double)i) * 2.0 / (3.0 * N);
    R.sth = std::sqrt((1.0 - R.z) * (1.0 + R.z));
    R.npix = 4 * nside;
    i64 s = (i - nside + 1) & 1;
    R.phi0 = (kPi / (2.0 * N)) * (1.0 - 0.5 * s);
  }
  return R;
}

// Centre of NESTED pixel p: z = cos(colatitude), sin(colatitude), longitude in [0, 2pi).
// The ring of face pixel (x, y) is (row+2)N - x - y - 1 and the longitude is
// (pi/4)(jpll + (x - y)/n_r), n_r = this face's share of the ring.
static void pix2zphi_nest(i64 nside, i64 p, double& z, double& sth, double& phi, i64* ring_out) {
  XYF c = nest2xyf(nside, p);
  i64 jr = (face_row(c.f) + 2) * nside - c.x - c.y - 1;
  double N = (double)nside;
  i64 nr;
  if (jr < nside) {
    nr = jr; double t = (double)nr * nr / (3.0 * N * N);
    z = 1.0 - t; sth = std::sqrt(t * (2.0 - t));
  } else if (jr > 3 * nside) {
    nr = 4 * nside - jr; double t = (double)nr * nr / (3.0 * N * N);
    z = t - 1.0; sth = std::sqrt(t * (2.0 - t));
  } else {
    nr = nside;
    z = (2.0 * N - (double)jr) * 2.0 / (3.0 * N);
    sth = std::sqrt((1.0 - z) * (1.0 + z));
  }
  phi = (kPi / 4.0) * ((double)face_jpll(c.f) + (double)(c.x - c.y) / (double)nr);
  if (phi < 0) phi += 2 * kPi;
  if (phi >= 2 * kPi) phi -= 2 * kPi;
  if (ring_out) *ring_out = jr;
}

static void pix2vec_nest(i64 nside, i64 p, double v[3]) {
  double z, sth, phi;
  pix2zphi_nest(nside, p, z, sth, phi, nullptr);
  v[0] = sth * std::cos(phi); v[1] = sth * std::sin(phi); v[2] = z;
}

// Planar HEALPix projection (Calabretta & Roukema 2007) in units of pi/4:
// belt |z| <= 2/3: (X, Y) = (phi / (pi/4), 3z/2); caps: sigma = sqrt(3(1-|z|)),
// X = phi_c + (phi - phi_c) sigma, Y = +-(2 - sigma). Faces are unit diamonds
// centred at (2f+1, 1) (north), (2e, 0) (equator), (2s+1, -1) (south).
static i64 zphi2pix_nest(i64 nside, double z, double phi) {
  phi = std::fmod(phi, 2 * kPi);
  if (phi < 0) phi += 2 * kPi;
  double X, Y; i64 f, Xc, Yc;
  if (std::fabs(z) <= 2.0 / 3.0) {
    X = phi / (kPi / 4.0); Y = 1.5 * z;
    i64 A = (i64)std::floor((X + Y + 1.0) / 2.0);
    i64 B = (i64)std::floor((Y - X + 1.0) / 2.0);
    if (A + B >= 1) { f = pmod(A - 1, 4); Xc = 2 * A - 1; Yc = 1; }
    else if (A + B == 0) { f = 4 + pmod(A, 4); Xc = 2 * A; Yc = 0; }
    else { f = 8 + pmod(A, 4); Xc = 2 * A + 1; Yc = -1; }
  } else {
    double sigma = std::sqrt(3.0 * (1.0 - std::fabs(z)));
    i64 fc = (i64)std::floor(phi / (kPi / 2.0));
    if (fc > 3) fc = 3;
    double phic = ((double)fc + 0.5) * (kPi / 2.0);
    X = (phic + (phi - phic) * sigma) / (kPi / 4.0);
    Y = (z > 0 ? 1.0 : -1.0) * (2.0 - sigma);
    Xc = 2 * fc + 1;
    if (z > 0) { f = fc; Yc = 1; } else { f = 8 + fc; Yc = -1; }
  }
  double u = (X - Xc + Y - Yc + 1.0) / 2.0;
  double v = (Y - Yc - (X - Xc) + 1.0) / 2.0;
  i64 x = (i64)std::floor(u * nside), y = (i64)std::floor(v * nside);
  x = std::min(std::max(x, (i64)0), nside - 1);
  y = std::min(std::max(y, (i64)0), nside - 1);
  return xyf2nest(nside, x, y, f);
}

static i64 vec2pix_nest(i64 nside, const double v[3]) {
  double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  return zphi2pix_nest(nside, v[2] / n, std::atan2(v[1], v[0]));
}

// Inverse of the planar projection for a point (u, v) in [0,1]^2 of face f.
static void face_uv2vec(i64 f, double u, double v, double out[3]) {
  i64 row = face_row(f);
  double Xc = (double)face_jpll(f), Yc = (row == 0) ? 1.0 : (row == 1 ? 0.0 : -1.0);
  double X = Xc + u - v, Y = Yc + u + v - 1.0;
  double z, phi;
  if (std::fabs(Y) <= 1.0) { z = 2.0 * Y / 3.0; phi = X * kPi / 4.0; }
  else {
    double sigma = 2.0 - std::fabs(Y);
    z = (Y > 0 ? 1.0 : -1.0) * (1.0 - sigma * sigma / 3.0);
    phi = Xc * kPi / 4.0 + (sigma > 0 ? (X - Xc) * (kPi / 4.0) / sigma : 0.0);
  }
  double sth = std::sqrt(std::max(0.0, (1.0 - z) * (1.0 + z)));
  out[0] = sth * std::cos(phi); out[1] = sth * std::sin(phi); out[2] = z;
}

// RING-scheme index of ring i, in-ring position j (Gorski et al. 2005 numbering).
static i64 ring_start(i64 nside, i64 i) {
  if (i <= nside) return 2 * i * (i - 1);
  if (i <= 3 * nside) return 2 * nside * (nside - 1) + 4 * nside * (i - nside);
  i64 ii = 4 * nside - i;
  return 12 * nside * nside - 2 * ii * (ii + 1);
}
static void ringpix_decompose(i64 nside, i64 pr, i64& i, i64& j) {
  i64 lo = 1, hi = 4 * nside - 1;
  while (lo < hi) {
    i64 mid = (lo + hi + 1) / 2;
    if (ring_start(nside, mid) <= pr) lo = mid; else hi = mid - 1;
  }
  i = lo; j = pr - ring_start(nside, lo);
}
static void ring2zphi(i64 nside, i64 i, i64 j, double& z, double& sth, double& phi) {
  Ring R = ring_info(nside, i);
  z = R.z; sth = R.sth;
  phi = R.phi0 + 2.0 * kPi * (double)j / (double)R.npix;
}
// ring -> nest: centre of the ring pixel, then the planar inverse map.
static i64 ring2nest(i64 nside, i64 pr) {
  i64 i, j; ringpix_decompose(nside, pr, i, j);
  double z, sth, phi; ring2zphi(nside, i, j, z, sth, phi);
  return zphi2pix_nest(nside, z, phi);
}
// nest -> ring: ring number of the face pixel, position from its longitude.
static i64 nest2ring(i64 nside, i64 p) {
  double z, sth, phi; i64 jr;
  pix2zphi_nest(nside, p, z, sth, phi, &jr);
  Ring R = ring_info(nside, jr);
  double jj = (phi - R.phi0) * (double)R.npix / (2.0 * kPi);
  i64 j = pmod((i64)std::llround(jj), R.npix);
  return ring_start(nside, jr) + j;
}

// 8-neighbourhood by geometry: the pixels sharing at least one vertex with p.
// Sample a small circle around each of p's four corners and look up each point.
static int neighbours_nest(i64 nside, i64 p, i64 out[8]) {
  XYF c = nest2xyf(nside, p);
  double N = (double)nside;
  double eps = 0.05 * std::sqrt(4.0 * kPi / (12.0 * N * N));
  std::vector<i64> found;
  for (int cu = 0; cu < 2; ++cu)
    for (int cv = 0; cv < 2; ++cv) {
      double vtx[3];
      face_uv2vec(c.f, (c.x + cu) / N, (c.y + cv) / N, vtx);
      double a[3] = {0, 0, 1};
      if (std::fabs(vtx[2]) > 0.9) { a[0] = 1; a[2] = 0; }
      double t1[3] = {a[1] * vtx[2] - a[2] * vtx[1], a[2] * vtx[0] - a[0] * vtx[2], a[0] * vtx[1] - a[1] * vtx[0]};
      double n1 = std::sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
      for (int k = 0; k < 3; ++k) t1[k] /= n1;
      double t2[3] = {vtx[1] * t1[2] - vtx[2] * t1[1], vtx[2] * t1[0] - vtx[0] * t1[2], vtx[0] * t1[1] - vtx[1] * t1[0]};
      const int K = 48;
      for (int s = 0; s < K; ++s) {
        double ang = 2.0 * kPi * (s + 0.5) / K;
        double q[3];
        for (int k = 0; k < 3; ++k)
          q[k] = vtx[k] * std::cos(eps) + (std::cos(ang) * t1[k] + std::sin(ang) * t2[k]) * std::sin(eps);
        i64 pp = vec2pix_nest(nside, q);
        if (pp != p && std::find(found.begin(), found.end(), pp) == found.end()) found.push_back(pp);
      }
    }
  std::sort(found.begin(), found.end());
  int n = (int)std::min<size_t>(found.size(), 8);
  for (int k = 0; k < 8; ++k) out[k] = k < n ? found[k] : -1;
  return (int)found.size();
}

// ===========================================================================
// Cameras and the FoV mask (Sec. 3.1; Sec. D.1)
// Camera directions d = (cos(phi) sin(omega), sin(phi), cos(phi) cos(omega)).
// Reading: HEALPix colatitude = pi/2 - phi and HEALPix longitude = omega, so a
// HEALPix unit vector (X, Y, Z) is the camera direction (d_z, d_x, d_y).
// ===========================================================================

enum { CAM_FULL = 0, CAM_PINHOLE = 1, CAM_FISHEYE = 2 };

// Signed margin of direction d (camera frame) against the camera's valid region:
// >= 0 inside. Pinhole (Eq. persp_sphere): d_z > 0 and the image point
// u = c_x + f_x d_x/d_z, v = c_y + f_y d_y/d_z inside [0,W] x [0,H], with
// f_x = W / (2 tan(FoV_x/2)) and the principal point c_x = (W/2)(1 + ppx),
// c_y = (H/2)(1 + ppy); in units of d_z: min(d_x - lo_x d_z, hi_x d_z - d_x, ...)
// with lo_x = -c_x / f_x, hi_x = (W - c_x) / f_x. Fisheye: incident angle
// psi <= (pi/2) w_eff(gamma) (Eqs. fish_weff, imaging_region, semi_axes).
static double camera_margin(int kind, double fovx_deg, double fovy_deg, double ppx, double ppy, const double d[3]) {
  if (kind == CAM_FULL) return 1.0;
  if (kind == CAM_PINHOLE) {
    double tx = std::tan(0.5 * fovx_deg * kPi / 180.0), ty = std::tan(0.5 * fovy_deg * kPi / 180.0);
    if (d[2] <= 0) return -1.0;
    // c_x / f_x = tan(FoV_x/2)(1 + ppx), (W - c_x) / f_x = tan(FoV_x/2)(1 - ppx)
    double lox = -tx * (1.0 + ppx), hix = tx * (1.0 - ppx);
    double loy = -ty * (1.0 + ppy), hiy = ty * (1.0 - ppy);
    double mx = std::min(d[0] - lox * d[2], hix * d[2] - d[0]);
    double my = std::min(d[1] - loy * d[2], hiy * d[2] - d[1]);
    return std::min(mx, my);
  }
  double wx = fovx_deg / 180.0, wy = fovy_deg / 180.0;
  double rxy = std::sqrt(d[0] * d[0] + d[1] * d[1]);
  double psi = std::atan2(rxy, d[2]);
  double gam = std::atan2(d[1], d[0]);
  double weff = std::sqrt(std::pow(wx * std::cos(gam), 2) + std::pow(wy * std::sin(gam), 2));
  return 0.5 * kPi * weff - psi;
}

// Adaptive resolution (Sec. 3.1; Table "resolution"): N* = sqrt(4 pi W H / (12 Omega_in)).
static double solid_angle_in(int kind, double fovx_deg, double fovy_deg) {
  double hx = 0.5 * fovx_deg * kPi / 180.0, hy = 0.5 * fovy_deg * kPi / 180.0;
  if (kind == CAM_FULL) return 4.0 * kPi;
  if (kind == CAM_FISHEYE) return 2.0 * kPi * (1.0 - std::cos(hx));
  return 4.0 * std::asin(std::sin(hx) * std::sin(hy));
}

// ===========================================================================
// Real spherical harmonics, degree <= 3 (3DGS colour convention inherited, Sec. 5.1):
// Y_l^m = K_l^m P_l^|m|(cos theta) {sqrt2 cos(m phi), 1, sqrt2 sin(|m| phi)},
// P_l^m with the Condon-Shortley phase, coefficients ordered k = l^2 + l + m.
// ===========================================================================

static double factorial(int n) { double r = 1; for (int k = 2; k <= n; ++k) r *= k; return r; }

// P_l^m(x) and dP_l^m/dx for 0 <= m <= l <= 3 by the standard upward recurrences.
static void legendre(double x, double P[4][4], double dP[4][4]) {
  for (int l = 0; l < 4; ++l) for (int m = 0; m < 4; ++m) { P[l][m] = 0; dP[l][m] = 0; }
  double s2 = std::max(0.0, 1.0 - x * x);
  double s = std::sqrt(s2);
  for (int m = 0; m < 4; ++m) {
    double dfact = 1; for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= k;  // (2m-1)!!
    double pmm = ((m & 1) ? -1.0 : 1.0) * dfact * std::pow(s, m);
    P[m][m] = pmm;
    dP[m][m] = (m == 0) ? 0.0 : -m * x * pmm / s2;
    if (m + 1 < 4) {
      P[m + 1][m] = x * (2 * m + 1) * P[m][m];
      dP[m + 1][m] = (2 * m + 1) * (P[m][m] + x * dP[m][m]);
    }
    for (int l = m + 2; l < 4; ++l) {
      P[l][m] = ((2 * l - 1) * x * P[l - 1][m] - (l + m - 1) * P[l - 2][m]) / (l - m);
      dP[l][m] = ((2 * l - 1) * (P[l - 1][m] + x * dP[l - 1][m]) - (l + m - 1) * dP[l - 2][m]) / (l - m);
    }
  }
}

// Y_k(dir) for k < (deg+1)^2 and dY_k/d(dir) (as a function on R^3 through z and azimuth).
static void sh_basis(const double dir[3], int deg, double Y[16], double dY[16][3]) {
  double P[4][4], dP[4][4];
  double z = dir[2];
  legendre(z, P, dP);
  double az = std::atan2(dir[1], dir[0]);
  double rxy2 = dir[0] * dir[0] + dir[1] * dir[1];
  double daz[3] = {rxy2 > 0 ? -dir[1] / rxy2 : 0.0, rxy2 > 0 ? dir[0] / rxy2 : 0.0, 0.0};
  for (int l = 0; l <= deg; ++l)
    for (int m = -l; m <= l; ++m) {
      int am = std::abs(m);
      double K = std::sqrt((2 * l + 1) / (4 * kPi) * factorial(l - am) / factorial(l + am));
      double trig, dtrig;
      if (m > 0) { trig = std::sqrt(2.0) * std::cos(m * az); dtrig = -std::sqrt(2.0) * m * std::sin(m * az); }
      else if (m < 0) { trig = std::sqrt(2.0) * std::sin(am * az); dtrig = std::sqrt(2.0) * am * std::cos(am * az); }
      else { trig = 1.0; dtrig = 0.0; }
      int k = l * l + l + m;
      Y[k] = K * P[l][am] * trig;
      for (int c = 0; c < 3; ++c) dY[k][c] = K * P[l][am] * dtrig * daz[c];
      dY[k][2] += K * dP[l][am] * trig;
    }
}

// ===========================================================================
// Stage 1: preprocessing (Algorithm 1, preprocessing loop; Eq. lonlat_projection,
// Eq. arc_scaling; r_s = 3 sqrt(lambda_max(Sigma_arc))).
// ===========================================================================

struct Cfg {
  double near, blur, eps_T, alpha_max, cutoff, bg[3];
};

struct Pre {
  int valid, pole;
  double t[3], r, omega, phi;
  double qn[4], qnorm, R[3][3], M[3][3], S3[3][3];
  double J[2][3], T[2][3], Srad[2][2], Sarc[2][2];
  double conic[3];  // (a, b, c): m = a dx^2 + 2 b dx dy + c dy^2
  double rs;
  double dir[3], dist;
  double Y[16], dY[16][3];
  double craw[3], col[3];
  double g[3];      // HEALPix-frame unit vector of the Gaussian centre
};

static void quat_to_rot(const double q[4], double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

static void preprocess_one(const double mu[3], const double s[3], const double q[4],
                           const double* sh, int deg, const double W[9], const double b[3],
                           const Cfg& cfg, Pre& o) {
  std::memset(&o, 0, sizeof(o));
  // t = W mu + b
  for (int i = 0; i < 3; ++i) o.t[i] = W[3 * i] * mu[0] + W[3 * i + 1] * mu[1] + W[3 * i + 2] * mu[2] + b[i];
  double tx = o.t[0], ty = o.t[1], tz = o.t[2];
  double rho2 = tx * tx + tz * tz, rho = std::sqrt(rho2);
  o.r = std::sqrt(rho2 + ty * ty);
  // Reading: Gaussians with r <= near are culled (3DGS near plane).
  o.valid = o.r > cfg.near;
  if (!o.valid) return;
  o.g[0] = tz / o.r; o.g[1] = tx / o.r; o.g[2] = ty / o.r;
  o.pole = rho < 1e-9 * o.r;
  // Eq. lonlat_projection: omega = atan2(t_x, t_z), phi = atan2(t_y, sqrt(t_x^2 + t_z^2))
  // Reading at the pole: omega = 0 (the limiting frame of the omega = 0 meridian).
  o.omega = o.pole ? 0.0 : std::atan2(tx, tz);
  o.phi = std::atan2(ty, rho);
  if (o.pole) o.phi = ty > 0 ? kPi / 2 : -kPi / 2;
  // Sigma_3D = R diag(s^2) R^T with R = QuatToMat(q / |q|)
  o.qnorm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) o.qn[k] = q[k] / o.qnorm;
  quat_to_rot(o.qn, o.R);
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) o.M[i][j] = o.R[i][j] * s[j];
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
    double acc = 0; for (int k = 0; k < 3; ++k) acc += o.M[i][k] * o.M[j][k];
    o.S3[i][j] = acc;
  }
  double Wm[3][3];
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Wm[i][j] = W[3 * i + j];
  double r2 = o.r * o.r;
  double cphi = std::cos(o.phi);
  if (!o.pole) {
    // J = dPi/dt
    o.J[0][0] = tz / rho2; o.J[0][1] = 0.0; o.J[0][2] = -tx / rho2;
    o.J[1][0] = -tx * ty / (r2 * rho); o.J[1][1] = rho / r2; o.J[1][2] = -tz * ty / (r2 * rho);
  } else {
    // Reading at the pole: S_phi J is replaced by its omega = 0 limit E / r
    // (cos(phi) folded in); the backward is not defined there.
    o.J[0][0] = 1.0 / o.r; o.J[0][1] = 0; o.J[0][2] = 0;
    o.J[1][0] = 0; o.J[1][1] = 0; o.J[1][2] = -(ty > 0 ? 1.0 : -1.0) / o.r;
    cphi = 1.0;
  }
  // T = J W ; Sigma_rad = T Sigma3D T^T ; Sigma_arc = S_phi Sigma_rad S_phi
  for (int a = 0; a < 2; ++a) for (int j = 0; j < 3; ++j) {
    double acc = 0; for (int k = 0; k < 3; ++k) acc += o.J[a][k] * Wm[k][j];
    o.T[a][j] = acc;
  }
  for (int a = 0; a < 2; ++a) for (int c = 0; c < 2; ++c) {
    double acc = 0;
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) acc += o.T[a][i] * o.S3[i][j] * o.T[c][j];
    o.Srad[a][c] = acc;
  }
  double S[2] = {cphi, 1.0};
  for (int a = 0; a < 2; ++a) for (int c = 0; c < 2; ++c) o.Sarc[a][c] = S[a] * o.Srad[a][c] * S[c];
  // Reading: a low-pass term blur * I (the radian analogue of 3DGS's 0.3 px^2 dilation).
  o.Sarc[0][0] += cfg.blur; o.Sarc[1][1] += cfg.blur;
  double A = o.Sarc[0][0], B = o.Sarc[0][1], C = o.Sarc[1][1];
  double det = A * C - B * B;
  if (!(det > 0)) { o.valid = 0; return; }
  o.conic[0] = C / det; o.conic[1] = -B / det; o.conic[2] = A / det;
  double lmax = 0.5 * (A + C) + std::sqrt(0.25 * (A - C) * (A - C) + B * B);
  o.rs = 3.0 * std::sqrt(lmax);
  // view-dependent colour: SH at the world direction from the camera centre -W^T b
  double cam[3];
  for (int j = 0; j < 3; ++j) cam[j] = -(W[j] * b[0] + W[3 + j] * b[1] + W[6 + j] * b[2]);
  double dv[3] = {mu[0] - cam[0], mu[1] - cam[1], mu[2] - cam[2]};
  o.dist = std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  for (int j = 0; j < 3; ++j) o.dir[j] = dv[j] / o.dist;
  sh_basis(o.dir, deg, o.Y, o.dY);
  int K = (deg + 1) * (deg + 1);
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0;
    for (int k = 0; k < K; ++k) acc += sh[k * 3 + ch] * o.Y[k];
    o.craw[ch] = acc + 0.5;
    o.col[ch] = std::max(0.0, o.craw[ch]);
  }
}

// ===========================================================================
// Stage 3: spherical offset (Sec. 3.4): haversine great-circle distance and the
// bearing at the Gaussian centre; d = d_gc (sin beta, cos beta) = (east, north).
// ===========================================================================

struct Offset { double d[2], uw, uf, c, s, theta; };

static void spherical_offset(double omega_p, double sphp, double cphp, double omega_g, double sphg,
                             double cphg, Offset& o) {
  double dw = omega_p - omega_g;
  double phip = std::atan2(sphp, cphp), phig = std::atan2(sphg, cphg);
  double h = std::pow(std::sin(0.5 * (phip - phig)), 2) + cphg * cphp * std::pow(std::sin(0.5 * dw), 2);
  double dgc = 2.0 * std::asin(std::sqrt(std::min(1.0, std::max(0.0, h))));
  o.uw = std::sin(dw) * cphp;                         // numerator of the bearing
  o.uf = cphg * sphp - sphg * cphp * std::cos(dw);    // denominator of the bearing
  o.c = sphg * sphp + cphg * cphp * std::cos(dw);     // cos of the great-circle distance
  o.s = std::sqrt(o.uw * o.uw + o.uf * o.uf);
  o.theta = dgc;
  double beta = std::atan2(o.uw, o.uf);
  o.d[0] = dgc * std::sin(beta);
  o.d[1] = dgc * std::cos(beta);
}

// ===========================================================================
// Tiles (Sec. 3.1, Table "resolution"): tile = ancestor at order k_t = k - b.
// Membership (reading, conservative 3-sigma support): tile t is listed for
// Gaussian i iff t is active and c_t . g_i >= cos(min(pi, r_s + rho + 1e-7)).
// ===========================================================================

// rho(k, b): largest angle between a tile centre and a pixel centre of that
// tile, rounded up to a multiple of 2^-20 rad.
static double tile_rho(int k, int b) {
  i64 nside = 1LL << k, nside_t = 1LL << (k - b);
  i64 ntile = 12 * nside_t * nside_t, per = 1LL << (2 * b);
  double worst = 1.0;
#pragma omp parallel for reduction(min : worst) schedule(static)
  for (i64 t = 0; t < ntile; ++t) {
    double ct[3]; pix2vec_nest(nside_t, t, ct);
    for (i64 j = 0; j < per; ++j) {
      double pv[3]; pix2vec_nest(nside, t * per + j, pv);
      double dt = ct[0] * pv[0] + ct[1] * pv[1] + ct[2] * pv[2];
      if (dt < worst) worst = dt;
    }
  }
  double rho = std::acos(std::min(1.0, worst));
  return std::ceil(rho * 1048576.0) / 1048576.0;
}

// Algorithm 3 (QueryDiscRing) at order k_t: candidate tiles whose centres may lie
// within angle R of g. Returns NESTED tile indices.
static void query_disc_ring(i64 nside_t, const double g[3], double R, std::vector<i64>& out) {
  out.clear();
  double zc = g[2];
  double phic = std::atan2(zc, std::sqrt(g[0] * g[0] + g[1] * g[1]));
  double omc = std::atan2(g[1], g[0]);
  double phimin = std::max(-kPi / 2, phic - R), phimax = std::min(kPi / 2, phic + R);
  // z = sin(latitude) (Algorithm 3)
  double zmin = std::sin(phimin), zmax = std::sin(phimax);
  // ZtoRingRange: continuous ring number of a latitude, then +-1 ring of margin
  auto ring_of = [&](double z) {
    double N = (double)nside_t;
    if (z > 2.0 / 3.0) return N * std::sqrt(3.0 * (1.0 - z));
    if (z < -2.0 / 3.0) return 4.0 * N - N * std::sqrt(3.0 * (1.0 + z));
    return N * (2.0 - 1.5 * z);
  };
  i64 ilo = std::max<i64>(1, (i64)std::floor(ring_of(zmax)) - 1);
  i64 ihi = std::min<i64>(4 * nside_t - 1, (i64)std::ceil(ring_of(zmin)) + 1);
  double cosR = std::cos(std::min(kPi, R));
  for (i64 i = ilo; i <= ihi; ++i) {
    Ring rg = ring_info(nside_t, i);
    if (rg.z < zmin - 1e-12 || rg.z > zmax + 1e-12) continue;
    double delta = std::sqrt(std::max(0.0, 1 - zc * zc)) * std::sqrt(std::max(0.0, 1 - rg.z * rg.z));
    i64 jlo = 0, jhi = -1;
    bool full = false;
    if (delta < 1e-12) {
      if (zc * rg.z >= cosR) full = true; else continue;
    } else {
      // Eq. ring_phi_range: cos(d omega) = (cos r_s - z_c z_ring) / (sqrt(1-z_c^2) sqrt(1-z_ring^2))
      double cw = (cosR - zc * rg.z) / delta;
      if (cw <= -1) full = true;
      else if (cw <= 1) {
        double dw = std::acos(std::min(1.0, std::max(-1.0, cw)));
        jlo = (i64)std::floor((omc - dw - rg.phi0) * rg.npix / (2 * kPi));
        jhi = (i64)std::ceil((omc + dw - rg.phi0) * rg.npix / (2 * kPi));
        if (jhi - jlo + 1 >= rg.npix) full = true;
      } else continue;
    }
    if (full) { jlo = 0; jhi = rg.npix - 1; }
    for (i64 j = jlo; j <= jhi; ++j) {
      double z, sth, ph; ring2zphi(nside_t, i, pmod(j, rg.npix), z, sth, ph);
      out.push_back(zphi2pix_nest(nside_t, z, ph));
    }
  }
}

// Enumeration radius for the membership test c . g >= cos(R) (Algorithm 3 enumerates the
// directions within a radius of a unit centre). The stored centre g is unit length only to
// its rounding, and the test holds for the directions within acos(cos R / |g|) of g / |g|:
// a little more than R when |g| > 1, by about (|g| - 1) / tan R. With
// h = (1 - cos R / |g|) / 2 = (|g| - 1 + 2 sin^2(R / 2)) / (2 |g|), that angle is 2 asin sqrt(h).
static double dot_disc_radius(double R, double glen) {
  if (R >= kPi) return kPi;
  const double s = std::sin(0.5 * R);
  const double h = (glen - 1.0 + 2.0 * s * s) / (2.0 * glen);
  if (h >= 1.0) return kPi;
  return std::max(R, h > 0.0 ? 2.0 * std::asin(std::sqrt(h)) : 0.0);
}

// Algorithm 3 candidates of the disc {c : c . g >= cos(R)} (g as stored, near unit length):
// the enumeration runs about g / |g| with the radius of that disc plus 1e-9.
static void query_dot_disc(i64 nside, const double g[3], double R, std::vector<i64>& out) {
  const double glen = std::sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  const double gu[3] = {g[0] / glen, g[1] / glen, g[2] / glen};
  query_disc_ring(nside, gu, std::min(kPi, dot_disc_radius(R, glen) + 1e-9), out);
}

// Membership of a Gaussian (centre g, radius r_s) in the tile with centre ct.
static bool tile_member_at(const double ct[3], const double g[3], double rs, double rho) {
  double dt = ct[0] * g[0] + ct[1] * g[1] + ct[2] * g[2];
  return dt >= std::cos(std::min(kPi, rs + rho + 1e-7));
}

static bool tile_member(i64 nside_t, i64 t, const double g[3], double rs, double rho) {
  double ct[3]; pix2vec_nest(nside_t, t, ct);
  return tile_member_at(ct, g, rs, rho);
}

// Per Gaussian: the sorted set of listed tiles (RING candidates, exact test).
static void tiles_of(i64 nside_t, const double g[3], double rs, double rho, const u8* active,
                     std::vector<i64>& out) {
  std::vector<i64> cand;
  query_dot_disc(nside_t, g, std::min(kPi, rs + rho + 1e-7), cand);
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  out.clear();
  for (i64 t : cand)
    if (active[t] && tile_member(nside_t, t, g, rs, rho)) out.push_back(t);
}

// Emission + sort (Algorithm 1): pairs ((tile, depth), i) ordered by tile, then
// increasing radial depth (as float32 bits), then Gaussian index (reading).
struct ListCSR { std::vector<i64> start; std::vector<i64> ids; };

static void build_lists(i64 nside_t, i64 P, const double* g, const double* rs, const int* valid,
                        const u32* depth_bits, double rho, const u8* active, ListCSR& L) {
  i64 ntile = 12 * nside_t * nside_t;
  std::vector<std::vector<i64>> per(P);
#pragma omp parallel for schedule(dynamic, 64)
  for (i64 i = 0; i < P; ++i)
    if (valid[i]) tiles_of(nside_t, g + 3 * i, rs[i], rho, active, per[i]);
  struct Pair { i64 tile; u32 depth; i64 id; };
  std::vector<Pair> pairs;
  for (i64 i = 0; i < P; ++i) for (i64 t : per[i]) pairs.push_back({t, depth_bits[i], i});
  std::stable_sort(pairs.begin(), pairs.end(), [](const Pair& a, const Pair& b) {
    if (a.tile != b.tile) return a.tile < b.tile;
    if (a.depth != b.depth) return a.depth < b.depth;
    return a.id < b.id;
  });
  L.start.assign(ntile + 1, 0);
  for (auto& p : pairs) L.start[p.tile + 1]++;
  for (i64 t = 0; t < ntile; ++t) L.start[t + 1] += L.start[t];
  L.ids.resize(pairs.size());
  for (size_t j = 0; j < pairs.size(); ++j) L.ids[j] = pairs[j].id;
}

// ===========================================================================
// Per-pixel compositing (Algorithm 1, rendering loop; Eq. unified_rendering).
// Readings: alpha = 0 beyond the 3-sigma ellipse (m > cutoff); alpha clamped to
// alpha_max; the entry that takes T below eps is included, then the loop breaks.
// ===========================================================================

struct GaussView {  // what compositing needs per Gaussian
  double omega, sphg, cphg, conic[3], opac, col[3], r;
};

struct PixOut { double C[3], T, D; i64 last; };   // D: composited inverse radial depth

// Forward at one pixel; optionally records alpha, T before each entry and exp(-m/2).
static void composite_pixel(double omega_p, double sphp, double cphp, const i64* ids, i64 n,
                            const std::vector<GaussView>& G, const Cfg& cfg, PixOut& out,
                            std::vector<double>* alphas, std::vector<double>* Ts,
                            std::vector<double>* Gs) {
  double T = 1.0, C[3] = {0, 0, 0}, D = 0.0;
  i64 j = 0;
  for (; j < n; ++j) {
    const GaussView& gv = G[ids[j]];
    Offset o;
    spherical_offset(omega_p, sphp, cphp, gv.omega, gv.sphg, gv.cphg, o);
    double m = gv.conic[0] * o.d[0] * o.d[0] + 2 * gv.conic[1] * o.d[0] * o.d[1] + gv.conic[2] * o.d[1] * o.d[1];
    double Gm = std::exp(-0.5 * m);
    double a = (m > cfg.cutoff) ? 0.0 : std::min(cfg.alpha_max, gv.opac * Gm);
    if (alphas) { alphas->push_back(a); Ts->push_back(T); Gs->push_back(Gm); }
    for (int c = 0; c < 3; ++c) C[c] += T * a * gv.col[c];
    D += T * a / gv.r;                        // depth channel: inverse radial depth (Sec. 3.2)
    T *= (1.0 - a);
    if (T < cfg.eps_T) { ++j; break; }
  }
  for (int c = 0; c < 3; ++c) out.C[c] = C[c] + T * cfg.bg[c];
  out.T = T; out.D = D; out.last = j;
}

// ---------------------------------------------------------------------------
// Decisions that single precision may take the other way (test bookkeeping, not part
// of the method). A rasterizer working in FP32 decides m <= cutoff and T < eps from
// values within a few parts in 1e6 (m) and 1e5 (T) of these FP64 ones. Where the FP64
// value lies within the bands below of its threshold, both outcomes are results of
// the method at that precision. composite_branches follows both outcomes of every such
// decision, up to kMaxFlips of them per pixel, and returns each resulting pixel value
// (a leaf); the leaf with the FP64 outcome of every decision comes first and equals
// composite_pixel's result. Flags: bit 0, a cutoff decision in its band; bit 1, a
// termination decision in its band; bit 2, more such decisions than kMaxFlips (the
// later ones take the FP64 outcome only, so the leaves do not cover every outcome).
// ---------------------------------------------------------------------------
constexpr double kAmbCut = 2e-5;     // |m - cutoff| < kAmbCut * cutoff
constexpr double kAmbTerm = 1e-4;    // |T - eps| < kAmbTerm * eps
constexpr int kMaxFlips = 4;
constexpr int kMaxLeaves = 1 << kMaxFlips;

struct Leaf { double C[3], T, D; i64 last; };

struct BranchCtx {
  double omega_p, sphp, cphp;
  const i64* ids;
  i64 n;
  const std::vector<GaussView>* G;
  const Cfg* cfg;
  Leaf leaves[kMaxLeaves];
  int nleaves;   // leaves[0] is the FP64 path's; the others follow from index 1
  int amb;
};

static void emit_leaf(BranchCtx& X, bool primary, const double C[3], double T, double D, i64 last) {
  int slot = primary ? 0 : X.nleaves++;
  Leaf& L = X.leaves[slot];
  for (int c = 0; c < 3; ++c) L.C[c] = C[c] + T * X.cfg->bg[c];
  L.T = T; L.D = D; L.last = last;
}

// From list position j with state (T, C, D); nd band decisions met so far on this path
// (each path meets at most kMaxFlips, so there are at most kMaxLeaves leaves).
// forced_in >= 0 imposes the cutoff outcome of entry j (the other branch of a decision
// the caller met).
static void composite_branches(BranchCtx& X, i64 j, double T, const double C0[3], double D, int nd,
                               bool primary, int forced_in) {
  const Cfg& cfg = *X.cfg;
  double C[3] = {C0[0], C0[1], C0[2]};
  for (; j < X.n; ++j, forced_in = -1) {
    const GaussView& gv = (*X.G)[X.ids[j]];
    Offset o;
    spherical_offset(X.omega_p, X.sphp, X.cphp, gv.omega, gv.sphg, gv.cphg, o);
    double m = gv.conic[0] * o.d[0] * o.d[0] + 2 * gv.conic[1] * o.d[0] * o.d[1] + gv.conic[2] * o.d[1] * o.d[1];
    bool in = !(m > cfg.cutoff);
    if (forced_in >= 0) {
      in = forced_in != 0;
    } else if (std::fabs(m - cfg.cutoff) < kAmbCut * cfg.cutoff) {
      X.amb |= 1;
      if (nd < kMaxFlips) composite_branches(X, j, T, C, D, ++nd, false, in ? 0 : 1);
      else X.amb |= 4;
    }
    double a = in ? std::min(cfg.alpha_max, gv.opac * std::exp(-0.5 * m)) : 0.0;
    for (int c = 0; c < 3; ++c) C[c] += T * a * gv.col[c];
    D += T * a / gv.r;
    T *= (1.0 - a);
    // only an entry that changes T can end the loop (on the FP64 path T >= eps whenever
    // a == 0; on a path that went on past a band decision T may already be below eps)
    bool stop = a > 0 && T < cfg.eps_T;
    if (a > 0 && std::fabs(T - cfg.eps_T) < kAmbTerm * cfg.eps_T) {
      X.amb |= 2;
      if (nd < kMaxFlips) {
        ++nd;
        if (stop) composite_branches(X, j + 1, T, C, D, nd, false, -1);   // went on
        else emit_leaf(X, false, C, T, D, j + 1);                          // stopped here
      } else {
        X.amb |= 4;
      }
    }
    if (stop) { emit_leaf(X, primary, C, T, D, j + 1); return; }
  }
  emit_leaf(X, primary, C, T, D, X.n);
}

static void composite_pixel_branches(double omega_p, double sphp, double cphp, const i64* ids, i64 n,
                                     const std::vector<GaussView>& G, const Cfg& cfg, BranchCtx& X) {
  X.omega_p = omega_p; X.sphp = sphp; X.cphp = cphp;
  X.ids = ids; X.n = n; X.G = &G; X.cfg = &cfg;
  X.nleaves = 1; X.amb = 0;
  const double C0[3] = {0, 0, 0};
  composite_branches(X, 0, 1.0, C0, 0.0, 0, true, -1);
}

static void pixel_lonlat(i64 nside, i64 p, double& omega_p, double& sphp, double& cphp) {
  double z, sth, phi;
  pix2zphi_nest(nside, p, z, sth, phi, nullptr);
  omega_p = phi; sphp = z; cphp = sth;   // latitude phi_p = pi/2 - colatitude
}

// ---------------------------------------------------------------------------
// Backward helpers (Sec. 3.2, Eqs. backward_lat_scale and grad_via_J_S).
// ---------------------------------------------------------------------------

// dJ_ab / dt_k for J = dPi/dt of Eq. lonlat_projection.
static void dJ_dt(const double t[3], double dJ[2][3][3]) {
  double tx = t[0], ty = t[1], tz = t[2];
  double rho2 = tx * tx + tz * tz, rho = std::sqrt(rho2), r2 = rho2 + ty * ty;
  double rho4 = rho2 * rho2;
  // row 0: (tz/rho^2, 0, -tx/rho^2)
  dJ[0][0][0] = -2 * tz * tx / rho4; dJ[0][0][1] = 0; dJ[0][0][2] = (tx * tx - tz * tz) / rho4;
  dJ[0][1][0] = 0; dJ[0][1][1] = 0; dJ[0][1][2] = 0;
  dJ[0][2][0] = (tx * tx - tz * tz) / rho4; dJ[0][2][1] = 0; dJ[0][2][2] = 2 * tx * tz / rho4;
  // row 1: (-tx ty h, rho/r^2, -tz ty h), h = 1/(r^2 rho)
  double h = 1.0 / (r2 * rho);
  double dh[3] = {-2 * tx / (r2 * r2 * rho) - tx / (r2 * rho * rho2),
                  -2 * ty / (r2 * r2 * rho),
                  -2 * tz / (r2 * r2 * rho) - tz / (r2 * rho * rho2)};
  double dtxty[3] = {ty, tx, 0}, dtzty[3] = {0, tz, ty};
  for (int k = 0; k < 3; ++k) {
    dJ[1][0][k] = -dtxty[k] * h - tx * ty * dh[k];
    dJ[1][2][k] = -dtzty[k] * h - tz * ty * dh[k];
  }
  dJ[1][1][0] = tx / (rho * r2) - 2 * rho * tx / (r2 * r2);
  dJ[1][1][1] = -2 * rho * ty / (r2 * r2);
  dJ[1][1][2] = tz / (rho * r2) - 2 * rho * tz / (r2 * r2);
}

// Per-pixel partial derivatives of d w.r.t. the Gaussian's (omega, phi),
// differentiating the haversine/bearing offset: d = theta (uw, uf)/s with
// theta = atan2(s, c), s = |(uw, uf)| (the same quantities as in the bearing).
static void offset_grad(double omega_p, double cphp, double omega_g, double sphg, double cphg,
                        const Offset& o, double dd_dw[2], double dd_dph[2]) {
  double dw = omega_p - omega_g;
  double sdw = std::sin(dw), cdw = std::cos(dw);
  double duw[2] = {-cphp * cdw, 0.0};                 // d(uw)/d(omega_g, phi_g)
  double duf[2] = {-sphg * cphp * sdw, -o.c};         // d(uf)/d(...)
  double dc[2] = {cphg * cphp * sdw, o.uf};           // d(c)/d(...)
  double s = o.s, c = o.c, th = std::atan2(s, c);
  double ss = s * s + c * c;
  double u[2] = {o.uw, o.uf};
  double f_over_s;  // th / s
  double kfac;      // (c s/ss - th) / s^3, so that d(th/s)/du_j = kfac u_j
  if (s < 1e-4 && c > 0) { f_over_s = 1.0 + s * s / 6.0; kfac = -2.0 / 3.0 - s * s / 5.0; }
  else { f_over_s = th / s; kfac = (c * s / ss - th) / (s * s * s); }
  for (int a = 0; a < 2; ++a) {
    double dua[2] = {duw[a], duf[a]};
    double out[2];
    double kdot = kfac * (u[0] * dua[0] + u[1] * dua[1]);
    for (int i = 0; i < 2; ++i)
      out[i] = f_over_s * dua[i] + u[i] * kdot + (s > 0 ? u[i] / s : 0.0) * (-s / ss) * dc[a];
    if (a == 0) { dd_dw[0] = out[0]; dd_dw[1] = out[1]; }
    else { dd_dph[0] = out[0]; dd_dph[1] = out[1]; }
  }
}

// ---------------------------------------------------------------------------
// HEALPix-SSIM (Sec. 4.1; masked mean Eq. supp_hssim_eval) helpers.
// Readings: window W(q) = q and its in-mask 8- (or 7-) neighbours; weights
// exp(-theta^2 / (2 sigma^2)) of the great-circle distance between pixel centres,
// sigma = 1.5 sqrt(Omega_pix), normalised over W(q); SSIM constants C1 = 0.01^2,
// C2 = 0.03^2; h_q = mean over channels; loss = (1 - lambda) L1 + lambda (1 - HSSIM).
// ---------------------------------------------------------------------------

struct Window { int n; i64 idx[9]; double w[9]; };

static void hssim_window(i64 nside, i64 q, const u8* mask, Window& W) {
  i64 nb[8];
  neighbours_nest(nside, q, nb);
  double Om = 4.0 * kPi / (12.0 * (double)nside * nside);
  double sig2 = 2.25 * Om;
  double cq[3]; pix2vec_nest(nside, q, cq);
  W.n = 0;
  W.idx[W.n] = q; W.w[W.n] = 1.0; W.n++;
  for (int k = 0; k < 8; ++k) {
    if (nb[k] < 0 || !mask[nb[k]]) continue;
    double cn[3]; pix2vec_nest(nside, nb[k], cn);
    double cr[3] = {cq[1] * cn[2] - cq[2] * cn[1], cq[2] * cn[0] - cq[0] * cn[2], cq[0] * cn[1] - cq[1] * cn[0]};
    double th = std::atan2(std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]),
                           cq[0] * cn[0] + cq[1] * cn[1] + cq[2] * cn[2]);
    W.idx[W.n] = nb[k]; W.w[W.n] = std::exp(-th * th / (2.0 * sig2)); W.n++;
  }
  double Z = 0; for (int j = 0; j < W.n; ++j) Z += W.w[j];
  for (int j = 0; j < W.n; ++j) W.w[j] /= Z;
}

static const double kC1 = 1e-4, kC2 = 9e-4;

// Local SSIM value per channel and its partials w.r.t. (mu_x, sigma_x^2, sigma_xy).
static double ssim_local(const Window& W, const double* I, const double* Gt, int ch, double* dmu,
                         double* dvar, double* dcov, double* mux_o, double* muy_o) {
  double mx = 0, my = 0, xx = 0, yy = 0, xy = 0;
  for (int j = 0; j < W.n; ++j) {
    double x = I[3 * W.idx[j] + ch], y = Gt[3 * W.idx[j] + ch], w = W.w[j];
    mx += w * x; my += w * y; xx += w * x * x; yy += w * y * y; xy += w * x * y;
  }
  double vx = xx - mx * mx, vy = yy - my * my, cxy = xy - mx * my;
  double A1 = 2 * mx * my + kC1, A2 = 2 * cxy + kC2, B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
  double s = (A1 * A2) / (B1 * B2);
  if (dmu) {
    *dmu = (2 * my * A2 * B1 - A1 * A2 * 2 * mx) / (B1 * B1 * B2);
    *dvar = -A1 * A2 / (B1 * B2 * B2);
    *dcov = 2 * A1 / (B1 * B2);
    *mux_o = mx; *muy_o = my;
  }
  return s;
}

// ===========================================================================
// extern "C" entry points (called from Python through ctypes)
// ===========================================================================

// ===========================================================================
// NESTED quadtree tile query (Algorithm 2; Sec. 3.3, "NESTED Quadtree
// Traversal"). A depth-first search from the 12 base pixels: each node (p, o)
// is classified by the haversine distance d from the disc centre to the node
// centre against r_s and PixRad(o): zone 0 (d > r_s + PixRad, pruned), 3 (fully
// inside, d + PixRad <= r_s), 2 (centre inside, d <= r_s), 1 (partial). A node of
// zone >= 2 at or below the tile order adds its tile; otherwise it is refined
// down to k_max = tile order + log2 f, where a zone-1 node adds its tile.
// Reading (the paper does not define PixRad): the largest angle from a node
// centre to its boundary over all nodes of order o, the boundary sampled at 9
// points along each edge (corners included), rounded up to 2^-20 rad.
// ===========================================================================

static double angle_between(const double a[3], const double b[3]) {
  const double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
  return std::atan2(std::sqrt(cx * cx + cy * cy + cz * cz), a[0] * b[0] + a[1] * b[1] + a[2] * b[2]);
}

static double pixrad_order(int o) {
  static std::mutex mu;
  static std::map<int, double> cache;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(o);
    if (it != cache.end()) return it->second;
  }
  const i64 nside = 1LL << o, npix = 12 * nside * nside;
  const double N = (double)nside;
  double mx = 0.0;
#pragma omp parallel for reduction(max : mx) schedule(static)
  for (i64 p = 0; p < npix; ++p) {
    XYF c = nest2xyf(nside, p);
    double ctr[3]; pix2vec_nest(nside, p, ctr);
    for (int t = 0; t <= 8; ++t) {
      const double s = t / 8.0;
      const double uv[4][2] = {{c.x + s, (double)c.y}, {c.x + s, c.y + 1.0}, {(double)c.x, c.y + s}, {c.x + 1.0, c.y + s}};
      for (int e = 0; e < 4; ++e) {
        double q[3]; face_uv2vec(c.f, uv[e][0] / N, uv[e][1] / N, q);
        mx = std::max(mx, angle_between(ctr, q));
      }
    }
  }
  const double r = std::ceil(mx * 1048576.0) / 1048576.0;
  std::lock_guard<std::mutex> lk(mu);
  cache[o] = r;
  return r;
}

static double haversine(double lon1, double lat1, double lon2, double lat2) {
  const double a = std::sin(0.5 * (lat2 - lat1)), b = std::sin(0.5 * (lon2 - lon1));
  const double h = a * a + std::cos(lat1) * std::cos(lat2) * b * b;
  return 2.0 * std::asin(std::min(1.0, std::sqrt(h)));
}

// Tiles at order k touched by the disc (centre g, radius rs) with refinement down to kmax.
static void query_disc_nested(int k, int kmax, const double g[3], double rs, std::vector<i64>& tiles) {
  const double lon = std::atan2(g[1], g[0]), lat = std::atan2(g[2], std::sqrt(g[0] * g[0] + g[1] * g[1]));
  struct Node { i64 p; int o; };
  std::vector<Node> stack;
  for (i64 p = 0; p < 12; ++p) stack.push_back({p, 0});
  tiles.clear();
  while (!stack.empty()) {
    const Node nd = stack.back();
    stack.pop_back();
    double z, sth, ph; pix2zphi_nest(1LL << nd.o, nd.p, z, sth, ph, nullptr);
    const double d = haversine(lon, lat, ph, std::atan2(z, sth));
    const double pr = pixrad_order(nd.o);
    const int zone = d > rs + pr ? 0 : (d + pr <= rs ? 3 : (d <= rs ? 2 : 1));
    if (zone == 0) continue;
    if (zone >= 2 && nd.o >= k) tiles.push_back(nd.p >> (2 * (nd.o - k)));
    else if (nd.o < kmax) for (i64 c = 0; c < 4; ++c) stack.push_back({4 * nd.p + c, nd.o + 1});
    else tiles.push_back(nd.p >> (2 * (nd.o - k)));
  }
  std::sort(tiles.begin(), tiles.end());
  tiles.erase(std::unique(tiles.begin(), tiles.end()), tiles.end());
}

// ===========================================================================
// Sphere <-> image resampling: the rendered map to a camera image
// (Eq. camera_synthesis) and a camera image to the HEALPix grid
// (Eqs. supp_image_to_healpix, supp_hssim_mask), with the camera models of
// Sec. D.1 (Eq. persp_sphere; Eqs. fish_weff, fish_sphere, imaging_region,
// semi_axes; the omnidirectional mapping).
// Readings (the paper names the operations, not the schemes):
//  - image samples sit at pixel centres (i + 1/2, j + 1/2);
//  - Interp_H is HEALPix ring-bilinear interpolation: along each of the two
//    rings that bracket the colatitude, linear in longitude between the two
//    pixel centres that bracket it; between the rings, linear in colatitude.
//    Above the first ring (below the last) it runs linearly in colatitude to a
//    pole value, the mean of that ring's 4 pixels;
//  - the image is sampled bilinearly between pixel centres, clamped at the
//    image edges and, for the panorama, wrapped in longitude;
//  - each camera's formula is taken as printed (image v grows with d_y for
//    the pinhole and fisheye; the panorama has phi = pi/2 on its top row).
// The HEALPix map lives in the camera frame: HEALPix (X, Y, Z) = (d_z, d_x, d_y).
// ===========================================================================

struct ImgCam { int kind; double W, H, fovx, fovy, ppx, ppy; };   // pp: pinhole principal point offset

// P_C: image point (u, v) -> unit camera direction d; false outside D_C.
static bool img_to_dir(const ImgCam& c, double u, double v, double d[3]) {
  if (c.kind == CAM_PINHOLE) {
    double fx = c.W / (2.0 * std::tan(0.5 * c.fovx * kPi / 180.0));
    double fy = c.H / (2.0 * std::tan(0.5 * c.fovy * kPi / 180.0));
    double x = (u - 0.5 * c.W * (1.0 + c.ppx)) / fx, y = (v - 0.5 * c.H * (1.0 + c.ppy)) / fy;
    double n = std::sqrt(x * x + y * y + 1.0);
    d[0] = x / n; d[1] = y / n; d[2] = 1.0 / n;
    return u >= 0 && u <= c.W && v >= 0 && v <= c.H;
  }
  if (c.kind == CAM_FISHEYE) {
    double fx = c.W / kPi, fy = c.H / kPi;
    double mx = (u - 0.5 * c.W) / fx, my = (v - 0.5 * c.H) / fy;
    double rm = std::sqrt(mx * mx + my * my);
    if (rm > 0.5 * kPi) return false;                 // outside the ellipse with a = fx pi/2, b = fy pi/2
    double gam = std::atan2(my, mx);
    double wx = c.fovx / 180.0, wy = c.fovy / 180.0;
    double weff = std::sqrt(std::pow(wx * std::cos(gam), 2) + std::pow(wy * std::sin(gam), 2));
    double psi = rm * weff;
    d[0] = std::sin(psi) * std::cos(gam); d[1] = std::sin(psi) * std::sin(gam); d[2] = std::cos(psi);
    return true;
  }
  double om = 2.0 * kPi * u / c.W - kPi, ph = 0.5 * kPi - kPi * v / c.H;
  d[0] = std::cos(ph) * std::sin(om); d[1] = std::sin(ph); d[2] = std::cos(ph) * std::cos(om);
  return true;
}

// Pi_C^{-1}: camera direction d -> image point (u, v); false outside D_C (the
// same test as the FoV mask, so the resampled mask is M_C itself).
static bool dir_to_img(const ImgCam& c, const double d[3], double& u, double& v) {
  if (c.kind == CAM_PINHOLE) {
    if (camera_margin(c.kind, c.fovx, c.fovy, c.ppx, c.ppy, d) < 0) return false;
    double fx = c.W / (2.0 * std::tan(0.5 * c.fovx * kPi / 180.0));
    double fy = c.H / (2.0 * std::tan(0.5 * c.fovy * kPi / 180.0));
    u = 0.5 * c.W * (1.0 + c.ppx) + fx * d[0] / d[2]; v = 0.5 * c.H * (1.0 + c.ppy) + fy * d[1] / d[2];
    return true;
  }
  if (c.kind == CAM_FISHEYE) {
    if (camera_margin(c.kind, c.fovx, c.fovy, 0.0, 0.0, d) < 0) return false;
    double psi = std::atan2(std::sqrt(d[0] * d[0] + d[1] * d[1]), d[2]);
    double gam = std::atan2(d[1], d[0]);
    double wx = c.fovx / 180.0, wy = c.fovy / 180.0;
    double weff = std::sqrt(std::pow(wx * std::cos(gam), 2) + std::pow(wy * std::sin(gam), 2));
    double rm = psi / weff;
    u = 0.5 * c.W + (c.W / kPi) * rm * std::cos(gam); v = 0.5 * c.H + (c.H / kPi) * rm * std::sin(gam);
    return true;
  }
  double om = std::atan2(d[0], d[2]), ph = std::asin(std::max(-1.0, std::min(1.0, d[1])));
  u = c.W * (om + kPi) / (2.0 * kPi); v = c.H * (0.5 * kPi - ph) / kPi;
  return true;
}

static double ring_theta(i64 nside, i64 i) { Ring R = ring_info(nside, i); return std::atan2(R.sth, R.z); }

// NESTED index of pixel j (mod n) of ring i.
static i64 ring_pixel_nest(i64 nside, i64 i, i64 j) {
  Ring R = ring_info(nside, i);
  double z, sth, phi; ring2zphi(nside, i, pmod(j, R.npix), z, sth, phi);
  return zphi2pix_nest(nside, z, phi);
}

// The two pixels of ring i that bracket longitude phi, with linear weights.
static void ring_bracket(i64 nside, i64 i, double phi, i64 pix[2], double w[2]) {
  Ring R = ring_info(nside, i);
  double t = (phi - R.phi0) * (double)R.npix / (2.0 * kPi);
  double j0 = std::floor(t), f = t - j0;
  pix[0] = ring_pixel_nest(nside, i, (i64)j0); pix[1] = ring_pixel_nest(nside, i, (i64)j0 + 1);
  w[0] = 1.0 - f; w[1] = f;
}

// Interp_H weights at colatitude theta in [0, pi], longitude phi: 4 NESTED pixels
// (a pixel may repeat) whose weights sum to 1.
static void interp_weights(i64 nside, double theta, double phi, i64 pix[4], double w[4]) {
  const i64 nr = 4 * nside - 1;
  i64 lo = 0, hi = nr;                                  // last ring with theta_i <= theta (0: above ring 1)
  while (lo < hi) { i64 mid = (lo + hi + 1) / 2; if (ring_theta(nside, mid) <= theta) lo = mid; else hi = mid - 1; }
  const i64 ir = lo;
  if (ir >= 1 && ir < nr) {
    double t0 = ring_theta(nside, ir), t1 = ring_theta(nside, ir + 1);
    double wt = (theta - t0) / (t1 - t0);
    i64 a[2], b[2]; double wa[2], wb[2];
    ring_bracket(nside, ir, phi, a, wa); ring_bracket(nside, ir + 1, phi, b, wb);
    pix[0] = a[0]; pix[1] = a[1]; pix[2] = b[0]; pix[3] = b[1];
    w[0] = (1 - wt) * wa[0]; w[1] = (1 - wt) * wa[1]; w[2] = wt * wb[0]; w[3] = wt * wb[1];
    return;
  }
  // polar caps: ring 1 (or 4N-1) has 4 pixels; the pole value is their mean
  const i64 ring = (ir == 0) ? 1 : nr;
  double tr = ring_theta(nside, ring);
  double wr = (ir == 0) ? theta / tr : (kPi - theta) / (kPi - tr);   // weight of the ring's bracket
  i64 a[2]; double wa[2];
  ring_bracket(nside, ring, phi, a, wa);
  for (int j = 0; j < 4; ++j) { pix[j] = ring_pixel_nest(nside, ring, j); w[j] = 0.25 * (1.0 - wr); }
  for (int q = 0; q < 2; ++q)
    for (int j = 0; j < 4; ++j)
      if (pix[j] == a[q]) w[j] += wr * wa[q];
}

static void dir_to_healpix_angles(const double d[3], double& theta, double& phi) {
  const double X = d[2], Y = d[0], Z = d[1];
  theta = std::atan2(std::sqrt(X * X + Y * Y), Z);
  phi = std::atan2(Y, X);
  if (phi < 0) phi += 2.0 * kPi;
}

// Bilinear image sample at (u, v): taps at pixel centres, clamped (panorama: wrapped in u).
static void image_sample(const double* img, const ImgCam& c, double u, double v, double out[3]) {
  const i64 W = (i64)c.W, H = (i64)c.H;
  double x = u - 0.5, y = v - 0.5;
  double x0 = std::floor(x), y0 = std::floor(y), fx = x - x0, fy = y - y0;
  i64 xs[2] = {(i64)x0, (i64)x0 + 1}, ys[2] = {(i64)y0, (i64)y0 + 1};
  for (int q = 0; q < 2; ++q) {
    xs[q] = (c.kind == CAM_FULL) ? pmod(xs[q], W) : std::max<i64>(0, std::min<i64>(W - 1, xs[q]));
    ys[q] = std::max<i64>(0, std::min<i64>(H - 1, ys[q]));
  }
  const double wx[2] = {1 - fx, fx}, wy[2] = {1 - fy, fy};
  out[0] = out[1] = out[2] = 0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int ch = 0; ch < 3; ++ch) out[ch] += wy[a] * wx[b] * img[3 * (ys[a] * W + xs[b]) + ch];
}

extern "C" {

void or_pix2vec_nest(i64 nside, i64 n, const i64* p, double* v) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i) pix2vec_nest(nside, p[i], v + 3 * i);
}
void or_pix2ang_nest(i64 nside, i64 n, const i64* p, double* theta, double* phi) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i) {
    double z, sth, ph; pix2zphi_nest(nside, p[i], z, sth, ph, nullptr);
    theta[i] = std::atan2(sth, z); phi[i] = ph;
  }
}
void or_vec2pix_nest(i64 nside, i64 n, const double* v, i64* p) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i) p[i] = vec2pix_nest(nside, v + 3 * i);
}
void or_ang2pix_nest(i64 nside, i64 n, const double* theta, const double* phi, i64* p) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i) p[i] = zphi2pix_nest(nside, std::cos(theta[i]), phi[i]);
}
void or_nest2ring(i64 nside, i64 n, const i64* in, i64* out) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i) out[i] = nest2ring(nside, in[i]);
}
void or_ring2nest(i64 nside, i64 n, const i64* in, i64* out) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i) out[i] = ring2nest(nside, in[i]);
}
void or_pix2ang_ring(i64 nside, i64 n, const i64* pr, double* theta, double* phi) {
#pragma omp parallel for schedule(static)
  for (i64 k = 0; k < n; ++k) {
    i64 i, j; ringpix_decompose(nside, pr[k], i, j);
    double z, sth, ph; ring2zphi(nside, i, j, z, sth, ph);
    theta[k] = std::atan2(sth, z); phi[k] = ph;
  }
}
// Pixel corners in face (u, v) order (0,0), (1,0), (0,1), (1,1), HEALPix frame.
void or_pixel_corners_nest(i64 nside, i64 n, const i64* p, double* out) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i) {
    XYF c = nest2xyf(nside, p[i]);
    double N = (double)nside;
    int k = 0;
    for (int cv = 0; cv < 2; ++cv) for (int cu = 0; cu < 2; ++cu)
      face_uv2vec(c.f, (c.x + cu) / N, (c.y + cv) / N, out + 12 * i + 3 * (k++));
  }
}
// 8-neighbourhood (sorted, -1 padded); returns the neighbour count per pixel in cnt.
void or_neighbours_nest(i64 nside, i64 n, const i64* p, i64* out, int* cnt) {
#pragma omp parallel for schedule(dynamic, 256)
  for (i64 i = 0; i < n; ++i) cnt[i] = neighbours_nest(nside, p[i], out + 8 * i);
}

// FoV mask M_C(p) = 1[(omega_p, phi_p) in R_C] and its signed margin.
void or_mask(i64 nside, int kind, double fovx, double fovy, double ppx, double ppy, u8* mask, double* margin) {
  i64 npix = 12 * nside * nside;
#pragma omp parallel for schedule(static)
  for (i64 p = 0; p < npix; ++p) {
    double v[3]; pix2vec_nest(nside, p, v);
    double d[3] = {v[1], v[2], v[0]};   // camera direction from the HEALPix vector
    double mg = camera_margin(kind, fovx, fovy, ppx, ppy, d);
    mask[p] = mg >= 0 ? 1 : 0;
    if (margin) margin[p] = mg;
  }
}

void or_adaptive_nside(int kind, double W, double H, double fovx, double fovy, double* nstar,
                       int* k, int* kL, int* kH) {
  double om = solid_angle_in(kind, fovx, fovy);
  *nstar = std::sqrt(4.0 * kPi * W * H / (12.0 * om));
  double l2 = std::log2(*nstar);
  *k = (int)std::lround(l2); *kL = (int)std::floor(l2); *kH = (int)std::ceil(l2);
}

double or_tile_rho(int k, int b) { return tile_rho(k, b); }

// Real SH basis values and their gradient (for pins against a library routine).
void or_sh_basis(i64 n, const double* dirs, int deg, double* Y, double* dY) {
  for (i64 i = 0; i < n; ++i) {
    double y[16], dy[16][3];
    sh_basis(dirs + 3 * i, deg, y, dy);
    int K = (deg + 1) * (deg + 1);
    for (int k = 0; k < K; ++k) {
      Y[i * K + k] = y[k];
      if (dY) for (int c = 0; c < 3; ++c) dY[(i * K + k) * 3 + c] = dy[k][c];
    }
  }
}

// Spherical offset for (pixel, Gaussian) lon/lat pairs (for pins).
void or_spherical_offset(i64 n, const double* omp, const double* php, const double* omg,
                         const double* phg, double* d) {
  for (i64 i = 0; i < n; ++i) {
    Offset o;
    spherical_offset(omp[i], std::sin(php[i]), std::cos(php[i]), omg[i], std::sin(phg[i]), std::cos(phg[i]), o);
    d[2 * i] = o.d[0]; d[2 * i + 1] = o.d[1];
  }
}

// Stage 1 for P Gaussians. Outputs (per Gaussian): valid, r, omega, phi, g[3],
// conic[3], sigma_arc[3] (a, b, c), r_s, colour[3].
void or_preprocess(i64 P, const double* means, const double* scales, const double* rots,
                   const double* sh, int deg, const double* W, const double* b,
                   double near, double blur, int* valid, double* r, double* omega, double* phi,
                   double* g, double* conic, double* sarc, double* rs, double* col) {
  Cfg cfg{}; cfg.near = near; cfg.blur = blur;
  int K = (deg + 1) * (deg + 1);
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < P; ++i) {
    Pre o;
    preprocess_one(means + 3 * i, scales + 3 * i, rots + 4 * i, sh + (size_t)i * K * 3, deg, W, b, cfg, o);
    valid[i] = o.valid;
    r[i] = o.r; omega[i] = o.omega; phi[i] = o.phi;
    for (int c = 0; c < 3; ++c) {
      g[3 * i + c] = o.g[c]; conic[3 * i + c] = o.conic[c]; col[3 * i + c] = o.col[c];
    }
    sarc[3 * i] = o.Sarc[0][0]; sarc[3 * i + 1] = o.Sarc[0][1]; sarc[3 * i + 2] = o.Sarc[1][1];
    rs[i] = o.rs;
  }
}

// Tile lists from given per-Gaussian (g, r_s, valid, depth bits): CSR over all
// tiles of order k - b. Returns the pair count; start/ids may be null.
i64 or_tile_lists(int k, int b, i64 P, const double* g, const double* rs, const int* valid,
                  const u32* depth_bits, double rho, const u8* active, i64* start, i64* ids) {
  i64 nside_t = 1LL << (k - b);
  ListCSR L;
  build_lists(nside_t, P, g, rs, valid, depth_bits, rho, active, L);
  if (start) std::copy(L.start.begin(), L.start.end(), start);
  if (ids) std::copy(L.ids.begin(), L.ids.end(), ids);
  return (i64)L.ids.size();
}

// Brute force over every tile of the membership definition (pin for the RING enumerator).
i64 or_tile_lists_bruteforce(int k, int b, i64 P, const double* g, const double* rs, const int* valid,
                             double rho, const u8* active, u8* member /* P x ntile */) {
  i64 nside_t = 1LL << (k - b), ntile = 12 * nside_t * nside_t;
  i64 total = 0;
#pragma omp parallel for reduction(+ : total) schedule(static)
  for (i64 i = 0; i < P; ++i)
    for (i64 t = 0; t < ntile; ++t) {
      u8 v = valid[i] && active[t] && tile_member(nside_t, t, g + 3 * i, rs[i], rho);
      member[i * ntile + t] = v;
      total += v;
    }
  return total;
}

// Lists of the chosen tiles only, by the membership definition over every
// Gaussian, in (depth bits, id) order; every other tile gets an empty list. For
// sampled checks of a large scene, where enumerating all tiles would be slow.
// `sel` holds distinct tile ids. Returns the pair count; start/ids may be null.
i64 or_tile_lists_subset(int k, int b, i64 P, const double* g, const double* rs, const int* valid,
                         const u32* depth_bits, double rho, const u8* active, i64 nsel, const i64* sel,
                         i64* start, i64* ids) {
  i64 nside_t = 1LL << (k - b), ntile = 12 * nside_t * nside_t;
  std::vector<std::vector<i64>> per(nsel);
#pragma omp parallel for schedule(dynamic, 1)
  for (i64 s = 0; s < nsel; ++s) {
    const i64 t = sel[s];
    if (!active[t]) continue;
    double ct[3]; pix2vec_nest(nside_t, t, ct);
    for (i64 i = 0; i < P; ++i)
      if (valid[i] && tile_member_at(ct, g + 3 * i, rs[i], rho)) per[s].push_back(i);
    std::stable_sort(per[s].begin(), per[s].end(),
                     [&](i64 a, i64 c) { return depth_bits[a] < depth_bits[c]; });   // ids ascending within a depth
  }
  std::vector<i64> cnt(ntile, 0);
  for (i64 s = 0; s < nsel; ++s) cnt[sel[s]] = (i64)per[s].size();
  i64 total = 0;
  for (i64 t = 0; t < ntile; ++t) {
    if (start) start[t] = total;
    total += cnt[t];
  }
  if (start) start[ntile] = total;
  if (ids && start)
    for (i64 s = 0; s < nsel; ++s) std::copy(per[s].begin(), per[s].end(), ids + start[sel[s]]);
  return total;
}

// Active tiles of a mask: tiles with at least one in-mask pixel.
void or_active_tiles(int k, int b, const u8* mask, u8* active) {
  i64 nside_t = 1LL << (k - b), ntile = 12 * nside_t * nside_t, per = 1LL << (2 * b);
  for (i64 t = 0; t < ntile; ++t) {
    u8 a = 0;
    for (i64 j = 0; j < per && !a; ++j) a = mask[t * per + j];
    active[t] = a;
  }
}

// Compositing given per-Gaussian values and sorted lists, for the in-mask pixels
// listed in `pix`: the FP64 result and the flags of composite_branches. With `var_*`
// non-null, also every leaf (up to kMaxLeaves per pixel, leaf 0 the FP64 result):
// var_n[q] leaves, var_img[q][l][3], var_T[q][l], var_last[q][l], var_D[q][l].
static void composite_many(int k, int b, i64 P, const double* omega, const double* phi, const double* conic,
                           const double* opac, const double* col, const double* r, const i64* start,
                           const i64* ids, i64 npix_q, const i64* pix, double eps_T, double alpha_max,
                           double cutoff, const double* bg, double* img, double* Tfin, i64* last, u8* amb,
                           double* depth, int* var_n, double* var_img, double* var_T, i64* var_last,
                           double* var_D) {
  std::vector<GaussView> G(P);
  for (i64 i = 0; i < P; ++i) {
    G[i].omega = omega[i]; G[i].sphg = std::sin(phi[i]); G[i].cphg = std::cos(phi[i]);
    for (int c = 0; c < 3; ++c) { G[i].conic[c] = conic[3 * i + c]; G[i].col[c] = col[3 * i + c]; }
    G[i].opac = opac[i]; G[i].r = r[i];
  }
  Cfg cfg{}; cfg.eps_T = eps_T; cfg.alpha_max = alpha_max; cfg.cutoff = cutoff;
  for (int c = 0; c < 3; ++c) cfg.bg[c] = bg[c];
  i64 nside = 1LL << k;
#pragma omp parallel for schedule(dynamic, 64)
  for (i64 q = 0; q < npix_q; ++q) {
    i64 p = pix[q];
    i64 t = p >> (2 * b);
    double om, sp, cp; pixel_lonlat(nside, p, om, sp, cp);
    BranchCtx X;
    composite_pixel_branches(om, sp, cp, ids + start[t], start[t + 1] - start[t], G, cfg, X);
    const Leaf& L0 = X.leaves[0];
    if (img) for (int c = 0; c < 3; ++c) img[3 * q + c] = L0.C[c];
    if (Tfin) Tfin[q] = L0.T;
    if (last) last[q] = L0.last;
    if (amb) amb[q] = (u8)X.amb;
    if (depth) depth[q] = L0.D;
    if (var_n) {
      var_n[q] = X.nleaves;
      for (int l = 0; l < kMaxLeaves; ++l) {
        const Leaf& Lf = X.leaves[l < X.nleaves ? l : 0];
        for (int c = 0; c < 3; ++c) var_img[(q * kMaxLeaves + l) * 3 + c] = Lf.C[c];
        var_T[q * kMaxLeaves + l] = Lf.T;
        var_last[q * kMaxLeaves + l] = Lf.last;
        if (var_D) var_D[q * kMaxLeaves + l] = Lf.D;
      }
    }
  }
}

void or_composite(int k, int b, i64 P, const double* omega, const double* phi, const double* conic,
                  const double* opac, const double* col, const double* r, const i64* start,
                  const i64* ids, i64 npix_q, const i64* pix, double eps_T, double alpha_max,
                  double cutoff, const double* bg, double* img, double* Tfin, i64* last, u8* amb,
                  double* depth) {
  composite_many(k, b, P, omega, phi, conic, opac, col, r, start, ids, npix_q, pix, eps_T, alpha_max, cutoff, bg,
                 img, Tfin, last, amb, depth, nullptr, nullptr, nullptr, nullptr, nullptr);
}

int or_max_leaves() { return kMaxLeaves; }

void or_composite_variants(int k, int b, i64 P, const double* omega, const double* phi, const double* conic,
                           const double* opac, const double* col, const double* r, const i64* start,
                           const i64* ids, i64 npix_q, const i64* pix, double eps_T, double alpha_max,
                           double cutoff, const double* bg, int* var_n, double* var_img, double* var_T,
                           i64* var_last, double* var_D) {
  composite_many(k, b, P, omega, phi, conic, opac, col, r, start, ids, npix_q, pix, eps_T, alpha_max, cutoff, bg,
                 nullptr, nullptr, nullptr, nullptr, nullptr, var_n, var_img, var_T, var_last, var_D);
}

// Full backward for one view (Sec. 3.2): dL/dI over the listed in-mask pixels ->
// gradients w.r.t. means, linear scales, unnormalised quaternions, opacities and SH.
// The cull, cutoff, clamp and termination sets are held fixed.
void or_backward(int k, int b, i64 P, const double* means, const double* scales, const double* rots,
                 const double* opac, const double* sh, int deg, const double* W, const double* bvec,
                 double near, double blur, double eps_T, double alpha_max, double cutoff,
                 const double* bg, const i64* start, const i64* ids, i64 npix_q, const i64* pix,
                 const double* dLdI, double* dmeans, double* dscales, double* drots, double* dopac,
                 double* dsh, const double* dLdD, double* dang) {
  Cfg cfg{}; cfg.near = near; cfg.blur = blur; cfg.eps_T = eps_T; cfg.alpha_max = alpha_max;
  cfg.cutoff = cutoff; for (int c = 0; c < 3; ++c) cfg.bg[c] = bg[c];
  int K = (deg + 1) * (deg + 1);
  std::vector<Pre> pre(P);
  std::vector<GaussView> G(P);
  for (i64 i = 0; i < P; ++i) {
    preprocess_one(means + 3 * i, scales + 3 * i, rots + 4 * i, sh + (size_t)i * K * 3, deg, W, bvec, cfg, pre[i]);
    G[i].omega = pre[i].omega; G[i].sphg = std::sin(pre[i].phi); G[i].cphg = std::cos(pre[i].phi);
    for (int c = 0; c < 3; ++c) { G[i].conic[c] = pre[i].conic[c]; G[i].col[c] = pre[i].col[c]; }
    G[i].opac = opac[i]; G[i].r = pre[i].r;
  }
  // per-Gaussian accumulators: dcol[3], dopac, dconic[3] (a, b-unique, c), domega, dphi,
  // d(1/r) from the depth channel
  const int NA = 10;
  i64 nside = 1LL << k;
  int nthr = 1;
#ifdef _OPENMP
  nthr = omp_get_max_threads();
#endif
  std::vector<std::vector<double>> acc(nthr, std::vector<double>(P * NA, 0.0));
#pragma omp parallel for schedule(dynamic, 64)
  for (i64 q = 0; q < npix_q; ++q) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* A = acc[tid].data();
    i64 p = pix[q];
    i64 t = p >> (2 * b);
    const i64* L = ids + start[t];
    i64 n = start[t + 1] - start[t];
    double om, sp, cp; pixel_lonlat(nside, p, om, sp, cp);
    std::vector<double> al, Ts, Gs;
    PixOut po;
    composite_pixel(om, sp, cp, L, n, G, cfg, po, &al, &Ts, &Gs);
    const double* dI = dLdI + 3 * q;
    // colour behind entry j, including the background seen through T_final; the depth
    // channel has no background term
    double Sacc[3] = {po.T * cfg.bg[0], po.T * cfg.bg[1], po.T * cfg.bg[2]};
    const double dD = dLdD ? dLdD[q] : 0.0;
    double SD = 0.0;
    for (i64 j = po.last - 1; j >= 0; --j) {
      double a = al[j];
      if (a <= 0) continue;
      i64 gi = L[j];
      const GaussView& gv = G[gi];
      double Tj = Ts[j];
      double dLda = 0;
      for (int c = 0; c < 3; ++c) {
        A[gi * NA + c] += Tj * a * dI[c];
        dLda += dI[c] * (Tj * gv.col[c] - Sacc[c] / (1.0 - a));
        Sacc[c] += Tj * a * gv.col[c];
      }
      A[gi * NA + 9] += Tj * a * dD;
      dLda += dD * (Tj / gv.r - SD / (1.0 - a));
      SD += Tj * a / gv.r;
      if (gv.opac * Gs[j] >= cfg.alpha_max) continue;   // clamped: no gradient to o, m
      A[gi * NA + 3] += dLda * Gs[j];
      double dLdm = -0.5 * dLda * gv.opac * Gs[j];
      Offset o;
      spherical_offset(om, sp, cp, gv.omega, gv.sphg, gv.cphg, o);
      double dx = o.d[0], dy = o.d[1];
      A[gi * NA + 4] += dLdm * dx * dx;
      A[gi * NA + 5] += dLdm * 2 * dx * dy;
      A[gi * NA + 6] += dLdm * dy * dy;
      double Ld[2] = {dLdm * 2 * (gv.conic[0] * dx + gv.conic[1] * dy),
                      dLdm * 2 * (gv.conic[1] * dx + gv.conic[2] * dy)};
      double ddw[2], ddp[2];
      offset_grad(om, cp, gv.omega, gv.sphg, gv.cphg, o, ddw, ddp);
      A[gi * NA + 7] += Ld[0] * ddw[0] + Ld[1] * ddw[1];
      A[gi * NA + 8] += Ld[0] * ddp[0] + Ld[1] * ddp[1];
    }
  }
  std::vector<double> tot(P * NA, 0.0);
  for (int th = 0; th < nthr; ++th) for (i64 i = 0; i < P * NA; ++i) tot[i] += acc[th][i];

  double Wm[3][3];
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Wm[i][j] = W[3 * i + j];
  for (i64 i = 0; i < P; ++i) {
    double* dmu = dmeans + 3 * i; double* ds = dscales + 3 * i; double* dq = drots + 4 * i;
    double* dshi = dsh + (size_t)i * K * 3;
    for (int c = 0; c < 3; ++c) { dmu[c] = 0; ds[c] = 0; }
    for (int c = 0; c < 4; ++c) dq[c] = 0;
    for (int c = 0; c < K * 3; ++c) dshi[c] = 0;
    dopac[i] = 0;
    if (dang) { dang[2 * i] = 0; dang[2 * i + 1] = 0; }
    const Pre& o = pre[i];
    if (!o.valid) continue;
    const double* Ai = tot.data() + i * NA;
    // the angular gradient of density control (Sec. 4.2, radian-space density control; reading): dL/domega
    // and dL/dphi of the centre through the pixel offsets, the conic held in the local (east, north) frame
    if (dang) { dang[2 * i] = Ai[7]; dang[2 * i + 1] = Ai[8]; }
    // colour -> SH (clamped channels give no gradient)
    double dcr[3];
    for (int c = 0; c < 3; ++c) dcr[c] = o.craw[c] > 0 ? Ai[c] : 0.0;
    double ddir[3] = {0, 0, 0};
    for (int kk = 0; kk < K; ++kk)
      for (int c = 0; c < 3; ++c) {
        dshi[kk * 3 + c] = o.Y[kk] * dcr[c];
        for (int e = 0; e < 3; ++e) ddir[e] += dcr[c] * sh[(size_t)i * K * 3 + kk * 3 + c] * o.dY[kk][e];
      }
    double pd = ddir[0] * o.dir[0] + ddir[1] * o.dir[1] + ddir[2] * o.dir[2];
    for (int e = 0; e < 3; ++e) dmu[e] += (ddir[e] - o.dir[e] * pd) / o.dist;
    dopac[i] = Ai[3];
    // conic -> Sigma_arc: G_Sarc = -Q G_Q Q, G_Q = [[La, Lb/2], [Lb/2, Lc]]
    double Q[2][2] = {{o.conic[0], o.conic[1]}, {o.conic[1], o.conic[2]}};
    double GQ[2][2] = {{Ai[4], 0.5 * Ai[5]}, {0.5 * Ai[5], Ai[6]}};
    double tmp[2][2], Gar[2][2];
    for (int a = 0; a < 2; ++a) for (int c = 0; c < 2; ++c) tmp[a][c] = Q[a][0] * GQ[0][c] + Q[a][1] * GQ[1][c];
    for (int a = 0; a < 2; ++a) for (int c = 0; c < 2; ++c) Gar[a][c] = -(tmp[a][0] * Q[0][c] + tmp[a][1] * Q[1][c]);
    // Eq. backward_lat_scale: L_Srad = S L_Sarc S ; L_phi|S = -sin(phi)(2 cos(phi) s_ww L_ww + s_wp L_wp),
    // L_wp the gradient of the single off-diagonal entry (sum of both matrix entries).
    double cphi = std::cos(o.phi), sphi = std::sin(o.phi);
    double S[2] = {cphi, 1.0};
    double Grad[2][2];
    for (int a = 0; a < 2; ++a) for (int c = 0; c < 2; ++c) Grad[a][c] = S[a] * Gar[a][c] * S[c];
    double Lphi_S = -sphi * (2 * cphi * o.Srad[0][0] * Gar[0][0] + o.Srad[0][1] * (Gar[0][1] + Gar[1][0]));
    // Sigma_rad = T Sigma3D T^T : G_T = 2 G_rad T Sigma3D ; G_S3 = T^T G_rad T
    double GT[2][3], GS3[3][3];
    for (int a = 0; a < 2; ++a) for (int j = 0; j < 3; ++j) {
      double acc2 = 0;
      for (int c = 0; c < 2; ++c) for (int kk = 0; kk < 3; ++kk) acc2 += Grad[a][c] * o.T[c][kk] * o.S3[kk][j];
      GT[a][j] = 2 * acc2;
    }
    for (int x = 0; x < 3; ++x) for (int y = 0; y < 3; ++y) {
      double acc2 = 0;
      for (int a = 0; a < 2; ++a) for (int c = 0; c < 2; ++c) acc2 += o.T[a][x] * Grad[a][c] * o.T[c][y];
      GS3[x][y] = acc2;
    }
    // T = J W : G_J = G_T W^T ; Eq. grad_via_J_S: the J path, the S_phi path, and mu' J
    double GJ[2][3];
    for (int a = 0; a < 2; ++a) for (int j = 0; j < 3; ++j) {
      double acc2 = 0; for (int kk = 0; kk < 3; ++kk) acc2 += GT[a][kk] * Wm[j][kk];
      GJ[a][j] = acc2;
    }
    double dJ[2][3][3];
    dJ_dt(o.t, dJ);
    // depth channel: d(1/r)/dt = -t / r^3
    const double ir3 = 1.0 / (o.r * o.r * o.r);
    double Lt[3] = {-Ai[9] * o.t[0] * ir3, -Ai[9] * o.t[1] * ir3, -Ai[9] * o.t[2] * ir3};
    double Lmu2[2] = {Ai[7], Ai[8] + Lphi_S};
    for (int kk = 0; kk < 3; ++kk) {
      Lt[kk] += o.J[0][kk] * Lmu2[0] + o.J[1][kk] * Lmu2[1];
      for (int a = 0; a < 2; ++a) for (int j = 0; j < 3; ++j) Lt[kk] += GJ[a][j] * dJ[a][j][kk];
    }
    // dL/dmu = W^T dL/dt
    for (int e = 0; e < 3; ++e) dmu[e] += Wm[0][e] * Lt[0] + Wm[1][e] * Lt[1] + Wm[2][e] * Lt[2];
    // Sigma3D = M M^T, M = R diag(s): G_M = (G_S3 + G_S3^T) M
    double GM[3][3];
    for (int x = 0; x < 3; ++x) for (int y = 0; y < 3; ++y) {
      double acc2 = 0; for (int kk = 0; kk < 3; ++kk) acc2 += (GS3[x][kk] + GS3[kk][x]) * o.M[kk][y];
      GM[x][y] = acc2;
    }
    double s3[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
    double GR[3][3];
    for (int y = 0; y < 3; ++y) {
      double acc2 = 0;
      for (int x = 0; x < 3; ++x) { acc2 += GM[x][y] * o.R[x][y]; GR[x][y] = GM[x][y] * s3[y]; }
      ds[y] = acc2;
    }
    double w = o.qn[0], x = o.qn[1], y = o.qn[2], z = o.qn[3];
    double dR[4][3][3] = {
        {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}},
        {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}},
        {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}},
        {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}}};
    double Lqn[4];
    for (int c = 0; c < 4; ++c) {
      double acc2 = 0;
      for (int a = 0; a < 3; ++a) for (int bb = 0; bb < 3; ++bb) acc2 += GR[a][bb] * dR[c][a][bb];
      Lqn[c] = acc2;
    }
    double qd = Lqn[0] * o.qn[0] + Lqn[1] * o.qn[1] + Lqn[2] * o.qn[2] + Lqn[3] * o.qn[3];
    for (int c = 0; c < 4; ++c) dq[c] = (Lqn[c] - o.qn[c] * qd) / o.qnorm;
  }
}

// Loss and its gradient w.r.t. I over the whole map (in-mask pixels only).
// Returns the loss; writes HSSIM, L1 and dL/dI (N_pix x 3; zero outside the mask).
double or_hssim_loss(i64 nside, const double* I, const double* Gt, const u8* mask, double lambda,
                     double* hssim_out, double* l1_out, double* dI) {
  i64 npix = 12 * nside * nside;
  std::vector<i64> qs;
  for (i64 p = 0; p < npix; ++p) if (mask[p]) qs.push_back(p);
  i64 nm = (i64)qs.size();
  std::vector<Window> win(nm);
  std::vector<double> coef(nm * 9);   // per channel: dmu, dvar, dcov
  std::vector<double> mus(nm * 6);
  double hsum = 0, l1 = 0;
#pragma omp parallel for reduction(+ : hsum, l1) schedule(dynamic, 256)
  for (i64 a = 0; a < nm; ++a) {
    i64 q = qs[a];
    hssim_window(nside, q, mask, win[a]);
    double h = 0;
    for (int ch = 0; ch < 3; ++ch) {
      h += ssim_local(win[a], I, Gt, ch, &coef[9 * a + 3 * ch], &coef[9 * a + 3 * ch + 1],
                      &coef[9 * a + 3 * ch + 2], &mus[6 * a + 2 * ch], &mus[6 * a + 2 * ch + 1]);
      l1 += std::fabs(I[3 * q + ch] - Gt[3 * q + ch]);
    }
    hsum += h / 3.0;
  }
  double hssim = nm ? hsum / nm : 0.0;
  double L1 = nm ? l1 / (3.0 * nm) : 0.0;
  if (hssim_out) *hssim_out = hssim;
  if (l1_out) *l1_out = L1;
  if (dI) {
    std::fill(dI, dI + 3 * npix, 0.0);
    for (i64 a = 0; a < nm; ++a) {
      i64 q = qs[a];
      for (int ch = 0; ch < 3; ++ch) {
        double dd = I[3 * q + ch] - Gt[3 * q + ch];
        dI[3 * q + ch] += (1.0 - lambda) * (dd > 0 ? 1.0 : (dd < 0 ? -1.0 : 0.0)) / (3.0 * nm);
      }
    }
    // HSSIM term: d(1 - HSSIM)/dx_p = -(1/nm) sum_q (1/3) w_qp [ds/dmu + 2 (x_p - mu_x) ds/dvar + (y_p - mu_y) ds/dcov]
    for (i64 a = 0; a < nm; ++a) {
      const Window& W = win[a];
      for (int j = 0; j < W.n; ++j) {
        i64 p = W.idx[j];
        for (int ch = 0; ch < 3; ++ch) {
          const double* cf = &coef[9 * a + 3 * ch];
          double mx = mus[6 * a + 2 * ch], my = mus[6 * a + 2 * ch + 1];
          double g = W.w[j] * (cf[0] + 2 * (I[3 * p + ch] - mx) * cf[1] + (Gt[3 * p + ch] - my) * cf[2]);
          dI[3 * p + ch] += -lambda * g / (3.0 * nm);
        }
      }
    }
  }
  return (1.0 - lambda) * L1 + lambda * (1.0 - hssim);
}

// Local HSSIM value h_q at selected pixels (for sampled checks at full size).
void or_hssim_local(i64 nside, const double* I, const double* Gt, const u8* mask, i64 n,
                    const i64* qs, double* h) {
#pragma omp parallel for schedule(dynamic, 64)
  for (i64 a = 0; a < n; ++a) {
    Window W; hssim_window(nside, qs[a], mask, W);
    double s = 0;
    for (int ch = 0; ch < 3; ++ch) s += ssim_local(W, I, Gt, ch, nullptr, nullptr, nullptr, nullptr, nullptr);
    h[a] = s / 3.0;
  }
}

int or_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Threads of the following parallel regions (timing at a chosen core count).
void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}


// ---- resampling ----
int or_img_to_dir(int kind, double W, double H, double fovx, double fovy,
                  double ppx, double ppy, i64 n, const double* uv, double* dir,
                  u8* valid) {
  ImgCam c{kind, W, H, fovx, fovy, ppx, ppy};
  for (i64 q = 0; q < n; ++q) valid[q] = img_to_dir(c, uv[2 * q], uv[2 * q + 1], dir + 3 * q);
  return 0;
}

int or_dir_to_img(int kind, double W, double H, double fovx, double fovy,
                  double ppx, double ppy, i64 n, const double* dir, double* uv,
                  u8* valid) {
  ImgCam c{kind, W, H, fovx, fovy, ppx, ppy};
  for (i64 q = 0; q < n; ++q) valid[q] = dir_to_img(c, dir + 3 * q, uv[2 * q], uv[2 * q + 1]);
  return 0;
}

void or_interp_weights(i64 nside, i64 n, const double* theta, const double* phi, i64* pix, double* w) {
#pragma omp parallel for schedule(static)
  for (i64 q = 0; q < n; ++q) interp_weights(nside, theta[q], phi[q], pix + 4 * q, w + 4 * q);
}

// I_C(u, v) = Interp_H(I_H, P_C(u, v)) at every pixel centre; 0 and valid = 0 outside D_C.
void or_sphere_to_image(i64 nside, const double* map, int kind, i64 W, i64 H, double fovx, double fovy,
                        double ppx, double ppy,
                        double* img, u8* valid) {
  ImgCam c{kind, (double)W, (double)H, fovx, fovy, ppx, ppy};
#pragma omp parallel for schedule(static)
  for (i64 p = 0; p < W * H; ++p) {
    const i64 row = p / W, col = p % W;
    double d[3];
    img[3 * p] = img[3 * p + 1] = img[3 * p + 2] = 0;
    valid[p] = img_to_dir(c, col + 0.5, row + 0.5, d);
    if (!valid[p]) continue;
    double th, ph; dir_to_healpix_angles(d, th, ph);
    i64 pix[4]; double w[4];
    interp_weights(nside, th, ph, pix, w);
    for (int k = 0; k < 4; ++k)
      for (int ch = 0; ch < 3; ++ch) img[3 * p + ch] += w[k] * map[3 * pix[k] + ch];
  }
}

// The adjoint of or_sphere_to_image: dmap = A^T dimg (overwrites dmap).
void or_sphere_to_image_adjoint(i64 nside, const double* dimg, int kind, i64 W, i64 H, double fovx, double fovy,
                                double ppx, double ppy,
                                double* dmap) {
  ImgCam c{kind, (double)W, (double)H, fovx, fovy, ppx, ppy};
  std::fill(dmap, dmap + 3 * 12 * nside * nside, 0.0);
  for (i64 p = 0; p < W * H; ++p) {
    const i64 row = p / W, col = p % W;
    double d[3];
    if (!img_to_dir(c, col + 0.5, row + 0.5, d)) continue;
    double th, ph; dir_to_healpix_angles(d, th, ph);
    i64 pix[4]; double w[4];
    interp_weights(nside, th, ph, pix, w);
    for (int k = 0; k < 4; ++k)
      for (int ch = 0; ch < 3; ++ch) dmap[3 * pix[k] + ch] += w[k] * dimg[3 * p + ch];
  }
}

// or_sphere_to_image at the given image points only (for sampled checks of large images).
void or_sphere_to_image_at(i64 nside, const double* map, int kind, i64 W, i64 H, double fovx, double fovy,
                           double ppx, double ppy, i64 n,
                           const double* uv, double* out, u8* valid) {
  ImgCam c{kind, (double)W, (double)H, fovx, fovy, ppx, ppy};
#pragma omp parallel for schedule(static)
  for (i64 q = 0; q < n; ++q) {
    double d[3];
    out[3 * q] = out[3 * q + 1] = out[3 * q + 2] = 0;
    valid[q] = img_to_dir(c, uv[2 * q], uv[2 * q + 1], d);
    if (!valid[q]) continue;
    double th, ph; dir_to_healpix_angles(d, th, ph);
    i64 pix[4]; double w[4];
    interp_weights(nside, th, ph, pix, w);
    for (int k = 0; k < 4; ++k)
      for (int ch = 0; ch < 3; ++ch) out[3 * q + ch] += w[k] * map[3 * pix[k] + ch];
  }
}

// or_image_to_sphere at the given NESTED pixels only.
void or_image_to_sphere_at(i64 nside, const double* img, int kind, i64 W, i64 H, double fovx, double fovy,
                           double ppx, double ppy, i64 n,
                           const i64* qs, double* out, u8* mask) {
  ImgCam c{kind, (double)W, (double)H, fovx, fovy, ppx, ppy};
#pragma omp parallel for schedule(static)
  for (i64 t = 0; t < n; ++t) {
    double v[3]; pix2vec_nest(nside, qs[t], v);
    const double d[3] = {v[1], v[2], v[0]};
    double u, vv;
    out[3 * t] = out[3 * t + 1] = out[3 * t + 2] = 0;
    mask[t] = dir_to_img(c, d, u, vv);
    if (mask[t]) image_sample(img, c, u, vv, out + 3 * t);
  }
}

// I_H(q) = I_C(Pi_C^{-1}(s_q)) and M_C(q) for every NESTED pixel q; 0 where M_C(q) = 0.
void or_image_to_sphere(i64 nside, const double* img, int kind, i64 W, i64 H, double fovx, double fovy,
                        double ppx, double ppy, double* map,
                        u8* mask) {
  ImgCam c{kind, (double)W, (double)H, fovx, fovy, ppx, ppy};
#pragma omp parallel for schedule(static)
  for (i64 q = 0; q < 12 * nside * nside; ++q) {
    double v[3]; pix2vec_nest(nside, q, v);
    const double d[3] = {v[1], v[2], v[0]};            // camera (d_x, d_y, d_z) = HEALPix (Y, Z, X)
    double u, vv;
    map[3 * q] = map[3 * q + 1] = map[3 * q + 2] = 0;
    mask[q] = dir_to_img(c, d, u, vv);
    if (mask[q]) image_sample(img, c, u, vv, map + 3 * q);
  }
}


// ---- NESTED quadtree query (Algorithm 2) ----
double or_pixrad(int o) { return pixrad_order(o); }

// Tiles (order k - b) of one disc by Algorithm 2 with refinement f; returns the count.
i64 or_query_disc_nested(int kt, int log2f, const double* g, double rs, i64* out, i64 cap) {
  std::vector<i64> t;
  query_disc_nested(kt, kt + log2f, g, rs, t);
  for (i64 i = 0; i < (i64)t.size() && i < cap; ++i) out[i] = t[i];
  return (i64)t.size();
}

// Lists as or_tile_lists but with Algorithm 2 (refinement 2^log2f) as the query:
// tiles without an in-mask pixel dropped, each list in (depth bits, id) order.
i64 or_tile_lists_nested(int k, int b, int log2f, i64 P, const double* g, const double* rs, const int* valid,
                         const u32* depth_bits, const u8* active, i64* start, i64* ids) {
  const int kt = k - b;
  const i64 ntile = 12LL << (2 * kt);
  pixrad_order(kt + log2f);                                  // fill the cache before the parallel region
  for (int o = 0; o <= kt + log2f; ++o) pixrad_order(o);
  std::vector<std::vector<i64>> per(P);
#pragma omp parallel for schedule(dynamic, 64)
  for (i64 i = 0; i < P; ++i) {
    if (!valid[i]) continue;
    std::vector<i64> t;
    query_disc_nested(kt, kt + log2f, g + 3 * i, rs[i], t);
    for (i64 x : t) if (active[x]) per[i].push_back(x);
  }
  struct Pair { i64 tile; u32 depth; i64 id; };
  std::vector<Pair> pairs;
  for (i64 i = 0; i < P; ++i) for (i64 t : per[i]) pairs.push_back({t, depth_bits[i], i});
  std::stable_sort(pairs.begin(), pairs.end(), [](const Pair& a, const Pair& c) {
    if (a.tile != c.tile) return a.tile < c.tile;
    if (a.depth != c.depth) return a.depth < c.depth;
    return a.id < c.id;
  });
  if (start) {
    std::fill(start, start + ntile + 1, 0);
    for (auto& q : pairs) start[q.tile + 1]++;
    for (i64 t = 0; t < ntile; ++t) start[t + 1] += start[t];
  }
  if (ids) for (size_t q = 0; q < pairs.size(); ++q) ids[q] = pairs[q].id;
  return (i64)pairs.size();
}

// ===========================================================================
// RING query at a finer search resolution (Sec. 3.3 and Sec. D.2, "x f" search;
// Algorithm 3 run at query order k_q = k_t + log2 f instead of the tile order).
// Reading: the disc is enumerated over the order-k_q pixels with Algorithm 3, each
// candidate pixel q is kept when its centre passes the membership test of the tile
// query at that order, c_q . g >= cos(min(pi, r_s + rho_q + 1e-7)) with rho_q =
// rho(k, b - log2 f) (the largest angle from an order-k_q centre to the render-pixel
// centres it holds), and a tile is listed once when any of its pixels is kept and
// it is active. With the m <= cutoff weight this is again conservative (a pixel
// within r_s of g lies in a query pixel whose centre is within r_s + rho_q), and
// finer f lists fewer tiles; log2 f = 0 is the tile-order query.
// ===========================================================================
static void tiles_of_ringf(int kt, int log2f, const double g[3], double rs, double rho_q, const u8* active,
                           std::vector<i64>& out) {
  const i64 nside_q = 1LL << (kt + log2f);
  std::vector<i64> cand;
  query_dot_disc(nside_q, g, std::min(kPi, rs + rho_q + 1e-7), cand);
  out.clear();
  for (i64 q : cand) {
    if (!tile_member(nside_q, q, g, rs, rho_q)) continue;
    const i64 t = q >> (2 * log2f);                  // the order-k_t ancestor (NESTED)
    if (active[t]) out.push_back(t);
  }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
}

i64 or_tile_lists_ringf(int k, int b, int log2f, i64 P, const double* g, const double* rs, const int* valid,
                        const u32* depth_bits, const u8* active, i64* start, i64* ids) {
  const int kt = k - b;
  const i64 ntile = 12LL << (2 * kt);
  // at log2 f = b the query pixels are the render pixels: rho_q = 0 exactly
  const double rho_q = (b == log2f) ? 0.0 : tile_rho(k, b - log2f);
  std::vector<std::vector<i64>> per(P);
#pragma omp parallel for schedule(dynamic, 64)
  for (i64 i = 0; i < P; ++i)
    if (valid[i]) tiles_of_ringf(kt, log2f, g + 3 * i, rs[i], rho_q, active, per[i]);
  struct Pair { i64 tile; u32 depth; i64 id; };
  std::vector<Pair> pairs;
  for (i64 i = 0; i < P; ++i) for (i64 t : per[i]) pairs.push_back({t, depth_bits[i], i});
  std::stable_sort(pairs.begin(), pairs.end(), [](const Pair& a, const Pair& c) {
    if (a.tile != c.tile) return a.tile < c.tile;
    if (a.depth != c.depth) return a.depth < c.depth;
    return a.id < c.id;
  });
  if (start) {
    std::fill(start, start + ntile + 1, 0);
    for (auto& q : pairs) start[q.tile + 1]++;
    for (i64 t = 0; t < ntile; ++t) start[t + 1] += start[t];
  }
  if (ids) for (size_t q = 0; q < pairs.size(); ++q) ids[q] = pairs[q].id;
  return (i64)pairs.size();
}

}  // extern "C"

