// Device-side HEALPix geometry for the rasterizer (Sec. 3.1).
//
// NESTED pixel p of order k (Nside N = 2^k): face f = p >> 2k, face-local
// (x, y) = de-interleaved bits of p (x on even bits). Ring formulas after
// Gorski et al. (2005): ring jr = (row+2)N - x - y - 1 counted from the north
// pole, z and longitude (pi/4)(jpll + (x - y)/n_r). The inverse map uses the
// HEALPix ang2pix construction of the same paper (edge lines jp/jm in the belt,
// scaled polar coordinates in the caps). Integer neighbour logic walks across
// face edges with the fixed face adjacency of the 12 base quadrilaterals.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hpx {

constexpr double kPi = 3.14159265358979323846;

__host__ __device__ __forceinline__ uint32_t even_bits(uint32_t v) {   // compact bits 0,2,4,.. -> 0,1,2,..
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0f0f0f0fu;
  v = (v | (v >> 4)) & 0x00ff00ffu;
  v = (v | (v >> 8)) & 0x0000ffffu;
  return v;
}
__host__ __device__ __forceinline__ uint32_t spread_bits(uint32_t v) {  // inverse of even_bits
  v &= 0x0000ffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

struct FaceXY { int f, x, y; };

__host__ __device__ __forceinline__ FaceXY nest_to_fxy(int k, uint32_t p) {
  FaceXY r;
  r.f = (int)(p >> (2 * k));
  uint32_t q = p & ((1u << (2 * k)) - 1u);
  r.x = (int)even_bits(q);
  r.y = (int)even_bits(q >> 1);
  return r;
}
__host__ __device__ __forceinline__ uint32_t fxy_to_nest(int k, int f, int x, int y) {
  return ((uint32_t)f << (2 * k)) | spread_bits((uint32_t)x) | (spread_bits((uint32_t)y) << 1);
}

// Longitude of a face's centre in units of pi/4.
__host__ __device__ __forceinline__ int face_jpll(int f) {
  return ((f >> 2) == 1) ? 2 * (f & 3) : 2 * (f & 3) + 1;
}

// Point of face f at continuous face coordinates (u, v) in [0, 1]^2 (x / Nside,
// y / Nside), FP64: ring coordinate j = row + 2 - u - v (units of Nside); polar caps
// z = +-(1 - j'^2 / 3) with j' the distance to the pole in rings, longitude
// (pi/4)(jpll + (u - v) / j'); the belt z = (2 - j) 2/3, longitude (pi/4)(jpll + u - v).
__device__ __forceinline__ double3 face_uv_vec_f64(int f, double u, double v) {
  const double jr = (double)((f >> 2) + 2) - u - v;
  double z, sth, nr;
  if (jr < 1.0) { nr = jr; const double t = nr * nr / 3.0; z = 1.0 - t; sth = sqrt(t * (2.0 - t)); }
  else if (jr > 3.0) { nr = 4.0 - jr; const double t = nr * nr / 3.0; z = t - 1.0; sth = sqrt(t * (2.0 - t)); }
  else { nr = 1.0; z = (2.0 - jr) * (2.0 / 3.0); sth = sqrt((1.0 - z) * (1.0 + z)); }
  const double phi = nr > 0.0 ? 0.25 * kPi * ((double)face_jpll(f) + (u - v) / nr) : 0.0;
  double sp, cp;
  sincos(phi, &sp, &cp);
  return make_double3(sth * cp, sth * sp, z);
}

// Pixel centre of NESTED p at order k, FP32, HEALPix frame.
__device__ __forceinline__ float3 pix2vec_f32(int k, uint32_t p) {
  const int N = 1 << k;
  FaceXY c = nest_to_fxy(k, p);
  const int row = c.f >> 2;
  const int jr = (row + 2) * N - c.x - c.y - 1;
  const float invN = 1.0f / (float)N;   // exact: N is a power of two
  int nr;
  float z, sth;
  if (jr < N) {
    nr = jr;
    float a = (float)nr * invN;
    float t = a * a * (1.0f / 3.0f);
    z = 1.0f - t;
    sth = sqrtf(t * (2.0f - t));
  } else if (jr > 3 * N) {
    nr = 4 * N - jr;
    float a = (float)nr * invN;
    float t = a * a * (1.0f / 3.0f);
    z = t - 1.0f;
    sth = sqrtf(t * (2.0f - t));
  } else {
    nr = N;
    z = (float)(2 * N - jr) * invN * (2.0f / 3.0f);
    sth = sqrtf((1.0f - z) * (1.0f + z));
  }
  const int num = face_jpll(c.f) * nr + c.x - c.y;           // longitude * 4 nr / pi
  const float tphi = (float)num / (float)(4 * nr);
  float sp, cp;
  sincospif(tphi, &sp, &cp);
  return make_float3(sth * cp, sth * sp, z);
}

// Same in FP64.
__device__ __forceinline__ double3 pix2vec_f64(int k, uint32_t p) {
  const int N = 1 << k;
  FaceXY c = nest_to_fxy(k, p);
  const int row = c.f >> 2;
  const int jr = (row + 2) * N - c.x - c.y - 1;
  const double invN = 1.0 / (double)N;
  int nr;
  double z, sth;
  if (jr < N) {
    nr = jr;
    double a = (double)nr * invN;
    double t = a * a / 3.0;
    z = 1.0 - t;
    sth = sqrt(t * (2.0 - t));
  } else if (jr > 3 * N) {
    nr = 4 * N - jr;
    double a = (double)nr * invN;
    double t = a * a / 3.0;
    z = t - 1.0;
    sth = sqrt(t * (2.0 - t));
  } else {
    nr = N;
    z = (double)(2 * N - jr) * invN * (2.0 / 3.0);
    sth = sqrt((1.0 - z) * (1.0 + z));
  }
  const int num = face_jpll(c.f) * nr + c.x - c.y;
  double sp, cp;
  sincospi((double)num / (double)(4 * nr), &sp, &cp);
  return make_double3(sth * cp, sth * sp, z);
}

// Ring geometry at order k: z of ring i (1..4N-1), pixel count, longitude of pixel 0.
struct RingF { float z, sth, phi0; int npix; };
__device__ __forceinline__ RingF ring_f32(int k, int i) {
  const int N = 1 << k;
  const float invN = 1.0f / (float)N;
  RingF R;
  if (i < N) {
    float a = (float)i * invN, t = a * a * (1.0f / 3.0f);
    R.z = 1.0f - t; R.sth = sqrtf(t * (2.0f - t)); R.npix = 4 * i;
    R.phi0 = (float)kPi / (4.0f * (float)i);
  } else if (i > 3 * N) {
    int ii = 4 * N - i;
    float a = (float)ii * invN, t = a * a * (1.0f / 3.0f);
    R.z = t - 1.0f; R.sth = sqrtf(t * (2.0f - t)); R.npix = 4 * ii;
    R.phi0 = (float)kPi / (4.0f * (float)ii);
  } else {
    R.z = (float)(2 * N - i) * invN * (2.0f / 3.0f);
    R.sth = sqrtf((1.0f - R.z) * (1.0f + R.z));
    R.npix = 4 * N;
    int s = (i - N + 1) & 1;
    R.phi0 = ((float)kPi * 0.5f * invN) * (1.0f - 0.5f * (float)s);
  }
  return R;
}

// Centre of ring pixel (i, j) in FP64 (for decisions re-checked in double precision).
__device__ __forceinline__ double3 ringpix_vec_f64(int k, int i, int j) {
  const int N = 1 << k;
  const double invN = 1.0 / (double)N;
  double z, sth, num, den;
  if (i < N) {
    double a = (double)i * invN, t = a * a / 3.0;
    z = 1.0 - t; sth = sqrt(t * (2.0 - t));
    num = 2.0 * j + 1.0; den = 4.0 * i;                       // phi / pi = (2j+1) / (4i)
  } else if (i > 3 * N) {
    int ii = 4 * N - i;
    double a = (double)ii * invN, t = a * a / 3.0;
    z = t - 1.0; sth = sqrt(t * (2.0 - t));
    num = 2.0 * j + 1.0; den = 4.0 * ii;
  } else {
    z = (double)(2 * N - i) * invN * (2.0 / 3.0);
    sth = sqrt((1.0 - z) * (1.0 + z));
    int s = (i - N + 1) & 1;
    num = 2.0 * j + 2.0 - s; den = 4.0 * N;                   // phi / pi = (2j + 2 - s) / (4N)
  }
  double sp, cp;
  sincospi(num / den, &sp, &cp);
  return make_double3(sth * cp, sth * sp, z);
}

__host__ __device__ __forceinline__ int floordiv(int a, int b) {   // b > 0
  int q = a / b;
  return (a % b != 0 && a < 0) ? q - 1 : q;
}

// RING coordinates (ring i 1-based, in-ring j 0-based) -> face (f, x, y) at order k.
// Caps: f = j / i, the position p = j mod i gives x = N - i + p, y = N - 1 - p (north)
// or x = p, y = i' - 1 - p (south). Belt: locate the face diamond from the pixel's
// plane coordinates (X = 2j + 2 - s in units of pi/(4N), Y = 2N - i in units of 1/N).
__host__ __device__ __forceinline__ FaceXY ring_to_fxy(int k, int i, int j) {
  const int N = 1 << k;
  FaceXY r;
  if (i < N) {                                   // j < 4i: face = number of whole multiples of i
    const int fq = (j >= i) + (j >= 2 * i) + (j >= 3 * i);
    const int p = j - fq * i;
    r.f = fq; r.x = N - i + p; r.y = N - 1 - p;
  } else if (i > 3 * N) {
    const int ii = 4 * N - i;
    const int fq = (j >= ii) + (j >= 2 * ii) + (j >= 3 * ii);
    const int p = j - fq * ii;
    r.f = 8 + fq; r.x = p; r.y = ii - 1 - p;
  } else {
    const int s = (i - N + 1) & 1;
    const int a = 2 * j + 2 - s;
    // floor division by 2N = 2^(k+1): arithmetic shift
    const int A = (a + 3 * N - i) >> (k + 1), B = (3 * N - i - a) >> (k + 1);
    int Xc, Yc;
    if (A + B >= 1) { r.f = (A - 1) & 3; Xc = 2 * A - 1; Yc = 1; }
    else if (A + B == 0) { r.f = 4 + (A & 3); Xc = 2 * A; Yc = 0; }
    else { r.f = 8 + (A & 3); Xc = 2 * A + 1; Yc = -1; }
    r.x = (a - Xc * N + 3 * N - i - Yc * N - 1) >> 1;
    r.y = ((2 * N - i) - Yc * N - a + Xc * N + N - 1) >> 1;
  }
  return r;
}

__host__ __device__ __forceinline__ int64_t ring_start(int k, int i) {
  const int64_t N = 1LL << k;
  if (i <= N) return 2LL * i * (i - 1);
  if (i <= 3 * N) return 2 * N * (N - 1) + 4 * N * (i - N);
  int64_t ii = 4 * N - i;
  return 12 * N * N - 2 * ii * (ii + 1);
}

__host__ __device__ __forceinline__ int64_t nest2ring(int k, uint32_t p) {
  const int N = 1 << k;
  FaceXY c = nest_to_fxy(k, p);
  const int row = c.f >> 2;
  const int jr = (row + 2) * N - c.x - c.y - 1;
  int j;
  if (jr < N) j = (c.f & 3) * jr + (c.x - c.y + jr - 1) / 2;
  else if (jr > 3 * N) { int ii = 4 * N - jr; j = (c.f & 3) * ii + (c.x - c.y + ii - 1) / 2; }
  else {
    int s = (jr - N + 1) & 1;
    int a = face_jpll(c.f) * N + c.x - c.y;
    j = floordiv(a + s - 2, 2);
    if (j < 0) j += 4 * N;
    if (j >= 4 * N) j -= 4 * N;
  }
  return ring_start(k, jr) + j;
}

__host__ __device__ __forceinline__ uint32_t ring2nest(int k, int64_t pr) {
  const int N = 1 << k;
  int lo = 1, hi = 4 * N - 1;       // ring containing pr: largest i with start(i) <= pr
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (ring_start(k, mid) <= pr) lo = mid; else hi = mid - 1;
  }
  FaceXY c = ring_to_fxy(k, lo, (int)(pr - ring_start(k, lo)));
  return fxy_to_nest(k, c.f, c.x, c.y);
}

// NESTED pixel containing direction v (FP64), HEALPix ang2pix construction.
__device__ __forceinline__ uint32_t vec2pix_f64(int k, double3 v) {
  const int N = 1 << k;
  double n = sqrt(v.x * v.x + v.y * v.y + v.z * v.z);
  double z = v.z / n;
  double phi = atan2(v.y, v.x);
  if (phi < 0) phi += 2.0 * kPi;
  double tt = phi / (0.5 * kPi);                 // in [0, 4)
  if (tt >= 4.0) tt -= 4.0;
  int f, ix, iy;
  if (fabs(z) <= 2.0 / 3.0) {
    double temp1 = N * (0.5 + tt), temp2 = N * (z * 0.75);
    int jp = (int)floor(temp1 - temp2);          // ascending edge line index
    int jm = (int)floor(temp1 + temp2);          // descending edge line index
    int ifp = jp >> k, ifm = jm >> k;
    f = (ifp == ifm) ? (ifp | 4) : ((ifp < ifm) ? ifp : ifm + 8);
    ix = jm & (N - 1);
    iy = N - (jp & (N - 1)) - 1;
  } else {
    int ntt = (int)tt; if (ntt > 3) ntt = 3;
    double tp = tt - ntt;
    double tmp = N * sqrt(3.0 * (1.0 - fabs(z)));
    int jp = (int)(tp * tmp), jm = (int)((1.0 - tp) * tmp);
    if (jp > N - 1) jp = N - 1;
    if (jm > N - 1) jm = N - 1;
    if (z >= 0) { f = ntt; ix = N - jm - 1; iy = N - jp - 1; }
    else { f = ntt + 8; ix = jp; iy = jm; }
  }
  f &= 15;
  if (f > 11) f = 11;
  return fxy_to_nest(k, f, ix, iy);
}

// Neighbour of face pixel (x, y) of face f after the step (dx, dy) in {-1,0,1}^2,
// following face edges; returns -1 across the 8 vertices where only three faces
// meet (those corner pixels have 7 neighbours). Faces: 0-3 north, 4-7 equator,
// 8-11 south; x grows to the north-east, y to the north-west.
__host__ __device__ __forceinline__ int64_t neighbour_nest(int k, int f, int x, int y, int dx, int dy) {
  const int N = 1 << k;
  int X = x + dx, Y = y + dy;
  bool xo = X >= N, xu = X < 0, yo = Y >= N, yu = Y < 0;
  if (!(xo || xu || yo || yu)) return (int64_t)fxy_to_nest(k, f, X, Y);
  const int row = f >> 2, e = f & 3;
  int nf = -1;
  auto wrap = [N](int v) { return v & (N - 1); };
  if (row == 0) {
    if (xo && yo) { nf = (e + 2) & 3; X = N - 1; Y = N - 1; }            // across the north pole
    else if ((xo && yu) || (xu && yo)) nf = -1;
    else if (xu && yu) { nf = 8 + e; X = wrap(X); Y = wrap(Y); }
    else if (xo) { nf = (e + 1) & 3; int t = X; X = Y; Y = 2 * N - 1 - t; }
    else if (yo) { nf = (e + 3) & 3; int t = Y; Y = X; X = 2 * N - 1 - t; }
    else if (xu) { nf = 4 + e; X = wrap(X); }
    else { nf = 4 + ((e + 1) & 3); Y = wrap(Y); }
  } else if (row == 1) {
    if ((xo && yo) || (xu && yu)) nf = -1;
    else if (xo && yu) { nf = 4 + ((e + 1) & 3); X = wrap(X); Y = wrap(Y); }
    else if (xu && yo) { nf = 4 + ((e + 3) & 3); X = wrap(X); Y = wrap(Y); }
    else if (xo) { nf = e; X = wrap(X); }
    else if (yo) { nf = (e + 3) & 3; Y = wrap(Y); }
    else if (xu) { nf = 8 + ((e + 3) & 3); X = wrap(X); }
    else { nf = 8 + e; Y = wrap(Y); }
  } else {
    if (xu && yu) { nf = 8 + ((e + 2) & 3); X = 0; Y = 0; }              // across the south pole
    else if ((xo && yu) || (xu && yo)) nf = -1;
    else if (xo && yo) { nf = e; X = wrap(X); Y = wrap(Y); }
    else if (xu) { nf = 8 + ((e + 3) & 3); int t = X; X = Y; Y = -1 - t; }
    else if (yu) { nf = 8 + ((e + 1) & 3); int t = Y; Y = X; X = -1 - t; }
    else if (xo) { nf = 4 + ((e + 1) & 3); X = wrap(X); }
    else { nf = 4 + e; Y = wrap(Y); }
  }
  if (nf < 0) return -1;
  return (int64_t)fxy_to_nest(k, nf, X, Y);
}

}  // namespace hpx
