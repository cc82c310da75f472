"""FP64 CPU oracle for the HEALPix spherical Gaussian rasterizer (UniTriSplat).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package. The
product library (``paper_2606_29794_b300``) never imports it and shares no code
with it: the oracle is plain C++ (``hpx_oracle.cpp``) in double precision,
loaded here through ctypes; the product path is CUDA.

Each wrapper names the passage of the paper it follows (section, equation,
algorithm or table). Readings of passages where the paper is silent are stated
in the C++ source next to the code that takes them.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force, a library routine (SciPy's
spherical harmonics), finite differences, or an independent dense PyTorch FP64
reference. What stays unpinned is only whether these readings reproduce the
authors' own (unreleased) rasterizer bit for bit: the paper prints no pixel,
tile or gradient value that could pin it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpx_oracle.cpp")
_LIB = os.path.join(_HERE, "libhpx_oracle.so")

CAM_FULL, CAM_PINHOLE, CAM_FISHEYE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, OpenMP, IEEE double: no fast-math and no contraction
    of a multiply and an add into one rounding)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.or_tile_rho.restype = ctypes.c_double
        _lib.or_tile_lists.restype = ctypes.c_int64
        _lib.or_tile_lists_bruteforce.restype = ctypes.c_int64
        _lib.or_tile_lists_subset.restype = ctypes.c_int64
        _lib.or_tile_lists_nested.restype = ctypes.c_int64
        _lib.or_query_disc_nested.restype = ctypes.c_int64
        _lib.or_pixrad.restype = ctypes.c_double
        _lib.or_hssim_loss.restype = ctypes.c_double
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_max_leaves.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _i64(x):
    return ctypes.c_int64(int(x))


def _f64(x):
    return ctypes.c_double(float(x))


def num_threads() -> int:
    return lib().or_num_threads()


def set_threads(n: int) -> None:
    """Use n OpenMP threads in the oracle's parallel loops from now on (timing only)."""
    lib().or_set_threads(ctypes.c_int(int(n)))


# ---------------------------------------------------------------------------
# HEALPix (Sec. 3.1; Gorski et al. 2005; Calabretta & Roukema 2007)
# ---------------------------------------------------------------------------

def npix(nside: int) -> int:
    return 12 * nside * nside


def pix2vec_nest(nside, p):
    p = np.ascontiguousarray(p, dtype=np.int64).ravel()
    out = np.empty((p.size, 3), np.float64)
    lib().or_pix2vec_nest(_i64(nside), _i64(p.size), _p(p), _p(out))
    return out


def pix2ang_nest(nside, p):
    p = np.ascontiguousarray(p, dtype=np.int64).ravel()
    th = np.empty(p.size); ph = np.empty(p.size)
    lib().or_pix2ang_nest(_i64(nside), _i64(p.size), _p(p), _p(th), _p(ph))
    return th, ph


def ang2pix_nest(nside, theta, phi):
    theta = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    phi = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    out = np.empty(theta.size, np.int64)
    lib().or_ang2pix_nest(_i64(nside), _i64(theta.size), _p(theta), _p(phi), _p(out))
    return out


def vec2pix_nest(nside, v):
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
    out = np.empty(v.shape[0], np.int64)
    lib().or_vec2pix_nest(_i64(nside), _i64(v.shape[0]), _p(v), _p(out))
    return out


def nest2ring(nside, p):
    p = np.ascontiguousarray(p, dtype=np.int64).ravel()
    out = np.empty_like(p)
    lib().or_nest2ring(_i64(nside), _i64(p.size), _p(p), _p(out))
    return out


def ring2nest(nside, p):
    p = np.ascontiguousarray(p, dtype=np.int64).ravel()
    out = np.empty_like(p)
    lib().or_ring2nest(_i64(nside), _i64(p.size), _p(p), _p(out))
    return out


def pix2ang_ring(nside, p):
    p = np.ascontiguousarray(p, dtype=np.int64).ravel()
    th = np.empty(p.size); ph = np.empty(p.size)
    lib().or_pix2ang_ring(_i64(nside), _i64(p.size), _p(p), _p(th), _p(ph))
    return th, ph


def pixel_corners_nest(nside, p):
    p = np.ascontiguousarray(p, dtype=np.int64).ravel()
    out = np.empty((p.size, 4, 3))
    lib().or_pixel_corners_nest(_i64(nside), _i64(p.size), _p(p), _p(out))
    return out


def neighbours_nest(nside, p):
    """8-neighbourhood by shared vertices: (n, 8) sorted, -1 padded, and counts."""
    p = np.ascontiguousarray(p, dtype=np.int64).ravel()
    out = np.empty((p.size, 8), np.int64)
    cnt = np.empty(p.size, np.int32)
    lib().or_neighbours_nest(_i64(nside), _i64(p.size), _p(p), _p(out), _p(cnt))
    return out, cnt


# ---------------------------------------------------------------------------
# Cameras (Sec. 3.1; Sec. D.1)
# ---------------------------------------------------------------------------

def mask(nside, kind, fov_x=360.0, fov_y=None, pp=(0.0, 0.0)):
    """FoV mask M_C(p) over all NESTED pixels (uint8) and the FP64 decision margin. pp: the
    pinhole principal point's offset from the image centre in half-image units."""
    fov_y = fov_x if fov_y is None else fov_y
    n = npix(nside)
    m = np.empty(n, np.uint8)
    mg = np.empty(n, np.float64)
    lib().or_mask(_i64(nside), ctypes.c_int(kind), _f64(fov_x), _f64(fov_y), _f64(pp[0]), _f64(pp[1]), _p(m),
                  _p(mg))
    return m, mg


def adaptive_nside(kind, W, H, fov_x=360.0, fov_y=None):
    """Table "resolution": N* = sqrt(4 pi W H / (12 Omega_in)); k = round, kL = floor, kH = ceil of log2 N*."""
    fov_y = fov_x if fov_y is None else fov_y
    ns = ctypes.c_double(); k = ctypes.c_int(); kl = ctypes.c_int(); kh = ctypes.c_int()
    lib().or_adaptive_nside(ctypes.c_int(kind), _f64(W), _f64(H), _f64(fov_x), _f64(fov_y),
                            ctypes.byref(ns), ctypes.byref(k), ctypes.byref(kl), ctypes.byref(kh))
    return ns.value, k.value, kl.value, kh.value


def tile_rho(k: int, b: int) -> float:
    """Largest tile-centre to pixel-centre angle at orders (k, k-b), rounded up to 2^-20 rad."""
    return lib().or_tile_rho(ctypes.c_int(k), ctypes.c_int(b))


def active_tiles(k, b, m):
    nt = 12 * 4 ** (k - b)
    out = np.empty(nt, np.uint8)
    m = np.ascontiguousarray(m, dtype=np.uint8)
    lib().or_active_tiles(ctypes.c_int(k), ctypes.c_int(b), _p(m), _p(out))
    return out


def sh_basis(dirs, deg, with_grad=False):
    dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    K = (deg + 1) ** 2
    Y = np.empty((dirs.shape[0], K))
    dY = np.empty((dirs.shape[0], K, 3)) if with_grad else None
    lib().or_sh_basis(_i64(dirs.shape[0]), _p(dirs), ctypes.c_int(deg), _p(Y), _p(dY))
    return (Y, dY) if with_grad else Y


def spherical_offset(omega_p, phi_p, omega_g, phi_g):
    """Sec. 3.4: haversine distance split by the bearing at the Gaussian -> (east, north)."""
    a = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (omega_p, phi_p, omega_g, phi_g)]
    n = a[0].size
    out = np.empty((n, 2))
    lib().or_spherical_offset(_i64(n), _p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), _p(out))
    return out


# ---------------------------------------------------------------------------
# Rasterizer (Algorithm 1; Sec. 3.2-3.4)
# ---------------------------------------------------------------------------

@dataclass
class Config:
    tile_level: int = 4          # B = 2^b, Table "resolution" (B = 16)
    eps_T: float = 1e-4          # Algorithm 1 termination threshold
    alpha_max: float = 0.99      # reading (3DGS clamp)
    cutoff: float = 9.0          # reading (3-sigma ellipse)
    blur: float | None = None    # reading: None -> 0.3 * Omega_pix
    near: float = 0.2            # reading (3DGS near plane)
    bg: tuple = (0.0, 0.0, 0.0)  # reading
    lam: float = 0.2             # reading (loss weight)

    def blur_for(self, nside):
        return 0.3 * 4.0 * np.pi / npix(nside) if self.blur is None else float(self.blur)


def _scene64(scene):
    K = (scene["sh_degree"] + 1) ** 2
    P = scene["means"].shape[0]
    return (np.ascontiguousarray(scene["means"], np.float64),
            np.ascontiguousarray(scene["scales"], np.float64),
            np.ascontiguousarray(scene["rotations"], np.float64),
            np.ascontiguousarray(scene["opacities"], np.float64),
            np.ascontiguousarray(np.asarray(scene["sh"], np.float64).reshape(P, K, 3)),
            int(scene["sh_degree"]), P)


def preprocess(scene, view, cfg: Config):
    """Stage 1 (Algorithm 1 preprocessing): returns per-Gaussian FP64 quantities."""
    mu, s, q, o, sh, deg, P = _scene64(scene)
    W = np.ascontiguousarray(view["W"], np.float64).ravel()
    b = np.ascontiguousarray(view["b"], np.float64).ravel()
    nside = 1 << view["nside_log2"]
    out = dict(valid=np.empty(P, np.int32), r=np.empty(P), omega=np.empty(P), phi=np.empty(P),
               g=np.empty((P, 3)), conic=np.empty((P, 3)), sigma_arc=np.empty((P, 3)),
               rs=np.empty(P), col=np.empty((P, 3)))
    lib().or_preprocess(_i64(P), _p(mu), _p(s), _p(q), _p(sh), ctypes.c_int(deg), _p(W), _p(b),
                        _f64(cfg.near), _f64(cfg.blur_for(nside)), _p(out["valid"]), _p(out["r"]),
                        _p(out["omega"]), _p(out["phi"]), _p(out["g"]), _p(out["conic"]),
                        _p(out["sigma_arc"]), _p(out["rs"]), _p(out["col"]))
    return out


def depth_bits(r):
    """Sort key of the radial depth: the bit pattern of float32(r) (monotone for r > 0)."""
    return np.ascontiguousarray(np.asarray(r, np.float64).astype(np.float32).view(np.uint32))


def tile_lists(k, b, g, rs, valid, dbits, rho, active):
    """Stage 2 (Algorithm 1 + Algorithm 3): CSR (start over all tiles, Gaussian ids)."""
    g = np.ascontiguousarray(g, np.float64); rs = np.ascontiguousarray(rs, np.float64)
    valid = np.ascontiguousarray(valid, np.int32); dbits = np.ascontiguousarray(dbits, np.uint32)
    active = np.ascontiguousarray(active, np.uint8)
    P = rs.size
    nt = 12 * 4 ** (k - b)
    start = np.empty(nt + 1, np.int64)
    m = lib().or_tile_lists(ctypes.c_int(k), ctypes.c_int(b), _i64(P), _p(g), _p(rs), _p(valid), _p(dbits),
                            _f64(rho), _p(active), _p(start), None)
    ids = np.empty(m, np.int64)
    lib().or_tile_lists(ctypes.c_int(k), ctypes.c_int(b), _i64(P), _p(g), _p(rs), _p(valid), _p(dbits),
                        _f64(rho), _p(active), None, _p(ids))
    return start, ids


def tile_lists_subset(k, b, g, rs, valid, dbits, rho, active, tiles):
    """Lists of the distinct tiles `tiles` only (membership definition over every
    Gaussian, depth order); CSR over all tiles with the other lists empty."""
    g = np.ascontiguousarray(g, np.float64); rs = np.ascontiguousarray(rs, np.float64)
    valid = np.ascontiguousarray(valid, np.int32); dbits = np.ascontiguousarray(dbits, np.uint32)
    active = np.ascontiguousarray(active, np.uint8)
    sel = np.ascontiguousarray(np.unique(np.asarray(tiles, np.int64)), np.int64)
    P = rs.size
    nt = 12 * 4 ** (k - b)
    start = np.empty(nt + 1, np.int64)
    m = lib().or_tile_lists_subset(ctypes.c_int(k), ctypes.c_int(b), _i64(P), _p(g), _p(rs), _p(valid), _p(dbits),
                                   _f64(rho), _p(active), _i64(sel.size), _p(sel), _p(start), None)
    ids = np.empty(m, np.int64)
    lib().or_tile_lists_subset(ctypes.c_int(k), ctypes.c_int(b), _i64(P), _p(g), _p(rs), _p(valid), _p(dbits),
                               _f64(rho), _p(active), _i64(sel.size), _p(sel), _p(start), _p(ids))
    return start, ids


def tile_lists_bruteforce(k, b, g, rs, valid, rho, active):
    g = np.ascontiguousarray(g, np.float64); rs = np.ascontiguousarray(rs, np.float64)
    valid = np.ascontiguousarray(valid, np.int32); active = np.ascontiguousarray(active, np.uint8)
    P = rs.size
    nt = 12 * 4 ** (k - b)
    member = np.empty((P, nt), np.uint8)
    lib().or_tile_lists_bruteforce(ctypes.c_int(k), ctypes.c_int(b), _i64(P), _p(g), _p(rs), _p(valid),
                                   _f64(rho), _p(active), _p(member))
    return member


def _composite_inputs(pre, opac, start, ids):
    return [np.ascontiguousarray(pre["omega"], np.float64), np.ascontiguousarray(pre["phi"], np.float64),
            np.ascontiguousarray(pre["conic"], np.float64), np.ascontiguousarray(opac, np.float64),
            np.ascontiguousarray(pre["col"], np.float64), np.ascontiguousarray(pre["r"], np.float64),
            np.ascontiguousarray(start, np.int64), np.ascontiguousarray(ids, np.int64)]


# Flags of composite / render (test bookkeeping, not the method): decisions an FP32
# rasterizer may take the other way, because the FP64 value lies within a narrow band
# of its threshold (m <= cutoff within 2e-5 relative; T < eps within 1e-4 relative).
AMB_CUTOFF = 1       # a cutoff decision in its band: composite_variants holds both outcomes
AMB_TERM = 2         # a termination decision in its band: likewise
AMB_UNRESOLVED = 4   # more band decisions than the variants follow: not comparable


def composite(k, b, pre, opac, start, ids, pix, cfg: Config, depth=False):
    """Stage 3 (Algorithm 1 rendering loop) at the NESTED pixels `pix`.
    Returns (image, T, last, amb) with the FP64 outcome of every decision; amb holds the
    AMB_* flags of decisions single precision may take the other way."""
    pix = np.ascontiguousarray(pix, np.int64)
    n = pix.size
    img = np.empty((n, 3)); T = np.empty(n); last = np.empty(n, np.int64); amb = np.empty(n, np.uint8)
    D = np.empty(n) if depth else None
    bg = np.asarray(cfg.bg, np.float64)
    P = pre["r"].size
    args = _composite_inputs(pre, opac, start, ids)
    lib().or_composite(ctypes.c_int(k), ctypes.c_int(b), _i64(P), *[_p(a) for a in args],
                       _i64(n), _p(pix), _f64(cfg.eps_T), _f64(cfg.alpha_max),
                       _f64(cfg.cutoff), _p(bg), _p(img), _p(T), _p(last), _p(amb), _p(D))
    if depth:
        return img, T, last, amb, D
    return img, T, last, amb


def max_leaves() -> int:
    return lib().or_max_leaves()


def composite_variants(k, b, pre, opac, start, ids, pix, cfg: Config):
    """Every result the rendering loop can give at `pix` when each decision within its FP32
    band takes either outcome (see AMB_*): dict with n (leaves per pixel), image (n, L, 3),
    T (n, L), last (n, L), D (n, L); leaf 0 is composite's FP64 result, slots past n[q]
    repeat it."""
    pix = np.ascontiguousarray(pix, np.int64)
    n = pix.size
    L = max_leaves()
    out = dict(n=np.empty(n, np.int32), image=np.empty((n, L, 3)), T=np.empty((n, L)),
               last=np.empty((n, L), np.int64), D=np.empty((n, L)))
    bg = np.asarray(cfg.bg, np.float64)
    args = _composite_inputs(pre, opac, start, ids)
    lib().or_composite_variants(ctypes.c_int(k), ctypes.c_int(b), _i64(pre["r"].size), *[_p(a) for a in args],
                                _i64(n), _p(pix), _f64(cfg.eps_T), _f64(cfg.alpha_max), _f64(cfg.cutoff), _p(bg),
                                _p(out["n"]), _p(out["image"]), _p(out["T"]), _p(out["last"]), _p(out["D"]))
    return out


@dataclass
class Render:
    image: np.ndarray            # (Npix, 3); outside the mask: bg
    T: np.ndarray                # (Npix,) final transmittance (1 outside the mask)
    last: np.ndarray             # (Npix,) processed entries of the tile list
    amb: np.ndarray              # (Npix,) AMB_* flags of FP32-undecidable decisions
    mask: np.ndarray
    active: np.ndarray
    pre: dict
    start: np.ndarray
    ids: np.ndarray
    rho: float
    pix: np.ndarray = field(default=None)


def render(scene, view, cfg: Config, pix=None, rho=None):
    """Forward render of one view end to end in FP64 (Algorithm 1)."""
    k = view["nside_log2"]; b = cfg.tile_level
    nside = 1 << k
    m, _ = mask(nside, view["cam"], view.get("fov_x", 360.0), view.get("fov_y"), view.get("pp", (0.0, 0.0)))
    act = active_tiles(k, b, m)
    pre = preprocess(scene, view, cfg)
    rho = tile_rho(k, b) if rho is None else rho
    start, ids = tile_lists(k, b, pre["g"], pre["rs"], pre["valid"], depth_bits(pre["r"]), rho, act)
    if pix is None:
        pix = np.nonzero(m)[0].astype(np.int64)
    img_q, T_q, last_q, amb_q = composite(k, b, pre, scene["opacities"], start, ids, pix, cfg)
    N = npix(nside)
    image = np.tile(np.asarray(cfg.bg, np.float64), (N, 1))
    T = np.ones(N); last = np.zeros(N, np.int64); amb = np.zeros(N, np.uint8)
    image[pix] = img_q; T[pix] = T_q; last[pix] = last_q; amb[pix] = amb_q
    return Render(image, T, last, amb, m, act, pre, start, ids, rho, pix)


def backward(scene, view, cfg: Config, dLdI, start, ids, pix, dLdD=None, angular=False):
    """Sec. 3.2 backward for one view: dL/dI at `pix` (n, 3) and optionally dL/dD of the
    inverse-depth channel at `pix` (n,) -> parameter gradients. With angular=True, out["angular"]
    (P, 2) holds dL/domega and dL/dphi of each centre through the pixel offsets with the conic held
    in the local (east, north) frame: the statistic of radian-space density control (Sec. 4.2)."""
    mu, s, q, o, sh, deg, P = _scene64(scene)
    k = view["nside_log2"]; b = cfg.tile_level
    nside = 1 << k
    W = np.ascontiguousarray(view["W"], np.float64).ravel()
    bv = np.ascontiguousarray(view["b"], np.float64).ravel()
    pix = np.ascontiguousarray(pix, np.int64)
    dLdI = np.ascontiguousarray(dLdI, np.float64).reshape(-1, 3)
    K = (deg + 1) ** 2
    out = dict(means=np.empty((P, 3)), scales=np.empty((P, 3)), rotations=np.empty((P, 4)),
               opacities=np.empty(P), sh=np.empty((P, K, 3)))
    if angular:
        out["angular"] = np.empty((P, 2))
    bg = np.asarray(cfg.bg, np.float64)
    lib().or_backward(ctypes.c_int(k), ctypes.c_int(b), _i64(P), _p(mu), _p(s), _p(q), _p(o), _p(sh),
                      ctypes.c_int(deg), _p(W), _p(bv), _f64(cfg.near), _f64(cfg.blur_for(nside)),
                      _f64(cfg.eps_T), _f64(cfg.alpha_max), _f64(cfg.cutoff), _p(bg),
                      _p(np.ascontiguousarray(start, np.int64)), _p(np.ascontiguousarray(ids, np.int64)),
                      _i64(pix.size), _p(pix), _p(dLdI), _p(out["means"]), _p(out["scales"]),
                      _p(out["rotations"]), _p(out["opacities"]), _p(out["sh"]),
                      _p(None if dLdD is None else np.ascontiguousarray(dLdD, np.float64).ravel()),
                      _p(out["angular"]) if angular else None)
    return out


def density_stats_update(rs_max, grad_acc, count, rs, angular, valid):
    """Radian-space density statistics of one view (Sec. 4.2), updated in place for the visible
    Gaussians: r_s,max <- max(r_s,max, r_s); grad_acc += |(dL/domega, dL/dphi)|; count += 1."""
    v = np.asarray(valid).astype(bool)
    rs_max[v] = np.maximum(rs_max[v], np.asarray(rs)[v])
    grad_acc[v] += np.hypot(angular[v, 0], angular[v, 1])
    count[v] += 1


# ---------------------------------------------------------------------------
# HEALPix-SSIM and the training loss (Sec. 4.1; Eq. supp_hssim_eval)
# ---------------------------------------------------------------------------

def hssim_loss(nside, I, G, m, lam=0.2, grad=True):
    """Returns (loss, hssim, l1, dL/dI) with dL/dI of shape (Npix, 3) (or None)."""
    I = np.ascontiguousarray(I, np.float64).reshape(-1, 3)
    G = np.ascontiguousarray(G, np.float64).reshape(-1, 3)
    m = np.ascontiguousarray(m, np.uint8)
    h = ctypes.c_double(); l1 = ctypes.c_double()
    dI = np.empty_like(I) if grad else None
    loss = lib().or_hssim_loss(_i64(nside), _p(I), _p(G), _p(m), _f64(lam), ctypes.byref(h),
                               ctypes.byref(l1), _p(dI))
    return loss, h.value, l1.value, dI


def hssim_local(nside, I, G, m, qs):
    I = np.ascontiguousarray(I, np.float64).reshape(-1, 3)
    G = np.ascontiguousarray(G, np.float64).reshape(-1, 3)
    m = np.ascontiguousarray(m, np.uint8)
    qs = np.ascontiguousarray(qs, np.int64)
    h = np.empty(qs.size)
    lib().or_hssim_local(_i64(nside), _p(I), _p(G), _p(m), _i64(qs.size), _p(qs), _p(h))
    return h


# ---------------------------------------------------------------------------
# Sphere <-> image resampling (Eq. camera_synthesis; Eqs. supp_image_to_healpix,
# supp_hssim_mask; camera models of Sec. D.1)
# ---------------------------------------------------------------------------

def _cam_args(kind, W, H, fovx, fovy, pp=(0.0, 0.0)):
    fovy = fovx if fovy is None else fovy
    return ctypes.c_int(kind), _f64(W), _f64(H), _f64(fovx), _f64(fovy), _f64(pp[0]), _f64(pp[1])


def _fov_pp(fovx, fovy, pp):
    return _f64(fovx), _f64(fovx if fovy is None else fovy), _f64(pp[0]), _f64(pp[1])


# The camera arguments: kind, image size W x H, FoV in degrees and, for the pinhole, the
# principal point's offset pp from the image centre in half-image units.

def img_to_dir(kind, W, H, fovx, fovy, uv, pp=(0.0, 0.0)):
    """P_C: image points (n, 2) -> camera directions (n, 3) and validity (D_C)."""
    uv = np.ascontiguousarray(uv, np.float64).reshape(-1, 2)
    d = np.empty((uv.shape[0], 3)); ok = np.empty(uv.shape[0], np.uint8)
    lib().or_img_to_dir(*_cam_args(kind, W, H, fovx, fovy, pp), _i64(uv.shape[0]), _p(uv), _p(d), _p(ok))
    return d, ok


def dir_to_img(kind, W, H, fovx, fovy, d, pp=(0.0, 0.0)):
    """Pi_C^{-1}: camera directions (n, 3) -> image points (n, 2) and validity."""
    d = np.ascontiguousarray(d, np.float64).reshape(-1, 3)
    uv = np.empty((d.shape[0], 2)); ok = np.empty(d.shape[0], np.uint8)
    lib().or_dir_to_img(*_cam_args(kind, W, H, fovx, fovy, pp), _i64(d.shape[0]), _p(d), _p(uv), _p(ok))
    return uv, ok


def interp_weights(nside, theta, phi):
    """Interp_H: 4 NESTED pixels and weights per (colatitude, longitude)."""
    theta = np.ascontiguousarray(theta, np.float64).ravel()
    phi = np.ascontiguousarray(phi, np.float64).ravel()
    pix = np.empty((theta.size, 4), np.int64); w = np.empty((theta.size, 4))
    lib().or_interp_weights(_i64(nside), _i64(theta.size), _p(theta), _p(phi), _p(pix), _p(w))
    return pix, w


def sphere_to_image(nside, hmap, kind, W, H, fovx=360.0, fovy=None, pp=(0.0, 0.0)):
    """Camera image (H, W, 3) from a HEALPix map (Npix, 3) in the camera frame, and validity (H, W)."""
    hmap = np.ascontiguousarray(hmap, np.float64).reshape(-1, 3)
    img = np.empty((H, W, 3)); ok = np.empty((H, W), np.uint8)
    lib().or_sphere_to_image(_i64(nside), _p(hmap), ctypes.c_int(kind), _i64(W), _i64(H),
                             *_fov_pp(fovx, fovy, pp), _p(img), _p(ok))
    return img, ok


def sphere_to_image_adjoint(nside, dimg, kind, W, H, fovx=360.0, fovy=None, pp=(0.0, 0.0)):
    dimg = np.ascontiguousarray(dimg, np.float64).reshape(H, W, 3)
    dmap = np.empty((12 * nside * nside, 3))
    lib().or_sphere_to_image_adjoint(_i64(nside), _p(dimg), ctypes.c_int(kind), _i64(W), _i64(H),
                                     *_fov_pp(fovx, fovy, pp), _p(dmap))
    return dmap


def image_to_sphere(nside, img, kind, W, H, fovx=360.0, fovy=None, pp=(0.0, 0.0)):
    """HEALPix map (Npix, 3) and mask M_C from a camera image (H, W, 3)."""
    img = np.ascontiguousarray(img, np.float64).reshape(H, W, 3)
    hmap = np.empty((12 * nside * nside, 3)); m = np.empty(12 * nside * nside, np.uint8)
    lib().or_image_to_sphere(_i64(nside), _p(img), ctypes.c_int(kind), _i64(W), _i64(H),
                             *_fov_pp(fovx, fovy, pp), _p(hmap), _p(m))
    return hmap, m


def sphere_to_image_at(nside, hmap, kind, W, H, fovx, fovy, uv, pp=(0.0, 0.0)):
    """sphere_to_image at image points uv (n, 2) only: values (n, 3) and validity."""
    hmap = np.ascontiguousarray(hmap, np.float64).reshape(-1, 3)
    uv = np.ascontiguousarray(uv, np.float64).reshape(-1, 2)
    out = np.empty((uv.shape[0], 3)); ok = np.empty(uv.shape[0], np.uint8)
    lib().or_sphere_to_image_at(_i64(nside), _p(hmap), ctypes.c_int(kind), _i64(W), _i64(H),
                                *_fov_pp(fovx, fovy, pp), _i64(uv.shape[0]), _p(uv), _p(out), _p(ok))
    return out, ok


def image_to_sphere_at(nside, img, kind, W, H, fovx, fovy, qs, pp=(0.0, 0.0)):
    """image_to_sphere at NESTED pixels qs only: values (n, 3) and M_C."""
    img = np.ascontiguousarray(img, np.float64).reshape(H, W, 3)
    qs = np.ascontiguousarray(qs, np.int64)
    out = np.empty((qs.size, 3)); m = np.empty(qs.size, np.uint8)
    lib().or_image_to_sphere_at(_i64(nside), _p(img), ctypes.c_int(kind), _i64(W), _i64(H),
                                *_fov_pp(fovx, fovy, pp), _i64(qs.size), _p(qs), _p(out), _p(m))
    return out, m



# ---------------------------------------------------------------------------
# NESTED quadtree tile query (Algorithm 2)
# ---------------------------------------------------------------------------

def pixrad(o: int) -> float:
    """PixRad(o): the largest node-centre-to-boundary angle at order o, rounded up to 2^-20."""
    return lib().or_pixrad(ctypes.c_int(o))


def query_disc_nested(kt, log2f, g, rs):
    """Tiles (order kt) of one disc (unit centre g, radius rs) by Algorithm 2 with refinement 2^log2f."""
    g = np.ascontiguousarray(g, np.float64)
    out = np.empty(1 << 16, np.int64)
    n = lib().or_query_disc_nested(ctypes.c_int(kt), ctypes.c_int(log2f), _p(g), _f64(rs), _p(out), _i64(out.size))
    if n > out.size:
        out = np.empty(n, np.int64)
        lib().or_query_disc_nested(ctypes.c_int(kt), ctypes.c_int(log2f), _p(g), _f64(rs), _p(out), _i64(out.size))
    return out[:n].copy()


def tile_lists_nested(k, b, log2f, g, rs, valid, dbits, active):
    """CSR lists like tile_lists, with Algorithm 2 (refinement 2^log2f) as the query."""
    g = np.ascontiguousarray(g, np.float64); rs = np.ascontiguousarray(rs, np.float64)
    valid = np.ascontiguousarray(valid, np.int32); dbits = np.ascontiguousarray(dbits, np.uint32)
    active = np.ascontiguousarray(active, np.uint8)
    P = rs.size
    nt = 12 * 4 ** (k - b)
    start = np.empty(nt + 1, np.int64)
    m = lib().or_tile_lists_nested(ctypes.c_int(k), ctypes.c_int(b), ctypes.c_int(log2f), _i64(P), _p(g), _p(rs),
                                   _p(valid), _p(dbits), _p(active), _p(start), None)
    ids = np.empty(m, np.int64)
    lib().or_tile_lists_nested(ctypes.c_int(k), ctypes.c_int(b), ctypes.c_int(log2f), _i64(P), _p(g), _p(rs),
                               _p(valid), _p(dbits), _p(active), None, _p(ids))
    return start, ids


# ---------------------------------------------------------------------------
# RING query at a finer search resolution (Sec. 3.3, Sec. D.2: Algorithm 3 at order
# k_t + log2 f, query pixels mapped to their tiles)
# ---------------------------------------------------------------------------

def tile_lists_ringf(k, b, log2f, g, rs, valid, dbits, active):
    """CSR lists like tile_lists, with Algorithm 3 run at query order k - b + log2f: a tile
    is listed once when one of its query pixels has its centre within r_s + rho(k, b - log2f)
    (+1e-7) of the Gaussian and the tile is active. log2f = 0 is tile_lists."""
    g = np.ascontiguousarray(g, np.float64); rs = np.ascontiguousarray(rs, np.float64)
    valid = np.ascontiguousarray(valid, np.int32); dbits = np.ascontiguousarray(dbits, np.uint32)
    active = np.ascontiguousarray(active, np.uint8)
    P = rs.size
    nt = 12 * 4 ** (k - b)
    start = np.empty(nt + 1, np.int64)
    lib().or_tile_lists_ringf.restype = ctypes.c_int64
    m = lib().or_tile_lists_ringf(ctypes.c_int(k), ctypes.c_int(b), ctypes.c_int(log2f), _i64(P), _p(g), _p(rs),
                                  _p(valid), _p(dbits), _p(active), _p(start), None)
    ids = np.empty(m, np.int64)
    lib().or_tile_lists_ringf(ctypes.c_int(k), ctypes.c_int(b), ctypes.c_int(log2f), _i64(P), _p(g), _p(rs),
                              _p(valid), _p(dbits), _p(active), None, _p(ids))
    return start, ids
