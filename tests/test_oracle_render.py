"""Pins for the oracle's preprocessing, offset, tile lists and compositing.

Sec. 3.2 (Eqs. lonlat_projection, arc_scaling), Sec. 3.3 (Eq. ring_phi_range,
Algorithm 3), Sec. 3.4 (Eq. unified_rendering, Algorithm 1).
"""
import math

import numpy as np
import pytest
import scipy.special as sps
import torch

import oracle as O
from paper_2606_29794_b300 import synth as S
from tests.dense_ref import params_from_scene, render_dense, sh_cartesian


def _single(mu, s, o, col, q=(1.0, 0.0, 0.0, 0.0)):
    sh0 = (np.asarray(col, np.float64) - 0.5) / (0.5 / math.sqrt(math.pi))
    return dict(means=np.array([mu], np.float64), scales=np.array([[s, s, s]], np.float64),
                rotations=np.array([q], np.float64), opacities=np.array([o], np.float64),
                sh=sh0.reshape(1, 1, 3), sh_degree=0)


def _f64view(v):
    v = dict(v)
    v["W"] = np.asarray(v["W"], np.float64); v["b"] = np.asarray(v["b"], np.float64)
    return v


# --------------------------------------------------------------------------- preprocess

def test_arc_jacobian_equals_tangent_frame_over_r():
    # S_phi J (Eqs. 1-2) equals [e_omega; e_phi] / r: FD Jacobian of Pi vs the frame.
    rng = np.random.default_rng(3)
    for _ in range(20):
        t = rng.standard_normal(3) * 3

        def Pi(t):
            return np.array([math.atan2(t[0], t[2]), math.atan2(t[1], math.hypot(t[0], t[2]))])
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = 1e-6
            J[:, k] = (Pi(t + e) - Pi(t - e)) / 2e-6
        r = np.linalg.norm(t); rho = math.hypot(t[0], t[2])
        SJ = np.diag([rho / r, 1.0]) @ J
        e_w = np.array([t[2], 0, -t[0]]) / rho
        e_p = np.array([-t[0] * t[1], rho * rho, -t[2] * t[1]]) / (rho * r)
        assert np.allclose(SJ, np.stack([e_w, e_p]) / r, atol=1e-8)


def test_isotropic_sigma_arc_and_radius():
    rng = np.random.default_rng(4)
    P = 50
    sc = dict(means=rng.standard_normal((P, 3)) * 3, scales=np.repeat(rng.uniform(0.01, 0.3, (P, 1)), 3, 1),
              rotations=rng.standard_normal((P, 4)), opacities=np.full(P, 0.5), sh=np.zeros((P, 1, 3)), sh_degree=0)
    Rw = S.random_rotation(rng)     # exactly orthonormal in FP64 (no float32 rounding)
    v = dict(W=Rw, b=-Rw @ np.array([0.2, 0.1, -0.3]), nside_log2=5, cam=0)
    blur = 1e-5
    pre = O.preprocess(sc, v, O.Config(blur=blur))
    t = sc["means"] @ v["W"].T + v["b"]
    r = np.linalg.norm(t, axis=1)
    ok = pre["valid"] == 1
    s2 = sc["scales"][:, 0] ** 2 / r ** 2 + blur
    assert np.allclose(pre["sigma_arc"][ok, 0], s2[ok], rtol=1e-10)
    assert np.allclose(pre["sigma_arc"][ok, 1], 0, atol=1e-12 * s2[ok].max())
    assert np.allclose(pre["sigma_arc"][ok, 2], s2[ok], rtol=1e-10)
    assert np.allclose(pre["rs"][ok], 3 * np.sqrt(s2[ok]), rtol=1e-10)


def test_radius_is_three_sigma_of_largest_eigenvalue():
    sc = S.make_scene(200, 0, seed=7)
    pre = O.preprocess(sc, S.make_view(6), O.Config())
    a, b, c = pre["sigma_arc"].T
    lam = np.array([np.linalg.eigvalsh(np.array([[x, y], [y, z]]))[-1] for x, y, z in zip(a, b, c)])
    ok = pre["valid"] == 1
    assert np.allclose(pre["rs"][ok], 3 * np.sqrt(lam[ok]), rtol=1e-12)
    for i in np.nonzero(ok)[0][:20]:
        Sm = np.array([[a[i], b[i]], [b[i], c[i]]])
        Q = np.array([[pre["conic"][i, 0], pre["conic"][i, 1]], [pre["conic"][i, 1], pre["conic"][i, 2]]])
        assert np.allclose(Sm @ Q, np.eye(2), atol=1e-9)


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(5)
    d = rng.standard_normal((500, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = O.sh_basis(d, 3)
    th = np.arccos(d[:, 2]); ph = np.arctan2(d[:, 1], d[:, 0])
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            c = sps.sph_harm_y(l, abs(m), th, ph)
            ref = c.real if m == 0 else (math.sqrt(2) * c.real if m > 0 else math.sqrt(2) * c.imag)
            assert np.allclose(Y[:, k], ref, atol=1e-12), (l, m)
            k += 1
    assert np.allclose(sh_cartesian(torch.as_tensor(d), 3).numpy(), Y, atol=1e-12)


def test_sh_gradient_fd():
    rng = np.random.default_rng(6)
    d = rng.standard_normal((50, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y, dY = O.sh_basis(d, 3, with_grad=True)
    for i in range(50):
        tdir = np.cross(d[i], rng.standard_normal(3)); tdir /= np.linalg.norm(tdir)
        h = 1e-6
        dp = d[i] + h * tdir; dp /= np.linalg.norm(dp)
        dm = d[i] - h * tdir; dm /= np.linalg.norm(dm)
        num = (O.sh_basis(dp, 3) - O.sh_basis(dm, 3))[0] / (2 * h)
        assert np.allclose(dY[i] @ tdir, num, atol=1e-7)


def test_offset_haversine_equals_tangent_frame():
    # d = d_gc (sin beta, cos beta) equals theta * u/|u| with u the pixel direction
    # in the (e_omega, e_phi) frame at the Gaussian (azimuthal equidistant coordinates).
    rng = np.random.default_rng(8)
    n = 2000
    wp, wg = rng.uniform(-np.pi, np.pi, (2, n))
    pp, pg = np.arcsin(rng.uniform(-0.99, 0.99, (2, n)))
    d = O.spherical_offset(wp, pp, wg, pg)
    P = np.stack([np.cos(pp) * np.sin(wp), np.sin(pp), np.cos(pp) * np.cos(wp)], 1)
    G = np.stack([np.cos(pg) * np.sin(wg), np.sin(pg), np.cos(pg) * np.cos(wg)], 1)
    e_w = np.stack([np.cos(wg), np.zeros(n), -np.sin(wg)], 1)
    e_p = np.stack([-np.sin(pg) * np.sin(wg), np.cos(pg), -np.sin(pg) * np.cos(wg)], 1)
    u = np.stack([(P * e_w).sum(1), (P * e_p).sum(1)], 1)
    th = np.arctan2(np.linalg.norm(u, axis=1), (P * G).sum(1))
    ref = th[:, None] * u / np.linalg.norm(u, axis=1, keepdims=True)
    assert np.allclose(d, ref, atol=1e-12)


# --------------------------------------------------------------------------- tile lists

@pytest.mark.parametrize("k,b", [(4, 1), (5, 2), (6, 3), (6, 4)])
def test_ring_query_equals_bruteforce_membership(k, b):
    rng = np.random.default_rng(k * 10 + b)
    P = 300
    g = rng.standard_normal((P, 3)); g /= np.linalg.norm(g, axis=1, keepdims=True)
    g[:4] = [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0.6, 0.8, 0]]     # poles and face seams
    rs = np.exp(rng.uniform(np.log(1e-3), np.log(2.5), P))
    valid = np.ones(P, np.int32)
    for kind, fov in [(O.CAM_FULL, 360.0), (O.CAM_FISHEYE, 190.0), (O.CAM_PINHOLE, 80.0)]:
        m, _ = O.mask(1 << k, kind, fov)
        act = O.active_tiles(k, b, m)
        rho = O.tile_rho(k, b)
        start, ids = O.tile_lists(k, b, g, rs, valid, np.arange(P, dtype=np.uint32), rho, act)
        mem = O.tile_lists_bruteforce(k, b, g, rs, valid, rho, act)
        for t in range(act.size):
            assert sorted(ids[start[t]:start[t + 1]]) == list(np.nonzero(mem[:, t])[0])


@pytest.mark.parametrize("k,b", [(5, 2), (6, 3)])
def test_subset_lists_equal_full_lists(k, b):
    # The per-tile builder used by the full-size sampled checks: same ids, same
    # order as the RING-built lists on the chosen tiles, empty lists elsewhere.
    rng = np.random.default_rng(40 + k)
    P = 400
    g = rng.standard_normal((P, 3)); g /= np.linalg.norm(g, axis=1, keepdims=True)
    g[:2] = [[0, 0, 1], [0, 0, -1]]
    rs = np.exp(rng.uniform(np.log(1e-3), np.log(1.5), P))
    valid = (rng.random(P) > 0.1).astype(np.int32)
    dbits = rng.integers(0, 40, P).astype(np.uint32)             # many equal depths: ties by id
    m, _ = O.mask(1 << k, O.CAM_FISHEYE, 200.0)
    act = O.active_tiles(k, b, m)
    rho = O.tile_rho(k, b)
    start, ids = O.tile_lists(k, b, g, rs, valid, dbits, rho, act)
    nt = act.size
    sel = np.concatenate([rng.choice(nt, 12, replace=False), [0, nt - 1], np.nonzero(act == 0)[0][:2]])
    s2, i2 = O.tile_lists_subset(k, b, g, rs, valid, dbits, rho, act, sel)
    for t in range(nt):
        got = list(i2[s2[t]:s2[t + 1]])
        want = list(ids[start[t]:start[t + 1]]) if t in set(sel.tolist()) else []
        assert got == want


def test_tile_rho_bounds_pixel_distance():
    for k, b in [(5, 2), (6, 4)]:
        rho = O.tile_rho(k, b)
        nt = 12 * 4 ** (k - b)
        ct = O.pix2vec_nest(1 << (k - b), np.arange(nt))
        pc = O.pix2vec_nest(1 << k, np.arange(12 * 4 ** k)).reshape(nt, 4 ** b, 3)
        ang = np.arccos(np.clip(np.einsum("tk,tjk->tj", ct, pc), -1, 1))
        assert ang.max() <= rho < ang.max() + 2 ** -19


def test_lists_sorted_by_depth_then_index():
    sc = S.make_scene(500, 0, seed=9)
    R = O.render(sc, S.make_view(5), O.Config(tile_level=2))
    key = O.depth_bits(R.pre["r"])
    for t in range(R.start.size - 1):
        ids = R.ids[R.start[t]:R.start[t + 1]]
        pairs = list(zip(key[ids], ids))
        assert pairs == sorted(pairs)


# --------------------------------------------------------------------------- compositing

@pytest.mark.parametrize("where", ["equator", "pole", "corner", "random"])
def test_single_isotropic_gaussian_closed_form(where):
    # I(p) = c min(0.99, o exp(-theta^2 / (2 sigma_a^2))) for theta <= 3 sigma_a, else 0,
    # sigma_a^2 = s^2 / r^2 + blur  (Eq. unified_rendering with one Gaussian).
    rng = np.random.default_rng(11)
    dist, s, o, col = 3.0, 0.09, 0.7, np.array([0.2, 0.5, 0.9])
    if where == "equator":
        dirc = np.array([0.3, 0.0, 1.0])
    elif where == "pole":
        dirc = np.array([0.0, 1.0, 0.0])
    elif where == "corner":
        # HEALPix vertex at longitude pi/4 on the equator (faces 0, 4, 5, 8 meet);
        # camera direction (d_x, d_y, d_z) = HEALPix (Y, Z, X)
        dirc = np.array([math.sin(math.pi / 4), 0.0, math.cos(math.pi / 4)])
    else:
        dirc = rng.standard_normal(3)
    dirc = dirc / np.linalg.norm(dirc)
    Rw = S.random_rotation(rng) if where == "random" else np.eye(3)
    mu_world = Rw.T @ (dirc * dist)
    sc = _single(mu_world, s, o, col, q=tuple(rng.standard_normal(4)))
    v = dict(W=Rw, b=np.zeros(3), nside_log2=6, cam=0)    # FP64 rotation, no float32 rounding
    blur = 2e-6
    R = O.render(sc, v, O.Config(blur=blur, tile_level=3))
    pv = O.pix2vec_nest(64, np.arange(O.npix(64)))
    pd = np.stack([pv[:, 1], pv[:, 2], pv[:, 0]], 1)
    th = np.arccos(np.clip(pd @ dirc, -1, 1))
    sa2 = s * s / dist ** 2 + blur
    a = np.where(th * th / sa2 <= 9.0, np.minimum(0.99, o * np.exp(-0.5 * th * th / sa2)), 0.0)
    ref = a[:, None] * col[None, :]
    keep = np.abs(th * th / sa2 - 9.0) > 1e-6
    assert np.abs(R.image - ref)[keep].max() < 1e-12
    assert (a > 0).sum() > 20


def test_single_gaussian_integral_equal_area():
    # sum_p I(p) Omega_pix approximates the integral of alpha over the sphere.
    dist, s, o = 3.0, 0.15, 0.6
    sc = _single([0.0, 0.0, dist], s, o, [1.0, 1.0, 1.0])
    nside = 256
    R = O.render(sc, S.make_view(8), O.Config(blur=0.0))
    total = R.image[:, 0].sum() * 4 * np.pi / O.npix(nside)
    sa2 = s * s / dist ** 2
    thg = np.linspace(0, 3 * np.sqrt(sa2), 200001)
    f = np.minimum(0.99, o * np.exp(-0.5 * thg ** 2 / sa2)) * np.sin(thg)
    exact = 2 * np.pi * np.trapezoid(f, thg)
    assert abs(total - exact) / exact < 2e-3


def test_two_gaussians_same_ray():
    # front-to-back: I = c1 a1 + c2 a2 (1 - a1), the nearer one first.
    c1, c2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    sc1 = _single([0, 0, 2.0], 0.05, 0.6, c1)
    sc2 = _single([0, 0, 4.0], 0.1, 0.5, c2)
    sc = {k: (np.concatenate([sc2[k], sc1[k]]) if k != "sh_degree" else 0) for k in sc1}
    R = O.render(sc, S.make_view(6), O.Config(blur=0.0))
    p = O.vec2pix_nest(64, np.array([[1.0, 0.0, 0.0]]))[0]     # camera +z axis
    th = np.arccos(O.pix2vec_nest(64, [p])[0][0])
    a1 = 0.6 * np.exp(-0.5 * th ** 2 / (0.05 ** 2 / 4.0))
    a2 = 0.5 * np.exp(-0.5 * th ** 2 / (0.1 ** 2 / 16.0))
    assert np.allclose(R.image[p], c1 * a1 + c2 * a2 * (1 - a1), atol=1e-13)


def test_permutation_invariance():
    sc = S.make_scene(300, 3, seed=12)
    perm = np.random.default_rng(0).permutation(300)
    sc2 = {k: (v[perm] if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    v = S.make_view(5)
    R1 = O.render(sc, v, O.Config()); R2 = O.render(sc2, v, O.Config())
    assert np.allclose(R1.image, R2.image, atol=1e-13)


@pytest.mark.parametrize("b", [1, 2, 3])
@pytest.mark.parametrize("kind,fov", [(O.CAM_FULL, 360.0), (O.CAM_FISHEYE, 190.0), (O.CAM_PINHOLE, 90.0)])
def test_tiled_equals_dense_bruteforce(b, kind, fov):
    rng = np.random.default_rng(b * 7 + kind)
    sc = S.make_scene(150, 3, seed=13 + b, r_min=1.5, r_max=4.0, logscale_mu=-1.8)
    v = _f64view(S.random_pose_view(rng, 4, kind, fov, fov, radius=0.3))
    cfg = O.Config(tile_level=b)
    R = O.render(sc, v, cfg)
    with torch.no_grad():
        C, T = render_dense(params_from_scene(sc), v, cfg, R.pix, 16)
    ok = R.amb[R.pix] == 0
    assert np.abs(C.numpy() - R.image[R.pix])[ok].max() < 1e-12
    assert np.abs(T.numpy() - R.T[R.pix])[ok].max() < 1e-12


@pytest.mark.parametrize("b", [2, 3])
@pytest.mark.parametrize("kind,fov", [(O.CAM_FULL, 360.0), (O.CAM_FISHEYE, 190.0)])
def test_literal_semantics_equals_dense_over_tile_members(b, kind, fov):
    # the paper's literal tile semantics (Sec. 3.3 ablation): every Gaussian listed for a tile
    # contributes at every pixel of the tile, with no m <= 9 cutoff; the oracle takes it with an
    # infinite cutoff (the lists keep their 3-sigma radius). Dense reference: all Gaussians in depth
    # order, restricted to the members of each pixel's tile (brute-force membership).
    rng = np.random.default_rng(b * 11 + kind)
    sc = S.make_scene(120, 3, seed=31 + b, r_min=1.5, r_max=4.0, logscale_mu=-1.8)
    v = _f64view(S.random_pose_view(rng, 4, kind, fov, fov, radius=0.3))
    cfg = O.Config(tile_level=b, cutoff=math.inf)
    R = O.render(sc, v, cfg)
    pre = R.pre
    member = O.tile_lists_bruteforce(4, b, pre["g"], pre["rs"], pre["valid"], O.tile_rho(4, b), R.active)
    members = member[:, R.pix >> (2 * b)].T.astype(bool)         # (n, P)
    with torch.no_grad():
        C, T = render_dense(params_from_scene(sc), v, cfg, R.pix, 16, members=members)
    ok = R.amb[R.pix] == 0
    assert ok.mean() > 0.95
    assert np.abs(C.numpy() - R.image[R.pix])[ok].max() < 1e-12
    assert np.abs(T.numpy() - R.T[R.pix])[ok].max() < 1e-12
    # the semantics differ: contributions beyond the 3-sigma ellipse change some pixels
    R9 = O.render(sc, v, O.Config(tile_level=b))
    assert np.abs(R9.image[R.pix] - R.image[R.pix]).max() > 1e-6


def _quat_mul(a, b):
    """Hamilton product of (w, x, y, z) quaternions, rows of a with rows of b: R(a b) = R(a) R(b)."""
    w1, v1 = a[..., :1], a[..., 1:]
    w2, v2 = b[..., :1], b[..., 1:]
    return np.concatenate([w1 * w2 - (v1 * v2).sum(-1, keepdims=True), w1 * v2 + w2 * v1 + np.cross(v1, v2)], -1)


@pytest.mark.parametrize("kind,fov", [(O.CAM_FISHEYE, 190.0), (O.CAM_PINHOLE, 90.0)])
def test_joint_rotation_of_scene_and_camera_leaves_the_map_unchanged(kind, fov):
    # the map lives in the camera frame: turning every Gaussian (position and orientation) and the
    # camera by the same world rotation Q (W' = W Q^T, b' = b) changes nothing the camera sees.
    # SH degree 0 (a colour that does not depend on the world direction). A wrong frame anywhere in
    # the view transform, the quaternion-to-rotation map or the covariance projection breaks it.
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(41 + kind)
    sc = S.make_scene(300, 0, seed=42 + kind, r_min=1.5, r_max=4.0, logscale_mu=-2.0)
    v = _f64view(S.random_pose_view(rng, 5, kind, fov, fov, radius=0.3))
    Q = S.random_rotation(rng)
    qQ = np.roll(Rotation.from_matrix(Q).as_quat(), 1)               # (x, y, z, w) -> (w, x, y, z)
    sc2 = dict(sc, means=sc["means"] @ Q.T, rotations=_quat_mul(np.broadcast_to(qQ, sc["rotations"].shape),
                                                                  np.asarray(sc["rotations"], np.float64)))
    v2 = dict(v, W=v["W"] @ Q.T)
    cfg = O.Config(tile_level=3)
    R1, R2 = O.render(sc, v, cfg), O.render(sc2, v2, cfg)
    assert np.array_equal(R1.mask, R2.mask)
    ok = (R1.amb == 0) & (R2.amb == 0)
    assert ok[R1.pix].mean() > 0.99 and (R1.T[R1.pix] < 1).mean() > 0.2       # a non-trivial image
    assert np.abs(R1.image - R2.image)[ok].max() < 1e-10
    assert np.abs(R1.T - R2.T)[ok].max() < 1e-10


@pytest.mark.parametrize("seed", [100, 101])
def test_band_variants_equal_dense_with_moved_thresholds(seed):
    # composite_variants follows both outcomes of a cutoff or termination decision whose FP64
    # value lies within its FP32 band. Where a pixel has exactly one such decision (two leaves),
    # the two leaves must be the dense reference's pixel value with that threshold moved to
    # either edge of its band: cutoff (1 -+ 2e-5) for a cutoff decision, eps (1 -+ 1e-4) for a
    # termination decision. An opaque scene makes both kinds frequent.
    sc = S.make_scene(1500, 0, seed=seed, r_min=1.5, r_max=4.0, logscale_mu=-1.2)
    sc["opacities"] = np.full_like(sc["opacities"], 0.9)
    v = _f64view(S.make_view(6))
    cfg = O.Config(tile_level=3)
    R = O.render(sc, v, cfg)
    a = R.amb[R.pix]
    params = params_from_scene(sc)
    for flag, field, band in ((O.AMB_CUTOFF, "cutoff", 2e-5), (O.AMB_TERM, "eps_T", 1e-4)):
        sel = R.pix[a == flag]
        V = O.composite_variants(6, 3, R.pre, sc["opacities"], R.start, R.ids, sel, cfg)
        two = V["n"] == 2
        assert two.sum() >= 15, (flag, two.sum())
        sel, img, T = sel[two], V["image"][two], V["T"][two]
        outs = []
        for f in (1 - band, 1 + band):
            c2 = O.Config(tile_level=3, **{field: getattr(cfg, field) * f})
            with torch.no_grad():
                C, Td = render_dense(params, v, c2, sel, 64)
            outs.append((C.numpy(), Td.numpy()))
        (Clo, Tlo), (Chi, Thi) = outs
        d = lambda C1, T1, l: np.maximum(np.abs(C1 - img[:, l]).max(1), np.abs(T1 - T[:, l]))
        straight = np.maximum(d(Clo, Tlo, 0), d(Chi, Thi, 1))
        crossed = np.maximum(d(Clo, Tlo, 1), d(Chi, Thi, 0))
        assert np.minimum(straight, crossed).max() < 1e-12
        # the leaves really differ (a termination decision at the end of the list may not)
        assert (np.abs(img[:, 0] - img[:, 1]).max(1) > 0).mean() > 0.9
