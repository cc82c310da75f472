"""Pins for the oracle's sphere <-> image resampling (Eq. camera_synthesis;
Eqs. supp_image_to_healpix, supp_hssim_mask; camera models of Sec. D.1).

Each check is fixed by something other than the oracle's own formulas: closed
forms of the printed camera models, interpolation identities (exactness at
pixel centres, reproduction of functions linear in colatitude and longitude,
partition of unity), the adjoint identity, and equality of the resampled mask
with the FoV mask pinned against the paper's solid angles.
"""
import math

import numpy as np
import pytest

import oracle as O

Z = (0.0, 0.0)
CAMS = [(O.CAM_PINHOLE, 90.0, 70.0, Z), (O.CAM_PINHOLE, 90.0, 70.0, (0.3, -0.45)), (O.CAM_FISHEYE, 190.0, 190.0, Z),
        (O.CAM_FISHEYE, 200.0, 170.0, Z), (O.CAM_FULL, 360.0, 180.0, Z)]


def _ring_thetas(nside):
    th, _ = O.pix2ang_nest(nside, np.arange(12 * nside * nside))
    return np.unique(np.round(th, 12))


@pytest.mark.parametrize("nside", [1, 2, 8, 32])
def test_interp_is_exact_at_pixel_centres(nside):
    q = np.arange(12 * nside * nside)
    th, ph = O.pix2ang_nest(nside, q)
    pix, w = O.interp_weights(nside, th, ph)
    # all weight on the pixel itself (other entries zero weight or the same pixel)
    on_self = np.where(pix == q[:, None], w, 0.0).sum(1)
    assert np.allclose(on_self, 1.0, atol=1e-12)


@pytest.mark.parametrize("nside", [4, 16])
def test_weights_partition_of_unity_and_nonnegative(nside):
    rng = np.random.default_rng(nside)
    v = rng.standard_normal((4000, 3)); v /= np.linalg.norm(v, axis=1, keepdims=True)
    th = np.arccos(np.clip(v[:, 2], -1, 1)); ph = np.mod(np.arctan2(v[:, 1], v[:, 0]), 2 * np.pi)
    th[:3] = [0.0, np.pi, 1e-9]
    pix, w = O.interp_weights(nside, th, ph)
    assert np.allclose(w.sum(1), 1.0, atol=1e-12) and (w >= -1e-15).all()
    assert ((pix >= 0) & (pix < 12 * nside * nside)).all()


@pytest.mark.parametrize("nside", [4, 16, 64])
def test_linear_in_colatitude_and_longitude_is_reproduced(nside):
    # between the first and the last ring, f(q) = a + b theta_q + c phi_q is interpolated exactly
    # where no bracket crosses the longitude wrap
    q = np.arange(12 * nside * nside)
    thq, phq = O.pix2ang_nest(nside, q)
    f = 0.2 + 1.3 * thq + 0.7 * phq
    rt = _ring_thetas(nside)
    rng = np.random.default_rng(1)
    th = rng.uniform(rt[0], rt[-1], 3000)
    ph = rng.uniform(np.pi / 4 + 1e-3, 2 * np.pi - np.pi / 4 - 1e-3, 3000)   # every ring's first pixel is at phi <= pi/4
    pix, w = O.interp_weights(nside, th, ph)
    assert np.allclose((w * f[pix]).sum(1), 0.2 + 1.3 * th + 0.7 * ph, atol=1e-10)


@pytest.mark.parametrize("nside", [2, 8])
def test_pole_value_is_mean_of_first_ring_and_interpolation_is_continuous(nside):
    rng = np.random.default_rng(3)
    f = rng.random(12 * nside * nside)
    thq, _ = O.pix2ang_nest(nside, np.arange(f.size))
    north = np.argsort(thq)[:4]
    south = np.argsort(-thq)[:4]
    for th0, ring in [(0.0, north), (np.pi, south)]:
        pix, w = O.interp_weights(nside, np.full(5, th0), np.linspace(0.1, 6.0, 5))
        assert np.allclose((w * f[pix]).sum(1), f[ring].mean(), atol=1e-12)
    # continuity: nearby directions give nearby values (a wrong bracket would jump)
    v = rng.standard_normal((2000, 3)); v /= np.linalg.norm(v, axis=1, keepdims=True)
    th = np.arccos(np.clip(v[:, 2], -1, 1)); ph = np.mod(np.arctan2(v[:, 1], v[:, 0]), 2 * np.pi)
    p1, w1 = O.interp_weights(nside, th, ph)
    p2, w2 = O.interp_weights(nside, np.clip(th + 1e-7, 0, np.pi), np.mod(ph + 1e-7, 2 * np.pi))
    assert np.abs((w1 * f[p1]).sum(1) - (w2 * f[p2]).sum(1)).max() < 1e-4 * nside


def test_camera_closed_forms():
    W, H = 64, 48
    # pinhole: principal point -> optical axis; image corner -> (-tan(fx/2), -tan(fy/2), 1) normalised
    d, ok = O.img_to_dir(O.CAM_PINHOLE, W, H, 90.0, 70.0, [[W / 2, H / 2], [0.0, 0.0]])
    assert ok.all() and np.allclose(d[0], [0, 0, 1])
    c = np.array([-1.0, -math.tan(math.radians(35.0)), 1.0])
    assert np.allclose(d[1], c / np.linalg.norm(c))
    # fisheye: the end of the ellipse's horizontal semi-axis a = f_x pi/2 has incident angle (pi/2) w_x
    for fx_deg, fy_deg in [(190.0, 190.0), (200.0, 170.0)]:
        wx, wy = fx_deg / 180, fy_deg / 180
        a, b = (W / math.pi) * math.pi / 2, (H / math.pi) * math.pi / 2
        d, ok = O.img_to_dir(O.CAM_FISHEYE, W, H, fx_deg, fy_deg, [[W / 2 + a, H / 2], [W / 2, H / 2 + b],
                                                                    [W / 2 + a * 1.01, H / 2]])
        assert ok.tolist() == [1, 1, 0]
        assert np.allclose(d[0], [math.sin(math.pi / 2 * wx), 0, math.cos(math.pi / 2 * wx)])
        assert np.allclose(d[1], [0, math.sin(math.pi / 2 * wy), math.cos(math.pi / 2 * wy)])
    # off-centre pinhole (Eq. persp_sphere with c_x = (W/2)(1 + ppx), c_y = (H/2)(1 + ppy)): the
    # principal point -> optical axis; corner (0, 0) -> x = -c_x / f_x; corner (W, H) -> (W - c_x) / f_x
    ppx, ppy = 0.3, -0.45
    cx, cy = W / 2 * (1 + ppx), H / 2 * (1 + ppy)
    fpx, fpy = W / (2 * math.tan(math.radians(45.0))), H / (2 * math.tan(math.radians(35.0)))
    d, ok = O.img_to_dir(O.CAM_PINHOLE, W, H, 90.0, 70.0, [[cx, cy], [0.0, 0.0], [W, H]], pp=(ppx, ppy))
    assert ok.all() and np.allclose(d[0], [0, 0, 1])
    for dd, (u, v) in zip(d[1:], [(0.0, 0.0), (W, H)]):
        c = np.array([(u - cx) / fpx, (v - cy) / fpy, 1.0])
        assert np.allclose(dd, c / np.linalg.norm(c))
    assert np.isclose(d[1, 0] / d[1, 2], -1.3) and np.isclose(d[2, 0] / d[2, 2], 0.7)      # tan 45 = 1
    # panorama: centre -> forward; left edge -> backward; top row -> +y (phi = pi/2)
    d, ok = O.img_to_dir(O.CAM_FULL, W, H, 360.0, 180.0, [[W / 2, H / 2], [0.0, H / 2], [W / 2, 0.0]])
    assert np.allclose(d, [[0, 0, 1], [0, 0, -1], [0, 1, 0]], atol=1e-12)


@pytest.mark.parametrize("kind,fx,fy,pp", CAMS)
def test_camera_round_trip(kind, fx, fy, pp):
    W, H = 96, 72
    rng = np.random.default_rng(kind)
    uv = np.stack([rng.uniform(0, W, 2000), rng.uniform(0, H, 2000)], 1)
    d, ok = O.img_to_dir(kind, W, H, fx, fy, uv, pp=pp)
    uv2, ok2 = O.dir_to_img(kind, W, H, fx, fy, d[ok == 1], pp=pp)
    assert ok2.all()
    assert np.allclose(uv2, uv[ok == 1], atol=1e-9)
    assert np.allclose(np.linalg.norm(d[ok == 1], axis=1), 1.0)


@pytest.mark.parametrize("kind,fx,fy,pp", CAMS)
def test_resampled_mask_is_the_fov_mask(kind, fx, fy, pp):
    nside = 16
    m_ref, _ = O.mask(nside, kind, fx, fy, pp=pp)
    _, m = O.image_to_sphere(nside, np.zeros((40, 50, 3)), kind, 50, 40, fx, fy, pp=pp)
    assert np.array_equal(m, m_ref)


@pytest.mark.parametrize("kind,fx,fy,pp", CAMS)
def test_adjoint_identity(kind, fx, fy, pp):
    nside, W, H = 8, 40, 30
    rng = np.random.default_rng(7)
    x = rng.standard_normal((12 * nside * nside, 3))
    y = rng.standard_normal((H, W, 3))
    Ax, ok = O.sphere_to_image(nside, x, kind, W, H, fx, fy, pp=pp)
    Aty = O.sphere_to_image_adjoint(nside, y, kind, W, H, fx, fy, pp=pp)
    assert ok.any()
    assert abs((Ax * y).sum() - (x * Aty).sum()) < 1e-9 * np.abs(Ax * y).sum()


@pytest.mark.parametrize("kind,fx,fy,pp", CAMS)
def test_linear_image_is_sampled_exactly(kind, fx, fy, pp):
    # bilinear sampling reproduces an image linear in (u, v) at interior points
    nside, W, H = 32, 80, 60
    uu, vv = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    img = np.stack([0.1 + 0.01 * uu, 0.2 - 0.005 * vv, 0.003 * uu + 0.004 * vv], -1)
    hmap, m = O.image_to_sphere(nside, img, kind, W, H, fx, fy, pp=pp)
    thq, phq = O.pix2ang_nest(nside, np.arange(12 * nside * nside))
    v = np.stack([np.sin(thq) * np.cos(phq), np.sin(thq) * np.sin(phq), np.cos(thq)], 1)
    d = v[:, [1, 2, 0]]                                     # camera (d_x, d_y, d_z) = HEALPix (Y, Z, X)
    uv, ok = O.dir_to_img(kind, W, H, fx, fy, d, pp=pp)
    inner = (ok == 1) & (uv[:, 0] > 0.5) & (uv[:, 0] < W - 0.5) & (uv[:, 1] > 0.5) & (uv[:, 1] < H - 0.5)
    assert inner.sum() > 100
    u, w = uv[inner, 0], uv[inner, 1]
    want = np.stack([0.1 + 0.01 * u, 0.2 - 0.005 * w, 0.003 * u + 0.004 * w], 1)
    assert np.allclose(hmap[inner], want, atol=1e-12)


def test_sphere_image_round_trip_is_close_at_matched_resolution():
    # a smooth panorama resampled to the sphere and back stays close (interpolation, not identity)
    nside, W, H = 64, 512, 256
    uu, vv = np.meshgrid((np.arange(W) + 0.5) / W, (np.arange(H) + 0.5) / H)
    img = np.stack([0.5 + 0.4 * np.cos(2 * np.pi * uu), 0.5 + 0.4 * np.sin(np.pi * vv), 0.3 + 0.2 * uu * 0], -1)
    hmap, m = O.image_to_sphere(nside, img, O.CAM_FULL, W, H)
    back, ok = O.sphere_to_image(nside, hmap, O.CAM_FULL, W, H)
    assert m.all() and ok.all()
    assert np.abs(back - img)[8:-8].max() < 0.02


@pytest.mark.parametrize("kind,fx,fy,pp", CAMS)
def test_pointwise_entries_equal_whole_image_entries(kind, fx, fy, pp):
    nside, W, H = 8, 30, 20
    rng = np.random.default_rng(11)
    hmap = rng.random((12 * nside * nside, 3))
    img, ok = O.sphere_to_image(nside, hmap, kind, W, H, fx, fy, pp=pp)
    uu, vv = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    out, ok2 = O.sphere_to_image_at(nside, hmap, kind, W, H, fx, fy, np.stack([uu.ravel(), vv.ravel()], 1), pp=pp)
    assert np.array_equal(ok2, ok.ravel()) and np.array_equal(out, img.reshape(-1, 3))
    im = rng.random((H, W, 3))
    hm, m = O.image_to_sphere(nside, im, kind, W, H, fx, fy, pp=pp)
    qs = np.arange(12 * nside * nside)
    o2, m2 = O.image_to_sphere_at(nside, im, kind, W, H, fx, fy, qs, pp=pp)
    assert np.array_equal(m2, m) and np.array_equal(o2, hm)
