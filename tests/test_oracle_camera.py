"""Pins for the oracle's camera masks and adaptive resolution (Sec. 3.1; Sec. D.1)."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "adaptive_nside.txt")


def test_full_mask_is_all_ones():
    m, _ = O.mask(32, O.CAM_FULL)
    assert m.all()


@pytest.mark.parametrize("fx,fy", [(90.0, 90.0), (60.0, 100.0), (120.0, 70.0)])
def test_pinhole_mask_solid_angle(fx, fy):
    # The masked fraction of an equal-area grid estimates the camera's solid angle,
    # which the paper gives as 4 arcsin(sin(theta_x) sin(theta_y)) for a pinhole.
    nside = 256
    m, _ = O.mask(nside, O.CAM_PINHOLE, fx, fy)
    om = 4 * np.arcsin(np.sin(np.radians(fx / 2)) * np.sin(np.radians(fy / 2)))
    assert abs(m.mean() - om / (4 * np.pi)) < 2e-3


def _rect_solid_angle(x1, x2, y1, y2):
    """Solid angle, seen from the origin, of the rectangle [x1, x2] x [y1, y2] on the plane z = 1:
    F(x, y) = atan(x y / sqrt(1 + x^2 + y^2)) is the solid angle of [0, x] x [0, y] (signed), and
    the rectangle is F(x2, y2) - F(x1, y2) - F(x2, y1) + F(x1, y1)."""
    F = lambda x, y: np.arctan(x * y / np.sqrt(1 + x * x + y * y))
    return F(x2, y2) - F(x1, y2) - F(x2, y1) + F(x1, y1)


def test_rect_solid_angle_closed_form_reduces_to_the_centred_pinhole():
    for fx, fy in [(90.0, 90.0), (60.0, 100.0)]:
        tx, ty = np.tan(np.radians(fx / 2)), np.tan(np.radians(fy / 2))
        om = 4 * np.arcsin(np.sin(np.radians(fx / 2)) * np.sin(np.radians(fy / 2)))
        assert np.isclose(_rect_solid_angle(-tx, tx, -ty, ty), om, rtol=1e-12)


@pytest.mark.parametrize("fx,fy,pp", [(90.0, 70.0, (0.3, -0.45)), (60.0, 100.0, (-0.7, 0.2)),
                                      (120.0, 80.0, (0.9, 0.9))])
def test_off_centre_pinhole_mask_solid_angle(fx, fy, pp):
    # principal point c = (W/2)(1 + pp): the frustum spans d_x/d_z in [-t_x(1 + ppx), t_x(1 - ppx)]
    nside = 256
    m, _ = O.mask(nside, O.CAM_PINHOLE, fx, fy, pp=pp)
    tx, ty = np.tan(np.radians(fx / 2)), np.tan(np.radians(fy / 2))
    om = _rect_solid_angle(-tx * (1 + pp[0]), tx * (1 - pp[0]), -ty * (1 + pp[1]), ty * (1 - pp[1]))
    assert abs(m.mean() - om / (4 * np.pi)) < 2e-3


def test_off_centre_pinhole_mask_containment_and_mirror():
    nside = 64
    fx, fy, pp = 90.0, 70.0, (0.3, -0.45)
    tx, ty = np.tan(np.radians(fx / 2)), np.tan(np.radians(fy / 2))
    m, mg = O.mask(nside, O.CAM_PINHOLE, fx, fy, pp=pp)
    fov = lambda t: 2 * np.degrees(np.arctan(t))
    inner, _ = O.mask(nside, O.CAM_PINHOLE, fov(tx * (1 - abs(pp[0]))), fov(ty * (1 - abs(pp[1]))))
    outer, _ = O.mask(nside, O.CAM_PINHOLE, fov(tx * (1 + abs(pp[0]))), fov(ty * (1 + abs(pp[1]))))
    assert np.all(m >= inner) and np.all(m <= outer) and inner.sum() < m.sum() < outer.sum()
    # mirroring d_x (HEALPix Y -> -Y) maps the mask at ppx to the mask at -ppx
    v = O.pix2vec_nest(nside, np.arange(O.npix(nside)))
    mirror = O.vec2pix_nest(nside, v * np.array([1.0, -1.0, 1.0]))
    m_neg, _ = O.mask(nside, O.CAM_PINHOLE, fx, fy, pp=(-pp[0], pp[1]))
    far = np.abs(mg) > 1e-12
    assert np.array_equal(m_neg[mirror][far], m[far])
    # pp = 0 is the centred camera
    assert np.array_equal(O.mask(nside, O.CAM_PINHOLE, fx, fy, pp=(0.0, 0.0))[0], O.mask(nside, O.CAM_PINHOLE, fx, fy)[0])


@pytest.mark.parametrize("fov", [120.0, 180.0, 190.0, 220.0])
def test_fisheye_mask_solid_angle(fov):
    nside = 256
    m, _ = O.mask(nside, O.CAM_FISHEYE, fov)
    om = 2 * np.pi * (1 - np.cos(np.radians(fov / 2)))
    assert abs(m.mean() - om / (4 * np.pi)) < 2e-3


def test_fisheye_180_is_the_front_hemisphere():
    # w_x = w_y = 1 reduces the anisotropic model to the 180-degree fisheye (Sec. D.1).
    nside = 64
    m, _ = O.mask(nside, O.CAM_FISHEYE, 180.0)
    v = O.pix2vec_nest(nside, np.arange(O.npix(nside)))
    dz = v[:, 0]                      # camera z is the HEALPix X axis
    far = np.abs(dz) > 1e-9
    assert np.array_equal(m[far].astype(bool), dz[far] > 0)


def test_anisotropic_fisheye_axes():
    # Along the image x axis (gamma = 0) the limit angle is (pi/2) w_x, along y it is (pi/2) w_y.
    nside = 512
    m, _ = O.mask(nside, O.CAM_FISHEYE, 200.0, 160.0)
    v = O.pix2vec_nest(nside, np.arange(O.npix(nside)))
    d = np.stack([v[:, 1], v[:, 2], v[:, 0]], 1)        # camera (x, y, z)
    psi = np.degrees(np.arctan2(np.hypot(d[:, 0], d[:, 1]), d[:, 2]))
    on_x = np.abs(d[:, 1]) < 2e-3
    on_y = np.abs(d[:, 0]) < 2e-3
    assert np.all(m[on_x & (psi < 99.0)]) and not np.any(m[on_x & (psi > 101.0)])
    assert np.all(m[on_y & (psi < 79.0)]) and not np.any(m[on_y & (psi > 81.0)])


def test_adaptive_nside_golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append(line.split())
    assert rows
    for r in rows:
        kind = dict(full=O.CAM_FULL, pinhole=O.CAM_PINHOLE, fisheye=O.CAM_FISHEYE)[r[0]]
        W, H, fov, kl, kh = float(r[1]), float(r[2]), float(r[3]), int(r[4]), int(r[5])
        ns, k, kL, kH = O.adaptive_nside(kind, W, H, fov)
        assert (kL, kH) == (kl, kh)
        if len(r) > 6:
            saving = 1 - O.npix(2 ** kL) / (W * H)
            assert abs(saving - float(r[6])) < 6e-4


def test_adaptive_nside_matches_pixel_solid_angle():
    # N* makes one HEALPix pixel cover the mean solid angle of one input pixel.
    for kind, fov in [(O.CAM_FULL, 360.0), (O.CAM_FISHEYE, 190.0), (O.CAM_PINHOLE, 90.0)]:
        ns, k, kL, kH = O.adaptive_nside(kind, 1920, 1080, fov, fov)
        om_in = 4 * np.pi if kind == O.CAM_FULL else (
            2 * np.pi * (1 - np.cos(np.radians(fov / 2))) if kind == O.CAM_FISHEYE else
            4 * np.arcsin(np.sin(np.radians(fov / 2)) ** 2))
        assert np.isclose(4 * np.pi / (12 * ns ** 2), om_in / (1920 * 1080))
        assert kL <= k <= kH and kH - kL <= 1
