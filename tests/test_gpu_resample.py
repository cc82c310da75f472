"""GPU parity of sphere <-> image resampling (Eq. camera_synthesis;
Eqs. supp_image_to_healpix, supp_hssim_mask) against the FP64 oracle.

Tolerances follow from FP32 positions. A direction in FP32 is fixed to about
1e-7 rad, and neighbouring HEALPix pixels are about 1/Nside apart, so an
interpolation weight can move by about 1e-7 Nside; on maps whose neighbours
differ by up to 1 (the random maps here) the value can move by as much. Hence
1e-6 + 6e-7 Nside for sphere -> image and its adjoint; likewise an FP32 image
coordinate is fixed to about 1e-7 max(W, H) pixels, hence 1e-6 + 2e-7 max(W, H)
for image -> sphere.

- sphere -> image: values within that bound, validity equal except where the
  oracle's point sits within 1e-5 of the fisheye ellipse;
- its adjoint: equal to the oracle's A^T within the bound times the largest
  entry, and <A x, y> = <x, A^T y> on the GPU's own results;
- image -> sphere: values within the bound inside the mask, the mask equal to
  the FoV mask of hpxgs_mask_build bit for bit;
- the sizes the benchmark times (fisheye 190 deg 1472^2 at Nside 512, pinhole
  90 deg 2048^2 and a 4096 x 2048 panorama at Nside 1024) on seeded samples.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import _lib as L
from paper_2606_29794_b300 import resample as RS
from tests.gpu_util import mask_from_words

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

def tol_s2i(k):
    return 1e-6 + 6e-7 * 2 ** k


def tol_i2s(W, H):
    return 1e-6 + 2e-7 * max(W, H)
Z = (0.0, 0.0)
CAMS = [(O.CAM_PINHOLE, 90.0, 70.0, Z), (O.CAM_PINHOLE, 90.0, 70.0, (0.3, -0.45)), (O.CAM_FISHEYE, 190.0, 190.0, Z),
        (O.CAM_FISHEYE, 200.0, 170.0, Z), (O.CAM_FULL, 360.0, 180.0, Z)]


def _cam(kind, fx, fy, pp=Z):
    return {"cam": kind, "fov_x": fx, "fov_y": fy, "pp": pp}


def _fisheye_edge(kind, W, H, uv):
    """Image points within 1e-5 (relative) of the fisheye ellipse, where FP32 may decide validity otherwise."""
    if kind != O.CAM_FISHEYE:
        return np.zeros(len(uv), bool)
    mx = (uv[:, 0] - W / 2) / (W / math.pi)
    my = (uv[:, 1] - H / 2) / (H / math.pi)
    return np.abs(np.hypot(mx, my) - math.pi / 2) < 1e-5


@pytest.mark.parametrize("kind,fx,fy,pp", CAMS)
def test_sphere_to_image(kind, fx, fy, pp):
    k, W, H = 6, 160, 120
    rng = np.random.default_rng(kind + 10)
    hmap = rng.random((12 * 4 ** k, 3))
    img, ok = RS.sphere_to_image_raw(torch.as_tensor(hmap, dtype=torch.float32, device="cuda"), k,
                                     _cam(kind, fx, fy, pp), W, H)
    ref, ok_ref = O.sphere_to_image(2 ** k, hmap, kind, W, H, fx, fy, pp=pp)
    uu, vv = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    edge = _fisheye_edge(kind, W, H, np.stack([uu.ravel(), vv.ravel()], 1)).reshape(H, W)
    okg = ok.cpu().numpy()
    assert np.array_equal(okg[~edge], ok_ref[~edge])
    both = (okg == 1) & (ok_ref == 1)
    assert both.sum() > 0.3 * W * H
    assert np.abs(img.cpu().numpy()[both] - ref[both]).max() < tol_s2i(k)
    assert np.all(img.cpu().numpy()[okg == 0] == 0)


@pytest.mark.parametrize("kind,fx,fy,pp", CAMS)
def test_sphere_to_image_adjoint(kind, fx, fy, pp):
    k, W, H = 5, 96, 64
    rng = np.random.default_rng(kind + 20)
    y = rng.standard_normal((H, W, 3))
    dmap = RS.sphere_to_image_backward(torch.as_tensor(y, dtype=torch.float32, device="cuda"), k,
                                       _cam(kind, fx, fy, pp), W, H).cpu().numpy().astype(np.float64)
    ref = O.sphere_to_image_adjoint(2 ** k, y, kind, W, H, fx, fy, pp=pp)
    assert np.abs(dmap - ref).max() < tol_s2i(k) * np.abs(ref).max() * 4
    # <A x, y> = <x, A^T y> with the GPU's forward and backward
    x = rng.standard_normal((12 * 4 ** k, 3))
    Ax, ok = RS.sphere_to_image_raw(torch.as_tensor(x, dtype=torch.float32, device="cuda"), k, _cam(kind, fx, fy, pp),
                                    W, H)
    lhs = (Ax.cpu().numpy().astype(np.float64) * y).sum()
    rhs = (x * dmap).sum()
    assert abs(lhs - rhs) < 1e-5 * np.abs(Ax.cpu().numpy() * y).sum()


def test_autograd_through_sphere_to_image():
    k, W, H = 5, 64, 48
    cam = _cam(O.CAM_PINHOLE, 80.0, 60.0)
    hmap = torch.rand((12 * 4 ** k, 3), device="cuda", requires_grad=True)
    img, valid = RS.sphere_to_image(hmap, k, cam, W, H)
    w = torch.rand_like(img)
    (img * w).sum().backward()
    want = RS.sphere_to_image_backward(w.contiguous(), k, cam, W, H)
    assert torch.allclose(hmap.grad, want)


@pytest.mark.parametrize("kind,fx,fy,pp", CAMS)
def test_image_to_sphere(kind, fx, fy, pp):
    k, W, H = 6, 150, 100
    rng = np.random.default_rng(kind + 30)
    img = rng.random((H, W, 3))
    hm, words = RS.image_to_sphere(torch.as_tensor(img, dtype=torch.float32, device="cuda"), _cam(kind, fx, fy, pp), k)
    n = 12 * 4 ** k
    m = mask_from_words(words.cpu().numpy().view(np.uint32), n)
    # the mask is M_C of the FoV mask kernel, bit for bit
    fov = torch.empty(n // 32, dtype=torch.int32, device="cuda")
    v = L.make_views([{"W": np.eye(3, dtype=np.float32), "b": np.zeros(3, np.float32), "nside_log2": k,
                       "cam": kind, "fov_x": fx, "fov_y": fy, "pp": pp}])
    cfg = L.default_config()
    L.check(L.lib().hpxgs_mask_build(v, ctypes.byref(cfg), ctypes.c_void_p(fov.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "mask")
    torch.cuda.synchronize()
    assert np.array_equal(m, mask_from_words(fov.cpu().numpy().view(np.uint32), n))
    ref, m_ref = O.image_to_sphere(2 ** k, img, kind, W, H, fx, fy, pp=pp)
    _, margin = O.mask(2 ** k, kind, fx, fy, pp=pp)
    assert np.all(np.abs(margin[m != m_ref]) < 1e-12)
    both = (m == 1) & (m_ref == 1)
    assert np.abs(hm.cpu().numpy()[both] - ref[both]).max() < tol_i2s(W, H)
    assert np.all(hm.cpu().numpy()[m == 0] == 0)


BENCH_CASES = [(O.CAM_FISHEYE, 190.0, 190.0, Z, 9, 1472, 1472), (O.CAM_PINHOLE, 90.0, 90.0, Z, 10, 2048, 2048),
               (O.CAM_PINHOLE, 90.0, 90.0, (0.25, 0.1), 10, 2048, 1536), (O.CAM_FULL, 360.0, 180.0, Z, 10, 4096, 2048)]


@pytest.mark.parametrize("kind,fx,fy,pp,k,W,H", BENCH_CASES)
def test_bench_sizes_sampled(kind, fx, fy, pp, k, W, H):
    rng = np.random.default_rng(W + k)
    n = 12 * 4 ** k
    hmap = rng.random((n, 3)).astype(np.float32)
    cam = _cam(kind, fx, fy, pp)
    img, ok = RS.sphere_to_image_raw(torch.as_tensor(hmap, device="cuda"), k, cam, W, H)
    sel = rng.choice(W * H, 20000, replace=False)
    uv = np.stack([sel % W + 0.5, sel // W + 0.5], 1)
    ref, ok_ref = O.sphere_to_image_at(2 ** k, hmap.astype(np.float64), kind, W, H, fx, fy, uv, pp=pp)
    okg = ok.cpu().numpy().ravel()[sel]
    edge = _fisheye_edge(kind, W, H, uv)
    assert np.array_equal(okg[~edge], ok_ref[~edge])
    both = (okg == 1) & (ok_ref == 1)
    assert np.abs(img.cpu().numpy().reshape(-1, 3)[sel][both] - ref[both]).max() < tol_s2i(k)
    # image -> sphere at the same sizes
    im = rng.random((H, W, 3)).astype(np.float32)
    hm, words = RS.image_to_sphere(torch.as_tensor(im, device="cuda"), cam, k)
    qs = rng.choice(n, 20000, replace=False)
    ref2, m2 = O.image_to_sphere_at(2 ** k, im.astype(np.float64), kind, W, H, fx, fy, qs, pp=pp)
    m = mask_from_words(words.cpu().numpy().view(np.uint32), n)[qs]
    _, margin = O.mask(2 ** k, kind, fx, fy, pp=pp)
    assert np.all(np.abs(margin[qs][m != m2]) < 1e-12)
    both = (m == 1) & (m2 == 1)
    assert np.abs(hm.cpu().numpy()[qs][both] - ref2[both]).max() < tol_i2s(W, H)


@pytest.mark.parametrize("kind,fx,fy,pp", CAMS)
def test_plans_equal_direct_calls(kind, fx, fy, pp):
    # a resampling plan holds the taps the direct kernels compute; applying it gives their results
    # bit for bit (the adjoint up to the order of its atomic sums), for float and 8-bit images
    k, W, H = 7, 180, 120
    cam = _cam(kind, fx, fy, pp)
    g = torch.Generator(device="cuda").manual_seed(kind + 50)
    hmap = torch.rand((12 * 4 ** k, 3), device="cuda", generator=g)
    ps = RS.Plan(L.PLAN_SPHERE_TO_IMAGE, cam, k, W, H)
    img0, val0 = RS.sphere_to_image_raw(hmap, k, cam, W, H)
    img1, val1 = ps.sphere_to_image(hmap)
    torch.cuda.synchronize()
    assert torch.equal(img0, img1) and torch.equal(val0, val1)
    dimg = torch.rand((H, W, 3), device="cuda", generator=g)
    d0 = RS.sphere_to_image_backward(dimg, k, cam, W, H)
    d1 = ps.sphere_to_image_backward(dimg)
    assert torch.allclose(d0, d1, rtol=1e-5, atol=1e-6)
    pi = RS.Plan(L.PLAN_IMAGE_TO_SPHERE, cam, k, W, H)
    img8 = torch.randint(0, 256, (H, W, 3), dtype=torch.uint8, device="cuda", generator=g)
    for im in (img8.float() / 255.0, img8):
        m0, w0 = RS.image_to_sphere(im, cam, k)
        w1 = torch.empty_like(w0)
        m1, _ = pi.image_to_sphere(im, words=w1)
        torch.cuda.synchronize()
        assert torch.equal(m0, m1) and torch.equal(w0, w1)
    with pytest.raises(ValueError):
        pi.sphere_to_image(hmap)
