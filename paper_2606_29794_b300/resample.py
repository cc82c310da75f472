"""Sphere <-> image resampling through the C ABI (Eq. camera_synthesis;
Eqs. supp_image_to_healpix, supp_hssim_mask): the rendered HEALPix map to a
camera image, its adjoint, and a camera image to the HEALPix grid. Argument
marshalling only; the work runs in libhpxgs kernels.

A camera is a dict with "cam" (CAM_FULL for the panorama, CAM_PINHOLE,
CAM_FISHEYE) and "fov_x", "fov_y" in degrees, and for the pinhole optionally "pp",
the principal point's offset from the image centre in half-image units (the views of
`synth` carry them).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L


def _cam(cam) -> L.Camera:
    c = L.Camera()
    c.kind = int(cam["cam"])
    c.fov_x_deg = float(cam.get("fov_x", 360.0))
    fy = cam.get("fov_y")
    c.fov_y_deg = float(c.fov_x_deg if fy is None else fy)
    c.ppx, c.ppy = (float(x) for x in cam.get("pp", (0.0, 0.0)))
    return c


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _f32(t):
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return t


def sphere_to_image_raw(hmap, nside_log2, cam, width, height, with_valid=True):
    """Image [height, width, 3] = Interp_H(hmap, P_C(u, v)) and validity [height, width] (uint8)."""
    hmap = _f32(hmap)
    if hmap.numel() != 3 * 12 * 4 ** nside_log2:
        raise ValueError("map size does not match nside_log2")
    img = torch.empty((height, width, 3), dtype=torch.float32, device=hmap.device)
    valid = torch.empty((height, width), dtype=torch.uint8, device=hmap.device) if with_valid else None
    c = _cam(cam)
    L.check(L.lib().hpxgs_sphere_to_image(_ptr(hmap), nside_log2, ctypes.byref(c), width, height, _ptr(img),
                                          _ptr(valid), _stream(hmap.device)), "sphere_to_image")
    return img, valid


def sphere_to_image_backward(dimage, nside_log2, cam, width, height):
    """dL/dmap [12 * 4^k, 3] = A^T dL/dimage."""
    dimage = _f32(dimage)
    if dimage.numel() != 3 * width * height:
        raise ValueError("dimage size does not match width x height x 3")
    dmap = torch.empty((12 * 4 ** nside_log2, 3), dtype=torch.float32, device=dimage.device)
    c = _cam(cam)
    L.check(L.lib().hpxgs_sphere_to_image_backward(_ptr(dimage), nside_log2, ctypes.byref(c), width, height,
                                                   _ptr(dmap), _stream(dimage.device)), "sphere_to_image_backward")
    return dmap


def image_to_sphere_into(image, cam, nside_log2, hmap, words=None, stream=None):
    """Writes the HEALPix map of a camera image [height, width, 3] (float32 values, or uint8 codes
    v read as v / 255) into `hmap` [12 * 4^k, 3] and, if given, the mask words of M_C into `words`,
    on `stream` (default: the current stream)."""
    if image.dim() != 3 or image.shape[2] != 3 or not image.is_cuda or not image.is_contiguous():
        raise ValueError("expected a contiguous CUDA image of shape [height, width, 3]")
    if image.dtype == torch.uint8:
        fn = L.lib().hpxgs_image_to_sphere_u8
    elif image.dtype == torch.float32:
        fn = L.lib().hpxgs_image_to_sphere
    else:
        raise ValueError("expected a float32 or uint8 image")
    npix = 12 * 4 ** nside_log2
    _f32(hmap)
    if hmap.numel() != 3 * npix or (words is not None and (words.numel() != npix // 32 or not words.is_contiguous())):
        raise ValueError("map or mask size does not match nside_log2")
    height, width = image.shape[0], image.shape[1]
    c = _cam(cam)
    s = ctypes.c_void_p((stream or torch.cuda.current_stream(image.device)).cuda_stream)
    L.check(fn(_ptr(image), width, height, ctypes.byref(c), nside_log2, _ptr(hmap), _ptr(words), s), "image_to_sphere")


def image_to_sphere(image, cam, nside_log2, with_mask=True):
    """HEALPix map [12 * 4^k, 3] of a camera image [height, width, 3] (float32, or uint8 codes read
    as v / 255) and the mask words of M_C."""
    npix = 12 * 4 ** nside_log2
    hmap = torch.empty((npix, 3), dtype=torch.float32, device=image.device)
    words = torch.empty(npix // 32, dtype=torch.int32, device=image.device) if with_mask else None
    image_to_sphere_into(image, cam, nside_log2, hmap, words)
    return hmap, words


class Plan:
    """A resampling plan (hpxgs_resample_plan_build): the taps of every output pixel for one
    camera, image size and HEALPix order, built once on the device. `direction` is
    L.PLAN_SPHERE_TO_IMAGE (serves sphere_to_image and its adjoint) or L.PLAN_IMAGE_TO_SPHERE
    (serves image_to_sphere); the planned calls give the direct calls' results bit for bit."""

    def __init__(self, direction, cam, nside_log2, width, height, device="cuda"):
        self.direction, self.k, self.W, self.H = int(direction), int(nside_log2), int(width), int(height)
        nb = ctypes.c_size_t()
        L.check(L.lib().hpxgs_resample_plan_size(self.direction, self.k, self.W, self.H, ctypes.byref(nb)),
                "plan size")
        self.nbytes = nb.value
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        c = _cam(cam)
        L.check(L.lib().hpxgs_resample_plan_build(self.direction, self.k, ctypes.byref(c), self.W, self.H,
                                                  _ptr(self.buf), self.nbytes, _stream(self.buf.device)),
                "plan build")

    def _need(self, direction):
        if self.direction != direction:
            raise ValueError("plan built for the other direction")

    def sphere_to_image(self, hmap, image=None, valid=None):
        """Image [H, W, 3] and validity [H, W] of a map through the plan."""
        self._need(L.PLAN_SPHERE_TO_IMAGE)
        hmap = _f32(hmap)
        if hmap.numel() != 3 * 12 * 4 ** self.k:
            raise ValueError("map size does not match the plan's order")
        image = torch.empty((self.H, self.W, 3), dtype=torch.float32, device=hmap.device) if image is None else image
        valid = torch.empty((self.H, self.W), dtype=torch.uint8, device=hmap.device) if valid is None else valid
        L.check(L.lib().hpxgs_sphere_to_image_planned(_ptr(hmap), self.k, self.W, self.H, _ptr(self.buf), self.nbytes,
                                                      _ptr(image), _ptr(valid), _stream(hmap.device)),
                "sphere_to_image_planned")
        return image, valid

    def sphere_to_image_backward(self, dimage):
        self._need(L.PLAN_SPHERE_TO_IMAGE)
        dimage = _f32(dimage)
        if dimage.numel() != 3 * self.W * self.H:
            raise ValueError("dimage size does not match the plan's image")
        dmap = torch.empty((12 * 4 ** self.k, 3), dtype=torch.float32, device=dimage.device)
        L.check(L.lib().hpxgs_sphere_to_image_backward_planned(_ptr(dimage), self.k, self.W, self.H, _ptr(self.buf),
                                                               self.nbytes, _ptr(dmap), _stream(dimage.device)),
                "sphere_to_image_backward_planned")
        return dmap

    def image_to_sphere(self, image, hmap=None, words=None, stream=None):
        """HEALPix map [12 * 4^k, 3] and mask words of an image [H, W, 3] (float32, or uint8 codes
        read as v / 255) through the plan."""
        self._need(L.PLAN_IMAGE_TO_SPHERE)
        if tuple(image.shape) != (self.H, self.W, 3) or not image.is_cuda or not image.is_contiguous():
            raise ValueError("expected a contiguous CUDA image of the plan's size")
        fn = {torch.uint8: L.lib().hpxgs_image_to_sphere_u8_planned,
              torch.float32: L.lib().hpxgs_image_to_sphere_planned}.get(image.dtype)
        if fn is None:
            raise ValueError("expected a float32 or uint8 image")
        npix = 12 * 4 ** self.k
        hmap = torch.empty((npix, 3), dtype=torch.float32, device=image.device) if hmap is None else _f32(hmap)
        if hmap.numel() != 3 * npix:
            raise ValueError("map size does not match the plan's order")
        s = ctypes.c_void_p((stream or torch.cuda.current_stream(image.device)).cuda_stream)
        L.check(fn(_ptr(image), self.W, self.H, self.k, _ptr(self.buf), self.nbytes, _ptr(hmap), _ptr(words), s),
                "image_to_sphere_planned")
        return hmap, words


class _SphereToImage(torch.autograd.Function):
    @staticmethod
    def forward(ctx, hmap, nside_log2, cam, width, height):
        img, valid = sphere_to_image_raw(hmap.contiguous(), nside_log2, cam, width, height)
        ctx.args = (nside_log2, cam, width, height)
        ctx.mark_non_differentiable(valid)
        return img, valid

    @staticmethod
    def backward(ctx, dimg, dvalid):
        return sphere_to_image_backward(dimg.contiguous(), *ctx.args), None, None, None, None


def sphere_to_image(hmap, nside_log2, cam, width, height):
    """Differentiable in `hmap`: returns (image, valid)."""
    return _SphereToImage.apply(hmap, nside_log2, cam, width, height)
