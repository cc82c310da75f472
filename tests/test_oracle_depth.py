"""Pins for the oracle's inverse-depth channel (Sec. 3.2: depth supervision by the
inverse radial depth 1/r, with d(1/r)/dt = -t / r^3).

- one Gaussian seen at its centre pixel: D = alpha / r in closed form;
- the composited D equals the dense FP64 PyTorch reference over all Gaussians;
- the backward with dL/dD (and dL/dI) equals torch.autograd through that reference;
- a loss on D alone against central finite differences of the means.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import synth as S
from tests.dense_ref import params_from_scene, render_dense

KEYS = ["means", "scales", "rotations", "opacities", "sh"]


def _view(rng, k, kind, fov):
    v = S.random_pose_view(rng, k, kind, fov, fov if kind == S.CAM_PINHOLE else None, 0.3)
    return dict(v, W=np.asarray(v["W"], np.float64), b=np.asarray(v["b"], np.float64))


def _scene(seed, P=120):
    sc = S.make_scene(P, 3, seed=seed, r_min=1.5, r_max=4.0, logscale_mu=-1.8)
    return {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}


def test_single_gaussian_depth_closed_form():
    r0, o = 3.0, 0.7
    sc = dict(means=np.array([[0.0, 0.0, r0]]), scales=np.full((1, 3), 0.05), rotations=np.array([[1.0, 0, 0, 0]]),
              opacities=np.array([o]), sh=np.zeros((1, 1, 3)), sh_degree=0)
    view = S.make_view(6)
    view = dict(view, W=np.asarray(view["W"], np.float64), b=np.asarray(view["b"], np.float64))
    cfg = O.Config(tile_level=3)
    R = O.render(sc, view, cfg)
    p = O.vec2pix_nest(64, np.array([[1.0, 0.0, 0.0]]))       # camera +z is HEALPix +X
    img, T, last, amb, D = O.composite(6, 3, R.pre, sc["opacities"], R.start, R.ids, p, cfg, depth=True)
    # the pixel centre is not exactly on the axis: evaluate the closed form at its offset
    th = float(np.arccos(np.clip(O.pix2vec_nest(64, p)[0] @ np.array([1.0, 0, 0]), -1, 1)))
    sig2 = (0.05 / r0) ** 2 + cfg.blur_for(64)
    alpha = min(0.99, o * math.exp(-0.5 * th * th / sig2))
    assert abs(D[0] - alpha / r0) < 1e-12


@pytest.mark.parametrize("kind,fov,b", [(O.CAM_FULL, 360.0, 2), (O.CAM_FISHEYE, 200.0, 3), (O.CAM_PINHOLE, 90.0, 3)])
def test_depth_equals_dense_reference(kind, fov, b):
    rng = np.random.default_rng(40 + b)
    sc = _scene(41 + b)
    v = _view(rng, 4, kind, fov)
    cfg = O.Config(tile_level=b)
    R = O.render(sc, v, cfg)
    img, T, last, amb, D = O.composite(4, b, R.pre, sc["opacities"], R.start, R.ids, R.pix, cfg, depth=True)
    C, Tr, Dr = render_dense(params_from_scene(sc), v, cfg, R.pix, 16, with_depth=True)
    ok = amb == 0
    assert ok.mean() > 0.9
    assert np.abs(D - Dr.numpy())[ok].max() < 1e-12
    assert np.abs(img - C.numpy())[ok].max() < 1e-12


@pytest.mark.parametrize("kind,fov,b", [(O.CAM_FULL, 360.0, 2), (O.CAM_FISHEYE, 190.0, 3), (O.CAM_PINHOLE, 90.0, 3)])
def test_depth_backward_matches_autograd_of_dense_reference(kind, fov, b):
    rng = np.random.default_rng(60 + b)
    sc = _scene(61 + b)
    sc["rotations"] = sc["rotations"] * 0.7
    v = _view(rng, 4, kind, fov)
    cfg = O.Config(tile_level=b)
    R = O.render(sc, v, cfg)
    pix = R.pix[R.amb[R.pix] == 0]
    dI = rng.standard_normal((pix.size, 3))
    dD = rng.standard_normal(pix.size)
    g = O.backward(sc, v, cfg, dI, R.start, R.ids, pix, dLdD=dD)
    prm = params_from_scene(sc, requires_grad=True)
    C, _, Dr = render_dense(prm, v, cfg, pix, 16, with_depth=True)
    ((C * torch.as_tensor(dI)).sum() + (Dr * torch.as_tensor(dD)).sum()).backward()
    for key in KEYS:
        ref = prm[key].grad.numpy().reshape(g[key].shape)
        assert np.abs(ref - g[key]).max() <= 1e-9 * max(1.0, np.abs(ref).max()), key


def test_depth_only_loss_finite_differences():
    rng = np.random.default_rng(77)
    sc = _scene(78, P=40)
    v = _view(rng, 4, O.CAM_FULL, 360.0)
    cfg = O.Config(tile_level=2)
    R = O.render(sc, v, cfg)
    pix = R.pix[R.amb[R.pix] == 0]
    dD = rng.standard_normal(pix.size)
    g = O.backward(sc, v, cfg, np.zeros((pix.size, 3)), R.start, R.ids, pix, dLdD=dD)

    def loss(means):
        s2 = dict(sc, means=means)
        R2 = O.render(s2, v, cfg, rho=R.rho)
        *_, D = O.composite(4, 2, R2.pre, sc["opacities"], R2.start, R2.ids, pix, cfg, depth=True)
        return float((D * dD).sum())

    h = 1e-6
    for i in rng.choice(np.nonzero(np.abs(g["means"]).sum(1) > 0)[0], 6, replace=False):
        for c in range(3):
            mp = sc["means"].copy(); mp[i, c] += h
            mm = sc["means"].copy(); mm[i, c] -= h
            fd = (loss(mp) - loss(mm)) / (2 * h)
            assert abs(fd - g["means"][i, c]) <= 1e-5 * max(1.0, abs(fd)), (i, c, fd, g["means"][i, c])
