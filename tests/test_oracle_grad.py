"""Pins for the oracle's hand-derived backward (Sec. 3.2, Eqs. backward_lat_scale,
grad_via_J_S): central finite differences in FP64 and torch.autograd through the
independent dense reference."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import synth as S
from tests.dense_ref import params_from_scene, render_dense

KEYS = ("means", "scales", "rotations", "opacities", "sh")


def _scene(deg, seed, P=6):
    sc = S.make_scene(P, deg, seed=seed, r_min=2, r_max=3, logscale_mu=-1.2, logscale_sd=0.3)
    sc = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    sc["opacities"] = np.clip(sc["opacities"], 0.05, 0.85)
    sc["rotations"] = sc["rotations"] * 1.3           # unnormalised quaternions
    return sc


def _view(rng, k=4, kind=0, fov=360.0):
    v = S.make_view(k, kind, fov, R=S.random_rotation(rng), position=(0.1, -0.2, 0.05))
    v["W"] = np.asarray(v["W"], np.float64); v["b"] = np.asarray(v["b"], np.float64)
    return v


@pytest.mark.parametrize("deg", [0, 3])
def test_backward_matches_central_differences(deg):
    rng = np.random.default_rng(1 + deg)
    sc = _scene(deg, 5 + deg)
    v = _view(rng)
    # no termination and no cutoff, so L is smooth in every parameter
    cfg = O.Config(tile_level=2, eps_T=0.0, cutoff=1e9)
    R = O.render(sc, v, cfg)
    pix = R.pix
    dI = rng.standard_normal((pix.size, 3))
    g = O.backward(sc, v, cfg, dI, R.start, R.ids, pix)

    def L(s):
        return (O.render(s, v, cfg, rho=R.rho).image[pix] * dI).sum()

    for key in KEYS:
        flat = sc[key].reshape(-1)
        idx = rng.choice(flat.size, size=min(flat.size, 12), replace=False)
        for j in idx:
            h = 1e-6 * max(1.0, abs(flat[j]))
            s2 = {k: (x.copy() if isinstance(x, np.ndarray) else x) for k, x in sc.items()}
            s2[key].reshape(-1)[j] += h
            lp = L(s2)
            s2[key].reshape(-1)[j] -= 2 * h
            lm = L(s2)
            num = (lp - lm) / (2 * h)
            an = g[key].reshape(-1)[j]
            assert abs(an - num) <= 1e-6 * max(1.0, np.abs(g[key]).max()), (key, j, an, num)


@pytest.mark.parametrize("kind,fov,b", [(O.CAM_FULL, 360.0, 2), (O.CAM_FISHEYE, 190.0, 1),
                                        (O.CAM_PINHOLE, 90.0, 3)])
def test_backward_matches_autograd_of_dense_reference(kind, fov, b):
    rng = np.random.default_rng(20 + b)
    sc = S.make_scene(120, 3, seed=31 + b, r_min=1.5, r_max=4.0, logscale_mu=-1.8)
    sc = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    sc["rotations"] = sc["rotations"] * 0.7
    v = _view(rng, 4, kind, fov)
    cfg = O.Config(tile_level=b)
    R = O.render(sc, v, cfg)
    keep = R.amb[R.pix] == 0
    pix = R.pix[keep]
    dI = rng.standard_normal((pix.size, 3))
    g = O.backward(sc, v, cfg, dI, R.start, R.ids, pix)
    prm = params_from_scene(sc, requires_grad=True)
    C, _ = render_dense(prm, v, cfg, pix, 16)
    (C * torch.as_tensor(dI)).sum().backward()
    for key in KEYS:
        ref = prm[key].grad.numpy().reshape(g[key].shape)
        err = np.abs(ref - g[key]).max()
        assert err <= 1e-9 * max(1.0, np.abs(ref).max()), (key, err)


def test_angular_gradient_of_density_control_by_finite_differences():
    # Sec. 4.2 radian-space density control: the statistic is |(dL/domega, dL/dphi)| of each
    # centre through the pixel offsets, the conic held in the local (east, north) frame (reading).
    # Pinned by central differences of the oracle's own composite over fixed lists, made smooth:
    # no cutoff (literal semantics), no early termination, opacities below the alpha clamp.
    sc = S.make_scene(60, 3, seed=77, r_min=1.5, r_max=3.5, logscale_mu=-1.6)
    sc["opacities"] = np.minimum(sc["opacities"], 0.9).astype(np.float32)
    v = dict(S.make_view(4, S.CAM_FISHEYE, 200.0))
    v["W"] = np.asarray(v["W"], np.float64); v["b"] = np.asarray(v["b"], np.float64)
    cfg = O.Config(tile_level=2, cutoff=math.inf, eps_T=0.0)
    R = O.render(sc, v, cfg)
    rng = np.random.default_rng(3)
    dI = rng.standard_normal((R.pix.size, 3))
    ang = O.backward(sc, v, cfg, dI, R.start, R.ids, R.pix, angular=True)["angular"]

    def loss(pre):
        img, *_ = O.composite(4, 2, pre, sc["opacities"], R.start, R.ids, R.pix, cfg)
        return float((img * dI).sum())

    idx = np.argsort(-np.hypot(ang[:, 0], ang[:, 1]))[:6]
    h = 1e-6
    for i in idx:
        for c, key in enumerate(("omega", "phi")):
            pp = {kk: np.array(vv, copy=True) for kk, vv in R.pre.items()}
            pm = {kk: np.array(vv, copy=True) for kk, vv in R.pre.items()}
            pp[key][i] += h
            pm[key][i] -= h
            fd = (loss(pp) - loss(pm)) / (2 * h)
            assert abs(fd - ang[i, c]) <= 1e-5 * max(1.0, abs(fd)), (i, key, fd, ang[i, c])
