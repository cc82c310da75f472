"""Pins for the oracle's HEALPix-SSIM and training loss (Sec. 4.1; Eq. supp_hssim_eval)."""
import numpy as np
import pytest
import torch

import oracle as O

C1, C2 = 1e-4, 9e-4


def test_identical_maps():
    nside = 8
    rng = np.random.default_rng(0)
    I = rng.random((O.npix(nside), 3))
    m, _ = O.mask(nside, O.CAM_FISHEYE, 190.0)
    loss, h, l1, _ = O.hssim_loss(nside, I, I, m, 0.2)
    assert abs(h - 1.0) < 1e-14 and l1 == 0.0 and abs(loss) < 1e-14


def test_constant_maps_closed_form():
    # constant maps: sigma terms vanish, SSIM = (2ab + C1) / (a^2 + b^2 + C1) per channel
    nside = 4
    a = np.array([0.2, 0.5, 0.9]); b = np.array([0.3, 0.1, 0.9])
    I = np.tile(a, (O.npix(nside), 1)); G = np.tile(b, (O.npix(nside), 1))
    m = np.ones(O.npix(nside), np.uint8)
    lam = 0.2
    loss, h, l1, _ = O.hssim_loss(nside, I, G, m, lam)
    ref = np.mean((2 * a * b + C1) / (a * a + b * b + C1))
    assert abs(h - ref) < 1e-14
    assert abs(l1 - np.abs(a - b).mean()) < 1e-14
    assert abs(loss - ((1 - lam) * l1 + lam * (1 - h))) < 1e-14


def test_loss_gradient_fd():
    nside = 4
    rng = np.random.default_rng(1)
    n = O.npix(nside)
    I = rng.random((n, 3)); G = rng.random((n, 3))
    m, _ = O.mask(nside, O.CAM_FISHEYE, 190.0)
    _, _, _, dI = O.hssim_loss(nside, I, G, m, 0.2)
    assert np.all(dI[m == 0] == 0)
    for _ in range(40):
        p = int(rng.choice(np.nonzero(m)[0])); c = int(rng.integers(3))
        h = 1e-6
        Ip = I.copy(); Ip[p, c] += h
        Im = I.copy(); Im[p, c] -= h
        num = (O.hssim_loss(nside, Ip, G, m, 0.2, grad=False)[0] - O.hssim_loss(nside, Im, G, m, 0.2, grad=False)[0]) / (2 * h)
        assert abs(num - dI[p, c]) < 1e-8


def test_loss_matches_torch_window_formula():
    # Direct SSIM over explicit windows (q and its in-mask neighbours, Gaussian weights
    # of the centre-to-centre angle, sigma = 1.5 sqrt(Omega_pix)), gradient by autograd.
    nside = 8
    rng = np.random.default_rng(2)
    n = O.npix(nside)
    I = rng.random((n, 3)); G = rng.random((n, 3))
    m, _ = O.mask(nside, O.CAM_PINHOLE, 100.0, 80.0)
    lam = 0.3
    loss, h, l1, dI = O.hssim_loss(nside, I, G, m, lam)
    nb, _ = O.neighbours_nest(nside, np.arange(n))
    c = O.pix2vec_nest(nside, np.arange(n))
    sig2 = 2.25 * 4 * np.pi / n
    It = torch.tensor(I, requires_grad=True); Gt = torch.tensor(G)
    hs = []
    qs = np.nonzero(m)[0]
    for q in qs:
        idx = [q] + [int(j) for j in nb[q] if j >= 0 and m[j]]
        ang = np.arccos(np.clip(c[idx] @ c[q], -1, 1))
        w = np.exp(-ang ** 2 / (2 * sig2)); w = torch.tensor(w / w.sum())
        x = It[idx]; y = Gt[idx]
        mx = (w[:, None] * x).sum(0); my = (w[:, None] * y).sum(0)
        vx = (w[:, None] * x * x).sum(0) - mx * mx; vy = (w[:, None] * y * y).sum(0) - my * my
        cxy = (w[:, None] * x * y).sum(0) - mx * my
        s = ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
        hs.append(s.mean())
    H = torch.stack(hs).mean()
    L1 = (It[qs] - Gt[qs]).abs().mean()
    Lt = (1 - lam) * L1 + lam * (1 - H)
    Lt.backward()
    assert abs(Lt.item() - loss) < 1e-13 and abs(H.item() - h) < 1e-13
    assert np.abs(It.grad.numpy() - dI).max() < 1e-13
