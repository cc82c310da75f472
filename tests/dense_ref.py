"""Dense all-Gaussians-per-pixel FP64 reference in PyTorch, used to pin the oracle.

Independent of the oracle's C++: it uses the basis-free tangent-frame form of the
projection (S_phi J = [e_omega; e_phi] / r), the azimuthal-equidistant form of the
spherical offset, Cartesian real SH polynomials, and a global depth sort with an
exclusive cumulative product instead of per-tile lists. Gradients come from
torch.autograd, so this reference also pins the oracle's hand-derived backward.
Only pixel-centre directions (pinned separately) are taken from the oracle.
"""
import math

import numpy as np
import torch

import oracle as O


def sh_cartesian(d, deg):
    """Real SH (Condon-Shortley phase, order m = -l..l) as Cartesian polynomials."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    pi = math.pi
    out = [torch.full_like(x, math.sqrt(1 / (4 * pi)))]
    if deg >= 1:
        c1 = math.sqrt(3 / (4 * pi))
        out += [-c1 * y, c1 * z, -c1 * x]
    if deg >= 2:
        a, b, c = math.sqrt(15 / (4 * pi)), math.sqrt(5 / (16 * pi)), math.sqrt(15 / (16 * pi))
        out += [a * x * y, -a * y * z, b * (2 * z * z - x * x - y * y), -a * x * z, c * (x * x - y * y)]
    if deg >= 3:
        a = math.sqrt(35 / (32 * pi)); b = math.sqrt(105 / (4 * pi)); c = math.sqrt(21 / (32 * pi))
        e = math.sqrt(7 / (16 * pi)); f = math.sqrt(105 / (16 * pi))
        out += [-a * y * (3 * x * x - y * y), b * x * y * z, -c * y * (4 * z * z - x * x - y * y),
                e * z * (2 * z * z - 3 * x * x - 3 * y * y), -c * x * (4 * z * z - x * x - y * y),
                f * z * (x * x - y * y), -a * x * (x * x - 3 * y * y)]
    return torch.stack(out, -1)


def quat_rot(q):
    q = q / q.norm(dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def render_dense(params, view, cfg, pix, nside, with_depth=False, members=None):
    """params: dict of float64 tensors (means, scales, rotations, opacities, sh (P,K,3)).

    Returns (colours at pix (n, 3), final transmittance (n,)) and, with with_depth, the
    composited inverse radial depth (n,) (Sec. 3.2: depth supervision by 1/r).
    members (optional, (n, P) bool): Gaussian i may contribute to pixel n only where set
    (the tile lists of the literal semantics, where the cutoff no longer decides)."""
    W = torch.as_tensor(np.asarray(view["W"], np.float64))
    b = torch.as_tensor(np.asarray(view["b"], np.float64))
    mu, s, q, o, sh = (params[k] for k in ("means", "scales", "rotations", "opacities", "sh"))
    deg = int(round(math.sqrt(sh.shape[1]))) - 1
    t = mu @ W.T + b
    r = t.norm(dim=-1)
    valid = r > cfg.near
    tx, ty, tz = t.unbind(-1)
    rho = torch.sqrt(tx * tx + tz * tz)
    e_w = torch.stack([tz, torch.zeros_like(tz), -tx], -1) / rho[:, None]
    e_p = torch.stack([-tx * ty, rho * rho, -tz * ty], -1) / (rho * r)[:, None]
    A = torch.stack([e_w, e_p], -2) / r[:, None, None]            # = S_phi J
    R = quat_rot(q)
    M = R * s[:, None, :]
    S3 = M @ M.transpose(-1, -2)
    Sc = W @ S3 @ W.T
    Sarc = A @ Sc @ A.transpose(-1, -2) + cfg.blur_for(nside) * torch.eye(2, dtype=torch.float64)
    det = Sarc[:, 0, 0] * Sarc[:, 1, 1] - Sarc[:, 0, 1] ** 2
    valid = valid & (det > 0)
    Q = torch.linalg.inv(Sarc)
    cam = -(W.T @ b)
    dv = mu - cam
    dirn = dv / dv.norm(dim=-1, keepdim=True)
    Y = sh_cartesian(dirn, deg)
    col = torch.clamp((Y[:, :, None] * sh).sum(1) + 0.5, min=0.0)
    g = t / r[:, None]
    # pixel directions in the camera frame (HEALPix (X, Y, Z) = camera (z, x, y))
    v = torch.as_tensor(O.pix2vec_nest(nside, pix))
    pd = torch.stack([v[:, 1], v[:, 2], v[:, 0]], -1)
    u1 = pd @ e_w.T; u2 = pd @ e_p.T; c = pd @ g.T                 # (n, P)
    sn = torch.sqrt(u1 * u1 + u2 * u2)
    th = torch.atan2(sn, c)
    fac = torch.where(sn > 0, th / torch.where(sn > 0, sn, torch.ones_like(sn)), torch.ones_like(sn))
    dx, dy = fac * u1, fac * u2
    m = Q[None, :, 0, 0] * dx * dx + 2 * Q[None, :, 0, 1] * dx * dy + Q[None, :, 1, 1] * dy * dy
    a = torch.clamp(o[None, :] * torch.exp(-0.5 * m), max=cfg.alpha_max)
    keep = (m <= cfg.cutoff) & valid[None, :]
    if members is not None:
        keep = keep & torch.as_tensor(members)
    a = torch.where(keep, a, torch.zeros_like(a))
    # global order by (float32 depth bits, index)
    key = O.depth_bits(r.detach().numpy()).astype(np.int64)
    key[~valid.numpy()] = np.iinfo(np.int64).max
    order = torch.as_tensor(np.argsort(key, kind="stable"))
    a = a[:, order]; colo = col[order]; invr = (1.0 / r)[order]
    one_minus = 1 - a
    T_ex = torch.cumprod(torch.cat([torch.ones_like(a[:, :1]), one_minus[:, :-1]], 1), 1)
    incl = (T_ex >= cfg.eps_T).to(a.dtype).detach()
    w = T_ex * a * incl
    C = w @ colo
    T_fin = torch.prod(torch.where(incl > 0, one_minus, torch.ones_like(one_minus)), 1)
    C = C + T_fin[:, None] * torch.as_tensor(np.asarray(cfg.bg, np.float64))[None, :]
    if with_depth:
        return C, T_fin, w @ torch.where(valid[order], invr, torch.zeros_like(invr))
    return C, T_fin


def params_from_scene(scene, requires_grad=False):
    P = scene["means"].shape[0]
    K = (scene["sh_degree"] + 1) ** 2
    out = {}
    for k in ("means", "scales", "rotations", "opacities"):
        out[k] = torch.tensor(np.asarray(scene[k], np.float64), requires_grad=requires_grad)
    out["sh"] = torch.tensor(np.asarray(scene["sh"], np.float64).reshape(P, K, 3), requires_grad=requires_grad)
    return out
