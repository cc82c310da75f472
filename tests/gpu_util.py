"""Helpers shared by the GPU parity tests (CUDA path vs the FP64 oracle)."""
import numpy as np
import torch

import oracle as O
from paper_2606_29794_b300 import raster as R
from paper_2606_29794_b300 import synth as S

DEV = "cuda"


def scene_tensors(sc):
    P = sc["means"].shape[0]
    K = (sc["sh_degree"] + 1) ** 2
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=DEV)
    return (t(sc["means"]), t(sc["scales"]), t(sc["rotations"]), t(sc["opacities"]),
            t(np.asarray(sc["sh"]).reshape(P, K, 3)))


def oracle_cfg(rast: R.Rasterizer) -> O.Config:
    c = rast.cfg
    return O.Config(tile_level=c.tile_level, eps_T=float(c.eps_T), alpha_max=float(c.alpha_max),
                    cutoff=float(c.cutoff_m), blur=None if c.blur_rad2 < 0 else float(c.blur_rad2),
                    near=float(c.near_plane), bg=tuple(float(x) for x in c.bg), lam=float(c.lambda_ssim))


def gpu_render(sc, views, rast, grad=False):
    ts = scene_tensors(sc)
    out, state = rast.forward_raw(*ts, sc["sh_degree"], views)
    torch.cuda.synchronize()
    return ts, out, state


def mask_from_words(words_np, n):
    w = words_np.astype(np.uint32)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1).astype(np.uint8)
    return bits.reshape(-1)[:n]


def c1_scene():
    return S.make_scene(2000, 0, seed=20261204)


def c1_view():
    return S.make_view(6)


def match_oracle(k, b, pre, opac, start, ids, pix, cfg, gpu_img, gpu_T, gpu_last=None, gpu_D=None, tol=2e-4):
    """GPU maps (and T, the last index, the depth channel where given) at NESTED pixels `pix`
    against the oracle's compositing (Algorithm 1) of the same lists.

    A pixel matches when it equals, within `tol` (the last index exactly), the oracle's FP64
    result or, where a cutoff or termination decision lies within its FP32 band, one of the
    results the other outcomes of those decisions give (O.composite_variants): both are results
    of the method at the GPU's precision. Pixels with more band decisions than the variants
    follow (O.AMB_UNRESOLVED) are not compared. Asserts that every other pixel matches and
    returns (pixels compared, pixels excluded, pixels matched by a non-FP64 variant, the
    oracle's AMB_* flags per pixel)."""
    depth = gpu_D is not None
    res = O.composite(k, b, pre, opac, start, ids, pix, cfg, depth=depth)
    img, T, last, amb = res[:4]
    gi, gT = np.asarray(gpu_img, np.float64), np.asarray(gpu_T, np.float64)
    ok = (np.abs(gi - img).max(1) < tol) & (np.abs(gT - T) < tol)
    if gpu_last is not None:
        ok &= np.asarray(gpu_last, np.int64) == last
    if depth:
        ok &= np.abs(np.asarray(gpu_D, np.float64) - res[4]) < tol
    excluded = (amb & O.AMB_UNRESOLVED) != 0
    alt = np.nonzero(~ok & ~excluded & ((amb & (O.AMB_CUTOFF | O.AMB_TERM)) != 0))[0]
    n_alt = 0
    if alt.size:
        V = O.composite_variants(k, b, pre, opac, start, ids, pix[alt], cfg)
        L = V["T"].shape[1]
        live = np.arange(L)[None, :] < V["n"][:, None]
        hit = live & (np.abs(gi[alt][:, None, :] - V["image"]).max(2) < tol) & (np.abs(gT[alt][:, None] - V["T"]) < tol)
        if gpu_last is not None:
            hit &= np.asarray(gpu_last, np.int64)[alt][:, None] == V["last"]
        if depth:
            hit &= np.abs(np.asarray(gpu_D, np.float64)[alt][:, None] - V["D"]) < tol
        good = hit.any(1)
        ok[alt[good]] = True
        n_alt = int(good.sum())
    bad = np.nonzero(~ok & ~excluded)[0]
    assert bad.size == 0, ("pixels matching no oracle outcome", pix[bad[:8]], amb[bad[:8]],
                           np.abs(gi - img).max(1)[bad[:8]], np.abs(gT - T)[bad[:8]])
    return int((~excluded).sum()), int(excluded.sum()), n_alt, amb


# Share of pixels the comparison may exclude (more FP32-undecidable decisions than the
# oracle's variants follow): at most 1e-5 of the pixels compared.
MAX_EXCLUDED_SHARE = 1e-5
