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
