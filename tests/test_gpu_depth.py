"""GPU parity of the inverse-depth channel (Sec. 3.2: depth supervision by 1/r)
against the FP64 oracle.

- the depth map, staged (oracle compositing from the GPU's records and lists) and
  end to end, within 2e-4 (ambiguous pixels excluded);
- colour maps, T and last are bit-identical with and without the channel;
- gradients of a loss on colour and depth within 1e-3 relative per tensor;
- views batched with the channel equal the views rendered alone.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import raster as R
from paper_2606_29794_b300 import synth as S
from tests.gpu_util import MAX_EXCLUDED_SHARE, match_oracle, mask_from_words, oracle_cfg, scene_tensors

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

TOL = 2e-4


def _f64view(v):
    return dict(v, W=np.asarray(v["W"], np.float64), b=np.asarray(v["b"], np.float64))


CASES = [("fisheye190_b4", lambda: (S.make_scene(3000, 3, seed=81), S.make_view(7, S.CAM_FISHEYE, 190.0)), 4),
         ("pinhole_b3", lambda: (S.make_scene(2500, 3, seed=82),
                                 S.random_pose_view(np.random.default_rng(8), 7, S.CAM_PINHOLE, 90.0, 70.0)), 3),
         ("full_b5", lambda: (S.make_scene(2500, 0, seed=83, logscale_mu=-2.0), S.make_view(7)), 5)]


@pytest.mark.parametrize("name,make,b", CASES, ids=[c[0] for c in CASES])
def test_depth_map_and_gradients(name, make, b):
    sc, view = make()
    k = view["nside_log2"]
    P = sc["means"].shape[0]
    rast = R.Rasterizer(tile_level=b)
    cfg = oracle_cfg(rast)
    ts = scene_tensors(sc)
    out, state = rast.forward_raw(*ts, sc["sh_degree"], [view], depth=True)
    plain, _ = R.Rasterizer(tile_level=b).forward_raw(*ts, sc["sh_degree"], [view])
    torch.cuda.synchronize()
    for key in ("maps", "T", "last"):
        assert torch.equal(out[key], plain[key]), key
    D = out["depth"].cpu().numpy()
    m_gpu = mask_from_words(out["mask"].cpu().numpy().view(np.uint32), O.npix(2 ** k))
    pix = np.nonzero(m_gpu)[0].astype(np.int64)
    assert np.all(D[m_gpu == 0] == 0)
    # staged: the oracle composites the GPU's FP32 records over the GPU's lists
    wv = R.workspace_view(rast, state)
    rec = R.device_array(wv.records, P * 16, torch.float32).view(P, 16).cpu().numpy().astype(np.float64)
    depth = R.device_array(wv.depth, P, torch.float32).cpu().numpy().astype(np.float64)
    radii = R.device_array(wv.radii, P, torch.float32).cpu().numpy()
    valid = radii > 0
    dbits = depth.astype(np.float32).view(np.uint32).copy()
    dbits[~valid] = 0xFFFFFFFF
    act = O.active_tiles(k, b, m_gpu)
    st, ids = O.tile_lists(k, b, rec[:, 0:3], radii.astype(np.float64), valid.astype(np.int32), dbits,
                           O.tile_rho(k, b), act)
    pre_g = dict(omega=np.arctan2(rec[:, 1], rec[:, 0]), phi=np.arctan2(rec[:, 2], np.hypot(rec[:, 0], rec[:, 1])),
                 conic=rec[:, [7, 11, 15]], col=rec[:, 12:15], r=depth)
    mg, Tg = out["maps"].cpu().numpy()[pix], out["T"].cpu().numpy()[pix]
    _, n_ex, _, _ = match_oracle(k, b, pre_g, rec[:, 3], st, ids, pix, cfg, mg, Tg, gpu_D=D[pix], tol=TOL)
    assert n_ex <= MAX_EXCLUDED_SHARE * pix.size
    # end to end from scratch
    full = O.render(sc, _f64view(view), cfg)
    m_ref, _ = O.mask(2 ** k, view["cam"], view["fov_x"], view["fov_y"])
    sel = m_ref[pix] == 1
    _, n_ex, _, amb2 = match_oracle(k, b, full.pre, sc["opacities"], full.start, full.ids, pix[sel], cfg, mg[sel],
                                    Tg[sel], gpu_D=D[pix][sel], tol=TOL)
    assert n_ex <= MAX_EXCLUDED_SHARE * sel.sum()
    okf = np.zeros(pix.size, bool)
    okf[np.nonzero(sel)[0][amb2 == 0]] = True
    # gradients of sum dI . maps + sum dD . depth
    rng = np.random.default_rng(b)
    keep = okf
    dI = rng.standard_normal((pix.size, 3)) * keep[:, None]
    dD = rng.standard_normal(pix.size) * keep
    ps = [t.clone().requires_grad_(True) for t in ts]
    maps, dep, *_ = R.render(*ps, [view], rasterizer=R.Rasterizer(tile_level=b), sh_degree=sc["sh_degree"],
                             with_depth=True)
    gI = np.zeros((O.npix(2 ** k), 3), np.float32); gI[pix] = dI
    gD = np.zeros(O.npix(2 ** k), np.float32); gD[pix] = dD
    ((maps * torch.as_tensor(gI, device="cuda")).sum() + (dep * torch.as_tensor(gD, device="cuda")).sum()).backward()
    ref = O.backward(sc, _f64view(view), cfg, dI, full.start, full.ids, pix, dLdD=dD)
    for t, name_ in zip(ps, ["means", "scales", "rotations", "opacities", "sh"]):
        g = t.grad.cpu().numpy().astype(np.float64).reshape(ref[name_].shape)
        r = ref[name_]
        assert np.linalg.norm(g - r) <= 1e-3 * np.linalg.norm(r), name_
        assert np.abs(g - r).max() <= 1e-3 * np.abs(r).max() + 1e-12, name_


def test_batched_views_with_depth_equal_single():
    sc = S.make_scene(3000, 3, seed=84)
    rng = np.random.default_rng(9)
    views = [S.random_pose_view(rng, 7, S.CAM_PINHOLE, 90.0, 90.0, 0.5), S.make_view(6, S.CAM_FISHEYE, 200.0)]
    ts = scene_tensors(sc)
    outb, _ = R.Rasterizer().forward_raw(*ts, 3, views, depth=True)
    lay = outb["layout"]
    for v, base in zip(views, lay.pix_base):
        outs, _ = R.Rasterizer().forward_raw(*ts, 3, [v], depth=True)
        n = R.npix(v["nside_log2"])
        assert torch.equal(outb["depth"][base:base + n], outs["depth"])
