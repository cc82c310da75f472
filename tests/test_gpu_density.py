"""GPU parity of the radian-space density-control statistics (Sec. 4.2) against the FP64 oracle.

After a forward and backward over two views (a 190-degree fisheye and an
asymmetric-FoV pinhole), hpxgs_density_stats updates per Gaussian:
r_s,max <- max(r_s,max, r_s), grad_accum += |(dL/domega, dL/dphi)|, count += 1 over
the (view, Gaussian) pairs in which the Gaussian is listed for an active tile.

- visibility: the Gaussians listed by the oracle's tile query run on the GPU's own
  FP32 records, bit for bit;
- dL/domega, dL/dphi per (view, Gaussian) against the oracle's angular gradient
  (its pin: central finite differences of the oracle's loss in omega and phi,
  tests/test_oracle_grad.py), within 1e-3 relative (norm and max);
- r_s,max against the oracle's FP64 r_s within 1e-5 relative; the counts exactly;
  grad_accum against the oracle's update within 1e-3 relative.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import raster as R
from paper_2606_29794_b300 import synth as S
from tests.gpu_util import mask_from_words, oracle_cfg, scene_tensors

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]


def _f64view(v):
    return dict(v, W=np.asarray(v["W"], np.float64), b=np.asarray(v["b"], np.float64))


def _setup(seed=81, b=4):
    sc = S.make_scene(3000, 3, seed=seed)
    views = [S.make_view(7, S.CAM_FISHEYE, 190.0),
             S.random_pose_view(np.random.default_rng(seed + 1), 7, S.CAM_PINHOLE, 100.0, 70.0, 0.3)]
    rast = R.Rasterizer(tile_level=b)
    return sc, views, rast


def test_density_statistics_match_oracle():
    sc, views, rast = _setup()
    cfg = oracle_cfg(rast)
    P = sc["means"].shape[0]
    ts = scene_tensors(sc)
    out, state = rast.forward_raw(*ts, sc["sh_degree"], views)
    torch.cuda.synchronize()
    lay = R.view_layout(views)
    mask_all = mask_from_words(out["mask"].cpu().numpy().view(np.uint32), lay.total_pix)
    rng = np.random.default_rng(7)
    dm = np.zeros((lay.total_pix, 3), np.float32)
    per_view = []
    for v, base in zip(views, lay.pix_base):
        k = v["nside_log2"]
        n = O.npix(2 ** k)
        pix = np.nonzero(mask_all[base:base + n])[0].astype(np.int64)
        full = O.render(sc, _f64view(v), cfg)
        ok = full.amb[pix] == 0                  # pixels with a decision FP32 cannot settle carry no loss
        assert ok.mean() > 0.99
        dI = rng.standard_normal((pix.size, 3)) * ok[:, None]
        dm[base + pix] = dI
        per_view.append((v, pix, full, dI))
    rast.backward_raw(state, torch.as_tensor(dm, device="cuda"))
    rs_max = torch.zeros(P, dtype=torch.float32, device="cuda")
    acc = torch.zeros(P, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(P, dtype=torch.int32, device="cuda")
    ang = torch.full((len(views), P, 2), float("nan"), dtype=torch.float32, device="cuda")
    rast.density_stats(state, rs_max, acc, cnt, ang)
    torch.cuda.synchronize()
    wv = R.workspace_view(rast, state)
    PV = len(views) * P
    rec = R.device_array(wv.records, PV * 16, torch.float32).view(len(views), P, 16).cpu().numpy().astype(np.float64)
    depth = R.device_array(wv.depth, PV, torch.float32).view(len(views), P).cpu().numpy()
    radii = R.device_array(wv.radii, PV, torch.float32).view(len(views), P).cpu().numpy()
    ang = ang.cpu().numpy().astype(np.float64)
    e_rs = np.zeros(P)
    e_acc = np.zeros(P)
    e_cnt = np.zeros(P, np.int64)
    for vi, (v, pix, full, dI) in enumerate(per_view):
        k = v["nside_log2"]
        b = rast.cfg.tile_level
        n = O.npix(2 ** k)
        # visibility: the oracle's tile query over the GPU's records of this view
        valid = radii[vi] > 0
        dbits = depth[vi].astype(np.float32).view(np.uint32).copy()
        dbits[~valid] = 0xFFFFFFFF
        m_v = mask_all[lay.pix_base[vi]:lay.pix_base[vi] + n]
        _, ids = O.tile_lists(k, b, rec[vi][:, 0:3], radii[vi].astype(np.float64), valid.astype(np.int32), dbits,
                              O.tile_rho(k, b), O.active_tiles(k, b, m_v))
        vis = np.zeros(P, bool)
        vis[np.asarray(ids, np.int64)] = True
        assert np.all(ang[vi][~vis] == 0), vi                   # angular is 0 off the visible set
        ref = O.backward(sc, _f64view(v), cfg, dI, full.start, full.ids, pix, angular=True)["angular"]
        g = ang[vi]
        assert np.linalg.norm(g - ref) <= 1e-3 * np.linalg.norm(ref), vi
        assert np.abs(g - ref).max() <= 1e-3 * np.abs(ref).max(), vi
        # the oracle's own listing (FP64 records) agrees with the GPU's records' listing
        vis_o = np.zeros(P, bool)
        vis_o[np.asarray(full.ids, np.int64)] = True
        assert (vis_o != vis).sum() <= max(2, P // 1000), vi
        O.density_stats_update(e_rs, e_acc, e_cnt, full.pre["rs"], ref, vis)
    assert np.array_equal(cnt.cpu().numpy().astype(np.int64), e_cnt)
    assert np.allclose(rs_max.cpu().numpy(), e_rs, rtol=1e-5, atol=0)
    a = acc.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(a - e_acc) <= 1e-3 * np.linalg.norm(e_acc)
    assert np.abs(a - e_acc).max() <= 1e-3 * np.abs(e_acc).max()


def test_density_statistics_accumulate_over_steps():
    # two calls add: counts double, grad_accum doubles, r_s,max unchanged; angular is
    # optional and the statistics do not depend on it
    sc, views, rast = _setup(seed=83)
    P = sc["means"].shape[0]
    out, state = rast.forward_raw(*scene_tensors(sc), sc["sh_degree"], views)
    gen = torch.Generator(device="cuda").manual_seed(3)
    rast.backward_raw(state, torch.randn(out["maps"].shape, device="cuda", generator=gen))
    bufs = [torch.zeros(P, dtype=torch.float32, device="cuda"), torch.zeros(P, dtype=torch.float32, device="cuda"),
            torch.zeros(P, dtype=torch.int32, device="cuda")]
    rast.density_stats(state, *bufs)
    once = [t.clone() for t in bufs]
    rast.density_stats(state, *bufs, angular=torch.zeros((len(views), P, 2), device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(bufs[0], once[0])
    assert torch.equal(bufs[2], 2 * once[2])
    assert torch.allclose(bufs[1], 2 * once[1], rtol=1e-6, atol=0)
    assert int(once[2].max()) <= len(views) and int((once[2] > 0).sum()) > P // 4
