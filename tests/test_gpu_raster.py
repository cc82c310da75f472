"""GPU parity of the rasterizer (forward Algorithm 1, backward Sec. 3.2) against the FP64 oracle.

Staged checks feed the oracle the GPU's stored FP32 per-Gaussian values so that
tile lists and sort order can be compared exactly; end-to-end checks compare
maps within 2e-4 per channel against the oracle from scratch, where a cutoff or
termination decision that FP32 cannot settle may take either outcome
(tests.gpu_util.match_oracle; at most 1e-5 of the pixels excluded), and
gradients within 1e-3 relative.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import raster as R
from paper_2606_29794_b300 import synth as S
from tests.gpu_util import (MAX_EXCLUDED_SHARE, c1_scene, c1_view, gpu_render, mask_from_words, match_oracle,
                            oracle_cfg, scene_tensors)

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

MAP_TOL = 2e-4


def _f64view(v):
    v = dict(v)
    v["W"] = np.asarray(v["W"], np.float64); v["b"] = np.asarray(v["b"], np.float64)
    return v


def _records(rast, state, P):
    wv = R.workspace_view(rast, state)
    rec = R.device_array(wv.records, P * 16, torch.float32).view(P, 16).cpu().numpy().astype(np.float64)
    radii = R.device_array(wv.radii, P, torch.float32).cpu().numpy()
    depth = R.device_array(wv.depth, P, torch.float32).cpu().numpy()
    return wv, rec, radii, depth


def _gpu_lists(rast, state, total_tiles):
    wv = R.workspace_view(rast, state)
    n = int(R.device_array(wv.n_pairs, 1, torch.int32).item())
    ids = R.device_array(wv.pair_ids, n, torch.int32).cpu().numpy().astype(np.int64)
    tiles = R.device_array(wv.pair_tiles, n, torch.int32).cpu().numpy().astype(np.int64)
    rng = R.device_array(wv.ranges, 2 * total_tiles, torch.int32).view(total_tiles, 2).cpu().numpy().astype(np.int64)
    return ids, tiles, rng


CASES = [
    ("c1_full", lambda: (c1_scene(), c1_view()), 4),
    ("fisheye190_sh3", lambda: (S.make_scene(3000, 3, seed=5), S.make_view(7, S.CAM_FISHEYE, 190.0)), 4),
    ("pinhole_rot", lambda: (S.make_scene(2500, 3, seed=6),
                             S.random_pose_view(np.random.default_rng(2), 7, S.CAM_PINHOLE, 90.0, 70.0)), 3),
    ("full_b5", lambda: (S.make_scene(2500, 0, seed=7, logscale_mu=-2.0), S.make_view(7)), 5),
    ("pinhole_off_centre", lambda: (S.make_scene(2500, 3, seed=8),
                                    S.random_pose_view(np.random.default_rng(12), 7, S.CAM_PINHOLE, 100.0, 75.0,
                                                       pp=(0.35, -0.5))), 4),
    # anisotropic fisheye, w_x != w_y (Sec. D.1, Eq. fish_weff)
    ("fisheye_aniso_220x180", lambda: (S.make_scene(3000, 3, seed=9),
                                       S.random_pose_view(np.random.default_rng(13), 7, S.CAM_FISHEYE, 220.0, 180.0)), 4),
]


@pytest.mark.parametrize("name,make,b", CASES, ids=[c[0] for c in CASES])
def test_staged_records_lists_and_maps(name, make, b):
    sc, view = make()
    rast = R.Rasterizer(tile_level=b)
    cfg = oracle_cfg(rast)
    k = view["nside_log2"]
    P = sc["means"].shape[0]
    ts, out, state = gpu_render(sc, [view], rast)
    wv, rec, radii, depth = _records(rast, state, P)
    # ---- stage 1: records vs oracle preprocessing (FP32 tolerance)
    pre = O.preprocess(sc, _f64view(view), cfg)
    valid = radii > 0
    # the GPU also culls Gaussians outside the FoV cap; they must be ones the oracle lists nowhere
    assert np.all(pre["valid"][valid] == 1)
    culled = np.nonzero((pre["valid"] == 1) & ~valid)[0]
    full0 = O.render(sc, _f64view(view), cfg)
    assert not np.isin(full0.ids, culled).any()
    assert np.allclose(rec[valid, 0:3], pre["g"][valid], atol=3e-7)
    assert np.allclose(rec[valid, 12:15], pre["col"][valid], atol=2e-6)
    assert np.allclose(radii[valid], pre["rs"][valid], rtol=2e-5)
    conic_gpu = rec[:, [7, 11, 15]]
    scale = np.abs(pre["conic"][valid]).max(1, keepdims=True)
    assert np.abs(conic_gpu[valid] - pre["conic"][valid]).max() <= 0 + (2e-4 * scale).max()
    # ---- mask and active tiles
    m_gpu = mask_from_words(out["mask"].cpu().numpy().view(np.uint32), O.npix(2 ** k))
    m_ref, margin = O.mask(2 ** k, view["cam"], view["fov_x"], view["fov_y"], view.get("pp", (0.0, 0.0)))
    assert np.all(np.abs(margin[m_gpu != m_ref]) < 1e-12)
    act = O.active_tiles(k, b, m_gpu)
    # ---- stage 2: tile lists from the GPU's stored FP32 values, exact
    rho = O.tile_rho(k, b)
    dbits = depth.astype(np.float32).view(np.uint32).copy()
    dbits[~valid] = 0xFFFFFFFF
    start, ids_ref = O.tile_lists(k, b, rec[:, 0:3], radii.astype(np.float64), valid.astype(np.int32), dbits, rho, act)
    nt = act.size
    ids, tiles, rng = _gpu_lists(rast, state, nt)
    assert ids.size == ids_ref.size
    for t in np.nonzero(act)[0]:
        a = ids[rng[t, 0]:rng[t, 1]] if rng[t, 1] > rng[t, 0] else np.zeros(0, np.int64)
        bref = ids_ref[start[t]:start[t + 1]]
        assert np.array_equal(a, bref), (t, a[:10], bref[:10])
    # ---- stage 3: compositing from the GPU's records and lists (FP64), then end to end
    pre_g = dict(omega=np.arctan2(rec[:, 1], rec[:, 0]), phi=np.arctan2(rec[:, 2], np.hypot(rec[:, 0], rec[:, 1])),
                 conic=conic_gpu, col=rec[:, 12:15], r=depth.astype(np.float64))
    pix = np.nonzero(m_gpu)[0].astype(np.int64)
    mg = out["maps"].cpu().numpy()[pix]
    Tg = out["T"].cpu().numpy()[pix]
    lg = out["last"].cpu().numpy()[pix]
    n_ok, n_ex, _, _ = match_oracle(k, b, pre_g, rec[:, 3], start, ids_ref, pix, cfg, mg, Tg, gpu_last=lg)
    assert n_ex <= MAX_EXCLUDED_SHARE * pix.size
    # end to end (oracle from scratch in FP64): the depth keys are the same float32 values
    # on both sides, so the order is the same; pixels whose mask decision the two sides take
    # differently sit on the FoV boundary itself (FP64 margin < 1e-12, checked above)
    full = O.render(sc, _f64view(view), cfg)
    assert np.array_equal(O.depth_bits(full.pre["r"])[valid], dbits[valid])
    both = pix[m_ref[pix] == 1]
    sel = m_ref[pix] == 1
    n_ok, n_ex, _, _ = match_oracle(k, b, full.pre, sc["opacities"], full.start, full.ids, both, cfg, mg[sel], Tg[sel])
    assert n_ex <= MAX_EXCLUDED_SHARE * both.size
    # outside the mask: background, T = 1
    outside = np.nonzero(m_gpu == 0)[0]
    if outside.size:
        assert np.all(out["maps"].cpu().numpy()[outside] == 0) and np.all(out["T"].cpu().numpy()[outside] == 1)


@pytest.mark.parametrize("b", [3, 4, 5])
def test_maps_independent_of_tile_level(b):
    sc, view = S.make_scene(4000, 3, seed=11), S.make_view(7, S.CAM_FISHEYE, 200.0)
    ref = None
    rast = R.Rasterizer(tile_level=b)
    _, out, _ = gpu_render(sc, [view], rast)
    full = O.render(sc, _f64view(view), oracle_cfg(rast))
    pix = full.pix
    n_ok, n_ex, _, _ = match_oracle(7, b, full.pre, sc["opacities"], full.start, full.ids, pix, oracle_cfg(rast),
                                 out["maps"].cpu().numpy()[pix], out["T"].cpu().numpy()[pix])
    assert n_ex <= MAX_EXCLUDED_SHARE * pix.size


def test_batched_views_equal_single_views():
    sc = S.make_scene(3000, 3, seed=21)
    rng = np.random.default_rng(3)
    views = [S.random_pose_view(rng, 7, S.CAM_PINHOLE, 90.0, 90.0, 0.5), S.random_pose_view(rng, 6, S.CAM_FISHEYE, 180.0, None, 0.5),
             S.random_pose_view(rng, 5, S.CAM_FULL, 360.0, None, 0.5)]
    rast = R.Rasterizer()
    _, outb, _ = gpu_render(sc, views, rast)
    lay = outb["layout"]
    for v, base in zip(views, lay.pix_base):
        _, outs, _ = gpu_render(sc, [v], R.Rasterizer())
        n = R.npix(v["nside_log2"])
        assert torch.equal(outb["maps"][base:base + n], outs["maps"])
        assert torch.equal(outb["last"][base:base + n], outs["last"])


def test_empty_and_degenerate_inputs():
    # no Gaussians; all Gaussians behind the near plane; a Gaussian at the pole of the camera frame
    rast = R.Rasterizer()
    empty = S.make_scene(0, 0, seed=1)
    _, out, _ = gpu_render(empty, [S.make_view(5)], rast)
    assert torch.all(out["maps"] == 0) and torch.all(out["T"] == 1) and torch.all(out["last"] == 0)
    near = S.make_scene(50, 0, seed=2, r_min=0.01, r_max=0.15)
    _, out, _ = gpu_render(near, [S.make_view(5)], R.Rasterizer())
    assert torch.all(out["T"] == 1)
    pole = S.make_scene(1, 0, seed=3)
    pole["means"][:] = [[0.0, 3.0, 0.0]]
    pole["scales"][:] = 0.1
    _, out, _ = gpu_render(pole, [S.make_view(6)], R.Rasterizer())
    full = O.render(pole, _f64view(S.make_view(6)), O.Config())
    assert np.abs(out["maps"].cpu().numpy() - full.image).max() < MAP_TOL


def test_capacity_overflow_is_reported_and_recovered():
    sc, view = c1_scene(), c1_view()
    rast = R.Rasterizer(capacity=100)
    ts, out, state = gpu_render(sc, [view], rast)     # grows the capacity and re-runs
    assert rast.capacity > 100
    rast2 = R.Rasterizer(capacity=100)
    out2, _ = rast2.forward_raw(*ts, 0, [view], check_status=False)
    torch.cuda.synchronize()
    assert int(out2["status"].item()) & 1
    assert torch.equal(out["maps"], R.Rasterizer().forward_raw(*ts, 0, [view])[0]["maps"])


def _grad_check(sc, view, b, seed):
    rast = R.Rasterizer(tile_level=b)
    cfg = oracle_cfg(rast)
    ts = [t.requires_grad_(True) for t in scene_tensors(sc)]
    maps, T, last, mask, radii = R.render(*ts, [view], rasterizer=rast, sh_degree=sc["sh_degree"])
    k = view["nside_log2"]
    full = O.render(sc, _f64view(view), cfg)
    pix = full.pix
    ok = full.amb[pix] == 0
    rng = np.random.default_rng(seed)
    dI = rng.standard_normal((pix.size, 3))
    dI[~ok] = 0.0
    dfull = np.zeros((O.npix(2 ** k), 3), np.float32)
    dfull[pix] = dI
    maps.backward(torch.as_tensor(dfull, device="cuda"))
    ref = O.backward(sc, _f64view(view), cfg, dI, full.start, full.ids, pix)
    names = ["means", "scales", "rotations", "opacities", "sh"]
    for t, name in zip(ts, names):
        g = t.grad.cpu().numpy().astype(np.float64).reshape(ref[name].shape)
        r = ref[name]
        rel = np.linalg.norm(g - r) / max(1e-30, np.linalg.norm(r))
        assert rel <= 1e-3, (name, rel)
        assert np.abs(g - r).max() <= 1e-3 * np.abs(r).max() + 1e-12, (name, np.abs(g - r).max(), np.abs(r).max())


def test_gradients_c1():
    _grad_check(c1_scene(), c1_view(), 4, 0)


def test_gradients_fisheye_sh3():
    sc = S.make_scene(5000, 3, seed=41, logscale_mu=-2.2)
    view = S.random_pose_view(np.random.default_rng(9), 7, S.CAM_FISHEYE, 190.0, None, 0.5)
    _grad_check(sc, view, 4, 1)


def test_gradients_pinhole_b3():
    sc = S.make_scene(3000, 3, seed=42)
    view = S.random_pose_view(np.random.default_rng(10), 7, S.CAM_PINHOLE, 80.0, 100.0, 0.5)
    _grad_check(sc, view, 3, 2)


def test_gradients_off_centre_pinhole():
    sc = S.make_scene(3000, 3, seed=43)
    view = S.random_pose_view(np.random.default_rng(11), 7, S.CAM_PINHOLE, 90.0, 70.0, 0.5, pp=(-0.6, 0.4))
    _grad_check(sc, view, 4, 3)


def test_gradients_anisotropic_fisheye():
    sc = S.make_scene(3000, 3, seed=44)
    view = S.random_pose_view(np.random.default_rng(14), 7, S.CAM_FISHEYE, 220.0, 180.0, 0.5)
    _grad_check(sc, view, 4, 4)

