"""Parity at the full sizes of the measured workloads, on sampled outputs.

Rendering a 300k-, 1M- or 6M-Gaussian scene end to end in FP64 takes the oracle
far longer than a test may run, but every pixel is defined by its own tile's
list alone (Algorithm 1; with the m <= 9 cutoff the map does not depend on
which other tiles exist). So for a seeded sample of active tiles the oracle
builds only those lists (membership definition over every Gaussian) and
composites a sample of their pixels. Each workload runs in the launch
configuration the benchmark times (order-5 lists blended by 16 x 16 quarters;
default pixels per thread):

- tile lists of the sampled tiles, rebuilt by the oracle from the GPU's stored
  FP32 (g, r_s, depth): exact, including order;
- compositing of the sampled pixels by the oracle from the GPU's FP32 records
  and those lists: maps and T within 2e-4 and the last index equal;
- the depth keys: the GPU forms the radial depth in FP64 in the oracle's order
  of operations, so the float32 sort keys are equal bit for bit;
- maps and T at the sampled pixels vs the oracle from scratch in FP64: 2e-4.
  In both comparisons a cutoff or termination decision that FP32 cannot settle
  may take either outcome (tests.gpu_util.match_oracle), and at most 1e-5 of
  the sampled pixels may be excluded (more such decisions than the oracle's
  variants follow); the counts are printed;
- gradients of a loss weighting only the sampled pixels vs the oracle's backward
  over the same pixels: 1e-3 relative (the oracle's backward runs on the
  Gaussians listed in the sampled tiles, the only ones those pixels see).

Workloads: Nside 512 fisheye 190 deg with 300k SH3 Gaussians (the training
step); 16 views of three cameras over 1M SH3 Gaussians; Nside 2048 full sphere
with 6M SH3 Gaussians (log-scales N(-3.5, 0.7)).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import raster as R
from paper_2606_29794_b300 import synth as S
from tests.gpu_util import MAX_EXCLUDED_SHARE, mask_from_words, match_oracle, oracle_cfg, scene_tensors

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]

MAP_TOL = 2e-4
GRAD_TOL = 1e-3


def _f64view(v):
    v = dict(v)
    v["W"] = np.asarray(v["W"], np.float64); v["b"] = np.asarray(v["b"], np.float64)
    return v


def _check_views(sc, views, rast, out, state, n_tiles, per_tile, seed):
    """Sampled list, map and T parity for every view of one batched forward.
    Returns per view (pixels, oracle lists (start, ids), ambiguity flags)."""
    cfg = oracle_cfg(rast)
    b = rast.tile_level
    P = sc["means"].shape[0]
    nv = len(views)
    lay = out["layout"]
    wv = R.workspace_view(rast, state)
    rec = R.device_array(wv.records, nv * P * 16, torch.float32).view(nv * P, 16)
    radii = R.device_array(wv.radii, nv * P, torch.float32)
    depth = R.device_array(wv.depth, nv * P, torch.float32)
    n_pairs = int(R.device_array(wv.n_pairs, 1, torch.int32).item())
    gids = R.device_array(wv.pair_ids, n_pairs, torch.int32).cpu().numpy().astype(np.int64)
    ranges = R.device_array(wv.ranges, 2 * lay.total_tiles, torch.int32).view(-1, 2).cpu().numpy().astype(np.int64)
    maps = out["maps"].cpu().numpy()
    Tg = out["T"].cpu().numpy()
    lastg = out["last"].cpu().numpy().astype(np.int64)
    words = out["mask"].cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(seed)
    res = []
    tile_base = 0
    total = excluded = staged_ex = alt = 0
    for v, view in enumerate(views):
        k = view["nside_log2"]
        N = O.npix(2 ** k)
        base = lay.pix_base[v]
        m_gpu = mask_from_words(words[base // 32:(base + N) // 32], N)
        m_ref, margin = O.mask(2 ** k, view["cam"], view["fov_x"], view["fov_y"])
        assert np.all(np.abs(margin[m_gpu != m_ref]) < 1e-12)
        act = O.active_tiles(k, b, m_gpu)
        cand = np.nonzero(act)[0]
        tiles = np.sort(rng.choice(cand, min(n_tiles, cand.size), replace=False))
        # ---- lists of the sampled tiles from the GPU's FP32 values: exact
        sl = slice(v * P, (v + 1) * P)
        g32 = rec[sl, 0:3].cpu().numpy().astype(np.float64)
        rs32 = radii[sl].cpu().numpy()
        valid = rs32 > 0
        dbits = depth[sl].cpu().numpy().astype(np.float32).view(np.uint32).copy()
        dbits[~valid] = 0xFFFFFFFF
        rho = O.tile_rho(k, b)
        st, ids_ref = O.tile_lists_subset(k, b, g32, rs32.astype(np.float64), valid.astype(np.int32), dbits, rho,
                                          act, tiles)
        for t in tiles:
            lo, hi = ranges[tile_base + t]
            got = gids[lo:hi] - v * P if hi > lo else np.zeros(0, np.int64)
            assert np.array_equal(got, ids_ref[st[t]:st[t + 1]]), (v, t, got[:8], ids_ref[st[t]:st[t] + 8])
        pix = []
        for t in tiles:
            inside = (t << (2 * b)) + np.nonzero((m_gpu & m_ref)[t << (2 * b):(t + 1) << (2 * b)])[0]
            pix.append(rng.choice(inside, min(per_tile, inside.size), replace=False))
        pix = np.sort(np.concatenate(pix)).astype(np.int64)
        # ---- staged compositing from the GPU's records and lists
        r32 = rec[sl].cpu().numpy().astype(np.float64)
        pre_g = dict(omega=np.arctan2(r32[:, 1], r32[:, 0]), phi=np.arctan2(r32[:, 2], np.hypot(r32[:, 0], r32[:, 1])),
                     conic=r32[:, [7, 11, 15]], col=r32[:, 12:15], r=depth[sl].cpu().numpy().astype(np.float64))
        _, n_ex, n_alt, _ = match_oracle(k, b, pre_g, r32[:, 3], st, ids_ref, pix, cfg, maps[base + pix], Tg[base + pix],
                                         gpu_last=lastg[base + pix])
        staged_ex += n_ex
        # ---- maps and T at sampled pixels vs the oracle from scratch
        pre = O.preprocess(sc, _f64view(view), cfg)
        # the depth keys: float32 of the same FP64 radial depth on both sides
        assert np.array_equal(O.depth_bits(pre["r"])[valid], dbits[valid])
        act_ref = O.active_tiles(k, b, m_ref)
        st2, ids2 = O.tile_lists_subset(k, b, pre["g"], pre["rs"], pre["valid"], O.depth_bits(pre["r"]), rho,
                                        act_ref, tiles)
        _, n_ex, n_alt, amb = match_oracle(k, b, pre, sc["opacities"], st2, ids2, pix, cfg, maps[base + pix],
                                           Tg[base + pix])
        excluded += n_ex; alt += n_alt; total += pix.size
        res.append((pix, st2, ids2, amb))
        tile_base += 12 * 4 ** (k - b)
    print(f"sampled pixels {total}: excluded {excluded} (staged {staged_ex}), matched by an FP32-band variant {alt}")
    assert staged_ex <= MAX_EXCLUDED_SHARE * total, (staged_ex, total)
    assert excluded <= MAX_EXCLUDED_SHARE * total, (excluded, total)
    return res


def _oracle_backward_listed(sc, view, cfg, dI, st, ids, pix):
    """The oracle's backward (Sec. 3.2) for the sampled pixels, run on the sub-scene of the
    Gaussians their lists hold (the others cannot reach these pixels); gradients scattered
    back to the full scene, zero elsewhere."""
    P = sc["means"].shape[0]
    used = np.unique(ids)
    remap = np.full(P, -1, np.int64)
    remap[used] = np.arange(used.size)
    sub = {k: (np.asarray(v)[used] if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    r = O.backward(sub, _f64view(view), cfg, dI, st, remap[ids], pix)
    out = {}
    for name, g in r.items():
        full = np.zeros((P,) + g.shape[1:])
        full[used] = g
        out[name] = full
    return out


def _check_grads(sc, views, rast, out, state, sampled, seed, use=None):
    """Gradients of sum_p dI_p . I_p over the sampled pixels of the views `use` (default all)
    that have no FP32-undecidable decision; the backward still walks every view's tiles."""
    cfg = oracle_cfg(rast)
    lay = out["layout"]
    rng = np.random.default_rng(seed)
    dmaps = np.zeros((lay.total_pix, 3), np.float32)
    ref = None
    for v, (view, (pix, st, ids, amb)) in enumerate(zip(views, sampled)):
        if use is not None and v not in use:
            continue
        dI = rng.standard_normal((pix.size, 3)).astype(np.float32)
        dI[amb != 0] = 0.0
        dmaps[lay.pix_base[v] + pix] = dI
        r = _oracle_backward_listed(sc, view, cfg, dI.astype(np.float64), st, ids, pix)
        ref = r if ref is None else {n: ref[n] + r[n] for n in ref}
    grads = rast.backward_raw(state, torch.as_tensor(dmaps, device="cuda"))
    torch.cuda.synchronize()
    for name, gt in zip(["means", "scales", "rotations", "opacities", "sh"], grads):
        g = gt.cpu().numpy().astype(np.float64).reshape(ref[name].shape)
        r = ref[name]
        assert np.linalg.norm(r) > 0, name
        rel = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert rel <= GRAD_TOL, (name, rel)
        assert np.abs(g - r).max() <= GRAD_TOL * np.abs(r).max(), (name, np.abs(g - r).max(), np.abs(r).max())


def test_training_step_nside512_fisheye190_p300k():
    sc = S.make_scene(300_000, 3, seed=20261205)
    view = S.make_view(9, S.CAM_FISHEYE, 190.0)
    rast = R.Rasterizer(tile_level=5)
    out, state = rast.forward_raw(*scene_tensors(sc), 3, [view])
    torch.cuda.synchronize()
    sampled = _check_views(sc, [view], rast, out, state, n_tiles=48, per_tile=24, seed=1)
    _check_grads(sc, [view], rast, out, state, sampled, seed=2)


@pytest.mark.parametrize("workload", ["train_p300k", "views16_p1m"])
def test_fused_loss_step_equals_two_pass_at_full_size(workload):
    # the bench times the training step with the L1 + HSSIM backward folded into the backward
    # blend (hpxgs_backward_hssim); the two-pass step (HSSIM backward writing dL/dmaps, then
    # hpxgs_backward, checked against the oracle above) must give the same losses and, up to
    # the order of the atomic sums, the same gradients, in the launch configuration timed
    if workload == "train_p300k":
        sc, views, b = S.make_scene(300_000, 3, seed=20261205), [S.make_view(9, S.CAM_FISHEYE, 190.0)], 5
    else:
        sc, views, b = S.make_scene(1_000_000, 3, seed=20261206), S.multiview_set(20261208), 5
    params = scene_tensors(sc)
    lay = R.view_layout(views)
    tgt = torch.rand((lay.total_pix, 3), generator=torch.Generator().manual_seed(7)).cuda()
    res = []
    for fused in (True, False):
        st = R.GraphStep(params, 3, views, tgt, R.Rasterizer(tile_level=b), fused=fused)
        losses, grads = st.replay()
        torch.cuda.synchronize()
        assert int(st.status.item()) == 0
        res.append((losses.clone(), [x.clone() for x in grads]))
        del st
        torch.cuda.empty_cache()
    (l1, g1), (l0, g0) = res
    assert torch.equal(l1, l0)
    for a, c in zip(g1, g0):
        assert float((a - c).double().norm()) <= 1e-4 * float(c.double().norm()) + 1e-12
        assert float((a - c).abs().max()) <= 1e-3 * float(c.abs().max()) + 1e-12


def test_sixteen_views_p1m():
    sc = S.make_scene(1_000_000, 3, seed=20261206)
    views = S.multiview_set(20261208)
    rast = R.Rasterizer(tile_level=5)       # the level the benchmark's autotuner picks for this workload
    out, state = rast.forward_raw(*scene_tensors(sc), 3, views)
    torch.cuda.synchronize()
    sampled = _check_views(sc, views, rast, out, state, n_tiles=6, per_tile=16, seed=3)
    _check_grads(sc, views, rast, out, state, sampled, seed=4, use=(0, 1, 6, 12))   # pinhole x2, fisheye, full


def test_nside2048_full_sphere_p6m():
    sc = S.make_scene(6_000_000, 3, seed=20261213, logscale_mu=-3.5, logscale_sd=0.7)
    view = S.make_view(11)
    rast = R.Rasterizer(tile_level=5)
    out, state = rast.forward_raw(*scene_tensors(sc), 3, [view])
    torch.cuda.synchronize()
    sampled = _check_views(sc, [view], rast, out, state, n_tiles=24, per_tile=16, seed=5)
    # the backward from the stored T_final and last index alone (recompute in backward)
    _check_grads(sc, [view], rast, out, state, sampled, seed=6)


def test_timed_fused_step_against_oracle_full_size():
    # the step the benchmark times (forward, L1 + HSSIM loss, the loss backward folded into the
    # backward blend; CUDA graph; order-5 lists in 16 x 16 units) on the 300k training workload,
    # against the oracle over every in-mask pixel: the oracle renders the scene, evaluates the loss
    # (Sec. 4.1) against the same target and runs its backward (Sec. 3.2) on dL/dI of every pixel.
    # The target is the oracle's own render of the perturbed scene (rounded to float32).
    sc = S.make_scene(300_000, 3, seed=20261205)
    tgt = S.perturb_scene(sc, 20261206)
    view = S.make_view(9, S.CAM_FISHEYE, 190.0)
    rast = R.Rasterizer(tile_level=5)
    cfg = oracle_cfg(rast)
    cfg.tile_level = 4
    v64 = _f64view(view)
    G32 = O.render(tgt, v64, cfg).image.astype(np.float32)
    step = R.GraphStep(scene_tensors(sc), 3, [view], torch.as_tensor(G32, device="cuda"), rast, fused=True)
    losses, grads = step.replay()
    torch.cuda.synchronize()
    assert int(step.status.item()) == 0
    full = O.render(sc, v64, cfg)
    loss, h, l1, dI = O.hssim_loss(2 ** 9, full.image, G32.astype(np.float64), full.mask, cfg.lam)
    got = losses[0].cpu().numpy().astype(np.float64)
    assert np.abs(got - np.array([loss, h, l1])).max() < 2e-6, (got, loss, h, l1)
    ref = O.backward(sc, v64, cfg, dI[full.pix], full.start, full.ids, full.pix)
    for name, gt in zip(["means", "scales", "rotations", "opacities", "sh"], grads):
        g = gt.cpu().numpy().astype(np.float64).reshape(ref[name].shape)
        r = ref[name]
        rel = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert rel <= GRAD_TOL, (name, rel)
        assert np.abs(g - r).max() <= GRAD_TOL * np.abs(r).max(), (name, np.abs(g - r).max(), np.abs(r).max())
