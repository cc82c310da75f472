"""GPU tests of the system layer: CUDA-graph training step, autotuner, serving loop.

- a graph replay of the training step gives the eager step's losses and gradients;
- the autotuner returns one of its candidates and timings for all that built;
- a request rendered alone equals the same request inside a mixed batch (bit for bit);
- the real-time server serves every request in batched and in plain mode, with
  each served map equal to the request rendered alone;
- a batch whose tile lists were under-predicted is detected and rendered again.
"""
import numpy as np
import pytest
import torch

from paper_2606_29794_b300 import raster as R
from paper_2606_29794_b300 import serve as SV
from paper_2606_29794_b300 import synth as S
from tests.gpu_util import scene_tensors

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]


def _views(seed=0):
    rng = np.random.default_rng(seed)
    return [S.random_pose_view(rng, 7, S.CAM_FISHEYE, 190.0, None, 0.5),
            S.random_pose_view(rng, 6, S.CAM_PINHOLE, 80.0, 80.0, 0.5),
            S.random_pose_view(rng, 5, S.CAM_FULL, 360.0, None, 0.5)]


def test_graph_step_matches_eager():
    sc = S.make_scene(20000, 3, seed=51)
    tgt = S.perturb_scene(sc, 52)
    views = _views(1)
    params = scene_tensors(sc)
    rast_t = R.Rasterizer()
    with torch.no_grad():
        tout, _ = rast_t.forward_raw(*scene_tensors(tgt), 3, views)
    targets = tout["maps"].clone()
    step = R.GraphStep(params, 3, views, targets, R.Rasterizer())
    losses, grads = step.replay()
    torch.cuda.synchronize()
    l_graph = losses.clone()
    g_graph = [g.clone() for g in grads]
    assert int(step.status.item()) == 0
    # eager reference through the public API
    rast = R.Rasterizer()
    ps = [p.clone().requires_grad_(True) for p in params]
    maps, T, last, mask, radii = R.render(*ps, views, rasterizer=rast, sh_degree=3)
    lay = R.view_layout(views)
    total = 0
    for vi, (v, base) in enumerate(zip(views, lay.pix_base)):
        n = R.npix(v["nside_log2"])
        loss, parts = R.hssim_loss(maps[base:base + n], targets[base:base + n], mask[base // 32:(base + n) // 32],
                                   v["nside_log2"], 0.2)
        assert torch.allclose(parts, l_graph[vi], atol=1e-6)
        total = total + loss
    total.backward()
    for p, g in zip(ps, g_graph):
        assert torch.allclose(p.grad, g, rtol=1e-4, atol=1e-6 * float(g.abs().max()) + 1e-12)
    # replay again: same losses
    losses2, _ = step.replay()
    torch.cuda.synchronize()
    assert torch.equal(losses2, l_graph)


def test_autotuner_picks_a_candidate():
    sc = S.make_scene(20000, 3, seed=53)
    params = scene_tensors(sc)
    views = _views(2)
    targets = torch.rand((R.view_layout(views).total_pix, 3), device="cuda")

    def make(kw):
        st = R.GraphStep(params, 3, views, targets, R.Rasterizer(**kw))
        return st.replay

    cands = [dict(tile_level=4), dict(tile_level=3), dict(tile_level=4, blocks_per_sm=2)]
    best, timings = R.autotune(make, cands, reps=2, warmup=1)
    assert best in cands and len(timings) == 3 and all(t > 0 for t in timings.values())


def test_request_alone_equals_request_in_mix():
    sc = S.make_scene(30000, 3, seed=54)
    srv = SV.RenderServer(scene_tensors(sc), 3, budget_bytes=2 << 30)
    views = _views(3)
    alone = [srv.render_batch([v]) for v in views]
    mix = srv.render_batch(views)
    lay = mix["layout"]
    for a, v, base in zip(alone, views, lay.pix_base):
        n = R.npix(v["nside_log2"])
        assert torch.equal(a["maps"], mix["maps"][base:base + n])
        assert torch.equal(a["T"], mix["T"][base:base + n])


@pytest.mark.parametrize("plain", [False, True])
def test_server_serves_stream(plain):
    sc = S.make_scene(30000, 3, seed=55)
    srv = SV.RenderServer(scene_tensors(sc), 3, budget_bytes=2 << 30, slots=3, max_views=4)
    reqs = S.request_stream(24, rate_hz=400.0, seed=56, nside_choices=(5, 6, 7))
    stats, results = srv.run(reqs, plain=plain, keep_outputs=True)
    summ = stats.summary()
    assert summ["served"] == 24 and summ["p99_ms"] >= summ["p50_ms"] > 0
    if plain:
        assert summ["mean_batch"] == 1.0
    for r in reqs[:6]:
        job = results[r["id"]]
        idx = [q["id"] for q in job["reqs"]].index(r["id"])
        base = job["layout"].pix_base[idx]
        n = R.npix(r["view"]["nside_log2"])
        alone = srv.render_batch([r["view"]])
        assert torch.equal(alone["maps"], job["maps"][base:base + n])


def test_underpredicted_capacity_is_rerun():
    sc = S.make_scene(30000, 3, seed=57)
    srv = SV.RenderServer(scene_tensors(sc), 3, budget_bytes=2 << 30)
    reqs = S.request_stream(6, rate_hz=1000.0, seed=58, nside_choices=(6,))
    for r in reqs:
        srv._count([r["view"]])
    for k in list(srv.pairs_per_pixel):
        srv.pairs_per_pixel[k] = 1e-6            # force a gross under-prediction
    srv.headroom = 1.0
    stats, results = srv.run(reqs, keep_outputs=True)
    assert stats.served == 6 and stats.reruns > 0
    r = reqs[0]
    job = results[r["id"]]
    idx = [q["id"] for q in job["reqs"]].index(r["id"])
    base = job["layout"].pix_base[idx]
    n = R.npix(r["view"]["nside_log2"])
    srv.headroom = 1.3
    assert torch.equal(srv.render_batch([r["view"]])["maps"], job["maps"][base:base + n])


def test_graph_step_with_host_targets_matches_device_targets():
    # the copy of pinned host targets inside the graph (overlapping the forward)
    # gives the same losses and gradients as targets already on the device
    sc = S.make_scene(20000, 3, seed=59)
    views = _views(4)
    params = scene_tensors(sc)
    lay = R.view_layout(views)
    g = torch.Generator().manual_seed(60)
    tgt = torch.rand((lay.total_pix, 3), generator=g)
    host = tgt.pin_memory()
    dev_step = R.GraphStep(params, 3, views, tgt.cuda(), R.Rasterizer())
    host_step = R.GraphStep(params, 3, views, torch.zeros_like(tgt, device="cuda"), R.Rasterizer(), host_targets=host)
    l1, g1 = dev_step.replay()
    l2, g2 = host_step.replay()
    torch.cuda.synchronize()
    l2 = l2.clone()                                  # replay returns the graph's static buffers
    assert torch.equal(l1, l2)
    # the same partials added by atomics in another order (rotation gradients cancel strongly)
    for a, b in zip(g1, g2):
        assert float((a - b).norm()) <= 1e-4 * float(a.norm()) + 1e-12
        assert float((a - b).abs().max()) <= 1e-3 * float(a.abs().max()) + 1e-12
    host.mul_(0.5)                                   # a new target written in place is picked up by the next replay
    l3, _ = host_step.replay()
    torch.cuda.synchronize()
    assert not torch.equal(l3, l2)


def test_graph_step_with_host_camera_images_matches_float_image_targets():
    # a pinned 8-bit camera image per view, copied in and resampled onto the view's grid inside
    # the graph (hpxgs_image_to_sphere_u8), gives the targets of the float image v / 255 resampled
    # on the device: the same losses, gradients up to the order of atomic sums
    from paper_2606_29794_b300 import resample as RS
    sc = S.make_scene(20000, 3, seed=62)
    views = [S.make_view(7, S.CAM_FISHEYE, 190.0), S.make_view(6, S.CAM_PINHOLE, 90.0, 70.0)]
    sizes = [(300, 300), (240, 180)]
    params = scene_tensors(sc)
    lay = R.view_layout(views)
    g = torch.Generator().manual_seed(63)
    imgs = [torch.randint(0, 256, (h, w, 3), dtype=torch.uint8, generator=g) for w, h in sizes]
    tgt = torch.zeros((lay.total_pix, 3), device="cuda")
    for v, base, im in zip(views, lay.pix_base, imgs):
        n = R.npix(v["nside_log2"])
        RS.image_to_sphere_into((im.float() / 255.0).cuda(), v, v["nside_log2"], tgt[base:base + n])
        # the 8-bit entry point itself: the float image's map bit for bit
        m8, w8 = RS.image_to_sphere(im.cuda(), v, v["nside_log2"])
        assert torch.equal(m8, tgt[base:base + n])
    dev_step = R.GraphStep(params, 3, views, tgt, R.Rasterizer())
    host_step = R.GraphStep(params, 3, views, torch.zeros_like(tgt), R.Rasterizer(),
                            host_images=[im.pin_memory() for im in imgs])
    l1, g1 = dev_step.replay()
    l2, g2 = host_step.replay()
    torch.cuda.synchronize()
    assert torch.equal(l1, l2.clone())
    assert torch.equal(host_step.targets, tgt)
    for a, b in zip(g1, g2):
        assert float((a - b).norm()) <= 1e-4 * float(a.norm()) + 1e-12
        assert float((a - b).abs().max()) <= 1e-3 * float(a.abs().max()) + 1e-12


@pytest.mark.parametrize("tile_level,views,split", [(5, "fisheye", 1), (5, "fisheye", 0), (4, "mixed", 1),
                                                    (3, "fisheye", 1)])
def test_fused_loss_backward_equals_two_pass(tile_level, views, split):
    # hpxgs_backward_hssim (dL/dI formed inside the backward blend) against the HSSIM
    # backward writing dL/dmaps followed by hpxgs_backward: same losses, gradients equal
    # up to the order of the atomic sums
    sc = S.make_scene(20000, 3, seed=61)
    vs = [S.make_view(7, S.CAM_FISHEYE, 190.0)] if views == "fisheye" else _views(5)
    params = scene_tensors(sc)
    lay = R.view_layout(vs)
    g = torch.Generator().manual_seed(62)
    tgt = torch.rand((lay.total_pix, 3), generator=g).cuda()
    res = []
    for fused in (True, False):
        st = R.GraphStep(params, 3, vs, tgt, R.Rasterizer(tile_level=tile_level, blend_split=split), fused=fused)
        losses, grads = st.replay()
        torch.cuda.synchronize()
        assert int(st.status.item()) == 0
        res.append((losses.clone(), [x.clone() for x in grads], st.launches_per_replay))
    (l1, g1, n1), (l0, g0, n0) = res
    assert torch.equal(l1, l0)
    assert n1 == n0 - len(vs)                          # one HSSIM backward launch fewer per view
    for a, b in zip(g1, g0):
        assert float((a - b).norm()) <= 1e-4 * float(b.norm()) + 1e-12
        assert float((a - b).abs().max()) <= 1e-3 * float(b.abs().max()) + 1e-12


def test_fused_loss_backward_direct_with_dloss():
    # the C ABI call with a per-view dL/dloss against the two-pass path with the same scale
    import ctypes
    from paper_2606_29794_b300 import _lib as L
    sc = S.make_scene(15000, 3, seed=63)
    vs = _views(6)
    params = scene_tensors(sc)
    lay = R.view_layout(vs)
    tgt = torch.rand((lay.total_pix, 3), generator=torch.Generator().manual_seed(64)).cuda()
    rast = R.Rasterizer()
    out, state = rast.forward_raw(*params, 3, vs)
    dl = torch.tensor([0.5, 2.0, 1.25], device="cuda")
    dmaps = torch.zeros((lay.total_pix, 3), device="cuda")
    loss_views = []
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for vi, (v, base) in enumerate(zip(vs, lay.pix_base)):
        k = v["nside_log2"]
        n = R.npix(k)
        I, G = out["maps"][base:base + n], tgt[base:base + n]
        m = out["mask"][base // 32:(base + n) // 32]
        tab = R.hssim_table(m, k)
        nb = ctypes.c_size_t()
        L.check(L.lib().hpxgs_hssim_workspace_size(k, ctypes.byref(nb)), "ws")
        ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
        l3 = torch.empty(3, device="cuda")
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        L.check(L.lib().hpxgs_hssim_forward_table(p(I), p(G), p(m), k, 0.2, p(tab), p(ws), nb.value, p(l3), s), "f")
        L.check(L.lib().hpxgs_hssim_backward_table(p(I), p(G), p(m), k, 0.2, p(tab), p(ws), nb.value, p(dl[vi:vi + 1]),
                                                   p(dmaps[base:base + n]), s), "b")
        loss_views.append((I, G, tab, ws, dl[vi:vi + 1]))
    ref = rast.backward_raw(state, dmaps)
    got = rast.backward_hssim_raw(state, loss_views, 0.2)
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert float((a - b).norm()) <= 1e-4 * float(b.norm()) + 1e-12
        assert float((a - b).abs().max()) <= 1e-3 * float(b.abs().max()) + 1e-12


def test_render_loss_autograd_equals_render_then_loss():
    # the one-pass autograd loss (hpxgs_backward_hssim) against render + hssim_loss per view,
    # summed; a scaled loss scales the gradients
    sc = S.make_scene(20000, 3, seed=65)
    vs = _views(7)
    lay = R.view_layout(vs)
    tgt = torch.rand((lay.total_pix, 3), generator=torch.Generator().manual_seed(66)).cuda()
    base = scene_tensors(sc)
    ps = [p.clone().requires_grad_(True) for p in base]
    rast = R.Rasterizer()
    loss, parts = R.render_loss(*ps, vs, tgt, rasterizer=rast, sh_degree=3)
    (2.5 * loss).backward()
    g_fused = [p.grad.clone() for p in ps]
    qs = [p.clone().requires_grad_(True) for p in base]
    maps, T, last, mask, radii = R.render(*qs, vs, rasterizer=R.Rasterizer(), sh_degree=3)
    total = 0
    for vi, (v, b0) in enumerate(zip(vs, lay.pix_base)):
        n = R.npix(v["nside_log2"])
        lv, pv = R.hssim_loss(maps[b0:b0 + n], tgt[b0:b0 + n], mask[b0 // 32:(b0 + n) // 32], v["nside_log2"], 0.2)
        assert torch.equal(pv, parts[vi])                      # table and direct HSSIM forward agree bit for bit
        total = total + lv
    assert torch.allclose(total, loss, rtol=1e-6, atol=0)
    (2.5 * total).backward()
    for a, q in zip(g_fused, qs):
        c = q.grad
        assert float((a - c).double().norm()) <= 1e-4 * float(c.double().norm()) + 1e-12
        assert float((a - c).abs().max()) <= 1e-3 * float(c.abs().max()) + 1e-12
