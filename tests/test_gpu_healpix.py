"""GPU parity of the device HEALPix geometry and FoV masks against the FP64 oracle.

Bit-exact: vec2pix on random directions, pix2vec round trip, NESTED<->RING,
neighbour sets, masks (mismatches only where the FP64 margin is below 1e-12),
tile rho. FP32 pixel centres within 2e-7 rad.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import _lib as L
from paper_2606_29794_b300 import raster as R
from paper_2606_29794_b300 import synth as S

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("k", [0, 3, 9, 13])
def test_pix2ang_and_ang2pix_match_oracle(k):
    nside = 2 ** k
    n = min(12 * nside * nside, 200_000)
    rng = np.random.default_rng(k + 40)
    pix = np.sort(rng.choice(12 * nside * nside, n, replace=False)).astype(np.int64)
    pg = torch.as_tensor(pix, device="cuda")
    th = torch.empty(n, dtype=torch.float64, device="cuda")
    ph = torch.empty(n, dtype=torch.float64, device="cuda")
    L.check(L.lib().hpxgs_pix2ang_nest(k, _p(pg), n, _p(th), _p(ph), _s()), "pix2ang")
    back = torch.empty(n, dtype=torch.int64, device="cuda")
    L.check(L.lib().hpxgs_ang2pix_nest(k, _p(th), _p(ph), n, _p(back), _s()), "ang2pix")
    # random directions
    u = rng.random(n)
    t2 = np.arccos(1 - 2 * u)
    p2 = rng.random(n) * 2 * np.pi
    got = torch.empty(n, dtype=torch.int64, device="cuda")
    t2g, p2g = torch.as_tensor(t2, device="cuda"), torch.as_tensor(p2, device="cuda")   # held until the kernel ran
    L.check(L.lib().hpxgs_ang2pix_nest(k, _p(t2g), _p(p2g), n, _p(got), _s()), "ang2pix random")
    torch.cuda.synchronize()
    tr, pr = O.pix2ang_nest(nside, pix)
    assert np.abs(th.cpu().numpy() - tr).max() < 1e-12
    dphi = np.abs(np.angle(np.exp(1j * (ph.cpu().numpy() - pr))))     # longitude modulo 2 pi
    assert dphi.max() < 1e-12
    assert np.all((ph.cpu().numpy() >= 0) & (ph.cpu().numpy() < 2 * np.pi))
    assert np.array_equal(back.cpu().numpy(), pix)                     # centres map to their pixel
    assert np.array_equal(got.cpu().numpy(), O.ang2pix_nest(nside, t2, p2))


@pytest.mark.parametrize("k", [0, 1, 3, 6, 9, 11])
def test_pix2vec_and_roundtrip(k):
    n = 12 * 4 ** k
    p = np.arange(n, dtype=np.int64) if n <= 4_000_000 else np.random.default_rng(k).integers(0, n, 2_000_000)
    pt = torch.as_tensor(p, device="cuda")
    v32 = torch.empty((p.size, 3), dtype=torch.float32, device="cuda")
    v64 = torch.empty((p.size, 3), dtype=torch.float64, device="cuda")
    L.check(L.lib().hpxgs_pix2vec_nest(k, _p(pt), p.size, _p(v32), _p(v64), _s()), "pix2vec")
    back = torch.empty_like(pt)
    L.check(L.lib().hpxgs_vec2pix_nest(k, _p(v64), p.size, _p(back), _s()), "vec2pix")
    torch.cuda.synchronize()
    ref = O.pix2vec_nest(2 ** k, p)
    assert np.abs(v64.cpu().numpy() - ref).max() < 1e-14
    ang32 = np.linalg.norm(v32.cpu().numpy().astype(np.float64) - ref, axis=1)
    assert ang32.max() < 2e-7
    assert np.array_equal(back.cpu().numpy(), p)


@pytest.mark.parametrize("k", [2, 7, 10])
def test_vec2pix_random_directions(k):
    rng = np.random.default_rng(100 + k)
    v = rng.standard_normal((1_000_000, 3))
    vt = torch.as_tensor(v, device="cuda")
    out = torch.empty(v.shape[0], dtype=torch.int64, device="cuda")
    L.check(L.lib().hpxgs_vec2pix_nest(k, _p(vt), v.shape[0], _p(out), _s()), "vec2pix")
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), O.vec2pix_nest(2 ** k, v))


@pytest.mark.parametrize("k", [0, 1, 4, 8])
def test_nest_ring_conversion(k):
    n = 12 * 4 ** k
    p = torch.arange(n, dtype=torch.int64, device="cuda")
    r = torch.empty_like(p); q = torch.empty_like(p)
    L.check(L.lib().hpxgs_nest2ring(k, _p(p), n, _p(r), _s()), "nest2ring")
    L.check(L.lib().hpxgs_ring2nest(k, _p(r), n, _p(q), _s()), "ring2nest")
    torch.cuda.synchronize()
    assert np.array_equal(r.cpu().numpy(), O.nest2ring(2 ** k, np.arange(n)))
    assert np.array_equal(q.cpu().numpy(), np.arange(n))


@pytest.mark.parametrize("k", [1, 2, 5, 7])
def test_neighbours_match_vertex_sharing(k):
    n = 12 * 4 ** k
    p = torch.arange(n, dtype=torch.int64, device="cuda")
    out = torch.empty((n, 8), dtype=torch.int64, device="cuda")
    L.check(L.lib().hpxgs_neighbours_nest(k, _p(p), n, _p(out), _s()), "neighbours")
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref, cnt = O.neighbours_nest(2 ** k, np.arange(n))
    for i in range(n):
        g = sorted(x for x in got[i] if x >= 0)
        r = sorted(x for x in ref[i] if x >= 0)
        assert g == r, (k, i, g, r)
    assert ((got >= 0).sum(1) == 7).sum() == 24


@pytest.mark.parametrize("k,kind,fx,fy", [(6, 0, 360, 360), (9, 2, 190, 190), (8, 1, 90, 90), (9, 1, 60, 100),
                                          (7, 2, 220, 180), (10, 2, 180, 180)])
def test_mask_bits_match_oracle(k, kind, fx, fy):
    view = S.make_view(k, kind, fx, fy)
    rast = R.Rasterizer()
    cv = L.make_views([view])
    words = torch.empty(12 * 4 ** k // 32, dtype=torch.int32, device="cuda")
    L.check(L.lib().hpxgs_mask_build(cv, ctypes.byref(rast.cfg), _p(words), _s()), "mask")
    torch.cuda.synchronize()
    w = words.cpu().numpy().view(np.uint32)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8).reshape(-1)
    ref, margin = O.mask(2 ** k, kind, fx, fy)
    bad = np.nonzero(bits != ref)[0]
    assert np.all(np.abs(margin[bad]) < 1e-12), (bad[:10], margin[bad[:10]])


@pytest.mark.parametrize("k,kind,fx,fy", [(6, 0, 360, 360), (9, 2, 190, 190), (8, 1, 90, 90), (9, 1, 60, 100),
                                          (7, 2, 220, 180), (10, 2, 180, 180), (4, 2, 200, 200), (9, 1, 120, 100)])
def test_forward_mask_equals_per_pixel_mask(k, kind, fx, fy):
    # the forward builds its own mask in its mask stage (one thread per pixel, an FP64 re-check
    # near the FoV boundary); it must equal the mask of hpxgs_mask_build bit for bit
    import numpy as np
    from tests.gpu_util import scene_tensors
    view = S.make_view(k, kind, fx, fy)
    rast = R.Rasterizer(tile_level=min(4, k))
    cv = L.make_views([view])
    words = torch.empty(12 * 4 ** k // 32, dtype=torch.int32, device="cuda")
    L.check(L.lib().hpxgs_mask_build(cv, ctypes.byref(rast.cfg), _p(words), _s()), "mask")
    sc = S.make_scene(500, 0, seed=7)
    out, _ = rast.forward_raw(*scene_tensors(sc), 0, [view])
    torch.cuda.synchronize()
    assert torch.equal(out["mask"], words)


@pytest.mark.parametrize("k,fx,fy,pp", [(8, 90.0, 70.0, (0.3, -0.45)), (9, 60.0, 100.0, (-0.7, 0.2)),
                                        (7, 120.0, 80.0, (0.9, 0.9))])
def test_off_centre_pinhole_mask_matches_oracle(k, fx, fy, pp):
    # principal point (W/2)(1 + ppx), (H/2)(1 + ppy): an asymmetric frustum; the per-pixel
    # mask equals the oracle's except on the boundary itself, and the forward's mask equals it
    from tests.gpu_util import scene_tensors
    view = S.make_view(k, S.CAM_PINHOLE, fx, fy, pp=pp)
    rast = R.Rasterizer(tile_level=4)
    cv = L.make_views([view])
    words = torch.empty(12 * 4 ** k // 32, dtype=torch.int32, device="cuda")
    L.check(L.lib().hpxgs_mask_build(cv, ctypes.byref(rast.cfg), _p(words), _s()), "mask")
    out, _ = rast.forward_raw(*scene_tensors(S.make_scene(500, 0, seed=8)), 0, [view])
    torch.cuda.synchronize()
    w = words.cpu().numpy().view(np.uint32)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8).reshape(-1)
    ref, margin = O.mask(2 ** k, S.CAM_PINHOLE, fx, fy, pp=pp)
    bad = np.nonzero(bits != ref)[0]
    assert np.all(np.abs(margin[bad]) < 1e-12), (bad[:10], margin[bad[:10]])
    centred, _ = O.mask(2 ** k, S.CAM_PINHOLE, fx, fy)
    assert (bits != centred).sum() > 100                  # the offset moves the frustum
    assert torch.equal(out["mask"], words)


@pytest.mark.parametrize("k,b", [(6, 3), (9, 4), (11, 4), (10, 5)])
def test_tile_rho_matches_oracle(k, b):
    rho = ctypes.c_double()
    L.check(L.lib().hpxgs_tile_rho(k, b, ctypes.byref(rho), _s()), "rho")
    assert rho.value == O.tile_rho(k, b)
