"""GPU parity of the RING query at a finer search resolution (Sec. 3.3, Sec. D.2:
Algorithm 3 at query order k_t + log2 f) against the FP64 oracle.

- the query-order bounds rho(k, b - log2 f) and rho(k_t + log2 f, log2 f) equal the
  oracle's;
- lists: rebuilt by the oracle's RING x f query (O.tile_lists_ringf) from the GPU's
  stored FP32 values (g, r_s, depth), compared exactly, for f = 2, 4, 8 and three
  cameras, and at the training-step workload (Nside 512 fisheye 190 deg, 300k SH3);
- every RING x f list holds every tile the m <= 9 ellipse can reach, so the maps and T
  of RING x f and RING x 1 are equal bit for bit, and their gradients agree to rounding.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import _lib as L
from paper_2606_29794_b300 import raster as R
from paper_2606_29794_b300 import synth as S
from tests.gpu_util import mask_from_words, scene_tensors

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]


def _lists_exact(sc, view, rast, out, state, log2f):
    P = sc["means"].shape[0]
    k, b = view["nside_log2"], rast.tile_level
    wv = R.workspace_view(rast, state)
    rec = R.device_array(wv.records, P * 16, torch.float32).view(P, 16).cpu().numpy().astype(np.float64)
    radii = R.device_array(wv.radii, P, torch.float32).cpu().numpy()
    depth = R.device_array(wv.depth, P, torch.float32).cpu().numpy()
    nt = 12 * 4 ** (k - b)
    n = int(R.device_array(wv.n_pairs, 1, torch.int32).item())
    ids = R.device_array(wv.pair_ids, n, torch.int32).cpu().numpy().astype(np.int64)
    rng = R.device_array(wv.ranges, 2 * nt, torch.int32).view(nt, 2).cpu().numpy().astype(np.int64)
    m = mask_from_words(out["mask"].cpu().numpy().view(np.uint32), O.npix(2 ** k))
    act = O.active_tiles(k, b, m)
    valid = radii > 0
    dbits = depth.astype(np.float32).view(np.uint32).copy()
    dbits[~valid] = 0xFFFFFFFF
    st, ref = O.tile_lists_ringf(k, b, log2f, rec[:, 0:3], radii.astype(np.float64), valid.astype(np.int32), dbits,
                                 act)
    assert ids.size == ref.size, (ids.size, ref.size)
    for t in np.nonzero(act)[0]:
        a = ids[rng[t, 0]:rng[t, 1]] if rng[t, 1] > rng[t, 0] else np.zeros(0, np.int64)
        assert np.array_equal(a, ref[st[t]:st[t + 1]]), (t, a[:8], ref[st[t]:st[t] + 8])
    return n


@pytest.mark.parametrize("k,b,log2f", [(7, 4, 1), (7, 4, 2), (7, 3, 3), (9, 5, 2), (8, 4, 4 - 1)])
def test_query_order_rho_equals_oracle(k, b, log2f):
    got = ctypes.c_double()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for kk, bb in ((k, b - log2f), (k - b + log2f, log2f)):
        if bb == 0:
            continue
        L.check(L.lib().hpxgs_tile_rho(kk, bb, ctypes.byref(got), s), "tile rho")
        assert got.value == O.tile_rho(kk, bb), (kk, bb, got.value, O.tile_rho(kk, bb))


CASES = [("fisheye200_b3", lambda: (S.make_scene(3000, 3, seed=51), S.make_view(7, S.CAM_FISHEYE, 200.0)), 3),
         ("pinhole_b4", lambda: (S.make_scene(3000, 3, seed=52),
                                 S.random_pose_view(np.random.default_rng(5), 8, S.CAM_PINHOLE, 90.0, 70.0)), 4),
         ("full_b4", lambda: (S.make_scene(2500, 0, seed=53, logscale_mu=-2.0), S.make_view(7)), 4)]


@pytest.mark.parametrize("log2f", [1, 2, 3])
@pytest.mark.parametrize("name,make,b", CASES, ids=[c[0] for c in CASES])
def test_ringf_lists_exact_and_maps_equal_ring(name, make, b, log2f):
    sc, view = make()
    ts = scene_tensors(sc)
    rf = R.Rasterizer(tile_level=b, query=L.QUERY_RING, query_log2f=log2f)
    out_f, st_f = rf.forward_raw(*ts, sc["sh_degree"], [view])
    torch.cuda.synchronize()
    n_f = _lists_exact(sc, view, rf, out_f, st_f, log2f)
    ring = R.Rasterizer(tile_level=b)
    out_r, st_r = ring.forward_raw(*ts, sc["sh_degree"], [view])
    torch.cuda.synchronize()
    assert torch.equal(out_f["maps"], out_r["maps"]) and torch.equal(out_f["T"], out_r["T"])
    gen = torch.Generator(device="cuda").manual_seed(8)
    g = torch.randn(out_r["maps"].shape, device="cuda", generator=gen)
    gf = rf.backward_raw(st_f, g)
    gr = ring.backward_raw(st_r, g)
    torch.cuda.synchronize()
    for a, c in zip(gf, gr):
        assert float((a - c).norm() / c.norm()) <= 1e-5
        assert float((a - c).abs().max()) <= 1e-4 * float(c.abs().max())


@pytest.mark.parametrize("b,log2f", [(4, 2), (5, 2)])
def test_training_step_workload_ringf(b, log2f):
    sc = S.make_scene(300_000, 3, seed=20261205)
    view = S.make_view(9, S.CAM_FISHEYE, 190.0)
    ts = scene_tensors(sc)
    rf = R.Rasterizer(tile_level=b, query=L.QUERY_RING, query_log2f=log2f)
    out_f, st_f = rf.forward_raw(*ts, 3, [view])
    ring = R.Rasterizer(tile_level=b)
    out_r, _ = ring.forward_raw(*ts, 3, [view])
    torch.cuda.synchronize()
    assert torch.equal(out_f["maps"], out_r["maps"]) and torch.equal(out_f["T"], out_r["T"])
    _lists_exact(sc, view, rf, out_f, st_f, log2f)
