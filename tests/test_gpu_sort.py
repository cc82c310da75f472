"""The depth order of the tile lists (Algorithm 1) under ties and ragged sort tiles, the
tile query's membership decisions next to the threshold, and the bounded grid barrier of
the count scan's cooperative launch.

- Tile lists from scenes whose Gaussians share centres (bit-identical depth keys) at
  sizes that end on, just past and well inside a 4096-element sort tile: every list
  equals the oracle's exactly, i.e. increasing depth bits, then Gaussian index.
- Every tile list of the training-step workload (Nside 512, fisheye 190 deg, 300k
  Gaussians, order-4 tiles) equals the oracle's, built from the GPU's FP32 centres and
  radii. The FP32 test leaves to FP64 the candidates within about 2e-6 rad of the
  threshold; the test checks that the workload has a few hundred (Gaussian, tile) pairs
  within 1e-6 rad of it, so that both the FP32 bounds and the FP64 test are exercised.
- The grid barrier: every block passes when all arrive; when an arrival is missing
  every block gives up within its limit, HPXGS_F_TIMEOUT is set, and the context
  stays usable (a render afterwards is unchanged).
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import _lib as L
from paper_2606_29794_b300 import raster as R
from paper_2606_29794_b300 import synth as S
from tests.gpu_util import gpu_render, mask_from_words

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]


def _tie_scene(P, distinct, seed):
    sc = S.make_scene(P, 0, seed=seed)
    rng = np.random.default_rng(seed)
    src = rng.integers(0, distinct, P)
    for key in ("means", "scales", "rotations"):
        sc[key] = np.ascontiguousarray(sc[key][src])   # shared centres: equal depth keys
    return sc


@pytest.mark.parametrize("P", [100, 4096, 4097, 13000])
def test_depth_ties_and_ragged_sort_tiles(P):
    k, b = 6, 3
    sc = _tie_scene(P, max(7, P // 9), seed=P)
    view = S.make_view(k, S.CAM_FISHEYE, 200.0)
    rast = R.Rasterizer(tile_level=b)
    _, out, state = gpu_render(sc, [view], rast)
    wv = R.workspace_view(rast, state)
    rec = R.device_array(wv.records, P * 16, torch.float32).view(P, 16).cpu().numpy().astype(np.float64)
    radii = R.device_array(wv.radii, P, torch.float32).cpu().numpy()
    depth = R.device_array(wv.depth, P, torch.float32).cpu().numpy()
    valid = radii > 0
    dbits = depth.astype(np.float32).view(np.uint32).copy()
    dbits[~valid] = 0xFFFFFFFF
    assert np.unique(dbits[valid]).size < valid.sum()          # the scene has ties
    m = mask_from_words(out["mask"].cpu().numpy().view(np.uint32), O.npix(2 ** k))
    act = O.active_tiles(k, b, m)
    start, ids_ref = O.tile_lists(k, b, rec[:, 0:3], radii.astype(np.float64), valid.astype(np.int32), dbits,
                                  O.tile_rho(k, b), act)
    n = int(R.device_array(wv.n_pairs, 1, torch.int32).item())
    ids = R.device_array(wv.pair_ids, n, torch.int32).cpu().numpy().astype(np.int64)
    nt = act.size
    rng = R.device_array(wv.ranges, 2 * nt, torch.int32).view(nt, 2).cpu().numpy().astype(np.int64)
    assert n == ids_ref.size
    for t in np.nonzero(act)[0]:
        got = ids[rng[t, 0]:rng[t, 1]] if rng[t, 1] > rng[t, 0] else np.zeros(0, np.int64)
        assert np.array_equal(got, ids_ref[start[t]:start[t + 1]]), t


def test_all_lists_training_workload_near_threshold():
    from scipy.spatial import cKDTree
    k, b, P = 9, 4, 300_000
    sc = S.make_scene(P, 3, seed=20261205)
    view = S.make_view(k, S.CAM_FISHEYE, 190.0)
    rast = R.Rasterizer(tile_level=b)
    _, out, state = gpu_render(sc, [view], rast)
    wv = R.workspace_view(rast, state)
    g = R.device_array(wv.records, P * 16, torch.float32).view(P, 16)[:, 0:3].cpu().numpy().astype(np.float64)
    radii = R.device_array(wv.radii, P, torch.float32).cpu().numpy()
    depth = R.device_array(wv.depth, P, torch.float32).cpu().numpy()
    valid = radii > 0
    dbits = depth.astype(np.float32).view(np.uint32).copy()
    dbits[~valid] = 0xFFFFFFFF
    m = mask_from_words(out["mask"].cpu().numpy().view(np.uint32), O.npix(2 ** k))
    act = O.active_tiles(k, b, m)
    rho = O.tile_rho(k, b)
    start, ids_ref = O.tile_lists(k, b, g, radii.astype(np.float64), valid.astype(np.int32), dbits, rho, act)
    n = int(R.device_array(wv.n_pairs, 1, torch.int32).item())
    assert n == ids_ref.size
    ids = R.device_array(wv.pair_ids, n, torch.int32).cpu().numpy().astype(np.int64)
    assert np.array_equal(ids, ids_ref)
    nt = act.size
    rng = R.device_array(wv.ranges, 2 * nt, torch.int32).view(nt, 2).cpu().numpy().astype(np.int64)
    lens = np.where(rng[:, 1] > rng[:, 0], rng[:, 1] - rng[:, 0], 0)
    assert np.array_equal(lens, np.diff(start))
    full = lens > 0
    assert np.array_equal(rng[full, 0], start[:-1][full])
    # (Gaussian, tile centre) pairs within 1e-6 rad of the threshold r_s + rho + 1e-7
    tree = cKDTree(O.pix2vec_nest(2 ** (k - b), np.arange(nt)))
    gv = g[valid] / np.linalg.norm(g[valid], axis=1)[:, None]
    R_ = np.minimum(np.pi, radii[valid].astype(np.float64) + rho + 1e-7)
    chord = lambda a: 2 * np.sin(np.clip(a, 0, np.pi) / 2)
    near = (tree.query_ball_point(gv, chord(R_ + 1e-6), return_length=True)
            - tree.query_ball_point(gv, chord(R_ - 1e-6), return_length=True))
    assert near.sum() > 200, near.sum()


def _probe(blocks, missing, limit_ns):
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    passed = torch.full((blocks,), 7, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    L.check(L.lib().hpxgs_probe_grid_barrier(blocks, missing, limit_ns, p(counter), p(passed), p(status),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "probe")
    torch.cuda.synchronize()
    return int(counter.item()), passed.cpu().numpy(), int(status.item())


def test_grid_barrier_passes_when_all_arrive():
    for blocks in (1, 148, 296):
        cnt, passed, st = _probe(blocks, 0, 200_000_000)
        assert cnt == blocks and np.all(passed == 1) and st == 0


def test_grid_barrier_wait_runs_out_and_context_survives():
    sc, view = S.make_scene(2000, 0, seed=3), S.make_view(6, S.CAM_FISHEYE, 190.0)
    rast = R.Rasterizer(tile_level=3)
    _, before, _ = gpu_render(sc, [view], rast)
    maps0 = before["maps"].clone()
    cnt, passed, st = _probe(64, 1, 20_000_000)             # one arrival that never comes: 20 ms limit
    assert cnt == 64 and np.all(passed == 0)
    assert st == 2                                         # HPXGS_F_TIMEOUT
    assert L.lib().hpxgs_status_error(st) == -3            # HPXGS_E_TIMEOUT
    _, after, _ = gpu_render(sc, [view], rast)
    assert torch.equal(after["maps"], maps0)


def test_grid_barrier_probe_checks_arguments():
    z = ctypes.c_void_p(0)
    s = ctypes.c_void_p(0)
    t = torch.zeros(4, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    assert L.lib().hpxgs_probe_grid_barrier(0, 0, 1000, p, p, p, s) == -1
    assert L.lib().hpxgs_probe_grid_barrier(1, -1, 1000, p, p, p, s) == -1
    assert L.lib().hpxgs_probe_grid_barrier(1, 0, 3_000_000_000, p, p, p, s) == -1
    assert L.lib().hpxgs_probe_grid_barrier(1, 0, 1000, z, p, p, s) == -1
    assert L.lib().hpxgs_probe_grid_barrier(10 ** 6, 0, 1000, p, p, p, s) == -1
