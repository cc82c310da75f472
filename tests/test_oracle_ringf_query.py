"""Pins for the oracle's RING query at a finer search resolution (Sec. 3.3 and Sec. D.2:
Algorithm 3 run at query order k_t + log2 f, the query pixels mapped to their tiles).

- the lists equal brute-force membership at the query order: tile t is listed iff it
  is active and one of its 4^log2f query pixels has its centre within
  r_s + rho(k, b - log2 f) + 1e-7 of the Gaussian (every tile and query pixel tested);
- log2 f = 0 gives the tile-order RING lists;
- conservative: every active tile holding a render-pixel centre within r_s of the
  Gaussian is listed, so with the m <= 9 cutoff the image is the RING x1 image value for
  value; finer search lists no more tiles than the tile-order query on these scenes;
- under the literal tile semantics (no cutoff) the image depends on the search resolution.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_29794_b300 import synth as S


def _scene_view(seed, kind=O.CAM_FISHEYE, fov=200.0, k=6):
    rng = np.random.default_rng(seed)
    sc = S.make_scene(400, 3, seed=seed, r_min=1.5, r_max=4.0, logscale_mu=-2.0)
    v = S.random_pose_view(rng, k, kind, fov, fov, 0.3)
    v = dict(v, W=np.asarray(v["W"], np.float64), b=np.asarray(v["b"], np.float64))
    return sc, v


def _csr_sets(start, ids, nt):
    return [set(ids[start[t]:start[t + 1]].tolist()) for t in range(nt)]


@pytest.mark.parametrize("b,log2f", [(3, 1), (3, 2), (3, 3), (4, 2)])
@pytest.mark.parametrize("kind,fov", [(O.CAM_FULL, 360.0), (O.CAM_FISHEYE, 200.0), (O.CAM_PINHOLE, 90.0)])
def test_lists_equal_bruteforce_at_query_order(b, log2f, kind, fov):
    sc, v = _scene_view(b * 10 + log2f + kind, kind, fov)
    k = v["nside_log2"]
    cfg = O.Config(tile_level=b)
    R = O.render(sc, v, cfg)
    pre = R.pre
    dbits = O.depth_bits(pre["r"])
    start, ids = O.tile_lists_ringf(k, b, log2f, pre["g"], pre["rs"], pre["valid"], dbits, R.active)
    nt = R.active.size
    rho_q = 0.0 if log2f == b else O.tile_rho(k, b - log2f)
    # brute force at the query order (every query pixel of every tile), then any over a tile's
    # 4^log2f query pixels; activity of the tile
    act_q = np.repeat(R.active, 4 ** log2f)
    member_q = O.tile_lists_bruteforce(k, b - log2f, pre["g"], pre["rs"], pre["valid"], rho_q, act_q)
    member = member_q.reshape(pre["rs"].size, nt, 4 ** log2f).any(2)
    got = _csr_sets(start, ids, nt)
    want = [set(np.nonzero(member[:, t])[0].tolist()) for t in range(nt)]
    assert got == want
    # each list in depth order (float32 depth bits, then Gaussian index)
    for t in range(nt):
        lst = ids[start[t]:start[t + 1]]
        key = dbits[lst].astype(np.int64) * (1 << 32) + lst
        assert np.all(np.diff(key) > 0)


def test_log2f_zero_is_the_tile_order_query():
    sc, v = _scene_view(5)
    k, b = v["nside_log2"], 3
    R = O.render(sc, v, O.Config(tile_level=b))
    dbits = O.depth_bits(R.pre["r"])
    s0, i0 = O.tile_lists_ringf(k, b, 0, R.pre["g"], R.pre["rs"], R.pre["valid"], dbits, R.active)
    assert np.array_equal(s0, R.start) and np.array_equal(i0, R.ids)


@pytest.mark.parametrize("log2f", [1, 2, 3])
def test_conservative_same_image_under_cutoff_and_fewer_pairs(log2f):
    sc, v = _scene_view(20 + log2f, O.CAM_FULL, 360.0)
    k, b = v["nside_log2"], 3
    cfg = O.Config(tile_level=b)
    R = O.render(sc, v, cfg)
    pre = R.pre
    start, ids = O.tile_lists_ringf(k, b, log2f, pre["g"], pre["rs"], pre["valid"], O.depth_bits(pre["r"]), R.active)
    # every tile holding a render-pixel centre within r_s is listed (brute force at b = 0, radius r_s + 1e-7)
    near = O.tile_lists_bruteforce(k, 0, pre["g"], pre["rs"], pre["valid"], 0.0, np.ones(O.npix(1 << k), np.uint8))
    need = near.reshape(pre["rs"].size, R.active.size, 4 ** b).any(2) & (R.active[None, :] == 1)
    got = _csr_sets(start, ids, R.active.size)
    for t in range(R.active.size):
        assert set(np.nonzero(need[:, t])[0].tolist()) <= got[t]
    img, T, last, amb = O.composite(k, b, pre, sc["opacities"], start, ids, R.pix, cfg)
    assert np.array_equal(img, R.image[R.pix]) and np.array_equal(T, R.T[R.pix])
    assert ids.size <= R.ids.size


def test_literal_semantics_depend_on_the_search_resolution():
    sc, v = _scene_view(31, O.CAM_FULL, 360.0)
    k, b = v["nside_log2"], 3
    cfg = O.Config(tile_level=b, cutoff=math.inf)
    R = O.render(sc, v, cfg)
    pre = R.pre
    s2, i2 = O.tile_lists_ringf(k, b, 2, pre["g"], pre["rs"], pre["valid"], O.depth_bits(pre["r"]), R.active)
    img, *_ = O.composite(k, b, pre, sc["opacities"], s2, i2, R.pix, cfg)
    assert np.abs(img - R.image[R.pix]).max() > 1e-6


@pytest.mark.parametrize("log2f", [0, 2])
def test_centres_off_unit_length_are_enumerated(log2f):
    # a stored centre is unit length only to its rounding (float32 records: |g| - 1 ~ 1e-7); the
    # membership test c . g >= cos(R) then reaches slightly beyond R, by about (|g| - 1) / tan R,
    # which is large against R for small discs. Algorithm 3's enumeration must cover that disc:
    # the lists still equal brute force over every query pixel.
    rng = np.random.default_rng(7 + log2f)
    k, b = 8, 2
    n = 300
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    g *= (1.0 + rng.choice([-3e-7, 3e-7], n))[:, None]
    rs = 10.0 ** rng.uniform(-4.5, -1.5, n)
    valid = np.ones(n, np.int32)
    act = np.ones(12 * 4 ** (k - b), np.uint8)
    dbits = np.arange(n, dtype=np.uint32) + np.uint32(0x40000000)
    start, ids = O.tile_lists_ringf(k, b, log2f, g, rs, valid, dbits, act)
    nt = act.size
    rho_q = 0.0 if log2f == b else O.tile_rho(k, b - log2f)
    member_q = O.tile_lists_bruteforce(k, b - log2f, g, rs, valid, rho_q, np.repeat(act, 4 ** log2f))
    member = member_q.reshape(n, nt, 4 ** log2f).any(2)
    assert _csr_sets(start, ids, nt) == [set(np.nonzero(member[:, t])[0].tolist()) for t in range(nt)]
