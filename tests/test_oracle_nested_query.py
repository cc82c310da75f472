"""Pins for the oracle's NESTED quadtree tile query (Algorithm 2; Sec. 3.3).

- PixRad(o) bounds the angle from every node centre to every pixel centre inside
  the node (checked three orders down) and to its corners;
- conservative: every tile holding a pixel centre within r_s of the disc centre
  is listed, for refinements 1, 2, 4;
- tight: every listed tile has a descendant at the refinement order whose centre
  lies within r_s + PixRad of the disc centre;
- the depth-first search equals a non-recursive statement of the same rule over
  all nodes (which nodes are reached, which add their tile);
- with the m <= 9 cutoff, compositing over the NESTED lists gives the same image,
  value for value, as over the RING lists.
"""
import numpy as np
import pytest

import oracle as O
from paper_2606_29794_b300 import synth as S


def _unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _ang(a, b):
    c = np.cross(a, b)
    return np.arctan2(np.linalg.norm(c, axis=-1), (a * b).sum(-1))


@pytest.mark.parametrize("o", [0, 1, 2, 3, 4])
def test_pixrad_bounds_descendants_and_corners(o):
    nside = 1 << o
    n = 12 * nside * nside
    ctr = O.pix2vec_nest(nside, np.arange(n))
    sub = 3
    kids = O.pix2vec_nest(nside << sub, np.arange(n * 4 ** sub)).reshape(n, 4 ** sub, 3)
    far = _ang(ctr[:, None, :], kids).max()
    corners = O.pixel_corners_nest(nside, np.arange(n)).reshape(n, 4, 3)
    far_c = _ang(ctr[:, None, :], corners).max()
    r = O.pixrad(o)
    assert far <= r and far_c <= r
    assert r < far_c * 1.05 + 2 ** -19                     # not loose either
    assert r * 2 ** 20 == np.round(r * 2 ** 20)


def _tiles_needed(kt, b, g, rs):
    k = kt + b
    pix = O.pix2vec_nest(1 << k, np.arange(12 * 4 ** k))
    near = np.nonzero(_ang(pix, g[None, :]) <= rs)[0]
    return set((near >> (2 * b)).tolist())


@pytest.mark.parametrize("log2f", [0, 1, 2])
def test_conservative_and_tight(log2f):
    rng = np.random.default_rng(log2f)
    kt, b = 3, 3
    kmax = kt + log2f
    g = _unit(rng, 40)
    g[:3] = [[0, 0, 1], [0, 0, -1], [1, 0, 0]]
    rs = np.exp(rng.uniform(np.log(0.01), np.log(0.8), 40))
    kid_ctr = O.pix2vec_nest(1 << kmax, np.arange(12 * 4 ** kmax))
    for gi, ri in zip(g, rs):
        t = O.query_disc_nested(kt, log2f, gi, ri)
        assert np.all(np.diff(t) > 0)
        assert _tiles_needed(kt, b, gi, ri) <= set(t.tolist())
        # each listed tile has a descendant at k_max within r_s + PixRad(k_max)
        d = _ang(kid_ctr, gi[None, :]).reshape(12 * 4 ** kt, 4 ** log2f)
        assert np.all(d[t].min(1) <= ri + O.pixrad(kmax) + 1e-12)


def test_dfs_equals_nonrecursive_rule():
    rng = np.random.default_rng(5)
    kt, log2f = 2, 2
    kmax = kt + log2f
    for gi, ri in zip(_unit(rng, 25), np.exp(rng.uniform(np.log(0.02), np.log(1.0), 25))):
        lon, lat = np.arctan2(gi[1], gi[0]), np.arctan2(gi[2], np.hypot(gi[0], gi[1]))
        added = set()
        reached = np.ones(12, bool)                        # base nodes
        for o in range(kmax + 1):
            th, ph = O.pix2ang_nest(1 << o, np.arange(12 * 4 ** o))
            latn = np.pi / 2 - th
            h = np.sin(0.5 * (latn - lat)) ** 2 + np.cos(lat) * np.cos(latn) * np.sin(0.5 * (ph - lon)) ** 2
            d = 2 * np.arcsin(np.minimum(1.0, np.sqrt(h)))
            pr = O.pixrad(o)
            zone = np.where(d > ri + pr, 0, np.where(d + pr <= ri, 3, np.where(d <= ri, 2, 1)))
            stop = (zone >= 2) & (o >= kt)
            add = reached & (zone >= 1) & (stop | (o == kmax))
            added |= set((np.nonzero(add)[0] >> (2 * (o - kt))).tolist()) if o >= kt else set()
            go = reached & (zone >= 1) & ~stop & (o < kmax)
            reached = np.repeat(go, 4)                     # children 4p + c
        assert sorted(added) == O.query_disc_nested(kt, log2f, gi, ri).tolist()


@pytest.mark.parametrize("log2f", [1, 2])
def test_same_image_as_ring_lists(log2f):
    sc = S.make_scene(1500, 3, seed=31)
    view = S.make_view(6, S.CAM_FISHEYE, 200.0)
    view = dict(view, W=np.asarray(view["W"], np.float64), b=np.asarray(view["b"], np.float64))
    cfg = O.Config(tile_level=3)
    full = O.render(sc, view, cfg)
    k, b = 6, 3
    st, ids = O.tile_lists_nested(k, b, log2f, full.pre["g"], full.pre["rs"], full.pre["valid"],
                                  O.depth_bits(full.pre["r"]), full.active)
    img, T, last, amb = O.composite(k, b, full.pre, sc["opacities"], st, ids, full.pix, cfg)
    assert np.array_equal(img, full.image[full.pix]) and np.array_equal(T, full.T[full.pix])
    # and the per-disc queries, filtered by active tiles, make up the lists
    for i in np.nonzero(full.pre["valid"])[0][:50]:
        t = O.query_disc_nested(k - b, log2f, full.pre["g"][i], full.pre["rs"][i])
        t = t[full.active[t] == 1]
        listed = [tt for tt in range(st.size - 1) if i in set(ids[st[tt]:st[tt + 1]].tolist())]
        assert listed == t.tolist()
