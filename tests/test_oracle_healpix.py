"""Pins for the oracle's HEALPix geometry (Sec. 3.1; Gorski et al. 2005).

Each test checks the oracle against a fact that does not come from the oracle's
own formulas: pixel counts, equal area by Monte Carlo, the inverse map being an
inverse, two independent derivations of pixel centres (NESTED ring formulas vs
the RING scheme), ring structure, the Euler-characteristic count of 7-neighbour
pixels, and hand-checked values at Nside = 1.
"""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 32, 128, 512])
def test_inverse_and_ring_roundtrip(nside):
    p = np.arange(O.npix(nside), dtype=np.int64)
    th, ph = O.pix2ang_nest(nside, p)
    assert np.array_equal(O.ang2pix_nest(nside, th, ph), p)
    v = O.pix2vec_nest(nside, p)
    assert np.array_equal(O.vec2pix_nest(nside, v), p)
    r = O.nest2ring(nside, p)
    assert np.array_equal(np.sort(r), p)          # a permutation of 0..Npix-1
    assert np.array_equal(O.ring2nest(nside, r), p)


@pytest.mark.parametrize("nside", [1, 4, 16, 64])
def test_nested_centres_equal_ring_scheme_centres(nside):
    # NESTED centres (face coordinates -> ring formulas) against RING-scheme centres
    # (ring index -> latitude and longitude): two independent derivations.
    p = np.arange(O.npix(nside), dtype=np.int64)
    th_n, ph_n = O.pix2ang_nest(nside, p)
    th_r, ph_r = O.pix2ang_ring(nside, O.nest2ring(nside, p))
    assert np.allclose(th_n, th_r, atol=1e-13)
    dphi = np.angle(np.exp(1j * (ph_n - ph_r)))
    assert np.allclose(dphi, 0, atol=1e-12)


@pytest.mark.parametrize("nside", [2, 8, 32])
def test_ring_structure(nside):
    # 4N-1 iso-latitude rings; ring i holds 4 min(i, N, 4N-i) pixels at equal z,
    # equally spaced in longitude; rings are ordered north to south.
    pr = np.arange(O.npix(nside), dtype=np.int64)
    th, ph = O.pix2ang_ring(nside, pr)
    z = np.round(np.cos(th), 12)
    zs, counts = np.unique(z, return_counts=True)
    assert zs.size == 4 * nside - 1
    rings = np.arange(1, 4 * nside)
    expect = 4 * np.minimum(np.minimum(rings, nside), 4 * nside - rings)
    assert np.array_equal(counts[::-1], expect)
    start = 0
    for n in expect:
        seg = ph[start:start + n]
        assert np.allclose(np.diff(seg), 2 * np.pi / n, atol=1e-12)
        start += n
    assert np.all(np.diff(z) <= 0)


def test_nside1_face_centres():
    # Base faces: north faces at z = 2/3, longitudes pi/4 + f pi/2; equatorial faces
    # at z = 0, longitudes f pi/2; south faces at z = -2/3 (Gorski et al. 2005).
    th, ph = O.pix2ang_nest(1, np.arange(12))
    z = np.cos(th)
    assert np.allclose(z[:4], 2 / 3) and np.allclose(z[4:8], 0, atol=1e-15) and np.allclose(z[8:], -2 / 3)
    f = np.arange(4)
    assert np.allclose(ph[:4], np.pi / 4 + f * np.pi / 2)
    assert np.allclose(ph[4:8], f * np.pi / 2)
    assert np.allclose(ph[8:], np.pi / 4 + f * np.pi / 2)


def test_equal_area_monte_carlo():
    # N_pix = 12 Nside^2 pixels of equal solid angle 4 pi / N_pix (Sec. 3.1):
    # uniform directions fall into pixels with equal probability (chi-square).
    rng = np.random.default_rng(0)
    nside, n = 4, 2_000_000
    v = rng.standard_normal((n, 3))
    p = O.vec2pix_nest(nside, v)
    counts = np.bincount(p, minlength=O.npix(nside))
    assert counts.size == 192
    e = n / 192
    chi2 = ((counts - e) ** 2 / e).sum()
    # chi-square with 191 dof: P(chi2 > 265) ~ 3e-4
    assert chi2 < 265, chi2


def test_pixel_contains_its_samples():
    rng = np.random.default_rng(1)
    nside = 16
    v = rng.standard_normal((20000, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    p = O.vec2pix_nest(nside, v)
    c = O.pix2vec_nest(nside, p)
    ang = np.arccos(np.clip((v * c).sum(1), -1, 1))
    assert ang.max() < 1.5 * np.sqrt(4 * np.pi / O.npix(nside))


@pytest.mark.parametrize("nside", [2, 4, 16, 64])
def test_neighbours(nside):
    p = np.arange(O.npix(nside), dtype=np.int64)
    nb, cnt = O.neighbours_nest(nside, p)
    # 8 neighbours everywhere except the 24 corner pixels at the 8 valence-3 vertices
    # (Euler: V - E + F = 2 with F = 12, E = 24 -> 14 vertices, valence sum 48).
    assert set(np.unique(cnt)) <= {7, 8}
    assert (cnt == 7).sum() == 24
    pairs = set()
    for a in range(p.size):
        for q in nb[a]:
            if q >= 0:
                pairs.add((a, int(q)))
    assert all((q, a) in pairs for (a, q) in pairs)
    c = O.pix2vec_nest(nside, p)
    size = np.sqrt(4 * np.pi / O.npix(nside))
    for a in range(0, p.size, max(1, p.size // 500)):
        qs = nb[a][nb[a] >= 0]
        ang = np.arccos(np.clip(c[qs] @ c[a], -1, 1))
        assert ang.max() < 2.5 * size


def test_corner_pixels_sit_at_valence3_vertices():
    nside = 8
    p = np.arange(O.npix(nside), dtype=np.int64)
    _, cnt = O.neighbours_nest(nside, p)
    v = O.pix2vec_nest(nside, p[cnt == 7])
    z = v[:, 2]
    assert np.all(np.abs(np.abs(z) - 2 / 3) < 0.2)
    assert (z > 0).sum() == 12
