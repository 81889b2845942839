"""Pins of the oracle's compact square a_lm storage (Sec. 5, equ:new alm save
scheme) and of its pixel-domain E/B projection (Sec. 2.3, equ:aeab mat form
pixel), against a hand-worked example and structural identities."""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _blocks():
    blocks, cur = [], None
    for line in open(os.path.join(HERE, "golden", "square_storage.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("lmax"):
            cur = (int(line.split()[1]), [])
            blocks.append(cur)
        else:
            cur[1].append(line.split())
    return blocks


def _random_alm(lmax, nmaps=2, seed=0):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((nmaps, oracle.nalm(lmax))) + 1j * rng.standard_normal((nmaps, oracle.nalm(lmax)))
    return a


@pytest.mark.parametrize("blk", range(2))
def test_square_storage_worked_example(blk):
    lmax, rows = _blocks()[blk]
    a = _random_alm(lmax)
    sq = oracle.alm_to_square(a, lmax)
    assert sq.shape == (2, lmax + 1, lmax + 1)
    for r, row in enumerate(rows):
        for c, name in enumerate(row):
            part, l, m = name.split(":")
            v = a[:, oracle.alm_index(lmax, int(l), int(m))]
            want = v.real if part == "Re" else v.imag
            assert np.array_equal(sq[:, r, c], want), (lmax, r, c, name)


@pytest.mark.parametrize("lmax", [0, 1, 6, 17])
def test_square_storage_is_a_bijection(lmax):
    # every element of the square is used exactly once: with all parts of a
    # distinct and non-zero (Im a_l0 is not stored), every cell is non-zero,
    # the stored values are distinct, and the round trip is exact
    a = _random_alm(lmax, nmaps=1, seed=lmax)
    a[..., [oracle.alm_index(lmax, l, 0) for l in range(lmax + 1)]] = \
        a[..., [oracle.alm_index(lmax, l, 0) for l in range(lmax + 1)]].real
    sq = oracle.alm_to_square(a, lmax)
    assert np.all(sq != 0.0)
    assert len(np.unique(sq)) == (lmax + 1) ** 2
    assert np.array_equal(oracle.square_to_alm(sq, lmax), a)


def test_square_storage_mmax_below_lmax():
    lmax, mmax = 9, 4
    rng = np.random.default_rng(3)
    a = rng.standard_normal((1, oracle.nalm(lmax, mmax))) + 1j * rng.standard_normal((1, oracle.nalm(lmax, mmax)))
    for l in range(lmax + 1):
        a[..., oracle.alm_index(lmax, l, 0)] = a[..., oracle.alm_index(lmax, l, 0)].real
    sq = oracle.alm_to_square(a, lmax, mmax)
    assert np.count_nonzero(sq) == 2 * oracle.nalm(lmax, mmax) - (lmax + 1)
    assert np.array_equal(oracle.square_to_alm(sq, lmax, mmax), a)


def _pure_e_map(nside, lmax, seed):
    """Q/U maps of random E-mode coefficients only (l >= 2, Im a_l0 = 0)."""
    rng = np.random.default_rng(seed)
    n = oracle.nalm(lmax)
    a = np.zeros((1, 2, n), dtype=np.complex128)
    a[0, 0] = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for m in range(lmax + 1):
        for l in range(m, lmax + 1):
            i = oracle.alm_index(lmax, l, m)
            if l < 2:
                a[0, 0, i] = 0.0
            elif m == 0:
                a[0, 0, i] = a[0, 0, i].real
    return a, oracle.alm2map(a, nside, lmax, spin=2)


def test_eb_projection_complementary():
    # the E and B parts add up to the band-limited map: lambda^E + lambda^B = I
    nside, lmax = 8, 15
    rng = np.random.default_rng(11)
    maps = rng.standard_normal((2, 2, oracle.npix(nside)))
    pe = oracle.eb_project(maps, nside, lmax, "E", niter=1)
    pb = oracle.eb_project(maps, nside, lmax, "B", niter=1)
    full = oracle.alm2map(oracle.map2alm(maps, nside, lmax, spin=2, niter=1), nside, lmax, spin=2)
    assert np.allclose(pe + pb, full, rtol=0, atol=1e-12 * np.abs(full).max())


def test_eb_projection_idempotent_on_band_limited_maps():
    # a band-limited pure-E map is its own E part and has no B part, up to
    # the quadrature error of map2alm, which the iteration (Algorithm 2) reduces
    nside, lmax = 8, 15
    _, s = _pure_e_map(nside, lmax, 5)
    rms = np.sqrt(np.mean(s ** 2))
    errs = []
    for niter in (0, 3):
        pe = oracle.eb_project(s, nside, lmax, "E", niter=niter)
        pb = oracle.eb_project(s, nside, lmax, "B", niter=niter)
        errs.append((np.abs(pe - s).max() / rms, np.abs(pb).max() / rms))
    assert errs[1][0] < 1e-2 and errs[1][1] < 1e-2
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]
