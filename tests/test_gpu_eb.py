"""GPU parity of the E-only / B-only spin-2 transforms (Sec. 3.1: a pipeline
that needs one of a_E, a_B gets it with half of the Legendre contraction)
against the CPU oracle's full transforms: map2alm_eb must equal the kept
component of the oracle's map2alm, alm2map_eb the oracle's alm2map with the
other component zero. Split form at 1e-6, FP64 at 1e-10 (max |err| / RMS
per map column)."""
import numpy as np
import pytest
import torch

from paper_2208_10154_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"split": 1e-6, "fp64": 1e-10}


def colerr(got, want):
    w = np.asarray(want).reshape(-1, np.asarray(want).shape[-1])
    g = np.asarray(got).reshape(w.shape)
    den = np.sqrt(np.mean(np.abs(w) ** 2, axis=1))
    return float(np.max(np.max(np.abs(g - w), axis=1) / np.where(den == 0, 1.0, den)))


@pytest.fixture(scope="module")
def sht():
    from paper_2208_10154_b300 import build, sht as s
    build.build()
    s.load()
    return s


def _qu(orc, seed, nside, lmax, mmax, nmaps, bb=0.01):
    cl = inputs.cl_inv_llp1(lmax)
    a = inputs.gaussian_alm(seed, nmaps, 2, lmax, mmax, cls=np.stack([cl, bb * cl]))
    ls, _ = inputs.lm_arrays(lmax, mmax)
    a[..., ls < 2] = 0
    T = orc.alm2map(a, nside, lmax, mmax, spin=2)
    rng = np.random.default_rng(seed)
    T += 0.01 * np.sqrt(np.mean(T ** 2, axis=-1, keepdims=True)) * rng.standard_normal(T.shape)
    return a, T


CASES = [
    (16, 47, 47, 3),        # aliasing
    (32, 64, 64, 4),
    (16, 40, 20, 5),        # mmax < lmax
    (64, 127, 127, 70),     # 140 contraction columns: two tiles, ragged
    (8, 23, 23, 130),       # 260 columns: three tiles, a cluster
    (1, 3, 3, 2),           # smallest grid
]


@pytest.mark.parametrize("prec", ["split", "fp64"])
@pytest.mark.parametrize("nside,lmax,mmax,nmaps", CASES)
def test_map2alm_eb_matches_oracle(orc, sht, prec, nside, lmax, mmax, nmaps):
    _, T = _qu(orc, nside + 3, nside, lmax, mmax, nmaps)
    want = orc.map2alm(T, nside, lmax, mmax, spin=2)
    plan = sht.Plan(nside, lmax, mmax, 2, prec)
    x = torch.from_numpy(T).cuda()
    for k, which in enumerate("EB"):
        got = plan.map2alm_eb(x, which).cpu().numpy()
        assert got.shape == (nmaps, 1, want.shape[-1])
        assert colerr(got[:, 0], want[:, k]) < TOL[prec], (which, prec)
    plan.device_status()


@pytest.mark.parametrize("prec", ["split", "fp64"])
def test_alm2map_eb_matches_oracle(orc, sht, prec):
    nside, lmax, nmaps = 32, 64, 3
    a, _ = _qu(orc, 7, nside, lmax, lmax, nmaps)
    plan = sht.Plan(nside, lmax, None, 2, prec)
    for k, which in enumerate("EB"):
        keep = np.zeros_like(a)
        keep[:, k] = a[:, k]
        want = orc.alm2map(keep, nside, lmax, spin=2)
        got = plan.alm2map_eb(torch.from_numpy(np.ascontiguousarray(a[:, k:k + 1])).cuda(), which).cpu().numpy()
        assert colerr(got, want) < TOL[prec], (which, prec)


def test_eb_needs_spin2(sht):
    plan = sht.Plan(8, 15, None, 0, "fp64")
    with pytest.raises(sht.ShtError):
        plan.map2alm_eb(torch.zeros((1, 2, 12 * 64), dtype=torch.float64, device="cuda"), "E")
