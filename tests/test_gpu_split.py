"""GPU parity of the split-precision tensor-core form (FP16 slices on tcgen05,
FP32 TMEM accumulation, FP64 lambda recurrence, lambda shared across a
thread-block cluster) against the CPU oracle, at the split-form bar:
max |err| / RMS(output) <= 1e-6 per map column."""
import numpy as np
import pytest
import torch

from paper_2208_10154_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-6


def colerr(got, want):
    w = np.asarray(want)
    w = w.reshape(w.shape[0] * w.shape[1], -1)
    g = np.asarray(got).reshape(w.shape)
    num = np.max(np.abs(g - w), axis=1)
    den = np.sqrt(np.mean(np.abs(w) ** 2, axis=1))
    den = np.where(den == 0, 1.0, den)
    return float(np.max(num / den))


@pytest.fixture(scope="module")
def sht():
    from paper_2208_10154_b300 import build, sht as s
    build.build()
    s.load()
    return s


CASES = [
    (32, 64, 64, 16, "inv_lp1_sq"),     # the small spin-0 workload
    (8, 31, 31, 3, "flat"),             # heavy aliasing, odd column count
    (16, 40, 20, 5, "flat"),            # mmax < lmax
    (1, 3, 3, 2, "flat"),               # smallest grid
    (64, 127, 127, 130, "inv_llp1"),    # two column tiles, ragged
    (128, 300, 300, 7, "inv_llp1"),     # several row / pair tiles
    (16, 40, 40, 300, "inv_llp1"),      # 5 column tiles: one cluster of 5 CTAs
    (8, 23, 23, 520, "flat"),           # 9 column tiles: clusters of 5, one padded tile
]


def _cls(kind, lmax):
    if kind == "flat":
        return np.ones(lmax + 1)
    return inputs.cl_inv_lp1_sq(lmax) if kind == "inv_lp1_sq" else inputs.cl_inv_llp1(lmax)


@pytest.mark.parametrize("nside,lmax,mmax,nmaps,cl", CASES)
def test_alm2map_split(orc, sht, nside, lmax, mmax, nmaps, cl):
    a = inputs.gaussian_alm(nside + 3, nmaps, 1, lmax, mmax, cls=_cls(cl, lmax))
    want = orc.alm2map(a, nside, lmax, mmax)
    plan = sht.Plan(nside, lmax, mmax, 0, "split")
    got = plan.alm2map(torch.from_numpy(a).cuda()).cpu().numpy()
    assert colerr(got, want) < TOL


@pytest.mark.parametrize("nside,lmax,mmax,nmaps,cl", CASES)
def test_map2alm_split(orc, sht, nside, lmax, mmax, nmaps, cl):
    a = inputs.gaussian_alm(nside + 4, nmaps, 1, lmax, mmax, cls=_cls(cl, lmax))
    T = orc.alm2map(a, nside, lmax, mmax)
    rng = np.random.default_rng(nside)
    T += 0.01 * np.sqrt(np.mean(T ** 2, axis=-1, keepdims=True)) * rng.standard_normal(T.shape)
    want = orc.map2alm(T, nside, lmax, mmax)
    plan = sht.Plan(nside, lmax, mmax, 0, "split")
    got = plan.map2alm(torch.from_numpy(T).cuda()).cpu().numpy()
    assert colerr(got, want) < TOL


def test_split_adjoints_and_iteration(orc, sht):
    nside, lmax, nmaps = 16, 32, 3
    plan = sht.Plan(nside, lmax, None, 0, "split")
    rng = np.random.default_rng(3)
    h = rng.standard_normal((nmaps, 1, 12 * nside * nside))
    assert colerr(plan.alm2map_adjoint(torch.from_numpy(h).cuda()).cpu().numpy(),
                  orc.alm2map_adjoint(h, nside, lmax)) < TOL
    g = inputs.gaussian_alm(5, nmaps, 1, lmax, cls=np.ones(lmax + 1))
    assert colerr(plan.map2alm_adjoint(torch.from_numpy(g).cuda()).cpu().numpy(),
                  orc.map2alm_adjoint(g, nside, lmax)) < TOL
    assert colerr(plan.map2alm(torch.from_numpy(h).cuda(), niter=2).cpu().numpy(),
                  orc.map2alm(h, nside, lmax, niter=2)) < TOL


@pytest.mark.parametrize("nside,lmax,nmaps", [(128, 300, 300), (64, 160, 1100)])
def test_split_clusters_many_chunks(orc, sht, nside, lmax, nmaps):
    """Several column tiles per cluster and more K chunks than pipeline stages
    (stage reuse across the cluster); the oracle checks a few maps spread over
    the column tiles (map columns are independent)."""
    a = inputs.gaussian_alm(nside + 5, nmaps, 1, lmax, cls=inputs.cl_inv_llp1(lmax))
    plan = sht.Plan(nside, lmax, None, 0, "split")
    pick = [0, nmaps // 2 + 1, nmaps - 1]
    got = plan.alm2map(torch.from_numpy(a).cuda()).cpu().numpy()
    assert colerr(got[pick], orc.alm2map(a[pick], nside, lmax)) < TOL
    rng = np.random.default_rng(nside)
    T = got + 0.01 * np.sqrt(np.mean(got ** 2, axis=-1, keepdims=True)) * rng.standard_normal(got.shape)
    ga = plan.map2alm(torch.from_numpy(T).cuda()).cpu().numpy()
    assert colerr(ga[pick], orc.map2alm(T[pick], nside, lmax)) < TOL
