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
    (96, 200, 200, 6, "inv_llp1"),      # 192 ring pairs: an alm2map CTA walks a full and a 64-row tile
    (560, 100, 100, 3, "flat"),         # 1120 ring pairs: two alm2map groups (8 tiles, then a 96-row tile)
    (128, 255, 180, 3, "inv_llp1"),     # mmax < lmax with polar ring pairs skipped per order (up to 64)
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


@pytest.mark.parametrize("nside,lmax,nmaps", [(128, 300, 300), (64, 160, 1100), (64, 160, 1024)])
def test_split_clusters_many_chunks(orc, sht, nside, lmax, nmaps):
    """Several column tiles per cluster and more K chunks than pipeline stages
    (stage reuse across the cluster); the oracle checks a few maps spread over
    the column tiles (map columns are independent). 1024 maps = 16 column
    tiles: clusters of 8, with the last work items (the highest m) in the
    small-cluster launch that fills the SMs the large clusters leave idle."""
    a = inputs.gaussian_alm(nside + 5, nmaps, 1, lmax, cls=inputs.cl_inv_llp1(lmax))
    plan = sht.Plan(nside, lmax, None, 0, "split")
    pick = [0, nmaps // 2 + 1, nmaps - 1]
    got = plan.alm2map(torch.from_numpy(a).cuda()).cpu().numpy()
    want = orc.alm2map(a[pick], nside, lmax)
    assert colerr(got[pick], want) < TOL
    # map2alm input: GPU maps in the unchecked columns, the oracle's maps in
    # the checked ones (no oracle input comes from the GPU), plus 1% noise
    T = got.copy()
    T[pick] = want
    rng = np.random.default_rng(nside)
    T += 0.01 * np.sqrt(np.mean(T ** 2, axis=-1, keepdims=True)) * rng.standard_normal(T.shape)
    ga = plan.map2alm(torch.from_numpy(T).cuda()).cpu().numpy()
    assert colerr(ga[pick], orc.map2alm(T[pick], nside, lmax)) < TOL


# ---------------------------------------------------------------- spin 2
S2_CASES = [
    (16, 47, 47, 3, 1.0),       # aliasing, lmax = 3 nside - 1
    (32, 64, 64, 4, 0.01),      # E/B spectra of the polarization workload (C_BB = 0.01 C_EE)
    (8, 20, 20, 1, 1.0),
    (1, 3, 3, 2, 1.0),          # smallest grid: only l = 2, 3
    (16, 40, 20, 5, 1.0),       # mmax < lmax
    (64, 127, 127, 70, 0.01),   # 280 columns: three column tiles, ragged
    (128, 300, 300, 5, 0.01),   # several row / pair tiles, K' = 2 x 256 ring pairs
    (8, 23, 23, 130, 1.0),      # 520 columns: clusters of column tiles
    (96, 150, 150, 2, 0.01),    # 192 ring pairs: a full and a 64-row tile in one alm2map CTA
]


def _s2_alm(seed, nmaps, lmax, mmax, bb):
    cl = inputs.cl_inv_llp1(lmax)
    a = inputs.gaussian_alm(seed, nmaps, 2, lmax, mmax, cls=np.stack([cl, bb * cl]))
    ls, _ = inputs.lm_arrays(lmax, mmax)
    a[..., ls < 2] = 0
    return a


@pytest.mark.parametrize("nside,lmax,mmax,nmaps,bb", S2_CASES)
def test_alm2map_split_spin2(orc, sht, nside, lmax, mmax, nmaps, bb):
    a = _s2_alm(nside + 11, nmaps, lmax, mmax, bb)
    want = orc.alm2map(a, nside, lmax, mmax, spin=2)
    plan = sht.Plan(nside, lmax, mmax, 2, "split")
    got = plan.alm2map(torch.from_numpy(a).cuda()).cpu().numpy()
    assert colerr(got, want) < TOL


@pytest.mark.parametrize("nside,lmax,mmax,nmaps,bb", S2_CASES)
def test_map2alm_split_spin2(orc, sht, nside, lmax, mmax, nmaps, bb):
    a = _s2_alm(nside + 12, nmaps, lmax, mmax, bb)
    T = orc.alm2map(a, nside, lmax, mmax, spin=2)
    rng = np.random.default_rng(nside + 1)
    T += 0.01 * np.sqrt(np.mean(T ** 2, axis=-1, keepdims=True)) * rng.standard_normal(T.shape)
    want = orc.map2alm(T, nside, lmax, mmax, spin=2)
    plan = sht.Plan(nside, lmax, mmax, 2, "split")
    got = plan.map2alm(torch.from_numpy(T).cuda()).cpu().numpy()
    assert colerr(got, want) < TOL


def test_split_spin2_adjoints(orc, sht):
    nside, lmax, nmaps = 16, 32, 2
    plan = sht.Plan(nside, lmax, None, 2, "split")
    rng = np.random.default_rng(7)
    h = rng.standard_normal((nmaps, 2, 12 * nside * nside))
    assert colerr(plan.alm2map_adjoint(torch.from_numpy(h).cuda()).cpu().numpy(),
                  orc.alm2map_adjoint(h, nside, lmax, spin=2)) < TOL
    g = _s2_alm(8, nmaps, lmax, lmax, 1.0)
    assert colerr(plan.map2alm_adjoint(torch.from_numpy(g).cuda()).cpu().numpy(),
                  orc.map2alm_adjoint(g, nside, lmax, spin=2)) < TOL


def test_split_spin2_many_chunks(orc, sht):
    """Spin 2 with 1100 Q/U pairs (4400 columns, clusters of column tiles) and
    many K chunks; the oracle checks maps spread over the column tiles."""
    nside, lmax, nmaps = 64, 160, 1100
    a = _s2_alm(21, nmaps, lmax, lmax, 0.01)
    plan = sht.Plan(nside, lmax, None, 2, "split")
    pick = [0, nmaps // 2 + 1, nmaps - 1]
    got = plan.alm2map(torch.from_numpy(a).cuda()).cpu().numpy()
    want = orc.alm2map(a[pick], nside, lmax, spin=2)
    assert colerr(got[pick], want) < TOL
    T = got.copy()
    T[pick] = want
    rng = np.random.default_rng(9)
    T += 0.01 * np.sqrt(np.mean(T ** 2, axis=-1, keepdims=True)) * rng.standard_normal(T.shape)
    ga = plan.map2alm(torch.from_numpy(T).cuda()).cpu().numpy()
    assert colerr(ga[pick], orc.map2alm(T[pick], nside, lmax, spin=2)) < TOL


@pytest.mark.parametrize("nside,lmax,spin,niter", [(16, 47, 0, 3), (16, 47, 2, 2), (64, 127, 0, 2), (32, 63, 2, 1)])
def test_split_iteration(orc, sht, nside, lmax, spin, niter):
    """Fourier-domain iteration in the split form against the oracle's
    pixel-domain Algorithm 2."""
    ncomp = 2 if spin else 1
    rng = np.random.default_rng(31 + nside)
    h = rng.standard_normal((3, ncomp, 12 * nside * nside))
    plan = sht.Plan(nside, lmax, None, spin, "split")
    got = plan.map2alm(torch.from_numpy(h).cuda(), niter=niter).cpu().numpy()
    assert colerr(got, orc.map2alm(h, nside, lmax, spin=spin, niter=niter)) < TOL


@pytest.mark.parametrize("prec,spin", [("split", 0), ("split", 2), ("fp64", 0), ("fp64", 2)])
def test_ring_optimisation_changes_nothing_measurable(sht, monkeypatch, prec, spin):
    """Sec. 3.1 (Implementation detail), the ring optimisation: a spin-0 split
    plan leaves out, per order m, the polar ring pairs where |lambda_lm| <
    1e-30 for every l, in the contraction and in the FFT order mapping. At
    nside 256 / lmax 511 that is about a tenth of the (m, l, ring pair) terms;
    the results match a plan that skips nothing (SHT_RING_SKIP=0) to far below
    the form's own error, for alm2map and for map2alm with the Fourier-domain
    iteration (whose residual folds only the kept orders). The FP64 form
    skips the same leading ring pairs in map2alm and writes zeros for
    alm2map's ring-pair tiles that lie wholly among them."""
    nside, lmax, nmaps = 256, 511, 3
    tol_a, tol_b = (1e-9, 2e-7) if prec == "split" else (1e-12, 1e-12)
    plan = sht.Plan(nside, lmax, None, spin, prec)
    monkeypatch.setenv("SHT_RING_SKIP", "0")
    full = sht.Plan(nside, lmax, None, spin, prec)
    monkeypatch.delenv("SHT_RING_SKIP")
    assert full.terms_kept() == 1.0
    assert 0.5 < plan.terms_kept() < 0.95
    ncomp = 2 if spin else 1
    cls = None
    if spin:
        cl = inputs.cl_inv_llp1(lmax)
        cls = np.stack([cl, 0.01 * cl])
    a = torch.from_numpy(inputs.gaussian_alm(11, nmaps, ncomp, lmax, cls=cls)).cuda()
    m_skip, m_full = plan.alm2map(a), full.alm2map(a)
    assert colerr(m_skip.cpu().numpy(), m_full.cpu().numpy()) < tol_a
    for niter in (0, 2):
        b_skip = plan.map2alm(m_full, niter=niter).cpu().numpy()
        b_full = full.map2alm(m_full, niter=niter).cpu().numpy()
        assert np.all(np.isfinite(b_skip))
        assert colerr(b_skip, b_full) < tol_b
    if spin:                             # one component: half of the contraction
        e_skip = plan.map2alm_eb(m_full, "B").cpu().numpy()
        e_full = full.map2alm_eb(m_full, "B").cpu().numpy()
        assert colerr(e_skip, e_full) < tol_b
    plan.device_status()


@pytest.mark.parametrize("prec,spin,nside", [("split", 0, 128), ("split", 2, 64), ("fp64", 0, 128),
                                             ("fp64", 2, 64), ("split", 0, 256)])
def test_ring_first_pairs_match_the_oracle(orc, sht, prec, spin, nside):
    """The plan's ring-optimisation table (index work: bit-exact) equals the
    oracle's restatement of the rule: per order, the first ring pair where
    some |lambda_lm| (spin 2: of s = +2 or -2) reaches 1e-30, made
    nondecreasing in m, rounded down to 32, 0 for m = 0. The split plan takes
    its maxima from its double-float lambda walk in FP32, the FP64 plan from
    its FP64 walk, the oracle from long double."""
    lmax = 2 * nside - 1
    plan = sht.Plan(nside, lmax, None, spin, prec)
    want = orc.ring_first_pairs(nside, lmax, spin)
    assert want[-1] > 0
    assert np.array_equal(plan.first_pairs(), want)
