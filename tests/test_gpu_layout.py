"""GPU parity of the compact square a_lm storage (Sec. 5, equ:new alm save
scheme: bit-exact element copies) and of the pixel-domain E/B projection
(Sec. 2.3, equ:aeab mat form pixel: 1e-10 FP64, 1e-6 split) against the CPU
oracle. Every call goes through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2208_10154_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    from paper_2208_10154_b300 import build, sht as s
    build.build()
    s.load()
    return s


def colerr(got, want):
    w = np.asarray(want)
    w = w.reshape(w.shape[0] * w.shape[1], -1)
    g = np.asarray(got).reshape(w.shape)
    den = np.sqrt(np.mean(np.abs(w) ** 2, axis=1))
    return float(np.max(np.max(np.abs(g - w), axis=1) / np.where(den == 0, 1.0, den)))


@pytest.mark.parametrize("nside,lmax,mmax,spin,nmaps", [
    (16, 20, 20, 0, 3), (16, 31, 31, 2, 2), (8, 17, 9, 0, 4), (4, 0, 0, 0, 1), (64, 140, 140, 0, 5)])
def test_square_storage_bit_exact(orc, sht, nside, lmax, mmax, spin, nmaps):
    ncomp = 2 if spin else 1
    a = inputs.gaussian_alm(lmax + nmaps, nmaps, ncomp, lmax, mmax, cls=np.ones(lmax + 1))
    plan = sht.Plan(nside, lmax, mmax, spin, "fp64")
    at = torch.from_numpy(a).cuda()
    sq = plan.alm_to_square(at)
    torch.cuda.synchronize()
    want = orc.alm_to_square(a, lmax, mmax)
    assert np.array_equal(sq.cpu().numpy(), want)
    back = plan.square_to_alm(sq)
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy(), orc.square_to_alm(want, lmax, mmax))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("split", 1e-6)])
@pytest.mark.parametrize("which", ["E", "B"])
@pytest.mark.parametrize("niter", [0, 2])
def test_eb_projection_matches_oracle(orc, sht, precision, tol, which, niter):
    nside, lmax, nmaps = 16, 31, 3
    rng = np.random.default_rng(7)
    maps = rng.standard_normal((nmaps, 2, orc.npix(nside)))
    plan = sht.Plan(nside, lmax, None, 2, precision)
    got = plan.eb_project(torch.from_numpy(maps).cuda(), which, niter)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    want = orc.eb_project(maps, nside, lmax, which, niter)
    assert colerr(got.cpu().numpy(), want) <= tol


def test_eb_projection_needs_spin2(sht):
    plan = sht.Plan(8, 15, None, 0, "fp64")
    with pytest.raises(Exception):
        plan.eb_project(torch.zeros((1, 1, 12 * 64), dtype=torch.float64, device="cuda"))


def test_plan_device_bytes_counts_tables_and_host_staging(sht):
    """sht_plan_device_bytes (HBM admission): the split plan's FP64
    checkpoints make it larger than the FP64 plan, and the host-buffer entry
    points' device buffers are added once used."""
    import numpy as np
    p64 = sht.Plan(32, 63, None, 0, "fp64")
    psp = sht.Plan(32, 63, None, 0, "split")
    b64, bsp = p64.device_bytes(), psp.device_bytes()
    assert 0 < b64 < bsp
    a = np.zeros((2, 1, p64.nalm), dtype=np.complex128)
    p64.alm2map_host(a)
    assert p64.device_bytes() > b64
