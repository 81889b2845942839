"""GPU parity of the FP64 form against the CPU oracle (tolerance 1e-10 of the
output RMS per map column, the FP64 bar). Every call goes through the C ABI."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2208_10154_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def colerr(got, want):
    """max over (map, comp) columns of max|got - want| / RMS(want)."""
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


def make_alm(nside, lmax, mmax, spin, nmaps, seed):
    ncomp = 2 if spin else 1
    a = inputs.gaussian_alm(seed, nmaps, ncomp, lmax, mmax, cls=np.ones(lmax + 1))
    if spin:
        ls, _ = inputs.lm_arrays(lmax, mmax)
        a[..., ls < 2] = 0
    return a


CASES = [
    (32, 64, 64, 0, 16),     # 12288 pixels, the small spin-0 workload
    (8, 31, 31, 0, 3),       # lmax = 4 nside - 1: heavy aliasing on cap rings
    (16, 40, 20, 0, 5),      # mmax < lmax
    (1, 3, 3, 0, 2),         # smallest grid (rings of 4 pixels only)
    (4, 0, 0, 0, 1),         # monopole only
    (64, 140, 140, 0, 37),   # several row / pair / column tiles, ragged tails
    (16, 47, 47, 2, 3),      # spin 2 with aliasing
    (32, 64, 64, 2, 4),
    (8, 20, 20, 2, 1),
]


@pytest.mark.parametrize("nside,lmax,mmax,spin,nmaps", CASES)
def test_alm2map_fp64(orc, sht, nside, lmax, mmax, spin, nmaps):
    a = make_alm(nside, lmax, mmax, spin, nmaps, seed=nside + lmax)
    want = orc.alm2map(a, nside, lmax, mmax, spin)
    plan = sht.Plan(nside, lmax, mmax, spin, "fp64")
    got = plan.alm2map(torch.from_numpy(a).cuda()).cpu().numpy()
    assert colerr(got, want) < TOL


@pytest.mark.parametrize("nside,lmax,mmax,spin,nmaps", CASES)
def test_map2alm_fp64(orc, sht, nside, lmax, mmax, spin, nmaps):
    ncomp = 2 if spin else 1
    rng = np.random.default_rng(nside * 7 + lmax)
    T = rng.standard_normal((nmaps, ncomp, 12 * nside * nside))
    want = orc.map2alm(T, nside, lmax, mmax, spin)
    plan = sht.Plan(nside, lmax, mmax, spin, "fp64")
    got = plan.map2alm(torch.from_numpy(T).cuda()).cpu().numpy()
    assert colerr(got, want) < TOL


@pytest.mark.parametrize("spin", [0, 2])
def test_adjoints_fp64(orc, sht, spin):
    nside, lmax, nmaps = 16, 40, 3
    ncomp = 2 if spin else 1
    plan = sht.Plan(nside, lmax, None, spin, "fp64")
    rng = np.random.default_rng(3)
    h = rng.standard_normal((nmaps, ncomp, 12 * nside * nside))
    want = orc.alm2map_adjoint(h, nside, lmax, spin=spin)
    got = plan.alm2map_adjoint(torch.from_numpy(h).cuda()).cpu().numpy()
    assert colerr(got, want) < TOL
    g = make_alm(nside, lmax, lmax, spin, nmaps, seed=5)
    want = orc.map2alm_adjoint(g, nside, lmax, spin=spin)
    got = plan.map2alm_adjoint(torch.from_numpy(g).cuda()).cpu().numpy()
    assert colerr(got, want) < TOL


@pytest.mark.parametrize("nside,lmax,mmax,spin,niter", [
    (16, 32, 32, 0, 3), (16, 32, 32, 2, 3),
    (8, 23, 23, 0, 2),        # lmax = 3 nside - 1: every cap ring folds several m onto a bin
    (16, 47, 47, 2, 2),
    (16, 40, 20, 0, 2),       # mmax < lmax
    (32, 64, 64, 0, 1),
])
def test_iteration_fp64(orc, sht, nside, lmax, mmax, spin, niter):
    """The iteration runs on the ring spectra (no FFT); it must equal the
    oracle's pixel-domain Algorithm 2 on white-noise maps (not band-limited)."""
    ncomp = 2 if spin else 1
    rng = np.random.default_rng(17 + nside + lmax)
    T = rng.standard_normal((2, ncomp, 12 * nside * nside))
    want = orc.map2alm(T, nside, lmax, mmax, spin=spin, niter=niter)
    plan = sht.Plan(nside, lmax, mmax, spin, "fp64")
    got = plan.map2alm(torch.from_numpy(T).cuda(), niter=niter).cpu().numpy()
    assert colerr(got, want) < TOL


def test_host_entry_points_match_device(sht):
    nside, lmax, nmaps = 16, 32, 3
    plan = sht.Plan(nside, lmax, None, 0, "fp64")
    a = make_alm(nside, lmax, lmax, 0, nmaps, seed=9)
    dev = plan.alm2map(torch.from_numpy(a).cuda()).cpu().numpy()
    host = plan.alm2map_host(a)
    np.testing.assert_array_equal(host, dev)
    back_dev = plan.map2alm(torch.from_numpy(dev).cuda(), niter=1).cpu().numpy()
    back_host = plan.map2alm_host(dev, niter=1)
    np.testing.assert_array_equal(back_host, back_dev)
    host2 = plan.alm2map_host(a)
    np.testing.assert_array_equal(host2, dev)


def test_invalid_calls_report_status(sht):
    plan = sht.Plan(4, 8, None, 0, "fp64")
    lib = sht.load()
    x = torch.zeros(1, 1, plan.npix, dtype=torch.float64, device="cuda")
    y = torch.zeros(1, 1, plan.nalm, dtype=torch.complex128, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    rc = lib.sht_map2alm(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 1, 0,
                         ctypes.c_void_p(ws.data_ptr()), 16, st)
    assert rc == sht.SHT_EINVAL and "workspace" in sht.sht_last_error()
    rc = lib.sht_alm2map(plan.handle, None, ctypes.c_void_p(x.data_ptr()), 1, None, 0, st)
    assert rc == sht.SHT_EINVAL
    rc = lib.sht_alm2map(plan.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), 0,
                         None, 0, st)
    assert rc == sht.SHT_EINVAL


@pytest.mark.parametrize("pinned", [False, True])
def test_host_entry_points_pipelined_chunks(sht, monkeypatch, pinned):
    """Several chunks through the copy / transform / copy pipeline (chunk size
    forced to 2 maps), pageable and pinned host buffers: bit-identical to the
    device entry points."""
    monkeypatch.setenv("SHT_HOST_CHUNK_MAPS", "2")
    nside, lmax, nmaps = 16, 32, 7
    plan = sht.Plan(nside, lmax, None, 2, "fp64")
    a = make_alm(nside, lmax, lmax, 2, nmaps, seed=19)
    dev = plan.alm2map(torch.from_numpy(a).cuda()).cpu().numpy()
    if pinned:
        a_h = torch.from_numpy(a).pin_memory()
        out = torch.empty(dev.shape, dtype=torch.float64).pin_memory()
        plan.alm2map_host(a_h.numpy(), out_host=out.numpy())
        host = out.numpy()
    else:
        host = plan.alm2map_host(a)
    np.testing.assert_array_equal(host, dev)
    back_dev = plan.map2alm(torch.from_numpy(dev).cuda(), niter=1).cpu().numpy()
    np.testing.assert_array_equal(plan.map2alm_host(dev, niter=1), back_dev)
