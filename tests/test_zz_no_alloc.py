"""GPU test of sht_alm2map_noalloc, the alm2map entry point for callers that
cannot allocate device memory while they run (allocation-free serving loops,
frameworks that own all GPU memory). It is called through the
C ABI twice in a row, on different inputs, and must match sht_alm2map (the
workspace-based entry point) within the FP64 tolerance of the other tests.
This file is collected last so a failure here cannot hide another test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2208_10154_b300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _rel(got, want):
    w = want.reshape(-1, want.shape[-1])
    g = got.reshape(w.shape)
    return float(np.max(np.max(np.abs(g - w), axis=1) / np.sqrt(np.mean(w ** 2, axis=1))))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_10154_b300 import build, sht
    build.build()
    L = sht.load()
    L.sht_alm2map_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_void_p]
    L.sht_alm2map_noalloc.restype = ctypes.c_int
    L.sht_noalloc_scratch_bytes.restype = ctypes.c_size_t
    return L


@pytest.mark.parametrize("spin", [0, 2])
def test_noalloc_matches_alm2map_twice(lib, spin):
    from paper_2208_10154_b300 import sht
    nside, lmax, nmaps = 32, 63, 5
    ncomp = 2 if spin else 1
    plan = sht.Plan(nside, lmax, None, spin, "fp64")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((11, 12)):
        a = inputs.gaussian_alm(seed, nmaps, ncomp, lmax, cls=np.ones(lmax + 1))
        if spin:
            ls, _ = inputs.lm_arrays(lmax)
            a[..., ls < 2] = 0
        alm = torch.from_numpy(a).cuda()
        want = plan.alm2map(alm).cpu().numpy()
        out = torch.full((nmaps, ncomp, plan.npix), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.sht_alm2map_noalloc(plan.handle, ctypes.c_void_p(alm.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), nmaps, stream)
        assert rc == sht.SHT_OK, sht.sht_last_error()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert _rel(got, want) < TOL, call


def test_noalloc_rejects_oversized_call(lib):
    from paper_2208_10154_b300 import sht
    plan = sht.Plan(128, 255, None, 0, "fp64")
    nmaps = 64          # G needs 256 * 2 * 256 * 128 * 8 bytes = 128 MiB > 64 MiB
    assert lib.sht_noalloc_scratch_bytes() == 64 << 20
    alm = torch.zeros((nmaps, 1, plan.nalm), dtype=torch.complex128, device="cuda")
    out = torch.zeros((nmaps, 1, plan.npix), dtype=torch.float64, device="cuda")
    rc = lib.sht_alm2map_noalloc(plan.handle, ctypes.c_void_p(alm.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 nmaps, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == sht.SHT_EINVAL
    assert "scratch" in sht.sht_last_error()
