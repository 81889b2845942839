"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no transform arithmetic: it only draws random numbers. It
is the one module that both the CUDA path's tests/benchmark and the CPU
oracle's tests import, so that both sides see bit-identical inputs.

Sky recipe (the paper's runs use Planck-2018 CMB spectra, Sec. 4 / Fig. 3,
which are not available here; analytic spectra of the same shape stand in):
  a_lm complex Gaussian with E|a_lm|^2 = C_l: Re, Im ~ N(0, C_l/2) for m > 0,
  a_l0 ~ N(0, C_l) real; one ``standard_normal((nmaps, ncomp, nalm, 2))`` draw
  from ``numpy.random.default_rng(seed)`` (PCG64), then scaled.
"""
from __future__ import annotations

import numpy as np


def nalm(lmax: int, mmax: int | None = None) -> int:
    mmax = lmax if mmax is None else mmax
    return (mmax + 1) * (2 * lmax + 2 - mmax) // 2


def npix(nside: int) -> int:
    return 12 * nside * nside


def lm_arrays(lmax: int, mmax: int | None = None):
    """l and m of every packed coefficient (m-major, idx = m(2lmax+1-m)/2 + l)."""
    mmax = lmax if mmax is None else mmax
    ls, ms = [], []
    for m in range(mmax + 1):
        ls.append(np.arange(m, lmax + 1))
        ms.append(np.full(lmax - m + 1, m))
    return np.concatenate(ls), np.concatenate(ms)


def cl_inv_lp1_sq(lmax: int) -> np.ndarray:
    """C_l = 1/(l+1)^2 for l >= 2, 0 below."""
    l = np.arange(lmax + 1, dtype=np.float64)
    c = 1.0 / (l + 1.0) ** 2
    c[:2] = 0.0
    return c


def cl_inv_llp1(lmax: int) -> np.ndarray:
    """C_l = 1/(l(l+1)) for l >= 2, 0 below."""
    l = np.arange(lmax + 1, dtype=np.float64)
    c = np.zeros(lmax + 1)
    c[2:] = 1.0 / (l[2:] * (l[2:] + 1.0))
    return c


def gaussian_alm(seed_or_rng, nmaps: int, ncomp: int, lmax: int, mmax: int | None = None,
                 cls=None) -> np.ndarray:
    """complex128 [nmaps, ncomp, nalm]; ``cls`` is [lmax+1] or [ncomp, lmax+1]."""
    mmax = lmax if mmax is None else mmax
    rng = np.random.default_rng(seed_or_rng) if not isinstance(seed_or_rng, np.random.Generator) else seed_or_rng
    n = nalm(lmax, mmax)
    cls = cl_inv_llp1(lmax) if cls is None else np.asarray(cls, dtype=np.float64)
    if cls.ndim == 1:
        cls = np.broadcast_to(cls, (ncomp, lmax + 1))
    ls, ms = lm_arrays(lmax, mmax)
    g = rng.standard_normal((nmaps, ncomp, n, 2))
    out = np.empty((nmaps, ncomp, n), dtype=np.complex128)
    for c in range(ncomp):
        cl = cls[c][ls]
        sd = np.where(ms == 0, np.sqrt(cl), np.sqrt(cl / 2.0))
        re = g[:, c, :, 0] * sd
        im = np.where(ms == 0, 0.0, g[:, c, :, 1] * sd)
        out[:, c, :] = re + 1j * im
    return out


def white_noise(seed_or_rng, shape, sigma) -> np.ndarray:
    rng = np.random.default_rng(seed_or_rng) if not isinstance(seed_or_rng, np.random.Generator) else seed_or_rng
    return rng.standard_normal(shape) * np.asarray(sigma)[..., None]


# Workloads (sizes, spectra, seeds) of the five configurations.
WORKLOADS = {
    "t_nside32": dict(nside=32, lmax=64, mmax=64, spin=0, nmaps=16, seed=0, cl="inv_lp1_sq"),
    "t_nside512": dict(nside=512, lmax=1023, mmax=1023, spin=0, nmaps=1000, seed=1, cl="inv_llp1",
                       noise_frac=0.01),
    "qu_nside1024": dict(nside=1024, lmax=2047, mmax=2047, spin=2, nmaps=200, seed=2, cl="inv_llp1",
                         bb_frac=0.01),
    "serve_mixed": dict(seed=3, nreq=20000, nsides=(64, 128, 256, 512, 1024),
                        nside_p=(0.3, 0.3, 0.2, 0.15, 0.05), spin2_p=0.3, max_maps=256,
                        hbm_budget_gb=150.0),
    "autograd_nside256": dict(nside=256, lmax=511, mmax=511, spin=0, nmaps=256, seed=4, cl="inv_llp1",
                              niter=3, fd_step=1e-6, n_fd=64),
}


def workload_cls(w: dict) -> np.ndarray:
    lmax = w["lmax"]
    base = cl_inv_lp1_sq(lmax) if w.get("cl") == "inv_lp1_sq" else cl_inv_llp1(lmax)
    if w.get("spin", 0) == 2:
        return np.stack([base, w.get("bb_frac", 1.0) * base])
    return base[None, :]


def gaussian_alm_torch(seed: int, nmaps: int, ncomp: int, lmax: int, mmax: int | None = None, cls=None,
                       device="cuda"):
    """The same sky recipe as ``gaussian_alm``, drawn on ``device`` with a
    seeded ``torch.Generator`` (for batches too large to draw on the host):
    complex128 tensor [nmaps, ncomp, nalm]. Not bit-identical to the numpy
    draw; parity tests copy the columns they check to the host."""
    import torch
    mmax = lmax if mmax is None else mmax
    n = nalm(lmax, mmax)
    cls = cl_inv_llp1(lmax) if cls is None else np.asarray(cls, dtype=np.float64)
    if cls.ndim == 1:
        cls = np.broadcast_to(cls, (ncomp, lmax + 1))
    ls, ms = lm_arrays(lmax, mmax)
    sd = np.stack([np.where(ms == 0, np.sqrt(cls[c][ls]), np.sqrt(cls[c][ls] / 2.0)) for c in range(ncomp)])
    sd = torch.from_numpy(sd).to(device)[None]
    m0 = torch.from_numpy(ms == 0).to(device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    re = torch.randn((nmaps, ncomp, n), generator=g, dtype=torch.float64, device=device) * sd
    im = torch.randn((nmaps, ncomp, n), generator=g, dtype=torch.float64, device=device) * sd
    im[..., m0] = 0.0
    out = torch.complex(re, im)
    del re, im
    return out.contiguous()


def white_noise_torch(seed: int, shape, device="cuda"):
    """Unit Gaussian noise of ``shape`` (float64) from a seeded torch.Generator."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.randn(tuple(shape), generator=g, dtype=torch.float64, device=device)
