"""CPU oracle for the HEALPix spherical harmonic transforms (arXiv:2208.10154).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (``paper_2208_10154_b300``) never imports it and
shares no code with it: the C source here (``sht_oracle.c``) is a plain,
slow, long-double restatement of the definitions in Sec. 2.1 (Eq. 1, eq:mm,
equ:backward equ), Sec. 2.3 (Q_lm+iU_lm, equ:alm-eb) and Algorithm 2.

Array layouts (numpy, C order):
  map  float64 [nmaps, ncomp, npix]       RING order
  alm  complex128 [nmaps, ncomp, nalm]    m-major packed, idx(l,m) = m(2lmax+1-m)/2 + l
with ncomp = 1 for spin 0 and 2 (Q,U resp. E,B) for spin 2.

Pins that tie each function to something other than itself live in
``tests/test_oracle_*.py`` (closed forms, mpmath, addition theorem,
orthonormality, brute force vs separable, quadrature identities, adjoint
identity, iteration convergence, E/B rotation, the compact square storage
against a worked example, the E/B projection's complementarity and
idempotence, the ring optimisation's criterion against mpmath).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sht_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        lib.oracle_npix.restype = ctypes.c_longlong
        lib.oracle_npix.argtypes = [I]
        lib.oracle_nalm.restype = ctypes.c_longlong
        lib.oracle_nalm.argtypes = [I, I]
        lib.oracle_ring_info.argtypes = [I, P, P, P, P, P]
        lib.oracle_pix_angles.argtypes = [I, P, P]
        lib.oracle_lambda_theta.argtypes = [I, I, I, P, P]
        lib.oracle_slambda_theta.argtypes = [I, I, I, I, P, P]
        for fn in ("oracle_alm2map_brute", "oracle_map2alm_brute",
                   "oracle_alm2map_sep", "oracle_map2alm_sep"):
            getattr(lib, fn).argtypes = [I, I, I, I, I, P, P]
        lib.oracle_map2alm_iter.argtypes = [I, I, I, I, I, P, P, I]
        lib.oracle_map2alm_immediate.argtypes = [I, I, I, I, P, P, I]
        lib.oracle_map2alm_immediate2.argtypes = [I, I, I, I, P, P, I]
        lib.oracle_map2alm_msel.argtypes = [I, I, I, I, I, P, I, P, P]
        lib.oracle_alm2map_rings.argtypes = [I, I, I, I, I, P, I, P, P]
        lib.oracle_lambda_scaled.argtypes = [I, I, ctypes.c_double, P, P]
        lib.oracle_num_threads.restype = I
        lib.oracle_set_num_threads.argtypes = [I]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def npix(nside: int) -> int:
    return 12 * nside * nside


def nalm(lmax: int, mmax: int | None = None) -> int:
    mmax = lmax if mmax is None else mmax
    return (mmax + 1) * (2 * lmax + 2 - mmax) // 2


def alm_index(lmax: int, l, m):
    return m * (2 * lmax + 1 - m) // 2 + l


def num_threads() -> int:
    return _load().oracle_num_threads()


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def ring_info(nside: int):
    """(z, sin(theta), phi0, n, start) per ring, rings 1..4nside-1."""
    lib = _load()
    nr = 4 * nside - 1
    z = np.empty(nr); s = np.empty(nr); p0 = np.empty(nr)
    n = np.empty(nr, dtype=np.int64); st = np.empty(nr, dtype=np.int64)
    lib.oracle_ring_info(nside, _ptr(z), _ptr(s), _ptr(p0), _ptr(n), _ptr(st))
    return z, s, p0, n, st


def pix_angles(nside: int):
    lib = _load()
    th = np.empty(npix(nside)); ph = np.empty(npix(nside))
    lib.oracle_pix_angles(nside, _ptr(th), _ptr(ph))
    return th, ph


def lambda_theta(lmax: int, mmax: int, theta) -> np.ndarray:
    """lambda_lm(theta) from the Legendre recurrence, shape [ntheta, nalm]."""
    lib = _load()
    th = np.ascontiguousarray(np.atleast_1d(theta), dtype=np.float64)
    out = np.empty((th.size, nalm(lmax, mmax)))
    lib.oracle_lambda_theta(lmax, mmax, th.size, _ptr(th), _ptr(out))
    return out


def lambda_scaled(lmax: int, m: int, theta: float):
    """lambda_lm(theta), l = m..lmax, as (mantissa, exponent10): value = mant * 10**exp10.
    Reaches far below the float64 range (the recurrence keeps a binary exponent)."""
    lib = _load()
    mant = np.empty(lmax - m + 1)
    e10 = np.empty(lmax - m + 1, dtype=np.int64)
    lib.oracle_lambda_scaled(lmax, m, float(theta), _ptr(mant), _ptr(e10))
    return mant, e10


def slambda_theta(lmax: int, mmax: int, s: int, theta) -> np.ndarray:
    """theta part of sY_lm via Wigner d, shape [ntheta, 2mmax+1, lmax+1] (m = -mmax..mmax)."""
    lib = _load()
    th = np.ascontiguousarray(np.atleast_1d(theta), dtype=np.float64)
    out = np.empty((th.size, 2 * mmax + 1, lmax + 1))
    lib.oracle_slambda_theta(lmax, mmax, s, th.size, _ptr(th), _ptr(out))
    return out


def ring_first_pairs(nside: int, lmax: int, spin: int = 0, eps: float = 1e-30, raw: bool = False):
    """The ring optimisation (Sec. 3.1, Implementation detail: for a given m
    the rings where P_lm has an extremely low amplitude are ignored), as the
    library reads it: for each order m, p0(m) = the first ring pair, counted
    from the north pole (pair p = north ring p + 1), where |lambda_lm(theta)|
    reaches eps for some l (spin 2: the theta parts of sY_lm for s = +2 and
    -2). With raw=False the result is then made nondecreasing in m (the
    smallest p0 of this and every higher order), rounded down to a multiple
    of 32, and 0 for m = 0. int array [lmax + 1] (mmax = lmax)."""
    z, sth, _, _, _ = ring_info(nside)
    R = 2 * nside
    theta = np.arctan2(sth[:R], z[:R])
    if spin == 0:
        lam = np.abs(lambda_theta(lmax, lmax, theta))                   # [R, nalm]
        live = np.zeros((lmax + 1, R), dtype=bool)
        for m in range(lmax + 1):
            i0 = m * (2 * lmax + 1 - m) // 2
            live[m] = lam[:, i0 + m:i0 + lmax + 1].max(axis=1) >= eps
    else:
        sp = np.abs(slambda_theta(lmax, lmax, 2, theta))[:, lmax:, :]   # [R, m >= 0, l]
        sm = np.abs(slambda_theta(lmax, lmax, -2, theta))[:, lmax:, :]
        live = (np.maximum(sp, sm).max(axis=2) >= eps).T                # [m, R]
    p0 = np.array([int(np.argmax(live[m])) if live[m, :R - 1].any() else R - 1 for m in range(lmax + 1)])
    if raw:
        return p0
    out = np.minimum.accumulate(p0[::-1])[::-1] // 32 * 32
    out[0] = 0
    return out.astype(np.int32)


def _check(nside, lmax, mmax, spin):
    if spin not in (0, 2):
        raise ValueError("spin must be 0 or 2")
    mmax = lmax if mmax is None else mmax
    if not (nside >= 1 and lmax >= 0 and 0 <= mmax <= lmax):
        raise ValueError("bad nside/lmax/mmax")
    return mmax


def alm2map(alm, nside: int, lmax: int, mmax: int | None = None, spin: int = 0,
            method: str = "sep") -> np.ndarray:
    """Backward transform. alm complex128 [nmaps, ncomp, nalm] -> map float64 [nmaps, ncomp, npix]."""
    mmax = _check(nside, lmax, mmax, spin)
    ncomp = 2 if spin else 1
    a = np.ascontiguousarray(alm, dtype=np.complex128).reshape(-1, ncomp, nalm(lmax, mmax))
    fn = "oracle_alm2map_brute" if method == "brute" else "oracle_alm2map_sep"
    lib = _load()
    out = np.zeros((a.shape[0], ncomp, npix(nside)))
    getattr(lib, fn)(nside, lmax, mmax, spin, a.shape[0], _ptr(a), _ptr(out))
    return out


def map2alm(maps, nside: int, lmax: int, mmax: int | None = None, spin: int = 0,
            method: str = "sep", niter: int = 0) -> np.ndarray:
    """Forward transform. map float64 [nmaps, ncomp, npix] -> alm complex128 [nmaps, ncomp, nalm]."""
    mmax = _check(nside, lmax, mmax, spin)
    ncomp = 2 if spin else 1
    x = np.ascontiguousarray(maps, dtype=np.float64).reshape(-1, ncomp, npix(nside))
    lib = _load()
    out = np.zeros((x.shape[0], ncomp, nalm(lmax, mmax)), dtype=np.complex128)
    if niter:
        if method == "brute":
            raise ValueError("iteration uses the separable tier")
        lib.oracle_map2alm_iter(nside, lmax, mmax, spin, x.shape[0], _ptr(x), _ptr(out), int(niter))
    else:
        fn = "oracle_map2alm_brute" if method == "brute" else "oracle_map2alm_sep"
        getattr(lib, fn)(nside, lmax, mmax, spin, x.shape[0], _ptr(x), _ptr(out))
    return out


def map2alm_immediate(maps, nside: int, lmax: int, npass: int, mmax: int | None = None,
                      spin: int = 0) -> np.ndarray:
    """Algorithm 3 (immediate / Gauss-Seidel iteration over m): ``npass`` >= 1
    sweeps from a = 0 on the ring spectra of the residual. spin 0: map float64
    [nmaps, 1, npix] -> alm complex128 [nmaps, 1, nalm]; spin 2: Q/U maps
    [nmaps, 2, npix] -> E/B alm [nmaps, 2, nalm]."""
    mmax = _check(nside, lmax, mmax, spin)
    if npass < 1:
        raise ValueError("npass must be >= 1")
    nc = 2 if spin else 1
    x = np.ascontiguousarray(maps, dtype=np.float64).reshape(-1, nc, npix(nside))
    out = np.zeros((x.shape[0], nc, nalm(lmax, mmax)), dtype=np.complex128)
    fn = "oracle_map2alm_immediate2" if spin else "oracle_map2alm_immediate"
    getattr(_load(), fn)(nside, lmax, mmax, x.shape[0], _ptr(x), _ptr(out), int(npass))
    return out


def map2alm_msel(maps, nside: int, lmax: int, ms, mmax: int | None = None, spin: int = 0):
    """map2alm restricted to the orders ``ms`` (separable tier, same formula):
    a list, one complex128 array [nmaps, ncomp, lmax - m + 1] (l = m..lmax) per m."""
    mmax = _check(nside, lmax, mmax, spin)
    ms = np.ascontiguousarray(ms, dtype=np.int32)
    if ms.size and (ms.min() < 0 or ms.max() > mmax):
        raise ValueError("selected m outside 0..mmax")
    ncomp = 2 if spin else 1
    x = np.ascontiguousarray(maps, dtype=np.float64).reshape(-1, ncomp, npix(nside))
    K = int(sum(lmax - int(m) + 1 for m in ms))
    out = np.zeros((x.shape[0], ncomp, K), dtype=np.complex128)
    _load().oracle_map2alm_msel(nside, lmax, mmax, spin, x.shape[0], _ptr(x), int(ms.size), _ptr(ms), _ptr(out))
    res, o = [], 0
    for m in ms:
        res.append(out[..., o:o + lmax - int(m) + 1])
        o += lmax - int(m) + 1
    return res


def alm2map_rings(alm, nside: int, lmax: int, rings, mmax: int | None = None, spin: int = 0):
    """alm2map restricted to the 1-based rings ``rings`` (separable tier, same
    formula): a list, one float64 array [nmaps, ncomp, N_ring] per ring."""
    mmax = _check(nside, lmax, mmax, spin)
    rings = np.ascontiguousarray(rings, dtype=np.int32)
    if rings.size and (rings.min() < 1 or rings.max() > 4 * nside - 1):
        raise ValueError("ring outside 1..4 nside - 1")
    ncomp = 2 if spin else 1
    a = np.ascontiguousarray(alm, dtype=np.complex128).reshape(-1, ncomp, nalm(lmax, mmax))
    _, _, _, n, _ = ring_info(nside)
    P = int(sum(int(n[r - 1]) for r in rings))
    out = np.zeros((a.shape[0], ncomp, P))
    _load().oracle_alm2map_rings(nside, lmax, mmax, spin, a.shape[0], _ptr(a), int(rings.size), _ptr(rings),
                                 _ptr(out))
    res, o = [], 0
    for r in rings:
        res.append(out[..., o:o + int(n[r - 1])])
        o += int(n[r - 1])
    return res


def alm2map_adjoint(maps, nside, lmax, mmax=None, spin=0):
    """Adjoint of alm2map in real parameters (Re a_l0; Re, Im a_lm for m>0):
    (Npix/4pi) * map2alm(h) * w_m, w_0 = 1 (real part only), w_{m>0} = 2."""
    mmax = lmax if mmax is None else mmax
    a = map2alm(maps, nside, lmax, mmax, spin) * (npix(nside) / (4 * np.pi))
    w = _mweights(lmax, mmax)
    a = a * w
    a[..., w == 1.0] = a[..., w == 1.0].real
    return a


def map2alm_adjoint(alm, nside, lmax, mmax=None, spin=0):
    """Adjoint of map2alm: (4pi/Npix) * alm2map(g'), g'_l0 = Re g_l0, g'_lm = g_lm / 2 (m>0)."""
    mmax = lmax if mmax is None else mmax
    w = _mweights(lmax, mmax)
    g = np.array(alm, dtype=np.complex128, copy=True) / w
    g[..., w == 1.0] = g[..., w == 1.0].real
    return alm2map(g, nside, lmax, mmax, spin) * (4 * np.pi / npix(nside))


def _mweights(lmax, mmax):
    w = np.empty(nalm(lmax, mmax))
    for m in range(mmax + 1):
        i0 = alm_index(lmax, m, m)
        w[i0:i0 + lmax - m + 1] = 1.0 if m == 0 else 2.0
    return w


# ---------------------------------------------------------------------------
# Compact square a_lm storage (Sec. 5, equ:new alm save scheme): a real
# (lmax+1) x (lmax+1) matrix per map and component, every element used:
#   Re a_lm -> (l, m)                 for 0 <= m <= l <= lmax
#   Im a_lm -> (l - m, lmax - m + 1)  for 1 <= m <= l <= lmax
# Entries with m > mmax stay zero. Plain loops over (l, m).
# ---------------------------------------------------------------------------
def alm_to_square(alm, lmax: int, mmax: int | None = None) -> np.ndarray:
    mmax = lmax if mmax is None else mmax
    a = np.asarray(alm, dtype=np.complex128)
    lead = a.shape[:-1]
    flat = a.reshape(-1, a.shape[-1])
    sq = np.zeros((flat.shape[0], lmax + 1, lmax + 1))
    for m in range(mmax + 1):
        for l in range(m, lmax + 1):
            v = flat[:, alm_index(lmax, l, m)]
            sq[:, l, m] = v.real
            if m >= 1:
                sq[:, l - m, lmax - m + 1] = v.imag
    return sq.reshape(lead + (lmax + 1, lmax + 1))


def square_to_alm(sq, lmax: int, mmax: int | None = None) -> np.ndarray:
    """Inverse of alm_to_square (Im a_l0 = 0)."""
    mmax = lmax if mmax is None else mmax
    q = np.asarray(sq, dtype=np.float64)
    lead = q.shape[:-2]
    flat = q.reshape(-1, lmax + 1, lmax + 1)
    out = np.zeros((flat.shape[0], nalm(lmax, mmax)), dtype=np.complex128)
    for m in range(mmax + 1):
        for l in range(m, lmax + 1):
            im = flat[:, l - m, lmax - m + 1] if m >= 1 else 0.0
            out[:, alm_index(lmax, l, m)] = flat[:, l, m] + 1j * im
    return out.reshape(lead + (out.shape[-1],))


# ---------------------------------------------------------------------------
# Pixel-domain E / B projection (Sec. 2.3, equ:aeab mat form pixel): the Q/U
# maps of the E (or B) part, i.e. alm2map of map2alm with the other
# component of every a_lm set to zero (lambda^{E,B} keeps one diagonal block).
# ---------------------------------------------------------------------------
def eb_project(maps, nside: int, lmax: int, which: str = "E", niter: int = 0,
               mmax: int | None = None) -> np.ndarray:
    a = map2alm(maps, nside, lmax, mmax, spin=2, niter=niter)
    a[:, 1 if which == "E" else 0, :] = 0.0
    return alm2map(a, nside, lmax, mmax, spin=2)
