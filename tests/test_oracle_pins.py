"""Pins that tie the CPU oracle to mathematics and to the paper, not to itself.

Every test here runs on the CPU (no GPU marker). Each one targets a mistake
that could hide in the oracle: a wrong normalisation or phase (closed forms,
mpmath, addition theorem, orthonormality), a wrong ring layout (equal-area
property), a wrong sign/index in a transform (brute force vs separable,
impulse responses, adjoint identity, iteration convergence, E/B rotation),
and the paper's one worked example (the N = 4 FFT circle, Appendix A.1).
"""
import math
import os

import numpy as np
import pytest

from paper_2208_10154_b300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    """max |a - b| / RMS(b)."""
    b = np.asarray(b)
    return float(np.max(np.abs(np.asarray(a) - b)) / np.sqrt(np.mean(np.abs(b) ** 2)))


def real_m0(a, lmax):
    a = a.copy()
    a[..., :lmax + 1] = a[..., :lmax + 1].real
    return a


# ----------------------------------------------------------------- geometry
@pytest.mark.parametrize("nside", [1, 2, 4, 8, 32, 512])
def test_ring_geometry_equal_area(orc, nside):
    """HEALPix defining property: the sphere area north of ring i's centre
    latitude equals the area of the pixels above it plus half of ring i."""
    z, sth, phi0, n, start = orc.ring_info(nside)
    npix = 12 * nside * nside
    assert n.sum() == npix
    assert start[0] == 0 and np.all(start[1:] == start[:-1] + n[:-1])
    frac = (start + n / 2.0) / npix
    np.testing.assert_allclose((1.0 - z) / 2.0, frac, rtol=0, atol=1e-15)
    np.testing.assert_allclose(sth ** 2 + z ** 2, 1.0, rtol=0, atol=1e-15)
    # mirror rings: same length and phase offset, opposite z
    nr = 4 * nside - 1
    np.testing.assert_array_equal(n, n[::-1])
    np.testing.assert_allclose(phi0, phi0[::-1], atol=0)
    np.testing.assert_allclose(z, -z[::-1], atol=1e-15)
    # first pixels: caps at pi/N, belt alternating pi/(4 nside) and 0
    i = np.arange(1, nr + 1)
    cap = (i < nside) | (i > 3 * nside)
    np.testing.assert_allclose(phi0[cap], np.pi / n[cap], rtol=1e-15)
    belt = ~cap
    want = np.where((i[belt] - nside) % 2 == 0, np.pi / (4 * nside), 0.0)
    np.testing.assert_allclose(phi0[belt], want, atol=1e-16)


def test_fft_circle_n4_golden(orc):
    """Appendix A.1 (paper's worked example): on a ring of N = 4 pixels,
    harmonic m lands on the FFT circle at phi = 2 pi m / N, i.e. FFT bin m mod 4.
    A map that lives only on ring 1 (N = 4) has a_lm = dsigma lambda_lm(theta_1)
    e^{-i m phi0} X(m mod 4), X the 4-point DFT of the ring."""
    rows = np.loadtxt(os.path.join(GOLDEN, "fft_circle_n4.txt"))
    nside, lmax = 2, 11
    z, sth, phi0, n, start = orc.ring_info(nside)
    assert n[0] == 4
    rng = np.random.default_rng(7)
    x = rng.standard_normal(4)
    T = np.zeros((1, 1, 12 * nside * nside))
    T[0, 0, :4] = x
    a = orc.map2alm(T, nside, lmax, method="brute")[0, 0]
    X = np.fft.fft(x)                       # X[j] = sum_n x_n e^{-2 pi i j n / 4}
    lam = orc.lambda_theta(lmax, lmax, np.arccos(z[0]))[0]
    dsig = 4 * np.pi / (12 * nside * nside)
    for m, b, ph in rows:
        m, b = int(m), int(b)
        assert b == m % 4 and abs(ph - 2 * np.pi * b / 4) < 1e-15
        for l in range(m, lmax + 1):
            q = orc.alm_index(lmax, l, m)
            want = dsig * lam[q] * np.exp(-1j * m * phi0[0]) * X[b]
            if m == 0:
                want = want.real
            assert abs(a[q] - want) < 1e-13 * max(1.0, abs(want)), (m, l)


# ----------------------------------------------------------- closed forms
def closed_Y(l, m, th, ph):
    c, s = np.cos(th), np.sin(th)
    e = np.exp(1j * m * ph)
    pi = np.pi
    tab = {
        (0, 0): 1 / np.sqrt(4 * pi) + 0 * c,
        (1, 0): np.sqrt(3 / (4 * pi)) * c,
        (1, 1): -np.sqrt(3 / (8 * pi)) * s,
        (2, 0): np.sqrt(5 / (16 * pi)) * (3 * c ** 2 - 1),
        (2, 1): -np.sqrt(15 / (8 * pi)) * s * c,
        (2, 2): np.sqrt(15 / (32 * pi)) * s ** 2,
        (3, 0): np.sqrt(7 / (16 * pi)) * (5 * c ** 3 - 3 * c),
        (3, 1): -np.sqrt(21 / (64 * pi)) * s * (5 * c ** 2 - 1),
        (3, 2): np.sqrt(105 / (32 * pi)) * s ** 2 * c,
        (3, 3): -np.sqrt(35 / (64 * pi)) * s ** 3,
    }
    return tab[(l, m)] * e


def test_lambda_closed_forms(orc):
    rng = np.random.default_rng(11)
    th = rng.uniform(0.01, np.pi - 0.01, 50)
    lam = orc.lambda_theta(3, 3, th)
    for l in range(4):
        for m in range(l + 1):
            want = closed_Y(l, m, th, 0.0).real
            np.testing.assert_allclose(lam[:, orc.alm_index(3, l, m)], want, rtol=1e-14, atol=1e-15)


def test_spin2_closed_forms(orc):
    rng = np.random.default_rng(12)
    th = rng.uniform(0.01, np.pi - 0.01, 40)
    c, s = np.cos(th), np.sin(th)
    p2 = orc.slambda_theta(2, 2, 2, th)     # [t, m + 2, l]
    m2 = orc.slambda_theta(2, 2, -2, th)
    pi = np.pi
    np.testing.assert_allclose(p2[:, 2, 2], np.sqrt(15 / (32 * pi)) * s ** 2, rtol=1e-14)
    np.testing.assert_allclose(m2[:, 2, 2], np.sqrt(15 / (32 * pi)) * s ** 2, rtol=1e-14)
    np.testing.assert_allclose(p2[:, 4, 2], np.sqrt(5 / (64 * pi)) * (1 - c) ** 2, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(m2[:, 4, 2], np.sqrt(5 / (64 * pi)) * (1 + c) ** 2, rtol=1e-13, atol=1e-16)


def _sympy_spin_harmonics(lmax):
    """+-2Y_lm from the spin-raising/lowering operators applied to Y_lm written
    with Rodrigues' formula (Condon-Shortley phase):
      eth eta  = -sin^s(t) (d_t + i/sin(t) d_p) (sin^-s(t) eta)
      ethb eta = -sin^-s(t) (d_t - i/sin(t) d_p) (sin^s(t) eta)
      2Y  = sqrt((l-2)!/(l+2)!) eth^2 Y,   -2Y = sqrt((l-2)!/(l+2)!) ethb^2 Y."""
    sp = pytest.importorskip("sympy")
    t, p, x = sp.symbols("t p x", real=True)

    def Ylm(l, m):
        am = abs(m)
        P = sp.diff((x ** 2 - 1) ** l, x, l) / (2 ** l * sp.factorial(l))
        Plm = (-1) ** am * (1 - x ** 2) ** sp.Rational(am, 2) * sp.diff(P, x, am)
        N = sp.sqrt((2 * l + 1) / (4 * sp.pi) * sp.factorial(l - am) / sp.factorial(l + am))
        Y = N * Plm.subs(x, sp.cos(t)) * sp.exp(sp.I * am * p)
        if m < 0:
            Y = (-1) ** am * sp.conjugate(Y)
        return Y

    def eth(eta, s):
        return -sp.sin(t) ** s * (sp.diff(sp.sin(t) ** (-s) * eta, t)
                                  + sp.I / sp.sin(t) * sp.diff(sp.sin(t) ** (-s) * eta, p))

    def ethb(eta, s):
        return -sp.sin(t) ** (-s) * (sp.diff(sp.sin(t) ** s * eta, t)
                                     - sp.I / sp.sin(t) * sp.diff(sp.sin(t) ** s * eta, p))

    out = {}
    for l in range(2, lmax + 1):
        f = sp.sqrt(sp.factorial(l - 2) / sp.factorial(l + 2))
        for m in range(-l, l + 1):
            Y = Ylm(l, m)
            out[(2, l, m)] = sp.lambdify((t, p), f * eth(eth(Y, 0), 1), "numpy")
            out[(-2, l, m)] = sp.lambdify((t, p), f * ethb(ethb(Y, 0), -1), "numpy")
    return out


def test_spin2_against_eth_operator(orc):
    """Wigner-d based +-2Y_lm equal the eth / eth-bar definition (l = 2..4, all m)."""
    fns = _sympy_spin_harmonics(4)
    rng = np.random.default_rng(13)
    th = rng.uniform(0.05, np.pi - 0.05, 12)
    ph = rng.uniform(0, 2 * np.pi, 12)
    for s in (2, -2):
        lam = orc.slambda_theta(4, 4, s, th)
        for l in range(2, 5):
            for m in range(-l, l + 1):
                want = np.asarray(fns[(s, l, m)](th, ph), dtype=np.complex128)
                got = lam[:, m + 4, l] * np.exp(1j * m * ph)
                np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12, err_msg=str((s, l, m)))


def test_lambda_vs_wigner_spin0(orc):
    """Two independent constructions of lambda_lm (Legendre recurrence vs
    Wigner-d recurrence with s = 0) agree up to l = 300."""
    th = np.array([0.003, 0.4, 1.2, np.pi / 2, 2.0, 3.1])
    L = orc.lambda_theta(300, 300, th)
    W = orc.slambda_theta(300, 300, 0, th)
    err = 0.0
    for m in range(0, 301, 7):
        q0 = orc.alm_index(300, m, m)
        err = max(err, np.max(np.abs(L[:, q0:q0 + 301 - m] - W[:, m + 300, m:])))
    assert err < 1e-12


def _plm_explicit(mp, l, m, th):
    """Textbook expansion of Rodrigues' formula (Condon-Shortley phase):
    P_l^m(x) = (-1)^m 2^-l (1-x^2)^(m/2) sum_k (-1)^k (2l-2k)! / (k! (l-k)! (l-2k-m)!) x^(l-2k-m),
    evaluated in enough digits to survive its ~4^l cancellation."""
    x = mp.cos(mp.mpf(th)); s = mp.sin(mp.mpf(th))
    tot = mp.mpf(0)
    for k in range((l - m) // 2 + 1):
        tot += (-1) ** k * mp.factorial(2 * l - 2 * k) / (
            mp.factorial(k) * mp.factorial(l - k) * mp.factorial(l - 2 * k - m)) * x ** (l - 2 * k - m)
    norm = mp.sqrt((2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m))
    return norm * (-1) ** m * tot * s ** m / mp.mpf(2) ** l


def _scaled_value(mp, orc, l, m, th):
    mant, e10 = orc.lambda_scaled(l, m, th)
    return mp.mpf(float(mant[-1])) * mp.power(10, int(e10[-1])), int(e10[-1])


def test_lambda_mpmath_spot_values(orc):
    """Low degree: mpmath's Ferrers function legenp at 50 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    for l, m, th in [(10, 3, 0.7), (40, 0, 1.9), (100, 40, 2.1), (120, 120, 0.9)]:
        x = mp.cos(mp.mpf(th))
        norm = mp.sqrt((2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m))
        want = norm * mp.legenp(l, m, x)
        got, _ = _scaled_value(mp, orc, l, m, th)
        assert abs(got / want - 1) < 1e-13, (l, m, th, got, want)


@pytest.mark.parametrize("l,m,th", [(1023, 17, 0.05), (1023, 1023, 1.0), (2047, 1000, 0.6),
                                    (2047, 2047, 1.5707), (1500, 700, 2.9)])
def test_lambda_high_degree_explicit_sum(orc, l, m, th):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = int(0.7 * l) + 60
    want = _plm_explicit(mp, l, m, th)
    got, _ = _scaled_value(mp, orc, l, m, th)
    assert abs(got / want - 1) < 1e-12, (l, m, th, got, want)


@pytest.mark.parametrize("l,m,th", [(2047, 2000, 0.01), (2047, 1500, 0.002), (1200, 1100, 0.02)])
def test_lambda_deep_underflow(orc, l, m, th):
    """Values thousands of decades below the float64 range (sin^m theta at
    high m near the pole) keep full relative accuracy in the scaled recurrence."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = int(0.7 * l) + 60
    want = _plm_explicit(mp, l, m, th)
    got, e10 = _scaled_value(mp, orc, l, m, th)
    assert e10 < -300
    assert abs(got / want - 1) < 1e-12, (l, m, th, got, want)


def test_lambda_scipy_low_l(orc):
    sc = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(14)
    th = rng.uniform(0.01, np.pi - 0.01, 20)
    lmax = 100
    lam = orc.lambda_theta(lmax, lmax, th)
    fn = getattr(sc, "sph_harm_y", None)
    for l in range(0, lmax + 1, 9):
        for m in range(0, l + 1, 5):
            if fn is not None:
                want = fn(l, m, th, 0.0).real
            else:
                want = sc.sph_harm(m, l, 0.0, th).real
            np.testing.assert_allclose(lam[:, orc.alm_index(lmax, l, m)], want, rtol=1e-10, atol=1e-13)


# ------------------------------------------------------ sum rules, grids
@pytest.mark.parametrize("nside,lmax", [(64, 191), (256, 767)])
def test_addition_theorem_every_ring(orc, nside, lmax):
    """sum_m w_m lambda_lm^2 = (2l+1)/4pi at every ring (w_0 = 1, w_{m>0} = 2)."""
    z, *_ = orc.ring_info(nside)
    th = np.arccos(z[: 2 * nside])
    lam = orc.lambda_theta(lmax, lmax, th)
    ls, ms = inputs.lm_arrays(lmax)
    w = np.where(ms == 0, 1.0, 2.0)
    tot = np.zeros((th.size, lmax + 1))
    for t in range(th.size):
        np.add.at(tot[t], ls, w * lam[t] ** 2)
    want = (2 * np.arange(lmax + 1) + 1) / (4 * np.pi)
    np.testing.assert_allclose(tot, np.broadcast_to(want, tot.shape), rtol=1e-12)


def test_addition_theorem_lmax2047(orc):
    th = np.array([0.0008, 0.3, 1.1, 1.57])
    lmax = 2047
    lam = orc.lambda_theta(lmax, lmax, th)
    ls, ms = inputs.lm_arrays(lmax)
    w = np.where(ms == 0, 1.0, 2.0)
    for t in range(th.size):
        tot = np.zeros(lmax + 1)
        np.add.at(tot, ls, w * lam[t] ** 2)
        np.testing.assert_allclose(tot, (2 * np.arange(lmax + 1) + 1) / (4 * np.pi), rtol=1e-11)


@pytest.mark.parametrize("s", [2, -2])
def test_addition_theorem_spin(orc, s):
    th = np.array([0.01, 0.5, 1.3, 2.2, 3.0])
    lmax = 200
    lam = orc.slambda_theta(lmax, lmax, s, th)   # [t, m, l]
    tot = (lam ** 2).sum(axis=1)
    want = (2 * np.arange(lmax + 1) + 1) / (4 * np.pi)
    want[:2] = 0.0
    np.testing.assert_allclose(tot, np.broadcast_to(want, tot.shape), rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("s", [0, 2, -2])
def test_orthonormality_gauss_legendre(orc, s):
    """2 pi sum_t w_t sl_lm(t) sl_l'm(t) = delta_ll' on Gauss-Legendre nodes
    (exact quadrature for these polynomial products), l, l' <= 64."""
    lmax = 64
    x, w = np.polynomial.legendre.leggauss(80)
    th = np.arccos(x)
    lam = orc.slambda_theta(lmax, lmax, s, th)
    for m in range(-lmax, lmax + 1, 3):
        A = lam[:, m + lmax, :]
        G = 2 * np.pi * (A * w[:, None]).T @ A
        l0 = max(abs(m), abs(s))
        want = np.diag([1.0 if l >= l0 else 0.0 for l in range(lmax + 1)])
        np.testing.assert_allclose(G, want, atol=1e-13)


# ---------------------------------------------- brute force vs separable
@pytest.mark.parametrize("nside", [1, 2, 4, 8])
@pytest.mark.parametrize("spin", [0, 2])
def test_brute_vs_separable_aliasing(orc, nside, spin):
    """lmax up to 4 nside - 1: heavy aliasing of m on the short cap rings."""
    lmax = 4 * nside - 1
    ncomp = 2 if spin else 1
    a = inputs.gaussian_alm(nside * 10 + spin, 2, ncomp, lmax, cls=np.ones(lmax + 1))
    if spin:
        ls, _ = inputs.lm_arrays(lmax)
        a[..., ls < 2] = 0
    mb = orc.alm2map(a, nside, lmax, spin=spin, method="brute")
    ms = orc.alm2map(a, nside, lmax, spin=spin, method="sep")
    assert rel(ms, mb) < 1e-13
    rng = np.random.default_rng(nside)
    T = rng.standard_normal(mb.shape)
    ab = orc.map2alm(T, nside, lmax, spin=spin, method="brute")
    as_ = orc.map2alm(T, nside, lmax, spin=spin, method="sep")
    assert rel(as_, ab) < 1e-13


@pytest.mark.parametrize("spin", [0, 2])
def test_brute_vs_separable_nside32(orc, spin):
    nside, lmax = 32, 64
    ncomp = 2 if spin else 1
    a = inputs.gaussian_alm(0, 2, ncomp, lmax, cls=inputs.cl_inv_lp1_sq(lmax))
    mb = orc.alm2map(a, nside, lmax, spin=spin, method="brute")
    ms = orc.alm2map(a, nside, lmax, spin=spin)
    assert rel(ms, mb) < 1e-13
    ab = orc.map2alm(mb, nside, lmax, spin=spin, method="brute")
    as_ = orc.map2alm(mb, nside, lmax, spin=spin)
    assert rel(as_, ab) < 1e-13


# ------------------------------------------------- quadrature identities
def test_constant_map(orc):
    nside, lmax = 8, 20
    c = 1.7
    T = np.full((1, 1, 12 * nside * nside), c)
    a = orc.map2alm(T, nside, lmax)[0, 0]
    assert abs(a[0] - c * np.sqrt(4 * np.pi)) < 1e-14
    # odd l at m = 0 vanish (north/south symmetry of a constant map)
    for l in range(1, lmax + 1, 2):
        assert abs(a[orc.alm_index(lmax, l, 0)]) < 1e-14
    # aliasing: only m = 0 mod N_r survives ring by ring
    z, sth, phi0, n, start = orc.ring_info(nside)
    lam = orc.lambda_theta(lmax, lmax, np.arccos(z))
    dsig = 4 * np.pi / (12 * nside * nside)
    for m in range(lmax + 1):
        keep = (m % n) == 0
        for l in range(m, lmax + 1):
            q = orc.alm_index(lmax, l, m)
            want = dsig * c * np.sum(n[keep] * lam[keep, q] * np.exp(-1j * m * phi0[keep]))
            if m == 0:
                want = want.real
            assert abs(a[q] - want) < 1e-13


def test_impulse_reproduces_closed_form(orc):
    """alm2map of a single coefficient reproduces (2 Re of) Y_lm at pixel centres."""
    nside, lmax = 4, 3
    th, ph = orc.pix_angles(nside)
    for l in range(4):
        for m in range(l + 1):
            for val in ([1.0, 1j] if m else [1.0]):
                a = np.zeros((1, 1, orc.nalm(lmax)), dtype=complex)
                a[0, 0, orc.alm_index(lmax, l, m)] = val
                T = orc.alm2map(a, nside, lmax)[0, 0]
                Y = closed_Y(l, m, th, ph)
                want = (Y.real if m == 0 else 2 * (val * Y).real)
                np.testing.assert_allclose(T, want, atol=1e-14)


# ------------------------------------------------------------- adjoints
@pytest.mark.parametrize("spin", [0, 2])
def test_adjoint_dot_product(orc, spin):
    nside, lmax = 16, 40
    ncomp = 2 if spin else 1
    a = real_m0(inputs.gaussian_alm(3, 1, ncomp, lmax, cls=np.ones(lmax + 1)), lmax)
    if spin:
        ls, _ = inputs.lm_arrays(lmax)
        a[..., ls < 2] = 0
    rng = np.random.default_rng(5)
    T = rng.standard_normal((1, ncomp, 12 * nside * nside))
    lhs = np.sum(orc.alm2map(a, nside, lmax, spin=spin) * T)
    b = orc.map2alm(T, nside, lmax, spin=spin)
    _, ms = inputs.lm_arrays(lmax)
    w = np.where(ms == 0, 1.0, 2.0)
    rhs = 12 * nside * nside / (4 * np.pi) * np.sum(w * (np.conj(a) * b).real)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _real_params(lmax):
    """(index, part) of every real parameter: Re a_l0, and Re, Im a_lm (m > 0)."""
    ls, ms = inputs.lm_arrays(lmax)
    out = []
    for q in range(ls.size):
        out.append((q, 0))
        if ms[q] > 0:
            out.append((q, 1))
    return out


@pytest.mark.parametrize("spin", [0, 2])
def test_adjoint_explicit_transpose(orc, spin):
    """Explicit matrices at nside 2: the adjoint formulas equal the transpose."""
    nside, lmax = 2, 5
    ncomp = 2 if spin else 1
    npx = 12 * nside * nside
    na = orc.nalm(lmax)
    params = [(c, q, part) for c in range(ncomp) for (q, part) in _real_params(lmax)]
    A = np.zeros((ncomp * npx, len(params)))        # alm2map
    for j, (c, q, part) in enumerate(params):
        a = np.zeros((1, ncomp, na), dtype=complex)
        a[0, c, q] = 1.0 if part == 0 else 1j
        A[:, j] = orc.alm2map(a, nside, lmax, spin=spin).ravel()
    B = np.zeros((len(params), ncomp * npx))        # map2alm
    for p in range(ncomp * npx):
        T = np.zeros(ncomp * npx); T[p] = 1.0
        b = orc.map2alm(T.reshape(1, ncomp, npx), nside, lmax, spin=spin)[0]
        B[:, p] = [b[c, q].real if part == 0 else b[c, q].imag for (c, q, part) in params]
    rng = np.random.default_rng(9)
    h = rng.standard_normal((1, ncomp, npx))
    adj = orc.alm2map_adjoint(h, nside, lmax, spin=spin)[0]
    got = np.array([adj[c, q].real if part == 0 else adj[c, q].imag for (c, q, part) in params])
    np.testing.assert_allclose(got, A.T @ h.ravel(), atol=1e-12)
    g = np.zeros((1, ncomp, na), dtype=complex)
    vals = rng.standard_normal(len(params))
    for v, (c, q, part) in zip(vals, params):
        g[0, c, q] += v if part == 0 else 1j * v
    adj2 = orc.map2alm_adjoint(g, nside, lmax, spin=spin).ravel()
    np.testing.assert_allclose(adj2, B.T @ vals, atol=1e-12)


# ------------------------------------------------------------ iteration
@pytest.mark.parametrize("spin", [0, 2])
def test_jacobi_iteration_converges(orc, spin):
    """Algorithm 2 on band-limited input (lmax = 2 nside): the error of
    map2alm_n(alm2map(a)) decreases monotonically with n."""
    nside = 16
    lmax = 2 * nside
    ncomp = 2 if spin else 1
    a = inputs.gaussian_alm(21, 2, ncomp, lmax, cls=inputs.cl_inv_lp1_sq(lmax))
    T = orc.alm2map(a, nside, lmax, spin=spin)
    errs = []
    for n in range(6):
        b = orc.map2alm(T, nside, lmax, spin=spin, niter=n)
        errs.append(np.max(np.abs(b - a)))
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-3 * errs[0]


# ------------------------------------------------------------------ E/B
def test_eb_rotation_identity(orc):
    """(Q, U) -> (U, -Q) multiplies Q+iU by -i, which maps (a_E, a_B) to
    (a_B, -a_E) by the E/B definition of Sec. 2.3 (equ:alm-eb)."""
    nside, lmax = 16, 32
    rng = np.random.default_rng(31)
    P = rng.standard_normal((1, 2, 12 * nside * nside))
    a = orc.map2alm(P, nside, lmax, spin=2)
    R = np.stack([P[:, 1], -P[:, 0]], axis=1)
    b = orc.map2alm(R, nside, lmax, spin=2)
    np.testing.assert_allclose(b[:, 0], a[:, 1], atol=1e-14)
    np.testing.assert_allclose(b[:, 1], -a[:, 0], atol=1e-14)


def test_pure_e_gives_small_b(orc):
    nside, lmax = 32, 48
    a = inputs.gaussian_alm(41, 1, 2, lmax)
    a[:, 1] = 0.0
    T = orc.alm2map(a, nside, lmax, spin=2)
    b = orc.map2alm(T, nside, lmax, spin=2, niter=3)
    assert np.max(np.abs(b[:, 1])) < 1e-4 * np.max(np.abs(b[:, 0]))


def test_spin2_impulse_fixes_the_eb_sign(orc):
    """The overall sign of the E/B combination (Sec. 2.3, equ:alm-eb with
    a_{+-2} = -(a_E +- i a_B)), fixed by the closed form
    2Y_20 = -2Y_20 = sqrt(15/(32 pi)) sin^2(theta) (spin raising twice on
    Y_20): a_E,20 = 1 gives Q = -sqrt(15/(32 pi)) sin^2 theta, U = 0, and
    a_B,20 = 1 gives Q = 0, U = -sqrt(15/(32 pi)) sin^2 theta at every pixel
    centre. Flipping both E/B signs together would pass the rotation, adjoint
    and projection pins but fails this one. map2alm of those maps (with
    Algorithm 2, band-limited input) must return +1 in the same slot."""
    nside, lmax = 8, 7
    th, _ = orc.pix_angles(nside)
    y20 = math.sqrt(15.0 / (32.0 * math.pi)) * np.sin(th) ** 2
    i20 = orc.alm_index(lmax, 2, 0)
    for comp in (0, 1):
        a = np.zeros((1, 2, orc.nalm(lmax)), dtype=complex)
        a[0, comp, i20] = 1.0
        for method in ("brute", "sep"):
            QU = orc.alm2map(a, nside, lmax, spin=2, method=method)[0]
            want_q = -y20 if comp == 0 else np.zeros_like(y20)
            want_u = np.zeros_like(y20) if comp == 0 else -y20
            np.testing.assert_allclose(QU[0], want_q, atol=1e-14)
            np.testing.assert_allclose(QU[1], want_u, atol=1e-14)
        back = orc.map2alm(QU[None], nside, lmax, spin=2, niter=4)[0]
        assert abs(back[comp, i20] - 1.0) < 1e-6
        assert abs(back[1 - comp, i20]) < 1e-6


@pytest.mark.parametrize("spin", [0, 2])
def test_sampled_tiers_equal_full_transform(orc, spin):
    """The sampled forms used at full size (map2alm for chosen m, alm2map on
    chosen rings) return exactly the corresponding entries of the full
    separable transform, which the pins above tie to the mathematics."""
    nside, lmax, mmax = 8, 23, 20
    ncomp = 2 if spin else 1
    a = inputs.gaussian_alm(5, 2, ncomp, lmax, mmax)
    full = orc.alm2map(a, nside, lmax, mmax, spin)
    _, _, _, n, st = orc.ring_info(nside)
    rings = [1, 3, 8, 16, 20, 31]
    for k, r in enumerate(orc.alm2map_rings(a, nside, lmax, rings, mmax, spin)):
        assert np.array_equal(r, full[..., st[rings[k] - 1]:st[rings[k] - 1] + n[rings[k] - 1]])
    x = np.random.default_rng(2).standard_normal(full.shape)
    af = orc.map2alm(x, nside, lmax, mmax, spin)
    ms = [0, 1, 7, 20]
    for k, blk in enumerate(orc.map2alm_msel(x, nside, lmax, ms, mmax, spin)):
        i0 = orc.alm_index(lmax, ms[k], ms[k])
        assert np.array_equal(blk, af[..., i0:i0 + lmax - ms[k] + 1])


# ------------------------------------------------- Algorithm 3 (immediate)
def _gs_pixel(orc, x, nside, lmax, npass, mmax, spin=0):
    """Algorithm 3 read as a block Gauss-Seidel sweep over m in the pixel
    domain: for each m in order, a_m += map2alm(S - alm2map(a))_m with the
    residual recomputed from the current a (every earlier order updated)."""
    nc = 2 if spin else 1
    a = np.zeros((x.shape[0], nc, orc.nalm(lmax, mmax)), dtype=complex)
    for _ in range(npass):
        for m in range(mmax + 1):
            r = x - orc.alm2map(a, nside, lmax, mmax, spin)
            c = orc.map2alm_msel(r, nside, lmax, [m], mmax, spin)[0]
            i0 = orc.alm_index(lmax, m, m)
            a[..., i0:i0 + lmax - m + 1] += c
    return a


@pytest.mark.parametrize("nside,lmax,mmax,npass", [(4, 15, 15, 2), (8, 20, 12, 2), (2, 7, 7, 3)])
def test_immediate_fourier_domain_equals_pixel_definition(orc, nside, lmax, mmax, npass):
    """The oracle's Algorithm 3 keeps the residual as ring spectra and updates
    them after every order (aliased bins included); it must equal the
    pixel-domain sweep, here with lmax up to 4 nside - 1 (heavy aliasing)."""
    x = np.random.default_rng(nside).standard_normal((2, 1, 12 * nside * nside))
    got = orc.map2alm_immediate(x, nside, lmax, npass, mmax)
    assert rel(got, _gs_pixel(orc, x, nside, lmax, npass, mmax)) < 1e-13


def test_immediate_without_aliasing_equals_traditional(orc):
    """With mmax = 1 no two orders share a ring bin, so the orders decouple and
    npass sweeps of Algorithm 3 equal Algorithm 2 with npass - 1 refinements."""
    nside, lmax, mmax = 4, 5, 1
    x = np.random.default_rng(0).standard_normal((2, 1, 12 * nside * nside))
    for npass in (1, 2, 3):
        g = orc.map2alm_immediate(x, nside, lmax, npass, mmax)
        j = orc.map2alm(x, nside, lmax, mmax, niter=npass - 1)
        assert rel(g, j) < 1e-13


@pytest.mark.parametrize("nside,lmax", [(16, 40), (32, 80)])
def test_immediate_more_accurate_for_lmax_below_3nside(orc, nside, lmax):
    """Sec. 4: for band-limited maps with 2 nside < lmax < 3 nside the
    immediate mode (Algorithm 3) is more accurate than the traditional one
    (Algorithm 2) after the same number of passes, and both converge."""
    a = inputs.gaussian_alm(3, 2, 1, lmax, cls=inputs.cl_inv_llp1(lmax))
    x = orc.alm2map(a, nside, lmax)
    eg, ej = [], []
    for npass in (1, 2, 3, 4):
        eg.append(rel(orc.map2alm_immediate(x, nside, lmax, npass), a))
        ej.append(rel(orc.map2alm(x, nside, lmax, niter=npass - 1), a))
    assert all(g < j for g, j in zip(eg[1:], ej[1:])), (eg, ej)
    assert eg[-1] < 0.05 * eg[0]


@pytest.mark.parametrize("nside,lmax,mmax,npass", [(4, 15, 15, 2), (8, 20, 12, 2), (2, 7, 7, 3)])
def test_immediate_spin2_fourier_domain_equals_pixel_definition(orc, nside, lmax, mmax, npass):
    """Spin 2: the residual's Q and U ring spectra, updated at orders m and -m
    after every order, give the same E/B as the pixel-domain sweep."""
    x = np.random.default_rng(nside + 7).standard_normal((2, 2, 12 * nside * nside))
    got = orc.map2alm_immediate(x, nside, lmax, npass, mmax, spin=2)
    assert rel(got, _gs_pixel(orc, x, nside, lmax, npass, mmax, spin=2)) < 1e-13


def test_immediate_spin2_without_aliasing_equals_traditional(orc):
    """Spin 2 with mmax = 1 on rings of at least 4 pixels: orders +-1 and 0
    share no bin, so npass sweeps equal Algorithm 2 with npass - 1 refinements."""
    nside, lmax, mmax = 4, 6, 1
    x = np.random.default_rng(1).standard_normal((2, 2, 12 * nside * nside))
    for npass in (1, 2, 3):
        g = orc.map2alm_immediate(x, nside, lmax, npass, mmax, spin=2)
        j = orc.map2alm(x, nside, lmax, mmax, spin=2, niter=npass - 1)
        assert rel(g, j) < 1e-13


def test_immediate_spin2_recovers_band_limited_eb(orc):
    """Sec. 4 for polarisation: band-limited E/B maps with 2 nside < lmax <
    3 nside; the immediate passes beat Algorithm 2 after the same number of
    passes and converge towards the true E and B."""
    nside, lmax = 16, 40
    cl = inputs.cl_inv_llp1(lmax)
    a = inputs.gaussian_alm(4, 2, 2, lmax, cls=cl)
    a[:, 1] *= 0.1                                   # C_BB = 0.01 C_EE
    a[..., inputs.lm_arrays(lmax, lmax)[0] < 2] = 0  # E and B start at l = 2
    x = orc.alm2map(a, nside, lmax, spin=2)
    eg, ej = [], []
    for npass in (1, 2, 3, 4):
        eg.append(rel(orc.map2alm_immediate(x, nside, lmax, npass, spin=2), a))
        ej.append(rel(orc.map2alm(x, nside, lmax, spin=2, niter=npass - 1), a))
    assert all(g < j for g, j in zip(eg[1:], ej[1:])), (eg, ej)
    assert eg[-1] < 0.05 * eg[0]


def test_immediate_spin2_planted_sign_error_fails_pixel_check(orc):
    """The pixel-domain check is sharp for spin 2: a U map with its sign
    flipped (a plausible Q/U mix-up) changes the result well beyond 1e-13."""
    nside, lmax = 4, 15
    x = np.random.default_rng(3).standard_normal((1, 2, 12 * nside * nside))
    y = x.copy()
    y[:, 1] *= -1
    got = orc.map2alm_immediate(y, nside, lmax, 2, spin=2)
    assert rel(got, _gs_pixel(orc, x, nside, lmax, 2, lmax, spin=2)) > 1e-2


def test_immediate_pixel_error_at_the_papers_configuration(orc):
    """Sec. 4's comparison (its figure of pixel-domain errors): nside 128, a
    sky band-limited to lmax = 383 < 3 nside, 3 rounds. The map resynthesised
    from the immediate mode's a_lm is much closer to the input than the
    traditional mode's (about 10x here), and both a_lm errors shrink."""
    nside, lmax = 128, 383
    a = inputs.gaussian_alm(1, 1, 1, lmax, cls=inputs.cl_inv_llp1(lmax))
    x = orc.alm2map(a, nside, lmax)

    def pix(b):
        return float(np.sqrt(np.mean((orc.alm2map(b, nside, lmax) - x) ** 2) / np.mean(x ** 2)))

    g1 = orc.map2alm_immediate(x, nside, lmax, 1)
    g = orc.map2alm_immediate(x, nside, lmax, 3)
    j = orc.map2alm(x, nside, lmax, niter=2)
    assert pix(g) < pix(j) / 4, (pix(g), pix(j))
    assert rel(g, a) < rel(j, a) and rel(g, a) < rel(g1, a)


@pytest.mark.parametrize("nside", [1, 2, 3, 8, 13, 64])
def test_every_ring_has_a_multiple_of_four_pixels(orc, nside):
    """HEALPix rings hold 4i (caps) or 4 nside (belt) pixels. So orders m, m'
    share a ring bin (m' = +-m mod N) only if m' = +-m mod 4: an even and an
    odd order never interact in Algorithm 3's sweep, which is what lets the
    GPU refine the orders 2t and 2t + 1 in one step."""
    _, _, _, n, _ = orc.ring_info(nside)
    assert np.all(np.asarray(n) % 4 == 0)
    assert len(n) == 4 * nside - 1 and int(np.sum(n)) == 12 * nside * nside


@pytest.mark.parametrize("m", [44, 55, 63])
def test_ring_first_pair_against_mpmath(orc, m):
    """The ring optimisation's criterion (Sec. 3.1, Implementation detail)
    checked with the explicit Rodrigues expansion in mpmath (enough digits
    for its cancellation), independently of the oracle's recurrence: at
    nside 32, lmax 63, every ring pair before the
    oracle's first pair of order m has |lambda_lm| < 1e-30 for all l, and the
    first pair has some l at or above it. The library's table follows from
    these by the stated rule (nondecreasing in m, multiples of 32, order 0
    keeps every pair)."""
    mp = pytest.importorskip("mpmath")
    nside, lmax = 32, 63
    mp.mp.dps = int(0.7 * lmax) + 60
    eps = mp.mpf("1e-30")
    p0 = int(orc.ring_first_pairs(nside, lmax, 0, raw=True)[m])
    assert p0 >= 3
    z, s, _, _, _ = orc.ring_info(nside)

    def lam_max(p):
        th = float(np.arctan2(s[p], z[p]))
        return max(abs(_plm_explicit(mp, l, m, th)) for l in range(m, lmax + 1))

    for p in range(p0):
        assert lam_max(p) < eps, (m, p)
    assert lam_max(p0) >= eps
    full = orc.ring_first_pairs(nside, lmax, 0)
    raw = orc.ring_first_pairs(nside, lmax, 0, raw=True)
    assert full[0] == 0 and np.all(np.diff(full) >= 0) and np.all(full % 32 == 0)
    assert np.all(full <= raw)
