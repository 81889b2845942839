/*
 * sht_oracle.c -- plain, slow, CPU reference for the HEALPix spherical
 * harmonic transforms (TEST INFRASTRUCTURE: only the tests, the smoke check
 * and the timed CPU baseline of the benchmark may load this library; the
 * product path never does).
 *
 * What it computes (arXiv:2208.10154, "Accelerating spherical harmonic
 * transforms for a large number of sky maps"):
 *   map2alm, spin 0   a_lm = dsigma * sum_p T_p lambda_lm(theta_p) e^{-i m phi_p}
 *                     dsigma = 4 pi / Npix                      (Sec. 2.1, Eq. 1 and eq:mm)
 *   alm2map, spin 0   T_p = sum_l a_l0 lambda_l0 + 2 Re sum_{m>0} sum_l a_lm lambda_lm e^{i m phi_p}
 *                     (Sec. 2.1, equ:backward equ; real field, m >= 0 stored)
 *   map2alm, spin 2   a_{+-2,lm} = dsigma * sum_p (Q +- iU)_p conj(+-2Y_lm(p)),
 *                     a_E = -(a_2 + a_-2)/2,  a_B = i (a_2 - a_-2)/2   (Sec. 2.3, Q_lm+iU_lm, equ:alm-eb)
 *   alm2map, spin 2   a_{+-2} = -(a_E +- i a_B) for every m (negative m from
 *                     a_{X,l,-m} = (-1)^m conj(a_{X,lm})), Q +- iU = sum_{l,|m|<=l} a_{+-2,lm} +-2Y_lm
 *   iteration         a^0 = map2alm(T), a^{n+1} = a^n + map2alm(T - alm2map(a^n))  (Sec. 4, Algorithm 2)
 *
 * Readings of points the paper leaves to HEALPix (cited there, not restated):
 *   - ring geometry: the standard HEALPix RING layout (ring_geom below);
 *   - lambda_lm = sqrt((2l+1)/4pi (l-m)!/(l+m)!) P_l^m(cos theta) with the
 *     Condon-Shortley phase (the "lam" of Sec. 2.1's footnote);
 *   - sY_lm(theta, phi) = (-1)^m sqrt((2l+1)/4pi) d^l_{-m,s}(theta) e^{i m phi},
 *     which equals the spin-raising (eth) definition used by the papers the
 *     paper cites for spin-2 harmonics.
 *
 * Two tiers:
 *   brute force : every pixel evaluates its own harmonics from (theta_p, phi_p);
 *   separable   : lambda once per ring, a direct (non-FFT) DFT per ring, then the
 *                 sum over l -- the same formula factored (Sec. 2.1, eq:mm rows 2-4).
 * lambda_lm uses a long-double three-term recurrence in l with an explicit
 * binary exponent (never underflows); spin-weighted harmonics use a separate
 * Wigner-d recurrence, so the two constructions check each other.
 *
 * Layouts: map  double [nmaps][ncomp][npix]   (RING order)
 *          alm  double [nmaps][ncomp][nalm][2] (complex, m-major packed,
 *               idx(l,m) = m(2 lmax + 1 - m)/2 + l, 0 <= m <= mmax, m <= l <= lmax)
 *          ncomp = 1 (T) or 2 (Q,U / E,B).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double ld;
static const ld PI_L = 3.141592653589793238462643383279502884L;

/* ------------------------------------------------------------------ */
/* geometry                                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    ld z, cth, sth;      /* cos(theta) = z, sin(theta)                 */
    ld chalf, shalf;     /* cos(theta/2), sin(theta/2)                 */
    ld phi0;             /* phi of the first pixel of the ring         */
    long long start;     /* index of the first pixel                   */
    int n;               /* pixels in the ring                         */
} ring_t;

/* HEALPix RING geometry, 1-based ring index i = 1 .. 4 nside - 1. Cap
 * rings take sin(theta) from the exact 1 -+ z to avoid cancellation. */
static void ring_geom(int nside, int i, ring_t* r)
{
    ld ns = (ld)nside;
    long long npix = 12LL * nside * nside;
    if (i < nside) {
        ld omz = (ld)i * (ld)i / (3.0L * ns * ns);           /* 1 - z */
        r->z = 1.0L - omz;
        r->sth = sqrtl(omz * (2.0L - omz));
        r->chalf = sqrtl(1.0L - 0.5L * omz);
        r->shalf = sqrtl(0.5L * omz);
        r->n = 4 * i;
        r->phi0 = PI_L / (4.0L * i);
        r->start = 2LL * i * (i - 1);
    } else if (i <= 3 * nside) {
        ld z = (ld)(4 * nside - 2 * i) / (3.0L * ns);
        r->z = z;
        r->sth = sqrtl((1.0L - z) * (1.0L + z));
        r->chalf = sqrtl(0.5L * (1.0L + z));
        r->shalf = sqrtl(0.5L * (1.0L - z));
        r->n = 4 * nside;
        r->phi0 = ((i - nside) % 2 == 0) ? PI_L / (4.0L * nside) : 0.0L;
        r->start = 2LL * nside * (nside - 1) + 4LL * nside * (i - nside);
    } else {
        int ip = 4 * nside - i;
        ld opz = (ld)ip * (ld)ip / (3.0L * ns * ns);         /* 1 + z */
        r->z = opz - 1.0L;
        r->sth = sqrtl(opz * (2.0L - opz));
        r->chalf = sqrtl(0.5L * opz);
        r->shalf = sqrtl(1.0L - 0.5L * opz);
        r->n = 4 * ip;
        r->phi0 = PI_L / (4.0L * ip);
        r->start = npix - 2LL * ip * (ip + 1);
    }
    r->cth = r->z;
}

long long oracle_npix(int nside) { return 12LL * nside * nside; }
int oracle_nrings(int nside) { return 4 * nside - 1; }
long long oracle_nalm(int lmax, int mmax)
{
    return (long long)(mmax + 1) * (2 * lmax + 2 - mmax) / 2;
}
static inline long long aidx(int lmax, int l, int m)
{
    return (long long)m * (2 * lmax + 1 - m) / 2 + l;
}

/* Ring table for tests: z, sin(theta), phi0 as double; n and start as int64. */
void oracle_ring_info(int nside, double* z, double* sth, double* phi0,
                      long long* n, long long* start)
{
    for (int i = 1; i <= 4 * nside - 1; i++) {
        ring_t r;
        ring_geom(nside, i, &r);
        z[i - 1] = (double)r.z;
        sth[i - 1] = (double)r.sth;
        phi0[i - 1] = (double)r.phi0;
        n[i - 1] = r.n;
        start[i - 1] = r.start;
    }
}

/* theta and phi of every pixel centre (double), for tests. */
void oracle_pix_angles(int nside, double* theta, double* phi)
{
    for (int i = 1; i <= 4 * nside - 1; i++) {
        ring_t r;
        ring_geom(nside, i, &r);
        ld th = atan2l(r.sth, r.cth);
        for (int k = 0; k < r.n; k++) {
            theta[r.start + k] = (double)th;
            phi[r.start + k] = (double)(r.phi0 + 2.0L * PI_L * k / r.n);
        }
    }
}

/* ------------------------------------------------------------------ */
/* lambda_lm: normalised associated Legendre functions                */
/* ------------------------------------------------------------------ */
/* out[l - m] = lambda_lm(theta) for l = m .. lmax.
 *   lambda_mm     = (-1)^m sqrt((2m+1)/(4 pi) prod_{k<=m} (2k-1)/(2k)) sin^m theta
 *   lambda_{m+1,m} = sqrt(2m+3) cos(theta) lambda_mm
 *   lambda_lm     = sqrt((4l^2-1)/(l^2-m^2)) [cos(theta) lambda_{l-1,m}
 *                   - sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)) lambda_{l-2,m}]
 * The running pair carries a separate binary exponent, so nothing underflows
 * inside the recurrence; the returned value is the true long-double value. */
static void lambda_lm(int lmax, int m, ld cth, ld sth, ld* out)
{
    int ex, E = 0;
    ld v = sqrtl((2.0L * m + 1.0L) / (4.0L * PI_L));
    v = frexpl(v, &ex); E += ex;
    for (int k = 1; k <= m; k++) {
        v *= sqrtl((2.0L * k - 1.0L) / (2.0L * k)) * sth;
        v = frexpl(v, &ex); E += ex;
    }
    if (m & 1) v = -v;
    out[0] = ldexpl(v, E);
    if (lmax == m) return;
    ld prev = v;
    ld cur = sqrtl(2.0L * m + 3.0L) * cth * v;
    out[1] = ldexpl(cur, E);
    for (int l = m + 2; l <= lmax; l++) {
        ld L = l, M = m;
        ld a = sqrtl((4.0L * L * L - 1.0L) / (L * L - M * M));
        ld b = sqrtl(((L - 1) * (L - 1) - M * M) / (4.0L * (L - 1) * (L - 1) - 1.0L));
        ld nxt = a * (cth * cur - b * prev);
        prev = cur;
        cur = nxt;
        if (fabsl(cur) > 0x1p64L) {
            cur = ldexpl(cur, -64);
            prev = ldexpl(prev, -64);
            E += 64;
        }
        out[l - m] = ldexpl(cur, E);
    }
}

/* Same recurrence, returning each lambda_lm as mantissa * 10^exp10 so values
 * far below the double range can be checked (tests of the scaled exponent). */
void oracle_lambda_scaled(int lmax, int m, double theta, double* mant, long long* exp10)
{
    int ex, E = 0;
    ld cth = cosl((ld)theta), sth = sinl((ld)theta);
    ld v = sqrtl((2.0L * m + 1.0L) / (4.0L * PI_L));
    v = frexpl(v, &ex); E += ex;
    for (int k = 1; k <= m; k++) {
        v *= sqrtl((2.0L * k - 1.0L) / (2.0L * k)) * sth;
        v = frexpl(v, &ex); E += ex;
    }
    if (m & 1) v = -v;
    ld prev = 0.0L, cur = v;
    for (int l = m; l <= lmax; l++) {
        if (l == m + 1) { prev = cur; cur = sqrtl(2.0L * m + 3.0L) * cth * prev; }
        else if (l > m + 1) {
            ld L = l, M = m;
            ld a = sqrtl((4.0L * L * L - 1.0L) / (L * L - M * M));
            ld b = sqrtl(((L - 1) * (L - 1) - M * M) / (4.0L * (L - 1) * (L - 1) - 1.0L));
            ld nxt = a * (cth * cur - b * prev);
            prev = cur; cur = nxt;
            if (fabsl(cur) > 0x1p64L) { cur = ldexpl(cur, -64); prev = ldexpl(prev, -64); E += 64; }
        }
        /* cur * 2^E  ->  mant * 10^e10 */
        if (cur == 0.0L) { mant[l - m] = 0.0; exp10[l - m] = 0; continue; }
        ld lg = log10l(fabsl(cur)) + (ld)E * 0.30102999566398119521373889472449302676818988146211L;
        ld fl = floorl(lg);
        ld mm = powl(10.0L, lg - fl);
        mant[l - m] = (double)(cur < 0 ? -mm : mm);
        exp10[l - m] = (long long)fl;
    }
}

/* ------------------------------------------------------------------ */
/* Wigner d^l_{mp,m}(theta)                                           */
/* ------------------------------------------------------------------ */
/* x^n for 0 <= x as (mantissa, binary exponent). */
static void spow(ld x, int n, ld* mant, long* ex)
{
    if (n == 0) { *mant = 1.0L; *ex = 0; return; }
    if (x == 0.0L) { *mant = 0.0L; *ex = 0; return; }
    int e;
    ld f = frexpl(x, &e);               /* x = f 2^e, f in [0.5, 1) */
    *mant = powl(f, (ld)n);             /* >= 2^-n, inside long double range */
    *ex = (long)e * n;
}

/* out[l - l0] = d^l_{mp,m}(theta) for l = l0 .. lmax, l0 = max(|mp|, |m|).
 * Start: the closed form
 *   d^j_{j,k}(t) = (-1)^{j-k} sqrt(C(2j, j+k)) cos^{j+k}(t/2) sin^{j-k}(t/2)
 * moved to the other edges with d^l_{a,b} = (-1)^{a-b} d^l_{b,a} = d^l_{-b,-a};
 * then the three-term recurrence in l
 *   (l-1) sqrt((l^2-m^2)(l^2-mp^2)) d^l = (2l-1)(l(l-1) cos t - m mp) d^{l-1}
 *                                      - l sqrt(((l-1)^2-m^2)((l-1)^2-mp^2)) d^{l-2}. */
static void wigner_d(int lmax, int mp, int m, ld cth, ld chalf, ld shalf, ld* out)
{
    int amp = abs(mp), am = abs(m);
    int j = amp > am ? amp : am;
    if (j > lmax) return;
    int k, a, b, neg;
    if (mp == j)       { k = j + m;  a = j + m;  b = j - m;  neg = (j - m) & 1; }
    else if (mp == -j) { k = j - m;  a = j - m;  b = j + m;  neg = 0; }
    else if (m == j)   { k = j + mp; a = j + mp; b = j - mp; neg = 0; }
    else               { k = j - mp; a = j - mp; b = j + mp; neg = (j + mp) & 1; }
    /* sqrt(C(2j, k)) in scaled form */
    int kk = k < 2 * j - k ? k : 2 * j - k;
    ld v = 1.0L; long E = 0; int ex;
    for (int i = 1; i <= kk; i++) {
        v *= (ld)(2 * j - kk + i) / (ld)i;
        v = frexpl(v, &ex); E += ex;
    }
    if (E & 1) { v *= 2.0L; E -= 1; }
    v = sqrtl(v); E /= 2;
    ld pm; long pe;
    spow(chalf, a, &pm, &pe); v *= pm; E += pe;
    spow(shalf, b, &pm, &pe); v *= pm; E += pe;
    v = frexpl(v, &ex); E += ex;
    if (neg) v = -v;
    out[0] = ldexpl(v, (int)(E < -40000 ? -40000 : E));
    if (lmax == j) return;
    ld prev = 0.0L, cur = v;
    int lstart = j + 1;
    if (j == 0) {                      /* m = mp = 0: d^1_00 = cos(t) */
        prev = cur;
        cur = cth * prev;
        out[1] = ldexpl(cur, (int)E);
        lstart = 2;
    }
    ld M = m, MP = mp;
    for (int l = lstart; l <= lmax; l++) {
        ld L = l;
        ld c1 = (2.0L * L - 1.0L) * (L * (L - 1.0L) * cth - M * MP);
        ld c2 = L * sqrtl(((L - 1) * (L - 1) - M * M) * ((L - 1) * (L - 1) - MP * MP));
        ld den = (L - 1.0L) * sqrtl((L * L - M * M) * (L * L - MP * MP));
        ld nxt = (c1 * cur - c2 * prev) / den;
        prev = cur;
        cur = nxt;
        if (fabsl(cur) > 0x1p64L) {
            cur = ldexpl(cur, -64);
            prev = ldexpl(prev, -64);
            E += 64;
        }
        long Ec = E < -40000 ? -40000 : E;
        out[l - j] = ldexpl(cur, (int)Ec);
    }
}

/* theta part of sY_lm: out[l - l0] = (-1)^m sqrt((2l+1)/4pi) d^l_{-m,s}(theta),
 * l0 = max(|m|, |s|). */
static void slambda(int lmax, int m, int s, ld cth, ld chalf, ld shalf, ld* out)
{
    int l0 = abs(m) > abs(s) ? abs(m) : abs(s);
    if (l0 > lmax) return;
    wigner_d(lmax, -m, s, cth, chalf, shalf, out);
    ld sg = (m & 1) ? -1.0L : 1.0L;
    for (int l = l0; l <= lmax; l++)
        out[l - l0] *= sg * sqrtl((2.0L * l + 1.0L) / (4.0L * PI_L));
}

/* ------------------------------------------------------------------ */
/* exported harmonic evaluators (tests)                               */
/* ------------------------------------------------------------------ */
/* lambda_lm(theta_t) via the Legendre recurrence, out[t][idx(l,m)] (double). */
void oracle_lambda_theta(int lmax, int mmax, int ntheta, const double* theta, double* out)
{
    long long nalm = oracle_nalm(lmax, mmax);
#pragma omp parallel
    {
        ld* buf = (ld*)malloc(sizeof(ld) * (lmax + 1));
#pragma omp for schedule(dynamic)
        for (int t = 0; t < ntheta; t++) {
            ld th = theta[t];
            ld c = cosl(th), s = sinl(th);
            for (int m = 0; m <= mmax; m++) {
                lambda_lm(lmax, m, c, s, buf);
                for (int l = m; l <= lmax; l++)
                    out[(long long)t * nalm + aidx(lmax, l, m)] = (double)buf[l - m];
            }
        }
        free(buf);
    }
}

/* Spin-s theta part via Wigner d, for m = -mmax..mmax:
 * out[t][(m + mmax) * (lmax+1) + l], zero where l < max(|m|,|s|). */
void oracle_slambda_theta(int lmax, int mmax, int s, int ntheta, const double* theta, double* out)
{
    long long stride = (long long)(2 * mmax + 1) * (lmax + 1);
#pragma omp parallel
    {
        ld* buf = (ld*)malloc(sizeof(ld) * (lmax + 1));
#pragma omp for schedule(dynamic)
        for (int t = 0; t < ntheta; t++) {
            ld th = theta[t];
            ld c = cosl(th), ch = cosl(0.5L * th), sh = sinl(0.5L * th);
            double* o = out + (long long)t * stride;
            memset(o, 0, sizeof(double) * stride);
            for (int m = -mmax; m <= mmax; m++) {
                int l0 = abs(m) > abs(s) ? abs(m) : abs(s);
                if (l0 > lmax) continue;
                slambda(lmax, m, s, c, ch, sh, buf);
                for (int l = l0; l <= lmax; l++)
                    o[(long long)(m + mmax) * (lmax + 1) + l] = (double)buf[l - l0];
            }
        }
        free(buf);
    }
}

/* ------------------------------------------------------------------ */
/* brute force: every pixel evaluates its own harmonics               */
/* ------------------------------------------------------------------ */
static void pix_ring(int nside, long long p, ring_t* r, int* k)
{
    /* find the ring holding pixel p by walking the ring table */
    int nr = 4 * nside - 1;
    int lo = 1, hi = nr;
    while (lo < hi) {              /* last ring whose start <= p */
        int mid = (lo + hi + 1) / 2;
        ring_t t;
        ring_geom(nside, mid, &t);
        if (t.start <= p) lo = mid; else hi = mid - 1;
    }
    ring_geom(nside, lo, r);
    *k = (int)(p - r->start);
}

void oracle_alm2map_brute(int nside, int lmax, int mmax, int spin, int nmaps,
                          const double* alm, double* map)
{
    long long npix = oracle_npix(nside);
    long long nalm = oracle_nalm(lmax, mmax);
    int ncomp = spin ? 2 : 1;
#pragma omp parallel
    {
        ld* lp = (ld*)malloc(sizeof(ld) * (lmax + 1));
        ld* lm = (ld*)malloc(sizeof(ld) * (lmax + 1));
#pragma omp for schedule(dynamic, 16)
        for (long long p = 0; p < npix; p++) {
            ring_t r; int k;
            pix_ring(nside, p, &r, &k);
            ld phi = r.phi0 + 2.0L * PI_L * k / r.n;
            for (int j = 0; j < nmaps; j++) {
                if (spin == 0) {
                    const double* a = alm + (long long)j * nalm * 2;
                    ld T = 0.0L;
                    for (int m = 0; m <= mmax; m++) {
                        lambda_lm(lmax, m, r.cth, r.sth, lp);
                        ld cr = cosl(m * phi), ci = sinl(m * phi);
                        for (int l = m; l <= lmax; l++) {
                            const double* c = a + 2 * aidx(lmax, l, m);
                            if (m == 0) T += (ld)c[0] * lp[l - m];
                            else T += 2.0L * lp[l - m] * ((ld)c[0] * cr - (ld)c[1] * ci);
                        }
                    }
                    map[(long long)j * npix + p] = (double)T;
                } else {
                    const double* aE = alm + ((long long)j * 2 + 0) * nalm * 2;
                    const double* aB = alm + ((long long)j * 2 + 1) * nalm * 2;
                    ld Pr = 0.0L, Pi = 0.0L;          /* Q + iU */
                    for (int m = -mmax; m <= mmax; m++) {
                        int am = abs(m);
                        int l0 = am > 2 ? am : 2;
                        if (l0 > lmax) continue;
                        slambda(lmax, m, 2, r.cth, r.chalf, r.shalf, lp);
                        ld cr = cosl(m * phi), ci = sinl(m * phi);
                        for (int l = l0; l <= lmax; l++) {
                            const double* e = aE + 2 * aidx(lmax, l, am);
                            const double* b = aB + 2 * aidx(lmax, l, am);
                            ld er = e[0], ei = e[1], br = b[0], bi = b[1];
                            if (m == 0) { ei = 0.0L; bi = 0.0L; }
                            if (m < 0) {   /* a_{X,l,-m} = (-1)^m conj(a_{X,lm}) */
                                ld sg = (am & 1) ? -1.0L : 1.0L;
                                er = sg * er; ei = -sg * ei; br = sg * br; bi = -sg * bi;
                            }
                            /* a_2 = -(a_E + i a_B) */
                            ld a2r = -(er - bi), a2i = -(ei + br);
                            ld y = lp[l - l0];
                            Pr += y * (a2r * cr - a2i * ci);
                            Pi += y * (a2r * ci + a2i * cr);
                        }
                    }
                    map[((long long)j * 2 + 0) * npix + p] = (double)Pr;
                    map[((long long)j * 2 + 1) * npix + p] = (double)Pi;
                }
            }
        }
        free(lp); free(lm);
    }
    (void)ncomp;
}

void oracle_map2alm_brute(int nside, int lmax, int mmax, int spin, int nmaps,
                          const double* map, double* alm)
{
    long long npix = oracle_npix(nside);
    long long nalm = oracle_nalm(lmax, mmax);
    int ncomp = spin ? 2 : 1;
    ld dsig = 4.0L * PI_L / (ld)npix;
    long long nacc = (long long)nmaps * ncomp * nalm * 2;   /* spin 2: a_{+2}, a_{-2} */
    ld* acc = (ld*)calloc(nacc, sizeof(ld));
#pragma omp parallel
    {
        ld* loc = (ld*)calloc(nacc, sizeof(ld));
        ld* lp = (ld*)malloc(sizeof(ld) * (lmax + 1));
        ld* lq = (ld*)malloc(sizeof(ld) * (lmax + 1));
#pragma omp for schedule(dynamic, 16)
        for (long long p = 0; p < npix; p++) {
            ring_t r; int k;
            pix_ring(nside, p, &r, &k);
            ld phi = r.phi0 + 2.0L * PI_L * k / r.n;
            for (int m = 0; m <= mmax; m++) {
                ld cr = cosl(m * phi), ci = -sinl(m * phi);    /* e^{-i m phi} */
                if (spin == 0) {
                    lambda_lm(lmax, m, r.cth, r.sth, lp);
                    for (int j = 0; j < nmaps; j++) {
                        ld T = map[(long long)j * npix + p];
                        ld* o = loc + (long long)j * nalm * 2;
                        for (int l = m; l <= lmax; l++) {
                            long long q = aidx(lmax, l, m);
                            o[2 * q] += T * lp[l - m] * cr;
                            o[2 * q + 1] += T * lp[l - m] * ci;
                        }
                    }
                } else {
                    int l0 = m > 2 ? m : 2;
                    if (l0 > lmax) continue;
                    slambda(lmax, m, 2, r.cth, r.chalf, r.shalf, lp);   /* +2 */
                    slambda(lmax, m, -2, r.cth, r.chalf, r.shalf, lq);  /* -2 */
                    for (int j = 0; j < nmaps; j++) {
                        ld Q = map[((long long)j * 2 + 0) * npix + p];
                        ld U = map[((long long)j * 2 + 1) * npix + p];
                        ld* o2 = loc + ((long long)j * 2 + 0) * nalm * 2;
                        ld* om = loc + ((long long)j * 2 + 1) * nalm * 2;
                        /* (Q + iU) e^{-i m phi} and (Q - iU) e^{-i m phi} */
                        ld pr = Q * cr - U * ci, pi = Q * ci + U * cr;
                        ld mr = Q * cr + U * ci, mi = Q * ci - U * cr;
                        for (int l = l0; l <= lmax; l++) {
                            long long q = aidx(lmax, l, m);
                            o2[2 * q] += lp[l - l0] * pr;
                            o2[2 * q + 1] += lp[l - l0] * pi;
                            om[2 * q] += lq[l - l0] * mr;
                            om[2 * q + 1] += lq[l - l0] * mi;
                        }
                    }
                }
            }
        }
#pragma omp critical
        for (long long q = 0; q < nacc; q++) acc[q] += loc[q];
        free(loc); free(lp); free(lq);
    }
    for (int j = 0; j < nmaps; j++) {
        if (spin == 0) {
            for (long long q = 0; q < nalm; q++) {
                double* o = alm + ((long long)j * nalm + q) * 2;
                o[0] = (double)(dsig * acc[((long long)j * nalm + q) * 2]);
                o[1] = (double)(dsig * acc[((long long)j * nalm + q) * 2 + 1]);
            }
            for (int l = 0; l <= lmax; l++) alm[((long long)j * nalm + aidx(lmax, l, 0)) * 2 + 1] = 0.0;
        } else {
            const ld* a2 = acc + ((long long)j * 2 + 0) * nalm * 2;
            const ld* am2 = acc + ((long long)j * 2 + 1) * nalm * 2;
            double* oE = alm + ((long long)j * 2 + 0) * nalm * 2;
            double* oB = alm + ((long long)j * 2 + 1) * nalm * 2;
            for (long long q = 0; q < nalm; q++) {
                ld pr = dsig * a2[2 * q], pi = dsig * a2[2 * q + 1];
                ld mr = dsig * am2[2 * q], mi = dsig * am2[2 * q + 1];
                /* a_E = -(a_2 + a_-2)/2 ; a_B = i (a_2 - a_-2)/2 */
                oE[2 * q] = (double)(-0.5L * (pr + mr));
                oE[2 * q + 1] = (double)(-0.5L * (pi + mi));
                oB[2 * q] = (double)(-0.5L * (pi - mi));
                oB[2 * q + 1] = (double)(0.5L * (pr - mr));
            }
            for (int l = 0; l <= lmax; l++) {
                oE[2 * aidx(lmax, l, 0) + 1] = 0.0;
                oB[2 * aidx(lmax, l, 0) + 1] = 0.0;
            }
        }
    }
    free(acc);
}

/* ------------------------------------------------------------------ */
/* separable: lambda per ring, direct per-ring DFT, sum over l        */
/* ------------------------------------------------------------------ */
/* unit-circle table w[k] = e^{+2 pi i k / n}, k = 0..n-1 (double) */
static void circle_table(int n, double* wr, double* wi)
{
    for (int k = 0; k < n; k++) {
        ld a = 2.0L * PI_L * k / n;
        wr[k] = (double)cosl(a);
        wi[k] = (double)sinl(a);
    }
}

/* F[r][m] = sum_n x[start_r + n] e^{-i m (phi0 + 2 pi n / N)}, m = mlo..mhi.
 * Direct DFT: the phase index m n is reduced mod N exactly in integers. */
static void ring_dft_fwd(int nside, const double* x, int mlo, int mhi, double* F)
{
    int nr = 4 * nside - 1;
    int nm = mhi - mlo + 1;
#pragma omp parallel
    {
        double* wr = (double*)malloc(sizeof(double) * 4 * nside);
        double* wi = (double*)malloc(sizeof(double) * 4 * nside);
#pragma omp for schedule(dynamic)
        for (int i = 1; i <= nr; i++) {
            ring_t r;
            ring_geom(nside, i, &r);
            circle_table(r.n, wr, wi);
            const double* xr = x + r.start;
            for (int m = mlo; m <= mhi; m++) {
                int mm = ((m % r.n) + r.n) % r.n;
                double sr = 0.0, si = 0.0;
                long long idx = 0;
                for (int k = 0; k < r.n; k++) {
                    sr += xr[k] * wr[idx];
                    si -= xr[k] * wi[idx];
                    idx += mm; if (idx >= r.n) idx -= r.n;
                }
                ld ph = -(ld)m * r.phi0;
                ld c = cosl(ph), s = sinl(ph);
                double* o = F + ((long long)(i - 1) * nm + (m - mlo)) * 2;
                o[0] = (double)(c * sr - s * si);
                o[1] = (double)(c * si + s * sr);
            }
        }
        free(wr); free(wi);
    }
}

/* One ring of the backward DFT: x[n] = Re (and Im) of
 * sum_m w_m G[m] e^{+i m (phi0 + 2 pi n / N)}, m = mlo..mhi, n = 0..N-1.
 * wr/wi: the ring's unit-circle table; gr/gi: scratch of mhi - mlo + 1. */
static void ring_bwd_one(const ring_t* r, const double* G, int mlo, int mhi, const double* wm,
                         const double* wr, const double* wi, double* gr, double* gi,
                         double* x, double* ximag)
{
    for (int m = mlo; m <= mhi; m++) {              /* fold in e^{i m phi0} and the weight */
        const double* g = G + (long long)(m - mlo) * 2;
        ld ph = (ld)m * r->phi0;
        ld c = cosl(ph), s = sinl(ph);
        gr[m - mlo] = (double)(wm[m - mlo] * (c * g[0] - s * g[1]));
        gi[m - mlo] = (double)(wm[m - mlo] * (c * g[1] + s * g[0]));
    }
    for (int k = 0; k < r->n; k++) {
        double sr = 0.0, si = 0.0;
        long long mm = (((long long)mlo * k) % r->n + r->n) % r->n;   /* m k mod N */
        for (int m = mlo; m <= mhi; m++) {
            sr += gr[m - mlo] * wr[mm] - gi[m - mlo] * wi[mm];
            si += gr[m - mlo] * wi[mm] + gi[m - mlo] * wr[mm];
            mm += k; if (mm >= r->n) mm -= r->n;
        }
        x[k] = sr;
        if (ximag) ximag[k] = si;
    }
}

/* x[start_r + n] = sum_m G[r][m] e^{+i m (phi0 + 2 pi n/N)} with weights:
 * real_out: x = sum over m of Re(w_m G e^{i m phi}) where w_m is supplied per m. */
static void ring_dft_bwd_real(int nside, const double* G, int mlo, int mhi,
                              const double* wm, double* x, double* ximag)
{
    int nr = 4 * nside - 1;
    int nm = mhi - mlo + 1;
#pragma omp parallel
    {
        double* wr = (double*)malloc(sizeof(double) * 4 * nside);
        double* wi = (double*)malloc(sizeof(double) * 4 * nside);
        double* gr = (double*)malloc(sizeof(double) * nm);
        double* gi = (double*)malloc(sizeof(double) * nm);
#pragma omp for schedule(dynamic)
        for (int i = 1; i <= nr; i++) {
            ring_t r;
            ring_geom(nside, i, &r);
            circle_table(r.n, wr, wi);
            ring_bwd_one(&r, G + (long long)(i - 1) * nm * 2, mlo, mhi, wm, wr, wi, gr, gi,
                         x + r.start, ximag ? ximag + r.start : NULL);
        }
        free(wr); free(wi); free(gr); free(gi);
    }
}

/* The sum over l of one m for spin 0 (separable map2alm): om[2 (l - m)] and
 * om[2 (l - m) + 1] receive dsigma sum_rings lambda_lm(ring) F_ring(m), with
 * F_ring(m) at F + ((ring - 1) fstride + fcol) * 2. lp, ar, ai: scratch. */
static void m2a_spin0_m(int nside, int lmax, int m, const double* F, int fstride, int fcol, ld dsig,
                        ld* lp, ld* ar, ld* ai, double* om)
{
    int nr = 4 * nside - 1;
    for (int l = m; l <= lmax; l++) { ar[l] = 0.0L; ai[l] = 0.0L; }
    for (int i = 1; i <= nr; i++) {
        ring_t r;
        ring_geom(nside, i, &r);
        lambda_lm(lmax, m, r.cth, r.sth, lp);
        const double* f = F + ((long long)(i - 1) * fstride + fcol) * 2;
        for (int l = m; l <= lmax; l++) {
            ar[l] += lp[l - m] * f[0];
            ai[l] += lp[l - m] * f[1];
        }
    }
    for (int l = m; l <= lmax; l++) {
        om[2 * (l - m)] = (double)(dsig * ar[l]);
        om[2 * (l - m) + 1] = (m == 0) ? 0.0 : (double)(dsig * ai[l]);
    }
}

/* The same for spin 2: a_{+-2} from F(Q +- iU) and +-2 lambda, then E and B
 * (Sec. 2.3 equ:alm-eb) into oE / oB at [2 (l - m)]; l < 2 is written as 0.
 * lp, lq: scratch of lmax + 1; acc: scratch of 4 (lmax + 1). */
static void m2a_spin2_m(int nside, int lmax, int m, const double* FQ, const double* FU, int fstride,
                        int fcol, ld dsig, ld* lp, ld* lq, ld* acc, double* oE, double* oB)
{
    int nr = 4 * nside - 1;
    int l0 = m > 2 ? m : 2;
    for (int l = m; l <= lmax; l++) {
        oE[2 * (l - m)] = oE[2 * (l - m) + 1] = oB[2 * (l - m)] = oB[2 * (l - m) + 1] = 0.0;
    }
    if (l0 > lmax) return;
    memset(acc, 0, sizeof(ld) * 4 * (lmax + 1));
    for (int i = 1; i <= nr; i++) {
        ring_t r;
        ring_geom(nside, i, &r);
        slambda(lmax, m, 2, r.cth, r.chalf, r.shalf, lp);
        slambda(lmax, m, -2, r.cth, r.chalf, r.shalf, lq);
        const double* fq = FQ + ((long long)(i - 1) * fstride + fcol) * 2;
        const double* fu = FU + ((long long)(i - 1) * fstride + fcol) * 2;
        /* F(Q + iU) and F(Q - iU) */
        ld pr = (ld)fq[0] - fu[1], pi = (ld)fq[1] + fu[0];
        ld mr = (ld)fq[0] + fu[1], mi = (ld)fq[1] - fu[0];
        for (int l = l0; l <= lmax; l++) {
            ld* a = acc + 4 * l;
            a[0] += lp[l - l0] * pr; a[1] += lp[l - l0] * pi;
            a[2] += lq[l - l0] * mr; a[3] += lq[l - l0] * mi;
        }
    }
    for (int l = l0; l <= lmax; l++) {
        ld* a = acc + 4 * l;
        ld pr = dsig * a[0], pi = dsig * a[1], mr = dsig * a[2], mi = dsig * a[3];
        oE[2 * (l - m)] = (double)(-0.5L * (pr + mr));
        oE[2 * (l - m) + 1] = (m == 0) ? 0.0 : (double)(-0.5L * (pi + mi));
        oB[2 * (l - m)] = (double)(-0.5L * (pi - mi));
        oB[2 * (l - m) + 1] = (m == 0) ? 0.0 : (double)(0.5L * (pr - mr));
    }
}

void oracle_map2alm_sep(int nside, int lmax, int mmax, int spin, int nmaps,
                        const double* map, double* alm)
{
    long long npix = oracle_npix(nside);
    long long nalm = oracle_nalm(lmax, mmax);
    int nr = 4 * nside - 1;
    ld dsig = 4.0L * PI_L / (ld)npix;
    int nm = mmax + 1;
    double* FQ = (double*)malloc(sizeof(double) * 2 * (size_t)nr * nm);
    double* FU = spin ? (double*)malloc(sizeof(double) * 2 * (size_t)nr * nm) : NULL;
    for (int j = 0; j < nmaps; j++) {
        if (spin == 0) {
            ring_dft_fwd(nside, map + (long long)j * npix, 0, mmax, FQ);
            double* o = alm + (long long)j * nalm * 2;
#pragma omp parallel
            {
                ld* lp = (ld*)malloc(sizeof(ld) * (lmax + 1));
                ld* ar = (ld*)malloc(sizeof(ld) * (lmax + 1));
                ld* ai = (ld*)malloc(sizeof(ld) * (lmax + 1));
#pragma omp for schedule(dynamic)
                for (int m = 0; m <= mmax; m++)
                    m2a_spin0_m(nside, lmax, m, FQ, nm, m, dsig, lp, ar, ai, o + 2 * aidx(lmax, m, m));
                free(lp); free(ar); free(ai);
            }
        } else {
            ring_dft_fwd(nside, map + ((long long)j * 2 + 0) * npix, 0, mmax, FQ);
            ring_dft_fwd(nside, map + ((long long)j * 2 + 1) * npix, 0, mmax, FU);
            double* oE = alm + ((long long)j * 2 + 0) * nalm * 2;
            double* oB = alm + ((long long)j * 2 + 1) * nalm * 2;
#pragma omp parallel
            {
                ld* lp = (ld*)malloc(sizeof(ld) * (lmax + 1));
                ld* lq = (ld*)malloc(sizeof(ld) * (lmax + 1));
                ld* acc = (ld*)malloc(sizeof(ld) * 4 * (lmax + 1));
#pragma omp for schedule(dynamic)
                for (int m = 0; m <= mmax; m++)
                    m2a_spin2_m(nside, lmax, m, FQ, FU, nm, m, dsig, lp, lq, acc,
                                oE + 2 * aidx(lmax, m, m), oB + 2 * aidx(lmax, m, m));
                free(lp); free(lq); free(acc);
            }
        }
    }
    free(FQ);
    if (FU) free(FU);
}

/* G of one ring for the separable alm2map (before the backward DFT).
 * spin 0: G[m] = sum_l a_lm lambda_lm(ring), m = 0..mmax (Im of m = 0 dropped);
 * spin 2: G[m + mmax] = sum_l a_{2,lm} 2lambda_lm(ring), m = -mmax..mmax, with
 * a_{2,lm} = -(a_E + i a_B) and a_{X,l,-m} = (-1)^m conj(a_{X,lm}). lp: scratch. */
static void a2m_ring_G(int lmax, int mmax, int spin, const ring_t* r, const double* a, const double* aB,
                       ld* lp, double* G)
{
    if (spin == 0) {
        for (int m = 0; m <= mmax; m++) {
            lambda_lm(lmax, m, r->cth, r->sth, lp);
            ld sr = 0.0L, si = 0.0L;
            for (int l = m; l <= lmax; l++) {
                const double* c = a + 2 * aidx(lmax, l, m);
                sr += lp[l - m] * c[0];
                if (m) si += lp[l - m] * c[1];
            }
            G[2 * m] = (double)sr; G[2 * m + 1] = (double)si;
        }
        return;
    }
    for (int m = -mmax; m <= mmax; m++) {
        int am = abs(m);
        int l0 = am > 2 ? am : 2;
        ld sr = 0.0L, si = 0.0L;
        if (l0 <= lmax) {
            slambda(lmax, m, 2, r->cth, r->chalf, r->shalf, lp);
            for (int l = l0; l <= lmax; l++) {
                const double* e = a + 2 * aidx(lmax, l, am);
                const double* b = aB + 2 * aidx(lmax, l, am);
                ld er = e[0], ei = e[1], br = b[0], bi = b[1];
                if (m == 0) { ei = 0.0L; bi = 0.0L; }
                if (m < 0) {
                    ld sg = (am & 1) ? -1.0L : 1.0L;
                    er = sg * er; ei = -sg * ei; br = sg * br; bi = -sg * bi;
                }
                ld a2r = -(er - bi), a2i = -(ei + br);
                sr += lp[l - l0] * a2r;
                si += lp[l - l0] * a2i;
            }
        }
        G[2 * (m + mmax)] = (double)sr; G[2 * (m + mmax) + 1] = (double)si;
    }
}

void oracle_alm2map_sep(int nside, int lmax, int mmax, int spin, int nmaps,
                        const double* alm, double* map)
{
    long long npix = oracle_npix(nside);
    long long nalm = oracle_nalm(lmax, mmax);
    int nr = 4 * nside - 1;
    int nm = spin ? 2 * mmax + 1 : mmax + 1;
    int mlo = spin ? -mmax : 0;
    double* G = (double*)malloc(sizeof(double) * 2 * (size_t)nr * nm);
    double* wm = (double*)malloc(sizeof(double) * nm);
    for (int k = 0; k < nm; k++) wm[k] = (spin || k == 0) ? 1.0 : 2.0;
    for (int j = 0; j < nmaps; j++) {
        const double* a = alm + (long long)j * (spin ? 2 : 1) * nalm * 2;
        const double* aB = spin ? a + nalm * 2 : NULL;
#pragma omp parallel
        {
            ld* lp = (ld*)malloc(sizeof(ld) * (lmax + 1));
#pragma omp for schedule(dynamic)
            for (int i = 1; i <= nr; i++) {
                ring_t r;
                ring_geom(nside, i, &r);
                a2m_ring_G(lmax, mmax, spin, &r, a, aB, lp, G + (long long)(i - 1) * nm * 2);
            }
            free(lp);
        }
        if (spin == 0)
            ring_dft_bwd_real(nside, G, 0, mmax, wm, map + (long long)j * npix, NULL);
        else
            ring_dft_bwd_real(nside, G, mlo, mmax, wm, map + ((long long)j * 2 + 0) * npix,
                              map + ((long long)j * 2 + 1) * npix);
    }
    free(G); free(wm);
}

/* Sampled outputs of the separable tier, for checks at sizes where the full
 * transform is too slow; every value is the same formula as above.
 *
 * map2alm restricted to the orders ms[0..nsel-1]: out [nmaps][ncomp][K][2]
 * with K = sum_k (lmax - ms[k] + 1), the coefficients l = m..lmax of each
 * selected m in selection order. */
void oracle_map2alm_msel(int nside, int lmax, int mmax, int spin, int nmaps, const double* map,
                         int nsel, const int* ms, double* out)
{
    long long npix = oracle_npix(nside);
    int nr = 4 * nside - 1;
    int ncomp = spin ? 2 : 1;
    ld dsig = 4.0L * PI_L / (ld)npix;
    long long K = 0;
    long long* off = (long long*)malloc(sizeof(long long) * (nsel + 1));
    for (int k = 0; k < nsel; k++) { off[k] = K; K += lmax - ms[k] + 1; }
    double* FQ = (double*)malloc(sizeof(double) * 2 * (size_t)nr * nsel);
    double* FU = (double*)malloc(sizeof(double) * 2 * (size_t)nr * nsel);
    double* col = (double*)malloc(sizeof(double) * 2 * (size_t)nr);
    (void)mmax;
    for (int j = 0; j < nmaps; j++) {
        for (int c = 0; c < ncomp; c++) {
            double* F = c ? FU : FQ;
            for (int k = 0; k < nsel; k++) {        /* F[ring][k] for the selected orders */
                ring_dft_fwd(nside, map + ((long long)j * ncomp + c) * npix, ms[k], ms[k], col);
                for (int i = 0; i < nr; i++) {
                    F[((long long)i * nsel + k) * 2] = col[2 * i];
                    F[((long long)i * nsel + k) * 2 + 1] = col[2 * i + 1];
                }
            }
        }
#pragma omp parallel
        {
            ld* lp = (ld*)malloc(sizeof(ld) * (lmax + 1));
            ld* lq = (ld*)malloc(sizeof(ld) * (lmax + 1));
            ld* acc = (ld*)malloc(sizeof(ld) * 4 * (lmax + 1));
#pragma omp for schedule(dynamic)
            for (int k = 0; k < nsel; k++) {
                double* o0 = out + (((long long)j * ncomp + 0) * K + off[k]) * 2;
                if (spin == 0) {
                    m2a_spin0_m(nside, lmax, ms[k], FQ, nsel, k, dsig, lp, lq, acc, o0);
                } else {
                    double* o1 = out + (((long long)j * ncomp + 1) * K + off[k]) * 2;
                    m2a_spin2_m(nside, lmax, ms[k], FQ, FU, nsel, k, dsig, lp, lq, acc, o0, o1);
                }
            }
            free(lp); free(lq); free(acc);
        }
    }
    free(FQ); free(FU); free(col); free(off);
}

/* alm2map restricted to the rings rings[0..nsel-1] (1-based): out
 * [nmaps][ncomp][P] with P = sum_k N(rings[k]), the pixels of each selected
 * ring in RING order, rings in selection order. */
void oracle_alm2map_rings(int nside, int lmax, int mmax, int spin, int nmaps, const double* alm,
                          int nsel, const int* rings, double* out)
{
    long long nalm = oracle_nalm(lmax, mmax);
    int ncomp = spin ? 2 : 1;
    int nm = spin ? 2 * mmax + 1 : mmax + 1;
    int mlo = spin ? -mmax : 0;
    long long P = 0;
    long long* off = (long long*)malloc(sizeof(long long) * (nsel + 1));
    for (int k = 0; k < nsel; k++) {
        ring_t r;
        ring_geom(nside, rings[k], &r);
        off[k] = P;
        P += r.n;
    }
    double* wm = (double*)malloc(sizeof(double) * nm);
    for (int k = 0; k < nm; k++) wm[k] = (spin || k == 0) ? 1.0 : 2.0;
    for (int j = 0; j < nmaps; j++) {
        const double* a = alm + (long long)j * ncomp * nalm * 2;
        const double* aB = spin ? a + nalm * 2 : NULL;
#pragma omp parallel
        {
            ld* lp = (ld*)malloc(sizeof(ld) * (lmax + 1));
            double* G = (double*)malloc(sizeof(double) * 2 * nm);
            double* wr = (double*)malloc(sizeof(double) * 4 * nside);
            double* wi = (double*)malloc(sizeof(double) * 4 * nside);
            double* gr = (double*)malloc(sizeof(double) * nm);
            double* gi = (double*)malloc(sizeof(double) * nm);
#pragma omp for schedule(dynamic)
            for (int k = 0; k < nsel; k++) {
                ring_t r;
                ring_geom(nside, rings[k], &r);
                a2m_ring_G(lmax, mmax, spin, &r, a, aB, lp, G);
                circle_table(r.n, wr, wi);
                double* x0 = out + ((long long)j * ncomp + 0) * P + off[k];
                double* x1 = spin ? out + ((long long)j * ncomp + 1) * P + off[k] : NULL;
                ring_bwd_one(&r, G, mlo, spin ? mmax : mmax, wm, wr, wi, gr, gi, x0, x1);
            }
            free(lp); free(G); free(wr); free(wi); free(gr); free(gi);
        }
    }
    free(wm); free(off);
}

/* Traditional (Jacobi) iteration, Algorithm 2, in its pixel-domain form:
 * a^0 = map2alm(T); a^{n+1} = a^n + map2alm(T - alm2map(a^n)). */
void oracle_map2alm_iter(int nside, int lmax, int mmax, int spin, int nmaps,
                         const double* map, double* alm, int niter)
{
    long long npix = oracle_npix(nside);
    long long nalm = oracle_nalm(lmax, mmax);
    int ncomp = spin ? 2 : 1;
    long long nm = (long long)nmaps * ncomp * npix;
    long long na = (long long)nmaps * ncomp * nalm * 2;
    oracle_map2alm_sep(nside, lmax, mmax, spin, nmaps, map, alm);
    if (niter <= 0) return;
    double* res = (double*)malloc(sizeof(double) * nm);
    double* da = (double*)malloc(sizeof(double) * na);
    for (int it = 0; it < niter; it++) {
        oracle_alm2map_sep(nside, lmax, mmax, spin, nmaps, alm, res);
        for (long long q = 0; q < nm; q++) res[q] = map[q] - res[q];
        oracle_map2alm_sep(nside, lmax, mmax, spin, nmaps, res, da);
        for (long long q = 0; q < na; q++) alm[q] += da[q];
    }
    free(res); free(da);
}

/* Immediate (Gauss-Seidel) iteration, Algorithm 3, spin 0. The ring
 * spectra F of the residual map S - alm2map(a) are kept per ring (the full
 * DFT, bins j = 0..N-1, no phase). Each pass walks m = 0..mmax in order:
 *   T_m(ring)  = e^{-i m phi0} F_{m mod N}                 (remap)
 *   c_lm       = dsigma sum_rings lambda_lm T_m             (this order's correction)
 *   a_lm      += c_lm                                       (updated at once)
 *   S_m(ring)  = sum_l c_lm lambda_lm                       (its synthesis)
 *   F_{ m mod N} -= (w_m / 2) N S_m e^{+i m phi0},
 *   F_{-m mod N} -= (w_m / 2) N conj(S_m) e^{-i m phi0}     (w_0 = 1, w_m = 2)
 * so every later order sharing a bin with m (aliasing on rings with
 * N <= 2 mmax) already sees the update. a starts at 0 and F at the DFT of
 * the map; npass >= 1 passes (npass = 1 is one sweep, not the plain
 * quadrature: without aliasing the two coincide). */
void oracle_map2alm_immediate(int nside, int lmax, int mmax, int nmaps, const double* map, double* alm,
                              int npass)
{
    long long npix = oracle_npix(nside);
    long long nalm = oracle_nalm(lmax, mmax);
    int nr = 4 * nside - 1;
    ld dsig = 4.0L * PI_L / (ld)npix;
    ld* F = (ld*)malloc(sizeof(ld) * 2 * (size_t)npix);      /* ring r's bins at start_r */
    ld* lam = (ld*)malloc(sizeof(ld) * (size_t)nr * (lmax + 1));
    ld* c = (ld*)malloc(sizeof(ld) * 2 * (lmax + 1));
    ring_t* rg = (ring_t*)malloc(sizeof(ring_t) * nr);
    for (int i = 1; i <= nr; i++) ring_geom(nside, i, &rg[i - 1]);
    for (int j = 0; j < nmaps; j++) {
        const double* x = map + (long long)j * npix;
        double* o = alm + (long long)j * nalm * 2;
        memset(o, 0, sizeof(double) * 2 * nalm);
#pragma omp parallel for schedule(dynamic)
        for (int i = 0; i < nr; i++) {                      /* F = DFT of each ring */
            const ring_t* r = &rg[i];
            for (int b = 0; b < r->n; b++) {
                ld sr = 0.0L, si = 0.0L;
                for (int k = 0; k < r->n; k++) {
                    long long t = ((long long)b * k) % r->n;
                    ld a = -2.0L * PI_L * (ld)t / r->n;
                    sr += x[r->start + k] * cosl(a);
                    si += x[r->start + k] * sinl(a);
                }
                F[2 * (r->start + b)] = sr;
                F[2 * (r->start + b) + 1] = si;
            }
        }
        for (int pass = 0; pass < npass; pass++) {
            for (int m = 0; m <= mmax; m++) {
                int nl = lmax - m + 1;
#pragma omp parallel for schedule(dynamic)
                for (int i = 0; i < nr; i++)
                    lambda_lm(lmax, m, rg[i].cth, rg[i].sth, lam + (long long)i * (lmax + 1));
                /* remap and correction */
                for (int l = 0; l < nl; l++) { c[2 * l] = 0.0L; c[2 * l + 1] = 0.0L; }
                for (int i = 0; i < nr; i++) {
                    const ring_t* r = &rg[i];
                    int b = m % r->n;
                    ld fr = F[2 * (r->start + b)], fi = F[2 * (r->start + b) + 1];
                    ld ph = -(ld)m * r->phi0, cph = cosl(ph), sph = sinl(ph);
                    ld tr = cph * fr - sph * fi, ti = cph * fi + sph * fr;
                    const ld* lp = lam + (long long)i * (lmax + 1);
                    for (int l = 0; l < nl; l++) { c[2 * l] += lp[l] * tr; c[2 * l + 1] += lp[l] * ti; }
                }
                for (int l = 0; l < nl; l++) {
                    c[2 * l] *= dsig;
                    c[2 * l + 1] = (m == 0) ? 0.0L : c[2 * l + 1] * dsig;
                    long long q = aidx(lmax, m + l, m);
                    o[2 * q] += (double)c[2 * l];
                    o[2 * q + 1] += (double)c[2 * l + 1];
                }
                /* synthesis of the correction, removed from the residual's bins */
                ld w = (m == 0) ? 1.0L : 2.0L;
                for (int i = 0; i < nr; i++) {
                    const ring_t* r = &rg[i];
                    const ld* lp = lam + (long long)i * (lmax + 1);
                    ld sr = 0.0L, si = 0.0L;
                    for (int l = 0; l < nl; l++) { sr += lp[l] * c[2 * l]; si += lp[l] * c[2 * l + 1]; }
                    ld ph = (ld)m * r->phi0, cph = cosl(ph), sph = sinl(ph);
                    ld ur = cph * sr - sph * si, ui = cph * si + sph * sr;     /* S e^{i m phi0} */
                    ld f = 0.5L * w * (ld)r->n;
                    int b1 = m % r->n, b2 = (r->n - b1) % r->n;
                    F[2 * (r->start + b1)] -= f * ur;
                    F[2 * (r->start + b1) + 1] -= f * ui;
                    F[2 * (r->start + b2)] -= f * ur;
                    F[2 * (r->start + b2) + 1] += f * ui;
                }
            }
        }
    }
    free(F); free(lam); free(c); free(rg);
}

/* Immediate iteration, Algorithm 3, spin 2 (Q/U -> E/B). The residual
 * map's Q and U rings are kept as their full DFTs FQ, FU (bins 0..N-1, no
 * phase). Each pass walks m = 0..mmax in order:
 *   TQ, TU     = e^{-i m phi0} FQ_{m mod N}, e^{-i m phi0} FU_{m mod N}   (remap)
 *   (cE, cB)_l = the spin-2 quadrature of order m from TQ, TU (as in the
 *                separable map2alm: F(Q +- iU) against +-2 lambda, Sec. 2.3)
 *   a_E, a_B  += cE, cB                                                  (at once)
 *   G_m'       = sum_l c_{2,l,m'} 2lambda_{l,m'}, m' = m and -m, with
 *                c_{2,lm} = -(cE + i cB), c_{X,l,-m} = (-1)^m conj(c_{X,lm})
 *                (the correction's Q + iU at order m')
 *   for each m' (once for m = 0), g = N G_m' e^{i m' phi0} (its DFT bin):
 *     FQ_{m'} -= g / 2,   FQ_{-m'} -= conj(g) / 2      (Q = Re of Q + iU)
 *     FU_{m'} -= g / 2i,  FU_{-m'} += conj(g) / 2i     (U = Im of Q + iU)
 * so every later order sharing a bin sees the update. a starts at 0 and the
 * residual at the map; npass >= 1 passes. map [nmaps][2][npix] (Q, U),
 * alm [nmaps][2][nalm] (E, B). */
void oracle_map2alm_immediate2(int nside, int lmax, int mmax, int nmaps, const double* map, double* alm,
                               int npass)
{
    long long npix = oracle_npix(nside);
    long long nalm = oracle_nalm(lmax, mmax);
    int nr = 4 * nside - 1;
    ld dsig = 4.0L * PI_L / (ld)npix;
    ld* FQ = (ld*)malloc(sizeof(ld) * 2 * (size_t)npix);
    ld* FU = (ld*)malloc(sizeof(ld) * 2 * (size_t)npix);
    ld* lpp = (ld*)malloc(sizeof(ld) * (size_t)nr * (lmax + 1));   /* 2lambda_{l,m} per ring */
    ld* lpm = (ld*)malloc(sizeof(ld) * (size_t)nr * (lmax + 1));   /* -2lambda_{l,m} */
    ld* lnp = (ld*)malloc(sizeof(ld) * (size_t)nr * (lmax + 1));   /* 2lambda_{l,-m} */
    ld* acc = (ld*)malloc(sizeof(ld) * 4 * (lmax + 1));
    ld* ce = (ld*)malloc(sizeof(ld) * 4 * (lmax + 1));             /* cE (re, im), cB (re, im) */
    ring_t* rg = (ring_t*)malloc(sizeof(ring_t) * nr);
    for (int i = 1; i <= nr; i++) ring_geom(nside, i, &rg[i - 1]);
    for (int j = 0; j < nmaps; j++) {
        const double* xq = map + ((long long)j * 2 + 0) * npix;
        const double* xu = map + ((long long)j * 2 + 1) * npix;
        double* oE = alm + ((long long)j * 2 + 0) * nalm * 2;
        double* oB = alm + ((long long)j * 2 + 1) * nalm * 2;
        memset(oE, 0, sizeof(double) * 2 * nalm);
        memset(oB, 0, sizeof(double) * 2 * nalm);
#pragma omp parallel for schedule(dynamic)
        for (int i = 0; i < nr; i++) {                      /* FQ, FU = DFT of each ring */
            const ring_t* r = &rg[i];
            for (int b = 0; b < r->n; b++) {
                ld qr = 0.0L, qi = 0.0L, ur = 0.0L, ui = 0.0L;
                for (int k = 0; k < r->n; k++) {
                    long long t = ((long long)b * k) % r->n;
                    ld a = -2.0L * PI_L * (ld)t / r->n, ca = cosl(a), sa = sinl(a);
                    qr += xq[r->start + k] * ca; qi += xq[r->start + k] * sa;
                    ur += xu[r->start + k] * ca; ui += xu[r->start + k] * sa;
                }
                FQ[2 * (r->start + b)] = qr; FQ[2 * (r->start + b) + 1] = qi;
                FU[2 * (r->start + b)] = ur; FU[2 * (r->start + b) + 1] = ui;
            }
        }
        for (int pass = 0; pass < npass; pass++) {
            for (int m = 0; m <= mmax; m++) {
                int l0 = m > 2 ? m : 2;
                if (l0 > lmax) continue;                     /* no coefficient of this order */
                int nl = lmax - l0 + 1;
#pragma omp parallel for schedule(dynamic)
                for (int i = 0; i < nr; i++) {
                    slambda(lmax, m, 2, rg[i].cth, rg[i].chalf, rg[i].shalf, lpp + (long long)i * (lmax + 1));
                    slambda(lmax, m, -2, rg[i].cth, rg[i].chalf, rg[i].shalf, lpm + (long long)i * (lmax + 1));
                    slambda(lmax, -m, 2, rg[i].cth, rg[i].chalf, rg[i].shalf, lnp + (long long)i * (lmax + 1));
                }
                /* remap and this order's correction */
                memset(acc, 0, sizeof(ld) * 4 * (lmax + 1));
                for (int i = 0; i < nr; i++) {
                    const ring_t* r = &rg[i];
                    int b = m % r->n;
                    ld ph = -(ld)m * r->phi0, cph = cosl(ph), sph = sinl(ph);
                    ld fqr = FQ[2 * (r->start + b)], fqi = FQ[2 * (r->start + b) + 1];
                    ld fur = FU[2 * (r->start + b)], fui = FU[2 * (r->start + b) + 1];
                    ld tqr = cph * fqr - sph * fqi, tqi = cph * fqi + sph * fqr;
                    ld tur = cph * fur - sph * fui, tui = cph * fui + sph * fur;
                    ld pr = tqr - tui, pi = tqi + tur;           /* F(Q + iU) */
                    ld mr = tqr + tui, mi = tqi - tur;           /* F(Q - iU) */
                    const ld* p2 = lpp + (long long)i * (lmax + 1);
                    const ld* m2 = lpm + (long long)i * (lmax + 1);
                    for (int l = 0; l < nl; l++) {
                        acc[4 * l] += p2[l] * pr; acc[4 * l + 1] += p2[l] * pi;
                        acc[4 * l + 2] += m2[l] * mr; acc[4 * l + 3] += m2[l] * mi;
                    }
                }
                for (int l = 0; l < nl; l++) {
                    ld pr = dsig * acc[4 * l], pi = dsig * acc[4 * l + 1];
                    ld mr = dsig * acc[4 * l + 2], mi = dsig * acc[4 * l + 3];
                    ld er = -0.5L * (pr + mr), ei = (m == 0) ? 0.0L : -0.5L * (pi + mi);
                    ld br = -0.5L * (pi - mi), bi = (m == 0) ? 0.0L : 0.5L * (pr - mr);
                    ce[4 * l] = er; ce[4 * l + 1] = ei; ce[4 * l + 2] = br; ce[4 * l + 3] = bi;
                    long long q = aidx(lmax, l0 + l, m);
                    oE[2 * q] += (double)er; oE[2 * q + 1] += (double)ei;
                    oB[2 * q] += (double)br; oB[2 * q + 1] += (double)bi;
                }
                /* synthesis of the correction at orders m and -m, removed from
                 * the residual's Q and U bins */
                for (int i = 0; i < nr; i++) {
                    const ring_t* r = &rg[i];
                    for (int sg = 1; sg >= -1; sg -= 2) {
                        if (sg < 0 && m == 0) break;
                        const int mp = sg * m;
                        const ld* lam = ((sg > 0) ? lpp : lnp) + (long long)i * (lmax + 1);
                        ld gr = 0.0L, gi = 0.0L;
                        for (int l = 0; l < nl; l++) {
                            ld er = ce[4 * l], ei = ce[4 * l + 1], br = ce[4 * l + 2], bi = ce[4 * l + 3];
                            if (sg < 0) {
                                ld sgn = (m & 1) ? -1.0L : 1.0L;
                                er = sgn * er; ei = -sgn * ei; br = sgn * br; bi = -sgn * bi;
                            }
                            ld a2r = -(er - bi), a2i = -(ei + br);
                            gr += lam[l] * a2r; gi += lam[l] * a2i;
                        }
                        ld ph = (ld)mp * r->phi0, cph = cosl(ph), sph = sinl(ph);
                        ld n = (ld)r->n;
                        ld g_r = n * (cph * gr - sph * gi), g_i = n * (cph * gi + sph * gr);
                        int b1 = ((mp % r->n) + r->n) % r->n, b2 = (r->n - b1) % r->n;
                        FQ[2 * (r->start + b1)] -= 0.5L * g_r; FQ[2 * (r->start + b1) + 1] -= 0.5L * g_i;
                        FQ[2 * (r->start + b2)] -= 0.5L * g_r; FQ[2 * (r->start + b2) + 1] += 0.5L * g_i;
                        FU[2 * (r->start + b1)] -= 0.5L * g_i; FU[2 * (r->start + b1) + 1] += 0.5L * g_r;
                        FU[2 * (r->start + b2)] -= 0.5L * g_i; FU[2 * (r->start + b2) + 1] -= 0.5L * g_r;
                    }
                }
            }
        }
    }
    free(FQ); free(FU); free(lpp); free(lpm); free(lnp); free(acc); free(ce); free(rg);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
