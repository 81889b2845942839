// plan.cu -- plan creation (ring geometry, lambda recurrence tables, FFT
// tables), workspace accounting, argument validation and the C ABI of
// include/sht.h. Tables are built once on the host in long double and stay
// resident on the device (the paper likewise separates this init overhead
// from the transform time, Sec. 3.3).
#include <cmath>
#include <cstring>
#include <algorithm>
#include <map>
#include <complex>

#include <cstdlib>
#include <climits>
#include "common.cuh"

namespace sht {

static thread_local std::string t_err;
static thread_local int t_launches = 0;
void set_error(const std::string& msg) { t_err = msg; }
void count_launch(int n) { t_launches += n; }
void reset_launches() { t_launches = 0; }

struct ProfRec { std::string name; cudaEvent_t a, b; };
static thread_local bool t_prof = false;
static thread_local std::vector<ProfRec> t_recs;
void prof_start(const char* name, cudaStream_t st)
{
    if (!t_prof) return;
    ProfRec r; r.name = name;
    if (cudaEventCreate(&r.a) != cudaSuccess) return;
    if (cudaEventCreate(&r.b) != cudaSuccess) { cudaEventDestroy(r.a); return; }
    cudaEventRecord(r.a, st);
    t_recs.push_back(r);
}
void prof_stop(cudaStream_t st)
{
    if (!t_prof || t_recs.empty()) return;
    cudaEventRecord(t_recs.back().b, st);
}

typedef long double ld;
static const ld PI_L = 3.141592653589793238462643383279502884L;
static const double PI_D = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// HEALPix RING geometry of ring i (1-based): z, sin(theta), pixels, phi0
// shift flag, first pixel. Caps take sin(theta) from the exact 1 -+ z.
// ---------------------------------------------------------------------------
struct RingH { ld z, s; int n; bool shifted; long long start; };

static RingH ring_h(int nside, int i)
{
    RingH r;
    long long npix = 12LL * nside * nside;
    ld ns = nside;
    if (i < nside) {
        ld omz = (ld)i * i / (3 * ns * ns);
        r.z = 1 - omz; r.s = sqrtl(omz * (2 - omz));
        r.n = 4 * i; r.shifted = true; r.start = 2LL * i * (i - 1);
    } else if (i <= 3 * nside) {
        ld z = (ld)(4 * nside - 2 * i) / (3 * ns);
        r.z = z; r.s = sqrtl((1 - z) * (1 + z));
        r.n = 4 * nside; r.shifted = ((i - nside) % 2 == 0);
        r.start = 2LL * nside * (nside - 1) + 4LL * nside * (i - nside);
    } else {
        int ip = 4 * nside - i;
        ld opz = (ld)ip * ip / (3 * ns * ns);
        r.z = opz - 1; r.s = sqrtl(opz * (2 - opz));
        r.n = 4 * ip; r.shifted = true; r.start = npix - 2LL * ip * (ip + 1);
    }
    return r;
}

static int next_pow2(int v) { int p = 1; while (p < v) p <<= 1; return p; }
static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// in-place iterative radix-2 FFT (host, double), forward sign e^{-2 pi i}
static void host_fft(std::vector<double>& re, std::vector<double>& im)
{
    int n = (int)re.size();
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { std::swap(re[i], re[j]); std::swap(im[i], im[j]); }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int h = len / 2;
        for (int k = 0; k < h; k++) {
            ld a = -2 * PI_L * k / len;
            double wr = (double)cosl(a), wi = (double)sinl(a);
            for (int i = k; i < n; i += len) {
                double xr = re[i + h] * wr - im[i + h] * wi;
                double xi = re[i + h] * wi + im[i + h] * wr;
                re[i + h] = re[i] - xr; im[i + h] = im[i] - xi;
                re[i] += xr; im[i] += xi;
            }
        }
    }
}

static int bitrev(int i, int logm)
{
    int r = 0;
    for (int b = 0; b < logm; b++) if (i & (1 << b)) r |= 1 << (logm - 1 - b);
    return r;
}

// ---- split form: FFT sizes M = 3^b 2^a (2^a >= 64 when b > 0) ----
// relative cost of one size-M transform in the split FFT (double-float
// operations per point: ~29.5 per radix-4 pass, ~16 per radix-2 pass, ~30 per
// radix-3 pass)
static double split_fft_cost(int M)
{
    int b = 0;
    while (M % 3 == 0) { M /= 3; b++; }
    int L = 0;
    while ((1 << L) < M) L++;
    const double p3 = std::pow(3.0, b);
    return p3 * (double)M * ((L / 2) * 29.5 + (L % 2) * 16.0 + b * 30.0);
}

static int pow3_part(int M) { int p = 1; while (M % 3 == 0) { M /= 3; p *= 3; } return p; }

// the split form's recipe for a ring of N pixels: a direct transform when N
// is a power of two or 3^b 2^a (2^a >= 64), else Bluestein with the cheapest
// M = 3^b 2^a >= 2N - 1 (never above the power-of-two size)
static void split_fft_choice(int N, int& M, int& bluestein)
{
    if (is_pow2(N)) { M = N; bluestein = 0; return; }
    double best = 1e300;
    const int p3n = pow3_part(N);
    if (is_pow2(N / p3n) && N / p3n >= 64) { best = split_fft_cost(N); M = N; bluestein = 0; }
    const int cap = next_pow2(2 * N - 1);
    for (int p3 = 1; p3 <= 243; p3 *= 3) {
        int a2 = 1;
        while ((long long)a2 * p3 < 2LL * N - 1) a2 *= 2;
        const int Mc = a2 * p3;
        if (Mc > cap || (p3 > 1 && a2 < 64)) continue;
        const double c = 2.0 * split_fft_cost(Mc) + 30.0 * Mc;
        if (c < best) { best = c; M = Mc; bluestein = 1; }
    }
}

// position of index k in a digit-reversed sequence of M = p3 2^a points (the
// output order of the split FFT's decimation-in-frequency passes: radix-3
// stages first, then the power-of-two passes), and its inverse
static int split_pos_of(int k, int M, int p3)
{
    const int a2 = M / p3;
    int logm = 0;
    while ((1 << logm) < a2) logm++;
    int p = 0, S = M;
    for (int q = p3; q > 1; q /= 3) { S /= 3; p += (k % 3) * S; k /= 3; }
    return p + bitrev(k, logm);
}
static int split_k_of(int p, int M, int p3)
{
    const int a2 = M / p3;
    int logm = 0;
    while ((1 << logm) < a2) logm++;
    int k = 0, mul = 1, S = M;
    for (int q = p3; q > 1; q /= 3) { S /= 3; const int j = p / S; p -= j * S; k += j * mul; mul *= 3; }
    return k + mul * bitrev(p, logm);
}

// forward DFT of n = 3^b 2^a points in long double (recursive decimation in time)
typedef std::complex<ld> cld;
static void host_dft_mixed(std::vector<cld>& x)
{
    const size_t n = x.size();
    if (n == 1) return;
    const int r = (n % 3 == 0) ? 3 : 2;
    const size_t m = n / r;
    std::vector<std::vector<cld>> sub(r, std::vector<cld>(m));
    for (size_t i = 0; i < m; i++)
        for (int j = 0; j < r; j++) sub[j][i] = x[i * r + j];
    for (int j = 0; j < r; j++) host_dft_mixed(sub[j]);
    for (size_t k = 0; k < n; k++) {
        cld acc(0.0L, 0.0L);
        for (int j = 0; j < r; j++) {
            const ld a = -2 * PI_L * (ld)((j * k) % n) / (ld)n;
            acc += sub[j][k % m] * cld(cosl(a), sinl(a));
        }
        x[k] = acc;
    }
}

// scaled long-double value: mant * 2^exp
struct Scaled { ld v; long e; };
static Scaled snorm(ld v, long e)
{
    if (v == 0) return {0, 0};
    int ex; ld f = frexpl(v, &ex);
    return {f, e + ex};
}
static Scaled smul(Scaled a, ld b) { return snorm(a.v * b, a.e); }
static Scaled spow(ld x, int n)   // x >= 0
{
    if (n == 0) return {0.5L, 1};
    if (x == 0) return {0, 0};
    int ex; ld f = frexpl(x, &ex);
    return snorm(powl(f, (ld)n), (long)ex * n);
}
static Scaled sprod(Scaled a, Scaled b) { return snorm(a.v * b.v, a.e + b.e); }

template <typename T>
static cudaError_t upload(T** d, const std::vector<T>& h, size_t* acc)
{
    size_t b = h.size() * sizeof(T);
    if (b == 0) { *d = nullptr; return cudaSuccess; }
    cudaError_t e = cudaMalloc((void**)d, b);
    if (e != cudaSuccess) return e;
    *acc += b;
    return cudaMemcpy(*d, h.data(), b, cudaMemcpyHostToDevice);
}

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------
static cudaError_t build_tables(sht_plan* p)
{
    const int nside = p->nside, lmax = p->lmax, mmax = p->mmax, R = p->R;
    size_t acc = 0;
    cudaError_t e;
    // ---- rings and FFT lengths ----
    std::map<int, int> len_index;
    p->h_pairs.resize(R);
    std::vector<ld> zs(R), ss(R);
    for (int q = 0; q < R; q++) {
        int i = q + 1;
        RingH r = ring_h(nside, i);
        RingH rs = ring_h(nside, 4 * nside - i);
        PairGeom g;
        g.x = (double)r.z; g.s = (double)r.s;
        g.phi0 = r.shifted ? (double)(PI_L / r.n) : 0.0;
        g.start_n = r.start;
        g.start_s = (i == 2 * nside) ? -1 : rs.start;
        g.n = r.n;
        if (!len_index.count(r.n)) { int k = (int)len_index.size(); len_index[r.n] = k; }
        g.fft = len_index[r.n];
        p->h_pairs[q] = g;
        zs[q] = r.z; ss[q] = r.s;
    }
    p->nfft = (int)len_index.size();
    p->h_fft.resize(p->nfft);
    std::vector<double2> chirp, bhat;
    int fftmax = 2;
    for (auto& kv : len_index) {
        int N = kv.first;
        FftLen f;
        f.n = N;
        f.bluestein = is_pow2(N) ? 0 : 1;
        f.m = f.bluestein ? next_pow2(2 * N - 1) : N;
        f.p3 = 1;
        f.chirp = (long long)chirp.size();
        f.bhat = (long long)bhat.size();
        if (f.bluestein) {
            std::vector<double2> w(N);
            for (int n = 0; n < N; n++) {
                long long n2 = ((long long)n * n) % (2LL * N);
                ld a = -PI_L * (ld)n2 / N;
                w[n] = make_double2((double)cosl(a), (double)sinl(a));
                chirp.push_back(w[n]);
            }
            int M = f.m, logm = 0;
            while ((1 << logm) < M) logm++;
            std::vector<double> br(M, 0.0), bi(M, 0.0);
            for (int j = 0; j < N; j++) {
                br[j] = w[j].x; bi[j] = -w[j].y;
                if (j > 0) { br[M - j] = w[j].x; bi[M - j] = -w[j].y; }
            }
            host_fft(br, bi);
            std::vector<double2> b(M);
            for (int i = 0; i < M; i++) { int s = bitrev(i, logm); b[i] = make_double2(br[s], bi[s]); }
            bhat.insert(bhat.end(), b.begin(), b.end());
        }
        fftmax = std::max(fftmax, f.m);
        p->h_fft[kv.second] = f;
    }
    p->fft_max = fftmax;
    std::vector<double2> tw(fftmax / 2);
    for (int t = 0; t < fftmax / 2; t++) {
        ld a = -2 * PI_L * t / fftmax;
        tw[t] = make_double2((double)cosl(a), (double)sinl(a));
    }
    if ((e = upload(&p->t.pairs, p->h_pairs, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->t.fft, p->h_fft, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->t.twiddle, tw, &acc)) != cudaSuccess) return e;
    if (chirp.empty()) chirp.push_back(make_double2(1, 0));
    if (bhat.empty()) bhat.push_back(make_double2(1, 0));
    if ((e = upload(&p->t.chirp, chirp, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->t.bhat, bhat, &acc)) != cudaSuccess) return e;
    if (p->precision != SHT_FP64) {
        // FP32 hi/lo pairs of every FFT table for the compensated FFT
        auto split = [](const std::vector<double2>& v, std::vector<float2>& h, std::vector<float2>& l) {
            h.resize(v.size()); l.resize(v.size());
            for (size_t i = 0; i < v.size(); i++) {
                float hx = (float)v[i].x, hy = (float)v[i].y;
                h[i] = make_float2(hx, hy);
                l[i] = make_float2((float)(v[i].x - (double)hx), (float)(v[i].y - (double)hy));
            }
        };
        std::vector<float2> h, l;
        split(tw, h, l);
        if ((e = upload(&p->t.twiddle_f, h, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->c.twiddle_l, l, &acc)) != cudaSuccess) return e;
        split(chirp, h, l);
        if ((e = upload(&p->t.chirp_f, h, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->c.chirp_l, l, &acc)) != cudaSuccess) return e;
        split(bhat, h, l);
        if ((e = upload(&p->t.bhat_f, h, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->c.bhat_l, l, &acc)) != cudaSuccess) return e;
        // exp(+i pi k / N), k < 2N, for every distinct ring length (long double)
        std::vector<float2> ph, pl;
        std::vector<long long> off(p->nfft);
        for (auto& kv : len_index) {
            int N = kv.first;
            off[kv.second] = (long long)ph.size();
            for (int k = 0; k < 2 * N; k++) {
                ld a = PI_L * k / N;
                ld c = cosl(a), sn = sinl(a);
                float hc = (float)c, hs = (float)sn;
                ph.push_back(make_float2(hc, hs));
                pl.push_back(make_float2((float)(c - hc), (float)(sn - hs)));
            }
        }
        if ((e = upload(&p->c.phase_h, ph, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->c.phase_l, pl, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->c.phase_off, off, &acc)) != cudaSuccess) return e;
        // the split form's own recipes: sizes 3^b 2^a where they need less
        // work, Bluestein filters in the digit-reversed order of its passes
        p->h_fft_s = p->h_fft;
        std::vector<float2> bsh, bsl;
        for (auto& kv : len_index) {
            sht::FftLen& fs = p->h_fft_s[kv.second];
            const int N = kv.first;
            split_fft_choice(N, fs.m, fs.bluestein);
            fs.p3 = pow3_part(fs.m);
            fs.bhat = (long long)bsh.size();
            if (!fs.bluestein) continue;
            const int M = fs.m;
            std::vector<cld> b(M, cld(0.0L, 0.0L));
            for (int j = 0; j < N; j++) {
                const long long n2 = ((long long)j * j) % (2LL * N);
                const ld a = PI_L * (ld)n2 / N;              // conj of w_j = exp(-i pi j^2 / N)
                b[j] = cld(cosl(a), sinl(a));
                if (j > 0) b[M - j] = b[j];
            }
            host_dft_mixed(b);
            ld bmax = 0.0L;
            for (int q = 0; q < M; q++) bmax = std::max(bmax, std::abs(b[q]) / (ld)M);
            fs.bexp = (bmax > 0.0L) ? (int)ceill(log2l(bmax)) : 0;
            for (int q = 0; q < M; q++) {
                const cld v = b[split_k_of(q, M, fs.p3)] / (ld)M;   // with the inverse transform's 1 / M
                const float hx = (float)v.real(), hy = (float)v.imag();
                bsh.push_back(make_float2(hx, hy));
                bsl.push_back(make_float2((float)(v.real() - (ld)hx), (float)(v.imag() - (ld)hy)));
            }
        }
        if (bsh.empty()) { bsh.push_back(make_float2(1, 0)); bsl.push_back(make_float2(0, 0)); }
        if ((e = upload(&p->c.fft_s, p->h_fft_s, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->c.bhs_h, bsh, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->c.bhs_l, bsl, &acc)) != cudaSuccess) return e;
        // ring pairs grouped by FFT size (one launch per size in the split
        // FFTs), each size with its twiddles exp(-2 pi i u / M), u < M / 2
        std::map<int, std::vector<int>> bym;
        for (int q = 0; q < R; q++) bym[p->h_fft_s[p->h_pairs[q].fft].m].push_back(q);
        std::vector<int> cls;
        std::vector<float2> twh, twl;
        std::vector<float4> twp;
        for (auto& kv : bym) {
            sht::FftClass c;
            c.m = kv.first;
            c.off = (int)cls.size();
            c.cnt = (int)kv.second.size();
            c.tw = (long long)twh.size();
            // per-pass twiddles of the power-of-two part Ms = 2^La: its
            // transforms run one radix-2 (La = 1 mod 3) or radix-4 (La = 2
            // mod 3) pass of span 1, which needs none, and radix-8 passes of
            // spans h = 2^(La mod 3), 8 times that, ..., h <= Ms / 8; for each
            // such h and k < h, the seven factors W_{8h}^{k e}, e = 1 .. 7
            // (decimation in time and in frequency use the same ones)
            c.twp = (long long)twp.size();
            {
                const int Ms = c.m / pow3_part(c.m);
                int La = 0;
                while ((1 << La) < Ms) La++;
                for (int h = 1 << (La % 3); 8 * h <= Ms; h *= 8)
                    for (int k = 0; k < h; k++)
                        for (int e = 1; e <= 7; e++) {
                            const ld a = -2 * PI_L * (ld)((long long)k * e) / (ld)(8 * h);
                            const ld cr = cosl(a), ci = sinl(a);
                            const float hx = (float)cr, hy = (float)ci;
                            twp.push_back(make_float4(hx, hy, (float)(cr - (ld)hx), (float)(ci - (ld)hy)));
                        }
            }
            c.twp_n = (int)(twp.size() - c.twp);
            for (int u = 0; u < std::max(1, c.m / 2); u++) {
                const ld a = -2 * PI_L * (ld)u / (ld)c.m;
                const ld cr = cosl(a), ci = sinl(a);
                const float hx = (float)cr, hy = (float)ci;
                twh.push_back(make_float2(hx, hy));
                twl.push_back(make_float2((float)(cr - (ld)hx), (float)(ci - (ld)hy)));
            }
            cls.insert(cls.end(), kv.second.begin(), kv.second.end());
            p->h_fcls.push_back(c);
        }
        if ((e = upload(&p->c.cls_pairs, cls, &acc)) != cudaSuccess) return e;
        if (twp.empty()) twp.push_back(make_float4(1, 0, 0, 0));
        if ((e = upload(&p->c.twp, twp, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->c.tws_h, twh, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->c.tws_l, twl, &acc)) != cudaSuccess) return e;
    }

    // ---- lambda seeds ----
    std::vector<double> smant((size_t)(mmax + 1) * 2 * R);
    std::vector<int> sexp((size_t)(mmax + 1) * 2 * R);
    if (p->spin == 0) {
        // lambda_mm = (-1)^m sqrt((2m+1)/4pi prod_{k<=m} (2k-1)/(2k)) sin^m,
        // lambda_{m+1,m} = sqrt(2m+3) cos lambda_mm  (Condon-Shortley phase)
        for (int q = 0; q < R; q++) {
            Scaled v = snorm(1.0L / sqrtl(4 * PI_L), 0);
            for (int m = 0; m <= mmax; m++) {
                if (m > 0) v = smul(v, sqrtl((ld)(2 * m - 1) / (2 * m)) * ss[q]);
                Scaled lmm = smul(v, sqrtl((ld)(2 * m + 1)) * ((m & 1) ? -1 : 1));
                Scaled lm1 = smul(lmm, sqrtl((ld)(2 * m + 3)) * zs[q]);
                size_t i0 = ((size_t)m * 2 + 0) * R + q, i1 = ((size_t)m * 2 + 1) * R + q;
                smant[i0] = (double)lmm.v; sexp[i0] = (int)lmm.e;
                smant[i1] = (double)lm1.v; sexp[i1] = (int)lm1.e;
            }
        }
    } else {
        // s lambda at l0 = max(m,2): (-1)^m sqrt((2 l0+1)/4pi) d^{l0}_{-m,s}(theta)
        //   m >= 2: d^m_{-m,s}  = sqrt(C(2m, m-s)) cos^{m-s}(t/2) sin^{m+s}(t/2)
        //   m <  2: d^2_{-m,2}  = sqrt(C(4, 2-m)) cos^{2-m}(t/2) sin^{2+m}(t/2)
        //           d^2_{-m,-2} = (-1)^{2-m} sqrt(C(4, 2+m)) cos^{2+m}(t/2) sin^{2-m}(t/2)
        for (int m = 0; m <= mmax; m++) {
            int l0 = m > 2 ? m : 2;
            for (int si = 0; si < 2; si++) {
                int s = si == 0 ? 2 : -2;
                int kbin, pc, ps; ld sign = 1;
                if (m >= 2) { kbin = m - s; pc = m - s; ps = m + s; }
                else if (s == 2) { kbin = 2 - m; pc = 2 - m; ps = 2 + m; }
                else { kbin = 2 + m; pc = 2 + m; ps = 2 - m; sign = ((2 - m) & 1) ? -1 : 1; }
                int kk = std::min(kbin, 2 * l0 - kbin);
                Scaled c = {0.5L, 1};
                for (int i = 1; i <= kk; i++) c = smul(c, (ld)(2 * l0 - kk + i) / i);
                if (c.e & 1) { c.v *= 2; c.e -= 1; }
                c.v = sqrtl(c.v); c.e /= 2;
                ld pre = sign * ((m & 1) ? -1 : 1) * sqrtl((2 * l0 + 1) / (4 * PI_L));
                c = smul(c, pre);
                for (int q = 0; q < R; q++) {
                    ld ch = sqrtl((1 + zs[q]) / 2), sh = sqrtl((1 - zs[q]) / 2);
                    if (zs[q] > 0.5L) sh = sqrtl((ss[q] * ss[q]) / (2 * (1 + zs[q])));
                    Scaled v = sprod(c, sprod(spow(ch, pc), spow(sh, ps)));
                    size_t i0 = ((size_t)m * 2 + si) * R + q;
                    smant[i0] = (double)v.v; sexp[i0] = (int)v.e;
                }
            }
        }
    }
    if ((e = upload(&p->t.seed_mant, smant, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->t.seed_exp, sexp, &acc)) != cudaSuccess) return e;

    // ---- recurrence coefficients ----
    const long long nalm = p->nalm;
    if (p->spin == 0) {
        // a_l = sqrt((4l^2-1)/(l^2-m^2)), 1/a_m := 0; two-step same-parity form
        //   lambda_{l+2} = (alpha_l x^2 + beta_l) lambda_l + gamma_l lambda_{l-2}
        //   alpha_l = a_{l+2} a_{l+1}
        //   beta_l  = -a_{l+2} (a_{l+1} / a_l^2 + 1 / a_{l+1})
        //   gamma_l = -a_{l+2} a_{l+1} / (a_l a_{l-1})
        std::vector<double> ra(nalm, 0.0), rb(nalm, 0.0), rc(nalm, 0.0);
        for (int m = 0; m <= mmax; m++) {
            auto ainv = [&](int l) -> ld {
                if (l <= m) return 0;
                ld L = l, M = m;
                return sqrtl((L * L - M * M) / (4 * L * L - 1));
            };
            auto aa = [&](int l) -> ld {
                ld L = l, M = m;
                return sqrtl((4 * L * L - 1) / (L * L - M * M));
            };
            for (int l = m; l <= lmax; l++) {
                long long ci = alm_index(lmax, l, m);
                ld a1 = aa(l + 1), a2 = aa(l + 2);
                ld ia0 = ainv(l), iam = ainv(l - 1);
                ra[ci] = (double)(a2 * a1);
                rb[ci] = (double)(-a2 * (a1 * ia0 * ia0 + 1 / a1));
                rc[ci] = (double)(-a2 * a1 * ia0 * iam);
            }
        }
        if ((e = upload(&p->t.rec_a, ra, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->t.rec_b, rb, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->t.rec_c, rc, &acc)) != cudaSuccess) return e;
    } else {
        // s lambda_l = (A_l x + A_l B_l) s lambda_{l-1} - C_l s lambda_{l-2}
        //   A_l = l sqrt((2l+1)(2l-1)) / sqrt((l^2-m^2)(l^2-s^2)),  B_l = m s / (l(l-1))
        //   C_l = (l/(l-1)) sqrt((2l+1)/(2l-3)) sqrt(((l-1)^2-m^2)((l-1)^2-s^2) / ((l^2-m^2)(l^2-s^2)))
        for (int si = 0; si < 2; si++) {
            ld s = si == 0 ? 2 : -2;
            std::vector<double> A(nalm, 0.0), AB(nalm, 0.0), C(nalm, 0.0);
            for (int m = 0; m <= mmax; m++) {
                int l0 = m > 2 ? m : 2;
                for (int l = l0 + 1; l <= lmax; l++) {
                    long long ci = alm_index(lmax, l, m);
                    ld L = l, M = m;
                    ld den = (L * L - M * M) * (L * L - s * s);
                    ld Al = L * sqrtl((2 * L + 1) * (2 * L - 1)) / sqrtl(den);
                    ld Bl = M * s / (L * (L - 1));
                    ld num = ((L - 1) * (L - 1) - M * M) * ((L - 1) * (L - 1) - s * s);
                    ld Cl = (L / (L - 1)) * sqrtl((2 * L + 1) / (2 * L - 3)) * sqrtl(num / den);
                    A[ci] = (double)Al; AB[ci] = (double)(Al * Bl); C[ci] = (double)Cl;
                }
            }
            if ((e = upload(&p->t.w_A[si], A, &acc)) != cudaSuccess) return e;
            if ((e = upload(&p->t.w_AB[si], AB, &acc)) != cudaSuccess) return e;
            if ((e = upload(&p->t.w_C[si], C, &acc)) != cudaSuccess) return e;
        }
    }

    // ---- FP64 Legendre work lists ----
    {
        int TL = legendre_f64_row_tile(), TP = legendre_f64_pair_tile();
        std::vector<int4> w1, w2;
        p->m2a_off.assign(mmax + 2, 0);
        p->a2m_off.assign(mmax + 2, 0);
        for (int m = 0; m <= mmax; m++) {
            p->m2a_off[m] = (int)w1.size();
            p->a2m_off[m] = (int)w2.size();
            for (int q = 0; q < 2; q++) {
                int lf = m + q;
                int nrows = (lmax >= lf) ? (lmax - lf) / 2 + 1 : 0;
                for (int t = 0; t * TL < nrows; t++) w1.push_back(make_int4(m, q, t, 0));
                for (int t = 0; t * TP < R; t++) w2.push_back(make_int4(m, q, t, 0));
            }
        }
        p->m2a_off[mmax + 1] = (int)w1.size();
        p->a2m_off[mmax + 1] = (int)w2.size();
        p->nwork_m2a = (int)w1.size();
        p->nwork_a2m = (int)w2.size();
        if ((e = upload(&p->work_m2a, w1, &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->work_a2m, w2, &acc)) != cudaSuccess) return e;
    }
    p->table_bytes = acc;
    return cudaSuccess;
}

// integer range Q of the slices for a contraction of length K: main (the sum
// of q q' plus the integer parts folded in after every span, at most
// Q (Q + 1) K + 12 K / 32) must stay below 2^24, where FP32 holds integers
// exactly, and Q <= 127 keeps a span of q r0' + r0 q' (multiples of 2^-G: 64
// wide with G = 11, at most 64 Q (1 + 2^-10) < 2^13, or 128 wide with G = 10,
// at most 128 Q (1 + 2^-9) < 2^14) below 2^(24 - G)
static float slice_range(double K)
{
    K = std::max(K, 1.0);
    double Q = std::min(std::floor(std::sqrt(16777216.0 / K)), 127.0);
    while (Q > 1 && Q * (Q + 1) * K + 12.0 * std::ceil(K / 32.0) > 16777216.0) Q -= 1;
    return (float)Q;
}

// Slicing units and image chunks of the pre-sliced data (32-wide units of K
// per (m, q)). map2alm: K = the ring pairs, for every (m, q) that has l rows;
// spin 2 stores two chunks per unit (T_q + P(T_{1-q}) and T_q - P(T_{1-q})).
// alm2map: K = the l of slot q (spin 0) or all l >= m (spin 2, one chunk per
// unit shared by the v+ and v- chunks of the contraction).
// Ring optimisation (Sec. 3.1, Implementation detail: for each m the rings
// where P_lm has an extremely low amplitude are left out, in the Legendre
// step and in the FFT mapping). Near the poles lambda_lm(theta)
// ~ sin^m(theta) underflows for large m, so for each order m the leading ring
// pairs p < pfirst[m] (from the north pole) where max_l |lambda_lm| stays below
// SPLIT_LAMBDA_EPS for both parities are skipped: map2alm contracts only the
// 32-wide chunks of ring pairs from pfirst[m], alm2map computes G only for
// those ring pairs, and the ring FFTs and the Fourier-domain residual use the
// orders m <= mlim[p] of ring pair p. pfirst is made nondecreasing in m (the
// smallest first pair of this and every higher order) and rounded down to a
// multiple of 32, so {m : p >= pfirst[m]} = {m <= mlim[p]}. A skipped term is
// below 1e-30 of lambda's O(1) peak times the data, far below FP64 rounding
// of the outputs. SHT_RING_SKIP=0 turns it off. Split plans (spin 2: the
// maxima over both slots are those of s = +2 and -2).
// whether ring skipping is on for plans created now (SHT_RING_SKIP=0: off)
bool ring_skip_enabled()
{
    const char* env = std::getenv("SHT_RING_SKIP");
    return !(env && std::atoi(env) == 0);
}

// pfirst[m] (host) and the kept share of the (m, l, ring pair) terms from
// live[m * R + p] = 1 where some |lambda_lm(theta_p)| >= SPLIT_LAMBDA_EPS:
// the first live pair of each order, made nondecreasing in m from the top
// and rounded down to 32; order 0 keeps every pair
void ring_first_pairs(sht_plan* p, const std::vector<char>& live)
{
    const int mmax = p->mmax, R = p->R, KCH = 32;
    p->h_pfirst.assign((size_t)mmax + 1, 0);
    int run = R - 1;                     // the equator pair is never skipped
    for (int m = mmax; m >= 0; m--) {
        int p0 = 0;
        while (p0 < R - 1 && !live[(size_t)m * R + p0]) p0++;
        run = std::min(run, p0);
        p->h_pfirst[m] = run / KCH * KCH;
    }
    p->h_pfirst[0] = 0;                  // (lambda_00 is constant: order 0 keeps every pair)
    double kept = 0.0, all = 0.0;
    for (int m = 0; m <= mmax; m++) {
        const double nl = (p->lmax >= m) ? (double)(p->lmax - m + 1) : 0.0;
        kept += nl * (R - p->h_pfirst[m]);
        all += nl * R;
    }
    p->terms_kept = all > 0.0 ? kept / all : 1.0;
}

static cudaError_t build_ring_skip(sht_plan* p, size_t* acc)
{
    const int mmax = p->mmax, R = p->R;
    p->h_pfirst.assign((size_t)mmax + 1, 0);
    if (!ring_skip_enabled()) return cudaSuccess;
    std::vector<float> pm((size_t)(mmax + 1) * 2 * R);
    cudaError_t e = cudaMemcpy(pm.data(), p->s.pairmax, pm.size() * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    std::vector<char> live((size_t)(mmax + 1) * R);
    for (int m = 0; m <= mmax; m++)
        for (int q = 0; q < R; q++)
            live[(size_t)m * R + q] = std::max(pm[((size_t)m * 2 + 0) * R + q], pm[((size_t)m * 2 + 1) * R + q]) >=
                                      SPLIT_LAMBDA_EPS;
    ring_first_pairs(p, live);
    std::vector<int> ml((size_t)R, 0);
    for (int q = 0, m = 0; q < R; q++) {
        while (m < mmax && p->h_pfirst[m + 1] <= q) m++;
        ml[q] = m;
    }
    if ((e = upload(&p->s.pfirst, p->h_pfirst, acc)) != cudaSuccess) return e;
    if ((e = upload(&p->s.mlim, ml, acc)) != cudaSuccess) return e;
    // alm2map work items over the ring pairs [pfirst[m], R) of each order
    const int TM = split_row_tile(), GA = split_a2m_tiles();
    std::vector<int4> w2;
    std::vector<int4> old((size_t)p->s.nwork_a2m);
    if (!old.empty() &&
        (e = cudaMemcpy(old.data(), p->s.work_a2m, old.size() * sizeof(int4), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    int last = -1;
    for (const int4& w : old) {          // keep each (m, q)'s checkpoint block, one pass per (m, q)
        const int mq = w.x * 2 + w.y;
        if (mq == last) continue;
        last = mq;
        const int ntR = (R - p->h_pfirst[w.x] + TM - 1) / TM;
        for (int t = 0; t < ntR; t += GA) w2.push_back(make_int4(w.x, w.y, t | (std::min(GA, ntR - t) << 16), w.w));
    }
    cudaFree(p->s.work_a2m);
    p->s.work_a2m = nullptr;
    p->s.nwork_a2m = (int)w2.size();
    return upload(&p->s.work_a2m, w2, acc);
}

static cudaError_t build_slice_lists(sht_plan* p, size_t* acc)
{
    const int lmax = p->lmax, mmax = p->mmax, KCH = 32;
    const int nuR = (p->R + KCH - 1) / KCH;
    std::vector<int> bm((size_t)(mmax + 1) * 2, 0), ba((size_t)(mmax + 1) * 2, 0);
    std::vector<int4> um, ua;
    long long cm = 0, ca = 0;
    for (int m = 0; m <= mmax; m++)
        for (int q = 0; q < 2; q++) {
            const int mq = m * 2 + q;
            const int nl = (lmax >= m + q) ? (lmax - m - q) / 2 + 1 : 0;
            bm[mq] = (int)cm;
            if (nl > 0) {
                // (units before the order's first ring pair are never contracted)
                const int u0 = p->h_pfirst.empty() ? 0 : p->h_pfirst[m] / KCH;
                for (int u = u0; u < nuR; u++) um.push_back(make_int4(m, q, u, (int)(cm + (p->spin ? 2 * u : u))));
                cm += p->spin ? 2 * nuR : nuR;
            }
            const int Ka = p->spin ? (lmax >= m ? lmax - m + 1 : 0) : nl;
            const int nua = (Ka + KCH - 1) / KCH;
            ba[mq] = (int)ca;
            for (int u = 0; u < nua; u++) ua.push_back(make_int4(m, q, u, (int)(ca + u)));
            ca += nua;
        }
    if (cm > INT_MAX || ca > INT_MAX) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = upload(&p->s.img_base_m2a, bm, acc)) != cudaSuccess) return e;
    if ((e = upload(&p->s.img_base_a2m, ba, acc)) != cudaSuccess) return e;
    if (!um.empty() && (e = upload(&p->s.sunits_m2a, um, acc)) != cudaSuccess) return e;
    if (!ua.empty() && (e = upload(&p->s.sunits_a2m, ua, acc)) != cudaSuccess) return e;
    p->s.nsunits_m2a = (int)um.size();
    p->s.nsunits_a2m = (int)ua.size();
    p->s.img_chunks_m2a = cm;
    p->s.img_chunks_a2m = ca;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// spin-2 split-form tables. The Wigner recurrence of build_tables,
//   s lambda_l = A_l (x + B_l) s lambda_{l-1} - C_l s lambda_{l-2},
// with s lambda_l = d_l mu_l and d_l = C_l d_{l-2} (d_{l0} = d_{l0+1} = 1)
// becomes mu_l = (A'_l x + B'_l) mu_{l-1} - mu_{l-2},
//   A'_l = A_l d_{l-1} / d_l,  B'_l = A_l B_l d_{l-1} / d_l
// (2 FP64 operations per step). C_l depends on s only through s^2, so d_l is
// the same for s = +2 and -2.
// ---------------------------------------------------------------------------
static cudaError_t build_split_tables_s2(sht_plan* p)
{
    const int lmax = p->lmax, mmax = p->mmax, R = p->R;
    const long long nalm = p->nalm;
    size_t acc = 0;
    cudaError_t e;
    std::vector<double> cA[2] = {std::vector<double>(nalm, 0.0), std::vector<double>(nalm, 0.0)};
    std::vector<double> cB[2] = {std::vector<double>(nalm, 0.0), std::vector<double>(nalm, 0.0)};
    std::vector<double> d64(nalm, 0.0);
    std::vector<float2> d2(nalm, make_float2(0.0f, 0.0f));
    for (int m = 0; m <= mmax; m++) {
        const int l0 = m > 2 ? m : 2;
        if (l0 > lmax) continue;
        const ld M = m, S2 = 4;
        std::vector<ld> d(lmax + 1, 0);
        d[l0] = 1;
        if (l0 + 1 <= lmax) d[l0 + 1] = 1;
        for (int l = l0 + 2; l <= lmax; l++) {
            const ld L = l;
            const ld den = (L * L - M * M) * (L * L - S2);
            const ld num = ((L - 1) * (L - 1) - M * M) * ((L - 1) * (L - 1) - S2);
            const ld Cl = (L / (L - 1)) * sqrtl((2 * L + 1) / (2 * L - 3)) * sqrtl(num / den);
            d[l] = Cl * d[l - 2];
        }
        for (int l = l0; l <= lmax; l++) {
            const long long ci = alm_index(lmax, l, m);
            d64[ci] = (double)d[l];
            const float dh = (float)d[l];
            d2[ci] = make_float2(dh, (float)(d[l] - (ld)dh));
        }
        for (int si = 0; si < 2; si++) {
            const ld s = si == 0 ? 2 : -2;
            for (int l = l0 + 1; l <= lmax; l++) {
                const long long ci = alm_index(lmax, l, m);
                const ld L = l;
                const ld Al = L * sqrtl((2 * L + 1) * (2 * L - 1)) / sqrtl((L * L - M * M) * (L * L - s * s));
                const ld Bl = M * s / (L * (L - 1));
                cA[si][ci] = (double)(Al * d[l - 1] / d[l]);
                cB[si][ci] = (double)(Al * Bl * d[l - 1] / d[l]);
            }
        }
    }
    for (int si = 0; si < 2; si++) {
        if ((e = upload(&p->s.s2A[si], cA[si], &acc)) != cudaSuccess) return e;
        if ((e = upload(&p->s.s2B[si], cB[si], &acc)) != cudaSuccess) return e;
    }
    if ((e = upload(&p->s.s2d64, d64, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->s.s2d2, d2, &acc)) != cudaSuccess) return e;
    // work lists; checkpoint blocks: every 32 l from m, per m
    const int TM = split_row_tile(), CKL = split_ck_rows();
    // alm2map work items cover GA ring-pair tiles each (first tile | count << 16)
    const int GA = split_a2m_tiles(), ntR = (R + TM - 1) / TM;
    std::vector<int4> w1, w2;
    std::vector<int> base((size_t)(mmax + 1));
    int nblk = 0;
    for (int m = 0; m <= mmax; m++) {
        base[m] = nblk;
        for (int q = 0; q < 2; q++) {
            const int lf = m + q;
            const int nrows = (lmax >= lf) ? (lmax - lf) / 2 + 1 : 0;
            for (int t = 0; t * TM < nrows; t++) w1.push_back(make_int4(m, q, t, nblk));
            if (lmax >= m)
                for (int t = 0; t * TM < R; t += GA) w2.push_back(make_int4(m, q, t | (std::min(GA, ntR - t) << 16), nblk));
        }
        nblk += (lmax >= m) ? (lmax - m + 1 + CKL - 1) / CKL : 0;
    }
    p->s.nwork_m2a = (int)w1.size();
    p->s.nwork_a2m = (int)w2.size();
    if ((e = upload(&p->s.work_m2a, w1, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->s.work_a2m, w2, &acc)) != cudaSuccess) return e;
    int* d_base = nullptr;
    if ((e = upload(&d_base, base, &acc)) != cudaSuccess) return e;
    const size_t nck = (size_t)std::max(nblk, 1) * 2 * R;
    const size_t npm = (size_t)(mmax + 1) * 2 * R;
    if ((e = cudaMalloc(&p->s.ck, nck * sizeof(double2))) != cudaSuccess) { cudaFree(d_base); return e; }
    if ((e = cudaMalloc(&p->s.ck_exp, nck * sizeof(int))) != cudaSuccess) { cudaFree(d_base); return e; }
    if ((e = cudaMalloc(&p->s.rowmax_bits, (size_t)nalm * sizeof(unsigned int))) != cudaSuccess) { cudaFree(d_base); return e; }
    if ((e = cudaMalloc(&p->s.pairmax, npm * sizeof(float))) != cudaSuccess) { cudaFree(d_base); return e; }
    if ((e = cudaMalloc(&p->s.err, sizeof(int))) != cudaSuccess) { cudaFree(d_base); return e; }
    acc += nck * (sizeof(double2) + sizeof(int)) + (size_t)nalm * 4 + npm * 4 + 4;
    cudaMemset(p->s.ck, 0, nck * sizeof(double2));
    cudaMemset(p->s.ck_exp, 0, nck * sizeof(int));
    cudaMemset(p->s.rowmax_bits, 0, (size_t)nalm * sizeof(unsigned int));
    cudaMemset(p->s.pairmax, 0, npm * sizeof(float));
    cudaMemset(p->s.err, 0, sizeof(int));
    e = run_split_tables(p, d_base);
    cudaFree(d_base);
    if (e != cudaSuccess) return e;
    if ((e = build_ring_skip(p, &acc)) != cudaSuccess) return e;
    // each contraction runs twice over its range (v+ and v- chunks)
    p->s.Q_m2a = slice_range(2.0 * R);
    p->s.Q_a2m = slice_range(2.0 * (lmax + 1));
    if ((e = build_slice_lists(p, &acc)) != cudaSuccess) return e;
    p->table_bytes += acc;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// split-form tables: normalised two-step recurrence (2 FP64 ops per lambda),
// plan-time checkpoints of the map2alm row tiles and lambda maxima
// ---------------------------------------------------------------------------
static cudaError_t build_split_tables(sht_plan* p)
{
    if (p->spin) return build_split_tables_s2(p);
    const int lmax = p->lmax, mmax = p->mmax, R = p->R;
    const long long nalm = p->nalm;
    size_t acc = 0;
    cudaError_t e;
    // lambda_{l+2} = (alpha x^2 + beta) lambda_l + gamma lambda_{l-2} (see build_tables);
    // with lambda_l = c_l mu_l and c_{l+2} = gamma_l c_{l-2} the chain becomes
    // mu_{l+2} = (A x^2 + B) mu_l + mu_{l-2}, A = alpha c_l / c_{l+2}, B = beta c_l / c_{l+2};
    // each parity chain starts with c_{l0} = c_{l0+2} = 1 (gamma_{l0} = 0).
    std::vector<double> nA(nalm, 0.0), nB(nalm, 0.0);
    std::vector<float> nc(nalm, 0.0f);
    std::vector<double> nc64(nalm, 0.0);
    std::vector<float2> nc2(nalm, make_float2(0.0f, 0.0f));
    for (int m = 0; m <= mmax; m++) {
        auto ainv = [&](int l) -> ld { if (l <= m) return 0; ld L = l, M = m; return sqrtl((L * L - M * M) / (4 * L * L - 1)); };
        auto aa = [&](int l) -> ld { ld L = l, M = m; return sqrtl((4 * L * L - 1) / (L * L - M * M)); };
        for (int q = 0; q < 2; q++) {
            int l0 = m + q;
            if (l0 > lmax) continue;
            std::vector<ld> c;       // c for l = l0 + 2j
            c.push_back(1.0L);
            for (int l = l0; l <= lmax; l += 2) {
                ld a1 = aa(l + 1), a2 = aa(l + 2);
                ld alpha = a2 * a1;
                ld beta = -a2 * (a1 * ainv(l) * ainv(l) + 1 / a1);
                ld gamma = -a2 * a1 * ainv(l) * ainv(l - 1);
                size_t j = (l - l0) / 2;
                ld cn = (l == l0) ? 1.0L : gamma * c[j - 1];
                c.push_back(cn);
                long long ci = alm_index(lmax, l, m);
                nA[ci] = (double)(alpha * c[j] / cn);
                nB[ci] = (double)(beta * c[j] / cn);
                nc[ci] = (float)c[j];
                nc64[ci] = (double)c[j];
                const float ch = (float)c[j];
                nc2[ci] = make_float2(ch, (float)(c[j] - (ld)ch));
            }
        }
    }
    if ((e = upload(&p->s.nA, nA, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->s.nB, nB, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->s.nc, nc, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->s.nc64, nc64, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->s.nc2, nc2, &acc)) != cudaSuccess) return e;
    // work lists and checkpoint blocks (one block every CKR rows of a chain)
    const int TM = split_row_tile(), CKR = split_ck_rows();
    // alm2map work items cover GA ring-pair tiles each (first tile | count << 16)
    const int GA = split_a2m_tiles(), ntR = (R + TM - 1) / TM;
    std::vector<int4> w1, w2;
    std::vector<int> base((size_t)(mmax + 1) * 2);
    int nblk = 0;
    for (int m = 0; m <= mmax; m++)
        for (int q = 0; q < 2; q++) {
            int lf = m + q;
            int nrows = (lmax >= lf) ? (lmax - lf) / 2 + 1 : 0;
            base[m * 2 + q] = nblk;
            for (int t = 0; t * TM < nrows; t++) w1.push_back(make_int4(m, q, t, nblk));
            for (int t = 0; t * TM < R; t += GA) w2.push_back(make_int4(m, q, t | (std::min(GA, ntR - t) << 16), nblk));
            nblk += (nrows + CKR - 1) / CKR;
        }
    p->s.nwork_m2a = (int)w1.size();
    p->s.nwork_a2m = (int)w2.size();
    if ((e = upload(&p->s.work_m2a, w1, &acc)) != cudaSuccess) return e;
    if ((e = upload(&p->s.work_a2m, w2, &acc)) != cudaSuccess) return e;
    int* d_base = nullptr;
    if ((e = upload(&d_base, base, &acc)) != cudaSuccess) return e;
    size_t nck = (size_t)std::max(nblk, 1) * R;
    if ((e = cudaMalloc(&p->s.ck, nck * sizeof(double2))) != cudaSuccess) { cudaFree(d_base); return e; }
    if ((e = cudaMalloc(&p->s.ck_exp, nck * sizeof(int))) != cudaSuccess) { cudaFree(d_base); return e; }
    if ((e = cudaMalloc(&p->s.rowmax_bits, (size_t)nalm * sizeof(unsigned int))) != cudaSuccess) { cudaFree(d_base); return e; }
    if ((e = cudaMalloc(&p->s.pairmax, (size_t)(mmax + 1) * 2 * R * sizeof(float))) != cudaSuccess) { cudaFree(d_base); return e; }
    if ((e = cudaMalloc(&p->s.err, sizeof(int))) != cudaSuccess) { cudaFree(d_base); return e; }
    acc += nck * (sizeof(double2) + sizeof(int)) + (size_t)nalm * 4 + (size_t)(mmax + 1) * 2 * R * 4 + 4;
    cudaMemset(p->s.rowmax_bits, 0, (size_t)nalm * sizeof(unsigned int));
    cudaMemset(p->s.pairmax, 0, (size_t)(mmax + 1) * 2 * R * sizeof(float));
    cudaMemset(p->s.err, 0, sizeof(int));
    e = run_split_tables(p, d_base);
    cudaFree(d_base);
    if (e != cudaSuccess) return e;
    if ((e = build_ring_skip(p, &acc)) != cudaSuccess) return e;
    p->s.Q_m2a = slice_range((double)R);
    p->s.Q_a2m = slice_range((double)(lmax / 2 + 1));
    if ((e = build_slice_lists(p, &acc)) != cudaSuccess) return e;
    p->table_bytes += acc;
    return cudaSuccess;
}

static void free_tables(sht_plan* p)
{
    void* ptrs[] = {p->t.pairs, p->t.fft, p->t.twiddle, p->t.chirp, p->t.bhat, p->t.twiddle_f,
                    p->t.chirp_f, p->t.bhat_f, p->t.seed_mant, p->t.seed_exp, p->t.rec_a, p->t.rec_b,
                    p->t.rec_c, p->t.w_A[0], p->t.w_A[1], p->t.w_AB[0], p->t.w_AB[1], p->t.w_C[0],
                    p->t.w_C[1], p->t.ck64, p->t.ck64_exp, p->t.ck64_off, p->t.pfirst64, p->work_m2a, p->work_a2m,
                    p->host_dev_in, p->host_dev_out, p->host_ws};
    for (void* q : ptrs) if (q) cudaFree(q);
    void* cp[] = {p->c.cls_pairs, p->c.twiddle_l, p->c.chirp_l, p->c.bhat_l, p->c.phase_h, p->c.phase_l, p->c.phase_off,
                  p->c.fft_s, p->c.twp, p->c.tws_h, p->c.tws_l, p->c.bhs_h, p->c.bhs_l};
    for (void* q : cp) if (q) cudaFree(q);
    void* sp[] = {p->s.nA, p->s.nB, p->s.nc, p->s.nc64, p->s.nc2, p->s.ck, p->s.ck_exp, p->s.rowmax_bits, p->s.pairmax, p->s.err,
                  p->s.work_m2a, p->s.work_a2m, p->s.s2A[0], p->s.s2A[1], p->s.s2B[0], p->s.s2B[1], p->s.s2d2,
                  p->s.s2d64, p->s.img_base_m2a, p->s.img_base_a2m, p->s.sunits_m2a, p->s.sunits_a2m,
                  p->s.pfirst, p->s.mlim};
    for (void* q : sp) if (q) cudaFree(q);
    for (cudaEvent_t ev : p->hp_ev) if (ev) cudaEventDestroy(ev);
    if (p->hp_h2d) cudaStreamDestroy(p->hp_h2d);
    if (p->hp_d2h) cudaStreamDestroy(p->hp_d2h);
    for (int i = 0; i < sht_plan::FFT_AUX; i++) {
        if (p->fft_aux[i]) cudaStreamDestroy(p->fft_aux[i]);
        if (p->fft_join[i]) cudaEventDestroy(p->fft_join[i]);
    }
    if (p->fft_fork) cudaEventDestroy(p->fft_fork);
    if (p->pin_in) cudaFreeHost(p->pin_in);
    if (p->pin_out) cudaFreeHost(p->pin_out);
}

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// split form, alm2map: G (FP32) first, then the transposed a_lm A2 (FP32 hi/lo)
size_t split_a2_offset(const sht_plan* p, int nmaps)
{
    return round_up((size_t)(p->mmax + 1) * 2 * (size_t)p->R * (size_t)ncols(p, nmaps) * sizeof(float), 256);
}

size_t tbuf_bytes(const sht_plan* p, int nmaps)
{
    const size_t n = (size_t)(p->mmax + 1) * 2 * (size_t)p->R * (size_t)ncols(p, nmaps);
    if (p->precision == SHT_FP64) return n * sizeof(double);
    // split form: map2alm keeps T as FP32 hi/lo pairs; alm2map holds G (FP32) and A2
    const size_t a2 = (size_t)p->nalm * (size_t)ncols(p, nmaps) * sizeof(float2);
    return std::max(n * sizeof(float2), split_a2_offset(p, nmaps) + a2);
}

static size_t colmax_bytes(const sht_plan* p, int nmaps)
{
    return p->precision == SHT_FP64 ? 0 : (size_t)(p->mmax + 1) * 2 * (size_t)ncols(p, nmaps) * sizeof(float);
}

static size_t img_bytes(const sht_plan* p, int nmaps)
{
    return p->precision == SHT_FP64 ? 0 : split_img_bytes(p, nmaps);
}

// Workspace layout: [T / G buffer][column maxima] for one transform. map2alm
// with niter > 0 keeps the ring spectra T of the first pass and adds, for the
// Fourier-domain iteration: [G buffer of alm2map (FP64: also the residual D)]
// [split form: residual D (FP32 hi/lo)][split: column maxima][delta a_lm].
// The split form ends with the pre-sliced data image of the contractions
// (one at a time, in stream order).
struct IterWs {
    size_t g, d, cm, da, img, end;
};
static IterWs iter_ws(const sht_plan* p, int nmaps)
{
    IterWs w;
    const size_t tb = round_up(tbuf_bytes(p, nmaps), 256), cb = round_up(colmax_bytes(p, nmaps), 256);
    const size_t n = (size_t)(p->mmax + 1) * 2 * (size_t)p->R * (size_t)ncols(p, nmaps);
    w.g = tb + cb;
    if (p->precision == SHT_FP64) {
        w.d = w.g;
        w.cm = w.g + tb;
        w.da = w.cm;
    } else {
        w.d = w.g + tb;
        w.cm = w.d + round_up(n * sizeof(float2), 256);
        w.da = w.cm + cb;
    }
    w.img = w.da + round_up((size_t)nmaps * p->ncomp * (size_t)p->nalm * 2 * sizeof(double), 256);
    w.end = w.img + round_up(img_bytes(p, nmaps), 256);
    return w;
}

// offset of the data image in the workspace of a transform without iteration
static size_t img_offset(const sht_plan* p, int nmaps)
{
    return round_up(tbuf_bytes(p, nmaps), 256) + round_up(colmax_bytes(p, nmaps), 256);
}

static size_t ws_bytes(const sht_plan* p, int nmaps, int niter)
{
    if (niter > 0) return iter_ws(p, nmaps).end;
    return img_offset(p, nmaps) + round_up(img_bytes(p, nmaps), 256);
}

// elementwise helpers for the iteration (Algorithm 2)
__global__ void k_add(double* __restrict__ a, const double* __restrict__ d, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long st = (long long)gridDim.x * blockDim.x;
    for (; i < n; i += st) a[i] += d[i];
}
static int ew_grid(long long n) { long long b = (n + 255) / 256; return (int)std::min<long long>(b, 148 * 16); }

// [nmaps][2][nalm] a_lm with component `which` from one [nmaps][1][nalm], the other zero
cudaError_t expand_component(const sht_plan* p, const void* one, void* full, int nmaps, int which, cudaStream_t st)
{
    const size_t row = (size_t)p->nalm * 2 * sizeof(double);
    cudaError_t e = cudaMemset2DAsync((char*)full + (size_t)(1 - which) * row, 2 * row, 0, row, (size_t)nmaps, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync((char*)full + (size_t)which * row, 2 * row, one, row, row, (size_t)nmaps,
                              cudaMemcpyDeviceToDevice, st);
    return e;
}

}  // namespace sht

using namespace sht;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* sht_last_error(void) { return t_err.c_str(); }
int sht_last_launch_count(void) { return t_launches; }

sht_status sht_plan_device_status(sht_plan* p, int* code)
{
    t_err.clear();
    if (code) *code = 0;
    if (!p) { set_error("plan is NULL"); return SHT_EINVAL; }
    if (!p->s.err) return SHT_OK;
    SHT_CUDA_TRY(cudaSetDevice(p->device));
    SHT_CUDA_TRY(cudaDeviceSynchronize());
    int v = 0;
    SHT_CUDA_TRY(cudaMemcpy(&v, p->s.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) SHT_CUDA_TRY(cudaMemset(p->s.err, 0, sizeof(int)));
    if (code) *code = v;
    if (v != 0) {
        set_error("a bounded device wait gave up (code " + std::to_string(v) + ")");
        return SHT_ETIMEOUT;
    }
    return SHT_OK;
}
const char* sht_version(void) { return "libsht 0.1 (sm_103a)"; }

void sht_profile_begin(void)
{
    for (auto& r : t_recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    t_recs.clear();
    t_prof = true;
}

int sht_profile_end(char* buf, int cap)
{
    t_prof = false;
    std::map<std::string, std::pair<int, double>> agg;
    for (auto& r : t_recs) {
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            auto& v = agg[r.name];
            v.first += 1;
            v.second += ms;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    t_recs.clear();
    std::string js = "{";
    bool first = true;
    for (auto& kv : agg) {
        char tmp[256];
        snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %d, \"ms\": %.6f}", first ? "" : ", ",
                 kv.first.c_str(), kv.second.first, kv.second.second);
        js += tmp;
        first = false;
    }
    js += "}";
    if (buf && cap > 0) {
        int n = (int)std::min<size_t>(js.size(), (size_t)cap - 1);
        memcpy(buf, js.data(), n);
        buf[n] = 0;
    }
    return (int)js.size() + 1;
}

sht_status sht_plan_create(int nside, int lmax, int mmax, int spin, int precision, int device,
                           sht_plan** out)
{
    t_err.clear();
    if (!out) { set_error("out is NULL"); return SHT_EINVAL; }
    *out = nullptr;
    if (mmax < 0) mmax = lmax;
    if (nside < 1 || nside > 8192) { set_error("nside must be in [1, 8192]"); return SHT_EINVAL; }
    if (lmax < 0 || lmax > 4 * 8192) { set_error("lmax out of range"); return SHT_EINVAL; }
    if (mmax > lmax) { set_error("mmax must be <= lmax"); return SHT_EINVAL; }
    if (spin != 0 && spin != 2) { set_error("spin must be 0 or 2"); return SHT_EINVAL; }
    if (precision != SHT_FP64 && precision != SHT_SPLIT_F16X4) { set_error("unknown precision"); return SHT_EINVAL; }
    if (precision == SHT_SPLIT_F16X4 && mmax > 2047) {
        set_error("SHT_SPLIT_F16X4 supports mmax <= 2047");
        return SHT_EUNSUPPORTED;
    }
    // the contraction lengths (ring pairs, l of one parity) bound the exact
    // integer sums of the tensor-core form
    // (spin 2 contracts twice over each range)
    const int kmul = spin ? 2 : 1;
    if (precision == SHT_SPLIT_F16X4 && (kmul * 2 * nside > 8192 || (spin ? lmax + 1 : lmax / 2 + 1) * kmul > 8192)) {
        set_error(spin ? "SHT_SPLIT_F16X4 spin 2 supports nside <= 2048 and lmax <= 4095"
                       : "SHT_SPLIT_F16X4 supports nside <= 4096 and lmax <= 16383");
        return SHT_EUNSUPPORTED;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        set_error("no such CUDA device");
        return SHT_EINVAL;
    }
    SHT_CUDA_TRY(cudaSetDevice(device));
    sht_plan* p = new sht_plan();
    p->nside = nside; p->lmax = lmax; p->mmax = mmax; p->spin = spin;
    p->precision = precision; p->device = device;
    p->ncomp = spin ? 2 : 1;
    p->npix = 12LL * nside * nside;
    p->nalm = (long long)(mmax + 1) * (2 * lmax + 2 - mmax) / 2;
    p->R = 2 * nside;
    cudaError_t e = build_tables(p);
    if (e == cudaSuccess && precision == SHT_FP64) {
        size_t ckb = 0;
        e = build_f64_checkpoints(p, &ckb);
        p->table_bytes += ckb;
    }
    if (e == cudaSuccess && precision == SHT_SPLIT_F16X4) e = build_split_tables(p);
    // the split FFTs' helper streams and events, made here rather than at the
    // first call (which may be under stream capture)
    if (e == cudaSuccess && precision == SHT_SPLIT_F16X4) {
        e = cudaEventCreateWithFlags(&p->fft_fork, cudaEventDisableTiming);
        for (int i = 0; i < sht_plan::FFT_AUX && e == cudaSuccess; i++) {
            e = cudaStreamCreateWithFlags(&p->fft_aux[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fft_join[i], cudaEventDisableTiming);
        }
    }
    if (e != cudaSuccess) {
        set_error(std::string("plan tables: ") + cudaGetErrorString(e));
        free_tables(p);
        delete p;
        return e == cudaErrorMemoryAllocation ? SHT_ENOMEM : SHT_ECUDA;
    }
    *out = p;
    return SHT_OK;
}

void sht_plan_destroy(sht_plan* p)
{
    if (!p) return;
    cudaSetDevice(p->device);
    free_tables(p);
    delete p;
}

size_t sht_workspace_bytes(const sht_plan* p, int nmaps)
{
    if (!p || nmaps < 1) return 0;
    return ws_bytes(p, nmaps, 0);
}

size_t sht_workspace_bytes_iter(const sht_plan* p, int nmaps, int niter)
{
    if (!p || nmaps < 1) return 0;
    return ws_bytes(p, nmaps, niter);
}

int sht_plan_nside(const sht_plan* p) { return p ? p->nside : 0; }
int sht_plan_lmax(const sht_plan* p) { return p ? p->lmax : 0; }
int sht_plan_mmax(const sht_plan* p) { return p ? p->mmax : 0; }
int sht_plan_spin(const sht_plan* p) { return p ? p->spin : 0; }
int sht_plan_precision(const sht_plan* p) { return p ? p->precision : 0; }
long long sht_plan_npix(const sht_plan* p) { return p ? p->npix : 0; }
long long sht_plan_nalm(const sht_plan* p) { return p ? p->nalm : 0; }
double sht_plan_terms_kept(const sht_plan* p) { return p ? p->terms_kept : 0.0; }
sht_status sht_plan_first_pairs(const sht_plan* p, int* out)
{
    if (!p || !out) { set_error("sht_plan_first_pairs: NULL argument"); return SHT_EINVAL; }
    for (int m = 0; m <= p->mmax; m++) out[m] = p->h_pfirst.empty() ? 0 : p->h_pfirst[m];
    return SHT_OK;
}
size_t sht_plan_device_bytes(const sht_plan* p)
{
    return p ? p->table_bytes + p->host_dev_in_bytes + p->host_dev_out_bytes + p->host_ws_bytes : 0;
}

static sht_status check_call(const sht_plan* p, const void* in, const void* out, int nmaps,
                             void* ws, size_t wsb, int niter)
{
    t_err.clear();
    reset_launches();
    if (!p) { set_error("plan is NULL"); return SHT_EINVAL; }
    if (nmaps < 1) { set_error("nmaps must be >= 1"); return SHT_EINVAL; }
    if (!in || !out) { set_error("data pointer is NULL"); return SHT_EINVAL; }
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) { set_error("data pointers must be 16-byte aligned"); return SHT_EINVAL; }
    if (niter < 0) { set_error("niter must be >= 0"); return SHT_EINVAL; }
    size_t need = ws_bytes(p, nmaps, niter);
    if (!ws || wsb < need) {
        set_error("workspace too small: need " + std::to_string(need) + " bytes");
        return SHT_EINVAL;
    }
    if ((uintptr_t)ws & 255) { set_error("workspace must be 256-byte aligned"); return SHT_EINVAL; }
    return SHT_OK;
}

static sht_status do_alm2map(sht_plan* p, const double* alm, double* map, int nmaps, void* ws,
                             double s0, double s1, cudaStream_t st)
{
    cudaError_t e;
    if (p->precision == SHT_FP64) {
        double* G = (double*)ws;
        e = launch_legendre_a2m_f64(p, alm, G, nmaps, s0, s1, st);
        if (e == cudaSuccess) e = launch_fft_backward_f64(p, G, map, nmaps, st);
    } else {
        float* G = (float*)ws;
        float2* A2 = (float2*)((char*)ws + split_a2_offset(p, nmaps));
        unsigned int* cm = (unsigned int*)((char*)ws + round_up(tbuf_bytes(p, nmaps), 256));
        uint8_t* img = (uint8_t*)ws + img_offset(p, nmaps);
        e = launch_alm_prep(p, alm, A2, cm, nmaps, st);
        if (e == cudaSuccess)
            e = launch_legendre_a2m_tc(p, A2, (const float*)cm, img, G, nmaps, (float)s0, (float)s1, st);
        if (e == cudaSuccess) e = launch_fft_backward_f32(p, G, map, nmaps, st);
    }
    if (e != cudaSuccess) { set_error(std::string("alm2map launch: ") + cudaGetErrorString(e)); return SHT_ECUDA; }
    return SHT_OK;
}

static sht_status do_map2alm(sht_plan* p, const double* map, double* alm, int nmaps, void* ws,
                             double s0, double s1, cudaStream_t st, uint8_t* img)
{
    cudaError_t e;
    if (p->precision == SHT_FP64) {
        double* T = (double*)ws;
        e = launch_fft_forward_f64(p, map, T, nmaps, st);
        if (e == cudaSuccess) e = launch_legendre_m2a_f64(p, T, alm, nmaps, s0, s1, st);
    } else {
        // s0, s1 are the complete output factors (dsigma for map2alm)
        float2* T = (float2*)ws;
        unsigned int* cm = (unsigned int*)((char*)ws + round_up(tbuf_bytes(p, nmaps), 256));
        e = launch_fft_forward_split(p, map, T, cm, nmaps, st);
        if (e == cudaSuccess)
            e = launch_legendre_m2a_tc(p, T, (const float*)cm, img, alm, nmaps, s0, s1, st);
    }
    if (e != cudaSuccess) { set_error(std::string("map2alm launch: ") + cudaGetErrorString(e)); return SHT_ECUDA; }
    return SHT_OK;
}

sht_status sht_alm2map(sht_plan* p, const void* alm, void* map, int nmaps, void* ws, size_t wsb,
                       void* stream)
{
    sht_status s = check_call(p, alm, map, nmaps, ws, wsb, 0);
    if (s != SHT_OK) return s;
    cudaSetDevice(p->device);
    return do_alm2map(p, (const double*)alm, (double*)map, nmaps, ws, 1.0, 1.0, (cudaStream_t)stream);
}

sht_status sht_map2alm(sht_plan* p, const void* map, void* alm, int nmaps, int niter, void* ws,
                       size_t wsb, void* stream)
{
    sht_status s = check_call(p, map, alm, nmaps, ws, wsb, niter);
    if (s != SHT_OK) return s;
    cudaSetDevice(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const double dsig = 4.0 * PI_D / (double)p->npix;
    uint8_t* img = (uint8_t*)ws + (niter > 0 ? iter_ws(p, nmaps).img : img_offset(p, nmaps));
    s = do_map2alm(p, (const double*)map, (double*)alm, nmaps, ws, dsig, dsig, st, img);
    if (s != SHT_OK || niter == 0) return s;
    // Algorithm 2, a += map2alm(T - alm2map(a)) niter times, restricted to the
    // ring spectra: T (kept from the first pass) - F(G) with G the Legendre
    // alm2map of a and F what the backward + forward FFTs do to it (the
    // Fourier-domain residual, fft.cu), so the iteration runs no FFT.
    const IterWs w = iter_ws(p, nmaps);
    char* base = (char*)ws;
    double* da = (double*)(base + w.da);
    const long long na = (long long)nmaps * p->ncomp * p->nalm * 2;
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < niter && e == cudaSuccess; it++) {
        if (p->precision == SHT_FP64) {
            double* G = (double*)(base + w.g);
            e = launch_legendre_a2m_f64(p, (const double*)alm, G, nmaps, 1.0, 1.0, st);
            if (e == cudaSuccess) e = launch_alias_residual(p, ws, G, G, nmaps, st);
            if (e == cudaSuccess) e = launch_legendre_m2a_f64(p, G, da, nmaps, dsig, dsig, st);
        } else {
            float* G = (float*)(base + w.g);
            float2* A2 = (float2*)(base + w.g + split_a2_offset(p, nmaps));
            float2* D = (float2*)(base + w.d);
            unsigned int* cm = (unsigned int*)(base + w.cm);
            e = launch_alm_prep(p, (const double*)alm, A2, cm, nmaps, st);
            uint8_t* img = (uint8_t*)(base + w.img);
            if (e == cudaSuccess) e = launch_legendre_a2m_tc(p, A2, (const float*)cm, img, G, nmaps, 1.0f, 1.0f, st);
            if (e == cudaSuccess) e = launch_alias_residual(p, ws, G, D, nmaps, st);
            if (e == cudaSuccess) e = launch_colmax_T(p, D, cm, nmaps, st);
            if (e == cudaSuccess) e = launch_legendre_m2a_tc(p, D, (const float*)cm, img, da, nmaps, dsig, dsig, st);
        }
        if (e != cudaSuccess) break;
        prof_start("k_add", st);
        k_add<<<ew_grid(na), 256, 0, st>>>((double*)alm, da, na);
        prof_stop(st);
        count_launch();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { set_error(std::string("map2alm iteration: ") + cudaGetErrorString(e)); return SHT_ECUDA; }
    return SHT_OK;
}

// E-only / B-only transforms of spin-2 plans (Sec. 3.1: pipelines that need
// one of a_E, a_B). map2alm: the ring FFTs of Q and U, then a contraction
// over the two columns per map that form the kept component (half of the
// spin-2 contraction). alm2map from one component: the other is zero.
static sht_status check_eb(const sht_plan* p, int which)
{
    if (p->spin != 2) { set_error("E/B transforms need a spin-2 plan"); return SHT_EINVAL; }
    if (which != 0 && which != 1) { set_error("which must be 0 (E) or 1 (B)"); return SHT_EINVAL; }
    return SHT_OK;
}

sht_status sht_map2alm_eb(sht_plan* p, const void* map, void* alm, int nmaps, int which, void* ws, size_t wsb,
                          void* stream)
{
    sht_status s = check_call(p, map, alm, nmaps, ws, wsb, 0);
    if (s != SHT_OK) return s;
    if ((s = check_eb(p, which)) != SHT_OK) return s;
    cudaSetDevice(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const double dsig = 4.0 * PI_D / (double)p->npix;
    cudaError_t e;
    if (p->precision == SHT_FP64) {
        double* T = (double*)ws;
        e = launch_fft_forward_f64(p, (const double*)map, T, nmaps, st);
        if (e == cudaSuccess)
            e = launch_legendre_m2a_f64_comp(p, T, (double*)alm, nmaps, dsig, dsig, which + 1, st);
    } else {
        float2* T = (float2*)ws;
        unsigned int* cm = (unsigned int*)((char*)ws + round_up(tbuf_bytes(p, nmaps), 256));
        e = launch_fft_forward_split(p, (const double*)map, T, cm, nmaps, st);
        if (e == cudaSuccess)
            e = launch_legendre_m2a_tc(p, T, (const float*)cm, (uint8_t*)ws + img_offset(p, nmaps), (double*)alm,
                                       nmaps, dsig, dsig, st, which + 1);
    }
    if (e != cudaSuccess) { set_error(std::string("map2alm_eb launch: ") + cudaGetErrorString(e)); return SHT_ECUDA; }
    return SHT_OK;
}

size_t sht_workspace_bytes_eb(const sht_plan* p, int nmaps)
{
    if (!p || nmaps < 1) return 0;
    return round_up((size_t)nmaps * 2 * (size_t)p->nalm * 2 * sizeof(double), 256) + ws_bytes(p, nmaps, 0);
}

sht_status sht_alm2map_eb(sht_plan* p, const void* alm, void* map, int nmaps, int which, void* ws, size_t wsb,
                          void* stream)
{
    t_err.clear();
    reset_launches();
    if (!p) { set_error("plan is NULL"); return SHT_EINVAL; }
    sht_status s = check_eb(p, which);
    if (s != SHT_OK) return s;
    if (nmaps < 1) { set_error("nmaps must be >= 1"); return SHT_EINVAL; }
    if (!alm || !map) { set_error("data pointer is NULL"); return SHT_EINVAL; }
    if (((uintptr_t)alm & 15) || ((uintptr_t)map & 15)) { set_error("data pointers must be 16-byte aligned"); return SHT_EINVAL; }
    const size_t need = sht_workspace_bytes_eb(p, nmaps);
    if (!ws || wsb < need) { set_error("workspace too small: need " + std::to_string(need) + " bytes"); return SHT_EINVAL; }
    if ((uintptr_t)ws & 255) { set_error("workspace must be 256-byte aligned"); return SHT_EINVAL; }
    cudaSetDevice(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t fb = round_up((size_t)nmaps * 2 * (size_t)p->nalm * 2 * sizeof(double), 256);
    cudaError_t e = expand_component(p, alm, ws, nmaps, which, st);
    if (e != cudaSuccess) { set_error(std::string("alm2map_eb copy: ") + cudaGetErrorString(e)); return SHT_ECUDA; }
    return do_alm2map(p, (const double*)ws, (double*)map, nmaps, (char*)ws + fb, 1.0, 1.0, st);
}

// Algorithm 3 (immediate iteration), FP64 plans: ring spectra T of the map,
// the current coefficients' spectra G and the residual D of one order at a
// time, each [m][q][p][c] in FP64. Spin 2 runs on the Q and U columns: the
// order-m spectra of the two real maps carry the orders m and -m of Q + iU,
// so one step refines a_E, a_B at order m and resynthesises both.
size_t sht_workspace_bytes_immediate(const sht_plan* p, int nmaps)
{
    if (!p || nmaps < 1) return 0;
    const size_t n = (size_t)(p->mmax + 1) * 2 * (size_t)p->R * (size_t)ncols(p, nmaps) * sizeof(double);
    return 3 * round_up(n, 256);
}

sht_status sht_map2alm_immediate(sht_plan* p, const void* map, void* alm, int nmaps, int npass, void* ws,
                                 size_t wsb, void* stream)
{
    t_err.clear();
    reset_launches();
    if (!p) { set_error("plan is NULL"); return SHT_EINVAL; }
    if (p->precision != SHT_FP64) {
        set_error("the immediate iteration is built for FP64 plans");
        return SHT_EUNSUPPORTED;
    }
    if (nmaps < 1) { set_error("nmaps must be >= 1"); return SHT_EINVAL; }
    if (npass < 1) { set_error("npass must be >= 1"); return SHT_EINVAL; }
    if (!map || !alm) { set_error("data pointer is NULL"); return SHT_EINVAL; }
    if (((uintptr_t)map & 15) || ((uintptr_t)alm & 15)) { set_error("data pointers must be 16-byte aligned"); return SHT_EINVAL; }
    const size_t need = sht_workspace_bytes_immediate(p, nmaps);
    if (!ws || wsb < need) { set_error("workspace too small: need " + std::to_string(need) + " bytes"); return SHT_EINVAL; }
    if ((uintptr_t)ws & 255) { set_error("workspace must be 256-byte aligned"); return SHT_EINVAL; }
    cudaSetDevice(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t tb = need / 3;
    double* T = (double*)ws;
    double* G = (double*)((char*)ws + tb);
    double* D = (double*)((char*)ws + 2 * tb);
    const double dsig = 4.0 * PI_D / (double)p->npix;
    // a = 0, so the coefficients' spectra G = 0 and the first residual is T
    cudaError_t e = launch_fft_forward_f64(p, (const double*)map, T, nmaps, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(alm, 0, (size_t)nmaps * p->ncomp * p->nalm * 2 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, tb, st);
    // each order m in turn: its residual from the current G of every order
    // sharing its ring bins, its correction added to a at once, and its G
    // recomputed from the updated a, so the orders after it see the update.
    // Orders m and m' share a bin of a ring of N pixels only if m' = +-m
    // (mod N), and every HEALPix ring has a multiple of 4 pixels, so an even
    // and an odd order never do: the orders 2t and 2t + 1 run in one step,
    // each seeing exactly the updates the sequential sweep gives it.
    for (int pass = 0; pass < npass && e == cudaSuccess; pass++)
        for (int m0 = 0; m0 <= p->mmax && e == cudaSuccess; m0 += 2) {
            const int nm = std::min(2, p->mmax + 1 - m0);
            e = launch_alias_residual_order(p, T, G, D, nmaps, m0, nm, st);
            if (e == cudaSuccess)
                e = launch_legendre_m2a_f64_order(p, D, (double*)alm, nmaps, dsig, dsig, m0, nm, true, st);
            if (e == cudaSuccess) e = launch_legendre_a2m_f64_order(p, (const double*)alm, G, nmaps, m0, nm, st);
        }
    if (e != cudaSuccess) { set_error(std::string("immediate iteration: ") + cudaGetErrorString(e)); return SHT_ECUDA; }
    return SHT_OK;
}

sht_status sht_alm2map_adjoint(sht_plan* p, const void* map, void* alm, int nmaps, void* ws,
                               size_t wsb, void* stream)
{
    // (Npix/4pi) map2alm(h) * w_m: the dsigma of map2alm cancels
    sht_status s = check_call(p, map, alm, nmaps, ws, wsb, 0);
    if (s != SHT_OK) return s;
    cudaSetDevice(p->device);
    return do_map2alm(p, (const double*)map, (double*)alm, nmaps, ws, 1.0, 2.0, (cudaStream_t)stream,
                      (uint8_t*)ws + img_offset(p, nmaps));
}

sht_status sht_map2alm_adjoint(sht_plan* p, const void* alm, void* map, int nmaps, void* ws,
                               size_t wsb, void* stream)
{
    // (4pi/Npix) alm2map(g'), g'_l0 = Re g_l0, g'_lm = g_lm / 2
    sht_status s = check_call(p, alm, map, nmaps, ws, wsb, 0);
    if (s != SHT_OK) return s;
    cudaSetDevice(p->device);
    const double dsig = 4.0 * PI_D / (double)p->npix;
    return do_alm2map(p, (const double*)alm, (double*)map, nmaps, ws, dsig, 0.5 * dsig,
                      (cudaStream_t)stream);
}

// ---- host-buffer entry points: a three-stage pipeline over map chunks ----
// Chunk k's host->device copy (copy stream), transform (the caller's stream)
// and device->host copy (second copy stream) overlap with chunk k+1's copy in
// and chunk k-1's copy out; two device buffers per direction alternate.
// Events order the stages: in_ready[b] (copy in done), comp_done[b]
// (transform done: buffer b's input may be overwritten, its output copied
// out) and out_done[b] (copy out done: buffer b's output may be overwritten).
// Pageable caller buffers go through pinned staging, one buffer per parity.
static sht_status host_call(sht_plan* p, const void* in_host, void* out_host, int nmaps, int niter,
                            bool to_map, cudaStream_t st)
{
    t_err.clear();
    if (!p || !in_host || !out_host || nmaps < 1 || niter < 0) { set_error("bad argument"); return SHT_EINVAL; }
    cudaSetDevice(p->device);
    const size_t map_b = (size_t)p->ncomp * p->npix * sizeof(double);
    const size_t alm_b = (size_t)p->ncomp * p->nalm * 2 * sizeof(double);
    const size_t in_b = to_map ? alm_b : map_b, out_b = to_map ? map_b : alm_b;
    int chunk = nmaps;
    // device memory of one call: two buffer pairs and a workspace of a chunk
    size_t cap = (size_t)48 << 30;
    if (const char* env = std::getenv("SHT_HOST_CHUNK_GB")) {
        const long long g = std::atoll(env);
        if (g >= 1) cap = (size_t)g << 30;
    }
    while (chunk > 1 && 2 * (size_t)chunk * (in_b + out_b) + ws_bytes(p, chunk, niter) > cap) chunk = (chunk + 1) / 2;
    if (const char* env = std::getenv("SHT_HOST_CHUNK_MAPS")) {      // smaller chunks (tests)
        const int c = std::atoi(env);
        if (c >= 1) chunk = std::min(chunk, c);
    }
    const size_t cin = round_up((size_t)chunk * in_b, 256), cout = round_up((size_t)chunk * out_b, 256);
    auto grow_dev = [&](void** ptr, size_t* have, size_t need) -> cudaError_t {
        if (*have >= need) return cudaSuccess;
        if (*ptr) cudaFree(*ptr);
        *ptr = nullptr; *have = 0;
        cudaError_t e = cudaMalloc(ptr, need);
        if (e == cudaSuccess) *have = need;
        return e;
    };
    auto grow_pin = [&](void** ptr, size_t* have, size_t need) -> cudaError_t {
        if (*have >= need) return cudaSuccess;
        if (*ptr) cudaFreeHost(*ptr);
        *ptr = nullptr; *have = 0;
        cudaError_t e = cudaMallocHost(ptr, need);
        if (e == cudaSuccess) *have = need;
        return e;
    };
    // pinned (page-locked) caller buffers are copied directly; pageable ones
    // are staged through the plan's pinned buffers
    auto is_pinned = [](const void* ptr) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
        return at.type == cudaMemoryTypeHost;
    };
    const bool in_pinned = is_pinned(in_host), out_pinned = is_pinned(out_host);
    SHT_CUDA_TRY(grow_dev(&p->host_dev_in, &p->host_dev_in_bytes, 2 * cin));
    SHT_CUDA_TRY(grow_dev(&p->host_dev_out, &p->host_dev_out_bytes, 2 * cout));
    SHT_CUDA_TRY(grow_dev(&p->host_ws, &p->host_ws_bytes, ws_bytes(p, chunk, niter)));
    if (!in_pinned) SHT_CUDA_TRY(grow_pin(&p->pin_in, &p->pin_in_bytes, 2 * cin));
    if (!out_pinned) SHT_CUDA_TRY(grow_pin(&p->pin_out, &p->pin_out_bytes, 2 * cout));
    if (!p->hp_h2d) {
        SHT_CUDA_TRY(cudaStreamCreateWithFlags(&p->hp_h2d, cudaStreamNonBlocking));
        SHT_CUDA_TRY(cudaStreamCreateWithFlags(&p->hp_d2h, cudaStreamNonBlocking));
        for (cudaEvent_t& ev : p->hp_ev) SHT_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    cudaEvent_t* in_ready = p->hp_ev;
    cudaEvent_t* comp_done = p->hp_ev + 2;
    cudaEvent_t* out_done = p->hp_ev + 4;
    char* dev_in = (char*)p->host_dev_in;
    char* dev_out = (char*)p->host_dev_out;
    const int nch = (nmaps + chunk - 1) / chunk;
    int launches = 0;
    // finish the pageable copy-out of chunk k (its device->host copy is queued)
    auto finish_out = [&](int k) -> cudaError_t {
        if (out_pinned || k < 0) return cudaSuccess;
        const int b = k & 1, b0 = k * chunk, nb = std::min(chunk, nmaps - b0);
        cudaError_t e = cudaEventSynchronize(out_done[b]);
        if (e == cudaSuccess) memcpy((char*)out_host + (size_t)b0 * out_b, (char*)p->pin_out + b * cout, (size_t)nb * out_b);
        return e;
    };
    for (int k = 0; k < nch; k++) {
        const int b = k & 1, b0 = k * chunk, nb = std::min(chunk, nmaps - b0);
        // copy in: the transform of chunk k - 2 must be done with buffer b
        const char* src = (const char*)in_host + (size_t)b0 * in_b;
        if (k >= 2) SHT_CUDA_TRY(cudaStreamWaitEvent(p->hp_h2d, comp_done[b], 0));
        if (!in_pinned) {
            if (k >= 2) SHT_CUDA_TRY(cudaEventSynchronize(in_ready[b]));    // staging b copied in
            memcpy((char*)p->pin_in + b * cin, src, (size_t)nb * in_b);
            src = (const char*)p->pin_in + b * cin;
        }
        SHT_CUDA_TRY(cudaMemcpyAsync(dev_in + b * cin, src, (size_t)nb * in_b, cudaMemcpyHostToDevice, p->hp_h2d));
        SHT_CUDA_TRY(cudaEventRecord(in_ready[b], p->hp_h2d));
        // transform: its input is in, and output buffer b has been copied out
        SHT_CUDA_TRY(cudaStreamWaitEvent(st, in_ready[b], 0));
        if (k >= 2) SHT_CUDA_TRY(cudaStreamWaitEvent(st, out_done[b], 0));
        sht_status s = to_map
            ? sht_alm2map(p, dev_in + b * cin, dev_out + b * cout, nb, p->host_ws, p->host_ws_bytes, st)
            : sht_map2alm(p, dev_in + b * cin, dev_out + b * cout, nb, niter, p->host_ws, p->host_ws_bytes, st);
        if (s != SHT_OK) {
            cudaStreamSynchronize(p->hp_h2d);
            cudaStreamSynchronize(p->hp_d2h);
            return s;
        }
        launches += t_launches;
        SHT_CUDA_TRY(cudaEventRecord(comp_done[b], st));
        // copy out
        char* dst = out_pinned ? (char*)out_host + (size_t)b0 * out_b : (char*)p->pin_out + b * cout;
        SHT_CUDA_TRY(cudaStreamWaitEvent(p->hp_d2h, comp_done[b], 0));
        SHT_CUDA_TRY(cudaMemcpyAsync(dst, dev_out + b * cout, (size_t)nb * out_b, cudaMemcpyDeviceToHost, p->hp_d2h));
        SHT_CUDA_TRY(cudaEventRecord(out_done[b], p->hp_d2h));
        SHT_CUDA_TRY(finish_out(k - 1));
    }
    SHT_CUDA_TRY(finish_out(nch - 1));
    SHT_CUDA_TRY(cudaStreamSynchronize(p->hp_d2h));
    SHT_CUDA_TRY(cudaStreamSynchronize(st));
    t_launches = launches;
    return SHT_OK;
}

sht_status sht_alm2map_host(sht_plan* p, const void* alm_host, void* map_host, int nmaps, void* stream)
{
    return host_call(p, alm_host, map_host, nmaps, 0, true, (cudaStream_t)stream);
}

sht_status sht_map2alm_host(sht_plan* p, const void* map_host, void* alm_host, int nmaps, int niter,
                            void* stream)
{
    return host_call(p, map_host, alm_host, nmaps, niter, false, (cudaStream_t)stream);
}

}  // extern "C"
