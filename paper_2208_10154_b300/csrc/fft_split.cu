// fft_split.cu -- ring FFTs of the split-precision form in compensated FP32.
//
// A plain FP32 radix-2 FFT of 2048 points has an RMS error of ~1.3e-7 of the
// signal RMS (5.96e-7 worst over 4e5 outputs), too close to the 1e-6 bar of
// the split form, and FP64 arithmetic runs at ~1/64 of FP32 on this GPU. So
// every complex value is carried as an unevaluated sum hi + lo of two FP32
// numbers. Outside the transforms (loading, bin assembly) these are
// double-float pairs (TwoSum additions, FMA products with hi/lo constants);
// inside, a fixed-grid form (below) makes every addition exact at the cost
// of two packed FP32 additions. Phases e^{+-i pi m / N} come from a hi/lo
// table per ring length.
//
// Structure (Sec. 2.1 eq:mm; Appendix A.1 for m -> bin m mod N) is that of
// fft.cu: one complex FFT of x_north + i x_south per ring pair, sizes 2^a and
// 3^b 2^a directly, Bluestein's chirp convolution otherwise. Each CTA
// transforms one ring pair for two map columns at once (so a T / G row write
// covers 32 contiguous bytes) with radix-8 passes (three radix-2 stages per
// shared-memory round trip), and the rings are launched in classes of equal
// FFT size so the shared-memory footprint and thread count fit each size; the
// classes of one call run on the caller's stream and two helper streams.
// Ring optimisation (Sec. 3.1): with a per-pair order limit mlim[p] (the
// orders whose lambda is not negligible on the pair), the forward transform
// writes T and its column maxima for m <= mlim[p] only and the backward one
// folds only those orders.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace sht {

struct __align__(16) cx { float hr, hi, lr, li; };   // (hr + lr) + i (hi + li); 16-byte aligned: one 128-bit access

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// additions on the (re, im) pairs as packed FP32x2 operations (both lanes at
// once; every lane rounds exactly as the scalar TwoSum would)
__device__ __forceinline__ unsigned long long pk2(float a, float b)
{
    return tc::f2_pack(__float_as_uint(a), __float_as_uint(b));
}
__device__ __forceinline__ void up2(unsigned long long v, float& a, float& b)
{
    uint32_t x, y;
    tc::f2_unpack(v, x, y);
    a = __uint_as_float(x);
    b = __uint_as_float(y);
}
__device__ __forceinline__ cx caddc(const cx& a, const cx& b)
{
    using namespace tc;
    const unsigned long long A = pk2(a.hr, a.hi), B = pk2(b.hr, b.hi);
    const unsigned long long S = f2_add(A, B), BB = f2_sub(S, A);
    const unsigned long long E = f2_add(f2_sub(A, f2_sub(S, BB)), f2_sub(B, BB));
    const unsigned long long L = f2_add(f2_add(pk2(a.lr, a.li), pk2(b.lr, b.li)), E);
    cx s;
    up2(S, s.hr, s.hi);
    up2(L, s.lr, s.li);
    return s;
}
// a - b: TwoSum of a and -b, written with subtractions ((-b) - bb = -(b + bb) exactly)
__device__ __forceinline__ cx csubc(const cx& a, const cx& b)
{
    using namespace tc;
    const unsigned long long A = pk2(a.hr, a.hi), B = pk2(b.hr, b.hi);
    const unsigned long long S = f2_sub(A, B), BB = f2_sub(S, A);
    const unsigned long long E = f2_sub(f2_sub(A, f2_sub(S, BB)), f2_add(B, BB));
    const unsigned long long L = f2_add(f2_sub(pk2(a.lr, a.li), pk2(b.lr, b.li)), E);
    cx s;
    up2(S, s.hr, s.hi);
    up2(L, s.lr, s.li);
    return s;
}
// x * w with w = wh + wl (hi/lo twiddle); the products of the hi parts are
// error-free (FMA residuals) and their sum a TwoSum, so only the lo terms
// round. Packed: lane 0 the real part, lane 1 the imaginary part.
__device__ __forceinline__ cx cmulc(const cx& x, float2 wh, float2 wl)
{
    using namespace tc;
    const unsigned long long WH = pk2(wh.x, wh.y), WS = pk2(-wh.y, wh.x);
    const unsigned long long XR = pk2(x.hr, x.hr), XI = pk2(x.hi, x.hi);
    const unsigned long long P1 = f2_mul(XR, WH), P2 = f2_mul(XI, WS);      // (hr wx, hr wy), (-hi wy, hi wx)
    // minus the rounding errors of P1 and P2 (exact)
    const unsigned long long N1 = f2_fma(pk2(-x.hr, -x.hr), WH, P1), N2 = f2_fma(pk2(-x.hi, -x.hi), WS, P2);
    const unsigned long long S = f2_add(P1, P2), BB = f2_sub(S, P1);
    const unsigned long long E = f2_add(f2_sub(P1, f2_sub(S, BB)), f2_sub(P2, BB));
    const unsigned long long Q1 = f2_fma(pk2(x.li, x.li), WS, f2_mul(pk2(x.lr, x.lr), WH));
    const unsigned long long Q2 = f2_fma(XI, pk2(-wl.y, wl.x), f2_mul(XR, pk2(wl.x, wl.y)));
    const unsigned long long L = f2_add(f2_add(f2_sub(E, f2_add(N1, N2)), Q1), Q2);
    cx t;
    up2(S, t.hr, t.hi);
    up2(L, t.lr, t.li);
    return t;
}
__device__ __forceinline__ cx cscale(cx a, float s) { a.hr *= s; a.hi *= s; a.lr *= s; a.li *= s; return a; }
__device__ __forceinline__ cx cconjc(cx a) { a.hi = -a.hi; a.li = -a.li; return a; }
__device__ __forceinline__ cx czero() { cx z; z.hr = z.hi = z.lr = z.li = 0.0f; return z; }
__device__ __forceinline__ float cre(const cx& a) { return a.hr + a.lr; }
__device__ __forceinline__ float cim(const cx& a) { return a.hi + a.li; }

__device__ __forceinline__ int brev_c(int i, int logm) { return (int)(__brev((unsigned)i) >> (32 - logm)); }

// ---- grid arithmetic: the transforms proper ----------------------------
// Inside a transform a value is hi + lo with hi an integer-valued FP32 number
// and lo an FP32 correction of at most a few units. The sequence is first
// scaled by a power of two 2^-K such that every partial sum of the transform
// stays below 2^hb in magnitude (the complex L1 bound: at most N nonzero
// points of components below max, 2 sqrt(2) N max; hb = 21 for the forward
// transforms, whose epilogue doubles the bins before a product, 22 for the
// backward ones). Then the hi parts of a sum are integers below 2^24 and add
// exactly, so an addition is two packed FP32 additions with no error term; a
// product rounds hi w to an integer inside the FMA (adding 1.5 2^23 puts the
// units digit at the last place; |hi w| <= 2^22) and keeps the remainder
// hi w - round(hi w), exact to 2^-25, with the lo terms in lo. Every pass
// moves the integer part of lo back into hi (grenorm), so lo stays below a
// few units and its FP32 rounding near 2^-23 units per step (without it lo
// sums the remainders of every product upstream, and at N = 2048 that alone
// doubled the split form's alm2map error).
constexpr float GRND = 12582912.0f;      // 1.5 * 2^23

__device__ __forceinline__ cx gadd(const cx& a, const cx& b)
{
    using namespace tc;
    cx s;
    up2(f2_add(pk2(a.hr, a.hi), pk2(b.hr, b.hi)), s.hr, s.hi);
    up2(f2_add(pk2(a.lr, a.li), pk2(b.lr, b.li)), s.lr, s.li);
    return s;
}
__device__ __forceinline__ cx gsub(const cx& a, const cx& b)
{
    using namespace tc;
    cx s;
    up2(f2_sub(pk2(a.hr, a.hi), pk2(b.hr, b.hi)), s.hr, s.hi);
    up2(f2_sub(pk2(a.lr, a.li), pk2(b.lr, b.li)), s.lr, s.li);
    return s;
}
// x * w, w = wh + wl a hi/lo twiddle, |x| <= 2^22. Lane 0 the real part,
// lane 1 the imaginary part: hi = round(xr w) + round(xi (-wy, wx)).
__device__ __forceinline__ cx gmul(const cx& x, float2 wh, float2 wl)
{
    using namespace tc;
    const unsigned long long CC = pk2(GRND, GRND);
    const unsigned long long WH = pk2(wh.x, wh.y), WS = pk2(-wh.y, wh.x);
    const unsigned long long XR = pk2(x.hr, x.hr), XI = pk2(x.hi, x.hi);
    const unsigned long long T1 = f2_fma(XR, WH, CC), T2 = f2_fma(XI, WS, CC);
    const unsigned long long N1 = f2_sub(CC, T1), N2 = f2_sub(CC, T2);    // -round(xr w), -round(xi ws)
    const unsigned long long H = f2_sub(f2_sub(T1, CC), N2);             // integers: exact
    unsigned long long L = f2_fma(XR, WH, N1);                           // xr w - round(xr w)
    L = f2_fma(pk2(x.lr, x.lr), WH, L);
    L = f2_fma(pk2(x.li, x.li), WS, L);
    L = f2_fma(XR, pk2(wl.x, wl.y), L);
    L = f2_fma(XI, pk2(-wl.y, wl.x), L);
    L = f2_add(L, f2_fma(XI, WS, N2));
    cx t;
    up2(H, t.hr, t.hi);
    up2(L, t.lr, t.li);
    return t;
}
// x * c for a real c = ch + cl (|x| <= 2^22)
__device__ __forceinline__ cx gmulr(const cx& x, float ch, float cl)
{
    using namespace tc;
    const unsigned long long CC = pk2(GRND, GRND), C = pk2(ch, ch);
    const unsigned long long XH = pk2(x.hr, x.hi);
    const unsigned long long T = f2_fma(XH, C, CC);
    unsigned long long L = f2_fma(XH, C, f2_sub(CC, T));
    L = f2_fma(pk2(x.lr, x.li), C, f2_fma(XH, pk2(cl, cl), L));
    cx t;
    up2(f2_sub(T, CC), t.hr, t.hi);
    up2(L, t.lr, t.li);
    return t;
}
// a double-float value (hi + lo, normalised) times sc = 2^-K onto the grid
// (|hi sc| <= 2^22); the scaling is exact, the remainder too
__device__ __forceinline__ cx gquant(const cx& x, float sc)
{
    using namespace tc;
    const unsigned long long CC = pk2(GRND, GRND), S = pk2(sc, sc);
    const unsigned long long XH = pk2(x.hr, x.hi);
    const unsigned long long T = f2_fma(XH, S, CC);
    const unsigned long long L = f2_fma(pk2(x.lr, x.li), S, f2_fma(XH, S, f2_sub(CC, T)));
    cx t;
    up2(f2_sub(T, CC), t.hr, t.hi);
    up2(L, t.lr, t.li);
    return t;
}
// the integer part of lo moved into hi (exact): keeps |lo| <= 1/2 so that
// the FP32 rounding of lo stays at 2^-25 units however many products fed it
__device__ __forceinline__ cx grenorm(const cx& x)
{
    using namespace tc;
    const unsigned long long CC = pk2(GRND, GRND), XL = pk2(x.lr, x.li);
    const unsigned long long G = f2_sub(f2_add(XL, CC), CC);
    cx r;
    up2(f2_add(pk2(x.hr, x.hi), G), r.hr, r.hi);
    up2(f2_sub(XL, G), r.lr, r.li);
    return r;
}
// 2^k as an FP32 (k clamped to the normal range)
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + min(max(k, -126), 127)) << 23); }
// |hi| of both components as the larger FP32 bit pattern (order-preserving)
__device__ __forceinline__ unsigned absbits(const cx& z)
{
    return max(__float_as_uint(z.hr) & 0x7FFFFFFFu, __float_as_uint(z.hi) & 0x7FFFFFFFu);
}
// block-wide maxima of v0 (sequence 0) and v1 (sequence 1) into red[0], red[1]
// (every thread of the block calls this, outside divergent code)
__device__ __forceinline__ void red_max2(unsigned* red, unsigned v0, unsigned v1)
{
    v0 = __reduce_max_sync(0xffffffffu, v0);
    v1 = __reduce_max_sync(0xffffffffu, v1);
    if ((threadIdx.x & 31) == 0) {
        if (v0) atomicMax(red, v0);
        if (v1) atomicMax(red + 1, v1);
    }
}
// grid exponent K of a sequence of at most N nonzero points whose largest
// component has the FP32 bit pattern mb: |x| < 2^(E - 126) for the exponent
// field E, so 4 N max 2^-K <= 2^hb with K = E + ceil(log2 N) - 124 - hb
__device__ __forceinline__ int grid_k(unsigned mb, int N, int hb)
{
    const int E = (int)(mb >> 23);
    if (E == 0) return 0;
    return max(E + (32 - __clz(N - 1)) - 124 - hb, -126);
}

// a * (-i) and a * (+i): component swaps, exact
__device__ __forceinline__ cx cmul_mi(const cx& a) { cx r; r.hr = a.hi; r.lr = a.li; r.hi = -a.hr; r.li = -a.lr; return r; }
__device__ __forceinline__ cx cmul_pi(const cx& a) { cx r; r.hr = -a.hi; r.lr = -a.li; r.hi = a.hr; r.li = a.lr; return r; }

struct FftTabsF {
    const float4* twp;            // per size class: per-pass radix-8 twiddles (hi re, hi im, lo re, lo im)
    const float2 *twh, *twl;      // per size class: exp(-2 pi i u / M), u < M / 2, hi / lo
    const float2 *chh, *chl;      // Bluestein chirp, hi / lo
    const float2 *bhh, *bhl;      // Bluestein filter spectrum / M (digit-reversed), hi / lo
    const float2 *phh, *phl;      // exp(+i pi k / N), k < 2N, per ring length, hi / lo
    const long long* phoff;       // offset of each ring length's phase table
};

// twiddles of one FFT size M, staged in shared memory: exp(-2 pi i u / M),
// u < M / 2, as (hi re, hi im, lo re, lo im), at slot tw_slot(u). A pass reads
// u = k s for a power-of-two stride s, which in a plain table puts every lane
// of a warp on the same banks; XOR-ing the low three bits of u (the 16-byte
// slot within 128 bytes) with a fold of the higher bits spreads them (a
// bijection within each aligned block of eight).
__device__ __forceinline__ int tw_slot(int u)
{
    const int v = u >> 3;
    return u ^ ((v ^ (v >> 3) ^ (v >> 6) ^ (v >> 9)) & 7);
}
__device__ __forceinline__ void twid(const float4* tw, int idx, bool inv, float2& wh, float2& wl)
{
    const float4 v = tw[tw_slot(idx)];
    wh = make_float2(v.x, inv ? -v.y : v.y);
    wl = make_float2(v.z, inv ? -v.w : v.w);
}
// twiddle exp(-+2 pi i u / M) for 0 <= u < M (the staged table holds u < M / 2;
// u >= M / 2 is the negative of u - M / 2), branch-free per lane
__device__ __forceinline__ void twid_full(const float4* tw, int u, int M, bool inv, float2& wh, float2& wl)
{
    const int hm = M >> 1;
    const bool up = u >= hm;
    twid(tw, up ? u - hm : u, inv, wh, wl);
    const float sg = up ? -1.0f : 1.0f;
    wh.x *= sg; wh.y *= sg; wl.x *= sg; wl.y *= sg;
}

// copy the size-M twiddles of the class (table at offset ctw) into shared memory
__device__ __forceinline__ void stage_twiddles(float4* tw, int M, long long ctw, const FftTabsF& t)
{
    for (int u = threadIdx.x; u < M / 2; u += blockDim.x) {
        const float2 h = t.twh[ctw + u], l = t.twl[ctw + u];
        tw[tw_slot(u)] = make_float4(h.x, h.y, l.x, l.y);
    }
}

// the class's per-pass radix-8 twiddles (n float4 at offset ctwp) into shared memory
__device__ __forceinline__ void stage_pass_twiddles(float4* twp, int n, long long ctwp, const FftTabsF& t)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) twp[i] = t.twp[ctwp + i];
}

// Per-pass twiddles: the radix-8 pass of span h of a 2^L-point transform
// (h = 2^(L mod 3), 8 times that, ...) takes, for k < h, the seven factors
// W_{8h}^{k e}, e = 1 .. 7, at slots off(h) + 7 k + e - 1 with
// off(h) = h - 2^(L mod 3) (the sum of 7 h' over the smaller spans); 7 is odd,
// so a warp's 16-byte reads of consecutive k fall on distinct banks.
__device__ __forceinline__ void twp_get(const float4* e, int t, bool inv, float2& wh, float2& wl)
{
    const float4 v = e[t];
    wh = make_float2(v.x, inv ? -v.y : v.y);
    wl = make_float2(v.z, inv ? -v.w : v.w);
}

// Transform buffers in shared memory: sequence s of a size-M class starts at
// s * fft_pad_len(M), and its point i sits at fft_pad(i). One 16-byte slot of
// padding per 8 points and one more per 64 keep the 16-byte accesses of a
// warp on distinct banks for the bit-reversed input scatter, the first
// small-span passes and the consecutive runs of the other phases.
__host__ __device__ __forceinline__ int fft_pad(int i) { return i + (i >> 3) + (i >> 6); }
__host__ __device__ __forceinline__ int fft_pad_len(int M) { return M + (M >> 3) + (M >> 6); }

// 1/sqrt(2) as a double-float pair
constexpr float R2H = 0.707106769084930419921875f;
constexpr float R2L = 1.21016175477703189729e-08f;

// x * W_8 and x * W_8^3 (W_8 = e^{-+i pi / 4}): the sums are exact on the
// grid, then one product by 1/sqrt(2)
__device__ __forceinline__ cx mul_w8(const cx& x, bool inv)
{
    cx t;                                          // x (1 -+ i)
    if (!inv) { t.hr = x.hr + x.hi; t.lr = x.lr + x.li; t.hi = x.hi - x.hr; t.li = x.li - x.lr; }
    else      { t.hr = x.hr - x.hi; t.lr = x.lr - x.li; t.hi = x.hi + x.hr; t.li = x.li + x.lr; }
    return gmulr(t, R2H, R2L);
}
__device__ __forceinline__ cx mul_w83(const cx& x, bool inv)
{
    cx t;                                          // x (-1 -+ i)
    if (!inv) { t.hr = x.hi - x.hr; t.lr = x.li - x.lr; t.hi = -(x.hr + x.hi); t.li = -(x.lr + x.li); }
    else      { t.hr = -(x.hr + x.hi); t.lr = -(x.lr + x.li); t.hi = x.hr - x.hi; t.li = x.lr - x.li; }
    return gmulr(t, R2H, R2L);
}

// the 8-point DFT X_m = sum_j x_j W_8^{j m} of x in natural order (three
// radix-2 stages, W_8^2 = -+i exact)
__device__ __forceinline__ void dft8(cx (&x)[8], bool inv)
{
    const cx a0 = gadd(x[0], x[4]), b0 = gsub(x[0], x[4]);
    const cx a1 = gadd(x[1], x[5]), b1 = gsub(x[1], x[5]);
    const cx a2 = gadd(x[2], x[6]), b2 = gsub(x[2], x[6]);
    const cx a3 = gadd(x[3], x[7]), b3 = gsub(x[3], x[7]);
    const cx c0 = gadd(a0, a2), c2 = gsub(a0, a2), c1 = gadd(a1, a3);
    const cx c3 = inv ? cmul_pi(gsub(a1, a3)) : cmul_mi(gsub(a1, a3));
    x[0] = gadd(c0, c1); x[4] = gsub(c0, c1);
    x[2] = gadd(c2, c3); x[6] = gsub(c2, c3);
    const cx d1 = mul_w8(b1, inv), d3 = mul_w83(b3, inv);
    const cx d2 = inv ? cmul_pi(b2) : cmul_mi(b2);
    const cx e0 = gadd(b0, d2), e2 = gsub(b0, d2), e1 = gadd(d1, d3);
    const cx e3 = inv ? cmul_pi(gsub(d1, d3)) : cmul_mi(gsub(d1, d3));
    x[1] = gadd(e0, e1); x[5] = gsub(e0, e1);
    x[3] = gadd(e2, e3); x[7] = gsub(e2, e3);
}

// One radix-8 pass (three radix-2 stages) over nseq sequences of M = 2^L
// points (padded layout, P apart), span h of the last stage merged in.
// Decimation in time: the points y0 + j h hold sub-transforms in bit-reversed
// order, so the one at j takes W_{8h}^{k rev(j)} before the 8-point DFT, whose
// output m goes to y0 + m h. (the twiddle branch is per pass, not per lane)
__device__ __forceinline__ void dit8_pass(cx* buf, int nseq, int L, int h, const float4* tp, bool inv)
{
    const int M = 1 << L, P = fft_pad_len(M);
    const int ng = M >> 3;
    constexpr int rev[8] = {0, 4, 2, 6, 1, 5, 3, 7};
    for (int b = threadIdx.x; b < nseq * ng; b += blockDim.x) {
        const int f = b >> (L - 3), g = b & (ng - 1);
        const int k = g & (h - 1);
        cx* y = buf + f * P;
        const int y0 = ((g - k) << 3) + k;
        int ix[8];
        cx x[8];
#pragma unroll
        for (int j = 0; j < 8; j++) { ix[j] = fft_pad(y0 + j * h); x[j] = y[ix[j]]; }
        if (h > 1) {
            const float4* e = tp + 7 * k - 1;
#pragma unroll
            for (int j = 1; j < 8; j++) {
                float2 wh, wl;
                twp_get(e, rev[j], inv, wh, wl);
                x[j] = gmul(x[j], wh, wl);
            }
        }
        cx z[8];
#pragma unroll
        for (int j = 0; j < 8; j++) z[rev[j]] = x[j];
        dft8(z, inv);
#pragma unroll
        for (int j = 0; j < 8; j++) y[ix[j]] = grenorm(z[j]);
    }
}

// Decimation in frequency: the 8-point DFT of the points y0 + j h (natural
// order), output m times W_{8h}^{k m} to y0 + rev(m) h.
__device__ __forceinline__ void dif8_pass(cx* buf, int nseq, int L, int h, const float4* tp, bool inv)
{
    const int M = 1 << L, P = fft_pad_len(M);
    const int ng = M >> 3;
    constexpr int rev[8] = {0, 4, 2, 6, 1, 5, 3, 7};
    for (int b = threadIdx.x; b < nseq * ng; b += blockDim.x) {
        const int f = b >> (L - 3), g = b & (ng - 1);
        const int k = g & (h - 1);
        cx* y = buf + f * P;
        const int y0 = ((g - k) << 3) + k;
        int ix[8];
        cx x[8];
#pragma unroll
        for (int j = 0; j < 8; j++) { ix[j] = fft_pad(y0 + j * h); x[j] = y[ix[j]]; }
        dft8(x, inv);
        if (h > 1) {
            const float4* e = tp + 7 * k - 1;
#pragma unroll
            for (int m = 1; m < 8; m++) {
                float2 wh, wl;
                twp_get(e, m, inv, wh, wl);
                x[m] = gmul(x[m], wh, wl);
            }
        }
#pragma unroll
        for (int m = 0; m < 8; m++) y[ix[rev[m]]] = grenorm(x[m]);
    }
}

// radix-4 pass of spans 1 and 2 (no twiddles), decimation in time (bit-
// reversed sub-transforms of length 1 at y0 .. y0 + 3) or in frequency
// (natural input, bit-reversed output), over nseq sequences
__device__ __forceinline__ void r4_span1(cx* buf, int nseq, int L, bool inv, bool dif)
{
    const int M = 1 << L, P = fft_pad_len(M);
    for (int b = threadIdx.x; b < nseq * (M >> 2); b += blockDim.x) {
        cx* y = buf + (b >> (L - 2)) * P;
        const int y0 = (b & ((M >> 2) - 1)) << 2;
        const int i0 = fft_pad(y0), i1 = fft_pad(y0 + 1), i2 = fft_pad(y0 + 2), i3 = fft_pad(y0 + 3);
        const cx x0 = y[i0], x1 = y[i1], x2 = y[i2], x3 = y[i3];
        if (!dif) {
            // x1 and x2 are the bit-reversed sub-transforms 2 and 1
            const cx b0 = gadd(x0, x1), b1 = gsub(x0, x1), b2 = gadd(x2, x3), d = gsub(x2, x3);
            const cx b3 = inv ? cmul_pi(d) : cmul_mi(d);
            y[i0] = grenorm(gadd(b0, b2)); y[i2] = grenorm(gsub(b0, b2));
            y[i1] = grenorm(gadd(b1, b3)); y[i3] = grenorm(gsub(b1, b3));
        } else {
            const cx c0 = gadd(x0, x2), c2 = gsub(x0, x2), c1 = gadd(x1, x3), d = gsub(x1, x3);
            const cx c3 = inv ? cmul_pi(d) : cmul_mi(d);
            y[i0] = grenorm(gadd(c0, c1)); y[i1] = grenorm(gsub(c0, c1));
            y[i2] = grenorm(gadd(c2, c3)); y[i3] = grenorm(gsub(c2, c3));
        }
    }
}

// radix-2 stage of span 1 (twiddle 1) over nb sequences
__device__ __forceinline__ void r2_span1(cx* buf, int nb, int L)
{
    const int M = 1 << L, P = fft_pad_len(M);
    for (int b = threadIdx.x; b < nb * (M >> 1); b += blockDim.x) {
        cx* x = buf + (b >> (L - 1)) * P;
        const int i = (b & ((M >> 1) - 1)) * 2, i0 = fft_pad(i), i1 = fft_pad(i + 1);
        const cx a = x[i0], c = x[i1];
        x[i0] = grenorm(gadd(a, c));
        x[i1] = grenorm(gsub(a, c));
    }
    __syncthreads();
}

// In-place decimation-in-time FFTs of nb sequences of M = 2^L points (padded
// layout above), input in bit-reversed order, output natural: one radix-2 or
// radix-4 pass of span 1 for L = 1, 2 mod 3, then radix-8 passes.
// twp: the per-pass twiddles of the 2^L-point transform; W = exp(-+2 pi i / M).
__device__ void fft_dit(cx* buf, int nb, int L, const float4* twp, bool inv)
{
    const int r0 = L % 3;
    if (r0 == 1) r2_span1(buf, nb, L);
    if (r0 == 2) { r4_span1(buf, nb, L, inv, false); __syncthreads(); }
    for (int h = 1 << r0; 8 * h <= (1 << L); h <<= 3) {
        dit8_pass(buf, nb, L, h, twp + (h - (1 << r0)), inv);
        __syncthreads();
    }
}

// In-place decimation-in-frequency FFTs (natural input, bit-reversed output):
// radix-8 passes from span M / 8 down, then the radix-4 or radix-2 pass of span 1.
__device__ void fft_dif(cx* buf, int nb, int L, const float4* twp, bool inv)
{
    const int r0 = L % 3;
    for (int h = (1 << L) >> 3; h >= (1 << r0); h >>= 3) {
        dif8_pass(buf, nb, L, h, twp + (h - (1 << r0)), inv);
        __syncthreads();
    }
    if (r0 == 2) { r4_span1(buf, nb, L, inv, true); __syncthreads(); }
    if (r0 == 1) r2_span1(buf, nb, L);
}

// sqrt(3) / 2 as a double-float pair
constexpr float R3H = 0.866025388240814208984375f;
constexpr float R3L = 1.55436244377793497517e-08f;

// the 3-point DFT y_j = sum_i x_i e^{-+2 pi i i j / 3} on the grid: y0 = x0 + t,
// y1,2 = (x0 - t / 2) -+ i (sqrt 3 / 2)(x1 - x2), t = x1 + x2 (forward sign);
// t / 2 is rounded back onto the grid like a product
__device__ __forceinline__ void dft3(const cx& x0, const cx& x1, const cx& x2, bool inv, cx& y0, cx& y1, cx& y2)
{
    const cx t = gadd(x1, x2);
    y0 = gadd(x0, t);
    const cx u = gsub(x0, gmulr(t, 0.5f, 0.0f));
    const cx d = gmulr(gsub(x1, x2), R3H, R3L);
    const cx v = inv ? cmul_pi(d) : cmul_mi(d);
    y1 = gadd(u, v);
    y2 = gsub(u, v);
}

// Radix-3 stages of a size M = 3^b 2^a transform (padded layout, nb
// sequences), on the full sequences: decimation in frequency with spans M,
// M / 3, ... (before the power-of-two passes on the 3^b blocks of 2^a), or
// decimation in time with spans 3 2^a, ..., M (after them). The staged
// twiddles are those of size M: W_S^{j k} = W_M^{j k M / S}.
__device__ void r3_passes(cx* buf, int nb, int M, int p3, const float4* tw, bool inv, bool dif)
{
    const int P = fft_pad_len(M);
    const int nbf = M / 3;                           // butterflies per sequence and stage
    for (int st = 0, S = dif ? M : 3 * (M / p3); st < 64 && (dif ? S > M / p3 : S <= M);
         st++, S = dif ? S / 3 : S * 3) {
        const int Sp = S / 3, ms = M / S;
        const float rsp = 1.0f / (float)Sp;
        for (int b = threadIdx.x; b < nb * nbf; b += blockDim.x) {
            const int f = (b >= nbf) ? 1 : 0;            // nb <= 2 sequences
            const int r = b - f * nbf;
            // r / Sp through the FP32 reciprocal (r < 2^14: off by at most one)
            int blk = __float2int_rz((float)r * rsp);
            int k = r - blk * Sp;
            if (k < 0) { blk--; k += Sp; } else if (k >= Sp) { blk++; k -= Sp; }
            cx* y = buf + f * P;
            const int o = blk * S + k;
            const int i0 = fft_pad(o), i1 = fft_pad(o + Sp), i2 = fft_pad(o + 2 * Sp);
            float2 w1h, w1l, w2h, w2l;
            twid_full(tw, k * ms, M, inv, w1h, w1l);
            twid_full(tw, 2 * k * ms, M, inv, w2h, w2l);
            cx x0 = y[i0], x1 = y[i1], x2 = y[i2], y0, y1, y2;
            if (dif) {
                dft3(x0, x1, x2, inv, y0, y1, y2);
                y[i0] = grenorm(y0); y[i1] = grenorm(gmul(y1, w1h, w1l)); y[i2] = grenorm(gmul(y2, w2h, w2l));
            } else {
                dft3(x0, gmul(x1, w1h, w1l), gmul(x2, w2h, w2l), inv, y0, y1, y2);
                y[i0] = grenorm(y0); y[i1] = grenorm(y1); y[i2] = grenorm(y2);
            }
        }
        __syncthreads();
    }
}

// transforms of size M = p3 2^L: natural in, digit-reversed out (DIF) and
// digit-reversed in, natural out (DIT); p3 = 1 is the plain power-of-two case.
// tw: the size-M twiddles of the radix-3 stages (p3 > 1 only), twp: the
// per-pass twiddles of the 2^L-point part
__device__ __forceinline__ void fft_dif_m(cx* buf, int nb, int L, int p3, const float4* tw, const float4* twp, bool inv)
{
    if (p3 > 1) r3_passes(buf, nb, p3 << L, p3, tw, inv, true);
    fft_dif(buf, nb * p3, L, twp, inv);
}
__device__ __forceinline__ void fft_dit_m(cx* buf, int nb, int L, int p3, const float4* tw, const float4* twp, bool inv)
{
    fft_dit(buf, nb * p3, L, twp, inv);
    if (p3 > 1) r3_passes(buf, nb, p3 << L, p3, tw, inv, false);
}

// The forward DFTs of the nb sequences in buf, which hold double-float
// values at their input positions (natural order for Bluestein, the
// digit-reversed order of the passes otherwise). red[0], red[1]: the largest
// |component| of each sequence (block-reduced and published by the caller);
// red[2], red[3] zero on entry. Output in natural order on the grid, true
// values (hi + lo) 2^k of the returned exponents (x: sequence 0, y: 1).
__device__ __noinline__ int2 dftc_forward(cx* buf, int nb, const FftLen& f, const float4* tw, const float4* twp,
                             const FftTabsF& t, unsigned* red, int hb)
{
    const int M = f.m, L = 31 - __clz(M / f.p3), P = fft_pad_len(M);
    const int K0 = grid_k(red[0], f.n, hb), K1 = grid_k(red[1], f.n, hb);
    const float sc0 = pow2f(-K0), sc1 = pow2f(-K1);
    // onto the grid; Bluestein: times the chirp, zero beyond N (the table
    // loads of DUB points per thread are in flight before the first is used)
    constexpr int DUB = 4;
    if (!f.bluestein)
        for (int i = threadIdx.x; i < nb * M; i += blockDim.x) {
            const int s = (i >= M) ? 1 : 0, ii = i - s * M;   // nb <= 2 sequences
            cx& z = buf[s * P + fft_pad(ii)];
            z = gquant(z, s ? sc1 : sc0);
        }
    else
    for (int i0 = threadIdx.x; i0 < nb * M; i0 += DUB * blockDim.x) {
        float2 ch[DUB], cl[DUB];
#pragma unroll
        for (int u = 0; u < DUB; u++) {
            const int i = i0 + u * blockDim.x;
            const int s = (i >= M) ? 1 : 0, ii = i - s * M;   // nb <= 2 sequences
            ch[u] = make_float2(1.0f, 0.0f); cl[u] = make_float2(0.0f, 0.0f);
            if (i < nb * M && ii < f.n) { ch[u] = t.chh[f.chirp + ii]; cl[u] = t.chl[f.chirp + ii]; }
        }
#pragma unroll
        for (int u = 0; u < DUB; u++) {
            const int i = i0 + u * blockDim.x;
            if (i >= nb * M) break;
            const int s = (i >= M) ? 1 : 0, ii = i - s * M;
            cx& z = buf[s * P + fft_pad(ii)];
            z = (ii < f.n) ? gmul(gquant(z, s ? sc1 : sc0), ch[u], cl[u]) : czero();
        }
    }
    __syncthreads();
    if (!f.bluestein) {
        fft_dit_m(buf, nb, L, f.p3, tw, twp, false);
        return make_int2(K0, K1);
    }
    fft_dif_m(buf, nb, L, f.p3, tw, twp, false);
    // the filter product Y = Z b / M is rescaled by 2^-D so that the inverse
    // transform's partial sums (at most M terms of components below
    // sqrt(2) max|Z| 2^bexp) stay below 2^20 too
    unsigned m0 = 0, m1 = 0;
    for (int i = threadIdx.x; i < nb * M; i += blockDim.x) {
        const int s = (i >= M) ? 1 : 0, ii = i - s * M;
        const unsigned v = absbits(buf[s * P + fft_pad(ii)]);
        if (s) m1 = max(m1, v); else m0 = max(m0, v);
    }
    red_max2(red + 2, m0, m1);
    __syncthreads();
    const int lgm = 32 - __clz(M - 1);
    const int e0 = (int)(red[2] >> 23), e1 = (int)(red[3] >> 23);
    const int D0 = e0 ? e0 - 126 + lgm + f.bexp + 2 - hb : 0, D1 = e1 ? e1 - 126 + lgm + f.bexp + 2 - hb : 0;
    const float fs0 = pow2f(-D0), fs1 = pow2f(-D1);
    for (int i0 = threadIdx.x; i0 < nb * M; i0 += DUB * blockDim.x) {
        float2 bh[DUB], bl[DUB];
#pragma unroll
        for (int u = 0; u < DUB; u++) {
            const int i = i0 + u * blockDim.x;
            const int s = (i >= M) ? 1 : 0, ii = i - s * M;   // nb <= 2 sequences
            if (i < nb * M) { bh[u] = t.bhh[f.bhat + ii]; bl[u] = t.bhl[f.bhat + ii]; }
        }
#pragma unroll
        for (int u = 0; u < DUB; u++) {
            const int i = i0 + u * blockDim.x;
            if (i >= nb * M) break;
            const int s = (i >= M) ? 1 : 0, ii = i - s * M;
            cx& z = buf[s * P + fft_pad(ii)];
            const float fsc = s ? fs1 : fs0;
            z = gmul(z, make_float2(bh[u].x * fsc, bh[u].y * fsc), make_float2(bl[u].x * fsc, bl[u].y * fsc));
        }
    }
    __syncthreads();
    fft_dit_m(buf, nb, L, f.p3, tw, twp, true);
    // (the filter spectrum carries the 1 / M of the inverse transform: an
    // FP32 scale by 1 / M would round for M = 3^b 2^a)
    for (int i0 = threadIdx.x; i0 < nb * f.n; i0 += DUB * blockDim.x) {
        float2 ch[DUB], cl[DUB];
#pragma unroll
        for (int u = 0; u < DUB; u++) {
            const int i = i0 + u * blockDim.x;
            const int s = (i >= f.n) ? 1 : 0, k = i - s * f.n;
            if (i < nb * f.n) { ch[u] = t.chh[f.chirp + k]; cl[u] = t.chl[f.chirp + k]; }
        }
#pragma unroll
        for (int u = 0; u < DUB; u++) {
            const int i = i0 + u * blockDim.x;
            if (i >= nb * f.n) break;
            const int s = (i >= f.n) ? 1 : 0, k = i - s * f.n;
            cx& z = buf[s * P + fft_pad(k)];
            z = gmul(z, ch[u], cl[u]);
        }
    }
    __syncthreads();
    return make_int2(K0 + D0, K1 + D1);
}

// where input n goes: natural for Bluestein (decimation in frequency), else
// the digit-reversed position the decimation-in-time passes take: the base-3
// digits of n (least significant first) at spans M / 3, M / 9, ..., then the
// bit-reversed rest
__device__ __forceinline__ int placec(const FftLen& f, int n)
{
    if (f.bluestein) return n;
    if (f.p3 == 1) return brev_c(n, 31 - __clz(f.m));
    int p = 0, S = f.m;
    for (int q = f.p3; q > 1; q /= 3) { S /= 3; const int d = n % 3; n /= 3; p += d * S; }
    return p + brev_c(n, 31 - __clz(f.m / f.p3));
}

// e^{sgn i pi k / N} for k = m mod 2N (hi/lo)
__device__ __forceinline__ void phase(const FftTabsF& t, int fidx, int N, int m, bool neg, float2& ph, float2& pl)
{
    long long o = t.phoff[fidx] + ((m < 2 * N) ? m : m % (2 * N));
    ph = t.phh[o]; pl = t.phl[o];
    if (neg) { ph.y = -ph.y; pl.y = -pl.y; }
}

// ---------------------------------------------------------------------------
// forward: maps -> T[m][q][p][c] (FP32 hi/lo pairs) and the per (m, slot,
// column) maxima used for the tensor-core column quanta. One launch per FFT
// size class; grid.x = pair of map columns (map * ncomp + comp), grid.y = block
// of FWD_PB ring pairs of the class (neighbouring column pairs, which share
// the cache lines of T, run together).
// ---------------------------------------------------------------------------
constexpr int FWD_PB = 32;

// NT threads; in the epilogue lane pairs own m = threadIdx.x / 2 + jj NT / 2,
// jj < 8 (mmax < 4 NT)
template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
k_fftc_forward(const double* __restrict__ map, float2* __restrict__ T, unsigned int* __restrict__ colmax,
               const int* __restrict__ cls, int ncls, const PairGeom* __restrict__ pairs,
               const FftLen* __restrict__ ffts, FftTabsF tb, long long ctw, long long ctwp, int ntwp, int M,
               int R_, int mmax,
               long long npix, long long ncol, int nmc, int mpc, int pf, const int* __restrict__ mlim)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx* buf = reinterpret_cast<cx*>(smem_raw);
    const int P = fft_pad_len(M);
    // shared memory: the transform buffers, the per-pass twiddles, and for
    // sizes 3^b 2^a the size-M twiddles of the radix-3 stages
    // (ntwp < 0: the per-pass twiddles do not fit and stay in global memory)
    float4* twp_s = reinterpret_cast<float4*>(smem_raw + (size_t)mpc * P * sizeof(cx));
    float4* tw = twp_s + max(ntwp, 0);
    const float4* twp = (ntwp >= 0) ? twp_s : tb.twp + ctwp;
    if (ntwp > 0) stage_pass_twiddles(twp_s, ntwp, ctwp, tb);   // (the first __syncthreads below publishes them)
    if (M % 3 == 0) stage_twiddles(tw, M, ctw, tb);
    __shared__ unsigned red[4];                    // per ring pair: largest |component| of each sequence
    if (threadIdx.x < 4) red[threadIdx.x] = 0u;
    __syncthreads();
    const int mc0 = blockIdx.x * mpc;
    const int nb = min(mpc, nmc - mc0);
    const long long qstride = (long long)R_ * ncol;
    // epilogue: lanes 2k and 2k + 1 take the two columns of one order m, so
    // that a warp's T stores cover whole 32-byte sectors
    constexpr int FWD_MJ = 8;
    const int es = threadIdx.x & 1, et = threadIdx.x >> 1, ent = NT / 2;
    float mx[FWD_MJ][4];
#pragma unroll
    for (int j = 0; j < FWD_MJ; j++) mx[j][0] = mx[j][1] = mx[j][2] = mx[j][3] = 0.0f;
    const int iend = min(ncls, (int)(blockIdx.y + 1) * FWD_PB);
    for (int ip = blockIdx.y * FWD_PB; ip < iend; ip++) {
        const int p = cls[ip];
        const PairGeom g = pairs[p];
        const FftLen f = ffts[g.fft];
        const int N = g.n;
        // the orders this ring pair takes part in (the contraction skips the
        // others, whose lambda is negligible on this ring): T and the column
        // maxima are written for m <= ml only
        const int ml = mlim ? min(mmax, mlim[p]) : mmax;
        // the next ring pair's rows into L2 while this one is transformed (pf:
        // the map is 16-byte aligned; rows start at even pixels, N = 4i)
        if (pf && ip + 1 < iend && threadIdx.x < 2 * nb) {
            const PairGeom gn = pairs[cls[ip + 1]];
            const int s = threadIdx.x >> 1, r = threadIdx.x & 1;
            if (!r || gn.start_s >= 0)
                tc::prefetch_l2_bulk(map + (long long)(mc0 + s) * npix + (r ? gn.start_s : gn.start_n),
                                     (uint32_t)gn.n * 8u);
        }
        // the ring's samples in batches of FWD_UB per thread: every load of a
        // batch is in flight before the first is used
        constexpr int FWD_UB = 8;
        unsigned m0 = 0, m1 = 0;
        for (int e0 = threadIdx.x; e0 < nb * N; e0 += FWD_UB * NT) {
            double vn[FWD_UB], vs[FWD_UB];
#pragma unroll
            for (int u = 0; u < FWD_UB; u++) {
                const int e = e0 + u * NT;
                vn[u] = 0.0; vs[u] = 0.0;
                if (e < nb * N) {
                    const int s = (e >= N) ? 1 : 0, n = e - s * N;     // nb <= 2 sequences
                    const double* mp = map + (long long)(mc0 + s) * npix;
                    vn[u] = mp[g.start_n + n];
                    if (g.start_s >= 0) vs[u] = mp[g.start_s + n];
                }
            }
#pragma unroll
            for (int u = 0; u < FWD_UB; u++) {
                const int e = e0 + u * NT;
                if (e < nb * N) {
                    const int s = (e >= N) ? 1 : 0, n = e - s * N;     // nb <= 2 sequences
                    cx z = czero();
                    tc::f64_split_scaled(vn[u], 0, z.hr, z.lr);
                    if (g.start_s >= 0) tc::f64_split_scaled(vs[u], 0, z.hi, z.li);
                    buf[s * P + fft_pad(placec(f, n))] = z;
                    const unsigned v = absbits(z);
                    if (s) m1 = max(m1, v); else m0 = max(m0, v);
                }
            }
        }
        red_max2(red, m0, m1);
        __syncthreads();
        const int2 kq = dftc_forward(buf, nb, f, tw, twp, tb, red, 21);
        // the bins hold 2^-K times the spectrum; E and O below are twice the
        // true ones (the halvings of the split fold into the output scale)
        const float osc0 = pow2f(kq.x - 1), osc1 = pow2f(kq.y - 1);
        if (threadIdx.x < 4) red[threadIdx.x] = 0u;    // (read by every thread before the syncs above)
        // the phases of this lane's orders first (all loads in flight)
        float2 PH[FWD_MJ], PL[FWD_MJ];
#pragma unroll
        for (int jj = 0; jj < FWD_MJ; jj++) {
            const int m = et + jj * ent;
            PH[jj] = make_float2(1.0f, 0.0f); PL[jj] = make_float2(0.0f, 0.0f);
            if (m <= ml && g.phi0 != 0.0) phase(tb, g.fft, N, m, true, PH[jj], PL[jj]);
        }
        const float osc = es ? osc1 : osc0;
#pragma unroll
        for (int jj = 0; jj < FWD_MJ; jj++) {
            const int m = et + jj * ent;
            if (m > ml) break;
            if (es < nb) {
                const int j = (m < N) ? m : m % N, jm = j ? N - j : 0;
                const cx a = buf[es * P + fft_pad(j)], b = cconjc(buf[es * P + fft_pad(jm)]);
                // 2 Xn = a + conj b, 2 Xs = (a - conj b) / i
                cx Xn = gadd(a, b);
                const cx d = gsub(a, b);
                cx Xs; Xs.hr = d.hi; Xs.lr = d.li; Xs.hi = -d.hr; Xs.li = -d.lr;
                if (g.phi0 != 0.0) { Xn = gmul(Xn, PH[jj], PL[jj]); Xs = gmul(Xs, PH[jj], PL[jj]); }
                const cx E = gadd(Xn, Xs), O = gsub(Xn, Xs);
                float2 e2, o2, el, ol;
                two_sum(E.hr, E.lr, e2.x, el.x); two_sum(E.hi, E.li, e2.y, el.y);
                two_sum(O.hr, O.lr, o2.x, ol.x); two_sum(O.hi, O.li, o2.y, ol.y);
                e2.x *= osc; e2.y *= osc; el.x *= osc; el.y *= osc;
                o2.x *= osc; o2.y *= osc; ol.x *= osc; ol.y *= osc;
                mx[jj][0] = fmaxf(mx[jj][0], fabsf(e2.x));
                mx[jj][1] = fmaxf(mx[jj][1], fabsf(e2.y));
                mx[jj][2] = fmaxf(mx[jj][2], fabsf(o2.x));
                mx[jj][3] = fmaxf(mx[jj][3], fabsf(o2.y));
                // T keeps hi and lo: (Re hi, Re lo, Im hi, Im lo) per complex column
                float4* t0 = reinterpret_cast<float4*>(T + ((long long)m * 2 + 0) * qstride + (long long)p * ncol + mc0 * 2);
                float4* t1 = reinterpret_cast<float4*>(T + ((long long)m * 2 + 1) * qstride + (long long)p * ncol + mc0 * 2);
                t0[es] = make_float4(e2.x, el.x, e2.y, el.y);
                t1[es] = make_float4(o2.x, ol.x, o2.y, ol.y);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int jj = 0; jj < FWD_MJ; jj++) {
        const int m = et + jj * ent;
        if (m > mmax || es >= nb) break;
        const long long col = (long long)(mc0 + es) * 2;
        unsigned int* c0 = colmax + ((long long)m * 2 + 0) * ncol + col;
        unsigned int* c1 = colmax + ((long long)m * 2 + 1) * ncol + col;
        if (mx[jj][0] > 0.0f) atomicMax(c0, __float_as_uint(mx[jj][0]));
        if (mx[jj][1] > 0.0f) atomicMax(c0 + 1, __float_as_uint(mx[jj][1]));
        if (mx[jj][2] > 0.0f) atomicMax(c1, __float_as_uint(mx[jj][2]));
        if (mx[jj][3] > 0.0f) atomicMax(c1 + 1, __float_as_uint(mx[jj][3]));
    }
}

// ---------------------------------------------------------------------------
// backward: G[m][q][p][c] (FP32) -> maps. Every m is folded onto bin m mod N
// with weight w_0 = 1, w_{m>0} = 2 and phase e^{+i m phi0}; the real ring is
// the IDFT of the Hermitian part. One launch per FFT size class; grid.x = pair
// of map columns, grid.y = block of BWD_PB ring pairs of the class.
// ---------------------------------------------------------------------------
constexpr int BWD_PB = 8;

template <int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
k_fftc_backward(const float* __restrict__ G, double* __restrict__ map, const int* __restrict__ cls, int ncls,
                const PairGeom* __restrict__ pairs, const FftLen* __restrict__ ffts, FftTabsF tb, long long ctw,
                long long ctwp, int ntwp,
                int M, int R_, int mmax, long long npix, long long ncol, int nmc, int mpc,
                const int* __restrict__ mlim)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx* buf = reinterpret_cast<cx*>(smem_raw);
    const int P = fft_pad_len(M);
    float4* twp_s = reinterpret_cast<float4*>(smem_raw + (size_t)mpc * P * sizeof(cx));
    float4* tw = twp_s + max(ntwp, 0);
    const float4* twp = (ntwp >= 0) ? twp_s : tb.twp + ctwp;
    if (ntwp > 0) stage_pass_twiddles(twp_s, ntwp, ctwp, tb);   // (published by the __syncthreads before the FFT)
    if (M % 3 == 0) stage_twiddles(tw, M, ctw, tb);
    __shared__ unsigned red[4];                    // per ring pair: largest |component| of each sequence
    if (threadIdx.x < 4) red[threadIdx.x] = 0u;
    __syncthreads();
    const int mc0 = blockIdx.x * mpc;
    const int nb = min(mpc, nmc - mc0);
    const long long qstride = (long long)R_ * ncol;
    const int iend = min(ncls, (int)(blockIdx.y + 1) * BWD_PB);
    for (int ip = blockIdx.y * BWD_PB; ip < iend; ip++) {
        const int p = cls[ip];
        const PairGeom g = pairs[p];
        const FftLen f = ffts[g.fft];
        const int N = g.n;
        const float* g0 = G + (long long)p * ncol + mc0 * 2;
        // the orders this ring pair takes part in (the contraction skips the
        // others: their lambda is negligible on this ring)
        const int ml = mlim ? min(mmax, mlim[p]) : mmax;
        // E and O of the two columns at order m (16-byte loads when aligned)
        auto load_eo = [&](int m, float4& E4, float4& O4) {
            const float* e = g0 + (long long)m * 2 * qstride;
            if (nb == 2 && (ncol & 3) == 0) {          // 16-byte aligned: ncol a multiple of 4
                E4 = *reinterpret_cast<const float4*>(e);
                O4 = *reinterpret_cast<const float4*>(e + qstride);
            } else if (nb == 2) {
                const float2 a0 = *reinterpret_cast<const float2*>(e), a1 = *reinterpret_cast<const float2*>(e + 2);
                const float2 b0 = *reinterpret_cast<const float2*>(e + qstride);
                const float2 b1 = *reinterpret_cast<const float2*>(e + qstride + 2);
                E4 = make_float4(a0.x, a0.y, a1.x, a1.y);
                O4 = make_float4(b0.x, b0.y, b1.x, b1.y);
            } else {
                const float2 E2 = *reinterpret_cast<const float2*>(e), O2 = *reinterpret_cast<const float2*>(e + qstride);
                E4 = make_float4(E2.x, E2.y, 0.0f, 0.0f);
                O4 = make_float4(O2.x, O2.y, 0.0f, 0.0f);
            }
        };
        // column s's north / south terms of order m: w_m (E +- O) e^{+i m phi0}
        auto term = [&](int m, const float4& E4, const float4& O4, float2 ph, float2 pl, int s, cx& tn, cx& ts) {
            const float er = s ? E4.z : E4.x, ei = s ? E4.w : E4.y;
            const float orr = s ? O4.z : O4.x, oi = s ? O4.w : O4.y;
            two_sum(er, orr, tn.hr, tn.lr); two_sum(ei, oi, tn.hi, tn.li);
            two_sum(er, -orr, ts.hr, ts.lr); two_sum(ei, -oi, ts.hi, ts.li);
            const float w = m ? 2.0f : 1.0f;
            tn = cscale(tn, w); ts = cscale(ts, w);
            if (g.phi0 != 0.0) { tn = cmulc(tn, ph, pl); ts = cmulc(ts, ph, pl); }
        };
        // bins j and N - j of both columns into the transform buffer. With
        // hn = B(j) + conj(B(N - j)) and hs likewise (twice the Hermitian parts
        // of the two rings), bin j takes conj(hn + i hs) and bin N - j, whose
        // Hermitian parts are the conjugates, hn - i hs (conjugated input: the
        // forward transform gives the inverse; the 1/2 goes to the output scale)
        unsigned m0 = 0, m1 = 0;
        auto emit = [&](int j, const cx (&Bn)[2][2], const cx (&Bs)[2][2]) {
            const int jm = j ? N - j : 0;
#pragma unroll
            for (int s = 0; s < 2; s++) {
                if (s >= nb) break;
                const cx hn = caddc(Bn[0][s], cconjc(Bn[1][s]));
                const cx hs = cmul_pi(caddc(Bs[0][s], cconjc(Bs[1][s])));
                const cx z = cconjc(caddc(hn, hs));
                buf[s * P + fft_pad(placec(f, j))] = z;
                unsigned v = absbits(z);
                if (jm != j) {
                    const cx z1 = csubc(hn, hs);
                    buf[s * P + fft_pad(placec(f, jm))] = z1;
                    v = max(v, absbits(z1));
                }
                if (s) m1 = max(m1, v); else m0 = max(m0, v);
            }
        };
        if (N > mmax) {
            // every bin receives at most one order (m = j or m = N - j): the
            // loads of BWD_JB bins per thread are all in flight before any is used
            constexpr int BWD_JB = 2;
            for (int j0 = threadIdx.x; j0 <= N / 2; j0 += BWD_JB * NT) {
                float4 E[BWD_JB][2], O[BWD_JB][2];
                float2 PH[BWD_JB][2], PL[BWD_JB][2];
#pragma unroll
                for (int u = 0; u < BWD_JB; u++) {
                    const int j = j0 + u * NT;
#pragma unroll
                    for (int t = 0; t < 2; t++) {
                        const int m = t ? (j ? N - j : 0) : j;
                        E[u][t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f); O[u][t] = E[u][t];
                        PH[u][t] = make_float2(1.0f, 0.0f); PL[u][t] = make_float2(0.0f, 0.0f);
                        if (j <= N / 2 && m <= ml) {
                            load_eo(m, E[u][t], O[u][t]);
                            if (g.phi0 != 0.0) phase(tb, g.fft, N, m, false, PH[u][t], PL[u][t]);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < BWD_JB; u++) {
                    const int j = j0 + u * NT;
                    if (j > N / 2) break;
                    cx Bn[2][2], Bs[2][2];                 // [bin j / N - j][column]
#pragma unroll
                    for (int t = 0; t < 2; t++) {
                        const int m = t ? (j ? N - j : 0) : j;
#pragma unroll
                        for (int s = 0; s < 2; s++) {
                            Bn[t][s] = czero(); Bs[t][s] = czero();
                            if (m <= ml) term(m, E[u][t], O[u][t], PH[u][t], PL[u][t], s, Bn[t][s], Bs[t][s]);
                        }
                    }
                    emit(j, Bn, Bs);
                }
            }
        } else {
            for (int j = threadIdx.x; j <= N / 2; j += NT) {
                const int jj[2] = {j, (j ? N - j : 0)};
                cx Bn[2][2], Bs[2][2];                     // [bin j / N - j][column]
#pragma unroll
                for (int t = 0; t < 2; t++) {
                    cx sn[2] = {czero(), czero()}, ss[2] = {czero(), czero()};
                    for (int m = jj[t]; m <= ml; m += N) {
                        float4 E4, O4;
                        load_eo(m, E4, O4);
                        float2 ph = make_float2(1.0f, 0.0f), pl = make_float2(0.0f, 0.0f);
                        if (g.phi0 != 0.0) phase(tb, g.fft, N, m, false, ph, pl);
#pragma unroll
                        for (int s = 0; s < 2; s++) {
                            cx tn, ts;
                            term(m, E4, O4, ph, pl, s, tn, ts);
                            sn[s] = caddc(sn[s], tn);
                            ss[s] = caddc(ss[s], ts);
                        }
                    }
                    Bn[t][0] = sn[0]; Bn[t][1] = sn[1]; Bs[t][0] = ss[0]; Bs[t][1] = ss[1];
                }
                emit(j, Bn, Bs);
            }
        }
        red_max2(red, m0, m1);
        __syncthreads();
        const int2 kq = dftc_forward(buf, nb, f, tw, twp, tb, red, 22);
        const float osc0 = pow2f(kq.x - 1), osc1 = pow2f(kq.y - 1);
        if (threadIdx.x < 4) red[threadIdx.x] = 0u;    // (read by every thread before the syncs above)
        for (int e = threadIdx.x; e < nb * N; e += blockDim.x) {
            const int s = (e >= N) ? 1 : 0, n = e - s * N;     // nb <= 2 sequences
            const cx z = buf[s * P + fft_pad(n)];      // conj of the inverse transform, times 2^-K
            const float osc = s ? osc1 : osc0;
            double* mp = map + (long long)(mc0 + s) * npix;
            mp[g.start_n + n] = tc::f32_to_f64(z.hr * osc) + tc::f32_to_f64(z.lr * osc);
            if (g.start_s >= 0) mp[g.start_s + n] = -(tc::f32_to_f64(z.hi * osc) + tc::f32_to_f64(z.li * osc));
        }
        __syncthreads();                               // buf is rewritten by the next ring pair
    }
}

static FftTabsF tabs(const sht_plan* p)
{
    FftTabsF t;
    t.twp = p->c.twp;
    t.twh = p->c.tws_h; t.twl = p->c.tws_l;
    t.chh = p->t.chirp_f; t.chl = p->c.chirp_l;
    t.bhh = p->c.bhs_h; t.bhl = p->c.bhs_l;
    t.phh = p->c.phase_h; t.phl = p->c.phase_l;
    t.phoff = p->c.phase_off;
    return t;
}

// Launch configuration of a size class: two map columns per CTA while their
// unpadded buffers fit in 128 KB; the per-pass twiddles staged in shared
// memory when everything fits in 227 KB (else read from global memory); the
// size-M twiddles for sizes 3^b 2^a; 512 threads where one CTA fills an
// SM's shared memory (16 warps per SM).
struct ClassCfg {
    int nt, mpc;
    size_t sm;
    bool twp_smem;
};
static ClassCfg class_cfg(const FftClass& c, int mmax, bool fwd)
{
    ClassCfg k;
    const int M = c.m;
    k.mpc = (2 * (size_t)M * sizeof(cx) <= (128u << 10)) ? 2 : 1;
    size_t sm = (size_t)k.mpc * fft_pad_len(M) * sizeof(cx) + ((M % 3 == 0) ? (size_t)(M / 2) * sizeof(float4) : 0);
    // (the backward kernels read the per-pass twiddles from global memory:
    // their G and phase loads keep more of the L1 that way; so do the forward
    // ones for tables above 40 KB, M >= 4096; measured)
    k.twp_smem = fwd && (size_t)c.twp_n * sizeof(float4) <= (40u << 10) &&
                 sm + (size_t)c.twp_n * sizeof(float4) <= (227u << 10);
    if (k.twp_smem) sm += (size_t)c.twp_n * sizeof(float4);
    k.sm = sm;
    k.nt = (M >= 4096 || mmax >= 1024 || sm > (113u << 10)) ? 512 : 256;
    return k;
}

static cudaError_t set_smem(const void* fn, const sht_plan* p, bool fwd)
{
    size_t mx = 0;
    for (const FftClass& c : p->h_fcls) mx = std::max(mx, class_cfg(c, p->mmax, fwd).sm);
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
}

// The size classes of a transform run beside one another: each class goes,
// in decreasing order of work (ring pairs x M log M), to whichever of the
// caller's stream and the plan's helper streams has the least work queued so
// far; the helpers are forked from and joined back into the caller's stream
// with events, so the call is ordered on `st` as a whole (and can be
// captured into a CUDA graph). The classes write disjoint ring pairs (the
// forward ones' column maxima with atomicMax).
struct ClassOrder {
    int n = 0;
    std::vector<int> idx;
    std::vector<int> stream;   // 0: the caller's stream, 1 + i: helper i
};
static ClassOrder class_order(const sht_plan* p)
{
    ClassOrder o;
    const int nc = (int)p->h_fcls.size();
    std::vector<std::pair<double, int>> w;
    for (int i = 0; i < nc; i++) {
        const FftClass& c = p->h_fcls[i];
        w.push_back({(double)c.cnt * c.m * std::log2((double)std::max(c.m, 2)), i});
    }
    std::sort(w.begin(), w.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
        return x.first > y.first;
    });
    const bool aux = p->fft_fork != nullptr && p->fft_aux[sht_plan::FFT_AUX - 1] != nullptr;
    double load[1 + sht_plan::FFT_AUX] = {0.0};
    for (auto& kv : w) {
        int s = 0;
        if (aux)
            for (int j = 1; j <= sht_plan::FFT_AUX; j++) if (load[j] < load[s]) s = j;
        load[s] += kv.first;
        o.idx.push_back(kv.second);
        o.stream.push_back(s);
        o.n++;
    }
    return o;
}
static cudaError_t fork_aux(const sht_plan* p, const ClassOrder& o, cudaStream_t st)
{
    bool any = false;
    for (int i = 0; i < o.n; i++) any = any || o.stream[i] > 0;
    if (!any) return cudaSuccess;
    cudaError_t e = cudaEventRecord(p->fft_fork, st);
    for (int j = 0; j < sht_plan::FFT_AUX && e == cudaSuccess; j++) e = cudaStreamWaitEvent(p->fft_aux[j], p->fft_fork, 0);
    return e;
}
static cudaError_t join_aux(const sht_plan* p, const ClassOrder& o, cudaStream_t st)
{
    bool any = false;
    for (int i = 0; i < o.n; i++) any = any || o.stream[i] > 0;
    if (!any) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < sht_plan::FFT_AUX && e == cudaSuccess; j++) {
        e = cudaEventRecord(p->fft_join[j], p->fft_aux[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->fft_join[j], 0);
    }
    return e;
}

cudaError_t launch_fft_forward_split(const sht_plan* p, const double* map, float2* T,
                                     unsigned int* colmax, int nmaps, cudaStream_t st)
{
    // the bulk L2 prefetches of the map rows want 16-byte aligned rows of a
    // multiple of 16 bytes: an aligned map, even row starts, even N
    int pf = ((uintptr_t)map & 15) == 0;
    for (const PairGeom& g : p->h_pairs)
        if ((g.start_n & 1) || (g.start_s >= 0 && (g.start_s & 1)) || (g.n & 1)) pf = 0;
    cudaError_t e = set_smem((const void*)k_fftc_forward<256>, p, true);
    if (e == cudaSuccess) e = set_smem((const void*)k_fftc_forward<512>, p, true);
    if (e != cudaSuccess) return e;
    const long long nc = ncols(p, nmaps);
    const int nmc = nmaps * p->ncomp;
    e = cudaMemsetAsync(colmax, 0, (size_t)(p->mmax + 1) * 2 * nc * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(p->fft_mu);
    const ClassOrder o = class_order(p);
    prof_start("k_fftc_forward", st);
    if ((e = fork_aux(p, o, st)) != cudaSuccess) return e;
    for (int i = 0; i < o.n; i++) {
        const FftClass& c = p->h_fcls[o.idx[i]];
        cudaStream_t ss = o.stream[i] ? p->fft_aux[o.stream[i] - 1] : st;
        const ClassCfg k = class_cfg(c, p->mmax, true);
        const int ntwp = k.twp_smem ? c.twp_n : -1;  // < 0: per-pass twiddles from global memory
        dim3 grid((nmc + k.mpc - 1) / k.mpc, (c.cnt + FWD_PB - 1) / FWD_PB);
        if (k.nt == 512)
            k_fftc_forward<512><<<grid, k.nt, k.sm, ss>>>(map, T, colmax, p->c.cls_pairs + c.off, c.cnt, p->t.pairs,
                                                          p->c.fft_s, tabs(p), c.tw, c.twp, ntwp, c.m, p->R, p->mmax,
                                                          p->npix, nc, nmc, k.mpc, pf, p->s.mlim);
        else
            k_fftc_forward<256><<<grid, k.nt, k.sm, ss>>>(map, T, colmax, p->c.cls_pairs + c.off, c.cnt, p->t.pairs,
                                                          p->c.fft_s, tabs(p), c.tw, c.twp, ntwp, c.m, p->R, p->mmax,
                                                          p->npix, nc, nmc, k.mpc, pf, p->s.mlim);
        count_launch();
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = join_aux(p, o, st);
    prof_stop(st);
    return e;
}

cudaError_t launch_fft_backward_f32(const sht_plan* p, const float* G, double* map, int nmaps, cudaStream_t st)
{
    cudaError_t e = set_smem((const void*)k_fftc_backward<256>, p, false);
    if (e == cudaSuccess) e = set_smem((const void*)k_fftc_backward<512>, p, false);
    if (e != cudaSuccess) return e;
    const int nmc = nmaps * p->ncomp;
    std::lock_guard<std::mutex> lk(p->fft_mu);
    const ClassOrder o = class_order(p);
    prof_start("k_fftc_backward", st);
    if ((e = fork_aux(p, o, st)) != cudaSuccess) return e;
    for (int i = 0; i < o.n; i++) {
        const FftClass& c = p->h_fcls[o.idx[i]];
        cudaStream_t ss = o.stream[i] ? p->fft_aux[o.stream[i] - 1] : st;
        const ClassCfg k = class_cfg(c, p->mmax, false);
        const int ntwp = k.twp_smem ? c.twp_n : -1;  // < 0: per-pass twiddles from global memory
        dim3 grid((nmc + k.mpc - 1) / k.mpc, (c.cnt + BWD_PB - 1) / BWD_PB);
        if (k.nt == 512)
            k_fftc_backward<512><<<grid, k.nt, k.sm, ss>>>(G, map, p->c.cls_pairs + c.off, c.cnt, p->t.pairs, p->c.fft_s,
                                                           tabs(p), c.tw, c.twp, ntwp, c.m, p->R, p->mmax, p->npix,
                                                           ncols(p, nmaps), nmc, k.mpc, p->s.mlim);
        else
            k_fftc_backward<256><<<grid, k.nt, k.sm, ss>>>(G, map, p->c.cls_pairs + c.off, c.cnt, p->t.pairs, p->c.fft_s,
                                                           tabs(p), c.tw, c.twp, ntwp, c.m, p->R, p->mmax, p->npix,
                                                           ncols(p, nmaps), nmc, k.mpc, p->s.mlim);
        count_launch();
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = join_aux(p, o, st);
    prof_stop(st);
    return e;
}

}  // namespace sht
