// fft_split.cu -- ring FFTs of the split-precision form in compensated FP32.
//
// A plain FP32 radix-2 FFT of 2048 points has an RMS error of ~1.3e-7 of the
// signal RMS (5.96e-7 worst over 4e5 outputs), too close to the 1e-6 bar of
// the split form, and FP64 arithmetic runs at ~1/64 of FP32 on this GPU. So
// every complex value is carried as an unevaluated sum hi + lo of two FP32
// numbers: butterfly additions are error-free (TwoSum, their rounding error
// goes to lo), products use FMA and a hi/lo twiddle, and lo is propagated in
// plain FP32. This halves the FFT error (6e-8 RMS) for ~4x the FP32 work.
// Phases e^{+-i pi m / N} come from a hi/lo table per ring length.
//
// Structure (Sec. 2.1 eq:mm; Appendix A.1 for m -> bin m mod N) is that of
// fft.cu: one complex FFT of x_north + i x_south per ring pair, radix-2 in
// shared memory for power-of-two N, Bluestein otherwise.
#include "common.cuh"
#include "tc.cuh"

namespace sht {

struct cx { float hr, hi, lr, li; };     // (hr + lr) + i (hi + li)

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// x * w with w = wh + wl (hi/lo twiddle); the products of the hi parts are
// error-free (FMA residuals) and their sum a TwoSum, so only the lo terms round
__device__ __forceinline__ cx cmulc(const cx& x, float2 wh, float2 wl)
{
    cx t;
    float s, e;
    {
        const float p1 = __fmul_rn(x.hr, wh.x), p2 = __fmul_rn(x.hi, wh.y);
        const float e1 = fmaf(x.hr, wh.x, -p1), e2 = fmaf(x.hi, wh.y, -p2);
        two_sum(p1, -p2, s, e);
        t.hr = s;
        t.lr = (e + (e1 - e2)) + (x.lr * wh.x - x.li * wh.y) + (x.hr * wl.x - x.hi * wl.y);
    }
    {
        const float p1 = __fmul_rn(x.hr, wh.y), p2 = __fmul_rn(x.hi, wh.x);
        const float e1 = fmaf(x.hr, wh.y, -p1), e2 = fmaf(x.hi, wh.x, -p2);
        two_sum(p1, p2, s, e);
        t.hi = s;
        t.li = (e + (e1 + e2)) + (x.lr * wh.y + x.li * wh.x) + (x.hr * wl.y + x.hi * wl.x);
    }
    return t;
}
__device__ __forceinline__ cx caddc(const cx& a, const cx& b)
{
    cx s; float e;
    two_sum(a.hr, b.hr, s.hr, e); s.lr = a.lr + b.lr + e;
    two_sum(a.hi, b.hi, s.hi, e); s.li = a.li + b.li + e;
    return s;
}
__device__ __forceinline__ cx csubc(const cx& a, const cx& b)
{
    cx s; float e;
    two_sum(a.hr, -b.hr, s.hr, e); s.lr = a.lr - b.lr + e;
    two_sum(a.hi, -b.hi, s.hi, e); s.li = a.li - b.li + e;
    return s;
}
__device__ __forceinline__ cx cscale(cx a, float s) { a.hr *= s; a.hi *= s; a.lr *= s; a.li *= s; return a; }
__device__ __forceinline__ cx cconjc(cx a) { a.hi = -a.hi; a.li = -a.li; return a; }
__device__ __forceinline__ cx czero() { cx z; z.hr = z.hi = z.lr = z.li = 0.0f; return z; }
__device__ __forceinline__ float cre(const cx& a) { return a.hr + a.lr; }
__device__ __forceinline__ float cim(const cx& a) { return a.hi + a.li; }

__device__ __forceinline__ int brev_c(int i, int logm) { return (int)(__brev((unsigned)i) >> (32 - logm)); }

__device__ __forceinline__ void twid(const float2* twh, const float2* twl, int k, bool inv, float2& wh, float2& wl)
{
    wh = twh[k]; wl = twl[k];
    if (inv) { wh.y = -wh.y; wl.y = -wl.y; }
}

__device__ void fftc_dif(cx* buf, int M, int fftmax, const float2* twh, const float2* twl, bool inv)
{
    for (int h = M >> 1; h >= 1; h >>= 1) {
        int step = fftmax / (2 * h);
        for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
            int k = b & (h - 1);
            int i0 = ((b - k) << 1) + k, i1 = i0 + h;
            float2 wh, wl;
            twid(twh, twl, k * step, inv, wh, wl);
            cx a = buf[i0], c = buf[i1];
            buf[i0] = caddc(a, c);
            buf[i1] = cmulc(csubc(a, c), wh, wl);
        }
        __syncthreads();
    }
}

__device__ void fftc_dit(cx* buf, int M, int fftmax, const float2* twh, const float2* twl, bool inv)
{
    for (int h = 1; h < M; h <<= 1) {
        int step = fftmax / (2 * h);
        for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
            int k = b & (h - 1);
            int i0 = ((b - k) << 1) + k, i1 = i0 + h;
            float2 wh, wl;
            twid(twh, twl, k * step, inv, wh, wl);
            cx t = cmulc(buf[i1], wh, wl);
            cx a = buf[i0];
            buf[i0] = caddc(a, t);
            buf[i1] = csubc(a, t);
        }
        __syncthreads();
    }
}

struct FftTabsF {
    const float2 *twh, *twl;      // exp(-2 pi i t / fftmax), hi / lo
    const float2 *chh, *chl;      // Bluestein chirp, hi / lo
    const float2 *bhh, *bhl;      // Bluestein filter spectrum (bit-reversed), hi / lo
    const float2 *phh, *phl;      // exp(+i pi k / N), k < 2N, per ring length, hi / lo
    const long long* phoff;       // offset of each ring length's phase table
};

// forward DFT (Z_k = sum z_n e^{-2 pi i k n / N}) of data placed by placec()
__device__ void dftc_forward(cx* buf, const FftLen& f, int fftmax, const FftTabsF& t)
{
    int M = f.m;
    if (!f.bluestein) {
        fftc_dit(buf, M, fftmax, t.twh, t.twl, false);
        return;
    }
    fftc_dif(buf, M, fftmax, t.twh, t.twl, false);
    for (int i = threadIdx.x; i < M; i += blockDim.x) buf[i] = cmulc(buf[i], t.bhh[f.bhat + i], t.bhl[f.bhat + i]);
    __syncthreads();
    fftc_dit(buf, M, fftmax, t.twh, t.twl, true);
    const float inv = 1.0f / (float)M;
    for (int k = threadIdx.x; k < f.n; k += blockDim.x)
        buf[k] = cscale(cmulc(buf[k], t.chh[f.chirp + k], t.chl[f.chirp + k]), inv);
    __syncthreads();
}

__device__ __forceinline__ int placec(const FftLen& f, int n)
{
    return f.bluestein ? n : brev_c(n, 31 - __clz(f.m));
}

__device__ __forceinline__ cx chirp_in(const FftLen& f, const FftTabsF& t, cx z, int n)
{
    return f.bluestein ? cmulc(z, t.chh[f.chirp + n], t.chl[f.chirp + n]) : z;
}

// e^{sgn i pi k / N} for k = m mod 2N (hi/lo)
__device__ __forceinline__ void phase(const FftTabsF& t, int fidx, int N, int m, bool neg, float2& ph, float2& pl)
{
    long long o = t.phoff[fidx] + (m % (2 * N));
    ph = t.phh[o]; pl = t.phl[o];
    if (neg) { ph.y = -ph.y; pl.y = -pl.y; }
}

// ---------------------------------------------------------------------------
// forward: maps -> T[m][q][p][c] (FP32 hi/lo pairs) and the
// per (m, slot, column) maxima used for the tensor-core column quanta.
// grid.x = block of FWD_PB ring pairs, grid.y = map * ncomp + comp
// ---------------------------------------------------------------------------
constexpr int FWD_PB = 64;
constexpr int FWD_MJ = 8;

__global__ void __launch_bounds__(256)
k_fftc_forward(const double* __restrict__ map, float2* __restrict__ T, unsigned int* __restrict__ colmax,
               const PairGeom* __restrict__ pairs, const FftLen* __restrict__ ffts, FftTabsF tb,
               int fftmax, int R_, int mmax, long long npix, long long ncol)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx* buf = reinterpret_cast<cx*>(smem_raw);
    const int mc = blockIdx.y;
    const long long col = (long long)mc * 2;
    const long long qstride = (long long)R_ * ncol;
    float mx[FWD_MJ][4];
#pragma unroll
    for (int j = 0; j < FWD_MJ; j++) mx[j][0] = mx[j][1] = mx[j][2] = mx[j][3] = 0.0f;
    const int pend = min(R_, (blockIdx.x + 1) * FWD_PB);
    for (int p = blockIdx.x * FWD_PB; p < pend; p++) {
        const PairGeom g = pairs[p];
        const FftLen f = ffts[g.fft];
        const int N = g.n;
        const double* xn = map + (long long)mc * npix + g.start_n;
        const double* xs = g.start_s >= 0 ? map + (long long)mc * npix + g.start_s : nullptr;
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
            cx z = czero();
            tc::f64_split_scaled(xn[n], 0, z.hr, z.lr);
            if (xs) tc::f64_split_scaled(xs[n], 0, z.hi, z.li);
            buf[placec(f, n)] = chirp_in(f, tb, z, n);
        }
        if (f.bluestein)
            for (int i = f.n + threadIdx.x; i < f.m; i += blockDim.x) buf[i] = czero();
        __syncthreads();
        dftc_forward(buf, f, fftmax, tb);
#pragma unroll
        for (int jj = 0; jj < FWD_MJ; jj++) {
            const int m = threadIdx.x + jj * 256;
            if (m > mmax) break;
            const int j = m % N, jm = (N - j) % N;
            const cx a = buf[j], b = cconjc(buf[jm]);
            // Xn = (a + conj b)/2, Xs = (a - conj b)/(2i)
            cx Xn = cscale(caddc(a, b), 0.5f);
            cx d = cscale(csubc(a, b), 0.5f);
            cx Xs; Xs.hr = d.hi; Xs.lr = d.li; Xs.hi = -d.hr; Xs.li = -d.lr;
            if (g.phi0 != 0.0) {
                float2 ph, pl;
                phase(tb, g.fft, N, m, true, ph, pl);
                Xn = cmulc(Xn, ph, pl);
                Xs = cmulc(Xs, ph, pl);
            }
            const cx E = caddc(Xn, Xs), O = csubc(Xn, Xs);
            float2 e2, o2, el, ol;
            two_sum(E.hr, E.lr, e2.x, el.x); two_sum(E.hi, E.li, e2.y, el.y);
            two_sum(O.hr, O.lr, o2.x, ol.x); two_sum(O.hi, O.li, o2.y, ol.y);
            // T keeps hi and lo: (Re hi, Re lo, Im hi, Im lo) per complex column
            float2* t0 = T + ((long long)m * 2 + 0) * qstride + (long long)p * ncol + col;
            *reinterpret_cast<float4*>(t0) = make_float4(e2.x, el.x, e2.y, el.y);
            *reinterpret_cast<float4*>(t0 + qstride) = make_float4(o2.x, ol.x, o2.y, ol.y);
            mx[jj][0] = fmaxf(mx[jj][0], fabsf(e2.x));
            mx[jj][1] = fmaxf(mx[jj][1], fabsf(e2.y));
            mx[jj][2] = fmaxf(mx[jj][2], fabsf(o2.x));
            mx[jj][3] = fmaxf(mx[jj][3], fabsf(o2.y));
        }
        __syncthreads();
    }
#pragma unroll
    for (int jj = 0; jj < FWD_MJ; jj++) {
        const int m = threadIdx.x + jj * 256;
        if (m > mmax) break;
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
// the IDFT of the Hermitian part. grid.x = ring pair, grid.y = map * ncomp + comp.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_fftc_backward(const float* __restrict__ G, double* __restrict__ map, const PairGeom* __restrict__ pairs,
                const FftLen* __restrict__ ffts, FftTabsF tb, int fftmax, int R_, int mmax, long long npix,
                long long ncol)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx* buf = reinterpret_cast<cx*>(smem_raw);
    const int p = blockIdx.x;
    const int mc = blockIdx.y;
    const PairGeom g = pairs[p];
    const FftLen f = ffts[g.fft];
    const int N = g.n;
    const long long col = (long long)mc * 2;
    const long long qstride = (long long)R_ * ncol;
    const float* g0 = G + (long long)p * ncol + col;
    for (int j = threadIdx.x; j <= N / 2; j += blockDim.x) {
        int jj[2] = {j, (N - j) % N};
        cx Bn[2], Bs[2];
        for (int t = 0; t < 2; t++) {
            cx sn = czero(), ss = czero();
            for (int m = jj[t]; m <= mmax; m += N) {
                const float* e = g0 + (long long)m * 2 * qstride;
                const float2 E = *reinterpret_cast<const float2*>(e);
                const float2 O = *reinterpret_cast<const float2*>(e + qstride);
                const float w = m ? 2.0f : 1.0f;
                cx tn, ts;
                two_sum(E.x, O.x, tn.hr, tn.lr); two_sum(E.y, O.y, tn.hi, tn.li);
                two_sum(E.x, -O.x, ts.hr, ts.lr); two_sum(E.y, -O.y, ts.hi, ts.li);
                tn = cscale(tn, w); ts = cscale(ts, w);
                if (g.phi0 != 0.0) {
                    float2 ph, pl;
                    phase(tb, g.fft, N, m, false, ph, pl);
                    tn = cmulc(tn, ph, pl);
                    ts = cmulc(ts, ph, pl);
                }
                sn = caddc(sn, tn);
                ss = caddc(ss, ts);
            }
            Bn[t] = sn; Bs[t] = ss;
        }
        for (int t = 0; t < 2; t++) {
            int jt = jj[t];
            if (t == 1 && jt == jj[0]) break;
            // H(j) = (B(j) + conj(B(N-j))) / 2 ; z = Hn + i Hs ; store conj(z)
            cx hn = cscale(caddc(Bn[t], cconjc(Bn[1 - t])), 0.5f);
            cx hs = cscale(caddc(Bs[t], cconjc(Bs[1 - t])), 0.5f);
            cx ihs; ihs.hr = -hs.hi; ihs.lr = -hs.li; ihs.hi = hs.hr; ihs.li = hs.lr;
            cx z = cconjc(caddc(hn, ihs));
            buf[placec(f, jt)] = chirp_in(f, tb, z, jt);
        }
    }
    if (f.bluestein)
        for (int i = f.n + threadIdx.x; i < f.m; i += blockDim.x) buf[i] = czero();
    __syncthreads();
    dftc_forward(buf, f, fftmax, tb);
    double* xn = map + (long long)mc * npix + g.start_n;
    double* xs = g.start_s >= 0 ? map + (long long)mc * npix + g.start_s : nullptr;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const cx z = buf[n];                 // conj of the inverse transform
        xn[n] = tc::f32_to_f64(cre(z));
        if (xs) xs[n] = -tc::f32_to_f64(cim(z));
    }
}

static FftTabsF tabs(const sht_plan* p)
{
    FftTabsF t;
    t.twh = p->t.twiddle_f; t.twl = p->c.twiddle_l;
    t.chh = p->t.chirp_f; t.chl = p->c.chirp_l;
    t.bhh = p->t.bhat_f; t.bhl = p->c.bhat_l;
    t.phh = p->c.phase_h; t.phl = p->c.phase_l;
    t.phoff = p->c.phase_off;
    return t;
}

cudaError_t launch_fft_forward_split(const sht_plan* p, const double* map, float2* T,
                                     unsigned int* colmax, int nmaps, cudaStream_t st)
{
    size_t sm = (size_t)p->fft_max * sizeof(cx);
    cudaError_t e = cudaFuncSetAttribute(k_fftc_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    long long nc = ncols(p, nmaps);
    e = cudaMemsetAsync(colmax, 0, (size_t)(p->mmax + 1) * 2 * nc * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    dim3 grid((p->R + FWD_PB - 1) / FWD_PB, nmaps * p->ncomp);
    prof_start("k_fftc_forward", st);
    k_fftc_forward<<<grid, 256, sm, st>>>(map, T, colmax, p->t.pairs, p->t.fft, tabs(p), p->fft_max, p->R,
                                          p->mmax, p->npix, nc);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fft_backward_f32(const sht_plan* p, const float* G, double* map, int nmaps, cudaStream_t st)
{
    size_t sm = (size_t)p->fft_max * sizeof(cx);
    cudaError_t e = cudaFuncSetAttribute(k_fftc_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid(p->R, nmaps * p->ncomp);
    prof_start("k_fftc_backward", st);
    k_fftc_backward<<<grid, 256, sm, st>>>(G, map, p->t.pairs, p->t.fft, tabs(p), p->fft_max, p->R, p->mmax,
                                           p->npix, ncols(p, nmaps));
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

}  // namespace sht
