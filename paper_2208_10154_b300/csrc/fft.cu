// fft.cu -- batched ring FFTs and the FFT mapping (Sec. 2.1 eq:mm, Algorithm 1
// "Batch FFT" and "remap F to T_m"; Appendix A.1 for the alias of m onto the
// FFT circle of a ring of N pixels).
//
// One CTA transforms one ring pair of one (map, component): the north ring
// and its mirror share N and phi0, so z = x_north + i x_south is transformed
// with a single complex FFT of length N and the two real spectra are split
// afterwards. Power-of-two N uses an in-place radix-2 FFT in shared memory;
// any other N (the 4i-pixel cap rings) uses Bluestein's chirp-z algorithm on
// the next power of two >= 2N-1 with resident chirp tables.
#include <algorithm>

#include "common.cuh"

namespace sht {

template <typename R> struct CT;
template <> struct CT<double> { using C = double2; };
template <> struct CT<float> { using C = float2; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

// (cos, sin) of pi * num / den
template <typename R> __device__ __forceinline__ void sincospi_r(int num, int den, R* sn, R* cs);
template <> __device__ __forceinline__ void sincospi_r<double>(int num, int den, double* sn, double* cs)
{
    sincospi((double)num / (double)den, sn, cs);
}
template <> __device__ __forceinline__ void sincospi_r<float>(int num, int den, float* sn, float* cs)
{
    sincospif((float)num / (float)den, sn, cs);
}

__device__ __forceinline__ int brev(int i, int logm) { return (int)(__brev((unsigned)i) >> (32 - logm)); }

// Decimation in frequency: natural-order input -> bit-reversed output.
// tw[t] = exp(-2 pi i t / fftmax), t < fftmax/2. inv conjugates the twiddles.
template <typename C>
__device__ void fft_dif(C* buf, int M, int fftmax, const C* __restrict__ tw, bool inv)
{
    for (int h = M >> 1; h >= 1; h >>= 1) {
        int step = fftmax / (2 * h);
        for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
            int k = b & (h - 1);
            int i0 = ((b - k) << 1) + k, i1 = i0 + h;
            C a = buf[i0], c = buf[i1];
            C w = tw[k * step];
            if (inv) w.y = -w.y;
            buf[i0] = cadd(a, c);
            buf[i1] = cmul(csub(a, c), w);
        }
        __syncthreads();
    }
}

// Decimation in time: bit-reversed input -> natural-order output.
template <typename C>
__device__ void fft_dit(C* buf, int M, int fftmax, const C* __restrict__ tw, bool inv)
{
    for (int h = 1; h < M; h <<= 1) {
        int step = fftmax / (2 * h);
        for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
            int k = b & (h - 1);
            int i0 = ((b - k) << 1) + k, i1 = i0 + h;
            C w = tw[k * step];
            if (inv) w.y = -w.y;
            C t = cmul(buf[i1], w);
            C a = buf[i0];
            buf[i0] = cadd(a, t);
            buf[i1] = csub(a, t);
        }
        __syncthreads();
    }
}

// Forward DFT of length N (Z_k = sum_n z_n e^{-2 pi i k n / N}) of the data
// the caller placed with place_index(): power-of-two N at brev(n), otherwise
// (Bluestein) at n, pre-multiplied by the chirp. Leaves Z in natural order.
template <typename C>
__device__ void dft_forward(C* buf, const FftLen& f, int fftmax, const C* tw, const C* chirp,
                            const C* bhat)
{
    int M = f.m;
    if (!f.bluestein) {
        fft_dit(buf, M, fftmax, tw, false);
        return;
    }
    fft_dif(buf, M, fftmax, tw, false);
    for (int i = threadIdx.x; i < M; i += blockDim.x) buf[i] = cmul(buf[i], bhat[i]);  // bhat bit-reversed
    __syncthreads();
    fft_dit(buf, M, fftmax, tw, true);
    typedef decltype(buf[0].x) Rl;
    Rl inv = (Rl)1 / (Rl)M;
    for (int k = threadIdx.x; k < f.n; k += blockDim.x) {   // Z_k = w_k c_k / M
        C c = cmul(buf[k], chirp[k]);
        c.x *= inv; c.y *= inv;
        buf[k] = c;
    }
    __syncthreads();
}

__device__ __forceinline__ int place_index(const FftLen& f, int n)
{
    return f.bluestein ? n : brev(n, 31 - __clz(f.m));
}

template <typename C>
__device__ __forceinline__ void zero_tail(C* buf, const FftLen& f)
{
    if (f.bluestein)
        for (int i = f.n + threadIdx.x; i < f.m; i += blockDim.x) { buf[i].x = 0; buf[i].y = 0; }
}

// ---------------------------------------------------------------------------
// map2alm side: maps -> T[m][q][p][c]
// grid.x = ring pair, grid.y = map * ncomp + comp
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
k_fft_forward(const double* __restrict__ map, R* __restrict__ T, const PairGeom* __restrict__ pairs,
              const FftLen* __restrict__ ffts, const typename CT<R>::C* __restrict__ tw,
              const typename CT<R>::C* __restrict__ chirp, const typename CT<R>::C* __restrict__ bhat,
              int fftmax, int R_, int mmax, long long npix, long long ncol)
{
    using C = typename CT<R>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int p = blockIdx.x;
    const int mc = blockIdx.y;                       // map * ncomp + comp
    const PairGeom g = pairs[p];
    const FftLen f = ffts[g.fft];
    const int N = g.n;
    const double* xn = map + (long long)mc * npix + g.start_n;
    const double* xs = g.start_s >= 0 ? map + (long long)mc * npix + g.start_s : nullptr;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        C z;
        z.x = (R)xn[n];
        z.y = xs ? (R)xs[n] : (R)0;
        if (f.bluestein) z = cmul(z, chirp[f.chirp + n]);
        buf[place_index(f, n)] = z;
    }
    zero_tail(buf, f);
    __syncthreads();
    dft_forward(buf, f, fftmax, tw, chirp + f.chirp, bhat + f.bhat);
    // split the two real spectra, apply the phase shift, write E / O
    const long long col = (long long)mc * 2;
    const long long qstride = (long long)R_ * ncol;
    for (int m = threadIdx.x; m <= mmax; m += blockDim.x) {
        int j = m % N;
        int jm = (N - j) % N;
        C a = buf[j], b = buf[jm];
        C Xn, Xs;
        Xn.x = (R)0.5 * (a.x + b.x); Xn.y = (R)0.5 * (a.y - b.y);
        Xs.x = (R)0.5 * (a.y + b.y); Xs.y = (R)0.5 * (b.x - a.x);
        if (g.phi0 != 0.0) {
            // e^{-i m phi0}, phi0 = pi / N: exact reduction of m mod 2N
            R sn, cs;
            sincospi_r<R>(-(m % (2 * N)), N, &sn, &cs);
            C ph; ph.x = cs; ph.y = sn;
            Xn = cmul(Xn, ph);
            Xs = cmul(Xs, ph);
        }
        C E = cadd(Xn, Xs), O = csub(Xn, Xs);
        R* t0 = T + ((long long)m * 2 + 0) * qstride + (long long)p * ncol + col;
        R* t1 = t0 + qstride;
        t0[0] = E.x; t0[1] = E.y;
        t1[0] = O.x; t1[1] = O.y;
    }
}

// ---------------------------------------------------------------------------
// alm2map side: G[m][q][p][c] -> maps
// north ring coefficient = G0 + G1, south = G0 - G1; bins fold every m with
// m = j mod N (the FFT circle of Appendix A.1) with weight w_0 = 1, w_{m>0} = 2
// and phase e^{+i m phi0}; the real ring is Re(IDFT) = IDFT of the Hermitian part.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
k_fft_backward(const R* __restrict__ G, double* __restrict__ map, const PairGeom* __restrict__ pairs,
               const FftLen* __restrict__ ffts, const typename CT<R>::C* __restrict__ tw,
               const typename CT<R>::C* __restrict__ chirp, const typename CT<R>::C* __restrict__ bhat,
               int fftmax, int R_, int mmax, long long npix, long long ncol)
{
    using C = typename CT<R>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int p = blockIdx.x;
    const int mc = blockIdx.y;
    const PairGeom g = pairs[p];
    const FftLen f = ffts[g.fft];
    const int N = g.n;
    const long long col = (long long)mc * 2;
    const long long qstride = (long long)R_ * ncol;
    const R* g0 = G + (long long)p * ncol + col;
    for (int j = threadIdx.x; j <= N / 2; j += blockDim.x) {
        int jj[2] = {j, (N - j) % N};
        C Bn[2], Bs[2];
        for (int t = 0; t < 2; t++) {
            C sn; sn.x = 0; sn.y = 0;
            C ss = sn;
            for (int m = jj[t]; m <= mmax; m += N) {
                const R* e = g0 + (long long)m * 2 * qstride;
                C E; E.x = e[0]; E.y = e[1];
                C O; O.x = e[qstride]; O.y = e[qstride + 1];
                C tn = cadd(E, O), ts = csub(E, O);
                R w = m ? (R)2 : (R)1;
                if (g.phi0 != 0.0) {
                    R sv, cv;
                    sincospi_r<R>(m % (2 * N), N, &sv, &cv);
                    C ph; ph.x = cv; ph.y = sv;
                    tn = cmul(tn, ph);
                    ts = cmul(ts, ph);
                }
                sn.x += w * tn.x; sn.y += w * tn.y;
                ss.x += w * ts.x; ss.y += w * ts.y;
            }
            Bn[t] = sn; Bs[t] = ss;
        }
        // Hermitian parts H(j) = (B(j) + conj(B(N-j))) / 2; spectrum z = Hn + i Hs;
        // IDFT(z) = conj(DFT(conj(z))): store conj(z) for the forward DFT.
        for (int t = 0; t < 2; t++) {
            int jt = jj[t];
            if (t == 1 && jt == jj[0]) break;
            C hn, hs;
            hn.x = (R)0.5 * (Bn[t].x + Bn[1 - t].x); hn.y = (R)0.5 * (Bn[t].y - Bn[1 - t].y);
            hs.x = (R)0.5 * (Bs[t].x + Bs[1 - t].x); hs.y = (R)0.5 * (Bs[t].y - Bs[1 - t].y);
            C z; z.x = hn.x - hs.y; z.y = hn.y + hs.x;
            z = cconj(z);
            if (f.bluestein) z = cmul(z, chirp[f.chirp + jt]);
            buf[place_index(f, jt)] = z;
        }
    }
    zero_tail(buf, f);
    __syncthreads();
    dft_forward(buf, f, fftmax, tw, chirp + f.chirp, bhat + f.bhat);
    double* xn = map + (long long)mc * npix + g.start_n;
    double* xs = g.start_s >= 0 ? map + (long long)mc * npix + g.start_s : nullptr;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        C z = buf[n];                 // conj of the inverse transform
        xn[n] = (double)z.x;
        if (xs) xs[n] = -(double)z.y;
    }
}

cudaError_t launch_fft_forward_f64(const sht_plan* p, const double* map, double* T, int nmaps,
                                   cudaStream_t st)
{
    size_t sm = (size_t)p->fft_max * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_fft_forward<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid(p->R, nmaps * p->ncomp);
    prof_start("k_fft_forward_f64", st);
    k_fft_forward<double><<<grid, 256, sm, st>>>(map, T, p->t.pairs, p->t.fft, p->t.twiddle, p->t.chirp,
                                                  p->t.bhat, p->fft_max, p->R, p->mmax, p->npix,
                                                  ncols(p, nmaps));
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fft_backward_f64(const sht_plan* p, const double* G, double* map, int nmaps,
                                    cudaStream_t st)
{
    size_t sm = (size_t)p->fft_max * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_fft_backward<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid(p->R, nmaps * p->ncomp);
    prof_start("k_fft_backward_f64", st);
    k_fft_backward<double><<<grid, 256, sm, st>>>(G, map, p->t.pairs, p->t.fft, p->t.twiddle, p->t.chirp,
                                                   p->t.bhat, p->fft_max, p->R, p->mmax, p->npix,
                                                   ncols(p, nmaps));
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fourier-domain residual of the iteration (Algorithm 2 restricted to the
// ring spectra): D = T - F(G), where F is what a backward FFT followed by a
// forward FFT does to the coefficients G[m][q][p][c] of a ring pair. Per ring
// of N pixels and phase offset phi0 (0 or pi/N), both steps fold m onto the
// FFT circle (Appendix A.1); with k0 = m div N, j = m mod N, j' = (N - j) mod N
// and sigma = -1 if phi0 != 0 else 1 (the phases e^{+-i m phi0} of two
// aliases differ by e^{i k N phi0} = sigma^k), for a ring's own coefficients
//     F(c)_m = (N / 2) sigma^{k0} [B(j) + sigma_j conj(B(j'))],
//     B(j) = sum_k sigma^k w_{j+kN} c_{j+kN}   (w_0 = 1, w_{m>0} = 2)
// with sigma_j = sigma for j > 0 and 1 for j = 0. For a pair of rings (north
// = E + O, south = E - O, the same N and phi0) it acts on the E and O slots
// separately with N in place of N / 2; the equator ring has no mirror (its
// forward FFT sees only the north ring), so there E' = O' = F(E + O).
// No trigonometry. One thread per complex column (coalesced over the
// columns); it walks the bin pairs (j, N - j), folding their aliases and
// writing D for every m on them. FP64, or for the split form FP32 G and
// double-float sums with FP32 hi/lo T and D. D may be G itself (FP64): each
// thread reads its G before it writes D on the same m.
// grid = (ring pair, column blocks of 128)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void df_add(float& hi, float& lo, float v)
{
    const float s = hi + v, bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}
__device__ __forceinline__ float2 df_norm(float hi, float lo)
{
    const float s = hi + lo;
    return make_float2(s, lo - (s - hi));
}

template <bool SPLIT>
__global__ void __launch_bounds__(128)
k_alias_residual(const void* __restrict__ Tv, const void* Gv, void* Dv, const PairGeom* __restrict__ pairs,
                 int R_, int mmax, long long ncol, int nmc, const int* __restrict__ mlim)
{
    const int p = blockIdx.x;
    const int mc = blockIdx.y * blockDim.x + threadIdx.x;
    if (mc >= nmc) return;
    const PairGeom g = pairs[p];
    const int N = g.n;
    const bool neg = g.phi0 != 0.0;               // sigma = -1
    const bool eq = g.start_s < 0;                // the equator ring: no mirror
    const long long qs = (long long)R_ * ncol;
    auto idx = [&](int m, int slot) -> long long {
        return ((long long)m * 2 + slot) * qs + (long long)p * ncol + (long long)mc * 2;
    };
    const int jmax = min(N / 2, mmax);
    if constexpr (SPLIT) {
        const float2* G = (const float2*)Gv;      // (re, im) of one complex column, FP32
        const float4* T = (const float4*)Tv;      // (re hi, re lo, im hi, im lo)
        float4* D = (float4*)Dv;
        // G holds the orders m <= ml of this ring pair (the split contraction
        // skips the others, whose lambda is negligible here)
        const int ml = mlim ? min(mmax, mlim[p]) : mmax;
        auto fold = [&](int j, int slot) -> float4 {
            float rh = 0.0f, rl = 0.0f, ih = 0.0f, il = 0.0f;
            bool odd = false;
            for (int m = j; m <= ml; m += N) {
                // w = w_m sigma^k: the products w G are exact in FP32
                const float w = (m ? 2.0f : 1.0f) * ((neg && odd) ? -1.0f : 1.0f);
                const float2 v = G[idx(m, slot) >> 1];
                df_add(rh, rl, w * v.x);
                df_add(ih, il, w * v.y);
                if (eq) {                          // the ring's coefficient E + O
                    const float2 o = G[idx(m, 1) >> 1];
                    df_add(rh, rl, w * o.x);
                    df_add(ih, il, w * o.y);
                }
                odd = !odd;
            }
            return make_float4(rh, rl, ih, il);
        };
        // D = T - f sigma^k0 (B + s conj(Bc)) on every m = j + k N
        auto unfold = [&](int j, int slot, float4 B, float4 Bc, bool sneg) {
            float xr = B.x, xrl = B.y, xi = B.z, xil = B.w;
            const float sj = sneg ? -1.0f : 1.0f;
            df_add(xr, xrl, sj * Bc.x);
            xrl += sj * Bc.y;
            df_add(xi, xil, -sj * Bc.z);
            xil -= sj * Bc.w;
            bool odd = false;
            for (int m = j; m <= ml; m += N) {
                // f = (N or N / 2) sigma^k0, exact in FP32
                const float f = (eq ? 0.5f : 1.0f) * (float)N * ((neg && odd) ? -1.0f : 1.0f);
                const float fr = xr * f, fi = xi * f;
                const float frl = fmaf(xr, f, -fr) + xrl * f, fil = fmaf(xi, f, -fi) + xil * f;
                for (int s2 = 0; s2 < (eq ? 2 : 1); s2++) {
                    const long long i = idx(m, eq ? s2 : slot) >> 1;
                    const float4 t = T[i];
                    float dr = t.x, drl = t.y, di = t.z, dil = t.w;
                    df_add(dr, drl, -fr);
                    drl -= frl;
                    df_add(di, dil, -fi);
                    dil -= fil;
                    const float2 a = df_norm(dr, drl), b = df_norm(di, dil);
                    D[i] = make_float4(a.x, a.y, b.x, b.y);
                }
                odd = !odd;
            }
        };
        // (D is written for the orders m <= ml only: the contraction reads no other)
        for (int slot = 0; slot < (eq ? 1 : 2); slot++) {
            for (int j = 0; j <= min(jmax, ml); j++) {
                const int jp = (N - j) % N;
                const float4 Bj = fold(j, slot);
                const float4 Bjp = (jp == j) ? Bj : (jp <= ml ? fold(jp, slot) : make_float4(0.0f, 0.0f, 0.0f, 0.0f));
                unfold(j, slot, Bj, Bjp, neg && j);
                if (jp != j && jp <= ml) unfold(jp, slot, Bjp, Bj, neg && jp);
            }
        }
    } else {
        const double2* G = (const double2*)Gv;
        const double2* T = (const double2*)Tv;
        double2* D = (double2*)Dv;
        auto fold = [&](int j, int slot) -> double2 {
            double2 b = make_double2(0.0, 0.0);
            double sk = 1.0;
            for (int m = j; m <= mmax; m += N) {
                double2 v = G[idx(m, slot) >> 1];
                if (eq) {                          // the ring's coefficient E + O
                    const double2 o = G[idx(m, 1) >> 1];
                    v.x += o.x;
                    v.y += o.y;
                }
                const double w = (m ? 2.0 : 1.0) * sk;
                b.x += w * v.x;
                b.y += w * v.y;
                if (neg) sk = -sk;
            }
            return b;
        };
        auto unfold = [&](int j, int slot, double2 B, double2 Bc, bool sneg) {
            const double sj = sneg ? -1.0 : 1.0;
            const double xr = B.x + sj * Bc.x, xi = B.y - sj * Bc.y;
            double fk = (eq ? 0.5 : 1.0) * (double)N;
            for (int m = j; m <= mmax; m += N) {
                for (int s2 = 0; s2 < (eq ? 2 : 1); s2++) {
                    const long long i = idx(m, eq ? s2 : slot) >> 1;
                    const double2 t = T[i];
                    D[i] = make_double2(t.x - fk * xr, t.y - fk * xi);
                }
                if (neg) fk = -fk;
            }
        };
        for (int slot = 0; slot < (eq ? 1 : 2); slot++) {
            for (int j = 0; j <= jmax; j++) {
                const int jp = (N - j) % N;
                const double2 Bj = fold(j, slot);
                const double2 Bjp = (jp == j) ? Bj : (jp <= mmax ? fold(jp, slot) : make_double2(0.0, 0.0));
                unfold(j, slot, Bj, Bjp, neg && j);
                if (jp != j && jp <= mmax) unfold(jp, slot, Bjp, Bj, neg && jp);
            }
        }
    }
}

// The same residual for single orders (Algorithm 3 updates the
// coefficients order by order): D[m] = T[m] - F(G)[m], with F(G)[m] =
// f sigma^{k0} [B(j) + sigma_j conj(B(j'))] folded from the current G of
// every order that shares the ring bin j = m mod N (and its mirror j').
// FP64. grid = (ring pair, column blocks of 128, order m0 + z)
__global__ void __launch_bounds__(128)
k_alias_residual_order(const double2* __restrict__ T, const double2* __restrict__ G, double2* __restrict__ D,
                       const PairGeom* __restrict__ pairs, int R_, int mmax, long long ncol, int nmc, int m0)
{
    const int m = m0 + (int)blockIdx.z;
    const int p = blockIdx.x;
    const int mc = blockIdx.y * blockDim.x + threadIdx.x;
    if (mc >= nmc) return;
    const PairGeom g = pairs[p];
    const int N = g.n;
    const bool neg = g.phi0 != 0.0;
    const bool eq = g.start_s < 0;
    const long long qs = (long long)R_ * ncol;
    auto idx = [&](int mm, int slot) -> long long {
        return (((long long)mm * 2 + slot) * qs + (long long)p * ncol + (long long)mc * 2) >> 1;
    };
    auto fold = [&](int j, int slot) -> double2 {
        double2 b = make_double2(0.0, 0.0);
        double sk = 1.0;
        for (int mm = j; mm <= mmax; mm += N) {
            double2 v = G[idx(mm, slot)];
            if (eq) {
                const double2 o = G[idx(mm, 1)];
                v.x += o.x;
                v.y += o.y;
            }
            const double w = (mm ? 2.0 : 1.0) * sk;
            b.x += w * v.x;
            b.y += w * v.y;
            if (neg) sk = -sk;
        }
        return b;
    };
    const int j = m % N, jp = (N - j) % N, k0 = m / N;
    const double sj = (neg && j) ? -1.0 : 1.0;
    const double fk = (eq ? 0.5 : 1.0) * (double)N * ((neg && (k0 & 1)) ? -1.0 : 1.0);
    for (int slot = 0; slot < (eq ? 1 : 2); slot++) {
        const double2 Bj = fold(j, slot);
        const double2 Bc = (jp == j) ? Bj : fold(jp, slot);
        const double xr = Bj.x + sj * Bc.x, xi = Bj.y - sj * Bc.y;
        for (int s2 = 0; s2 < (eq ? 2 : 1); s2++) {
            const long long i = idx(m, eq ? s2 : slot);
            const double2 t = T[i];
            D[i] = make_double2(t.x - fk * xr, t.y - fk * xi);
        }
    }
}

cudaError_t launch_alias_residual_order(const sht_plan* p, const double* T, const double* G, double* D, int nmaps,
                                        int m0, int nm, cudaStream_t st)
{
    const int nmc = nmaps * p->ncomp;
    dim3 grid(p->R, (nmc + 127) / 128, nm);
    prof_start("k_alias_residual_order", st);
    k_alias_residual_order<<<grid, 128, 0, st>>>((const double2*)T, (const double2*)G, (double2*)D, p->t.pairs,
                                                 p->R, p->mmax, ncols(p, nmaps), nmc, m0);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

// column maxima of T[m][q][p][c] (FP32 hi/lo) over the ring pairs, as float
// bits: the quanta of the split map2alm. grid = ((mmax + 1) * 2, column
// blocks of 256)
__global__ void __launch_bounds__(256)
k_colmax_T(const float2* __restrict__ T, unsigned int* __restrict__ colmax, int R_, long long ncol,
           const int* __restrict__ pfirst)
{
    const long long c = (long long)blockIdx.y * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const float2* t = T + (long long)blockIdx.x * R_ * ncol + c;
    float mx = 0.0f;
    // (the ring pairs the order's contraction reads: from pfirst[m])
    for (int p = pfirst ? pfirst[blockIdx.x >> 1] : 0; p < R_; p++) mx = fmaxf(mx, fabsf(t[(long long)p * ncol].x));
    colmax[(long long)blockIdx.x * ncol + c] = __float_as_uint(mx);
}

cudaError_t launch_alias_residual(const sht_plan* p, const void* T, const void* G, void* D, int nmaps,
                                  cudaStream_t st)
{
    const bool split = p->precision != SHT_FP64;
    const int nmc = nmaps * p->ncomp;
    dim3 grid(p->R, (nmc + 127) / 128);
    prof_start("k_alias_residual", st);
    if (split)
        k_alias_residual<true><<<grid, 128, 0, st>>>(T, G, D, p->t.pairs, p->R, p->mmax, ncols(p, nmaps), nmc, p->s.mlim);
    else
        k_alias_residual<false><<<grid, 128, 0, st>>>(T, G, D, p->t.pairs, p->R, p->mmax, ncols(p, nmaps), nmc, nullptr);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_colmax_T(const sht_plan* p, const float2* T, unsigned int* colmax, int nmaps, cudaStream_t st)
{
    const long long nc = ncols(p, nmaps);
    dim3 grid((unsigned)((p->mmax + 1) * 2), (unsigned)((nc + 255) / 256));
    prof_start("k_colmax_T", st);
    k_colmax_T<<<grid, 256, 0, st>>>(T, colmax, p->R, nc, p->s.pfirst);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

}  // namespace sht
