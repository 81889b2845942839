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

}  // namespace sht
