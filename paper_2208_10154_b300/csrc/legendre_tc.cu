// legendre_tc.cu -- split-precision Legendre contraction on the B300 tensor
// cores (tcgen05.mma kind::f16, FP16 operands, FP32 accumulation in TMEM).
//
// The paper's per-m GEMMs (Sec. 2.2 equ:matrix form: A_m = P_m T_m and
// T_m = P_m^t A_m) are evaluated per (m, slot q) with lambda generated on the
// fly in FP64 (normalised same-parity two-step recurrence, scaled exponents),
// so the Legendre matrix never lands in HBM.
//
// Accuracy scheme. The TMEM accumulator truncates toward zero on every MMA,
// which would cost ~1e-6 over K = 1024. Instead each operand x is written, per
// row (lambda) or column (data), in units of a power-of-two quantum u with
// |x/u| <= Q, Q^2 K <= 2^24, as
//     x/u = q + r0 + r1,   q integer (exact in FP16), r0, r1 FP16 residuals
// (FP16 rather than BF16: the residual keeps 22 bits relative to itself, so
// elements far below their row / column maximum stay accurate).
// The products q_a q_b are integers and their sum over K stays below 2^24, so
// the main accumulator is EXACT whatever the rounding mode. The five residual
// products (q r0', q r1', r0 q', r1 q', r0 r0') go to a second accumulator
// whose magnitude is ~2^-7 of the main one, so its truncation is harmless.
// Dropped terms are below 2^-25 of the largest product.
//
// CTA (256 threads, one CTA per SM: 216 KB of SMEM, all 512 TMEM columns):
//   warp 0      TMEM allocation; lane 0 issues the MMAs
//   map2alm:    warps 1-3 generate lambda (one ring pair per lane, walking
//               the 128 rows of the tile from a plan-time checkpoint),
//               warps 4-7 slice the FP32 ring spectra T and then run the epilogue
//   alm2map:    warps 4-7 generate lambda (one ring pair per thread, walking l
//               along K), warps 1-3 slice the FP64 a_lm, warps 4-7 epilogue
// Tile: M = 128 rows (l or ring pairs), N = 256 columns, K chunks of 32, three
// pipeline stages, SWIZZLE_64B K-major operand tiles.
#include "common.cuh"
#include "tc.cuh"

namespace sht {

using namespace tc;

constexpr int TM = 128, TN = 256, KC = 32, NST = 3;
constexpr int A_PLANE = TM * KC * 2;                 // 8 KB
constexpr int B_PLANE = TN * KC * 2;                 // 16 KB
constexpr int STAGE_BYTES = 3 * A_PLANE + 3 * B_PLANE;   // 72 KB
constexpr uint32_t IDESC = idesc_f16(TM, TN);

struct TcArgs {
    const int4* work;          // (m, q, tile, index of its checkpoint block)
    const PairGeom* pairs;
    const double* seed_mant;   // [m][q][p]
    const int* seed_exp;
    const double* nA;          // normalised recurrence: mu_{l+2} = (A x^2 + B) mu_l + mu_{l-2}
    const double* nB;
    const float* nc;           // lambda_l = c_l mu_l
    const double* nc64;        // the same c_l in FP64 (map2alm applies it per output row)
    const double2* ck;         // map2alm checkpoints [block][p] (mu at row r0, mu at row r0-1)
    const int* ck_exp;
    const float* rowmax;       // map2alm: max_p |mu_l(theta_p) 2^E| per packed (l, m)
    const float* pairmax;      // alm2map: max_{l in q} |lambda_lm(theta_p)| per [m][q][p]
    const float* colmax;       // data: max |x| per [m][q][col]
    int* err;
    int lmax, mmax, R, mlo;
    long long ncol, nalm;
    float Q;                   // integer range of the main slices
    double fs0, fs1;           // map2alm: output factor (dsigma times any adjoint weight), m = 0 / m > 0
    float s0, s1;              // alm2map: extra output scale for m = 0 / m > 0
};

// quantum exponent: smallest e with max / 2^e <= Q
__device__ __forceinline__ int quantum_exp(float mx, float Q)
{
    if (!(mx > 0.0f)) return 0;
    int e;
    frexpf(mx / Q, &e);           // mx/Q = f 2^e, f in [0.5, 1)  ->  mx/Q < 2^e
    return e;
}

__device__ __forceinline__ long long a_idx(int lmax, int l, int m)
{
    return (long long)m * (2 * lmax + 1 - m) / 2 + l;
}

// write one (q, r0, r1) triple of element (row, k) into the three planes
__device__ __forceinline__ void put3(uint8_t* planes, int plane_bytes, int row, int k, float v)
{
    float q, r0, r1;
    slice3(v, q, r0, r1);
    uint32_t off = sw64_off(row, k);
    *reinterpret_cast<__half*>(planes + off) = __float2half_rn(q);
    *reinterpret_cast<__half*>(planes + plane_bytes + off) = __float2half_rn(r0);
    *reinterpret_cast<__half*>(planes + 2 * plane_bytes + off) = __float2half_rn(r1);
}

// write 8 consecutive k (chunk j) of one row into the three planes
__device__ __forceinline__ void put3x8(uint8_t* planes, int plane_bytes, int row, int j, const float (&v)[8])
{
    uint32_t qq[4], a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float q0, x0, y0, q1, x1, y1;
        slice3(v[2 * i], q0, x0, y0);
        slice3(v[2 * i + 1], q1, x1, y1);
        qq[i] = pack_h2(q0, q1);
        a[i] = pack_h2(x0, x1);
        b[i] = pack_h2(y0, y1);
    }
    uint32_t off = sw64_chunk(row, j);
    *reinterpret_cast<uint4*>(planes + off) = make_uint4(qq[0], qq[1], qq[2], qq[3]);
    *reinterpret_cast<uint4*>(planes + plane_bytes + off) = make_uint4(a[0], a[1], a[2], a[3]);
    *reinterpret_cast<uint4*>(planes + 2 * plane_bytes + off) = make_uint4(b[0], b[1], b[2], b[3]);
}

// the same with FP32 remainders vl (value = v + vl)
__device__ __forceinline__ void put3x8l(uint8_t* planes, int plane_bytes, int row, int j, const float (&v)[8],
                                        const float (&vl)[8])
{
    uint32_t qq[4], a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float q0, x0, y0, q1, x1, y1;
        slice3x(v[2 * i], vl[2 * i], q0, x0, y0);
        slice3x(v[2 * i + 1], vl[2 * i + 1], q1, x1, y1);
        qq[i] = pack_h2(q0, q1);
        a[i] = pack_h2(x0, x1);
        b[i] = pack_h2(y0, y1);
    }
    uint32_t off = sw64_chunk(row, j);
    *reinterpret_cast<uint4*>(planes + off) = make_uint4(qq[0], qq[1], qq[2], qq[3]);
    *reinterpret_cast<uint4*>(planes + plane_bytes + off) = make_uint4(a[0], a[1], a[2], a[3]);
    *reinterpret_cast<uint4*>(planes + 2 * plane_bytes + off) = make_uint4(b[0], b[1], b[2], b[3]);
}

__device__ __forceinline__ void issue_chunk(uint32_t tmem, uint32_t stage_addr, bool first)
{
    const uint32_t A0 = stage_addr, A1 = A0 + A_PLANE, A2 = A1 + A_PLANE;
    const uint32_t B0 = stage_addr + 3 * A_PLANE, B1 = B0 + B_PLANE, B2 = B1 + B_PLANE;
#pragma unroll
    for (int kk = 0; kk < 2; kk++) {
        const uint32_t o = kk * 32;
        const uint32_t acc = (first && kk == 0) ? 0u : 1u;
        umma_f16(tmem, desc_sw64(A0 + o), desc_sw64(B0 + o), IDESC, acc);             // main: q q'
        umma_f16(tmem + TN, desc_sw64(A0 + o), desc_sw64(B1 + o), IDESC, acc);        // q r0'
        umma_f16(tmem + TN, desc_sw64(A0 + o), desc_sw64(B2 + o), IDESC, 1u);         // q r1'
        umma_f16(tmem + TN, desc_sw64(A1 + o), desc_sw64(B0 + o), IDESC, 1u);         // r0 q'
        umma_f16(tmem + TN, desc_sw64(A2 + o), desc_sw64(B0 + o), IDESC, 1u);         // r1 q'
        umma_f16(tmem + TN, desc_sw64(A1 + o), desc_sw64(B1 + o), IDESC, 1u);         // r0 r0'
    }
}

struct TcShared {
    uint64_t full[NST];
    uint64_t empty[NST];
    uint64_t accf;
    uint32_t tmem;
    int colexp[TN];
    int rowexp[TM];
    double cA[TM], cB[TM];
    float2 rfac[TM];           // map2alm: c_l * factor as an FP32 hi/lo pair
};
constexpr int SMEM_TC = NST * STAGE_BYTES + (int)sizeof(TcShared) + 1024;

// ===========================================================================
// map2alm: a[l, c] = sum_p lambda_lm(theta_p) dsig T[p, c]   (rows l = m + q + 2r)
// ===========================================================================
__global__ void __launch_bounds__(256, 1)
k_leg_m2a_tc(const float* __restrict__ T, const float* __restrict__ Tlo, double* __restrict__ alm, TcArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcShared& sh = *reinterpret_cast<TcShared*>(smem + NST * STAGE_BYTES);
    const int4 w = a.work[blockIdx.x];
    const int m = w.x, q = w.y, rt = w.z, ckb = w.w;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c0 = blockIdx.y * TN;
    const int l_first = m + q;
    const int nrows = (a.lmax >= l_first) ? (a.lmax - l_first) / 2 + 1 : 0;
    const int r0 = rt * TM;
    const int nch = (a.R + KC - 1) / KC;
    const long long qstride = (long long)a.R * a.ncol;
    const float* Tq = T + ((long long)m * 2 + q) * qstride;
    const float* Tlq = (m < a.mlo) ? Tlo + ((long long)m * 2 + q) * qstride : nullptr;

    // per-row constants and scales
    for (int r = tid; r < TM; r += blockDim.x) {
        int row = r0 + r;
        if (row < nrows) {
            int l = l_first + 2 * row;
            long long ci = a_idx(a.lmax, l, m);
            sh.cA[r] = a.nA[ci];
            sh.cB[r] = a.nB[ci];
            sh.rowexp[r] = quantum_exp(a.rowmax[ci], a.Q);
            // the row factor c_l * dsigma is applied once per output, in
            // double-float, so its rounding is not a coherent error on the row
            double f = a.nc64[ci] * (m == 0 ? a.fs0 : a.fs1);
            float fh = (float)f;
            sh.rfac[r] = make_float2(fh, (float)(f - (double)fh));
        } else {
            sh.cA[r] = 0.0; sh.cB[r] = 0.0; sh.rowexp[r] = 0; sh.rfac[r] = make_float2(0.0f, 0.0f);
        }
    }
    for (int c = tid; c < TN; c += blockDim.x) {
        long long cg = c0 + c;
        sh.colexp[c] = (cg < a.ncol) ? quantum_exp(a.colmax[((long long)m * 2 + q) * a.ncol + cg], a.Q) : 0;
    }
    if (tid == 0) {
        for (int s = 0; s < NST; s++) { mbar_init(&sh.full[s], 32 + 128); mbar_init(&sh.empty[s], 1); }
        mbar_init(&sh.accf, 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(&sh.tmem, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem;
    const uint32_t smem_base = smem_u32(smem);

    if (warp == 0) {
        if (lane == 0) {
            for (int kc = 0; kc < nch; kc++) {
                const int s = kc % NST;
                const uint32_t u = kc / NST;
                if (!mbar_wait(&sh.full[s], u & 1, a.err, 1)) break;
                tc_fence_after();
                issue_chunk(tmem, smem_base + s * STAGE_BYTES, kc == 0);
                umma_commit(&sh.empty[s]);
            }
            umma_commit(&sh.accf);
        }
    } else if (warp < 4) {
        // ---- lambda producers: chunk kc belongs to warp 1 + kc % 3 ----
        for (int kc = warp - 1; kc < nch; kc += 3) {
            const int s = kc % NST;
            const uint32_t u = kc / NST;
            if (u >= 1 && !mbar_wait(&sh.empty[s], (u - 1) & 1, a.err, 2)) break;
            uint8_t* A = smem + s * STAGE_BYTES;
            const int p = kc * KC + lane;
            double cur = 0.0, prev = 0.0, x2 = 0.0;
            int E = 0;
            if (p < a.R) {
                double2 v = a.ck[(long long)ckb * a.R + p];
                cur = v.x; prev = v.y;
                E = a.ck_exp[(long long)ckb * a.R + p];
                double x = a.pairs[p].x;
                x2 = x * x;
            }
            for (int r = 0; r < TM; r++) {
                float v = 0.0f;
                if (r0 + r < nrows) {
                    v = f64_to_f32_scaled(cur, E - sh.rowexp[r]);
                    double t = fma(sh.cA[r], x2, sh.cB[r]);
                    double nxt = fma(t, cur, prev);
                    prev = cur;
                    cur = nxt;
                    if (((__double2hiint(cur) >> 20) & 0x7FF) > 1023 + 500) {
                        cur *= 0x1p-500; prev *= 0x1p-500; E += 500;
                    }
                }
                put3(A, A_PLANE, r, lane, v);
            }
            fence_proxy_async_smem();
            mbar_arrive(&sh.full[s]);
        }
    } else {
        // ---- data producers: slice T[p][c] for two columns per thread ----
        const int t4 = tid - 128;
        const int cl = 2 * t4;
        const long long cg = c0 + cl;
        const int e0 = sh.colexp[cl], e1 = sh.colexp[cl + 1];
        for (int kc = 0; kc < nch; kc++) {
            const int s = kc % NST;
            const uint32_t u = kc / NST;
            if (u >= 1 && !mbar_wait(&sh.empty[s], (u - 1) & 1, a.err, 3)) break;
            uint8_t* B = smem + s * STAGE_BYTES + 3 * A_PLANE;
#pragma unroll
            for (int j = 0; j < KC / 8; j++) {
                float va[8], vb[8], la[8], lb[8];
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    int p = kc * KC + j * 8 + i;
                    float2 x = make_float2(0.0f, 0.0f), xl = make_float2(0.0f, 0.0f);
                    if (p < a.R && cg < a.ncol) {
                        x = *reinterpret_cast<const float2*>(Tq + (long long)p * a.ncol + cg);
                        if (Tlq) xl = *reinterpret_cast<const float2*>(Tlq + (long long)p * a.ncol + cg);
                    }
                    va[i] = ldexpf_fast(x.x, -e0);
                    vb[i] = ldexpf_fast(x.y, -e1);
                    la[i] = ldexpf_fast(xl.x, -e0);
                    lb[i] = ldexpf_fast(xl.y, -e1);
                }
                put3x8l(B, B_PLANE, cl, j, va, la);
                put3x8l(B, B_PLANE, cl + 1, j, vb, lb);
            }
            fence_proxy_async_smem();
            mbar_arrive(&sh.full[s]);
        }
        // ---- epilogue: a_lm = (main + corr) * 2^(e_row + e_col), FP64 final add ----
        const int quarter = warp & 3;
        const int r = quarter * 32 + lane;
        const int row = r0 + r;
        bool ok = mbar_wait(&sh.accf, 0, a.err, 4);
        tc_fence_after();
        const int l = l_first + 2 * row;
        const bool live = ok && row < nrows;
        const long long li = live ? a_idx(a.lmax, l, m) : 0;
        const float2 F = sh.rfac[r];
        for (int c = 0; c < TN; c += 16) {
            uint32_t vm[16], vc[16];
            const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
            tmem_ld16(tl + c, vm);
            tmem_ld16(tl + TN + c, vc);
            tmem_wait_ld();
            if (!live) continue;
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                long long cgj = c0 + c + j;
                if (cgj >= a.ncol) break;
                double out[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    // (main + corr) * (Fh + Fl): main is an exact integer, the
                    // product error of main * Fh is recovered with an FMA
                    const float mn = __uint_as_float(vm[j + h]), cr = __uint_as_float(vc[j + h]);
                    const float p1 = mn * F.x;
                    const float e1 = fmaf(mn, F.x, -p1);
                    const float lo = e1 + cr * F.x + (mn + cr) * F.y;
                    double v = f32_to_f64(p1) + f32_to_f64(lo);          // final FP64 accumulation
                    out[h] = ldexp_fast(v, sh.rowexp[r] + sh.colexp[c + j + h]);
                }
                if (m == 0) out[1] = 0.0;
                long long mc = cgj >> 1;
                *reinterpret_cast<double2*>(alm + (mc * a.nalm + li) * 2) = make_double2(out[0], out[1]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ===========================================================================
// alm2map: G[m][q][p][c] = sum_{l in q} lambda_lm(theta_p) a[l, c]
// ===========================================================================
__global__ void __launch_bounds__(256, 1)
k_leg_a2m_tc(const double* __restrict__ alm, float* __restrict__ G, TcArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcShared& sh = *reinterpret_cast<TcShared*>(smem + NST * STAGE_BYTES);
    const int4 w = a.work[blockIdx.x];
    const int m = w.x, q = w.y, pt = w.z;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c0 = blockIdx.y * TN;
    const int p0 = pt * TM;
    const int lk0 = m + q;
    const int K = (a.lmax >= lk0) ? (a.lmax - lk0) / 2 + 1 : 0;
    const int nch = (K + KC - 1) / KC;
    const long long qstride = (long long)a.R * a.ncol;

    for (int c = tid; c < TN; c += blockDim.x) {
        long long cg = c0 + c;
        sh.colexp[c] = (cg < a.ncol) ? quantum_exp(a.colmax[((long long)m * 2 + q) * a.ncol + cg], a.Q) : 0;
    }
    for (int r = tid; r < TM; r += blockDim.x) {
        int p = p0 + r;
        sh.rowexp[r] = (p < a.R) ? quantum_exp(a.pairmax[((long long)m * 2 + q) * a.R + p], a.Q) : 0;
    }
    if (tid == 0) {
        for (int s = 0; s < NST; s++) { mbar_init(&sh.full[s], 128 + 96); mbar_init(&sh.empty[s], 1); }
        mbar_init(&sh.accf, 1);
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(&sh.tmem, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem;
    const uint32_t smem_base = smem_u32(smem);

    if (warp == 0) {
        if (lane == 0 && nch > 0) {
            for (int kc = 0; kc < nch; kc++) {
                const int s = kc % NST;
                const uint32_t u = kc / NST;
                if (!mbar_wait(&sh.full[s], u & 1, a.err, 5)) break;
                tc_fence_after();
                issue_chunk(tmem, smem_base + s * STAGE_BYTES, kc == 0);
                umma_commit(&sh.empty[s]);
            }
            umma_commit(&sh.accf);
        }
    } else if (warp < 4) {
        // ---- data producers: a_lm (FP64) -> slices; item = (map, octet of k) ----
        const int t3 = tid - 32;
        for (int kc = 0; kc < nch; kc++) {
            const int s = kc % NST;
            const uint32_t u = kc / NST;
            if (u >= 1 && !mbar_wait(&sh.empty[s], (u - 1) & 1, a.err, 6)) break;
            uint8_t* B = smem + s * STAGE_BYTES + 3 * A_PLANE;
            for (int it = t3; it < (TN / 2) * (KC / 8); it += 96) {
                const int mp = it >> 2, j = it & 3;
                const int cl = 2 * mp;
                const long long cg = c0 + cl;
                const int e0 = sh.colexp[cl], e1 = sh.colexp[cl + 1];
                float va[8], vb[8];
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    int k = kc * KC + j * 8 + i;
                    double2 x = make_double2(0.0, 0.0);
                    if (k < K && cg < a.ncol) {
                        int l = lk0 + 2 * k;
                        x = *reinterpret_cast<const double2*>(alm + ((cg >> 1) * a.nalm + a_idx(a.lmax, l, m)) * 2);
                        if (m == 0) x.y = 0.0;
                    }
                    va[i] = f64_to_f32_scaled(x.x, -e0);
                    vb[i] = f64_to_f32_scaled(x.y, -e1);
                }
                put3x8(B, B_PLANE, cl, j, va);
                put3x8(B, B_PLANE, cl + 1, j, vb);
            }
            fence_proxy_async_smem();
            mbar_arrive(&sh.full[s]);
        }
    } else {
        // ---- lambda producers: one ring pair per thread, walking l along K ----
        const int r = tid - 128;
        const int p = p0 + r;
        double cur = 0.0, prev = 0.0, x2 = 0.0;
        int E = 0;
        const int erow = sh.rowexp[r];
        if (p < a.R) {
            long long si = ((long long)m * 2 + q) * a.R + p;
            cur = a.seed_mant[si];
            E = a.seed_exp[si];
            double x = a.pairs[p].x;
            x2 = x * x;
        }
        for (int kc = 0; kc < nch; kc++) {
            const int s = kc % NST;
            const uint32_t u = kc / NST;
            if (u >= 1 && !mbar_wait(&sh.empty[s], (u - 1) & 1, a.err, 7)) break;
            uint8_t* A = smem + s * STAGE_BYTES;
#pragma unroll
            for (int j = 0; j < KC / 8; j++) {
                float v[8];
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    int k = kc * KC + j * 8 + i;
                    v[i] = 0.0f;
                    if (k < K) {
                        int l = lk0 + 2 * k;
                        long long ci = a_idx(a.lmax, l, m);
                        v[i] = f64_to_f32_scaled(cur, E - erow) * a.nc[ci];
                        double t = fma(a.nA[ci], x2, a.nB[ci]);
                        double nxt = fma(t, cur, prev);
                        prev = cur;
                        cur = nxt;
                        if (((__double2hiint(cur) >> 20) & 0x7FF) > 1023 + 500) {
                            cur *= 0x1p-500; prev *= 0x1p-500; E += 500;
                        }
                    }
                }
                put3x8(A, A_PLANE, r, j, v);
            }
            fence_proxy_async_smem();
            mbar_arrive(&sh.full[s]);
        }
        // ---- epilogue: G = (main + corr) * 2^(e_row + e_col) in FP32 ----
        const int quarter = warp & 3;
        const int rr = quarter * 32 + lane;
        const int pp = p0 + rr;
        bool ok = (nch == 0) || mbar_wait(&sh.accf, 0, a.err, 8);
        tc_fence_after();
        const float sc = (m == 0) ? a.s0 : a.s1;
        float* Gq = G + ((long long)m * 2 + q) * qstride + (long long)pp * a.ncol;
        for (int c = 0; c < TN; c += 16) {
            uint32_t vm[16], vc[16];
            if (nch > 0) {
                const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
                tmem_ld16(tl + c, vm);
                tmem_ld16(tl + TN + c, vc);
                tmem_wait_ld();
            }
            if (pp >= a.R || !ok) continue;
            float out[16];
#pragma unroll
            for (int j = 0; j < 16; j++) {
                out[j] = 0.0f;
                if (nch > 0)
                    out[j] = sc * ldexpf_fast(__uint_as_float(vm[j]) + __uint_as_float(vc[j]),
                                              sh.rowexp[rr] + sh.colexp[c + j]);
            }
            long long cg = c0 + c;
            if (cg + 16 <= a.ncol && (a.ncol & 3) == 0) {
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    *reinterpret_cast<float4*>(Gq + cg + j) = make_float4(out[j], out[j + 1], out[j + 2], out[j + 3]);
            } else {
                for (int j = 0; j < 16 && cg + j < a.ncol; j++) Gq[cg + j] = out[j];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ===========================================================================
// plan-time walk: checkpoints of the map2alm chains at every row tile, the
// per-row maxima over ring pairs (map2alm scales) and the per-pair maxima
// over l (alm2map scales). grid = (mmax+1, 2), threads over ring pairs.
// ===========================================================================
__global__ void __launch_bounds__(256)
k_split_tables(TcArgs a, const int* __restrict__ ck_base, double2* __restrict__ ck, int* __restrict__ ck_exp,
               unsigned int* __restrict__ rowmax_bits, float* __restrict__ pairmax)
{
    const int m = blockIdx.x, q = blockIdx.y;
    const int l_first = m + q;
    const int nrows = (a.lmax >= l_first) ? (a.lmax - l_first) / 2 + 1 : 0;
    const int base = ck_base[m * 2 + q];
    for (int p0 = 0; p0 < a.R; p0 += blockDim.x) {
        const int p = p0 + threadIdx.x;
        const bool valid = p < a.R;
        double cur = 0.0, prev = 0.0, x2 = 0.0;
        int E = 0;
        if (valid) {
            long long si = ((long long)m * 2 + q) * a.R + p;
            cur = a.seed_mant[si];
            E = a.seed_exp[si];
            double x = a.pairs[p].x;
            x2 = x * x;
        }
        float pmax = 0.0f;
        for (int row = 0; row < nrows; row++) {
            if (valid && (row % TM) == 0) {
                long long ci = (long long)(base + row / TM) * a.R + p;
                ck[ci] = make_double2(cur, prev);
                ck_exp[ci] = E;
            }
            int l = l_first + 2 * row;
            long long ci = a_idx(a.lmax, l, m);
            float v = 0.0f, vmu = 0.0f;
            if (valid) {
                // |mu 2^E| for the map2alm row quanta; |lambda| = |c_l mu 2^E| for alm2map
                vmu = fabsf(f64_to_f32_scaled(cur, E));
                v = vmu * fabsf(a.nc[ci]);
                double t = fma(a.nA[ci], x2, a.nB[ci]);
                double nxt = fma(t, cur, prev);
                prev = cur;
                cur = nxt;
                if (((__double2hiint(cur) >> 20) & 0x7FF) > 1023 + 500) {
                    cur *= 0x1p-500; prev *= 0x1p-500; E += 500;
                }
            }
            pmax = fmaxf(pmax, v);
            // max over the ring pairs of this warp, then one atomic per warp
            float wv = vmu;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wv = fmaxf(wv, __shfl_xor_sync(0xffffffffu, wv, o));
            if ((threadIdx.x & 31) == 0 && wv > 0.0f) atomicMax(rowmax_bits + ci, __float_as_uint(wv));
        }
        if (valid) pairmax[((long long)m * 2 + q) * a.R + p] = pmax;
    }
}

// ===========================================================================
// alm2map data scales: max over l in slot q of |a_lm| per column
// grid = (mmax+1, ceil(ncol/256)); thread = column
// ===========================================================================
__global__ void __launch_bounds__(256)
k_alm_colmax(const double* __restrict__ alm, float* __restrict__ colmax, int lmax, long long nalm, long long ncol)
{
    const int m = blockIdx.x;
    const long long c = (long long)blockIdx.y * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const long long mc = c >> 1;
    const int reim = (int)(c & 1);
    float mx[2] = {0.0f, 0.0f};
    const double* base = alm + (mc * nalm + a_idx(lmax, m, m)) * 2 + reim;
    for (int l = m; l <= lmax; l++) {
        double v = base[(long long)(l - m) * 2];
        if (m == 0 && reim) v = 0.0;
        float f = fabsf(f64_to_f32_scaled(v, 0));
        mx[(l - m) & 1] = fmaxf(mx[(l - m) & 1], f * 1.0000002f);
    }
    colmax[((long long)m * 2 + 0) * ncol + c] = mx[0];
    colmax[((long long)m * 2 + 1) * ncol + c] = mx[1];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static TcArgs make_tc(const sht_plan* p, int nmaps, const float* colmax, float Q, float s0, float s1)
{
    TcArgs a;
    a.pairs = p->t.pairs;
    a.seed_mant = p->t.seed_mant;
    a.seed_exp = p->t.seed_exp;
    a.nA = p->s.nA; a.nB = p->s.nB; a.nc = p->s.nc; a.nc64 = p->s.nc64;
    a.ck = p->s.ck; a.ck_exp = p->s.ck_exp;
    a.rowmax = (const float*)p->s.rowmax_bits;
    a.pairmax = p->s.pairmax;
    a.colmax = colmax;
    a.err = p->s.err;
    a.lmax = p->lmax; a.mmax = p->mmax; a.R = p->R; a.mlo = p->s.mlo;
    a.ncol = ncols(p, nmaps); a.nalm = p->nalm;
    a.Q = Q;
    a.fs0 = a.fs1 = 1.0;
    a.s0 = s0; a.s1 = s1;
    a.work = nullptr;
    return a;
}

cudaError_t launch_legendre_m2a_tc(const sht_plan* p, const float* T, const float* Tlo, const float* colmax, double* alm,
                                   int nmaps, double fs0, double fs1, cudaStream_t st)
{
    if (p->s.nwork_m2a == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_leg_m2a_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC);
    if (e != cudaSuccess) return e;
    TcArgs a = make_tc(p, nmaps, colmax, p->s.Q_m2a, 1.0f, 1.0f);
    a.fs0 = fs0; a.fs1 = fs1;
    a.work = p->s.work_m2a;
    long long nc = ncols(p, nmaps);
    dim3 grid((unsigned)p->s.nwork_m2a, (unsigned)((nc + TN - 1) / TN));
    prof_start("k_leg_m2a_tc", st);
    k_leg_m2a_tc<<<grid, 256, SMEM_TC, st>>>(T, Tlo, alm, a);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_legendre_a2m_tc(const sht_plan* p, const double* alm, const float* colmax, float* G,
                                   int nmaps, float s0, float s1, cudaStream_t st)
{
    if (p->s.nwork_a2m == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_leg_a2m_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC);
    if (e != cudaSuccess) return e;
    TcArgs a = make_tc(p, nmaps, colmax, p->s.Q_a2m, s0, s1);
    a.work = p->s.work_a2m;
    long long nc = ncols(p, nmaps);
    dim3 grid((unsigned)p->s.nwork_a2m, (unsigned)((nc + TN - 1) / TN));
    prof_start("k_leg_a2m_tc", st);
    k_leg_a2m_tc<<<grid, 256, SMEM_TC, st>>>(alm, G, a);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_alm_colmax(const sht_plan* p, const double* alm, float* colmax, int nmaps, cudaStream_t st)
{
    long long nc = ncols(p, nmaps);
    dim3 grid((unsigned)(p->mmax + 1), (unsigned)((nc + 255) / 256));
    prof_start("k_alm_colmax", st);
    k_alm_colmax<<<grid, 256, 0, st>>>(alm, colmax, p->lmax, p->nalm, nc);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t run_split_tables(sht_plan* p, const int* d_ck_base)
{
    TcArgs a = make_tc(p, 1, nullptr, 1.0f, 1.0f, 1.0f);
    dim3 grid(p->mmax + 1, 2);
    k_split_tables<<<grid, 256>>>(a, d_ck_base, p->s.ck, p->s.ck_exp, p->s.rowmax_bits, p->s.pairmax);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaDeviceSynchronize();
}

int split_row_tile() { return TM; }
int split_col_tile() { return TN; }

}  // namespace sht
