// legendre_tc.cu -- split-precision Legendre contraction on the B300 tensor
// cores (tcgen05.mma kind::f16, FP16 operands, FP32 accumulation in TMEM).
//
// The paper's per-m GEMMs (Sec. 2.2 equ:matrix form: A_m = P_m T_m and
// T_m = P_m^t A_m) are evaluated per (m, slot q) with lambda generated on the
// fly by the FP64 recurrence with scaled exponents (normalised same-parity
// two-step form), so the Legendre matrix never lands in HBM.
//
// Orientation. The MMA's M dimension (TMEM lanes) is 128 map columns
// (map, component, Re/Im); its N dimension is the lambda side: l rows for
// map2alm (N = the rows left in the l tile, rounded up to 16, so short tiles at
// high m cost only what they hold) and ring pairs for alm2map. K is the
// contraction: ring pairs (map2alm) or l (alm2map).
//
// Accuracy. Every operand x is written, per row or column, in units of a
// power-of-two quantum u with |x/u| <= Q (K Q^2 <= 2^24, Q <= 127) as three
// FP16 slices q + r0 + r1 (tc::slice3d: integer, a multiple of 2^-12, and the
// rest below 2^-13). Eight products per K step, in three TMEM accumulators:
//     main = sum q q'                        integers below 2^24: exact
//     ex   = q r0' + r0 q'                   multiples of 2^-12 below 2^12 per
//                                            32-wide K chunk: exact
//     sm   = q r1' + r1 q' + r0 r0' + r0 r1' + r1 r0'     below ~9 per chunk
// The TMEM accumulator truncates toward zero on every MMA, so a sum that is not
// exact picks up a bias that grows with its magnitude and length. After every
// 32-wide K chunk the epilogue warps drain both into an exact integer count of
// 2^-12 kept in a fourth TMEM region: all of ex (which the next chunk
// restarts), and sm rounded to the 2^-12 grid, leaving in sm only its residual
// (below 2^-13) for the next chunk to accumulate onto. sm thus never grows past
// one chunk's worth, and nothing but the truncation of those small partial sums
// and the dropped r1 r1' (< 2^-26) is lost.
//
// Cluster sharing of lambda. The FP64 recurrence is the costly part (FP64 runs
// at ~1/64 of FP32 here), so the CTAs of a thread-block cluster, which work on
// the same (m, q, tile) for different column tiles, split the lambda work:
// lambda for one stage is cut into 32-row pieces, each produced by one warp of
// one CTA, written to its own shared memory and copied to every other CTA of
// the cluster with cp.async.bulk (shared::cta -> shared::cluster), completing
// on the destination's mbarrier. Each CTA's MMA completion is multicast to the
// "stage free" barriers of all CTAs of the cluster.
//
// CTA: 256 threads, one per SM (192 KB of pipeline stages, 512 TMEM columns).
//   warp 0       TMEM allocation; lane 0 issues the MMAs
//   warps 1-3    lambda pieces (32 ring pairs x 32 rows / steps each)
//   warps 4-7    slice the data (one map column per thread), then the epilogue
#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "tc.cuh"

namespace sht {

using namespace tc;

constexpr int TC_M = 128;                        // map columns per CTA (MMA M)
constexpr int TC_N = 128;                        // lambda rows per CTA (MMA N, max)
constexpr int KC = 32;                           // K per pipeline stage (2 MMA K-steps)
constexpr int NST = 3;                           // pipeline stages
constexpr int PR = 32;                           // rows per lambda piece
constexpr int A_PLANE = TC_M * KC * 2;           // 8 KB (data, one slice)
constexpr int B_PLANE = TC_N * KC * 2;           // 8 KB (lambda, one slice)
constexpr int PIECE_BYTES = PR * KC * 2;         // 2 KB of one B plane
constexpr int STAGE_BYTES = 3 * A_PLANE + 3 * B_PLANE;   // 48 KB
constexpr int STG_ROW = TC_M * 8;                // one K row of raw data (FP32 hi/lo per column): 1 KB
constexpr int STG_BYTES = KC * STG_ROW;          // 32 KB: one K chunk of raw data for the CTA's columns
constexpr uint32_t ACC_EX = 128;                 // TMEM columns: exact corrections of one chunk
constexpr uint32_t ACC_SM = 256;                 //   small corrections (+ the residual of earlier chunks)
constexpr uint32_t ACC_HX = 384;                 //   int32 count of 2^-12 drained so far
constexpr int CK_ROWS = 32;                      // rows between recurrence checkpoints
constexpr int MAX_CLUSTER = 8;

struct TcArgs {
    const int4* work;          // (m, q, tile, first checkpoint block of (m, q))
    const PairGeom* pairs;
    const double* nA;          // normalised recurrence: mu_{l+2} = (A x^2 + B) mu_l + mu_{l-2}
    const double* nB;
    const float* nc;           // lambda_l = c_l mu_l (FP32 copy, for maxima)
    const double* nc64;        // c_l in FP64 (map2alm applies it per output row)
    const float2* nc2;         // c_l as an FP32 hi/lo pair (alm2map applies it to lambda)
    const double2* ck;         // checkpoints [block][p]: (mu at row 32b, mu at row 32b - 1)
    const int* ck_exp;
    const float* rowmax;       // map2alm: max_p |mu_l(theta_p) 2^E| per packed (l, m)
    const float* pairmax;      // alm2map: max_{l in q} |lambda_lm(theta_p)| per [m][q][p]
    const float* colmax;       // data: max |x| per [m][q][col]
    int* err;
    int lmax, mmax, R;
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

// 8 consecutive k (16-byte chunk j) of row `row`, three slice planes
__device__ __forceinline__ void put3x8(uint8_t* planes, int plane_bytes, int row, int j, const float (&v)[8],
                                       const float (&vl)[8])
{
    uint32_t qq[4], a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float q0, x0, y0, q1, x1, y1;
        slice3d(v[2 * i], vl[2 * i], q0, x0, y0);
        slice3d(v[2 * i + 1], vl[2 * i + 1], q1, x1, y1);
        qq[i] = pack_h2(q0, q1);
        a[i] = pack_h2(x0, x1);
        b[i] = pack_h2(y0, y1);
    }
    const uint32_t off = sw64_chunk(row, j);
    *reinterpret_cast<uint4*>(planes + off) = make_uint4(qq[0], qq[1], qq[2], qq[3]);
    *reinterpret_cast<uint4*>(planes + plane_bytes + off) = make_uint4(a[0], a[1], a[2], a[3]);
    *reinterpret_cast<uint4*>(planes + 2 * plane_bytes + off) = make_uint4(b[0], b[1], b[2], b[3]);
}

// one stage (two MMA K-steps), A = data, B = lambda: the main products into
// TMEM column 0 (accumulated over the whole of K) ...
__device__ __forceinline__ void issue_main(uint32_t tmem, uint32_t st_addr, uint32_t idesc, bool first)
{
    const uint32_t A0 = st_addr, B0 = st_addr + 3 * A_PLANE;
#pragma unroll
    for (int kk = 0; kk < 2; kk++) {
        const uint32_t o = kk * 32;
        umma_f16(tmem, desc_sw64(A0 + o), desc_sw64(B0 + o), idesc, (first && kk == 0) ? 0u : 1u);   // q q'
    }
}
// ... and the seven correction products into the ex accumulator, which this
// stage restarts, and the sm accumulator, which only the first stage restarts
__device__ __forceinline__ void issue_corr(uint32_t tmem, uint32_t st_addr, uint32_t idesc, bool first)
{
    const uint32_t A0 = st_addr, A1 = A0 + A_PLANE, A2 = A1 + A_PLANE;
    const uint32_t B0 = st_addr + 3 * A_PLANE, B1 = B0 + B_PLANE, B2 = B1 + B_PLANE;
    const uint32_t ex = tmem + ACC_EX, sm = tmem + ACC_SM;
#pragma unroll
    for (int kk = 0; kk < 2; kk++) {
        const uint32_t o = kk * 32;
        const uint32_t acc = kk == 0 ? 0u : 1u;
        umma_f16(ex, desc_sw64(A0 + o), desc_sw64(B1 + o), idesc, acc);                              // q r0'
        umma_f16(ex, desc_sw64(A1 + o), desc_sw64(B0 + o), idesc, 1u);                               // r0 q'
        umma_f16(sm, desc_sw64(A0 + o), desc_sw64(B2 + o), idesc, (first && kk == 0) ? 0u : 1u);     // q r1'
        umma_f16(sm, desc_sw64(A2 + o), desc_sw64(B0 + o), idesc, 1u);                               // r1 q'
        umma_f16(sm, desc_sw64(A1 + o), desc_sw64(B1 + o), idesc, 1u);                               // r0 r0'
        umma_f16(sm, desc_sw64(A1 + o), desc_sw64(B2 + o), idesc, 1u);                               // r0 r1'
        umma_f16(sm, desc_sw64(A2 + o), desc_sw64(B1 + o), idesc, 1u);                               // r1 r0'
    }
}

struct TcShared {
    uint64_t full[NST];        // stage filled: 4 data warps + one arrival per lambda piece
    uint64_t empty[NST];       // stage consumed by the MMAs of every CTA of the cluster
    uint64_t accf;             // all MMAs of this CTA done
    uint64_t cdone;            // the correction accumulators hold a finished chunk
    uint64_t cfree;            // the correction accumulators drained (4 epilogue warps)
    uint64_t sfull[2];         // raw-data staging buffer b filled (bulk copies)
    int released;              // highest chunk whose stage is free in every CTA of the cluster
    uint32_t tmem;
    int colexp[TC_M];
    int rowexp[TC_N];          // quantum exponent per lambda row (l or ring pair)
    double cA[TC_N], cB[TC_N]; // map2alm: recurrence coefficients of the tile's rows
    float2 rfac[TC_N];         // map2alm: c_l * factor as an FP32 hi/lo pair
};
constexpr int SMEM_TC = NST * STAGE_BYTES + 2 * STG_BYTES + (int)sizeof(TcShared) + 1024;

// x * 2^-500 by exponent arithmetic (x is either 0 or has a biased exponent
// above 500 here, or is flushed to 0 if it does not)
__device__ __forceinline__ double down500(double x)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    return e > 500 ? __longlong_as_double(b - (500ll << 52)) : 0.0;
}
// rescale of the scaled-exponent recurrence (mu 2^E). Integer exponent
// arithmetic instead of an FP64 multiply: FP64 latency is ~185 cycles on
// this GPU and the rescale test sits on the recurrence's critical path.
__device__ __forceinline__ void rescale(double& cur, double& prev, int& E)
{
    if (((__double2hiint(cur) >> 20) & 0x7FF) > 1023 + 500) {
        cur = down500(cur);
        prev = down500(prev);
        E += 500;
    }
}

// ===========================================================================
// map2alm (M2A = true):  a[l, c] = f_l sum_p lambda_lm(theta_p) T[p, c]
// alm2map (M2A = false): G[p, c] = s   sum_l lambda_lm(theta_p) a[l, c]
// grid.x = work item (m, q, tile), grid.y = column tile; clusters along y
// ===========================================================================
template <bool M2A>
__global__ void __launch_bounds__(256, 1)
k_leg_tc(const void* __restrict__ src, void* __restrict__ dst, TcArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcShared& sh = *reinterpret_cast<TcShared*>(smem + NST * STAGE_BYTES + 2 * STG_BYTES);
    const int4 w = a.work[blockIdx.x];
    const int m = w.x, q = w.y, tile = w.z, ckb = w.w;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t crank = cluster_ctarank(), csize = cluster_nctarank();
    const long long c0 = (long long)blockIdx.y * TC_M;
    const int l_first = m + q;
    const int nl = (a.lmax >= l_first) ? (a.lmax - l_first) / 2 + 1 : 0;   // l rows of slot q
    const int n0 = tile * TC_N;                                         // first lambda row of the tile
    const int nrows = M2A ? min(TC_N, nl - n0) : min(TC_N, a.R - n0);
    const int K = M2A ? a.R : nl;
    const int nch = (K + KC - 1) / KC;
    const int npieces = (nrows + PR - 1) / PR;
    const int nmma = (nrows + 15) & ~15;
    const uint32_t idesc = idesc_f16(TC_M, nmma);
    const long long qstride = (long long)a.R * a.ncol;

    for (int r = tid; r < TC_N; r += blockDim.x) {
        if (M2A) {
            if (r < nrows) {
                const int l = l_first + 2 * (n0 + r);
                const long long ci = a_idx(a.lmax, l, m);
                sh.cA[r] = a.nA[ci];
                sh.cB[r] = a.nB[ci];
                sh.rowexp[r] = quantum_exp(a.rowmax[ci], a.Q);
                // c_l * dsigma applied once per output in double-float, so its
                // rounding is not a coherent error along the row
                const double f = a.nc64[ci] * (m == 0 ? a.fs0 : a.fs1);
                const float fh = (float)f;
                sh.rfac[r] = make_float2(fh, (float)(f - (double)fh));
            } else {
                sh.cA[r] = 0.0; sh.cB[r] = 0.0; sh.rowexp[r] = 0; sh.rfac[r] = make_float2(0.0f, 0.0f);
            }
        } else {
            sh.rowexp[r] = (r < nrows) ? quantum_exp(a.pairmax[((long long)m * 2 + q) * a.R + n0 + r], a.Q) : 0;
        }
    }
    for (int c = tid; c < TC_M; c += blockDim.x) {
        const long long cg = c0 + c;
        sh.colexp[c] = (cg < a.ncol) ? quantum_exp(a.colmax[((long long)m * 2 + q) * a.ncol + cg], a.Q) : 0;
    }
    if (tid == 0) {
        for (int s = 0; s < NST; s++) {
            mbar_init(&sh.full[s], 4 + npieces);
            mbar_init(&sh.empty[s], csize);
        }
        mbar_init(&sh.accf, 1);
        mbar_init(&sh.cdone, 1);
        mbar_init(&sh.cfree, 4);
        for (int b = 0; b < 2; b++) mbar_init(&sh.sfull[b], 1);
        sh.released = NST - 1;
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(&sh.tmem, 512);
    tc_fence_before();
    cluster_sync();            // barriers of every CTA initialised before any remote arrival
    tc_fence_after();
    const uint32_t tmem = sh.tmem;
    const uint32_t smem_base = smem_u32(smem);

    if (warp == 0) {
        // ---------------- MMA issuer ----------------
        if (lane == 0 && nch > 0) {
            const uint16_t mask = (uint16_t)((1u << csize) - 1u);
            for (int kc = 0; kc < nch; kc++) {
                const int s = kc % NST;
                const uint32_t u = kc / NST;
                if (!mbar_wait_cl(&sh.full[s], u & 1, a.err, 1)) break;
                tc_fence_after();
                issue_main(tmem, smem_base + s * STAGE_BYTES, idesc, kc == 0);
                // the correction accumulators of chunk kc - 1 must have been drained
                if (kc >= 1 && !mbar_wait_cl(&sh.cfree, (kc - 1) & 1, a.err, 5)) break;
                tc_fence_after();
                issue_corr(tmem, smem_base + s * STAGE_BYTES, idesc, kc == 0);
                umma_commit_mc(&sh.empty[s], mask);
                umma_commit(&sh.cdone);
            }
            umma_commit(&sh.accf);
        }
    } else if (warp < 4) {
        // ---------------- lambda pieces ----------------
        // A piece is computed into registers first (32 recurrence steps, ~one
        // FP64 FMA latency each) and only then does the warp wait for its stage
        // to be released, so the recurrence overlaps the MMAs of earlier chunks.
        const int total = nch * npieces;
        for (int g = (int)crank + (int)csize * (warp - 1); g < total; g += (int)csize * 3) {
            const int kc = g / npieces, j = g - kc * npieces;
            const int s = kc % NST;
            float hb[PR], lb[PR];
            int prow;                                   // row of the B tile this lane writes (alm2map)
            if (M2A) {
                // lane = ring pair (k), walking the 32 l rows of piece j
                const int p = kc * KC + lane;
                double cur = 0.0, prev = 0.0, x2 = 0.0;
                int E = 0;
                const bool live = p < a.R;
                if (live) {
                    const long long ci = (long long)(ckb + (n0 + j * PR) / CK_ROWS) * a.R + p;
                    const double2 v = a.ck[ci];
                    cur = v.x; prev = v.y;
                    E = a.ck_exp[ci];
                    const double x = a.pairs[p].x;
                    x2 = x * x;
                }
                const int rn = min(PR, nrows - j * PR);  // rows of this piece (warp-uniform)
                double tn = fma(sh.cA[j * PR], x2, sh.cB[j * PR]);
#pragma unroll
                for (int i = 0; i < PR; i++) {
                    hb[i] = 0.0f; lb[i] = 0.0f;
                    if (i < rn) {
                        const int r = j * PR + i;
                        if (live) f64_split_scaled(cur, E - sh.rowexp[r], hb[i], lb[i]);
                        const double t = tn;            // coefficient FMA one step ahead
                        if (i + 1 < rn) tn = fma(sh.cA[r + 1], x2, sh.cB[r + 1]);
                        const double nxt = fma(t, cur, prev);
                        prev = cur;
                        cur = nxt;
                        rescale(cur, prev, E);
                    }
                }
                prow = 0;
            } else {
                // lane = ring pair (row), walking the 32 l of stage kc; the
                // coefficients of those 32 l are loaded once (lane k holds l_k)
                // and broadcast with shuffles
                const int r = j * PR + lane;
                const int p = n0 + r;
                const bool live = r < nrows;
                double cur = 0.0, prev = 0.0, x2 = 0.0;
                int E = 0, pe = 0;
                if (live) {
                    const long long ci = (long long)(ckb + kc * KC / CK_ROWS) * a.R + p;
                    const double2 v = a.ck[ci];
                    cur = v.x; prev = v.y;
                    E = a.ck_exp[ci];
                    const double x = a.pairs[p].x;
                    x2 = x * x;
                    pe = sh.rowexp[r];
                }
                double cAk = 0.0, cBk = 0.0;
                float2 cck = make_float2(0.0f, 0.0f);
                {
                    const int k = kc * KC + lane;
                    if (k < K) {
                        const long long ci = a_idx(a.lmax, l_first + 2 * k, m);
                        cAk = a.nA[ci]; cBk = a.nB[ci]; cck = a.nc2[ci];
                    }
                }
                const int kn = min(KC, K - kc * KC);    // valid l of this chunk (warp-uniform)
                double tn = fma(__shfl_sync(0xffffffffu, cAk, 0), x2, __shfl_sync(0xffffffffu, cBk, 0));
#pragma unroll
                for (int i = 0; i < PR; i++) {
                    hb[i] = 0.0f; lb[i] = 0.0f;
                    const float c0_ = __shfl_sync(0xffffffffu, cck.x, i);
                    const float c1_ = __shfl_sync(0xffffffffu, cck.y, i);
                    const double cAn = __shfl_sync(0xffffffffu, cAk, (i + 1) & (PR - 1));
                    const double cBn = __shfl_sync(0xffffffffu, cBk, (i + 1) & (PR - 1));
                    if (i < kn) {
                        float h = 0.0f, lo = 0.0f;
                        if (live) f64_split_scaled(cur, E - pe, h, lo);
                        const float p1 = h * c0_;               // lambda = c_l mu in double-float
                        hb[i] = p1;
                        lb[i] = fmaf(h, c0_, -p1) + (h * c1_ + lo * c0_);
                        const double t = tn;
                        if (i + 1 < kn) tn = fma(cAn, x2, cBn);
                        const double nxt = fma(t, cur, prev);
                        prev = cur;
                        cur = nxt;
                        rescale(cur, prev, E);
                    }
                }
                prow = r;
            }
            // A warp's pieces can be several chunks apart, more than the parity
            // of the stage barrier can tell apart, so it waits on the monotonic
            // count of released chunks that the data warps publish instead.
            if (!__all_sync(0xffffffffu, wait_counter(&sh.released, kc, a.err, 2))) break;
            uint8_t* B = smem + s * STAGE_BYTES + 3 * A_PLANE;
            if (M2A) {
#pragma unroll
                for (int i = 0; i < PR; i++) {
                    float q0, q1, q2;
                    slice3d(hb[i], lb[i], q0, q1, q2);
                    const uint32_t off = sw64_off(j * PR + i, lane);
                    *reinterpret_cast<__half*>(B + off) = __float2half_rn(q0);
                    *reinterpret_cast<__half*>(B + B_PLANE + off) = __float2half_rn(q1);
                    *reinterpret_cast<__half*>(B + 2 * B_PLANE + off) = __float2half_rn(q2);
                }
            } else {
#pragma unroll
                for (int jj = 0; jj < KC / 8; jj++) {
                    float hv[8], lv[8];
#pragma unroll
                    for (int i = 0; i < 8; i++) { hv[i] = hb[jj * 8 + i]; lv[i] = lb[jj * 8 + i]; }
                    put3x8(B, B_PLANE, prow, jj, hv, lv);
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            // lane d sends the piece to CTA d of the cluster (its own CTA: a plain arrival)
            if (lane < (int)csize) {
                const uint32_t d = (uint32_t)lane;
                if (d == crank) {
                    mbar_arrive(&sh.full[s]);
                } else {
                    const uint32_t src0 = smem_u32(B) + j * PIECE_BYTES;
                    const uint32_t fb = mapa_shared(smem_u32(&sh.full[s]), d);
                    mbar_arrive_expect_tx_cl(fb, 3 * PIECE_BYTES);
#pragma unroll
                    for (int b = 0; b < 3; b++) {
                        const uint32_t sa = src0 + b * B_PLANE;
                        bulk_copy_s2cluster(mapa_shared(sa, d), sa, PIECE_BYTES, fb);
                    }
                }
            }
        }
    } else {
        // ---------------- data slices: one map column per thread ----------------
        const int t = tid - 128;
        const long long cg = c0 + t;
        const bool cok = cg < a.ncol;
        const int ce = sh.colexp[t];
        const int quarter = warp & 3;                 // TMEM lanes 32 quarter .. + 31
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        bool dok = true;
        // Move chunk c's corrections into the 2^-12 count and hand the
        // accumulators back to the MMA. Per chunk |ex| <= 32 Q (1 + 2^-11) and
        // |sm| < 10 + Q / 128, so the count stays below 2^12 (K Q (1 + 2^-11) +
        // 11 nch) < 2^31 for K Q^2 <= 2^24 and K <= 8192.
        // (A rolled loop: this runs once per chunk between other code, and a
        // short body stays in the instruction cache.)
        auto drain_cols = [&](uint32_t (&ve)[32], uint32_t (&vs)[32], uint32_t (&vh)[32], int n, bool first) {
#pragma unroll
            for (int i = 0; i < 32; i++) {
                if (i < n) {
                    // ex: a multiple of 2^-12 below 2^12, so ex 2^12 is an exact integer
                    const int ne = __float2int_rn(__uint_as_float(ve[i]) * 4096.0f);
                    // sm to the nearest multiple of 2^-12 (|sm| 2^12 < 2^22) and its exact residual
                    const float v = __uint_as_float(vs[i]);
                    const float y = fmaf(v, 4096.0f, 12582912.0f);
                    const int ns = __float_as_int(y) - 0x4B400000;
                    vs[i] = __float_as_uint(fmaf(y - 12582912.0f, -1.0f / 4096.0f, v));
                    vh[i] = (uint32_t)((first ? 0 : (int)vh[i]) + ne + ns);
                }
            }
        };
        auto drain = [&](int c) {
            dok = dok && __all_sync(0xffffffffu, mbar_wait_cl(&sh.cdone, c & 1, a.err, 6));
            tc_fence_after();
            uint32_t ve[32], vs[32], vh[32];
#pragma unroll 1
            for (int g = 0; g + 32 <= nmma; g += 32) {
                tmem_ld32(tl + ACC_EX + g, ve);
                tmem_ld32(tl + ACC_SM + g, vs);
                tmem_ld32(tl + ACC_HX + g, vh);
                tmem_wait_ld();
                drain_cols(ve, vs, vh, 32, c == 0);
                tmem_st32(tl + ACC_SM + g, vs);
                tmem_st32(tl + ACC_HX + g, vh);
            }
            if (nmma & 16) {                          // a last group of 16 columns
                const int g = nmma - 16;
                uint32_t e16[16], s16[16], h16[16];
                tmem_ld16(tl + ACC_EX + g, e16);
                tmem_ld16(tl + ACC_SM + g, s16);
                tmem_ld16(tl + ACC_HX + g, h16);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; i++) { ve[i] = e16[i]; vs[i] = s16[i]; vh[i] = h16[i]; }
                drain_cols(ve, vs, vh, 16, c == 0);
#pragma unroll
                for (int i = 0; i < 16; i++) { s16[i] = vs[i]; h16[i] = vh[i]; }
                tmem_st16(tl + ACC_SM + g, s16);
                tmem_st16(tl + ACC_HX + g, h16);
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.cfree);
        };
        // Raw data: K row kc of the CTA's 128 columns is contiguous in global
        // memory (T[m][q][p][c] for map2alm, the transposed a_lm A2[l,m][c] for
        // alm2map, both FP32 hi/lo pairs), so one thread moves each chunk with
        // 32 bulk copies (1 KB each) into staging buffer kc & 1.
        const int ncv = (int)max(0ll, min((long long)TC_M, a.ncol - c0));   // valid columns of the tile
        const float2* raw = (const float2*)src;
        auto fetch = [&](int c) {
            const int b = c & 1;
            const int i1 = min(KC, K - c * KC);
            const uint32_t rowb = (uint32_t)ncv * 8u;
            mbar_arrive_expect_tx(&sh.sfull[b], rowb * (uint32_t)max(i1, 0));
            if (rowb == 0) return;
            const uint32_t dst = smem_u32(smem + NST * STAGE_BYTES + b * STG_BYTES);
            for (int i = 0; i < i1; i++) {
                const int k = c * KC + i;
                const long long row = M2A ? ((long long)m * 2 + q) * a.R + k : a_idx(a.lmax, l_first + 2 * k, m);
                bulk_copy_g2s(dst + i * STG_ROW, raw + row * a.ncol + c0, rowb, &sh.sfull[b]);
            }
        };
        const bool issuer = (warp == 4 && lane == 0);
        if (issuer) {
            if (nch > 0) fetch(0);
            if (nch > 1) fetch(1);
        }
        // the quantum 2^ce as an FP32 factor (exact scaling)
        const float csc = __int_as_float((127 - ce) << 23);
        // (a wait that gives up turns dok off; the loop still runs to the end so
        // that all four data warps keep meeting at the named barrier)
        // (the stage of chunk kc is free: one of the first NST, or released at
        // the end of iteration kc - 1)
        for (int kc = 0; kc < nch; kc++) {
            const int s = kc % NST;
            if (dok) dok = __all_sync(0xffffffffu, mbar_wait(&sh.sfull[kc & 1], (kc >> 1) & 1, a.err, 8));
            if (dok) {
                const float2* stg =
                    reinterpret_cast<const float2*>(smem + NST * STAGE_BYTES + (kc & 1) * STG_BYTES) + t;
                const int kv = K - kc * KC;             // valid rows of this chunk
                uint8_t* A = smem + s * STAGE_BYTES;
#pragma unroll 1
                for (int jj = 0; jj < KC / 8; jj++) {
                    float hv[8], lv[8];
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int r = jj * 8 + i;
                        float2 x = make_float2(0.0f, 0.0f);
                        if (cok && r < kv) x = stg[r * TC_M];
                        hv[i] = x.x * csc;
                        lv[i] = x.y * csc;
                    }
                    put3x8(A, A_PLANE, t, jj, hv, lv);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.full[s]);
            }
            // all four data warps are done with staging buffer kc & 1: refill it
            named_bar_sync(1, 128);
            if (dok && issuer && kc + 2 < nch) fetch(kc + 2);
            // once every CTA of the cluster has consumed the previous use of the
            // stage of chunk kc + 1, release it to the lambda warps
            const int kn = kc + 1;
            if (dok && kn < nch && kn >= NST) {
                dok = __all_sync(0xffffffffu, mbar_wait_cl(&sh.empty[kn % NST], (kn / NST - 1) & 1, a.err, 3));
                if (dok && issuer) publish_counter(&sh.released, kn);
            }
            if (kc >= 1 && dok) drain(kc - 1);
        }
        // Tail: wait until every CTA of the cluster has consumed the last use of
        // each stage. All their MMA commits then have arrived on this CTA's
        // barriers, so none can land after it exits. (These waits continue the
        // sequential phase walk of the loop above.)
        for (int kc = nch; kc < nch + NST && dok; kc++) {
            const int s = kc % NST;
            const uint32_t u = kc / NST;
            if (u >= 1)
                dok = __all_sync(0xffffffffu, mbar_wait_cl(&sh.empty[s], (u - 1) & 1, a.err, 7));
        }
        if (dok && nch >= 1) drain(nch - 1);

        // ---------------- epilogue: out = (main + ex + sm) * scales ----------------
        const bool ok = dok && ((nch == 0) || __all_sync(0xffffffffu, mbar_wait_cl(&sh.accf, 0, a.err, 4)));
        tc_fence_after();
#pragma unroll
        for (int g = 0; g < TC_N / 32; g++) {
            if (g * 32 >= nmma) continue;
            uint32_t v0[32], vh[32], vr[32];
            if (nch > 0) {
                tmem_ld32(tl + g * 32, v0);
                tmem_ld32(tl + ACC_HX + g * 32, vh);
                tmem_ld32(tl + ACC_SM + g * 32, vr);
                tmem_wait_ld();
            }
            if (!ok || !cok) continue;
            if (M2A) {
                double* alm = (double*)dst;
                const long long mp = cg >> 1;
                const int reim = (int)(cg & 1);
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const int r = g * 32 + i;
                    if (r < nrows) {
                        // main + the count (integer and 2^-12 parts) + the residual as
                        // an FP32 pair (two TwoSums), times c_l f (hi/lo)
                        const float x0 = __uint_as_float(v0[i]);
                        const int hc = (int)vh[i];
                        const float eh = (float)(hc >> 12);                        // exact, < 2^19
                        const float el = (float)(hc & 4095) * (1.0f / 4096.0f);    // exact
                        const float s1 = x0 + eh;
                        const float b1 = s1 - x0;
                        const float e1 = (x0 - (s1 - b1)) + (eh - b1);             // exact (an integer)
                        const float t1 = (el + e1) + __uint_as_float(vr[i]);
                        const float sm = s1 + t1;
                        const float bb = sm - s1;
                        const float er = (s1 - (sm - bb)) + (t1 - bb);
                        const float2 F = sh.rfac[r];
                        const float p1 = __fmul_rn(sm, F.x);
                        const float lo = fmaf(sm, F.x, -p1) + er * F.x + sm * F.y;
                        double v = f32_to_f64(p1) + f32_to_f64(lo);            // final FP64 accumulation
                        v = ldexp_fast(v, sh.rowexp[r] + ce);
                        if (m == 0 && reim) v = 0.0;
                        const int l = l_first + 2 * (n0 + r);
                        alm[(mp * a.nalm + a_idx(a.lmax, l, m)) * 2 + reim] = v;
                    }
                }
            } else {
                float* Gq = (float*)dst + ((long long)m * 2 + q) * qstride + cg;
                const float sc = (m == 0) ? a.s0 : a.s1;
#pragma unroll
                for (int i = 0; i < 32; i++) {
                    const int r = g * 32 + i;
                    if (r < nrows) {
                        float gv = 0.0f;
                        if (nch > 0) {
                            const int hc = (int)vh[i];
                            const float x = (__uint_as_float(v0[i]) + (float)(hc >> 12)) +
                                            ((float)(hc & 4095) * (1.0f / 4096.0f) + __uint_as_float(vr[i]));
                            gv = sc * ldexpf_fast(x, sh.rowexp[r] + ce);
                        }
                        Gq[(long long)(n0 + r) * a.ncol] = gv;
                    }
                }
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    cluster_sync();            // no CTA leaves while others may still copy into it
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ===========================================================================
// plan-time walk: recurrence checkpoints every 32 rows of each (m, q) chain,
// the per-row maxima over ring pairs (map2alm quanta) and the per-pair maxima
// over l (alm2map quanta). grid = (mmax+1, 2), threads over ring pairs.
// ===========================================================================
__global__ void __launch_bounds__(256)
k_split_tables(TcArgs a, const int* __restrict__ ck_base, double2* __restrict__ ck, int* __restrict__ ck_exp,
               const double* __restrict__ seed_mant, const int* __restrict__ seed_exp,
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
            const long long si = ((long long)m * 2 + q) * a.R + p;
            cur = seed_mant[si];
            E = seed_exp[si];
            const double x = a.pairs[p].x;
            x2 = x * x;
        }
        float pmax = 0.0f;
        for (int row = 0; row < nrows; row++) {
            if (valid && (row % CK_ROWS) == 0) {
                const long long ci = (long long)(base + row / CK_ROWS) * a.R + p;
                ck[ci] = make_double2(cur, prev);
                ck_exp[ci] = E;
            }
            const int l = l_first + 2 * row;
            const long long ci = a_idx(a.lmax, l, m);
            float v = 0.0f, vmu = 0.0f;
            if (valid) {
                // |mu 2^E| for the map2alm row quanta; |lambda| = |c_l mu 2^E| for alm2map
                vmu = fabsf(f64_to_f32_scaled(cur, E));
                v = vmu * fabsf(a.nc[ci]);
                const double t = fma(a.nA[ci], x2, a.nB[ci]);
                const double nxt = fma(t, cur, prev);
                prev = cur;
                cur = nxt;
                rescale(cur, prev, E);
            }
            pmax = fmaxf(pmax, v * 1.0000003f);
            // max over the ring pairs of this warp, then one atomic per warp
            float wv = vmu * 1.0000003f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wv = fmaxf(wv, __shfl_xor_sync(0xffffffffu, wv, o));
            if ((threadIdx.x & 31) == 0 && wv > 0.0f) atomicMax(rowmax_bits + ci, __float_as_uint(wv));
        }
        if (valid) pairmax[((long long)m * 2 + q) * a.R + p] = pmax;
    }
}

// ===========================================================================
// alm2map input preparation: the a_lm of the batch, transposed to
// A2[idx(l, m)][col] (col = (map, component, Re/Im)) as FP32 hi/lo pairs, so
// each K row of the contraction is contiguous, plus the column maxima per
// (m, slot q, col) for the quanta. Block: 64 l x 32 map-components of one m.
// grid = (ceil((lmax+1)/64), mmax+1, ceil(nmaps ncomp / 32))
// ===========================================================================
constexpr int PREP_L = 64, PREP_M = 32;
__global__ void __launch_bounds__(256)
k_alm_prep(const double* __restrict__ alm, float2* __restrict__ A2, unsigned int* __restrict__ colmax,
           int lmax, long long nalm, long long ncol)
{
    __shared__ double2 tile[PREP_L][PREP_M + 1];
    __shared__ float cmx[2][2 * PREP_M];
    const int m = blockIdx.y;
    const int l0 = m + blockIdx.x * PREP_L;
    if (l0 > lmax) return;
    const long long nmc = ncol / 2;
    const long long mp0 = (long long)blockIdx.z * PREP_M;
    const int tid = threadIdx.x;
    if (tid < 4 * PREP_M) cmx[tid / (2 * PREP_M)][tid % (2 * PREP_M)] = 0.0f;
    const long long base = a_idx(lmax, l0, m);
    for (int e = tid; e < PREP_L * PREP_M; e += blockDim.x) {
        const int j = e / PREP_L, li = e % PREP_L;            // consecutive threads: consecutive l
        double2 v = make_double2(0.0, 0.0);
        if (l0 + li <= lmax && mp0 + j < nmc) {
            v = reinterpret_cast<const double2*>(alm)[(mp0 + j) * nalm + base + li];
            if (m == 0) v.y = 0.0;
        }
        tile[li][j] = v;
    }
    __syncthreads();
    const int cc = tid % (2 * PREP_M);                        // column within the block (fixed per thread)
    float mx[2] = {0.0f, 0.0f};
    for (int e = tid; e < PREP_L * 2 * PREP_M; e += blockDim.x) {
        const int li = e / (2 * PREP_M);
        const long long col = mp0 * 2 + cc;
        if (l0 + li > lmax || col >= ncol) continue;
        const double2 v = tile[li][cc >> 1];
        float h, lo;
        f64_split_scaled((cc & 1) ? v.y : v.x, 0, h, lo);
        A2[(base + li) * ncol + col] = make_float2(h, lo);
        mx[(l0 + li - m) & 1] = fmaxf(mx[(l0 + li - m) & 1], fabsf(h));
    }
    for (int qq = 0; qq < 2; qq++)
        if (mx[qq] > 0.0f) atomicMax(reinterpret_cast<unsigned int*>(&cmx[qq][cc]), __float_as_uint(mx[qq]));
    __syncthreads();
    if (tid < 4 * PREP_M) {
        const int qq = tid / (2 * PREP_M), c = tid % (2 * PREP_M);
        const long long col = mp0 * 2 + c;
        const float v = cmx[qq][c];
        if (col < ncol && v > 0.0f) atomicMax(colmax + ((long long)m * 2 + qq) * ncol + col, __float_as_uint(v));
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static TcArgs make_tc(const sht_plan* p, int nmaps, const float* colmax, float Q)
{
    TcArgs a;
    a.pairs = p->t.pairs;
    a.nA = p->s.nA; a.nB = p->s.nB; a.nc = p->s.nc; a.nc64 = p->s.nc64; a.nc2 = p->s.nc2;
    a.ck = p->s.ck; a.ck_exp = p->s.ck_exp;
    a.rowmax = (const float*)p->s.rowmax_bits;
    a.pairmax = p->s.pairmax;
    a.colmax = colmax;
    a.err = p->s.err;
    a.lmax = p->lmax; a.mmax = p->mmax; a.R = p->R;
    a.ncol = ncols(p, nmaps); a.nalm = p->nalm;
    a.Q = Q;
    a.fs0 = a.fs1 = 1.0;
    a.s0 = a.s1 = 1.0f;
    a.work = nullptr;
    return a;
}

// largest cluster: 8 (portable limit), or SHT_MAX_CLUSTER from the environment
static int max_cluster()
{
    static int mc = [] {
        const char* e = std::getenv("SHT_MAX_CLUSTER");
        int v = e ? std::atoi(e) : MAX_CLUSTER;
        return std::max(1, std::min(v, MAX_CLUSTER));
    }();
    return mc;
}

// cluster size along the column tiles: all of them up to the largest size,
// else the size in [largest/2, largest] that wastes the fewest padded tiles
// (ties: the larger)
static int pick_cluster(long long ntiles)
{
    const int cmax = max_cluster();
    if (ntiles <= cmax) return (int)std::max(1ll, ntiles);
    int best = cmax;
    long long waste = (cmax - ntiles % cmax) % cmax;
    for (int c = cmax - 1; c >= std::max(1, cmax / 2); c--) {
        long long wc = (c - ntiles % c) % c;
        if (wc < waste) { waste = wc; best = c; }
    }
    return best;
}

template <bool M2A>
static cudaError_t launch_tc(const sht_plan* p, int nwork, const void* src, void* dst,
                             const TcArgs& a, const char* name, cudaStream_t st)
{
    (void)p;
    auto kern = k_leg_tc<M2A>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC);
    if (e != cudaSuccess) return e;
    const long long ntiles = (a.ncol + TC_M - 1) / TC_M;
    int C = pick_cluster(ntiles);
    prof_start(name, st);
    for (;;) {
        const long long gy = (ntiles + C - 1) / C * C;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)nwork, (unsigned)gy, 1);
        cfg.blockDim = dim3(256, 1, 1);
        cfg.dynamicSmemBytes = SMEM_TC;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 1;
        at[0].val.clusterDim.y = (unsigned)C;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, kern, src, dst, a);
        if (e == cudaSuccess || C == 1) break;
        (void)cudaGetLastError();      // clear a failed cluster launch, retry smaller
        C = std::max(1, C / 2);
    }
    prof_stop(st);
    count_launch();
    return e;
}

cudaError_t launch_legendre_m2a_tc(const sht_plan* p, const float2* T, const float* colmax, double* alm,
                                   int nmaps, double fs0, double fs1, cudaStream_t st)
{
    if (p->s.nwork_m2a == 0) return cudaSuccess;
    TcArgs a = make_tc(p, nmaps, colmax, p->s.Q_m2a);
    a.fs0 = fs0; a.fs1 = fs1;
    a.work = p->s.work_m2a;
    return launch_tc<true>(p, p->s.nwork_m2a, T, alm, a, "k_leg_m2a_tc", st);
}

cudaError_t launch_legendre_a2m_tc(const sht_plan* p, const float2* A2, const float* colmax, float* G,
                                   int nmaps, float s0, float s1, cudaStream_t st)
{
    if (p->s.nwork_a2m == 0) return cudaSuccess;
    TcArgs a = make_tc(p, nmaps, colmax, p->s.Q_a2m);
    a.s0 = s0; a.s1 = s1;
    a.work = p->s.work_a2m;
    return launch_tc<false>(p, p->s.nwork_a2m, A2, G, a, "k_leg_a2m_tc", st);
}

cudaError_t launch_alm_prep(const sht_plan* p, const double* alm, float2* A2, unsigned int* colmax, int nmaps,
                            cudaStream_t st)
{
    const long long nc = ncols(p, nmaps);
    cudaError_t e = cudaMemsetAsync(colmax, 0, (size_t)(p->mmax + 1) * 2 * nc * sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((p->lmax + PREP_L) / PREP_L), (unsigned)(p->mmax + 1),
              (unsigned)((nc / 2 + PREP_M - 1) / PREP_M));
    prof_start("k_alm_prep", st);
    k_alm_prep<<<grid, 256, 0, st>>>(alm, A2, colmax, p->lmax, p->nalm, nc);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t run_split_tables(sht_plan* p, const int* d_ck_base)
{
    TcArgs a = make_tc(p, 1, nullptr, p->s.Q_m2a);
    dim3 grid((unsigned)(p->mmax + 1), 2);
    k_split_tables<<<grid, 256>>>(a, d_ck_base, p->s.ck, p->s.ck_exp, p->t.seed_mant, p->t.seed_exp,
                                  p->s.rowmax_bits, p->s.pairmax);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

int split_row_tile() { return TC_N; }
int split_ck_rows() { return CK_ROWS; }
int split_col_tile() { return TC_M; }

}  // namespace sht
