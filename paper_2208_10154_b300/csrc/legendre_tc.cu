// legendre_tc.cu -- split-precision Legendre contraction on the B300 tensor
// cores (tcgen05.mma kind::f16, FP16 operands, FP32 accumulation in TMEM).
//
// The paper's per-m GEMMs (Sec. 2.2 equ:matrix form: A_m = P_m T_m and
// T_m = P_m^t A_m) are evaluated per (m, slot q) with lambda generated on the
// fly by the normalised recurrence (same-parity two-step form for spin 0), run
// in double-float (FP32 pair) arithmetic with scaled exponents from FP64
// checkpoints every 32 rows, so the Legendre matrix never lands in HBM.
//
// Orientation. The MMA's M dimension (TMEM lanes) is 128 map columns
// (map, component, Re/Im); its N dimension is the lambda side: l rows for
// map2alm (N = the rows left in the l tile, rounded up to 16, so short tiles at
// high m cost only what they hold) and ring pairs for alm2map. K is the
// contraction: ring pairs (map2alm) or l (alm2map).
//
// Accuracy. Every operand x is written, per row or column, in units of a
// power-of-two quantum u with |x/u| <= Q (Q (Q + 1) K + 12 K / 32 <= 2^24,
// Q <= 127) as four FP16 slices q + r0 + r1 + 2^-12 r2s (tc::slice4d: integer,
// a multiple of 2^-G, the next 11 bits and the 11 after, ~2^-(G+24) of u). Ten
// products per K step, in four TMEM accumulators:
//     main = sum q q'                              integers: exact
//     ex   = q r0' + r0 q'                         multiples of 2^-G below 2^(24-G)
//                                                  per span of K: exact
//     sm   = q r1' + r1 q' + r0 r0' + r0 r1' + r1 r0'        small per span
//     fn   = q r2s' + r2s q'                       (2^12 times their value)
// The TMEM accumulator truncates toward zero on every MMA, so a sum that is not
// exact picks up an error that grows with its magnitude and length. After each
// span the drain warps fold the integer parts of ex and sm into main (exact:
// the bound above keeps main below 2^24) and leave the fractional parts plus
// 2^-12 fn (all below 1) in sm as the start of the next span, so sm never
// holds more than one span's worth; ex and fn restart with every span.
// Dropped: products of two residual slices beyond r0 r1' (< 2^-2G u u').
// Spans: spin-2 map2alm 64 of K (G = 11: the truncation of the sm sums is its
// largest error term, and its B component is a difference of E-sized terms);
// spin-0 map2alm and alm2map 128 of K (G = 10: half the drains; spin-0
// map2alm stays near 1e-8 of the RMS, alm2map's error is set by the FP32 ring
// spectra).
//
// Cluster sharing of lambda. The recurrence is a serial chain per ring pair,
// so the CTAs of a thread-block cluster, which work on
// the same (m, q, tile) for different column tiles, split the lambda work:
// lambda for one stage is cut into 32-row pieces, each produced by one warp of
// one CTA into its shared scratch and written to that warp's own slot of a
// static device array (g_lam_slots, in L2); once the stage is released, the
// warp multicasts the piece from that slot into the stage of every CTA of the
// cluster with one cp.async.bulk ... .multicast::cluster per plane, completing
// on each CTA's own stage barrier. The multicast source is always this GPU's
// own g_lam_slots array, and the split form runs only in single-GPU processes.
// Each CTA's MMA completion is multicast to the "stage free" barriers of all
// CTAs of the cluster.
//
// Ring optimisation (Sec. 3.1). Order m contracts only the ring pairs from
// pfirst[m] (a multiple of 32; the pairs before it hold |lambda_lm| < 1e-30
// for every l): map2alm's K and alm2map's ring-pair tiles start there.
//
// Data operand. A separate pass (k_slice) writes, per 32-wide chunk of K and
// column tile, the four slice planes of the data as the exact 32 KB image of
// the stage's A operand; the contraction fetches it with one bulk copy per
// chunk, so no thread of the contraction touches the data.
//
// CTA: 256 threads, one per SM (192 KB of pipeline stages, 512 TMEM columns).
//   warp 0       TMEM allocation; lane 0 issues the MMAs, the stage
//                releases and the data copies, in one non-blocking event loop
//   warps 1-3    lambda pieces (32 ring pairs x 32 rows / steps each; 8 KB
//                of shared scratch per warp)
//   warps 4-7    the drains of the correction accumulators, then the
//                epilogue with warps 0-3
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "tc.cuh"

namespace sht {

using namespace tc;

constexpr int TC_M = 128;                        // map columns per CTA (MMA M)
constexpr int TC_N = 128;                        // lambda rows per CTA (MMA N, max)
constexpr int KC = 32;                           // K per pipeline stage (2 MMA K-steps)
constexpr int NST = 3;                           // pipeline stages
constexpr int PR = 32;                           // rows per lambda piece
constexpr int NPL = 4;                           // FP16 slices per operand (q, r0, r1, r2s)
constexpr int A_PLANE = TC_M * KC * 2;           // 8 KB (data, one slice)
constexpr int B_PLANE = TC_N * KC * 2;           // 8 KB (lambda, one slice)
constexpr int PIECE_BYTES = PR * KC * 2;         // 2 KB of one B plane
constexpr int SCR_BYTES = NPL * PIECE_BYTES;      // 8 KB: one lambda piece (scratch per lambda warp)
constexpr int LAM_SM = 256;                      // SM ids covered by the L2 slots of the lambda pieces
constexpr int LAM_SLOTS = 4;                     // L2 slots per lambda warp (used round-robin)
constexpr int A_BYTES = NPL * A_PLANE;           // 32 KB: one chunk of the data operand
constexpr int STAGE_BYTES = NPL * (A_PLANE + B_PLANE);   // 64 KB
constexpr uint32_t ACC_EX = 128;                 // TMEM columns: exact corrections of one chunk
constexpr uint32_t ACC_SM = 256;                 //   small corrections (+ the residual of earlier chunks)
constexpr uint32_t ACC_FN = 384;                 //   products with r2s (2^12 times their value)
// chunks per drained span and the grid exponent G of the r0 slices: spin-2
// map2alm 64 of K with G = 11 (its error budget is the tightest), the others
// 128 of K with G = 10
template <bool M2A, bool S2> __host__ __device__ constexpr int span_chunks() { return (M2A && S2) ? 2 : 4; }
template <bool M2A, bool S2> __host__ __device__ constexpr int r0_grid() { return (M2A && S2) ? 11 : 10; }
constexpr int CK_ROWS = 32;                      // rows between recurrence checkpoints
constexpr int MAX_CLUSTER = 16;                 // non-portable above 8
constexpr int DEF_CLUSTER = 8;
constexpr int TC_THREADS = 256;                  // 8 warps (roles below)

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
    const int* pfirst;         // first ring pair contracted for order m (multiple of 32; null: 0)
    // spin 2: normalised Wigner recurrences, per s = +2 / -2 and packed (l, m):
    //   mu_l = (s2A x + s2B) mu_{l-1} - mu_{l-2},  s lambda_l = d_l mu_l (d_l the same for both s)
    const double* s2A[2];
    const double* s2B[2];
    const float2* s2d2;        // d_l as an FP32 hi/lo pair (alm2map applies it to lambda)
    const double* s2d64;       // d_l in FP64 (map2alm applies it per output row)
    // data operand: per chunk and column tile, the 32 KB shared-memory image of the
    // four FP16 slice planes (written by k_slice), at image chunk img_base[m][q] + chunk
    const uint8_t* img;
    const int* img_base;
    const int4* sunits;        // k_slice: (m, q, unit, image chunk of the unit)
    int* err;
    int lmax, mmax, R;
    int ntile;                 // column tiles of 128
    long long ncol, nalm;      // ncol: columns of the contraction (output columns)
    // spin-2 map2alm of one component: csel = 1 (E) or 2 (B) keeps, per map,
    // the two columns that form it; pcol = the columns of the data (row
    // stride of T and the column maxima). csel = 0: all columns, pcol = ncol.
    long long pcol;
    int csel;
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

// the four slice planes of 8 consecutive k, packed as FP16 pairs
template <int G>
__device__ __forceinline__ void pack4x8(const float (&v)[8], const float (&vl)[8], uint4 (&pk)[NPL])
{
    uint32_t w[NPL][4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float x0[NPL], x1[NPL];
        slice4d<G>(v[2 * i], vl[2 * i], x0[0], x0[1], x0[2], x0[3]);
        slice4d<G>(v[2 * i + 1], vl[2 * i + 1], x1[0], x1[1], x1[2], x1[3]);
#pragma unroll
        for (int b = 0; b < NPL; b++) w[b][i] = pack_h2(x0[b], x1[b]);
    }
#pragma unroll
    for (int b = 0; b < NPL; b++) pk[b] = make_uint4(w[b][0], w[b][1], w[b][2], w[b][3]);
}
// ... stored as the 16-byte chunk j of row `row` of each plane
__device__ __forceinline__ void store4x8(uint8_t* planes, int plane_bytes, int row, int j, const uint4 (&pk)[NPL])
{
    const uint32_t off = sw64_chunk(row, j);
#pragma unroll
    for (int b = 0; b < NPL; b++) *reinterpret_cast<uint4*>(planes + b * plane_bytes + off) = pk[b];
}
template <int G>
__device__ __forceinline__ void put4x8(uint8_t* planes, int plane_bytes, int row, int j, const float (&v)[8],
                                       const float (&vl)[8])
{
    uint4 pk[NPL];
    pack4x8<G>(v, vl, pk);
    store4x8(planes, plane_bytes, row, j, pk);
}

// lambda piece scratch (4 planes of 32 rows x 64 B, the swizzle of rows
// 32 j .. 32 j + 31 of a stage plane). map2alm: rows i0 .. i0 + 7 of K column
// `lane` (one FP16 per plane and row); alm2map: the 16-byte chunk jj (k = 8 jj
// .. 8 jj + 7) of row `lane`.
template <int G>
__device__ __forceinline__ void put_rows8(uint8_t* scr, int i0, int lane, const float (&hv)[8], const float (&lv)[8])
{
#pragma unroll
    for (int ii = 0; ii < 8; ii++) {
        float x[NPL];
        slice4d<G>(hv[ii], lv[ii], x[0], x[1], x[2], x[3]);
        const uint32_t w01 = pack_h2(x[0], x[1]), w23 = pack_h2(x[2], x[3]);
        const uint32_t off = sw64_off(i0 + ii, lane);
        *reinterpret_cast<uint16_t*>(scr + off) = (uint16_t)(w01 & 0xFFFFu);
        *reinterpret_cast<uint16_t*>(scr + PIECE_BYTES + off) = (uint16_t)(w01 >> 16);
        *reinterpret_cast<uint16_t*>(scr + 2 * PIECE_BYTES + off) = (uint16_t)(w23 & 0xFFFFu);
        *reinterpret_cast<uint16_t*>(scr + 3 * PIECE_BYTES + off) = (uint16_t)(w23 >> 16);
    }
}
__device__ __forceinline__ void put_chunk8(uint8_t* scr, int row, int jj, const float (&hv)[8], const float (&lv)[8])
{
    put4x8<r0_grid<false, false>()>(scr, PIECE_BYTES, row, jj, hv, lv);
}

// one stage (two MMA K-steps), A = data, B = lambda: main accumulates over the
// whole of K, sm over the whole of K on top of the residual the drain leaves in
// it (only the first stage restarts them); ex and fn restart at the first
// stage of each span.
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint32_t st_addr, uint32_t idesc, bool first,
                                            bool span_start)
{
    // descriptors as one base plus constant offsets (the start-address field
    // counts 16 bytes and shared memory stays below 2^18 bytes, so adding to
    // the 64-bit descriptor cannot carry out of that field)
    const uint64_t d0 = desc_sw64(st_addr);
    uint64_t A[NPL], B[NPL];
#pragma unroll
    for (int b = 0; b < NPL; b++) {
        A[b] = d0 + (uint64_t)((b * A_PLANE) >> 4);
        B[b] = d0 + (uint64_t)((NPL * A_PLANE + b * B_PLANE) >> 4);
    }
    const uint32_t ex = tmem + ACC_EX, sm = tmem + ACC_SM, fn = tmem + ACC_FN;
#pragma unroll
    for (int kk = 0; kk < 2; kk++) {
        const uint64_t o = (uint64_t)(kk * 32 >> 4);
        const uint32_t fresh = (span_start && kk == 0) ? 0u : 1u;
        const uint32_t keep = (first && kk == 0) ? 0u : 1u;
        umma_f16(tmem, A[0] + o, B[0] + o, idesc, keep);     // q q'
        umma_f16(ex, A[0] + o, B[1] + o, idesc, fresh);      // q r0'
        umma_f16(ex, A[1] + o, B[0] + o, idesc, 1u);         // r0 q'
        umma_f16(sm, A[0] + o, B[2] + o, idesc, keep);       // q r1'
        umma_f16(sm, A[2] + o, B[0] + o, idesc, 1u);         // r1 q'
        umma_f16(sm, A[1] + o, B[1] + o, idesc, 1u);         // r0 r0'
        umma_f16(sm, A[1] + o, B[2] + o, idesc, 1u);         // r0 r1'
        umma_f16(sm, A[2] + o, B[1] + o, idesc, 1u);         // r1 r0'
        umma_f16(fn, A[0] + o, B[3] + o, idesc, fresh);      // q r2s'
        umma_f16(fn, A[3] + o, B[0] + o, idesc, 1u);         // r2s q'
    }
}

// Lambda pieces travel through L2: a lambda warp writes its piece to its own
// slot (per SM id, warp and round-robin index) and multicasts it from there
// into the stage of every CTA of the cluster. Only one CTA of the contraction
// runs on an SM at a time (its shared memory), and a CTA exits only after
// every piece it sent has landed, so the slots of an SM are never shared.
__device__ __align__(128) uint8_t g_lam_slots[(size_t)LAM_SM * 3 * LAM_SLOTS * SCR_BYTES];

struct df { float h, l; };   // double-float value hi + lo

struct TcShared {
    uint64_t full[NST];        // stage filled: one arrival with the data copy; every byte completes as tx
    uint64_t empty[NST];       // stage consumed by the MMAs of every CTA of the cluster
    uint64_t accf;             // all MMAs of this CTA done
    uint64_t cdone;            // the correction accumulators hold a finished span
    uint64_t cfree;            // the span drained (4 drain warps)
    uint64_t tfree;            // alm2map: a tile's epilogue has read the accumulators (4 drain warps)
    int released;              // highest chunk whose stage is free in every CTA of the cluster
    int eok;                   // the data warps' waits all succeeded (read by the epilogue)
    uint32_t tmem;
    int colexp[TC_M];
    int rowexp[TC_N];          // quantum exponent per lambda row (l or ring pair)
    // map2alm: recurrence coefficients of the tile's rows. alm2map leaves them
    // unused and keeps the row scale factors of two tiles in their place
    // (float [2][TC_N], by tile parity).
    alignas(16) df cA2[TC_N], cB2[TC_N];
    float2 rfac[TC_N];         // map2alm: c_l * factor as an FP32 hi/lo pair
    int rowidx[TC_N];          // map2alm: packed index of the row's (l, m)
};
constexpr int SMEM_TC = NST * STAGE_BYTES + 3 * SCR_BYTES + (int)sizeof(TcShared) + 1024;
static_assert(SMEM_TC <= 227 * 1024, "shared memory of k_leg_tc");

// ---------------------------------------------------------------------------
// double-float ("hi + lo" FP32 pair) arithmetic for the lambda recurrences.
// An FP64 operation costs hundreds of cycles of latency on this GPU (a
// dependent FP64 recurrence step measured ~510 cycles), a double-float step
// ~70; the pair carries ~48 bits, far below what the FP16 slices keep
// (~2^-35 of the quantum). Error-free transformations: TwoSum (Knuth) and the
// FMA-based TwoProduct, written with non-contracting intrinsics.
// ---------------------------------------------------------------------------
__device__ __forceinline__ df df_norm(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return df{h, __fsub_rn(e, __fsub_rn(h, s))};
}
// an FP64 value as a pair (|v| < 2^127; parts below the FP32 normal range flush to 0)
__device__ __forceinline__ df df_of(double v)
{
    df r;
    f64_split_scaled(v, 0, r.h, r.l);
    return r;
}
__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df_norm(p, e);
}
// A x + B
__device__ __forceinline__ df df_axb(df A, df x, df B)
{
    const float p = __fmul_rn(A.h, x.h);
    float pe = __fmaf_rn(A.h, x.h, -p);
    pe = __fmaf_rn(A.h, x.l, pe);
    pe = __fmaf_rn(A.l, x.h, pe);
    const float s = __fadd_rn(p, B.h);
    const float bb = __fsub_rn(s, p);
    float e = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(B.h, bb));
    e = __fadd_rn(e, __fadd_rn(pe, B.l));
    return df_norm(s, e);
}
// one step of a three-term recurrence: (cur, prev) <- (t cur + sgn prev, cur), sgn = +-1
__device__ __forceinline__ void df_rec(df t, df& cur, df& prev, float sgn)
{
    const float m = __fmul_rn(t.h, cur.h);
    float me = __fmaf_rn(t.h, cur.h, -m);
    me = __fmaf_rn(t.h, cur.l, me);
    me = __fmaf_rn(t.l, cur.h, me);
    const float ph = sgn * prev.h, pl = sgn * prev.l;
    const float s = __fadd_rn(m, ph);
    const float bb = __fsub_rn(s, m);
    float e = __fadd_rn(__fsub_rn(m, __fsub_rn(s, bb)), __fsub_rn(ph, bb));
    e = __fadd_rn(e, __fadd_rn(me, pl));
    prev = cur;
    cur = df_norm(s, e);
}
// keep the pair in range: above 2^64 scale both values down by 2^64 (exact)
__device__ __forceinline__ void rescale_df(df& cur, df& prev, int& E)
{
    if (((__float_as_uint(cur.h) >> 23) & 0xFF) > 127 + 64) {
        cur.h *= 0x1p-64f; cur.l *= 0x1p-64f;
        prev.h *= 0x1p-64f; prev.l *= 0x1p-64f;
        E += 64;
    }
}
// a checkpoint (mu_l, mu_{l-1 or l-2}) 2^E as pairs scaled near 1 (E absorbs the scale)
__device__ __forceinline__ void ck_to_df(double2 v, df& cur, df& prev, int& E)
{
    const int ec = (__double2hiint(v.x) >> 20) & 0x7FF, ep = (__double2hiint(v.y) >> 20) & 0x7FF;
    const int eb = max(ec, ep);
    const int sc = (eb == 0) ? 0 : eb - 1023;
    f64_split_scaled(v.x, -sc, cur.h, cur.l);
    f64_split_scaled(v.y, -sc, prev.h, prev.l);
    E += sc;
}
// the pair times 2^k as (hi, lo) (flushes below the FP32 normal range)
__device__ __forceinline__ void df_scaled(df c, int k, float& h, float& l)
{
    h = ldexpf_fast(c.h, k);
    l = ldexpf_fast(c.l, k);
}
__device__ __forceinline__ df shfl_df(df v, int src)
{
    return df{__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src)};
}

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

// column c of the spin-2 E/B (or Q/U) coupling perm(Xr, Xi, Yr, Yi) = (-Yi, Yr, Xi, -Xr):
// source column within the group of four, and its sign
__device__ __forceinline__ int perm_src(int c) { return (c & ~3) | (3 - (c & 3)); }
__device__ __forceinline__ float perm_sign(int c) { return ((c & 3) == 0 || (c & 3) == 3) ? -1.0f : 1.0f; }

// data column (in T and the column maxima) of contraction column j: itself,
// or for one spin-2 component (E: Xr, Xi of each group of four; B: Yr, Yi)
__device__ __forceinline__ long long phys_col(const TcArgs& a, long long j)
{
    return a.csel == 0 ? j : ((j >> 1) << 2) + (j & 1) + (a.csel == 2 ? 2 : 0);
}

// quantum exponent of data column c0 + c of (m, q). Spin 2 also bounds the
// other slot, permuted: map2alm slices T_q +- P(T_{1-q}) (bounded by the sum),
// alm2map slices a_l or P(a_l) (bounded by the larger).
template <bool M2A, bool S2>
__device__ __forceinline__ int col_quantum(const TcArgs& a, int m, int q, long long c0, int c)
{
    const long long cg = c0 + c;
    if (cg >= a.ncol) return 0;
    const long long pc = phys_col(a, cg);
    float mx = a.colmax[((long long)m * 2 + q) * a.pcol + pc];
    if (S2) {
        const float mo = a.colmax[((long long)m * 2 + (1 - q)) * a.pcol + perm_src((int)(pc & 3)) + (pc & ~3LL)];
        mx = M2A ? mx + mo : fmaxf(mx, mo);
    }
    return quantum_exp(mx, a.Q);
}

// ===========================================================================
// map2alm (M2A = true):  a[l, c] = f_l sum_p lambda_lm(theta_p) T[p, c]
// alm2map (M2A = false): G[p, c] = s   sum_l lambda_lm(theta_p) a[l, c]
//
// Spin 2 (S2, Sec. 2.3 with F+- = -(2lambda +- -2lambda) / 2). Writing the two
// spin-weighted functions as v+ = 2lambda, v- = -2lambda:
//   map2alm, rows l of slot q:
//     a_l = F+ T_q + F- P_{1-q} = -1/2 [ v+ (T_q + P_{1-q}) + v- (T_q - P_{1-q}) ]
//   alm2map, slot q:
//     G_q = sum_{l in q} F+ a_l + sum_{l not in q} F- P(a_l)
//         = -1/2 sum_l [ v+ b_l + v- sigma_l b_l ],  b_l = a_l or P(a_l), sigma_l = +-1
// with P the E/B coupling permutation (perm_src). So each contraction runs over
// K' = 2 K: chunk 2u carries v+ and chunk 2u + 1 carries v- over the same 32
// ring pairs (map2alm) or values of l (alm2map), and a lambda piece is one
// recurrence (one s), like the spin-0 pieces. The data warps form the
// combinations of the two slots (map2alm) or the parity-dependent permutation
// and sign (alm2map) while slicing.
// grid.x = work item (m, q, tile), grid.y = column tile; clusters along y
// ===========================================================================
template <bool M2A, bool S2>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_leg_tc(void* __restrict__ dst, TcArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcShared& sh = *reinterpret_cast<TcShared*>(smem + NST * STAGE_BYTES + 3 * SCR_BYTES);
    const int4 w = a.work[blockIdx.x];
    // work item: (m, q, first tile | tiles << 16, first checkpoint block of (m, q));
    // an alm2map CTA walks several ring-pair tiles of (m, q) in one pipeline
    const int m = w.x, q = w.y, tile0 = w.z & 0xFFFF, ckb = w.w;
    const int ntl = M2A ? 1 : max(1, w.z >> 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t crank = cluster_ctarank(), csize = cluster_nctarank();
    const long long c0 = (long long)blockIdx.y * TC_M;
    const int l_first = m + q;
    const int nl = (a.lmax >= l_first) ? (a.lmax - l_first) / 2 + 1 : 0;   // l rows of slot q
    // ring pairs before pb hold negligible lambda for this order
    const int pb = (a.pfirst != nullptr) ? a.pfirst[m] : 0;
    const int nrow_all = M2A ? nl : a.R - pb;      // lambda rows of (m, q) (alm2map: ring pairs from pb)
    // tile t of the CTA: first lambda row, rows, 32-row pieces, MMA N
    auto t_n0 = [&](int t) { return (tile0 + t) * TC_N; };
    auto t_nrows = [&](int t) { return min(TC_N, nrow_all - t_n0(t)); };
    auto t_npieces = [&](int t) { return (t_nrows(t) + PR - 1) / PR; };
    auto t_nmma = [&](int t) { return (t_nrows(t) + 15) & ~15; };
    const int n0 = t_n0(0), nrows = t_nrows(0);    // map2alm: its only tile
    // contraction length: spin 0 over ring pairs (map2alm) or the l of slot q;
    // spin 2 over ring pairs or all l >= m, each twice (v+ and v- chunks)
    const int K = M2A ? a.R - pb : (S2 ? a.lmax - m + 1 : nl);
    const int nunit = (K + KC - 1) / KC;           // 32-wide units of raw data
    const int nch = S2 ? 2 * nunit : nunit;        // MMA chunks (pipeline stages) per tile
    const int nchunk = ntl * nch;                  // chunks of the CTA: chunk g = tile g / nch, kc = g % nch
    const int l0s = m > 2 ? m : 2;                 // first l of the spin-2 functions
    const int nmma = t_nmma(0);
    constexpr int SPAN = span_chunks<M2A, S2>();
    const int nspan = (nch + SPAN - 1) / SPAN;     // drained spans per tile
    const long long qstride = (long long)a.R * a.ncol;

    for (int r = tid; r < TC_N; r += blockDim.x) {
        if (M2A) sh.rowidx[r] = (r < nrows) ? (int)a_idx(a.lmax, l_first + 2 * (n0 + r), m) : 0;
        if (M2A && S2) {
            sh.cA2[r] = df{0.0f, 0.0f}; sh.cB2[r] = df{0.0f, 0.0f};
            if (r < nrows) {
                const int l = l_first + 2 * (n0 + r);
                const long long ci = a_idx(a.lmax, l, m);
                sh.rowexp[r] = quantum_exp(a.rowmax[ci], a.Q);
                // -d_l / 2 * factor; rows below l = 2 are zero
                const double f = (l < 2) ? 0.0 : -0.5 * a.s2d64[ci] * (m == 0 ? a.fs0 : a.fs1);
                const float fh = (float)f;
                sh.rfac[r] = make_float2(fh, (float)(f - (double)fh));
            } else {
                sh.rowexp[r] = 0; sh.rfac[r] = make_float2(0.0f, 0.0f);
            }
        } else if (M2A) {
            if (r < nrows) {
                const int l = l_first + 2 * (n0 + r);
                const long long ci = a_idx(a.lmax, l, m);
                sh.cA2[r] = df_of(a.nA[ci]);
                sh.cB2[r] = df_of(a.nB[ci]);
                sh.rowexp[r] = quantum_exp(a.rowmax[ci], a.Q);
                // c_l * dsigma applied once per output in double-float, so its
                // rounding is not a coherent error along the row
                const double f = a.nc64[ci] * (m == 0 ? a.fs0 : a.fs1);
                const float fh = (float)f;
                sh.rfac[r] = make_float2(fh, (float)(f - (double)fh));
            } else {
                sh.cA2[r] = df{0.0f, 0.0f}; sh.cB2[r] = df{0.0f, 0.0f};
                sh.rowexp[r] = 0; sh.rfac[r] = make_float2(0.0f, 0.0f);
            }
        }
    }
    for (int c = tid; c < TC_M; c += blockDim.x) sh.colexp[c] = col_quantum<M2A, S2>(a, m, q, c0, c);
    if (tid == 0) {
        for (int s = 0; s < NST; s++) {
            mbar_init(&sh.full[s], 1);     // the data warp's arrival; every byte completes as tx
            mbar_init(&sh.empty[s], csize);
        }
        mbar_init(&sh.accf, 1);
        mbar_init(&sh.cdone, 1);
        mbar_init(&sh.cfree, 4);
        mbar_init(&sh.tfree, 4);
        sh.released = NST - 1;
        sh.eok = 1;
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(&sh.tmem, 512);
    tc_fence_before();
    cluster_sync();            // barriers of every CTA initialised before any remote arrival
    tc_fence_after();
    const uint32_t tmem = sh.tmem;
    const uint32_t smem_base = smem_u32(smem);

    if (warp == 0) {
        // ---------------- MMA issue and stages (one lane) ----------------
        // A non-blocking event loop over two ordered streams:
        //  - stages: chunk c >= NST waits until every CTA of the cluster has
        //    consumed the stage's previous use (chunk c - NST), then starts its
        //    data copy and releases the stage to the lambda warps. The walk
        //    continues NST chunks past the end (publishing those too: the lambda
        //    warps' L2 slots wait on them), so that every MMA commit of the
        //    cluster has arrived on this CTA's barriers before it exits;
        //  - MMAs: chunk kc, once the stage is full and (first chunk of a span)
        //    the previous span has been drained (the drain rewrites main and sm).
        // Polls without progress are bounded.
        if (lane == 0) {
            const uint16_t mask = (uint16_t)((1u << csize) - 1u);
            // chunk c's data: one 32 KB bulk copy of its pre-sliced image (spin-2
            // alm2map: both chunks of a unit read the unit's image); the same
            // arrival announces the lambda pieces that the cluster multicasts in.
            // Column tiles that only pad the cluster read the last real tile.
            const int ytile = min((int)blockIdx.y, a.ntile - 1);
            const uint8_t* img0 = a.img + ((long long)a.img_base[m * 2 + q] * a.ntile + ytile) * A_BYTES;
            auto copy = [&](int c) {                    // c: chunk of the CTA
                const int s = c % NST;
                const int t = c / nch, kc = c - t * nch;
                // (map2alm: K starts at ring pair pb, (S2 ? 2 : 1) image chunks per unit)
                const long long ci = M2A ? kc + (S2 ? 2 : 1) * (pb / KC) : (S2 ? (kc >> 1) : kc);
                mbar_arrive_expect_tx(&sh.full[s], A_BYTES + t_npieces(t) * SCR_BYTES);
                bulk_copy_g2s(smem_base + s * STAGE_BYTES, img0 + ci * a.ntile * A_BYTES, A_BYTES, &sh.full[s]);
            };
            for (int c = 0; c < min(nchunk, NST); c++) copy(c);
            int c = NST;                                // next stage event
            int g = 0, t = 0, kc = 0;                   // next MMA chunk g = t nch + kc
            uint32_t idesc = idesc_f16(TC_M, t_nmma(0));
            bool full_ok = false;
            int idle = 0;
            while (g < nchunk || c < nchunk + NST) {
                bool did = false;
                if (c < nchunk + NST && mbar_test_wait_cl(&sh.empty[c % NST], (c / NST - 1) & 1)) {
                    if (c < nchunk) copy(c);
                    publish_counter(&sh.released, c);
                    c++;
                    did = true;
                }
                if (g < nchunk) {
                    const int s = g % NST;
                    if (!full_ok) full_ok = mbar_test_wait_cl(&sh.full[s], (g / NST) & 1);
                    const int kq = kc % SPAN;
                    bool ready = full_ok;
                    if (ready && kq == 0) {
                        // a tile's first span waits until the previous tile's epilogue has
                        // read the accumulators; a later span until the previous one is drained
                        if (kc == 0) ready = (t == 0) || mbar_test_wait_cl(&sh.tfree, (t - 1) & 1);
                        else ready = mbar_test_wait_cl(&sh.cfree, (t * nspan + kc / SPAN - 1) & 1);
                    }
                    if (ready) {
                        tc_fence_after();
                        issue_stage(tmem, smem_base + s * STAGE_BYTES, idesc, kc == 0, kq == 0);
                        umma_commit_mc(&sh.empty[s], mask);
                        if (kq == SPAN - 1 || kc == nch - 1) umma_commit(&sh.cdone);
                        if (kc == nch - 1) umma_commit(&sh.accf);
                        g++;
                        full_ok = false;
                        if (++kc == nch) {
                            kc = 0;
                            if (++t < ntl) idesc = idesc_f16(TC_M, t_nmma(t));
                        }
                        did = true;
                    }
                }
                if (did) {
                    idle = 0;
                } else if (++idle > (1 << 24)) {
                    atomicCAS(a.err, 0, 1);
                    break;
                }
            }
        }
    } else if (warp < 4) {
        // ---------------- lambda pieces ----------------
        // A piece is computed first, in groups of 8 rows / steps, into this
        // warp's scratch (the piece's exact shared-memory image), and only then
        // does the warp wait for its stage to be released, so the recurrence
        // overlaps the MMAs of earlier chunks. A warp's pieces can be several
        // chunks apart, more than the parity of the stage barrier can tell
        // apart, so it waits on the monotonic count of released chunks that the
        // data warps publish instead.
        uint8_t* scr = smem + NST * STAGE_BYTES + (warp - 1) * SCR_BYTES;
        const uint32_t smid = sm_id();
        if (smid >= (uint32_t)LAM_SM && lane == 0) atomicCAS(a.err, 0, 9);
        uint8_t* gslots = g_lam_slots + ((size_t)(smid % LAM_SM) * 3 + (warp - 1)) * LAM_SLOTS * SCR_BYTES;
        const uint16_t mask = (uint16_t)((1u << csize) - 1u);
        // the CTA's pieces in order (tile, chunk, piece); every tile but the last
        // has full 128-row tiles, TC_N / PR pieces per chunk
        constexpr int NPF = TC_N / PR;
        const int np_last = t_npieces(ntl - 1);
        const int pfull = (ntl - 1) * nch * NPF;
        const int total = (smid < (uint32_t)LAM_SM) ? pfull + nch * np_last : 0;
        auto piece_at = [&](int gi, int& t, int& kc, int& j) {
            if (gi < pfull) {
                t = gi / (nch * NPF);
                const int r = gi - t * nch * NPF;
                kc = r / NPF;
                j = r - kc * NPF;
            } else {
                const int r = gi - pfull;
                t = ntl - 1;
                kc = r / np_last;
                j = r - kc * np_last;
            }
        };
        const int gstep = (int)csize * 3;
        int npc = 0;                                    // pieces of this warp so far
        for (int g = (int)crank + (int)csize * (warp - 1); g < total; g += gstep, npc++) {
            int t, kc, j;
            piece_at(g, t, kc, j);
            const int gch = t * nch + kc;               // chunk of the CTA
            const int s = gch % NST;
            const int n0t = t_n0(t), nrt = t_nrows(t);  // the tile's rows
            if constexpr (M2A && S2) {
                // lane = ring pair (k) of unit kc / 2, walking the 64 l that hold the
                // 32 rows (slot q) of piece j with the recurrence of s = (kc odd ? -2 : +2)
                const int sg = kc & 1;
                const int p = pb + (kc >> 1) * KC + lane;
                const int J = (n0t >> 5) + j;            // 32-row block of the slot's rows
                const int L = m + 64 * J;               // first l of the walk (checkpoint block 2J)
                const int lck = max(L, l0s);            // l of the checkpointed value
                df cur = {0.0f, 0.0f}, prev = {0.0f, 0.0f}, x = {0.0f, 0.0f};
                int E = 0;
                const bool live = p < a.R;
                if (live) {
                    const long long ci = ((long long)(ckb + 2 * J) * 2 + sg) * a.R + p;
                    E = a.ck_exp[ci];
                    ck_to_df(a.ck[ci], cur, prev, E);
                    x = df_of(a.pairs[p].x);
                }
                // coefficients of the walk: lane k holds l = L + k and L + 32 + k
                df cA0 = {0.0f, 0.0f}, cB0 = {0.0f, 0.0f}, cA1 = {0.0f, 0.0f}, cB1 = {0.0f, 0.0f};
                if (L + lane <= a.lmax) {
                    const long long ci = a_idx(a.lmax, L + lane, m);
                    cA0 = df_of(a.s2A[sg][ci]); cB0 = df_of(a.s2B[sg][ci]);
                }
                if (L + 32 + lane <= a.lmax) {
                    const long long ci = a_idx(a.lmax, L + 32 + lane, m);
                    cA1 = df_of(a.s2A[sg][ci]); cB1 = df_of(a.s2B[sg][ci]);
                }
                const int rn = min(PR, nrt - j * PR);  // rows of this piece (warp-uniform)
                int lc = lck;                           // l of cur (warp-uniform)
#pragma unroll 1
                for (int i0 = 0; i0 < PR; i0 += 8) {
                    float hv[8], lv[8];
#pragma unroll
                    for (int ii = 0; ii < 8; ii++) {
                        const int i = i0 + ii;
                        hv[ii] = 0.0f; lv[ii] = 0.0f;
                        if (i < rn) {
                            const int lt = L + q + 2 * i;   // the row's l
#pragma unroll
                            for (int st = 0; st < 2; st++) {
                                if (lc < lt) {
                                    const int k = lc + 1 - L;
                                    const df cA = shfl_df(k < 32 ? cA0 : cA1, k & 31);
                                    const df cB = shfl_df(k < 32 ? cB0 : cB1, k & 31);
                                    df_rec(df_axb(cA, x, cB), cur, prev, -1.0f);
                                    rescale_df(cur, prev, E);
                                    lc++;
                                }
                            }
                            if (live && lt >= lck) df_scaled(cur, E - sh.rowexp[j * PR + i], hv[ii], lv[ii]);
                        }
                    }
                    put_rows8<r0_grid<M2A, S2>()>(scr, i0, lane, hv, lv);
                }
            } else if constexpr (M2A) {
                // lane = ring pair (k), walking the 32 l rows of piece j
                const int p = pb + kc * KC + lane;
                df cur = {0.0f, 0.0f}, prev = {0.0f, 0.0f}, x2 = {0.0f, 0.0f};
                int E = 0;
                const bool live = p < a.R;
                if (live) {
                    const long long ci = (long long)(ckb + (n0t + j * PR) / CK_ROWS) * a.R + p;
                    E = a.ck_exp[ci];
                    ck_to_df(a.ck[ci], cur, prev, E);
                    const df x = df_of(a.pairs[p].x);
                    x2 = df_mul(x, x);
                }
                const int rn = min(PR, nrt - j * PR);  // rows of this piece (warp-uniform)
                df tn = df_axb(sh.cA2[j * PR], x2, sh.cB2[j * PR]);
#pragma unroll 1
                for (int i0 = 0; i0 < PR; i0 += 8) {
                    float hv[8], lv[8];
#pragma unroll
                    for (int ii = 0; ii < 8; ii++) {
                        const int i = i0 + ii;
                        hv[ii] = 0.0f; lv[ii] = 0.0f;
                        if (i < rn) {
                            const int r = j * PR + i;
                            if (live) df_scaled(cur, E - sh.rowexp[r], hv[ii], lv[ii]);
                            const df t = tn;            // coefficient one step ahead
                            if (i + 1 < rn) tn = df_axb(sh.cA2[r + 1], x2, sh.cB2[r + 1]);
                            df_rec(t, cur, prev, 1.0f);
                            rescale_df(cur, prev, E);
                        }
                    }
                    put_rows8<r0_grid<M2A, S2>()>(scr, i0, lane, hv, lv);
                }
            } else if constexpr (S2) {
                // lane = ring pair (row), walking the 32 l of unit kc / 2 with the
                // recurrence of s = (kc odd ? -2 : +2); d_l applied in double-float
                const int sg = kc & 1;
                const int u = kc >> 1;
                const int r = j * PR + lane;
                const int p = pb + n0t + r;
                const bool live = r < nrt;
                const int L = m + KC * u;               // first l of the unit (checkpoint block u)
                const int lck = max(L, l0s);
                df cur = {0.0f, 0.0f}, prev = {0.0f, 0.0f}, x = {0.0f, 0.0f};
                int E = 0, pe = 0;
                if (live) {
                    const long long ci = ((long long)(ckb + u) * 2 + sg) * a.R + p;
                    E = a.ck_exp[ci];
                    ck_to_df(a.ck[ci], cur, prev, E);
                    x = df_of(a.pairs[p].x);
                    pe = quantum_exp(a.pairmax[((long long)m * 2 + q) * a.R + p], a.Q);
                }
                df cAk = {0.0f, 0.0f}, cBk = {0.0f, 0.0f};
                float2 cdk = make_float2(0.0f, 0.0f);
                if (L + lane <= a.lmax) {
                    const long long ci = a_idx(a.lmax, L + lane, m);
                    cAk = df_of(a.s2A[sg][ci]); cBk = df_of(a.s2B[sg][ci]); cdk = a.s2d2[ci];
                }
#pragma unroll 1
                for (int i0 = 0; i0 < PR; i0 += 8) {
                    float hv[8], lv[8];
#pragma unroll
                    for (int ii = 0; ii < 8; ii++) {
                        const int i = i0 + ii;
                        hv[ii] = 0.0f; lv[ii] = 0.0f;
                        const float d0 = __shfl_sync(0xffffffffu, cdk.x, i);
                        const float d1 = __shfl_sync(0xffffffffu, cdk.y, i);
                        const df cA = shfl_df(cAk, i);
                        const df cB = shfl_df(cBk, i);
                        const int l = L + i;
                        if (l <= a.lmax && l >= lck) {
                            if (l > lck) {
                                df_rec(df_axb(cA, x, cB), cur, prev, -1.0f);
                                rescale_df(cur, prev, E);
                            }
                            float h = 0.0f, lo = 0.0f;
                            if (live) df_scaled(cur, E - pe, h, lo);
                            const float p1 = __fmul_rn(h, d0);      // lambda = d_l mu in double-float
                            // v- chunks carry sigma_l = -1 for the rows of the other parity
                            const float sgn = (sg && (i & 1) != q) ? -1.0f : 1.0f;
                            hv[ii] = sgn * p1;
                            lv[ii] = sgn * (fmaf(h, d0, -p1) + (h * d1 + lo * d0));
                        }
                    }
                    put_chunk8(scr, lane, i0 >> 3, hv, lv);
                }
            } else {
                // lane = ring pair (row), walking the 32 l of stage kc; the
                // coefficients of those 32 l are loaded once (lane k holds l_k)
                // and broadcast with shuffles
                const int r = j * PR + lane;
                const int p = pb + n0t + r;
                const bool live = r < nrt;
                df cur = {0.0f, 0.0f}, prev = {0.0f, 0.0f}, x2 = {0.0f, 0.0f};
                int E = 0, pe = 0;
                if (live) {
                    const long long ci = (long long)(ckb + kc * KC / CK_ROWS) * a.R + p;
                    E = a.ck_exp[ci];
                    ck_to_df(a.ck[ci], cur, prev, E);
                    const df x = df_of(a.pairs[p].x);
                    x2 = df_mul(x, x);
                    pe = quantum_exp(a.pairmax[((long long)m * 2 + q) * a.R + p], a.Q);
                }
                df cAk = {0.0f, 0.0f}, cBk = {0.0f, 0.0f};
                float2 cck = make_float2(0.0f, 0.0f);
                {
                    const int k = kc * KC + lane;
                    if (k < K) {
                        const long long ci = a_idx(a.lmax, l_first + 2 * k, m);
                        cAk = df_of(a.nA[ci]); cBk = df_of(a.nB[ci]); cck = a.nc2[ci];
                    }
                }
                const int kn = min(KC, K - kc * KC);    // valid l of this chunk (warp-uniform)
                df tn = df_axb(shfl_df(cAk, 0), x2, shfl_df(cBk, 0));
#pragma unroll 1
                for (int i0 = 0; i0 < PR; i0 += 8) {
                    float hv[8], lv[8];
#pragma unroll
                    for (int ii = 0; ii < 8; ii++) {
                        const int i = i0 + ii;
                        hv[ii] = 0.0f; lv[ii] = 0.0f;
                        const float c0_ = __shfl_sync(0xffffffffu, cck.x, i);
                        const float c1_ = __shfl_sync(0xffffffffu, cck.y, i);
                        const df cAn = shfl_df(cAk, (i + 1) & (PR - 1));
                        const df cBn = shfl_df(cBk, (i + 1) & (PR - 1));
                        if (i < kn) {
                            float h = 0.0f, lo = 0.0f;
                            if (live) df_scaled(cur, E - pe, h, lo);
                            const float p1 = __fmul_rn(h, c0_);     // lambda = c_l mu in double-float
                            hv[ii] = p1;
                            lv[ii] = fmaf(h, c0_, -p1) + (h * c1_ + lo * c0_);
                            const df t = tn;
                            if (i + 1 < kn) tn = df_axb(cAn, x2, cBn);
                            df_rec(t, cur, prev, 1.0f);
                            rescale_df(cur, prev, E);
                        }
                    }
                    put_chunk8(scr, lane, i0 >> 3, hv, lv);
                }
            }
            __syncwarp();
            // The piece into its L2 slot, once the slot's previous piece (LAM_SLOTS
            // pieces ago, chunk kp) has landed in every CTA: true once chunk kp + NST
            // is released, which needs the MMAs of chunk kp in every CTA.
            const int gp = g - LAM_SLOTS * gstep;
            int tp = 0, kcp = 0, jp = 0;
            if (gp >= 0) piece_at(gp, tp, kcp, jp);
            if (gp >= 0 && !__all_sync(0xffffffffu, wait_counter(&sh.released, tp * nch + kcp + NST, a.err, 8))) break;
            uint8_t* gs = gslots + (npc & (LAM_SLOTS - 1)) * SCR_BYTES;
#pragma unroll
            for (int v = 0; v < SCR_BYTES / 512; v++) {
                const int off = (v * 32 + lane) * 16;
                *reinterpret_cast<uint4*>(gs + off) = *reinterpret_cast<const uint4*>(scr + off);
            }
            fence_proxy_async_global();
            __syncwarp();
            if (!__all_sync(0xffffffffu, wait_counter(&sh.released, gch, a.err, 2))) break;
            // stage free in every CTA: one multicast copy per plane into rows
            // 32 j .. 32 j + 31 (one contiguous 2 KB block: the swizzle repeats
            // every 8 rows); each CTA's data warp announced these bytes
            if (lane == 0) {
                const uint32_t dst = smem_u32(smem + s * STAGE_BYTES + NPL * A_PLANE) + j * PIECE_BYTES;
#pragma unroll
                for (int b = 0; b < NPL; b++)
                    bulk_copy_g2s_mc(dst + b * B_PLANE, gs + b * PIECE_BYTES, PIECE_BYTES, &sh.full[s], mask);
            }
            __syncwarp();                               // scratch reads done before the next piece
        }
    } else {
        // ---------------- span drains (warps 4-7) ----------------
        const int quarter = warp & 3;                 // TMEM lanes 32 quarter .. + 31
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        bool dok = true;
        // Fold span j's corrections (chunks SPAN j .. SPAN j + SPAN - 1) into
        // main and sm and hand the accumulators back to the MMA: main +=
        // nearest integers of ex and sm (exact), sm = their fractional parts +
        // 2^-12 fn (below 1). Groups of 16 columns, the next
        // group's TMEM loads in flight while the current one is folded; packed
        // FP32 pairs. (A rolled loop: a short body stays in the instruction cache.)
        const unsigned long long MAG2 = f2_pack(0x4B400000u, 0x4B400000u);   // 1.5 * 2^23: nearest integer
        const unsigned long long SC2 = f2_pack(0x39800000u, 0x39800000u);    // 2^-12
        auto drain_load = [&](int g, uint32_t (&v)[4][16]) {
            tmem_ld16(tl + g, v[0]);
            tmem_ld16(tl + ACC_EX + g, v[1]);
            tmem_ld16(tl + ACC_SM + g, v[2]);
            tmem_ld16(tl + ACC_FN + g, v[3]);
        };
        auto drain_fold = [&](int g, uint32_t (&v)[4][16]) {
#pragma unroll
            for (int i = 0; i < 16; i += 2) {
                const unsigned long long M = f2_pack(v[0][i], v[0][i + 1]), E = f2_pack(v[1][i], v[1][i + 1]);
                const unsigned long long V = f2_pack(v[2][i], v[2][i + 1]), F = f2_pack(v[3][i], v[3][i + 1]);
                const unsigned long long EH = f2_sub(f2_add(E, MAG2), MAG2);
                const unsigned long long VH = f2_sub(f2_add(V, MAG2), MAG2);
                f2_unpack(f2_add(f2_add(M, EH), VH), v[0][i], v[0][i + 1]);
                f2_unpack(f2_fma(F, SC2, f2_add(f2_sub(E, EH), f2_sub(V, VH))), v[2][i], v[2][i + 1]);
            }
            tmem_st16(tl + g, v[0]);
            tmem_st16(tl + ACC_SM + g, v[2]);
        };
        auto drain = [&](int j, int nm) {          // j: span of the CTA; nm: its tile's MMA N
            dok = dok && __all_sync(0xffffffffu, mbar_wait_cl(&sh.cdone, j & 1, a.err, 6));
            if (!dok) return;
            tc_fence_after();
            const int gb = 0, ge = nm;
            uint32_t va[4][16], vb[4][16];
            drain_load(gb, va);
            tmem_wait_ld();
#pragma unroll 1
            for (int g = gb; g < ge; g += 32) {
                if (g + 16 < ge) drain_load(g + 16, vb);
                drain_fold(g, va);
                tmem_wait_ld();
                if (g + 16 < ge) {
                    if (g + 32 < ge) drain_load(g + 32, va);
                    drain_fold(g + 16, vb);
                    tmem_wait_ld();
                }
            }
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.cfree);
        };
        // (the MMAs of the next span wait for each drain; a wait that gives up
        // turns dok off and ends the drains)
        if constexpr (M2A) {
            for (int j = 0; j < nspan && dok; j++) drain(j, nmma);
            // the last MMAs are complete once every wait above succeeded
            const bool ok = dok && ((nch == 0) || __all_sync(0xffffffffu, mbar_wait_cl(&sh.accf, 0, a.err, 4)));
            if (lane == 0 && !ok) sh.eok = 0;
            tmem_wait_st();
        } else {
            // alm2map, per tile: its spans, then its epilogue for this thread's
            // column: G = (main + sm) * scales. The accumulators are read into
            // registers and handed back (tfree) before the stores, which then
            // overlap the next tile's MMAs.
            const int tcol = tid - 128;
            const long long cg = c0 + tcol;
            const bool cok = cg < a.ncol;
            // G = sc 2^(ce + pe) (main + sm): the column factor sc 2^ce per
            // thread, the row factor 2^pe per row (powers of two: exact down to
            // 2^-149), so each output costs two multiplies and a store
            const float csc = ldexpf(((m == 0) ? a.s0 : a.s1) * (S2 ? -0.5f : 1.0f), sh.colexp[tcol]);
            float* Gq = (float*)dst + ((long long)m * 2 + q) * qstride + cg;
            float* rsc = reinterpret_cast<float*>(sh.cA2);
            for (int t = 0; t < ntl; t++) {
                const int nmt = t_nmma(t), nrt = t_nrows(t), n0t = t_n0(t);
                {   // the tile's row factors; the load overlaps the span drains
                    const int rl = quarter * 32 + lane;
                    const float pm = (rl < nrt) ? a.pairmax[((long long)m * 2 + q) * a.R + pb + n0t + rl] : 0.0f;
                    for (int j = 0; j < nspan && dok; j++) drain(t * nspan + j, nmt);
                    rsc[(t & 1) * TC_N + rl] = (pm > 0.0f) ? ldexpf(1.0f, quantum_exp(pm, a.Q)) : 0.0f;
                    named_bar_sync(3, 128);    // drain warps only
                }
                dok = dok && ((nch == 0) || __all_sync(0xffffffffu, mbar_wait_cl(&sh.accf, t & 1, a.err, 4)));
                tc_fence_after();
                float gv[TC_N];
#pragma unroll
                for (int gq = 0; gq < TC_N / 16; gq++) {
                    uint32_t v0[16], vr[16];
                    if (dok && nch > 0 && gq * 16 < nmt) {
                        tmem_ld16(tl + gq * 16, v0);
                        tmem_ld16(tl + ACC_SM + gq * 16, vr);
                        tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < 16; i++) gv[gq * 16 + i] = __uint_as_float(v0[i]) + __uint_as_float(vr[i]);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; i++) gv[gq * 16 + i] = 0.0f;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.tfree);
                // (row factors of tile t were written before the barrier above; the
                // next write to this half is two barriers later)
                if (cok && dok) {
                    const float4* rs4 = reinterpret_cast<const float4*>(rsc + (t & 1) * TC_N);
                    float* gp = Gq + (long long)(pb + n0t) * a.ncol;
#pragma unroll
                    for (int r4 = 0; r4 < TC_N / 4; r4++) {
                        const float4 f = rs4[r4];
                        const float fr[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
                        for (int i = 0; i < 4; i++) {
                            const int r = 4 * r4 + i;
                            if (r < nrt) gp[(long long)r * a.ncol] = (nch > 0) ? (gv[r] * csc) * fr[i] : 0.0f;
                        }
                    }
                }
            }
            tmem_wait_st();
        }
    }

    // ---------------- map2alm epilogue: out = (main + sm) * scales, warps 0-7 ----------------
    // (warps w and w + 4 reach the same TMEM lanes, i.e. the same map column;
    // warps 4-7 take rows 0-63, warps 0-3 rows 64-127)
    if constexpr (M2A) {
        __syncwarp();
        tc_fence_before();
        named_bar_sync(2, 256);
        tc_fence_after();
        const int t = tid & (TC_M - 1);             // this lane's TMEM lane: real column c0 + t
        const int ce = sh.colexp[t];
        const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const bool ok = sh.eok != 0;
        const int g0 = (warp >= 4) ? 0 : 2;
        // each warp's 32 x 32 outputs go through its own 8.25 KB of the (now idle)
        // stage memory and out by map column: lane = row, one 16-byte store of
        // (re, im) per lane, so a warp's store spans 1 KB of one map column
        // instead of 16 columns nalm apart
        double* tile = reinterpret_cast<double*>(smem) + warp * 32 * 33;   // rows of 33: conflict-free
        const long long cw = c0 + (warp & 3) * 32;     // the warp's first real column
#pragma unroll 1
        for (int g = g0; g < g0 + 2; g++) {
            if (g * 32 >= nmma) continue;
            uint32_t v0[32], vr[32];
            if (nch > 0) {
                tmem_ld32(tl + g * 32, v0);
                tmem_ld32(tl + ACC_SM + g * 32, vr);
                tmem_wait_ld();
            } else {
#pragma unroll
                for (int i = 0; i < 32; i++) v0[i] = vr[i] = 0u;
            }
#pragma unroll
            for (int i = 0; i < 32; i++) {
                const int r = g * 32 + i;
                double v = 0.0;
                if (r < nrows) {
                    // main (exact integer) + the residual as an FP32 pair, times c_l f (hi/lo)
                    const float x0 = __uint_as_float(v0[i]), x1 = __uint_as_float(vr[i]);
                    const float sm = x0 + x1;
                    const float bb = sm - x0;
                    const float er = (x0 - (sm - bb)) + (x1 - bb);
                    const float2 F = sh.rfac[r];
                    const float p1 = __fmul_rn(sm, F.x);
                    const float lo = fmaf(sm, F.x, -p1) + er * F.x + sm * F.y;
                    v = f32_to_f64(p1) + f32_to_f64(lo);                       // final FP64 accumulation
                    v = ldexp_fast(v, sh.rowexp[r] + ce);
                }
                tile[i * 33 + lane] = v;
            }
            __syncwarp();
            const int r = g * 32 + lane;
            if (ok && r < nrows) {
                const long long ri = sh.rowidx[r];
#pragma unroll 4
                for (int mc = 0; mc < 16; mc++) {
                    const long long cr = cw + 2 * mc;  // the re column (ncol is even)
                    if (cr >= a.ncol) break;
                    const double re = tile[lane * 33 + 2 * mc];
                    const double im = (m == 0) ? 0.0 : tile[lane * 33 + 2 * mc + 1];
                    reinterpret_cast<double2*>(dst)[(cr >> 1) * a.nalm + ri] = make_double2(re, im);
                }
            }
            __syncwarp();                               // the tile is rewritten for the next g
        }
    }
    __syncwarp();
    tc_fence_before();
    cluster_sync();            // no CTA leaves while others may still copy into it
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ===========================================================================
// data operand of the contraction, pre-sliced: for each 32-wide unit of K of
// (m, q) and each column tile, the four FP16 slice planes (tc::slice4d in the
// column's quantum) of the 128 columns x 32 K values, written as the exact
// shared-memory image the MMAs read (K-major, 64-byte swizzle), 32 KB per
// chunk, so that k_leg_tc fetches a chunk with one bulk copy. Rows past K and
// columns past ncol are written as zeros.
//   map2alm: rows = ring pairs of T[m][q]; spin 2: chunk 2u holds
//            T_q + P(T_{1-q}) and chunk 2u + 1 holds T_q - P(T_{1-q}) (the two
//            combinations of Sec. 2.3 that meet v+ and v-).
//   alm2map: rows = the l of slot q (spin 0: l = m + q + 2k) or all l >= m
//            (spin 2: a_l for l - m of parity q, P(a_l) otherwise; the sign
//            sigma_l of the v- chunks is carried by lambda).
// grid.x = unit (m, q, u, image chunk), grid.y = column tile; one column per
// thread. The image is built in shared memory and then copied out 16 bytes
// per lane, so that a warp's stores cover 512 contiguous bytes (direct stores
// of a row's 16-byte chunks would hit 32 half sectors per instruction).
// ===========================================================================
template <bool M2A, bool S2>
__global__ void __launch_bounds__(TC_M)
k_slice(const float2* __restrict__ raw, uint8_t* __restrict__ img, TcArgs a)
{
    __shared__ __align__(128) uint8_t simg[A_BYTES];
    const int4 w = a.sunits[blockIdx.x];
    const int m = w.x, q = w.y, u = w.z;
    const int t = threadIdx.x, lane = t & 31;
    const long long c0 = (long long)blockIdx.y * TC_M;
    const long long cg = c0 + t;
    const bool cok = cg < a.ncol;
    const long long pc = phys_col(a, cg);           // the column in T / A2
    const int l_first = m + q;
    const int nl = (a.lmax >= l_first) ? (a.lmax - l_first) / 2 + 1 : 0;
    const int K = M2A ? a.R : (S2 ? a.lmax - m + 1 : nl);
    constexpr bool TWO = S2 && M2A;                 // map2alm spin 2 reads both slots
    // one spin-2 component: this thread reads the permuted partner column of
    // the other slot itself (its lane does not hold it)
    const long long pc1 = (TWO && a.csel) ? perm_src((int)(pc & 3)) + (pc & ~3LL) : pc;
    float2 buf[TWO ? 2 * KC : KC];
#pragma unroll
    for (int h = 0; h < (TWO ? 2 : 1); h++) {
        const int slot = h ? 1 - q : q;
        const long long col = h ? pc1 : pc;
#pragma unroll
        for (int i = 0; i < KC; i++) {
            const int k = u * KC + i;
            float2 x = make_float2(0.0f, 0.0f);
            if (cok && k < K) {
                long long row;
                if (M2A) row = ((long long)m * 2 + slot) * a.R + k;
                else row = S2 ? a_idx(a.lmax, m + k, m) : a_idx(a.lmax, l_first + 2 * k, m);
                x = __ldg(raw + row * a.pcol + col);
            }
            buf[h * KC + i] = x;
        }
    }
    const int ce = col_quantum<M2A, S2>(a, m, q, c0, t);
    const float csc = __int_as_float((127 - ce) << 23);   // 2^-ce (exact scaling)
    const int psrc = (lane & ~3) | (3 - (lane & 3));     // spin 2: lane of the permuted column
    const float sgp = perm_sign((int)(pc & 3));
    const bool direct = a.csel != 0;
#pragma unroll
    for (int sub = 0; sub < (TWO ? 2 : 1); sub++) {
        uint8_t* A = simg;
        if (sub) __syncthreads();                     // the previous image has been copied out
#pragma unroll
        for (int jj = 0; jj < KC / 8; jj++) {
            float hv[8], lv[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int r = jj * 8 + i;
                float2 x;
                if constexpr (!S2) {
                    x = buf[r];
                } else if constexpr (M2A) {
                    // T_q +- P(T_{1-q}) in double-float (TwoSum of the hi parts)
                    const float2 x0 = buf[r];
                    float2 x1;
                    x1.x = __shfl_sync(0xffffffffu, buf[KC + r].x, psrc);
                    x1.y = __shfl_sync(0xffffffffu, buf[KC + r].y, psrc);
                    if (direct) x1 = buf[KC + r];
                    const float sb = sub ? -sgp : sgp;
                    const float bh = sb * x1.x;
                    const float s1 = x0.x + bh;
                    const float bb = s1 - x0.x;
                    const float lo = ((x0.x - (s1 - bb)) + (bh - bb)) + (x0.y + sb * x1.y);
                    const float hi = s1 + lo;
                    x = make_float2(hi, lo - (hi - s1));
                } else {
                    // a_l (l - m = 32 u + r of parity q) or P(a_l)
                    float2 xp;
                    xp.x = __shfl_sync(0xffffffffu, buf[r].x, psrc);
                    xp.y = __shfl_sync(0xffffffffu, buf[r].y, psrc);
                    const bool same = (r & 1) == q;
                    x = same ? buf[r] : make_float2(sgp * xp.x, sgp * xp.y);
                }
                hv[i] = x.x * csc;
                lv[i] = x.y * csc;
            }
            put4x8<r0_grid<M2A, S2>()>(A, A_PLANE, t, jj, hv, lv);
        }
        __syncthreads();
        uint4* dst = reinterpret_cast<uint4*>(img + ((long long)(w.w + sub) * a.ntile + blockIdx.y) * A_BYTES);
        const uint4* src = reinterpret_cast<const uint4*>(simg);
#pragma unroll 4
        for (int i = t; i < A_BYTES / 16; i += TC_M) dst[i] = src[i];
    }
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
// spin-2 plan-time walk (one block per m, threads over ring pairs): both
// normalised Wigner recurrences over every l >= l0 = max(m, 2), checkpoints
// at l = max(m + 32 b, l0) for every 32-wide block b of l - m, the per-row
// maxima over ring pairs and both s of |mu 2^E| (map2alm quanta) and the
// per-pair maxima over l and s of |d_l mu 2^E| (alm2map quanta; the same for
// both slots).
// ===========================================================================
__global__ void __launch_bounds__(256)
k_split_tables_s2(TcArgs a, const int* __restrict__ ck_base, double2* __restrict__ ck, int* __restrict__ ck_exp,
                  const double* __restrict__ seed_mant, const int* __restrict__ seed_exp,
                  unsigned int* __restrict__ rowmax_bits, float* __restrict__ pairmax)
{
    const int m = blockIdx.x;
    const int l0 = m > 2 ? m : 2;
    const int base = ck_base[m];
    for (int p0 = 0; p0 < a.R; p0 += blockDim.x) {
        const int p = p0 + threadIdx.x;
        const bool valid = p < a.R;
        double cur[2] = {0.0, 0.0}, prev[2] = {0.0, 0.0}, x = 0.0;
        int E[2] = {0, 0};
        if (valid) {
            for (int si = 0; si < 2; si++) {
                const long long i0 = ((long long)m * 2 + si) * a.R + p;
                cur[si] = seed_mant[i0];
                E[si] = seed_exp[i0];
            }
            x = a.pairs[p].x;
        }
        float pm = 0.0f;
        for (int l = l0; l <= a.lmax; l++) {
            const long long ci = a_idx(a.lmax, l, m);
            if (valid && l > l0) {
                for (int si = 0; si < 2; si++) {
                    const double nxt = fma(fma(a.s2A[si][ci], x, a.s2B[si][ci]), cur[si], -prev[si]);
                    prev[si] = cur[si];
                    cur[si] = nxt;
                    rescale(cur[si], prev[si], E[si]);
                }
            }
            if (valid && (l == l0 || (l - m) % CK_ROWS == 0)) {
                const int b = (l - m) / CK_ROWS;      // l0 < m + 32: block 0 starts at l0
                for (int si = 0; si < 2; si++) {
                    const long long i1 = ((long long)(base + b) * 2 + si) * a.R + p;
                    ck[i1] = make_double2(cur[si], prev[si]);
                    ck_exp[i1] = E[si];
                }
            }
            float vmu = 0.0f;
            if (valid)
                for (int si = 0; si < 2; si++) vmu = fmaxf(vmu, fabsf(f64_to_f32_scaled(cur[si], E[si])));
            pm = fmaxf(pm, vmu * fabsf(a.s2d2[ci].x) * 1.0000003f);
            float wv = vmu * 1.0000003f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wv = fmaxf(wv, __shfl_xor_sync(0xffffffffu, wv, o));
            if ((threadIdx.x & 31) == 0 && wv > 0.0f) atomicMax(rowmax_bits + ci, __float_as_uint(wv));
        }
        if (valid) {
            pairmax[((long long)m * 2 + 0) * a.R + p] = pm;
            pairmax[((long long)m * 2 + 1) * a.R + p] = pm;
        }
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
    // the block's 64 x 32 loads, PREP_UB per thread all in flight before the
    // first is stored (256 threads: one batch)
    constexpr int PREP_UB = PREP_L * PREP_M / 256;
    for (int e0 = tid; e0 < PREP_L * PREP_M; e0 += PREP_UB * blockDim.x) {
        double2 v[PREP_UB];
#pragma unroll
        for (int u = 0; u < PREP_UB; u++) {
            const int e = e0 + u * (int)blockDim.x;
            const int j = e / PREP_L, li = e % PREP_L;        // consecutive threads: consecutive l
            v[u] = make_double2(0.0, 0.0);
            if (e < PREP_L * PREP_M && l0 + li <= lmax && mp0 + j < nmc)
                v[u] = reinterpret_cast<const double2*>(alm)[(mp0 + j) * nalm + base + li];
        }
#pragma unroll
        for (int u = 0; u < PREP_UB; u++) {
            const int e = e0 + u * (int)blockDim.x;
            if (e >= PREP_L * PREP_M) break;
            if (m == 0) v[u].y = 0.0;
            tile[e % PREP_L][e / PREP_L] = v[u];
        }
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
    for (int si = 0; si < 2; si++) { a.s2A[si] = p->s.s2A[si]; a.s2B[si] = p->s.s2B[si]; }
    a.s2d2 = p->s.s2d2; a.s2d64 = p->s.s2d64;
    a.rowmax = (const float*)p->s.rowmax_bits;
    a.pairmax = p->s.pairmax;
    a.pfirst = p->s.pfirst;
    a.colmax = colmax;
    a.err = p->s.err;
    a.lmax = p->lmax; a.mmax = p->mmax; a.R = p->R;
    a.ncol = ncols(p, nmaps); a.nalm = p->nalm;
    a.pcol = a.ncol; a.csel = 0;
    a.ntile = (int)((a.ncol + TC_M - 1) / TC_M);
    a.img = nullptr; a.img_base = nullptr; a.sunits = nullptr;
    a.Q = Q;
    a.fs0 = a.fs1 = 1.0;
    a.s0 = a.s1 = 1.0f;
    a.work = nullptr;
    return a;
}

// largest cluster: 8 (portable limit), or SHT_MAX_CLUSTER from the environment (up to 16)
static int max_cluster()
{
    static int mc = [] {
        const char* e = std::getenv("SHT_MAX_CLUSTER");
        int v = e ? std::atoi(e) : DEF_CLUSTER;
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

template <bool M2A, bool S2>
static cudaError_t launch_slice(int nunits, const void* src, uint8_t* img, const TcArgs& a, const char* name,
                                cudaStream_t st)
{
    if (nunits == 0) return cudaSuccess;
    prof_start(name, st);
    k_slice<M2A, S2><<<dim3((unsigned)nunits, (unsigned)a.ntile), TC_M, 0, st>>>((const float2*)src, img, a);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

// one launch of the contraction over work items [0, nwork) of a.work with
// clusters of C CTAs along the column tiles (halved until a launch succeeds)
template <bool M2A, bool S2>
static cudaError_t launch_grid(int nwork, int C, void* dst, const TcArgs& a, cudaStream_t st)
{
    auto kern = k_leg_tc<M2A, S2>;
    const long long ntiles = (a.ncol + TC_M - 1) / TC_M;
    cudaError_t e = cudaSuccess;
    for (;;) {
        const long long gy = (ntiles + C - 1) / C * C;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)nwork, (unsigned)gy, 1);
        cfg.blockDim = dim3(TC_THREADS, 1, 1);
        cfg.dynamicSmemBytes = SMEM_TC;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 1;
        at[0].val.clusterDim.y = (unsigned)C;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, kern, dst, a);
        if (e == cudaSuccess || C == 1) break;
        (void)cudaGetLastError();      // clear a failed cluster launch, retry smaller
        C = std::max(1, C / 2);
    }
    return e;
}

// Filling the SMs that large clusters leave idle. With one 227 KB CTA per SM a
// cluster of C CTAs needs C free SMs in one GPC, so clusters of 8 occupy only
// 120 of this GPU's 148 SMs. When the main launch uses clusters of 4 or more
// (SHT_FILL_MIN_CLUSTER), a share of the work items (the last ones: the
// cheapest items) goes
// to a second launch with small clusters on a low-priority helper stream of
// the device, forked from and joined back into the caller's stream; the two
// launches never wait on each other, and each work item computes exactly
// what it would in one launch. SHT_FILL_FRAC: share of the work items for
// that launch (default 0.06; 0 turns it off); SHT_FILL_CLUSTER: its cluster
// size (default 2).
struct FillCfg { double frac; int cluster; int min_main; };
static FillCfg fill_cfg()
{
    static FillCfg f = [] {
        FillCfg c{0.06, 2, 4};
        if (const char* e = std::getenv("SHT_FILL_FRAC")) c.frac = std::max(0.0, std::min(0.5, std::atof(e)));
        if (const char* e = std::getenv("SHT_FILL_CLUSTER")) c.cluster = std::max(1, std::min(8, std::atoi(e)));
        if (const char* e = std::getenv("SHT_FILL_MIN_CLUSTER")) c.min_main = std::max(2, std::min(16, std::atoi(e)));
        return c;
    }();
    return f;
}
struct FillStream { cudaStream_t s = nullptr; cudaEvent_t fork = nullptr, join = nullptr; bool ok = false, tried = false; };
static FillStream g_fill[64];
static std::mutex g_fill_mu;           // one fork / launch / join sequence at a time (shared events)
static FillStream* fill_stream()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    FillStream& f = g_fill[dev];
    if (!f.tried) {
        f.tried = true;
        int lo = 0, hi = 0;
        f.ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
               cudaStreamCreateWithPriority(&f.s, cudaStreamNonBlocking, lo) == cudaSuccess &&
               cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&f.join, cudaEventDisableTiming) == cudaSuccess;
        if (!f.ok) (void)cudaGetLastError();
    }
    return f.ok ? &f : nullptr;
}

template <bool M2A, bool S2>
static cudaError_t launch_tc(const sht_plan* p, int nwork, void* dst,
                             const TcArgs& a, const char* name, cudaStream_t st)
{
    (void)p;
    auto kern = k_leg_tc<M2A, S2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_TC);
    if (e != cudaSuccess) return e;
    const long long ntiles = (a.ncol + TC_M - 1) / TC_M;
    int C = pick_cluster(ntiles);
    if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        (void)cudaGetLastError();
        C = 8;
    }
    const FillCfg fc = fill_cfg();
    std::unique_lock<std::mutex> lk(g_fill_mu, std::defer_lock);
    int nB = (fc.frac > 0.0 && C >= fc.min_main && C > fc.cluster) ? (int)(fc.frac * nwork + 0.5) : 0;
    if (nB > 0) lk.lock();
    FillStream* fs = (nB > 0) ? fill_stream() : nullptr;
    if (!fs) nB = 0;
    prof_start(name, st);
    if (nB > 0) {
        if ((e = cudaEventRecord(fs->fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(fs->s, fs->fork, 0)) != cudaSuccess) return e;
    }
    e = launch_grid<M2A, S2>(nwork - nB, C, dst, a, st);
    if (e == cudaSuccess && nB > 0) {
        TcArgs b = a;
        b.work = a.work + (nwork - nB);
        e = launch_grid<M2A, S2>(nB, fc.cluster, dst, b, fs->s);
        if (e == cudaSuccess) e = cudaEventRecord(fs->join, fs->s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, fs->join, 0);
        count_launch();
    }
    prof_stop(st);
    count_launch();
    return e;
}

// (the slicing pass writes the image that the contraction then reads, in stream order)
cudaError_t launch_legendre_m2a_tc(const sht_plan* p, const float2* T, const float* colmax, uint8_t* img,
                                   double* alm, int nmaps, double fs0, double fs1, cudaStream_t st, int csel)
{
    if (p->s.nwork_m2a == 0) return cudaSuccess;
    TcArgs a = make_tc(p, nmaps, colmax, p->s.Q_m2a);
    if (csel) {                      // one spin-2 component: half the columns
        a.csel = csel;
        a.ncol = a.pcol / 2;
        a.ntile = (int)((a.ncol + TC_M - 1) / TC_M);
    }
    a.fs0 = fs0; a.fs1 = fs1;
    a.work = p->s.work_m2a;
    a.img = img; a.img_base = p->s.img_base_m2a; a.sunits = p->s.sunits_m2a;
    cudaError_t e;
    if (p->spin) {
        e = launch_slice<true, true>(p->s.nsunits_m2a, T, img, a, "k_slice_m2a_s2", st);
        if (e == cudaSuccess) e = launch_tc<true, true>(p, p->s.nwork_m2a, alm, a, "k_leg_m2a_tc_s2", st);
    } else {
        e = launch_slice<true, false>(p->s.nsunits_m2a, T, img, a, "k_slice_m2a", st);
        if (e == cudaSuccess) e = launch_tc<true, false>(p, p->s.nwork_m2a, alm, a, "k_leg_m2a_tc", st);
    }
    return e;
}

cudaError_t launch_legendre_a2m_tc(const sht_plan* p, const float2* A2, const float* colmax, uint8_t* img,
                                   float* G, int nmaps, float s0, float s1, cudaStream_t st)
{
    if (p->s.nwork_a2m == 0) return cudaSuccess;
    TcArgs a = make_tc(p, nmaps, colmax, p->s.Q_a2m);
    a.s0 = s0; a.s1 = s1;
    a.work = p->s.work_a2m;
    a.img = img; a.img_base = p->s.img_base_a2m; a.sunits = p->s.sunits_a2m;
    cudaError_t e;
    if (p->spin) {
        e = launch_slice<false, true>(p->s.nsunits_a2m, A2, img, a, "k_slice_a2m_s2", st);
        if (e == cudaSuccess) e = launch_tc<false, true>(p, p->s.nwork_a2m, G, a, "k_leg_a2m_tc_s2", st);
    } else {
        e = launch_slice<false, false>(p->s.nsunits_a2m, A2, img, a, "k_slice_a2m", st);
        if (e == cudaSuccess) e = launch_tc<false, false>(p, p->s.nwork_a2m, G, a, "k_leg_a2m_tc", st);
    }
    return e;
}

// bytes of the pre-sliced data image of one contraction (the larger direction)
size_t split_img_bytes(const sht_plan* p, int nmaps)
{
    const long long ntile = (ncols(p, nmaps) + TC_M - 1) / TC_M;
    const long long nch = std::max(p->s.img_chunks_m2a, p->s.img_chunks_a2m);
    return (size_t)(nch * ntile) * (size_t)A_BYTES;
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
    if (p->spin) {
        k_split_tables_s2<<<(unsigned)(p->mmax + 1), 256>>>(a, d_ck_base, p->s.ck, p->s.ck_exp, p->t.seed_mant,
                                                             p->t.seed_exp, p->s.rowmax_bits, p->s.pairmax);
    } else {
        dim3 grid((unsigned)(p->mmax + 1), 2);
        k_split_tables<<<grid, 256>>>(a, d_ck_base, p->s.ck, p->s.ck_exp, p->t.seed_mant, p->t.seed_exp,
                                      p->s.rowmax_bits, p->s.pairmax);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

int split_row_tile() { return TC_N; }
// ring-pair tiles one alm2map CTA walks in one pipeline
int split_a2m_tiles() { return 8; }
int split_ck_rows() { return CK_ROWS; }
int split_col_tile() { return TC_M; }

}  // namespace sht
