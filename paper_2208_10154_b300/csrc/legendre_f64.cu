// legendre_f64.cu -- FP64 form of the Legendre contraction (Sec. 2.2
// equ:matrix form; spin 2: Sec. 2.3 equ:aeab mat form and its transpose),
// with lambda generated on the fly per (m, ring tile) from resident seeds and
// recurrence coefficients, so the Legendre matrix never lands in HBM.
//
// Slot convention (see common.cuh): for spin 0, slot q holds rows / K entries
// with (l - m) % 2 == q and uses T_q. For spin 2 (F+- = -(2lambda +- -2lambda)/2):
//   map2alm  slot q rows (l-m)%2 == q:  A = F+ T_q + F- perm(T_{1-q})
//   alm2map  slot q:  G_q = sum_{(l-m)%2==q} F+ a + sum_{(l-m)%2!=q} F- perm(a)
// with perm(Qr,Qi,Ur,Ui) = (-Ui,Ur,Qi,-Qr) (E/B coupling through i U, Sec. 2.3).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace sht {

// v * 2^E as a double (0 far below the double range)
__device__ __forceinline__ double scale2(double v, int E)
{
    if (E >= -1022) {
        if (E > 1023) E = 1023;
        return v * __longlong_as_double((long long)(E + 1023) << 52);
    }
    if (E < -2100) return 0.0;
    double t = v * __longlong_as_double((long long)(-1000 + 1023) << 52);
    int E2 = E + 1000;
    if (E2 < -1022) return 0.0;
    return t * __longlong_as_double((long long)(E2 + 1023) << 52);
}

constexpr double RESCALE_UP = 0x1p500;
constexpr double RESCALE_DN = 0x1p-500;

struct LegArgs {
    const int4* work;            // (m, q, tile, 0)
    const PairGeom* pairs;
    const double* seed_mant;
    const int* seed_exp;
    const double *ra, *rb, *rc;
    const double *wA0, *wAB0, *wC0, *wA1, *wAB1, *wC1;
    int spin, lmax, mmax, R;
    long long ncol, nalm;
    int ncomp;
    double scale;      // output scale for m > 0
    double scale0;     // output scale for m = 0
    int accum;         // map2alm: add into alm instead of overwriting
    // spin-2 map2alm of one component: csel = 1 (E) / 2 (B) keeps the two
    // columns per map that form it (ncol = output columns); pcol = columns
    // of T. csel = 0: pcol = ncol.
    long long pcol;
    int csel;
    // checkpoints of the recurrences (FP64 plans; null: walk from the seeds)
    const double2* ck64;
    const int* ck64_exp;
    const int* ck64_off;
    // ring optimisation: first ring pair of order m with a non-negligible
    // lambda (a multiple of 32; null: 0)
    const int* pfirst;
};

__device__ __forceinline__ long long d_alm_index(int lmax, int l, int m)
{
    return (long long)m * (2 * lmax + 1 - m) / 2 + l;
}

// ---------------------------------------------------------------------------
// map2alm: a[l, c] (rows l = m + q + 2 r) = sum_k Lambda[l, k] B[k, c]
// CTA tile: 128 rows x 32 cols, K chunk = 32 ring pairs.
// grid.x = work item (m, q, row tile), grid.y = column tile
// ---------------------------------------------------------------------------
constexpr int M2A_TL = 128, M2A_TN = 32, M2A_TK = 32;
constexpr int M2A_TLP = M2A_TL + 1;     // padded row stride of the lambda tile: the
                                        // lanes' stores (one ring pair each) hit distinct banks
// two buffers of (lambda + data) per type (spin 2: two types)
__host__ __device__ constexpr int m2a_smem(int spin, int tn)
{
    return 2 * (spin ? 2 : 1) * (M2A_TK * M2A_TLP + M2A_TK * tn) * (int)sizeof(double);
}
// column tiles: 32 (map2alm) / 64 (alm2map) map columns per CTA, 4 / 8 for
// batches of at most that many columns (one map or one Q/U pair)
constexpr int M2A_TN_SMALL = 4, A2M_TN_SMALL = 8;

// One step of each recurrence. The checkpoint walk at plan time and the
// kernels run these same operations, so a chain resumed from a checkpoint
// gives the values of the serial walk bit for bit.
// spin 0, row r -> r + 1 of slot q (ci = index of l = m + q + 2r)
__device__ __forceinline__ void step0(const double* ra, const double* rb, const double* rc, long long ci, double x2,
                                      double& cur, double& prev, int& E)
{
    const double t = fma(ra[ci], x2, rb[ci]);
    const double nxt = fma(t, cur, rc[ci] * prev);
    prev = cur;
    cur = nxt;
    if (fabs(cur) > RESCALE_UP) { cur *= RESCALE_DN; prev *= RESCALE_DN; E += 500; }
}
// spin 2, one of s = +-2: l - 1 -> l (ci = index of l)
__device__ __forceinline__ void step2(const double* A, const double* AB, const double* C, long long ci, double x,
                                      double& cur, double& prev, int& E)
{
    const double t = fma(A[ci], x, AB[ci]);
    const double nxt = fma(t, cur, -C[ci] * prev);
    prev = cur;
    cur = nxt;
    if (fabs(cur) > RESCALE_UP) { cur *= RESCALE_DN; prev *= RESCALE_DN; E += 500; }
}

// Roles: warps 0-3 produce the next K chunk (lambda rows from the
// checkpoints, the data tile) into one buffer while warps 4-7 run the FMAs of
// the current chunk from the other, 8 rows x 4 columns per thread, so the
// recurrence's FP64 latency overlaps the contraction (each output sums its
// products in the same order as a single-buffered tile would).
template <int TN>
__global__ void __launch_bounds__(256, 2)
k_leg_m2a_f64(const double* __restrict__ T, double* __restrict__ alm, LegArgs a)
{
    extern __shared__ __align__(16) double sm[];
    const int4 w = a.work[blockIdx.x];
    const int m = w.x, q = w.y, rt = w.z;
    const int tid = threadIdx.x;
    const int c0 = blockIdx.y * TN;
    const int l_first = m + q;
    const int nrows = (a.lmax >= l_first) ? (a.lmax - l_first) / 2 + 1 : 0;
    const int r0 = rt * M2A_TL;
    const int ntypes = a.spin ? 2 : 1;
    // buffer b, type t: lambda [TK][TLP], data [TK][TN]
    double* const lam0 = sm;
    double* const dat0 = sm + 2 * ntypes * M2A_TK * M2A_TLP;
    auto lam_buf = [&](int b, int t) { return lam0 + (long long)(b * ntypes + t) * M2A_TK * M2A_TLP; };
    auto dat_buf = [&](int b, int t) { return dat0 + (long long)(b * ntypes + t) * M2A_TK * TN; };
    const long long qstride = (long long)a.R * a.pcol;     // T holds every data column
    const double* Tq = T + ((long long)m * 2 + q) * qstride;
    const double* To = T + ((long long)m * 2 + (1 - q)) * qstride;
    const bool producer = tid < 128;
    const int ct = tid - 128;                   // consumer thread
    // TN / 4 column groups of 4; rows ty + RG i, i < RPT
    constexpr int CG = TN / 4, RG = 128 / CG, RPT = M2A_TL / RG;
    const int tx = ct % CG, ty = ct / CG;
    double acc[RPT][4];
#pragma unroll
    for (int i = 0; i < RPT; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

    // the producers' part: chunk k0 into buffer b
    auto produce = [&](int k0, int b) {
        // ---- lambda tile: warp v < 4 holds the rows rb = r0 + 32 v .. rb + 31
        // of the 32 ring pairs (one per lane), resuming each chain from its
        // checkpoint at row rb (the seed at row 0) ----
        {
            const int lane = tid & 31;
            const int rb = r0 + 32 * (tid >> 5);
            const int bk = rb >> 5;
            const int p = k0 + lane;
            const bool valid = p < a.R;
            const bool live = valid && rb < nrows;
            const double x = valid ? a.pairs[p].x : 0.0;
            double* l0row = lam_buf(b, 0) + (long long)lane * M2A_TLP + (rb - r0);
            if (a.spin == 0) {
                double cur = 0.0, prev = 0.0;
                int E = 0;
                const double x2 = x * x;
                if (live) {
                    if (bk > 0 && a.ck64) {
                        const long long ci = (long long)(a.ck64_off[m * 2 + q] + bk - 1) * a.R + p;
                        const double2 v = a.ck64[ci];
                        cur = v.x; prev = v.y; E = a.ck64_exp[ci];
                    } else {
                        const long long si = ((long long)m * 2 + q) * a.R + p;
                        cur = a.seed_mant[si];
                        E = a.seed_exp[si];
                        for (int r = 0; r < rb; r++)             // (plans without checkpoints)
                            step0(a.ra, a.rb, a.rc, d_alm_index(a.lmax, l_first + 2 * r, m), x2, cur, prev, E);
                    }
                }
                for (int i = 0; i < 32; i++) {
                    const int r = rb + i;
                    l0row[i] = (r < nrows) ? scale2(cur, E) : 0.0;
                    if (i + 1 < 32 && r + 1 < nrows)
                        step0(a.ra, a.rb, a.rc, d_alm_index(a.lmax, l_first + 2 * r, m), x2, cur, prev, E);
                }
            } else {
                // spin 2: walk every l from the start state; rows are l with (l-m)%2 == q
                double* l1row = lam_buf(b, 1) + (long long)lane * M2A_TLP + (rb - r0);
                const int l0 = m > 2 ? m : 2;
                double c2 = 0.0, p2 = 0.0, c3 = 0.0, p3 = 0.0;   // s=+2: cur, prev; s=-2: cur, prev
                int E2 = 0, E3 = 0;
                int ls = l0;                                     // l of the state
                if (live) {
                    if (bk > 0 && a.ck64) {
                        const long long ci = (long long)(a.ck64_off[m] + bk - 1) * a.R + p;
                        const double2 v2 = a.ck64[2 * ci], v3 = a.ck64[2 * ci + 1];
                        c2 = v2.x; p2 = v2.y; c3 = v3.x; p3 = v3.y;
                        E2 = a.ck64_exp[2 * ci]; E3 = a.ck64_exp[2 * ci + 1];
                        ls = m + 64 * bk;
                    } else {
                        long long si = ((long long)m * 2 + 0) * a.R + p;
                        c2 = a.seed_mant[si]; E2 = a.seed_exp[si];
                        si = ((long long)m * 2 + 1) * a.R + p;
                        c3 = a.seed_mant[si]; E3 = a.seed_exp[si];
                    }
                    const int lend = min(a.lmax, l_first + 2 * (rb + 31));
                    for (int l = ls; l <= lend; l++) {
                        if (l > ls) {
                            const long long ci = d_alm_index(a.lmax, l, m);
                            step2(a.wA0, a.wAB0, a.wC0, ci, x, c2, p2, E2);
                            step2(a.wA1, a.wAB1, a.wC1, ci, x, c3, p3, E3);
                        }
                        if (((l - m) & 1) == q && l >= l_first) {
                            const int r = (l - l_first) >> 1;
                            if (r >= rb) {
                                const double v2 = scale2(c2, E2), v3 = scale2(c3, E3);
                                l0row[r - rb] = -0.5 * (v2 + v3);
                                l1row[r - rb] = -0.5 * (v2 - v3);
                            }
                        }
                    }
                }
                // rows not produced above (l < l0 or beyond lmax) are zero
                for (int i = 0; i < 32; i++) {
                    const int l = l_first + 2 * (rb + i);
                    if (l < l0 || l > a.lmax || !live) {
                        l0row[i] = 0.0;
                        l1row[i] = 0.0;
                    }
                }
            }
        }
        // ---- data tile ----
        double* d0 = dat_buf(b, 0);
        double* d1 = a.spin ? dat_buf(b, 1) : nullptr;
        for (int i = tid; i < M2A_TK * TN; i += 128) {
            int k = i / TN, c = i % TN;
            int p = k0 + k;
            long long cg = c0 + c;
            double v0 = 0.0, v1 = 0.0;
            if (p < a.R && cg < a.ncol) {
                const long long pc = a.csel == 0 ? cg : ((cg >> 1) << 2) + (cg & 1) + (a.csel == 2 ? 2 : 0);
                v0 = Tq[(long long)p * a.pcol + pc];
                if (a.spin) {
                    long long base = pc & ~3LL;
                    int wsel = (int)(pc & 3);
                    const double* o = To + (long long)p * a.pcol + base;
                    v1 = (wsel == 0) ? -o[3] : (wsel == 1) ? o[2] : (wsel == 2) ? o[1] : -o[0];
                }
            }
            d0[k * TN + c] = v0;
            if (a.spin) d1[k * TN + c] = v1;
        }
    };

    // (ring pairs before pb hold negligible lambda for this order)
    const int pb = a.pfirst ? a.pfirst[m] : 0;
    const int nch = (a.R - pb + M2A_TK - 1) / M2A_TK;
    if (producer) produce(pb, 0);
    __syncthreads();
    for (int ch = 0; ch < nch; ch++) {
        const int cb = ch & 1;
        if (producer) {
            if (ch + 1 < nch) produce(pb + (ch + 1) * M2A_TK, cb ^ 1);
        } else {
            // row groups i with RG i >= nv hold no row of the tile (short last
            // tiles at high m): skipped, block-uniformly
            const int nv = nrows - r0;
            for (int t = 0; t < ntypes; t++) {
                const double* L = lam_buf(cb, t);
                const double* D = dat_buf(cb, t);
#pragma unroll 4
                for (int k = 0; k < M2A_TK; k++) {
                    double lv[RPT], dv[4];
#pragma unroll
                    for (int i = 0; i < RPT; i++) lv[i] = (RG * i < nv) ? L[k * M2A_TLP + ty + RG * i] : 0.0;
#pragma unroll
                    for (int j = 0; j < 4; j++) dv[j] = D[k * TN + tx * 4 + j];
#pragma unroll
                    for (int i = 0; i < RPT; i++)
                        if (RG * i < nv)
#pragma unroll
                            for (int j = 0; j < 4; j++) acc[i][j] = fma(lv[i], dv[j], acc[i][j]);
                }
            }
        }
        __syncthreads();
    }
    if (producer) return;
    // ---- write a_lm ----
#pragma unroll
    for (int i = 0; i < RPT; i++) {
        int r = r0 + ty + RG * i;
        if (r >= nrows) continue;
        int l = l_first + 2 * r;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            long long cg = c0 + tx * 4 + j;
            if (cg >= a.ncol) continue;
            long long mc = cg >> 1;           // map * ncomp + comp
            int reim = (int)(cg & 1);
            double v = (m == 0 ? a.scale0 : a.scale) * acc[i][j];
            if ((m == 0 && reim) || (a.spin && l < 2)) v = 0.0;
            double* dst = alm + (mc * a.nalm + d_alm_index(a.lmax, l, m)) * 2 + reim;
            if (a.accum) *dst += v; else *dst = v;
        }
    }
}

// ---------------------------------------------------------------------------
// alm2map: G[m][q][p][c] = sum_k Lambda[k, p] B[k, c]
// CTA tile: 64 ring pairs x 64 cols, K chunk = 32 values of l.
// grid.x = work item (m, q, pair tile), grid.y = column tile
// ---------------------------------------------------------------------------
constexpr int A2M_TP = 64, A2M_TN = 64, A2M_TK = 32;

// Roles as in map2alm: warps 0-3 produce the next chunk (threads 0-63 step
// the lambda chains of the tile's ring pairs, all four warps load the a_lm
// tile) while warps 4-7 run the FMAs of the current one, 8 ring pairs x 4
// columns per thread.
template <int TN>
__global__ void __launch_bounds__(256, 2)
k_leg_a2m_f64(const double* __restrict__ alm, double* __restrict__ G, LegArgs a)
{
    extern __shared__ __align__(16) double sm[];
    // buffer b: lambda [TK][TP] at sm + b * TK * TP, data [TK][TN] after both
    double* const lam0 = sm;
    double* const dat0 = sm + 2 * A2M_TK * A2M_TP;
    const int4 w = a.work[blockIdx.x];
    const int m = w.x, q = w.y, pt = w.z;
    const int tid = threadIdx.x;
    const int c0 = blockIdx.y * TN;
    const int p0 = pt * A2M_TP;
    const long long qstride = (long long)a.R * a.ncol;
    const bool producer = tid < 128;
    const int ct = tid - 128;                    // consumer thread
    // TN / 4 column groups of 4; ring pairs ty + PG i, i < PPT
    constexpr int CG = TN / 4, PG = 128 / CG, PPT = A2M_TP / PG;
    const int tx = ct % CG, ty = ct / CG;
    double acc[PPT][4];
#pragma unroll
    for (int i = 0; i < PPT; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

    int lk0, lstep, K;
    if (a.spin == 0) {
        lk0 = m + q; lstep = 2;
        K = (a.lmax >= lk0) ? (a.lmax - lk0) / 2 + 1 : 0;
    } else {
        lk0 = m > 2 ? m : 2; lstep = 1;
        K = (a.lmax >= lk0) ? a.lmax - lk0 + 1 : 0;
    }
    // a tile of ring pairs that all hold negligible lambda for this order
    // writes zeros (the ring optimisation)
    if (a.pfirst && p0 + A2M_TP <= a.pfirst[m]) K = 0;
    // chain state (threads 0..63: one ring pair each, carried across chunks)
    double c2 = 0.0, p2 = 0.0, c3 = 0.0, p3 = 0.0;
    int E2 = 0, E3 = 0;
    double x = 0.0;
    const int myp = p0 + tid;
    if (tid < A2M_TP && myp < a.R) {
        x = a.pairs[myp].x;
        if (a.spin == 0) {
            long long si = ((long long)m * 2 + q) * a.R + myp;
            c2 = a.seed_mant[si]; E2 = a.seed_exp[si];
        } else {
            long long si = ((long long)m * 2 + 0) * a.R + myp;
            c2 = a.seed_mant[si]; E2 = a.seed_exp[si];
            si = ((long long)m * 2 + 1) * a.R + myp;
            c3 = a.seed_mant[si]; E3 = a.seed_exp[si];
        }
    }
    const double x2 = x * x;
    auto produce = [&](int k0, int b) {
        double* lam = lam0 + b * A2M_TK * A2M_TP;
        double* dat = dat0 + b * A2M_TK * TN;
        if (tid < A2M_TP) {
            const bool valid = myp < a.R;
            for (int kk = 0; kk < A2M_TK; kk++) {
                int k = k0 + kk;
                double v = 0.0;
                if (k < K && valid) {
                    int l = lk0 + lstep * k;
                    if (a.spin == 0) {
                        v = scale2(c2, E2);
                        if (k + 1 < K) step0(a.ra, a.rb, a.rc, d_alm_index(a.lmax, l, m), x2, c2, p2, E2);
                    } else {
                        if (k > 0) {
                            const long long ci = d_alm_index(a.lmax, l, m);
                            step2(a.wA0, a.wAB0, a.wC0, ci, x, c2, p2, E2);
                            step2(a.wA1, a.wAB1, a.wC1, ci, x, c3, p3, E3);
                        }
                        double v2 = scale2(c2, E2), v3 = scale2(c3, E3);
                        v = (((l - m) & 1) == q) ? -0.5 * (v2 + v3) : -0.5 * (v2 - v3);
                    }
                }
                lam[kk * A2M_TP + tid] = v;
            }
        }
        // data tile: a[l][c] (or perm(a) for spin-2 rows of the other parity)
        for (int i = tid; i < A2M_TK * TN; i += 128) {
            int kk = i / TN, c = i % TN;
            int k = k0 + kk;
            long long cg = c0 + c;
            double v = 0.0;
            if (k < K && cg < a.ncol) {
                int l = lk0 + lstep * k;
                long long li = d_alm_index(a.lmax, l, m);
                if (a.spin == 0) {
                    long long mc = cg >> 1;
                    int reim = (int)(cg & 1);
                    v = (m == 0 && reim) ? 0.0 : alm[(mc * a.nalm + li) * 2 + reim];
                } else {
                    long long mp = cg >> 2;
                    int wsel = (int)(cg & 3);
                    bool perm = ((l - m) & 1) != q;
                    int src = wsel; double sg = 1.0;
                    if (perm) {   // (Er, Ei, Br, Bi) -> (-Bi, Br, Ei, -Er)
                        src = 3 - wsel;
                        sg = (wsel == 0 || wsel == 3) ? -1.0 : 1.0;
                    }
                    int comp = src >> 1, reim = src & 1;
                    v = (m == 0 && reim) ? 0.0
                        : sg * alm[((mp * 2 + comp) * a.nalm + li) * 2 + reim];
                }
            }
            dat[kk * TN + c] = v;
        }
    };

    const int nch = (K + A2M_TK - 1) / A2M_TK;
    if (producer && nch > 0) produce(0, 0);
    __syncthreads();
    for (int ch = 0; ch < nch; ch++) {
        const int cb = ch & 1;
        if (producer) {
            if (ch + 1 < nch) produce((ch + 1) * A2M_TK, cb ^ 1);
        } else {
            const double* lam = lam0 + cb * A2M_TK * A2M_TP;
            const double* dat = dat0 + cb * A2M_TK * TN;
            const int kn = min(A2M_TK, K - ch * A2M_TK);     // (the last chunk's rest is zero)
#pragma unroll 4
            for (int kk = 0; kk < kn; kk++) {
                double lv[PPT], dv[4];
#pragma unroll
                for (int i = 0; i < PPT; i++) lv[i] = lam[kk * A2M_TP + ty + PG * i];
#pragma unroll
                for (int j = 0; j < 4; j++) dv[j] = dat[kk * TN + tx * 4 + j];
#pragma unroll
                for (int i = 0; i < PPT; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = fma(lv[i], dv[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
    if (producer) return;
    double* Gq = G + ((long long)m * 2 + q) * qstride;
    const double gs = (m == 0) ? a.scale0 : a.scale;
#pragma unroll
    for (int i = 0; i < PPT; i++) {
        int p = p0 + ty + PG * i;
        if (p >= a.R) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            long long cg = c0 + tx * 4 + j;
            if (cg < a.ncol) Gq[(long long)p * a.ncol + cg] = gs * acc[i][j];
        }
    }
}

// ---------------------------------------------------------------------------
static LegArgs make_args(const sht_plan* p, int nmaps, double scale0, double scale, const int4* work)
{
    LegArgs a;
    a.work = work;
    a.pairs = p->t.pairs;
    a.seed_mant = p->t.seed_mant;
    a.seed_exp = p->t.seed_exp;
    a.ra = p->t.rec_a; a.rb = p->t.rec_b; a.rc = p->t.rec_c;
    a.wA0 = p->t.w_A[0]; a.wAB0 = p->t.w_AB[0]; a.wC0 = p->t.w_C[0];
    a.pfirst = p->t.pfirst64;
    a.wA1 = p->t.w_A[1]; a.wAB1 = p->t.w_AB[1]; a.wC1 = p->t.w_C[1];
    a.spin = p->spin; a.lmax = p->lmax; a.mmax = p->mmax; a.R = p->R;
    a.ncol = ncols(p, nmaps); a.nalm = p->nalm; a.ncomp = p->ncomp;
    a.scale = scale;
    a.scale0 = scale0;
    a.accum = 0;
    a.pcol = a.ncol;
    a.csel = 0;
    a.ck64 = p->t.ck64;
    a.ck64_exp = p->t.ck64_exp;
    a.ck64_off = p->t.ck64_off;
    return a;
}

// work items [w0, w0 + nwork) of the plan's list (the list runs over m in
// order, so one order's items are one range); accum adds into alm
// one map2alm launch over work items [w0, w0 + nwork) with the column tile TN
template <int TN>
static cudaError_t launch_m2a_tn(const LegArgs& a, const double* T, double* alm, int nwork, int spin,
                                 cudaStream_t st)
{
    const size_t sm = (size_t)m2a_smem(spin, TN);
    cudaError_t e = cudaFuncSetAttribute(k_leg_m2a_f64<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)nwork, (unsigned)((a.ncol + TN - 1) / TN));
    prof_start("k_leg_m2a_f64", st);
    k_leg_m2a_f64<TN><<<grid, 256, sm, st>>>(T, alm, a);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}
static cudaError_t launch_m2a(const LegArgs& a, const double* T, double* alm, int nwork, int spin, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    return a.ncol <= M2A_TN_SMALL ? launch_m2a_tn<M2A_TN_SMALL>(a, T, alm, nwork, spin, st)
                                  : launch_m2a_tn<M2A_TN>(a, T, alm, nwork, spin, st);
}

// work items [w0, w0 + nwork) of the plan's list (the list runs over m in
// order, so one order's items are one range); accum adds into alm
static cudaError_t launch_m2a_range(const sht_plan* p, const double* T, double* alm, int nmaps, double scale0,
                                    double scale, int w0, int nwork, bool accum, cudaStream_t st)
{
    LegArgs a = make_args(p, nmaps, scale0, scale, p->work_m2a + w0);
    a.accum = accum ? 1 : 0;
    return launch_m2a(a, T, alm, nwork, p->spin, st);
}

cudaError_t launch_legendre_m2a_f64(const sht_plan* p, const double* T, double* alm, int nmaps,
                                    double scale0, double scale, cudaStream_t st)
{
    return launch_m2a_range(p, T, alm, nmaps, scale0, scale, 0, p->nwork_m2a, false, st);
}

cudaError_t launch_legendre_m2a_f64_comp(const sht_plan* p, const double* T, double* alm, int nmaps,
                                         double scale0, double scale, int csel, cudaStream_t st)
{
    LegArgs a = make_args(p, nmaps, scale0, scale, p->work_m2a);
    a.csel = csel;
    a.ncol = a.pcol / 2;
    return launch_m2a(a, T, alm, p->nwork_m2a, p->spin, st);
}

cudaError_t launch_legendre_m2a_f64_order(const sht_plan* p, const double* T, double* alm, int nmaps,
                                          double scale0, double scale, int m0, int nm, bool accum, cudaStream_t st)
{
    const int w0 = p->m2a_off[m0];
    return launch_m2a_range(p, T, alm, nmaps, scale0, scale, w0, p->m2a_off[m0 + nm] - w0, accum, st);
}

template <int TN>
static cudaError_t launch_a2m_tn(const LegArgs& a, const double* alm, double* G, int nwork, cudaStream_t st)
{
    const size_t sm = (size_t)(2 * (A2M_TK * A2M_TP + A2M_TK * TN)) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_leg_a2m_f64<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)nwork, (unsigned)((a.ncol + TN - 1) / TN));
    prof_start("k_leg_a2m_f64", st);
    k_leg_a2m_f64<TN><<<grid, 256, sm, st>>>(alm, G, a);
    prof_stop(st);
    count_launch();
    return cudaGetLastError();
}

static cudaError_t launch_a2m_range(const sht_plan* p, const double* alm, double* G, int nmaps, double scale0,
                                    double scale, int w0, int nwork, cudaStream_t st)
{
    if (nwork <= 0) return cudaSuccess;
    const LegArgs a = make_args(p, nmaps, scale0, scale, p->work_a2m + w0);
    return a.ncol <= A2M_TN_SMALL ? launch_a2m_tn<A2M_TN_SMALL>(a, alm, G, nwork, st)
                                  : launch_a2m_tn<A2M_TN>(a, alm, G, nwork, st);
}

cudaError_t launch_legendre_a2m_f64(const sht_plan* p, const double* alm, double* G, int nmaps,
                                    double scale0, double scale, cudaStream_t st)
{
    return launch_a2m_range(p, alm, G, nmaps, scale0, scale, 0, p->nwork_a2m, st);
}

cudaError_t launch_legendre_a2m_f64_order(const sht_plan* p, const double* alm, double* G, int nmaps, int m0,
                                          int nm, cudaStream_t st)
{
    const int w0 = p->a2m_off[m0];
    return launch_a2m_range(p, alm, G, nmaps, 1.0, 1.0, w0, p->a2m_off[m0 + nm] - w0, st);
}

// ---------------------------------------------------------------------------
// plan-time walk of every chain the map2alm kernel resumes mid-tile (the
// layout of DevTables::ck64): spin 0, thread (p, m, q); spin 2, thread (p, m)
// ---------------------------------------------------------------------------
// (and live[(m * 2 + q) * R + p] = 1 where some |lambda| of the chain reaches
// SPLIT_LAMBDA_EPS: the ring optimisation's first pairs)
__global__ void k_ck64(LegArgs a, double2* __restrict__ ck, int* __restrict__ cke, char* __restrict__ live)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y, q = blockIdx.z;
    if (p >= a.R) return;
    const double x = a.pairs[p].x;
    const double eps = (double)SPLIT_LAMBDA_EPS;
    bool lv = false;
    if (a.spin == 0) {
        const int l_first = m + q;
        const int nrows = (a.lmax >= l_first) ? (a.lmax - l_first) / 2 + 1 : 0;
        const long long si = ((long long)m * 2 + q) * a.R + p;
        double cur = a.seed_mant[si], prev = 0.0;
        int E = a.seed_exp[si];
        const double x2 = x * x;
        const int o = a.ck64_off[m * 2 + q];
        if (nrows > 0) lv = fabs(scale2(cur, E)) >= eps;
        for (int r = 0; r + 1 < nrows; r++) {
            step0(a.ra, a.rb, a.rc, d_alm_index(a.lmax, l_first + 2 * r, m), x2, cur, prev, E);
            lv = lv || fabs(scale2(cur, E)) >= eps;
            if (((r + 1) & 31) == 0) {
                const long long i = (long long)(o + ((r + 1) >> 5) - 1) * a.R + p;
                ck[i] = make_double2(cur, prev);
                cke[i] = E;
            }
        }
    } else {
        if (q) return;
        const int l0 = m > 2 ? m : 2;
        long long si = ((long long)m * 2 + 0) * a.R + p;
        double c2 = a.seed_mant[si], p2 = 0.0;
        int E2 = a.seed_exp[si];
        si = ((long long)m * 2 + 1) * a.R + p;
        double c3 = a.seed_mant[si], p3 = 0.0;
        int E3 = a.seed_exp[si];
        const int o = a.ck64_off[m];
        if (a.lmax >= l0) lv = fabs(scale2(c2, E2)) >= eps || fabs(scale2(c3, E3)) >= eps;
        for (int l = l0 + 1; l <= a.lmax; l++) {
            const long long ci = d_alm_index(a.lmax, l, m);
            step2(a.wA0, a.wAB0, a.wC0, ci, x, c2, p2, E2);
            step2(a.wA1, a.wAB1, a.wC1, ci, x, c3, p3, E3);
            lv = lv || fabs(scale2(c2, E2)) >= eps || fabs(scale2(c3, E3)) >= eps;
            if (((l - m) & 63) == 0) {                  // l = m + 64 b, b >= 1 (l > l0 >= m)
                const long long i = (long long)(o + ((l - m) >> 6) - 1) * a.R + p;
                ck[2 * i] = make_double2(c2, p2);
                ck[2 * i + 1] = make_double2(c3, p3);
                cke[2 * i] = E2;
                cke[2 * i + 1] = E3;
            }
        }
    }
    live[((long long)m * 2 + q) * a.R + p] = lv ? 1 : 0;
}

cudaError_t build_f64_checkpoints(sht_plan* p, size_t* acc)
{
    const int lmax = p->lmax, mmax = p->mmax;
    std::vector<int> off;
    long long n = 0;                                   // checkpoints per ring pair
    if (p->spin == 0) {
        for (int m = 0; m <= mmax; m++)
            for (int q = 0; q < 2; q++) {
                const int nrows = (lmax >= m + q) ? (lmax - m - q) / 2 + 1 : 0;
                off.push_back((int)n);
                n += std::max(0, (nrows + 31) / 32 - 1);
            }
    } else {
        for (int m = 0; m <= mmax; m++) {
            off.push_back((int)n);
            n += (lmax - m) / 64;
        }
    }
    const long long ne = n * p->R * (p->spin ? 2 : 1);
    cudaError_t e;
    if ((e = cudaMalloc(&p->t.ck64_off, off.size() * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(p->t.ck64_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    *acc += off.size() * sizeof(int);
    if (ne > 0) {
        if ((e = cudaMalloc(&p->t.ck64, (size_t)ne * sizeof(double2))) != cudaSuccess) return e;
        if ((e = cudaMalloc(&p->t.ck64_exp, (size_t)ne * sizeof(int))) != cudaSuccess) return e;
        *acc += (size_t)ne * (sizeof(double2) + sizeof(int));
    }
    // (with no checkpoints, no chain is long enough to write one)
    const size_t nlive = (size_t)(mmax + 1) * 2 * p->R;
    char* d_live = nullptr;
    if ((e = cudaMalloc(&d_live, nlive)) != cudaSuccess) return e;
    cudaMemset(d_live, 0, nlive);
    LegArgs a = make_args(p, 1, 1.0, 1.0, nullptr);
    dim3 grid((unsigned)((p->R + 127) / 128), (unsigned)(mmax + 1), p->spin ? 1u : 2u);
    k_ck64<<<grid, 128>>>(a, p->t.ck64, p->t.ck64_exp, d_live);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    std::vector<char> lq(nlive);
    if (e == cudaSuccess) e = cudaMemcpy(lq.data(), d_live, nlive, cudaMemcpyDeviceToHost);
    cudaFree(d_live);
    if (e != cudaSuccess || !ring_skip_enabled()) return e;
    // the ring optimisation: first ring pair of each order (either slot live)
    const int R = p->R;
    std::vector<char> live((size_t)(mmax + 1) * R);
    for (int m = 0; m <= mmax; m++)
        for (int q = 0; q < R; q++)
            live[(size_t)m * R + q] = lq[((size_t)m * 2 + 0) * R + q] || lq[((size_t)m * 2 + 1) * R + q];
    ring_first_pairs(p, live);
    if ((e = cudaMalloc(&p->t.pfirst64, p->h_pfirst.size() * sizeof(int))) != cudaSuccess) return e;
    *acc += p->h_pfirst.size() * sizeof(int);
    return cudaMemcpy(p->t.pfirst64, p->h_pfirst.data(), p->h_pfirst.size() * sizeof(int), cudaMemcpyHostToDevice);
}

int legendre_f64_row_tile() { return M2A_TL; }
int legendre_f64_pair_tile() { return A2M_TP; }

}  // namespace sht
