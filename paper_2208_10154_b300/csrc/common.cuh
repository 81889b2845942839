// common.cuh -- internal types shared by the libsht translation units.
//
// Internal data layout (HBM). The Legendre step works per (m, slot q) on the
// "FFT-mapped" ring spectra of Sec. 2.1 (the matrices T_m of equ:mat form def),
// stored m-major so that every (m, q) block is one dense [pair][col] matrix:
//
//   T[m][q][p][c]   m = 0..mmax, q = 0/1, p = ring pair 0..R-1, c = column
//
// Ring pair p joins north ring p+1 and its mirror 4 nside - 1 - p (same
// length and phase offset); pair R-1 = 2 nside - 1 is the equator ring alone.
// With lambda_lm(pi - theta) = (-1)^{l+m} lambda_lm(theta), the ring sum of
// eq:mm splits into  E = T_north + T_south  (slot 0, rows with l+m even) and
// O = T_north - T_south (slot 1, rows with l+m odd). For spin 2 the slot is
// the parity of the output row for F+ (F- has the opposite parity, Sec. 2.3).
// A column c = (map, comp, re/im): c = (map * ncomp + comp) * 2 + reim.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <mutex>

#include "../../include/sht.h"

namespace sht {

// Per ring-pair geometry (north ring of the pair).
struct PairGeom {
    double x;          // cos(theta) of the north ring (>= 0)
    double s;          // sin(theta)
    double phi0;       // phi of the first pixel (0 or pi/N; same for both rings)
    long long start_n; // first pixel of the north ring
    long long start_s; // first pixel of the south ring (-1 for the equator pair)
    int n;             // pixels per ring
    int fft;           // index into the FFT length table
};

// One distinct ring length and its FFT recipe. The FP64 form uses
// power-of-two sizes (p3 = 1); the split form's own table also uses sizes
// M = 3^b 2^a (p3 = 3^b, 2^a >= 64), whichever needs the least work.
struct FftLen {
    int n;             // ring length N
    int m;             // FFT size used (N itself or the Bluestein size)
    int bluestein;     // 1 if N itself is not transformed directly
    long long chirp;   // offset of w_n = exp(-i pi n^2 / N) (n < N) in the chirp table
    long long bhat;    // offset of FFT_M(conj chirp, circular) (digit-reversed order)
    int p3;            // 3^b of M (1: M is a power of two)
    int bexp = 0;      // split form, Bluestein: max_k |filter_k| <= 2^bexp (filter with the 1 / M)
};

struct DevTables {
    PairGeom* pairs = nullptr;      // [R]
    FftLen* fft = nullptr;          // [nfft]
    double2* twiddle = nullptr;     // [fft_max/2]  exp(-2 pi i k / fft_max)
    double2* chirp = nullptr;       // Bluestein chirps
    double2* bhat = nullptr;        // Bluestein filter spectra
    float2* twiddle_f = nullptr;    // FP32 copies for the split form
    float2* chirp_f = nullptr;
    float2* bhat_f = nullptr;
    // lambda seeds: value at the first row of each chain, per pair, as
    // mantissa * 2^exponent. Spin 0: [m][q][p] (l0 = m + q);
    // spin 2: [m][s = +2, -2][p] at l0 = max(m, 2).
    double* seed_mant = nullptr;
    int* seed_exp = nullptr;
    // spin-0 two-step recurrence (same parity), per (m, l) at packed index
    // idx(l,m): lambda_{l+2} = (alpha x^2 + beta) lambda_l + gamma lambda_{l-2}
    double* rec_a = nullptr;
    double* rec_b = nullptr;
    double* rec_c = nullptr;
    // spin-2 three-term recurrence for s = +2 / -2 (Wigner d), per (m, l):
    // sl_l = (A x + AB) sl_{l-1} - C sl_{l-2}
    double* w_A[2] = {nullptr, nullptr};
    double* w_AB[2] = {nullptr, nullptr};
    double* w_C[2] = {nullptr, nullptr};
    // FP64 plans: states of the recurrences above where the FP64 map2alm
    // resumes a chain mid-tile. Spin 0, chain (m, q, p): (value at row 32b,
    // value at row 32b - 1) and the exponent, b >= 1; spin 2, chain (m, p):
    // both recurrences (s = +2, then -2) at l = m + 64b, b >= 1.
    // [off[chain] + b - 1][p] (spin 2: two entries per [..][p]).
    double2* ck64 = nullptr;
    int* ck64_exp = nullptr;
    int* ck64_off = nullptr;       // spin 0: [m][q]; spin 2: [m]
    // FP64 plans, ring optimisation: the first ring pair each order m
    // contracts (a multiple of 32, nondecreasing in m; null: every pair)
    int* pfirst64 = nullptr;
};

// lo parts of the FP32 FFT tables and hi/lo ring phase tables (compensated FFT)
// ring pairs grouped by FFT size (split form: one launch per class)
struct FftClass {
    int m;             // FFT size of the class
    int off, cnt;      // its ring pairs: cls_pairs[off .. off + cnt)
    long long tw;      // split form: offset of its twiddles exp(-2 pi i u / m), u < m / 2
    long long twp;     // split form: offset of its per-pass radix-8 twiddles (float4 units)
    int twp_n;         //   their count
};

struct CompTables {
    int* cls_pairs = nullptr;      // ring pair indices ordered by FFT size class
    float2* twiddle_l = nullptr;
    float2* chirp_l = nullptr;
    float2* bhat_l = nullptr;
    float2* phase_h = nullptr;     // exp(+i pi k / N), k < 2N, per ring length
    float2* phase_l = nullptr;
    long long* phase_off = nullptr;
    // the split form's FFT recipes (sizes 2^a or 3^b 2^a), per-class twiddles
    // and digit-reversed Bluestein filters, FP32 hi/lo
    FftLen* fft_s = nullptr;
    float4* twp = nullptr;         // per-pass radix-8 twiddles (hi re, hi im, lo re, lo im)
    float2* tws_h = nullptr;
    float2* tws_l = nullptr;
    float2* bhs_h = nullptr;
    float2* bhs_l = nullptr;
};

// tables of the split-precision (tensor-core) form
struct SplitTables {
    double* nA = nullptr;          // normalised recurrence per packed (l, m):
    double* nB = nullptr;          //   mu_{l+2} = (nA x^2 + nB) mu_l + mu_{l-2}
    float* nc = nullptr;           //   lambda_l = nc * mu_l
    double* nc64 = nullptr;        //   the same factor in FP64
    float2* nc2 = nullptr;         //   and as an FP32 hi/lo pair
    double2* ck = nullptr;         // recurrence checkpoints every 32 rows [block][p]
    int* ck_exp = nullptr;         //   (spin 2: every 32 l, [block][s][p])
    unsigned int* rowmax_bits = nullptr;   // max_p |lambda_lm| per packed (l, m) (float bits)
    float* pairmax = nullptr;      // max_{l in q} |lambda_lm(theta_p)| per [m][q][p]
    // spin 2: normalised Wigner recurrences mu_l = (s2A x + s2B) mu_{l-1} - mu_{l-2}
    // per s = +2 / -2, with s lambda_l = d_l mu_l (d_l the same for both s)
    double* s2A[2] = {nullptr, nullptr};
    double* s2B[2] = {nullptr, nullptr};
    float2* s2d2 = nullptr;
    double* s2d64 = nullptr;
    int* err = nullptr;            // device error word of the bounded waits
    int4* work_m2a = nullptr; int nwork_m2a = 0;
    int4* work_a2m = nullptr; int nwork_a2m = 0;
    float Q_m2a = 0.0f, Q_a2m = 0.0f;   // integer range of the main slices (K Q^2 <= 2^24)
    // pre-sliced data images (32 KB per 32-wide chunk of K and 128-column tile):
    // first image chunk per [m][q], slicing units (m, q, unit, image chunk) and
    // the image chunks of one contraction, per direction
    int* img_base_m2a = nullptr;
    int* img_base_a2m = nullptr;
    int4* sunits_m2a = nullptr; int nsunits_m2a = 0;
    int4* sunits_a2m = nullptr; int nsunits_a2m = 0;
    long long img_chunks_m2a = 0, img_chunks_a2m = 0;
    // ring optimisation: orders m are contracted only over the ring
    // pairs p >= pfirst[m] (a multiple of 32, nondecreasing in m); the polar
    // pairs before it hold |lambda_lm| < SPLIT_LAMBDA_EPS for every l. mlim[p]:
    // the highest order whose ring spectra pair p takes part in. Null: no
    // ring pair is skipped.
    int* pfirst = nullptr;
    int* mlim = nullptr;
};

// |lambda_lm(theta)| below which an (m, ring pair) term of the split form is
// skipped (lambda peaks at O(1): a dropped term is below 1e-30 of it)
constexpr float SPLIT_LAMBDA_EPS = 1e-30f;

}  // namespace sht

struct sht_plan {
    int nside = 0, lmax = 0, mmax = 0, spin = 0, precision = 0, device = 0;
    int ncomp = 1;
    long long npix = 0, nalm = 0;
    int R = 0;                  // ring pairs = 2 nside
    int fft_max = 0;            // largest power-of-two FFT size
    int nfft = 0;
    sht::DevTables t;
    sht::SplitTables s;
    sht::CompTables c;
    std::vector<sht::PairGeom> h_pairs;
    std::vector<sht::FftLen> h_fft;
    std::vector<sht::FftLen> h_fft_s;       // split form's FFT recipes
    std::vector<sht::FftClass> h_fcls;
    std::vector<int> h_pfirst;              // split form: host copy of s.pfirst (empty: none)
    double terms_kept = 1.0;                // share of the (m, l, ring pair) terms contracted
    size_t table_bytes = 0;
    // Legendre work lists (m, q, tile, 0) for the FP64 kernels
    int4* work_m2a = nullptr; int nwork_m2a = 0;
    int4* work_a2m = nullptr; int nwork_a2m = 0;
    std::vector<int> m2a_off, a2m_off;   // first work item of each order m (mmax + 2 entries)
    // staging for the host-buffer entry points (allocated lazily)
    void* pin_in = nullptr;
    void* pin_out = nullptr;
    size_t pin_in_bytes = 0, pin_out_bytes = 0;
    void* host_ws = nullptr;
    size_t host_ws_bytes = 0;
    void* host_dev_in = nullptr;
    void* host_dev_out = nullptr;
    size_t host_dev_in_bytes = 0, host_dev_out_bytes = 0;
    // the host entry points' copy streams and their events (created lazily)
    cudaStream_t hp_h2d = nullptr, hp_d2h = nullptr;
    cudaEvent_t hp_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // split FFTs: helper streams that run size classes beside the caller's
    // stream, forked and joined with events (made with the plan; one call's
    // fork / launch / join sequence at a time under fft_mu)
    static constexpr int FFT_AUX = 2;
    cudaStream_t fft_aux[FFT_AUX] = {nullptr, nullptr};
    cudaEvent_t fft_fork = nullptr;
    cudaEvent_t fft_join[FFT_AUX] = {nullptr, nullptr};
    mutable std::mutex fft_mu;
};

namespace sht {

// thread-local error message and launch counter
void set_error(const std::string& msg);
void count_launch(int n = 1);
void reset_launches();
// optional per-kernel timing (sht_profile_begin / sht_profile_end): CUDA events
// recorded on the launching stream around each launch
void prof_start(const char* name, cudaStream_t st);
void prof_stop(cudaStream_t st);

inline long long alm_index(int lmax, int l, int m)
{
    return (long long)m * (2 * lmax + 1 - m) / 2 + l;
}

// columns of the GEMMs for a batch
inline long long ncols(const sht_plan* p, int nmaps) { return (long long)nmaps * p->ncomp * 2; }

// workspace: the T / G buffer [m][q][p][c] in the compute precision
size_t tbuf_bytes(const sht_plan* p, int nmaps);

// kernels (launchers), return cudaSuccess or the launch error
cudaError_t launch_fft_forward_f64(const sht_plan* p, const double* map, double* T, int nmaps,
                                   cudaStream_t st);
cudaError_t launch_fft_backward_f64(const sht_plan* p, const double* G, double* map, int nmaps,
                                    cudaStream_t st);
cudaError_t launch_legendre_m2a_f64(const sht_plan* p, const double* T, double* alm, int nmaps,
                                    double scale0, double scale, cudaStream_t st);
// [nmaps][2][nalm] a_lm with component `which` copied from [nmaps][1][nalm], the other zero
cudaError_t expand_component(const sht_plan* p, const void* one, void* full, int nmaps, int which, cudaStream_t st);
// spin-2 map2alm of one component (csel = 1: E, 2: B) into alm [nmaps][1][nalm]
cudaError_t launch_legendre_m2a_f64_comp(const sht_plan* p, const double* T, double* alm, int nmaps,
                                         double scale0, double scale, int csel, cudaStream_t st);
// one order m only (its work items); map2alm may add into alm
// the orders m0 .. m0 + nm - 1 (one contiguous range of the work lists)
cudaError_t launch_legendre_m2a_f64_order(const sht_plan* p, const double* T, double* alm, int nmaps,
                                          double scale0, double scale, int m0, int nm, bool accum, cudaStream_t st);
cudaError_t launch_legendre_a2m_f64_order(const sht_plan* p, const double* alm, double* G, int nmaps, int m0,
                                          int nm, cudaStream_t st);
// Fourier-domain residual of the orders m0 .. m0 + nm - 1 only:
// D[m] = T[m] - F(G)[m] (FP64)
cudaError_t launch_alias_residual_order(const sht_plan* p, const double* T, const double* G, double* D, int nmaps,
                                        int m0, int nm, cudaStream_t st);
// plan-time walk of the FP64 recurrences that stores their checkpoints
cudaError_t build_f64_checkpoints(sht_plan* p, size_t* acc);
bool ring_skip_enabled();
void ring_first_pairs(sht_plan* p, const std::vector<char>& live);
cudaError_t launch_legendre_a2m_f64(const sht_plan* p, const double* alm, double* G, int nmaps,
                                    double scale0, double scale, cudaStream_t st);
int legendre_f64_row_tile();
int legendre_f64_pair_tile();
// split (tensor-core) form
cudaError_t launch_fft_forward_split(const sht_plan* p, const double* map, float2* T,
                                     unsigned int* colmax, int nmaps, cudaStream_t st);
cudaError_t launch_fft_backward_f32(const sht_plan* p, const float* G, double* map, int nmaps, cudaStream_t st);
// (each runs the slicing pass into `img`, split_img_bytes long, then the contraction;
// csel = 1 / 2: spin-2 map2alm of the E / B component only, alm [nmaps][1][nalm])
cudaError_t launch_legendre_m2a_tc(const sht_plan* p, const float2* T, const float* colmax, uint8_t* img,
                                   double* alm, int nmaps, double fs0, double fs1, cudaStream_t st,
                                   int csel = 0);
cudaError_t launch_legendre_a2m_tc(const sht_plan* p, const float2* A2, const float* colmax, uint8_t* img,
                                   float* G, int nmaps, float s0, float s1, cudaStream_t st);
size_t split_img_bytes(const sht_plan* p, int nmaps);
cudaError_t launch_alm_prep(const sht_plan* p, const double* alm, float2* A2, unsigned int* colmax, int nmaps,
                            cudaStream_t st);
// Fourier-domain residual of the iteration, D = T - F(G) (fft.cu), and the
// split form's column maxima of a T-layout buffer
cudaError_t launch_alias_residual(const sht_plan* p, const void* T, const void* G, void* D, int nmaps,
                                  cudaStream_t st);
cudaError_t launch_colmax_T(const sht_plan* p, const float2* T, unsigned int* colmax, int nmaps, cudaStream_t st);
// split form, alm2map: offset of the transposed a_lm (A2) inside the T / G buffer
size_t split_a2_offset(const sht_plan* p, int nmaps);
cudaError_t run_split_tables(sht_plan* p, const int* d_ck_base);
int split_row_tile();
int split_a2m_tiles();
int split_ck_rows();
int split_col_tile();

}  // namespace sht

#define SHT_CUDA_TRY(call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            sht::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));         \
            return SHT_ECUDA;                                                           \
        }                                                                               \
    } while (0)
