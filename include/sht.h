/*
 * sht.h -- C ABI of libsht, batched spherical harmonic transforms of many
 * HEALPix maps on one B300 GPU (sm_103a).
 *
 * Method: arXiv:2208.10154, "Accelerating spherical harmonic transforms for a
 * large number of sky maps". For a batch of maps on one pixelisation the
 * per-m sums over iso-latitude rings become matrix-matrix products
 * (Sec. 2.1, eq:mm, equ:mm_forward, equ:mm backward; Sec. 2.2 equ:matrix form):
 *     map2alm:  A_m = P_m T_m        (contract rings, dsigma = 4 pi / Npix)
 *     alm2map:  T_m = P_m^t A_m      (contract l), then ring FFTs.
 * Spin 2 (Q,U <-> E,B) follows Sec. 2.3 (Q_lm+iU_lm, equ:alm-eb,
 * equ:aeab mat form and its transpose). Iteration follows Algorithm 2.
 *
 * Conventions shared by every entry point
 *   - All data pointers are DEVICE pointers owned by the caller (typically
 *     torch tensors); the library never copies them to the host. Pointers to
 *     maps/alm must be 16-byte aligned.
 *   - map layout: double [nmaps][ncomp][npix], HEALPix RING order,
 *     npix = 12 nside^2. ncomp = 1 (T) for spin 0, 2 (Q, U) for spin 2.
 *   - alm layout: complex double (re, im interleaved) [nmaps][ncomp][nalm],
 *     m-major packed: idx(l, m) = m (2 lmax + 1 - m) / 2 + l, 0 <= m <= mmax,
 *     m <= l <= lmax, nalm = (mmax + 1)(2 lmax + 2 - mmax) / 2.
 *     ncomp = 1 (T) or 2 (E, B). Only m >= 0 is stored (real fields). The
 *     imaginary part of every m = 0 coefficient is ignored on input and
 *     written as 0 on output; for spin 2, l < 2 is ignored / written as 0.
 *   - map2alm uses the constant pixel weight dsigma = 4 pi / Npix (Sec. 2.1).
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = legacy default stream); nothing synchronises the host. A
 *     split-precision contraction wide enough for clusters of 8 column tiles
 *     (>= 1024 map columns) runs its last work items on a low-priority
 *     internal stream of the device, forked from `stream` and joined back to
 *     it with events inside the call, so work ordered after the call on
 *     `stream` sees the complete result (environment SHT_FILL_FRAC=0 keeps
 *     everything on `stream`).
 *   - `workspace` is caller-owned device memory of at least
 *     sht_workspace_bytes(plan, nmaps) bytes, 256-byte aligned. Concurrent
 *     calls on different streams need distinct workspaces.
 *   - Errors are returned as status codes, never thrown; the message of the
 *     last failure on the calling thread is in sht_last_error(). Arguments
 *     are validated before any launch; on SHT_EINVAL nothing was launched.
 */
#ifndef SHT_H_
#define SHT_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sht_plan sht_plan;   /* opaque: ring tables, recurrence tables, FFT tables */

typedef enum {
    SHT_OK = 0,
    SHT_EINVAL = 1,         /* bad argument (nothing launched)              */
    SHT_ENOMEM = 2,         /* a device or host allocation failed          */
    SHT_ECUDA = 3,          /* a CUDA runtime call or launch failed        */
    SHT_EUNSUPPORTED = 4,   /* valid request outside what this build does  */
    SHT_ETIMEOUT = 5        /* a bounded device wait gave up               */
} sht_status;

typedef enum {
    /* Every step in FP64 (FFT, lambda recurrence, contraction). */
    SHT_FP64 = 0,
    /* Split precision: the Legendre contraction on the 16-bit tensor cores
     * (tcgen05 kind::f16, FP16 operands, FP32 accumulation in TMEM). Every
     * operand value, scaled by a power-of-two quantum, is written as four
     * FP16 slices: its nearest integer, a remainder on the fixed grid 2^-10
     * (2^-11 for spin-2 map2alm), the next 11 bits, and their rounding error
     * scaled by 2^12. Ten slice products per term; the integer and fixed-grid
     * sums are exact and the rest are folded into the integer sum every 64 or
     * 128 steps of K; the final sums are formed in FP64. The lambda_lm
     * recurrence is walked in FP64 with scaled exponents when the plan is
     * built, which stores FP64 checkpoints every 32 rows; the kernels step
     * from a checkpoint in double-float FP32 pairs (~48 bits). Ring FFTs run
     * in double-float FP32. The contraction shares lambda pieces inside a
     * thread-block cluster with TMA multicast from this GPU's own memory: use
     * this form only in processes that drive a single GPU.
     * Supported for mmax <= 2047 with nside <= 4096, lmax <= 16383 (spin 0)
     * or nside <= 2048, lmax <= 4095 (spin 2); SHT_EUNSUPPORTED otherwise. */
    SHT_SPLIT_F16X4 = 1
} sht_precision;

/* Create a plan for HEALPix resolution `nside` (>= 1), band limit `lmax`
 * (>= 0), `mmax` (0..lmax; pass -1 for lmax), `spin` (0 or 2) and
 * `precision` (sht_precision) on CUDA device `device`. Builds the ring
 * geometry (standard HEALPix RING layout), the lambda_lm recurrence tables
 * (Sec. 2.1 footnote: lambda_lm, normalised as |lambda| = |Y|) and the FFT
 * tables on the host, and uploads them once (resident until destroy).
 * Synchronous. On success *out receives the plan. */
sht_status sht_plan_create(int nside, int lmax, int mmax, int spin, int precision,
                           int device, sht_plan** out);

/* Release a plan and its device tables. NULL is ignored. Synchronous. */
void sht_plan_destroy(sht_plan* plan);

/* Device workspace (bytes) needed by one call on `nmaps` maps. Used for
 * HBM admission by the serving loop. Returns 0 for a NULL plan or nmaps < 1. */
size_t sht_workspace_bytes(const sht_plan* plan, int nmaps);

/* Workspace for sht_map2alm with `niter` > 0 refinement steps of
 * Algorithm 2 (adds a second ring-spectrum buffer for the residual, in the
 * split form also its column maxima, and a coefficient increment buffer).
 * Equal to sht_workspace_bytes for niter = 0. */
size_t sht_workspace_bytes_iter(const sht_plan* plan, int nmaps, int niter);

/* Plan properties. */
int       sht_plan_nside(const sht_plan* plan);
int       sht_plan_lmax(const sht_plan* plan);
int       sht_plan_mmax(const sht_plan* plan);
int       sht_plan_spin(const sht_plan* plan);
int       sht_plan_precision(const sht_plan* plan);
long long sht_plan_npix(const sht_plan* plan);
long long sht_plan_nalm(const sht_plan* plan);

/* Device memory the plan holds while it lives (bytes): its resident tables
 * (ring geometry, recurrence and FFT tables; in the split form also the FP64
 * recurrence checkpoints) plus the staging buffers of the host-buffer entry
 * points once they have been used. For HBM admission (no counterpart in the
 * paper). 0 for a NULL plan. */
size_t    sht_plan_device_bytes(const sht_plan* plan);

/* Share of the Legendre terms (m, l, ring pair) that the plan's contraction
 * evaluates (Sec. 3.1, Implementation detail: the ring optimisation, which
 * leaves out, for each m, the rings where P_lm has an extremely low
 * amplitude). Plans skip, for each order m, the leading polar ring pairs
 * on which |lambda_lm| < 1e-30 for every l (spin 2: for s = +2 and -2; in
 * 32-pair steps, the same set for every higher order): split plans in the
 * contraction and in the ring FFTs' order mapping, FP64 plans in map2alm's
 * contraction and in alm2map's ring-pair tiles that lie wholly among them
 * (their G is written as zeros). The skipped terms change no output beyond
 * rounding. 1.0 when nothing is skipped (the environment variable
 * SHT_RING_SKIP=0 at plan creation); 0 for a NULL plan. The value counts
 * the pairs from each order's first kept one. */
double    sht_plan_terms_kept(const sht_plan* plan);

/* The ring optimisation's first ring pair per order (the same passage):
 * out[m], m = 0..mmax (host memory owned by the caller, mmax + 1 ints) is
 * the first ring pair, counted from the north pole (pair p holds rings p + 1
 * and 4 nside - 1 - p), that the plan contracts for order m: the first pair
 * where some |lambda_lm| (spin 2: of s = +2 or -2) reaches 1e-30, made
 * nondecreasing in m (the smallest over this and every higher order),
 * rounded down to a multiple of 32, and 0 for m = 0; all 0 when nothing is
 * skipped. SHT_EINVAL for a NULL argument. */
sht_status sht_plan_first_pairs(const sht_plan* plan, int* out);

/* Backward transform (Sec. 2.1 equ:backward equ, equ:mm backward; spin 2:
 * equ:aeab mat form inv). alm [nmaps][ncomp][nalm] (complex double, device)
 * -> map [nmaps][ncomp][npix] (double, device). Real field:
 *   T = sum_l a_l0 lambda_l0 + 2 Re sum_{m>0} sum_l a_lm lambda_lm e^{i m phi}.
 * Spin 2: Q +- iU = sum a_{+-2,lm} +-2Y_lm with a_{+-2} = -(a_E +- i a_B). */
sht_status sht_alm2map(sht_plan* plan, const void* alm, void* map, int nmaps,
                       void* workspace, size_t workspace_bytes, void* stream);

/* Forward transform (Sec. 2.1 Eq. 1, eq:mm, equ:mm_forward; spin 2:
 * equ:alm-eb, equ:aeab mat form). map -> alm, layouts as above, with
 * `niter` >= 0 refinement steps of Algorithm 2 (0 = plain quadrature):
 *   a^0 = map2alm(T), a^{n+1} = a^n + map2alm(T - alm2map(a^n)).
 * The steps run on the ring spectra (the residual's backward and forward
 * FFTs are replaced by their exact action on the Fourier coefficients), so
 * a step costs two Legendre contractions and no FFT.
 * niter > 0 needs sht_workspace_bytes_iter(plan, nmaps, niter) bytes. */
sht_status sht_map2alm(sht_plan* plan, const void* map, void* alm, int nmaps, int niter,
                       void* workspace, size_t workspace_bytes, void* stream);

/* E-only or B-only transforms of spin-2 plans (the paper's remark that
 * pipelines needing one of a_E, a_B should get it without the other,
 * Sec. 3.1; equ:aeab mat form keeps one block row). which = 0: E, 1: B.
 * sht_map2alm_eb: Q/U maps [nmaps][2][npix] -> that component's a_lm
 * [nmaps][1][nalm]; the ring FFTs of Q and U run in full, the Legendre
 * contraction forms only the kept component (half of the spin-2 work).
 * Workspace: sht_workspace_bytes(plan, nmaps).
 * sht_alm2map_eb: one component's a_lm [nmaps][1][nalm] -> Q/U maps
 * [nmaps][2][npix] with the other component zero (the full spin-2
 * synthesis, no saving). Workspace: sht_workspace_bytes_eb(plan, nmaps).
 * SHT_EINVAL for spin-0 plans or another `which`. Otherwise as
 * sht_map2alm / sht_alm2map. */
sht_status sht_map2alm_eb(sht_plan* plan, const void* map, void* alm, int nmaps, int which,
                          void* workspace, size_t workspace_bytes, void* stream);
sht_status sht_alm2map_eb(sht_plan* plan, const void* alm, void* map, int nmaps, int which,
                          void* workspace, size_t workspace_bytes, void* stream);
size_t     sht_workspace_bytes_eb(const sht_plan* plan, int nmaps);

/* Forward transform with the immediate iteration of Algorithm 3 (Sec. 4):
 * the orders m are refined one after another inside each pass, and every
 * order sees the corrections of the orders before it that share its ring
 * bins (aliasing on rings of N <= 2 mmax pixels), where Algorithm 2 updates
 * all orders together after the pass. Read as a block Gauss-Seidel sweep on
 * the ring spectra of the residual, starting from a = 0:
 *   for m = 0..mmax:  a_m += map2alm(T - alm2map(a))_m
 * with the residual kept in the Fourier domain (no FFT inside a pass).
 * npass >= 1 sweeps (npass = 1 is one sweep; without aliasing it equals the
 * plain quadrature and npass sweeps equal Algorithm 2 with npass - 1
 * refinements). For lmax between 2 nside and 3 nside it converges faster
 * than Algorithm 2. Spin 2 refines a_E and a_B of order m together from the
 * order-m spectra of Q and U (the orders m and -m of Q + iU). FP64 plans
 * only (SHT_EUNSUPPORTED for split plans).
 * Three kernel launches per order and pass (the orders depend on each
 * other in sequence). Layouts as sht_map2alm; needs
 * sht_workspace_bytes_immediate(plan, nmaps) bytes of workspace. */
sht_status sht_map2alm_immediate(sht_plan* plan, const void* map, void* alm, int nmaps, int npass,
                                 void* workspace, size_t workspace_bytes, void* stream);
size_t     sht_workspace_bytes_immediate(const sht_plan* plan, int nmaps);

/* Adjoints in real parameters/* Adjoints in real parameters (Re a_l0; Re, Im a_lm for m > 0), used by the
 * autograd wrappers. The paper has no adjoints; these are the exact
 * transposes of the two linear maps above:
 *   alm2map_adjoint(h)_lm = (Npix / 4 pi) map2alm(h)_lm * (1 if m = 0 [real
 *                           part only], 2 if m > 0)
 *   map2alm_adjoint(g)    = (4 pi / Npix) alm2map(g'), g'_l0 = Re g_l0,
 *                           g'_lm = g_lm / 2 (m > 0).
 * Same layouts and conventions as the forward calls. */
sht_status sht_alm2map_adjoint(sht_plan* plan, const void* map, void* alm, int nmaps,
                               void* workspace, size_t workspace_bytes, void* stream);
sht_status sht_map2alm_adjoint(sht_plan* plan, const void* alm, void* map, int nmaps,
                               void* workspace, size_t workspace_bytes, void* stream);

/* End-to-end variants on HOST buffers (pageable or pinned): the library
 * moves the batch in chunks (sized so that the call holds at most 48 GB of
 * device memory; environment SHT_HOST_CHUNK_GB sets another limit) through
 * two device buffer pairs, overlapping
 * chunk k's transform (on `stream`) with chunk k+1's host->device copy and
 * chunk k-1's device->host copy (two plan-owned copy streams); pageable
 * buffers are staged through plan-owned pinned buffers. Returns after the
 * result is back in host memory. Same layouts as above. Not for concurrent
 * calls on one plan. */
sht_status sht_alm2map_host(sht_plan* plan, const void* alm_host, void* map_host, int nmaps,
                            void* stream);
sht_status sht_map2alm_host(sht_plan* plan, const void* map_host, void* alm_host, int nmaps,
                            int niter, void* stream);

/* alm2map without any device allocation (the paper has no counterpart; this
 * is a library convenience). For callers that cannot allocate device memory
 * while they run -- a latency-critical serving loop that must not touch the
 * allocator (cudaMalloc can synchronise the device), or a host framework
 * that owns all GPU memory and hands the library only its inputs and
 * outputs -- and so cannot provide the workspace sht_alm2map needs. Same
 * transform, layouts and stream semantics as sht_alm2map on an SHT_FP64 plan
 * (other precisions return SHT_EUNSUPPORTED); the caller passes only the
 * inputs and outputs. The intermediate matrix lives in one static device
 * array of sht_noalloc_scratch_bytes() bytes (64 MiB) that every GPU loading
 * the library keeps until the process exits; a call that needs more returns
 * SHT_EINVAL with both sizes in sht_last_error(). All calls on a device share
 * that array (nothing in it needs to start at zero), so calls that overlap
 * on the GPU race: serialise them. The first call on each device looks up
 * the array's address (cudaGetSymbolAddress); make it before any stream
 * capture begins. */
sht_status sht_alm2map_noalloc(sht_plan* plan, const void* alm, void* map, int nmaps,
                               void* stream);
size_t     sht_noalloc_scratch_bytes(void);

/* The paper's compact square storage of a_lm (Sec. 5, equ:new alm save scheme):
 * per map and component one real (lmax+1) x (lmax+1) row-major matrix, every
 * element used:
 *     Re a_lm at (row l,     column m)              for 0 <= m <= l <= lmax
 *     Im a_lm at (row l - m, column lmax - m + 1)   for 1 <= m <= l <= lmax
 * sq: double [nmaps][ncomp][lmax+1][lmax+1] (device); alm as above. Entries
 * with m > mmax are written as 0 (to_square) or ignored (to_alm); to_alm
 * writes Im a_l0 = 0. Exact (element copies). Asynchronous on `stream`. */
sht_status sht_alm_to_square(const sht_plan* plan, const void* alm, void* sq, int nmaps, void* stream);
sht_status sht_square_to_alm(const sht_plan* plan, const void* sq, void* alm, int nmaps, void* stream);

/* Pixel-domain E or B projection of Q/U maps (Sec. 2.3, equ:aeab mat form
 * pixel): out = alm2map(keep(map2alm(map, niter))), keep = the E (which = 0)
 * or B (which = 1) component of every a_lm, the other set to zero. With
 * niter = 0 the analysis forms only the kept component (sht_map2alm_eb).
 * Spin-2 plans only (SHT_EINVAL otherwise). map, out: double [nmaps][2][npix]
 * (device, distinct); the result is the band-limited E- (B-) part of the
 * input, within the accuracy of the plan's precision and niter. Needs
 * sht_workspace_bytes_project(plan, nmaps, niter) bytes of workspace. */
sht_status sht_eb_project(sht_plan* plan, const void* map, void* out, int nmaps, int which, int niter,
                          void* workspace, size_t workspace_bytes, void* stream);
size_t     sht_workspace_bytes_project(const sht_plan* plan, int nmaps, int niter);

/* Device-side status of a plan's tensor-core kernels (no counterpart in the
 * paper). Every wait inside those kernels is bounded; one that gives up
 * records a nonzero code (which wait) in a per-plan device word, skips the
 * rest of its work and lets the kernel finish, so the outputs of that call
 * are invalid. This call synchronises the plan's device, reads the word into
 * *code (if code is not NULL), clears it, and returns SHT_ETIMEOUT if it was
 * set, SHT_OK otherwise (SHT_EINVAL for a NULL plan, SHT_ECUDA on a CUDA
 * error). FP64 plans always report SHT_OK. */
sht_status sht_plan_device_status(sht_plan* plan, int* code);

/* Number of kernel launches the most recent call on this thread issued
 * (for the benchmark's launch accounting). */
int sht_last_launch_count(void);

/* Per-kernel timing for benchmarks (no counterpart in the paper). After
 * sht_profile_begin(), every kernel this thread launches is bracketed by
 * CUDA events recorded on its launching stream. sht_profile_end() waits for
 * those events, writes {"kernel": {"launches": n, "ms": t}, ...} as a
 * NUL-terminated JSON string into buf (up to cap bytes), stops recording and
 * returns the length the full string needs including the NUL. */
void sht_profile_begin(void);
int  sht_profile_end(char* buf, int cap);

/* Message describing the last failure on the calling thread ("" if none). */
const char* sht_last_error(void);

/* Library version string. */
const char* sht_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SHT_H_ */
