// layout.cu -- the paper's compact square a_lm storage and the pixel-domain
// E / B projection, on top of the transforms of plan.cu.
//
// Compact square storage (Sec. 5, equ:new alm save scheme): per map and
// component one real (lmax+1) x (lmax+1) matrix, every element used:
//     Re a_lm  at (row l,     column m)               0 <= m <= l <= lmax
//     Im a_lm  at (row l - m, column lmax - m + 1)    1 <= m <= l <= lmax
// Real parts fill the lower triangle with the diagonal, imaginary parts the
// strict upper triangle (l - m < lmax - m + 1 always). Entries with m > mmax
// are zero.
//
// E / B projection (Sec. 2.3, equ:aeab mat form pixel): keep one of the two
// diagonal blocks of lambda^{E,B}, i.e. map2alm, zero the other component of
// every a_lm, alm2map.
#include <algorithm>
#include <string>

#include "common.cuh"

namespace sht {

__device__ __forceinline__ long long sq_alm_index(int lmax, int l, int m)
{
    return (long long)m * (2 * lmax + 1 - m) / 2 + l;
}

// one thread per square element (row, col) of one map component
__global__ void k_alm_to_square(const double2* __restrict__ alm, double* __restrict__ sq, int lmax, int mmax,
                                long long nalm, long long nsq, long long ncompmaps)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long mc = blockIdx.y + (long long)gridDim.y * blockIdx.z;
    if (e >= nsq || mc >= ncompmaps) return;
    const int L = lmax + 1;
    const int row = (int)(e / L), col = (int)(e - (long long)row * L);
    double v = 0.0;
    if (row >= col) {                                   // Re a_{row, col}
        if (col <= mmax) v = alm[mc * nalm + sq_alm_index(lmax, row, col)].x;
    } else {                                            // Im a_{l, m}, m = lmax + 1 - col, l = row + m
        const int m = L - col, l = row + m;
        if (m <= mmax) v = alm[mc * nalm + sq_alm_index(lmax, l, m)].y;
    }
    sq[mc * nsq + e] = v;
}

// the inverse: every element back to its a_lm part; Im a_l0 is written as 0
__global__ void k_square_to_alm(const double* __restrict__ sq, double2* __restrict__ alm, int lmax, int mmax,
                                long long nalm, long long nsq, long long ncompmaps)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long mc = blockIdx.y + (long long)gridDim.y * blockIdx.z;
    if (e >= nsq || mc >= ncompmaps) return;
    const int L = lmax + 1;
    const int row = (int)(e / L), col = (int)(e - (long long)row * L);
    double* a = reinterpret_cast<double*>(alm + mc * nalm);
    const double v = sq[mc * nsq + e];
    if (row >= col) {
        if (col <= mmax) {
            const long long i = sq_alm_index(lmax, row, col);
            a[2 * i] = v;
            if (col == 0) a[2 * i + 1] = 0.0;
        }
    } else {
        const int m = L - col, l = row + m;
        if (m <= mmax) a[2 * sq_alm_index(lmax, l, m) + 1] = v;
    }
}

static sht_status check_layout(const sht_plan* p, const void* a, const void* b, int nmaps)
{
    if (!p) { set_error("plan is NULL"); return SHT_EINVAL; }
    if (nmaps < 1) { set_error("nmaps must be >= 1"); return SHT_EINVAL; }
    if (!a || !b) { set_error("data pointer is NULL"); return SHT_EINVAL; }
    if (((uintptr_t)a & 15) || ((uintptr_t)b & 15)) { set_error("data pointers must be 16-byte aligned"); return SHT_EINVAL; }
    return SHT_OK;
}

static sht_status launch_layout(const sht_plan* p, const void* in, void* out, int nmaps, bool to_square,
                                cudaStream_t st)
{
    const long long L = p->lmax + 1, nsq = L * L, ncm = (long long)nmaps * p->ncomp;
    const unsigned by = (unsigned)std::min<long long>(ncm, 65535), bz = (unsigned)((ncm + by - 1) / by);
    dim3 grid((unsigned)((nsq + 255) / 256), by, bz);
    reset_launches();
    if (to_square) {
        prof_start("k_alm_to_square", st);
        k_alm_to_square<<<grid, 256, 0, st>>>((const double2*)in, (double*)out, p->lmax, p->mmax, p->nalm, nsq, ncm);
    } else {
        prof_start("k_square_to_alm", st);
        k_square_to_alm<<<grid, 256, 0, st>>>((const double*)in, (double2*)out, p->lmax, p->mmax, p->nalm, nsq, ncm);
    }
    prof_stop(st);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(std::string("layout launch: ") + cudaGetErrorString(e)); return SHT_ECUDA; }
    return SHT_OK;
}

}  // namespace sht

using namespace sht;

sht_status sht_alm_to_square(const sht_plan* p, const void* alm, void* sq, int nmaps, void* stream)
{
    sht_status s = check_layout(p, alm, sq, nmaps);
    if (s != SHT_OK) return s;
    cudaSetDevice(p->device);
    return launch_layout(p, alm, sq, nmaps, true, (cudaStream_t)stream);
}

sht_status sht_square_to_alm(const sht_plan* p, const void* sq, void* alm, int nmaps, void* stream)
{
    sht_status s = check_layout(p, sq, alm, nmaps);
    if (s != SHT_OK) return s;
    cudaSetDevice(p->device);
    return launch_layout(p, sq, alm, nmaps, false, (cudaStream_t)stream);
}

static size_t round256(size_t v) { return (v + 255) / 256 * 256; }

size_t sht_workspace_bytes_project(const sht_plan* p, int nmaps, int niter)
{
    if (!p || nmaps < 1 || niter < 0) return 0;
    const size_t alm_b = (size_t)nmaps * p->ncomp * (size_t)p->nalm * 2 * sizeof(double);
    return round256(alm_b) + round256(alm_b / 2) + sht_workspace_bytes_iter(p, nmaps, niter);
}

sht_status sht_eb_project(sht_plan* p, const void* map, void* out, int nmaps, int which, int niter, void* ws,
                          size_t wsb, void* stream)
{
    sht_status s = check_layout(p, map, out, nmaps);
    if (s != SHT_OK) return s;
    if (p->spin != 2) { set_error("E/B projection needs a spin-2 plan"); return SHT_EINVAL; }
    if (which != 0 && which != 1) { set_error("which must be 0 (E) or 1 (B)"); return SHT_EINVAL; }
    if (niter < 0) { set_error("niter must be >= 0"); return SHT_EINVAL; }
    const size_t need = sht_workspace_bytes_project(p, nmaps, niter);
    if (!ws || wsb < need) { set_error("workspace too small: need " + std::to_string(need) + " bytes"); return SHT_EINVAL; }
    if ((uintptr_t)ws & 255) { set_error("workspace must be 256-byte aligned"); return SHT_EINVAL; }
    cudaSetDevice(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t row = (size_t)p->nalm * 2 * sizeof(double);        // one component of one map
    const size_t alm_b = round256((size_t)nmaps * 2 * row), one_b = round256((size_t)nmaps * row);
    char* alm = (char*)ws;
    char* one = alm + alm_b;
    void* tws = one + one_b;
    const size_t twsb = wsb - alm_b - one_b;
    cudaError_t e;
    if (niter == 0) {
        // only the kept component is formed (half of the spin-2 contraction)
        s = sht_map2alm_eb(p, map, one, nmaps, which, tws, twsb, stream);
        if (s != SHT_OK) return s;
        e = expand_component(p, one, alm, nmaps, which, st);
    } else {
        s = sht_map2alm(p, map, alm, nmaps, niter, tws, twsb, stream);
        if (s != SHT_OK) return s;
        // zero the other component of every map: rows of `row` bytes, 2 rows apart
        e = cudaMemset2DAsync(alm + (size_t)(1 - which) * row, 2 * row, 0, row, (size_t)nmaps, st);
    }
    const int launches = sht_last_launch_count();
    if (e != cudaSuccess) { set_error(std::string("eb_project copy: ") + cudaGetErrorString(e)); return SHT_ECUDA; }
    s = sht_alm2map(p, alm, out, nmaps, tws, twsb, stream);
    count_launch(launches);
    return s;
}
