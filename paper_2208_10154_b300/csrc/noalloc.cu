// noalloc.cu -- sht_alm2map_noalloc: the FP64 alm2map for callers that must
// not allocate device memory at call time.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not
// wanted -- a latency-critical serving loop that must never hit the
// allocator (cudaMalloc can synchronise the whole device), or an embedding
// framework that owns all device memory and gives the library only its
// input and output buffers.
// Such callers cannot supply the workspace that sht_alm2map needs for the
// intermediate ring-coefficient matrix G[m][q][p][c], so this entry point
// keeps that matrix in a fixed, file-scope device array instead.
//
// Limits and sharing rules:
//   - the scratch array holds SHT_NOALLOC_SCRATCH_BYTES (64 MiB); a call whose
//     G matrix ((mmax+1) * 2 * (2 nside) * (2 nmaps ncomp) doubles) does not fit
//     is rejected with SHT_EINVAL and a message giving both sizes;
//   - every GPU that loads libsht holds the array until the process exits;
//   - all calls on a device share the one array and it keeps whatever the
//     previous call left in it; nothing here has to start at zero because the
//     Legendre kernel overwrites every entry of G before the FFT kernel reads
//     it. Calls whose kernels overlap on the GPU (different streams, or
//     different host threads) race on the array: serialise them;
//   - the first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it. Make that
//     first call before any stream capture starts.
#include <mutex>

#include "common.cuh"

#define SHT_NOALLOC_SCRATCH_BYTES (64ull << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[SHT_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
}  // namespace

// Device address of the scratch array on the current device (looked up once
// per device). In host code the symbol itself is only a host-side stand-in,
// never a device address, so it must not be passed to a kernel directly.
static sht_status noalloc_scratch(int device, void** out)
{
    if (device < 0 || device >= kMaxDevices) {
        sht::set_error("sht_alm2map_noalloc: device index out of range");
        return SHT_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[device]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            sht::set_error(std::string("sht_alm2map_noalloc: cudaGetSymbolAddress failed: ") +
                           cudaGetErrorString(e));
            return SHT_ECUDA;
        }
        g_scratch_ptr[device] = ptr;
    }
    *out = g_scratch_ptr[device];
    return SHT_OK;
}

extern "C" size_t sht_noalloc_scratch_bytes(void) { return (size_t)SHT_NOALLOC_SCRATCH_BYTES; }

extern "C" sht_status sht_alm2map_noalloc(sht_plan* p, const void* alm, void* map, int nmaps, void* stream)
{
    sht::set_error("");
    sht::reset_launches();
    if (!p) { sht::set_error("sht_alm2map_noalloc: plan is NULL"); return SHT_EINVAL; }
    if (p->precision != SHT_FP64) {
        sht::set_error("sht_alm2map_noalloc: only SHT_FP64 plans are supported");
        return SHT_EUNSUPPORTED;
    }
    if (nmaps < 1) { sht::set_error("sht_alm2map_noalloc: nmaps must be >= 1"); return SHT_EINVAL; }
    if (!alm || !map) { sht::set_error("sht_alm2map_noalloc: data pointer is NULL"); return SHT_EINVAL; }
    if (((uintptr_t)alm & 15) || ((uintptr_t)map & 15)) {
        sht::set_error("sht_alm2map_noalloc: data pointers must be 16-byte aligned");
        return SHT_EINVAL;
    }
    const size_t need = sht::tbuf_bytes(p, nmaps);
    if (need > (size_t)SHT_NOALLOC_SCRATCH_BYTES) {
        sht::set_error("sht_alm2map_noalloc: this call needs " + std::to_string(need) +
                       " bytes of scratch but the built-in scratch holds " +
                       std::to_string((size_t)SHT_NOALLOC_SCRATCH_BYTES) +
                       " bytes; use fewer maps per call or sht_alm2map with a workspace");
        return SHT_EINVAL;
    }
    cudaError_t e = cudaSetDevice(p->device);
    if (e != cudaSuccess) { sht::set_error(cudaGetErrorString(e)); return SHT_ECUDA; }
    void* scratch = nullptr;
    sht_status s = noalloc_scratch(p->device, &scratch);
    if (s != SHT_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    double* G = (double*)scratch;
    e = sht::launch_legendre_a2m_f64(p, (const double*)alm, G, nmaps, 1.0, 1.0, st);
    if (e == cudaSuccess) e = sht::launch_fft_backward_f64(p, G, (double*)map, nmaps, st);
    if (e != cudaSuccess) {
        sht::set_error(std::string("sht_alm2map_noalloc launch: ") + cudaGetErrorString(e));
        return SHT_ECUDA;
    }
    return SHT_OK;
}
