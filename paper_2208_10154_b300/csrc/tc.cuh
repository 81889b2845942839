// tc.cuh -- inline-PTX helpers for the sm_103a tensor-core path: mbarriers,
// tensor memory (TMEM) allocation and loads, UMMA shared-memory descriptors and
// tcgen05.mma (kind::f16 with FP16 operands, FP32 accumulation in TMEM).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace sht {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}"
                 :: "r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait: gives up after ~2^22 polls (each poll may itself suspend for a
// while), records `code` in *err and returns false. Every spin in the
// tensor-core kernels goes through here, so a kernel can never hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err, int code)
{
    for (int it = 0; it < (1 << 22); it++)
        if (mbar_try_wait(b, parity)) return true;
    atomicCAS(err, 0, code);
    return false;
}

// acquire at cluster scope: for barriers that other CTAs of the cluster arrive on
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cl(uint64_t* b, uint32_t parity, int* err, int code)
{
    for (int it = 0; it < (1 << 22); it++)
        if (mbar_try_wait_cl(b, parity)) return true;
    atomicCAS(err, 0, code);
    return false;
}

// one non-blocking test of a barrier phase (cluster-scope acquire)
__device__ __forceinline__ bool mbar_test_wait_cl(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait until a monotonic shared-memory counter reaches `target`
// (acquire); records `code` in *err and returns false after ~2^22 polls.
__device__ __forceinline__ bool wait_counter(const int* ctr, int target, int* err, int code)
{
    for (int it = 0; it < (1 << 22); it++) {
        int v;
        asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(ctr)) : "memory");
        if (v >= target) return true;
        __nanosleep(32);
    }
    atomicCAS(err, 0, code);
    return false;
}
__device__ __forceinline__ void publish_counter(int* ctr, int v)
{
    asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(ctr)), "r"(v) : "memory");
}

// ------------------------------------------------------------------ clusters
__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// all threads of all CTAs of the cluster (also a CTA-wide barrier)
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of the same shared-memory location in CTA `rank`
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
// arrive on a (possibly remote) mbarrier and announce `tx` bytes that an async copy will deliver
__device__ __forceinline__ void mbar_arrive_expect_tx_cl(uint32_t mbar_cl, uint32_t tx)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cluster.shared::cluster.b64 _, [%0], %1;"
                 :: "r"(mbar_cl), "r"(tx) : "memory");
}
// bulk copy from this CTA's shared memory into the shared memory of a CTA of the
// cluster; completion is signalled on that CTA's mbarrier (complete_tx)
__device__ __forceinline__ void bulk_copy_s2cluster(uint32_t dst_cl, uint32_t src, uint32_t bytes, uint32_t mbar_cl)
{
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst_cl), "r"(src), "r"(bytes), "r"(mbar_cl) : "memory");
}

// arrive on this CTA's mbarrier and announce `tx` bytes of async copies
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t tx)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_u32(b)), "r"(tx) : "memory");
}
// 1-D bulk copy global -> this CTA's shared memory (16-byte aligned, size a
// multiple of 16), completing on an mbarrier of this CTA
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(smem_u32(mbar)) : "memory");
}
// 1-D bulk copy global -> the shared memory at the same offset in every CTA of
// `mask` (cluster multicast; source in this GPU's own memory), completing on the
// mbarrier at the same offset in each destination CTA
__device__ __forceinline__ void bulk_copy_g2s_mc(uint32_t dst, const void* src, uint32_t bytes, uint64_t* mbar,
                                                 uint16_t mask)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
                 " [%0], [%1], %2, [%3], %4;"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(smem_u32(mbar)), "h"(mask) : "memory");
}
// generic-proxy writes to global memory made visible to later async-proxy reads
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ uint32_t sm_id()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}
// named barrier over `n` threads (id 1..15; id 0 is __syncthreads)
__device__ __forceinline__ void named_bar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(n) : "memory");
}

// ------------------------------------------------------ cp.async (LDGSTS)
// 8-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// L2 prefetch of a bulk range (16-byte aligned address, size a multiple of 16 bytes)
__device__ __forceinline__ void prefetch_l2_bulk(const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(src), "r"(bytes) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// ------------------------------------------------------------------- fences
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// --------------------------------------------------------------------- TMEM
// executed by one full warp
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(slot)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns; warp w may only touch lanes 32*(w%4)..
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                   "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr));
}
// 32 lanes x 32 consecutive 32-bit columns
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                   "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                   "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                   "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                   "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 32 lanes x 16 consecutive 32-bit columns, stored
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
                 "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                    "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
                    "r"(v[15])
                 : "memory");
}
// 32 lanes x 32 consecutive 32-bit columns, stored
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
                 "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                 "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                 :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                    "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
                    "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
                    "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
                    "r"(v[29]), "r"(v[30]), "r"(v[31])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- UMMA
// K-major operand tile in the 64-byte swizzle layout: rows of 32 16-bit values (64 B),
// 8-row atoms of 512 B, 16-byte chunk c of row r stored at chunk c ^ ((r>>1)&3).
// The tile base must be 512-byte aligned; the K = 16 half of a row starts 32 B in.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);   // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;          // stride byte offset: 8-row atom
    d |= (uint64_t)1 << 46;                   // descriptor version (tcgen05)
    d |= (uint64_t)4 << 61;                   // SWIZZLE_64B
    return d;
}
// byte offset of element (r, k) (k < 32) in such a tile
__device__ __forceinline__ uint32_t sw64_off(int r, int k)
{
    return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((((k >> 3)) ^ ((r >> 1) & 3)) << 4) + (k & 7) * 2);
}
// byte offset of the 16-byte chunk holding k = 8j..8j+7 of row r
__device__ __forceinline__ uint32_t sw64_chunk(int r, int j)
{
    return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((j ^ ((r >> 1) & 3)) << 4));
}

// instruction descriptor: kind::f16, A = B = BF16, D = F32, K-major A and B
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// instruction descriptor: kind::f16, A = B = FP16, D = F32, K-major A and B
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}
// arrive on an mbarrier once all previously issued tcgen05 ops of this thread completed
__device__ __forceinline__ void umma_commit(uint64_t* b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(b)) : "memory");
}

// the same arrival on the mbarrier at this offset in every CTA of `mask`
__device__ __forceinline__ void umma_commit_mc(uint64_t* b, uint16_t mask)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 :: "r"(smem_u32(b)), "h"(mask) : "memory");
}

// ------------------------------------------------------- number conversions
// The FP64 pipe of this GPU is ~2 lanes/clk/SM, and cvt between FP64 and FP32
// runs on it too, so FP64 <-> FP32 conversions are done with integer ops.
//
// FP64 value v times 2^sh as an FP32 (round to nearest on the 29 dropped bits,
// results below the FP32 normal range flush to 0; |v 2^sh| must stay < 2^127).
__device__ __forceinline__ float f64_to_f32_scaled(double v, int sh)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    unsigned int hi = (unsigned int)(b >> 32);
    int e = (int)((hi >> 20) & 0x7FF);
    if (e == 0) return 0.0f;
    unsigned long long mr = (b & 0x000FFFFFFFFFFFFFull) + (1ull << 28);   // round mantissa to 23 bits
    int carry = (int)(mr >> 52);
    unsigned int m23 = (unsigned int)((mr >> 29) & 0x7FFFFF);
    int ef = e - 1023 + 127 + sh + carry;
    if (ef <= 0) return 0.0f;
    unsigned int f = (hi & 0x80000000u) | ((unsigned int)ef << 23) | m23;
    return __uint_as_float(f);
}
// v * 2^sh as an FP32 pair hi + lo (|v 2^sh| < 2^127; parts below the FP32
// normal range flush to 0). Integer and FP32 operations only: the 29 mantissa
// bits below hi become lo through the 1.5 * 2^23 magic constant (their lowest
// 6 bits are dropped, a 2^-46 relative error), with no int-to-float
// conversion instruction.
__device__ __forceinline__ void f64_split_scaled(double v, int sh, float& hi, float& lo)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned int h32 = (unsigned int)(b >> 32);
    const int e = (int)((h32 >> 20) & 0x7FF);
    hi = f64_to_f32_scaled(v, sh);
    int r = (int)(b & ((1ull << 29) - 1));              // the 29 dropped mantissa bits
    r -= (r >= (1 << 28)) ? (1 << 29) : 0;              // hi was rounded up
    // (r >> 6) 2^-22, exact (|r >> 6| <= 2^22), then times 2^(e - 1075 + 28 + sh)
    const float fr = (__int_as_float(0x4B400000 + (r >> 6)) - 12582912.0f) * 2.384185791015625e-07f;
    const int es = e - 1075 + 28 + sh + 127;
    const float sc = (es > 0 && es < 255 && e != 0) ? __int_as_float(es << 23) : 0.0f;
    lo = (h32 & 0x80000000u) ? -(fr * sc) : fr * sc;
}
// exact FP32 -> FP64 (normal inputs; zero and subnormals give 0)
__device__ __forceinline__ double f32_to_f64(float x)
{
    unsigned int u = __float_as_uint(x);
    unsigned int e = (u >> 23) & 0xFF;
    if (e == 0) return 0.0;
    unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                           ((unsigned long long)(e - 127 + 1023) << 52) |
                           ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}
// x * 2^k for an FP64 x (exact; 0 stays 0)
__device__ __forceinline__ double ldexp_fast(double x, int k)
{
    const long long b = __double_as_longlong(x);
    return ((b & 0x7FF0000000000000ll) == 0) ? 0.0 : __longlong_as_double(b + ((long long)k << 52));
}
// x * 2^k for an FP32 x (exact when the result stays normal; flushes below)
// (selects, no early exits: the callers' unrolled loops stay one basic block)
__device__ __forceinline__ float ldexpf_fast(float x, int k)
{
    const int u = __float_as_int(x);
    const int e = (u >> 23) & 0xFF;
    const int en = e + k;
    const int r = (u & ~0x7F800000) | (en << 23);
    return (e != 0 && en > 0) ? __int_as_float(r) : 0.0f;
}

// Slice v + vl (|v| <= Q, |vl| <= 2^-23 |v|; units of the quantum) into four
// FP16 pieces, with r0 on the grid 2^-G (G = 10 or 11):
//     q   = nearest integer                           (exact in FP16 for Q <= 2048)
//     r0  = v - q rounded to the grid 2^-G            (|r0| <= 1/2: exact in FP16)
//     r1  = rem = (v - q - r0) + vl rounded to FP16   (|rem| <= 2^-G-1)
//     r2s = (rem - r1) 2^12 rounded to FP16           (the next 11 bits, scaled up)
// v - q and v - q - r0 are exact, so v + vl = q + r0 + r1 + 2^-12 r2s to
// ~2^-(G+24) of the quantum. The fixed grid of r0 makes every product q r0' a
// multiple of 2^-G, so sums of them are exact in FP32 while they stay below
// 2^(24-G).
template <int G>
__device__ __forceinline__ void slice4d(float v, float vl, float& q, float& r0, float& r1, float& r2s)
{
    static_assert(G == 10 || G == 11, "r0 grid");
    constexpr float magic = (G == 10) ? 12288.0f : 6144.0f;  // 1.5 * 2^(23-G): ulp 2^-G
    q = __fadd_rn(__fadd_rn(v, 12582912.0f), -12582912.0f);   // 1.5 * 2^23: nearest integer
    const float r = __fadd_rn(v, -q);
    r0 = __fadd_rn(__fadd_rn(r, magic), -magic);
    const float rem = __fadd_rn(__fadd_rn(r, -r0), vl);
    r1 = __half2float(__float2half_rn(rem));
    r2s = __fmul_rn(__fadd_rn(rem, -r1), 4096.0f);
}
// packed FP32 pairs (two lanes per instruction, each rounded to nearest)
__device__ __forceinline__ unsigned long long f2_pack(uint32_t lo, uint32_t hi)
{
    unsigned long long d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(lo), "r"(hi));
    return d;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, uint32_t& lo, uint32_t& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// nearest integer of |x| < 2^22 (exact)
__device__ __forceinline__ float rint_magic(float x)
{
    return __fadd_rn(__fadd_rn(x, 12582912.0f), -12582912.0f);
}
__device__ __forceinline__ uint32_t pack_h2(float lo, float hi)
{
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

}  // namespace tc
}  // namespace sht
