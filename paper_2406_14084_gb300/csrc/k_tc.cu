// k_tc.cu -- wide fused gates on the 5th-generation tensor cores (tcgen05), complex64 states.
//
// A 6-qubit fused gate U (64x64 complex) acts on every group of 64 amplitudes that differ only
// in its target bits.  Each CTA gathers a slab of 2^13 amplitudes (the 6 target bits plus 7
// further bits) into shared memory and views it as a 128 x 64 complex matrix S (rows = the 7
// other bits, columns = the target index).  With the real embedding of U,
//     E[2j][2l] = Re U[j][l], E[2j][2l+1] = -Im U[j][l], E[2j+1][2l] = Im U[j][l],
//     E[2j+1][2l+1] = Re U[j][l],
// the update is the real GEMM  D (128 x 128) = S_r (128 x 128) * E^T  on interleaved (re, im)
// columns.  Split precision: S_r = S_hi + S_lo and E = E_hi + E_lo with BF16 parts (E is split
// on the host in FP64); D = S_hi E_hi^T + S_hi E_lo^T + S_lo E_hi^T, accumulated in FP32 in
// tensor memory (the S_lo E_lo^T term, of relative size 2^-16 squared, is dropped).
//
// Per slab: 16-byte cp.async gather of the slab -> FP32-to-BF16 hi/lo split into the
// 128-byte-swizzled K-major operand layout -> 24 tcgen05.mma (3 products x 8 K-steps of 16)
// issued by one thread into a 128-lane x 128-column FP32 accumulator in TMEM ->
// tcgen05.commit to an mbarrier -> tcgen05.ld of the accumulator by the 4 warps (warp w owns
// TMEM lanes 32w..32w+31 = rows) -> into the (now free) A operand region -> 16-byte stores.
// The next slab's gather is issued as soon as the split has read the slab buffer, so it
// overlaps the MMAs, the accumulator read-back and the stores.  The E operand stays in shared
// memory for the whole launch.  Every mbarrier wait is bounded; on expiry the CTA
// records QS_ETIMEOUT, releases its tensor memory and exits.
//
// TF32 x 3 mode (kind::tf32): the same three products with TF32 parts (10 stored mantissa bits
// each, so hi + lo carries about 22 bits against BF16's 16).  The 4-byte operands take twice the
// space, so each slab is multiplied in two K halves of 64 (targets 0..31, then 32..63), both
// accumulating into the same TMEM columns; the E half-images (hi and lo, 32 KiB each) are copied
// from global memory (L2-resident) before each half.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdio>

#include "qs_internal.h"

namespace qs {
namespace {

constexpr int kThreads = 512;  // 16 warps: four per TMEM lane quarter
constexpr uint32_t kChunksPerThread = 16 * kTcRows / kThreads;  // 16-byte operand chunks of a row part
// One operand part in shared memory: a BF16 operand (128 x 128 x 2 B), or half the K range of a
// TF32 operand (128 x 64 x 4 B): 32 KiB either way.
constexpr uint32_t kOpBytes = kTcRows * kTcK * 2;
constexpr uint32_t kSlabBytes = (1u << kTcSlabBits) * 8;
constexpr uint32_t kOffAhi = kSlabBytes, kOffAlo = kOffAhi + kOpBytes, kOffBhi = kOffAlo + kOpBytes,
                   kOffBlo = kOffBhi + kOpBytes, kOffCtl = kOffBlo + kOpBytes;
constexpr uint32_t kWaitLimit = 1u << 24;

struct TcCtl {
    unsigned long long mbar;  // MMA completion
    unsigned long long bbar;  // E-image bulk copies landed
    uint32_t tmem;
    uint32_t pad;
    DevTc tc;
    uint64_t seg_lo[64], seg_hi[64];
    uint16_t joff[64];   // slab-local offset of target index j
    uint16_t moff[128];  // slab-local offset of row m
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

// One thread: expect `bytes` of bulk copies on the mbarrier (one arrival).
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bulk (TMA, non-tensor) copy global -> shared of `bytes` (16-byte aligned, multiple of 16),
// completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= uint64_t((addr >> 4) & 0x3FFF);          // start address
    d |= uint64_t(1) << 16;                       // leading byte offset (unused for swizzled K-major)
    d |= uint64_t(1024 >> 4) << 32;               // stride byte offset between 8-row groups
    d |= uint64_t(1) << 46;                       // descriptor version (tcgen05)
    d |= uint64_t(2) << 61;                       // layout: 128-byte swizzle
    return d;
}

// Instruction descriptors: D FP32 (bits 4-5 = 1), A and B both K-major, N = 128 (bits 17-22 hold
// N / 8), M = 128 (bits 24-28 hold M / 16); operand format in bits 7-9 (A) and 10-12 (B):
// kind::f16 with BF16 = 1, kind::tf32 with TF32 = 2.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t(kTcK) >> 3) << 17) |
                                ((uint32_t(kTcRows) >> 4) << 24);
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t(kTcK) >> 3) << 17) |
                                ((uint32_t(kTcRows) >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdescBf16), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdescTf32), "r"(accumulate)
        : "memory");
}

// TF32 value nearest to x (round to nearest, ties away), as FP32 bits with the low 13 bits clear.
__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&r)[32])
{
    uint32_t u[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
          "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
          "=r"(u[14]), "=r"(u[15]), "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]),
          "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]), "=r"(u[25]),
          "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) r[i] = __uint_as_float(u[i]);
}

// Byte offset of element (row, k) of a 128-row BF16 operand in the swizzled K-major layout:
// K is split into 128-byte atoms (64 elements) stored one after the other for all rows.
__device__ __forceinline__ uint32_t op_chunk_offset(uint32_t row, uint32_t chunk16)
{
    const uint32_t kb = chunk16 >> 3, c = chunk16 & 7;
    return kb * (kTcRows * 128u) + row * 128u + ((c ^ (row & 7u)) << 4);
}

// MODE = QS_TC_BF16X3: each GEMM is over K = 128.  MODE = QS_TC_TF32X3: the operands are 4-byte
// TF32, so each GEMM runs in two K halves of 64.  NB = 1: a 6-qubit gate, one GEMM per slab; for
// BF16 its E images stay in shared memory for the whole launch.  NB = 4: a 7-qubit gate (see
// below), four GEMMs per slab into four TMEM accumulators.  Whenever E is not resident, its
// (half-)images are copied from global memory (L2) by bulk TMA copies completing on an
// mbarrier, one block or half at a time.
template <int MODE, int NB>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(float2 *__restrict__ state, const DevTc *__restrict__ d_tc,
                   const unsigned char *__restrict__ images, uint64_t nslabs, int *status)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float2 *slab = reinterpret_cast<float2 *>(base);
    TcCtl &K = *reinterpret_cast<TcCtl *>(base + kOffCtl);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar = saddr(&K.mbar);

    const uint32_t bbar = saddr(&K.bbar);
    if (tid == 0) {
        K.tc = *d_tc;
        mbar_init(bar, 1);
        mbar_init(bbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    constexpr uint32_t kCols = uint32_t(kTcK) * NB;  // one 128-column FP32 accumulator per GEMM
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&K.tmem)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    constexpr bool kTf32 = MODE == QS_TC_TF32X3;
    constexpr int kParts = kTf32 ? 2 : 1;
    constexpr bool kResident = !kTf32 && NB == 1;
    const unsigned char *img = images + d_tc->img;
    // thread 0: bulk-copy half h of E block eb (per block: hi halves, then lo halves, 32 KiB each)
    // into the B region; the B region must be free (the previous GEMM has completed)
    auto load_b = [&](int eb, int h) {
        const unsigned char *blk = img + size_t(eb) * (2 * kParts) * kOpBytes;
        mbar_expect_tx(bbar, 2 * kOpBytes);
        bulk_g2s(saddr(base + kOffBhi), blk + h * kOpBytes, kOpBytes, bbar);
        bulk_g2s(saddr(base + kOffBlo), blk + (kParts + h) * kOpBytes, kOpBytes, bbar);
    };
    if (kResident) {
        // resident E_hi / E_lo images (64 KiB contiguous in global memory)
        const uint32_t dst = saddr(base + kOffBhi);
        for (uint32_t v = tid; v < (2 * kOpBytes) / 16; v += kThreads) cp_async16(dst + 16 * v, img + 16 * v);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = K.tmem;
    const DevPass &P = K.tc.slab;
    const int lo = P.lo, nhi = P.nhi;
    for (uint32_t j = tid; j < 128; j += kThreads) {
        const uint32_t x = j & 63, sh = (j < 64) ? 0 : 6;
        uint64_t o = 0;
        for (int m = 0; m < 6; ++m)
            if ((x >> m & 1) && int(m + sh) < nhi) o |= 1ull << P.hipos[m + sh];
        if (j < 64) K.seg_lo[x] = o; else K.seg_hi[x] = o;
    }
    for (uint32_t j = tid; j < 64; j += kThreads) {
        uint32_t o = 0;
        for (int t = 0; t < kTcTargets; ++t)
            if (j >> t & 1) o |= 1u << K.tc.tpos[t];
        K.joff[j] = (uint16_t)o;
    }
    for (uint32_t m = tid; m < 128; m += kThreads) {
        uint32_t o = 0;
        for (int t = 0; t < 7; ++t)
            if (m >> t & 1) o |= 1u << K.tc.mpos[t];
        K.moff[m] = (uint16_t)o;
    }
    cp_async_wait_all();
    __syncthreads();

    const int vps_log = lo - 1;  // 16-byte vectors per segment (complex64: 2 per vector)
    const uint32_t nvec = 1u << (kTcSlabBits - 1);
    const uint32_t sAhi = saddr(base + kOffAhi), sAlo = saddr(base + kOffAlo);
    const uint32_t sBhi = saddr(base + kOffBhi), sBlo = saddr(base + kOffBlo);
    uint32_t phase = 0;
    bool failed = false;

    auto slab_ptr = [&](uint64_t s) -> float2 * {
        uint64_t gb = s << lo;
        for (int m = 0; m < nhi; ++m) {
            const uint64_t lowm = (1ull << P.hipos[m]) - 1;
            gb = ((gb & ~lowm) << 1) | (gb & lowm);
        }
        return state + gb;
    };
    auto issue_load = [&](const float2 *g) {
        for (uint32_t v = tid; v < nvec; v += kThreads) {
            const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
            const uint64_t so = K.seg_lo[seg & 63] | K.seg_hi[(seg >> 6) & 63];
            cp_async16(saddr(slab) + 16u * v, reinterpret_cast<const uint4 *>(g + so) + w);
        }
        cp_async_commit();
    };
    // Results go to the operand region A (64 KiB, free once the MMAs have completed) so that the
    // next slab can stream into the slab buffer while this one is multiplied and stored.
    float2 *res = reinterpret_cast<float2 *>(base + kOffAhi);
    uint32_t bphase = 0;
    bool b_pending = false;
    if (uint64_t(blockIdx.x) < nslabs) issue_load(slab_ptr(blockIdx.x));
    for (uint64_t s = blockIdx.x; s < nslabs && !failed; s += gridDim.x) {
        float2 *g = slab_ptr(s);
        cp_async_wait_all();
        __syncthreads();
        const bool more = s + gridDim.x < nslabs;
        for (int eb = 0; eb < NB && !failed; ++eb) {
            for (int h = 0; h < kParts; ++h) {
                if (!kResident && tid == 0) load_b(eb, h);  // lands while the split runs
                b_pending = !kResident;
                // BF16: one split per slab (the A operand serves all blocks); TF32: A holds one
                // K half, so every (block, half) is split again
                const bool do_split = kTf32 || eb == 0;
                if (do_split) {
                    // split row m into hi / lo in the swizzled operand layout: thread (m, p) =
                    // (tid % 128, tid / 128) converts 16-byte chunks p*4 .. p*4+3 of the row's 16
                    const uint32_t m = tid & 127u, mo = K.moff[m], c16b = (tid >> 7) * kChunksPerThread;
                    if (!kTf32) {
#pragma unroll
                        for (uint32_t c16 = c16b; c16 < c16b + kChunksPerThread; ++c16) {
                            __nv_bfloat162 hv[4], lv[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float2 a = slab[mo | K.joff[c16 * 4 + q]];
                                const __nv_bfloat16 hx = __float2bfloat16_rn(a.x), hy = __float2bfloat16_rn(a.y);
                                hv[q] = __halves2bfloat162(hx, hy);
                                lv[q] = __halves2bfloat162(__float2bfloat16_rn(a.x - __bfloat162float(hx)),
                                                           __float2bfloat16_rn(a.y - __bfloat162float(hy)));
                            }
                            const uint32_t off = op_chunk_offset(m, c16);
                            *reinterpret_cast<uint4 *>(base + kOffAhi + off) = *reinterpret_cast<const uint4 *>(hv);
                            *reinterpret_cast<uint4 *>(base + kOffAlo + off) = *reinterpret_cast<const uint4 *>(lv);
                        }
                    } else {
                        // K half h holds targets j = 32h .. 32h + 31; a chunk is 2 amplitudes
#pragma unroll
                        for (uint32_t c16 = c16b; c16 < c16b + kChunksPerThread; ++c16) {
                            const uint32_t j = 32u * uint32_t(h) + 2u * c16;
                            const float2 a0 = slab[mo | K.joff[j]], a1 = slab[mo | K.joff[j + 1]];
                            const float xs[4] = {a0.x, a0.y, a1.x, a1.y};
                            uint32_t hv[4], lv[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                hv[q] = to_tf32(xs[q]);
                                lv[q] = to_tf32(xs[q] - __uint_as_float(hv[q]));
                            }
                            const uint32_t off = op_chunk_offset(m, c16);
                            *reinterpret_cast<uint4 *>(base + kOffAhi + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                            *reinterpret_cast<uint4 *>(base + kOffAlo + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
                        }
                    }
                }
                const bool last_split = do_split && (kTf32 ? (eb == NB - 1 && h == kParts - 1) : true);
                if (last_split) {
                    __syncthreads();  // every split has read the slab buffer
                    // prefetch this CTA's next slab into it; it lands while the GEMMs run
                    if (more) issue_load(slab_ptr(s + gridDim.x));
                }
                if (!kResident) {
                    const bool okb = mbar_wait_bounded(bbar, bphase);
                    if (__syncthreads_or(!okb)) {  // the copy stays pending: waited for at exit
                        if (tid == 0) atomicExch(status, QS_ETIMEOUT);
                        failed = true;
                        break;
                    }
                    bphase ^= 1u;
                    b_pending = false;
                }
                fence_proxy_async();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    // D_eb (+)= A_hi E_hi^T + A_hi E_lo^T + A_lo E_hi^T over 8 K-steps of 32 bytes
                    const uint32_t ops[3][2] = {{sAhi, sBhi}, {sAhi, sBlo}, {sAlo, sBhi}};
                    const uint32_t dcol = tmem + uint32_t(eb) * kTcK;
#pragma unroll
                    for (int pr = 0; pr < 3; ++pr)
#pragma unroll
                        for (int ks = 0; ks < 8; ++ks) {
                            const uint32_t koff = (uint32_t(ks) >> 2) * (kTcRows * 128u) + (uint32_t(ks) & 3u) * 32u;
                            const uint32_t acc = (h | pr | ks) ? 1u : 0u;
                            if (kTf32) mma_tf32(dcol, smem_desc(ops[pr][0] + koff), smem_desc(ops[pr][1] + koff), acc);
                            else mma_bf16(dcol, smem_desc(ops[pr][0] + koff), smem_desc(ops[pr][1] + koff), acc);
                        }
                    mma_commit(bar);
                }
                const bool ok = mbar_wait_bounded(bar, phase);
                phase ^= 1u;
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) atomicExch(status, QS_ETIMEOUT);
                    mbar_wait_bounded(bar, phase ^ 1u);  // bounded grace for the MMAs in flight
                    failed = true;
                    break;
                }
                tc_fence_after();
            }
        }
        if (failed) break;
        // epilogue: warp w reads rows 32q..32q+31 of its TMEM lane quarter q = w % 4, columns
        // 32h..32h+31 with h = w / 4, into the free operand region
        {
            constexpr uint32_t kColsW = kTcK / (kThreads / 128);
            const uint32_t q4 = warp & 3u, m = q4 * 32 + lane, cb = (warp >> 2) * kColsW;
            if (NB == 1) {
                const uint32_t mo = K.moff[m];
#pragma unroll 1
                for (uint32_t c0 = cb; c0 < cb + kColsW; c0 += 32) {
                    float r[32];
                    tmem_ld32(tmem + ((q4 * 32u) << 16) + c0, r);
#pragma unroll
                    for (int q = 0; q < 16; ++q) res[mo | K.joff[c0 / 2 + q]] = make_float2(r[2 * q], r[2 * q + 1]);
                }
            } else {
                // 7-qubit gate: row bit 6 is the gate's target 6.  Output row (t', rr) is
                // D_{2t'}(0, rr) + D_{2t'+1}(1, rr): rows with bit 6 clear write their part of both
                // outputs, then rows with bit 6 set add theirs.
                const uint32_t hi = m >> 6, rr = m & 63u;
                const uint32_t mo0 = K.moff[rr], mo1 = K.moff[rr | 64u];
#pragma unroll 1
                for (int ph = 0; ph < 2; ++ph) {
                    if (uint32_t(ph) == hi) {
#pragma unroll 1
                        for (int t = 0; t < 2; ++t) {
                            const uint32_t acc = 2u * uint32_t(t) + hi, mo = t ? mo1 : mo0;
                            float r[32];
                            tmem_ld32(tmem + ((q4 * 32u) << 16) + acc * kTcK + cb, r);
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                float2 &o = res[mo | K.joff[cb / 2 + q]];
                                if (ph == 0) o = make_float2(r[2 * q], r[2 * q + 1]);
                                else o = make_float2(o.x + r[2 * q], o.y + r[2 * q + 1]);
                            }
                        }
                    }
                    __syncthreads();
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        for (uint32_t v = tid; v < nvec; v += kThreads) {
            const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
            const uint64_t so = K.seg_lo[seg & 63] | K.seg_hi[(seg >> 6) & 63];
            __stcs(reinterpret_cast<float4 *>(g + so) + w, reinterpret_cast<const float4 *>(res)[v]);
        }
        __syncthreads();  // the operand region is rewritten by the next split
    }
    if (b_pending) mbar_wait_bounded(bbar, bphase);  // a bulk copy issued before a timeout
    cp_async_wait_all();  // no copy may land after the CTA has left (timeout path)
    (void)failed;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
}

}  // namespace

size_t tc_image_bytes(int mode, int width)
{
    return (mode == QS_TC_TF32X3 ? 4 : 2) * size_t(kOpBytes) * (width == 7 ? 4 : 1);
}

namespace {
template <int MODE, int NB>
int launch_tc_t(const LaunchCtx &c, const DevTc *d_tc, const void *d_images, char *err, size_t errlen)
{
    const size_t smem = kOffCtl + sizeof(TcCtl) + 1024;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaFuncSetAttribute(tc_kernel<MODE, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_dev = dev;
    }
    const uint64_t nslabs = 1ull << (c.n - kTcSlabBits);
    uint64_t grid = uint64_t(num_sms());
    if (grid > nslabs) grid = nslabs;
    tc_kernel<MODE, NB><<<(unsigned)grid, kThreads, smem, (cudaStream_t)c.stream>>>(
        reinterpret_cast<float2 *>(c.amp), d_tc, reinterpret_cast<const unsigned char *>(d_images), nslabs,
        device_status_ptr());
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "tensor-core launch failed: %s", cudaGetErrorString(e));
        return QS_ECUDA;
    }
    return QS_OK;
}
}  // namespace

int launch_tc(const LaunchCtx &c, const DevTc *d_tc, const DevTc &h, const void *d_images, char *err,
              size_t errlen)
{
    if (c.dt != QS_C64) {
        snprintf(err, errlen, "tensor-core path: complex64 states only");
        return QS_EUNSUPPORTED;
    }
    if (h.width != 6 && h.width != 7) {
        snprintf(err, errlen, "tensor-core path: gate width %d (6 or 7)", h.width);
        return QS_EINVAL;
    }
    const bool w7 = h.width == 7;
    if (h.mode == QS_TC_BF16X3)
        return w7 ? launch_tc_t<QS_TC_BF16X3, 4>(c, d_tc, d_images, err, errlen)
                  : launch_tc_t<QS_TC_BF16X3, 1>(c, d_tc, d_images, err, errlen);
    if (h.mode == QS_TC_TF32X3)
        return w7 ? launch_tc_t<QS_TC_TF32X3, 4>(c, d_tc, d_images, err, errlen)
                  : launch_tc_t<QS_TC_TF32X3, 1>(c, d_tc, d_images, err, errlen);
    snprintf(err, errlen, "tensor-core path: unknown mode %d", h.mode);
    return QS_EINVAL;
}

}  // namespace qs
