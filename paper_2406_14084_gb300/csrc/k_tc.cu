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
// tcgen05.commit to an mbarrier -> tcgen05.ld of the accumulator by the 16 warps (four per TMEM
// lane quarter) -> straight to HBM when the slab's 4 lowest bits are row bits (one read-back
// instruction then covers two whole 128-byte segments), else through the (now free), swizzled
// operand region and 16-byte stores.  The next slab's gather is issued as soon as the split has
// read the slab buffer, so it overlaps the MMAs, the accumulator read-back and the stores.
// BF16 x 3 6-qubit gates in that usual layout run in tc_pipe_kernel (below), which keeps two
// slabs in flight per CTA.  Every mbarrier wait is bounded; on expiry the CTA
// records QS_ETIMEOUT, waits (bounded) for its copies in flight, releases its tensor memory
// and exits.
//
// TF32 x 3 mode (kind::tf32): the same three products with TF32 parts (10 stored mantissa bits
// each, so hi + lo carries about 22 bits against BF16's 16).  The 4-byte operands take twice the
// space, so each slab is split and multiplied in two K halves of 64 (targets 0..31, then
// 32..63), both accumulating into the same TMEM columns.
//
// 7-qubit gates: the 7th target is row bit 6 of S, and the 128x128 unitary is applied as its
// four 64x64 blocks in transposed form (E as the M = 128 operand, each half of S as an N = 64
// operand; see the kernel).  E images that do not stay in shared memory come from L2 by bulk
// copies: for TF32 6-qubit gates one 64 KiB copy per K half, issued before that half's split;
// for 7-qubit gates a stream of 32 KiB chunks through two buffers.
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
// shared memory: FP32 slab buffer | slab operand hi | lo | E region (64 KiB: the resident image,
// one K half's image or two stream buffers) | control block
constexpr uint32_t kOffAhi = kSlabBytes, kOffAlo = kOffAhi + kOpBytes, kOffBhi = kOffAlo + kOpBytes,
                   kOffCtl = kOffBhi + 2 * kOpBytes;
constexpr uint32_t kWaitLimit = 1u << 24;

struct TcCtl {
    unsigned long long mbar;      // all MMAs issued so far completed (every thread waits)
    unsigned long long full[2];   // E buffer b: bulk copies landed (warp 0 waits)
    unsigned long long mdone[2];  // E buffer b: its MMAs completed (warp 0 waits)
    uint32_t tmem;
    uint32_t pad;
    DevTc tc;
    uint64_t seg_lo[64], seg_hi[64];
    uint64_t jg[64];     // offset in the state (from the slab's base) of target index j
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
// the same with N = 64 (7-qubit blocks: operand B is the 64 slab rows of one 7th-bit value)
constexpr uint32_t kIdescBf16N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((uint32_t(kTcRows) >> 4) << 24);
constexpr uint32_t kIdescTf32N64 = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((uint32_t(kTcRows) >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
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

// Result-buffer slot of slab amplitude x: bits 0-3 XORed with bits 4-7, 8-11 and 12 (an
// involution).  A read-back instruction writes 32 values whose slab indices differ in 5 bits
// (32 rows of one target value for 6-qubit gates, 16 target values of two rows for 7-qubit
// gates); unswizzled, whenever those bits lie above bit 3 they all fall into one bank group.
__device__ __forceinline__ uint32_t res_swz(uint32_t x) { return x ^ (((x >> 4) ^ (x >> 8) ^ (x >> 12)) & 15u); }

// Byte offset of element (row, k) of a 128-row BF16 operand in the swizzled K-major layout:
// K is split into 128-byte atoms (64 elements) stored one after the other for all rows.
__device__ __forceinline__ uint32_t op_chunk_offset(uint32_t row, uint32_t chunk16)
{
    const uint32_t kb = chunk16 >> 3, c = chunk16 & 7;
    return kb * (kTcRows * 128u) + row * 128u + ((c ^ (row & 7u)) << 4);
}

// The kernel.  MODE = QS_TC_BF16X3 (kind::f16, K = 16 per instruction) or QS_TC_TF32X3
// (kind::tf32, K = 8; the 4-byte operands hold one K half of 64 at a time, so the slab is split
// and multiplied in two halves).  NB = 1: a 6-qubit gate, D (rows x 128) = S E^T with the slab
// matrix S as operand A.  NB = 4: a 7-qubit gate whose 7th target is row bit 6; with t', t the
// 7th bit of output and input and S_t the 64 rows with row bit 6 = t, the transposed products
//     D_t'^T (128 x 64) = sum_t E_t't S_t^T
// take E as operand A (M = 128 output reals) and S_t as operand B (N = 64 rows starting at row
// 64 t), accumulating both t in one TMEM accumulator per t' (columns 64 t' .. 64 t' + 63).
//
// E operand: for BF16 x 3 with NB = 1 the hi and lo images (64 KiB) stay in shared memory for
// the whole launch.  For TF32 x 3 with NB = 1 the half of the image that a K half needs (two
// atoms, 64 KiB) is copied in one bulk copy before that half's split.  For NB = 4 E is streamed
// from global memory (L2-resident) in chunks of one 128-byte K atom (16 KiB hi + 16 KiB lo) by
// bulk copies into two alternating buffers: chunk c + 1 is copied while chunk c is multiplied,
// and the stream runs on across slabs.  Chunk order within a slab: K half h, then E block
// eb (= 2 t' + t), then atom a of the half.
template <int MODE, int NB>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(float2 *__restrict__ state, const DevTc *__restrict__ d_tc,
              const unsigned char *__restrict__ images, uint64_t nslabs, int *status)
{
    constexpr bool kTf32 = MODE == QS_TC_TF32X3;
    constexpr int kParts = kTf32 ? 2 : 1;               // K halves per slab
    constexpr bool kResident = !kTf32 && NB == 1;
    // TF32 6-qubit: one 64 KiB copy per K half, issued before that half's split so that it
    // lands while the split runs; 7-qubit: the two-buffer chunk stream
    constexpr bool kHalfCopy = kTf32 && NB == 1;
    constexpr bool kStream = !kResident && !kHalfCopy;
    constexpr int kChunks = kParts * NB * 2;             // E chunks (K atoms) per slab
    constexpr uint32_t kAtom = kTcRows * 128u;           // one 128-row K atom: 16 KiB
    constexpr uint32_t kAtoms = 2u * kParts;             // K atoms of one E block
    constexpr uint32_t kCols = uint32_t(kTcK);           // TMEM columns: one 128-column accumulator
    constexpr uint32_t kIdesc = NB == 1 ? (kTf32 ? kIdescTf32 : kIdescBf16) : (kTf32 ? kIdescTf32N64 : kIdescBf16N64);

    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float2 *slab = reinterpret_cast<float2 *>(base);
    TcCtl &K = *reinterpret_cast<TcCtl *>(base + kOffCtl);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar = saddr(&K.mbar);
    const uint32_t full0 = saddr(&K.full[0]), mdone0 = saddr(&K.mdone[0]);  // [1] at +8

    if (tid == 0) {
        K.tc = *d_tc;
        mbar_init(bar, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(full0 + 8u * b, 1);
            mbar_init(mdone0 + 8u * b, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&K.tmem)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const unsigned char *img = images + d_tc->img;
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
    // state offset of a slab-local index: bits below lo stay, bit lo + i goes to hipos[i]; the
    // bits of a row and of a target index are disjoint, so an amplitude's offset is the OR
    for (uint32_t j = tid; j < 64; j += kThreads) {
        const uint32_t x = K.joff[j];
        K.jg[j] = K.seg_lo[(x >> lo) & 63] | K.seg_hi[(x >> (lo + 6)) & 63] | (x & ((1u << lo) - 1));
    }
    // 6-qubit gates whose 4 lowest row bits are the slab's lowest bits (the usual layout): a
    // read-back instruction covers 32 rows of one target value = two whole 128-byte segments,
    // so it stores straight to HBM; other layouts go through the swizzled result buffer
    const bool direct = NB == 1 && lo >= 4 && K.moff[1] == 1 && K.moff[2] == 2 && K.moff[4] == 4 && K.moff[8] == 8;
    __syncthreads();

    const int vps_log = lo - 1;  // 16-byte vectors per segment (complex64: 2 per vector)
    const uint32_t nvec = 1u << (kTcSlabBits - 1);
    const uint32_t sS[2] = {saddr(base + kOffAhi), saddr(base + kOffAlo)};  // slab operand hi, lo
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

    // ---- the E stream, driven by warp 0 (lane 0 issues the copies and MMAs; the whole warp
    // waits, so that no lane of it sits in another wait meanwhile): chunk c of this CTA's
    // sequence goes to buffer c & 1
    const uint64_t nmine = uint64_t(blockIdx.x) < nslabs ? (nslabs - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const uint64_t total = kStream ? nmine * kChunks : 0;
    uint64_t c_next = 0;                 // next chunk to multiply
    uint64_t c_issued = 0, c_landed = 0; // chunks whose copies were issued / waited for
    uint32_t fph = 0, mph = 0;           // per-buffer parities (bit b)
    bool ok0 = true;                     // warp 0: every wait so far succeeded
    // chunk = K atom a of E block eb, hi then lo: one contiguous 32 KiB bulk copy
    auto chunk_load = [&](uint64_t c) {
        const uint32_t cl = uint32_t(c % kChunks), b = uint32_t(c & 1);
        const uint32_t h = cl / (NB * 2), eb = (cl >> 1) % NB, a = 2 * h + (cl & 1);
        const unsigned char *src = img + size_t(eb * kAtoms + a) * 2 * kAtom;
        mbar_expect_tx(full0 + 8u * b, 2 * kAtom);
        bulk_g2s(saddr(base + kOffBhi) + b * 2 * kAtom, src, 2 * kAtom, full0 + 8u * b);
    };
    if (warp == 0 && total > 0) {
        if (lane == 0) chunk_load(0);
        c_issued = 1;
    }
    // multiply chunk c_next (warp 0): refill the other buffer once its chunk's MMAs are done,
    // wait for this chunk's copy, issue 3 products x 4 K-steps
    auto chunk_mma = [&]() {
        const uint64_t c = c_next++;
        const uint32_t cl = uint32_t(c % kChunks), b = uint32_t(c & 1);
        const uint32_t h = cl / (NB * 2), eb = (cl >> 1) % NB, ah = cl & 1;
        uint32_t bhi;
        if constexpr (!kStream) {
            if (!ok0) return;
            bhi = saddr(base + kOffBhi) + ah * 2 * kAtom;  // atom ah of the resident image or the half
        } else {
            if (!ok0) return;
            if (c >= 1) {
                const uint32_t pb = b ^ 1u;
                ok0 = __all_sync(0xffffffffu, mbar_wait_bounded(mdone0 + 8u * pb, (mph >> pb) & 1u));
                mph ^= 1u << pb;
                if (!ok0) return;
            }
            if (c + 1 < total) {
                if (lane == 0) chunk_load(c + 1);
                __syncwarp();
                c_issued = c + 2;
            }
            ok0 = __all_sync(0xffffffffu, mbar_wait_bounded(full0 + 8u * b, (fph >> b) & 1u));
            if (!ok0) return;  // the copy stays pending: waited for at exit
            fph ^= 1u << b;
            c_landed = c + 1;
            bhi = saddr(base + kOffBhi) + b * 2 * kAtom;
        }
        if (lane != 0) return;
        tc_fence_after();
        const uint32_t ehl[2] = {bhi, bhi + kAtom};
        // (slab part, E part) of the three products: hi.hi, hi.lo, lo.hi
        const uint32_t pr_s[3] = {0, 0, 1}, pr_e[3] = {0, 1, 0};
        const uint32_t tp = eb >> 1, t = eb & 1;
#pragma unroll
        for (int pr = 0; pr < 3; ++pr)
#pragma unroll
            for (uint32_t ks = 0; ks < 4; ++ks) {
                const uint32_t soff = ah * kAtom + ks * 32u, eoff = ks * 32u;
                if (NB == 1) {
                    const uint32_t acc = (h | ah | uint32_t(pr) | ks) ? 1u : 0u;
                    const uint64_t ad = smem_desc(sS[pr_s[pr]] + soff), bd = smem_desc(ehl[pr_e[pr]] + eoff);
                    if (kTf32) mma_tf32(tmem, ad, bd, kIdesc, acc);
                    else mma_bf16(tmem, ad, bd, kIdesc, acc);
                } else {
                    const uint32_t acc = (t | h | ah | uint32_t(pr) | ks) ? 1u : 0u;
                    const uint64_t ad = smem_desc(ehl[pr_e[pr]] + eoff), bd = smem_desc(sS[pr_s[pr]] + soff + t * 8192u);
                    if (kTf32) mma_tf32(tmem + tp * 64u, ad, bd, kIdesc, acc);
                    else mma_bf16(tmem + tp * 64u, ad, bd, kIdesc, acc);
                }
            }
        if (kStream) mma_commit(mdone0 + 8u * b);
    };

    // Results go to the operand region A (64 KiB, free once the MMAs have completed) so that the
    // next slab can stream into the slab buffer while this one is multiplied and stored.
    float2 *res = reinterpret_cast<float2 *>(base + kOffAhi);
    if (nmine > 0) issue_load(slab_ptr(blockIdx.x));
    for (uint64_t s = blockIdx.x; s < nslabs && !failed; s += gridDim.x) {
        float2 *g = slab_ptr(s);
        cp_async_wait_all();
        __syncthreads();
        for (int h = 0; h < kParts; ++h) {
            if (kHalfCopy && warp == 0) {  // every MMA so far has completed: the buffer is free
                if (lane == 0) {
                    mbar_expect_tx(full0, 4 * kAtom);
                    bulk_g2s(saddr(base + kOffBhi), img + size_t(h) * 4 * kAtom, 4 * kAtom, full0);
                }
                __syncwarp();
                ++c_issued;
            }
            // split row m into hi / lo in the swizzled K-major operand layout: thread (m, p) =
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
            if (h == kParts - 1) {
                __syncthreads();  // every split has read the slab buffer
                // prefetch this CTA's next slab into it; it lands while the GEMMs run
                if (s + gridDim.x < nslabs) issue_load(slab_ptr(s + gridDim.x));
            }
            fence_proxy_async();
            __syncthreads();
            if (warp == 0) {
                if (kHalfCopy && ok0) {
                    ok0 = __all_sync(0xffffffffu, mbar_wait_bounded(full0, fph & 1u));
                    if (ok0) {
                        fph ^= 1u;
                        c_landed = c_issued;
                    }
                }
                for (int k = 0; k < NB * 2; ++k) chunk_mma();
                if (lane == 0) mma_commit(bar);  // arrives once every MMA issued so far has completed
                __syncwarp();
            }
            const bool ok = mbar_wait_bounded(bar, phase);
            phase ^= 1u;
            if (__syncthreads_or(!ok || (tid == 0 && !ok0))) {
                if (tid == 0) atomicExch(status, QS_ETIMEOUT);
                if (!ok) mbar_wait_bounded(bar, phase ^ 1u);  // bounded grace for the MMAs in flight
                failed = true;
                break;
            }
            tc_fence_after();
        }
        if (failed) break;
        // epilogue: warp w reads TMEM lane quarter q = w % 4 (lanes 32q .. 32q + 31), columns
        // 32g .. 32g + 31 with g = w / 4, into the free operand region
        {
            const uint32_t q4 = warp & 3u, g4 = warp >> 2;
            float r[32];
            tmem_ld32(tmem + ((q4 * 32u) << 16) + 32u * g4, r);
            if (NB == 1) {
                // lane = slab row m, columns = output reals 2j + (re, im) for j = 16 g .. 16 g + 15
                const uint32_t mo = K.moff[q4 * 32 + lane];
                if (direct) {
                    const uint64_t mg = K.seg_lo[(mo >> lo) & 63] | K.seg_hi[(mo >> (lo + 6)) & 63] | (mo & ((1u << lo) - 1));
#pragma unroll
                    for (int q = 0; q < 16; ++q) __stcs(g + (mg | K.jg[16 * g4 + q]), make_float2(r[2 * q], r[2 * q + 1]));
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) res[res_swz(mo | K.joff[16 * g4 + q])] = make_float2(r[2 * q], r[2 * q + 1]);
                }
            } else {
                // lane = output real 2j + c (j = 16 q + lane / 2), columns = rows rr0 .. rr0 + 31
                // of output half t' = g / 2 (rr0 = 32 (g % 2)); lanes 2i, 2i + 1 swap halves so
                // that each writes whole complex values
                const uint32_t c = lane & 1u, jo = K.joff[16 * q4 + (lane >> 1)];
                const uint32_t row0 = ((g4 >> 1) << 6) | ((g4 & 1u) << 5);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float send = c ? r[i] : r[16 + i];
                    const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
                    if (c == 0) res[res_swz(K.moff[row0 + i] | jo)] = make_float2(r[i], recv);
                    else res[res_swz(K.moff[row0 + 16 + i] | jo)] = make_float2(recv, r[16 + i]);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        if (!direct) {
            for (uint32_t v = tid; v < nvec; v += kThreads) {
                const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
                const uint64_t so = K.seg_lo[seg & 63] | K.seg_hi[(seg >> 6) & 63];
                const float2 a0 = res[res_swz(2 * v)], a1 = res[res_swz(2 * v + 1)];
                __stcs(reinterpret_cast<float4 *>(g + so) + w, make_float4(a0.x, a0.y, a1.x, a1.y));
            }
            __syncthreads();  // the operand region is rewritten by the next split
        }
    }
    // timeout path: no copy may land after the CTA has left
    if (warp == 0)
        for (uint64_t c = c_landed; c < c_issued; ++c) {
            const uint32_t b = kHalfCopy ? 0u : uint32_t(c & 1);
            mbar_wait_bounded(full0 + 8u * b, (fph >> b) & 1u);
            fph ^= 1u << b;
        }
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
}


// ---------------------------------------------------------------------------------------------
// Pipelined BF16 x 3 kernel for 6-qubit gates whose 4 lowest row bits are the slab's 4 lowest
// bits (the usual layout; the read-back then stores straight to HBM).  The split converts the
// FP32 slab in place -- hi and lo BF16 parts take exactly the FP32 footprint -- so two slab
// buffers X0, X1 and the resident E images fit shared memory (3 x 64 KiB), and two TMEM
// accumulators let slab i's split and MMAs overlap slab i-1's read-back, while slab i+2's
// gather is in flight:
//   iteration i:  wait gather(i) -> split(i) in X(i&1) -> MMAs(i) into accumulator i&1
//                 -> wait MMAs(i-1) -> read-back(i-1) to HBM
//                 -> wait MMAs(i) (X(i&1) free) -> gather(i+2) into X(i&1)
constexpr uint32_t kPipeX = 1u << 16;                   // one slab buffer: 64 KiB
constexpr uint32_t kPipeOffE = 2 * kPipeX, kPipeOffCtl = 3 * kPipeX;

struct TcPipeCtl {
    unsigned long long bar[2];  // MMAs into accumulator b completed
    uint32_t tmem;
    uint32_t pad;
    DevTc tc;
    uint64_t seg_lo[64], seg_hi[64];
    uint64_t jg[64];     // state offset (from the slab's base) of target index j
    uint16_t joff[64];   // slab-local offset of target index j
    uint16_t moff[128];  // slab-local offset of row m
};

__global__ void __launch_bounds__(kThreads, 1)
    tc_pipe_kernel(float2 *__restrict__ state, const DevTc *__restrict__ d_tc,
                   const unsigned char *__restrict__ images, uint64_t nslabs, int *status)
{
    constexpr uint32_t kCols = 2u * kTcK;  // two 128-column accumulators
    constexpr uint32_t kAtom = kTcRows * 128u;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    TcPipeCtl &K = *reinterpret_cast<TcPipeCtl *>(base + kPipeOffCtl);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar0 = saddr(&K.bar[0]);

    if (tid == 0) {
        K.tc = *d_tc;
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8u, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&K.tmem)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    {
        // resident E images: per K atom, hi then lo (64 KiB)
        const unsigned char *img = images + d_tc->img;
        const uint32_t dst = saddr(base + kPipeOffE);
        for (uint32_t v = tid; v < (4 * kAtom) / 16; v += kThreads) cp_async16(dst + 16 * v, img + 16 * v);
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
    for (uint32_t j = tid; j < 64; j += kThreads) {
        const uint32_t x = K.joff[j];
        K.jg[j] = K.seg_lo[(x >> lo) & 63] | K.seg_hi[(x >> (lo + 6)) & 63] | (x & ((1u << lo) - 1));
    }
    __syncthreads();

    const int vps_log = lo - 1;  // 16-byte vectors per segment
    const uint32_t nvec = 1u << (kTcSlabBits - 1);
    const uint64_t nmine = uint64_t(blockIdx.x) < nslabs ? (nslabs - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto slab_ptr = [&](uint64_t i) -> float2 * {  // this CTA's i-th slab
        uint64_t gb = (uint64_t(blockIdx.x) + i * gridDim.x) << lo;
        for (int m = 0; m < nhi; ++m) {
            const uint64_t lowm = (1ull << P.hipos[m]) - 1;
            gb = ((gb & ~lowm) << 1) | (gb & lowm);
        }
        return state + gb;
    };
    auto issue_gather = [&](uint64_t i) {
        const float2 *g = slab_ptr(i);
        const uint32_t X = saddr(base + uint32_t(i & 1) * kPipeX);
        for (uint32_t v = tid; v < nvec; v += kThreads) {
            const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
            const uint64_t so = K.seg_lo[seg & 63] | K.seg_hi[(seg >> 6) & 63];
            cp_async16(X + 16u * v, reinterpret_cast<const uint4 *>(g + so) + w);
        }
        cp_async_commit();
    };
    if (nmine > 0) issue_gather(0);
    if (nmine > 1) issue_gather(1);
    uint32_t ph = 0;       // bit b: parity of accumulator b's next completion
    uint32_t pending = 0;  // bit b: a commit on bar[b] not yet waited for
    bool failed = false;
    auto wait_acc = [&](uint32_t b) -> bool {  // every thread; false (for all) on a timeout
        const bool ok = mbar_wait_bounded(bar0 + 8u * b, (ph >> b) & 1u);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(status, QS_ETIMEOUT);
            return false;
        }
        ph ^= 1u << b;
        pending &= ~(1u << b);
        return true;
    };
    for (uint64_t i = 0; i <= nmine; ++i) {
        if (i < nmine) {
            // gather(i) is the older of at most two outstanding copy groups
            if (i + 1 < nmine) cp_async_wait<1>();
            else cp_async_wait<0>();
            __syncthreads();
            unsigned char *X = base + uint32_t(i & 1) * kPipeX;
            const float2 *slab = reinterpret_cast<const float2 *>(X);
            // split in place: thread (m, p) = (tid % 128, tid / 128) reads its 16 amplitudes,
            // then (after every thread has read) writes its 4 hi and 4 lo 16-byte chunks
            const uint32_t m = tid & 127u, mo = K.moff[m], c16b = (tid >> 7) * kChunksPerThread;
            uint4 hv[kChunksPerThread], lv[kChunksPerThread];
#pragma unroll
            for (uint32_t c = 0; c < kChunksPerThread; ++c) {
                __nv_bfloat162 h2[4], l2[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 a = slab[mo | K.joff[(c16b + c) * 4 + q]];
                    const __nv_bfloat16 hx = __float2bfloat16_rn(a.x), hy = __float2bfloat16_rn(a.y);
                    h2[q] = __halves2bfloat162(hx, hy);
                    l2[q] = __halves2bfloat162(__float2bfloat16_rn(a.x - __bfloat162float(hx)),
                                               __float2bfloat16_rn(a.y - __bfloat162float(hy)));
                }
                hv[c] = *reinterpret_cast<const uint4 *>(h2);
                lv[c] = *reinterpret_cast<const uint4 *>(l2);
            }
            __syncthreads();
#pragma unroll
            for (uint32_t c = 0; c < kChunksPerThread; ++c) {
                const uint32_t off = op_chunk_offset(m, c16b + c);
                *reinterpret_cast<uint4 *>(X + off) = hv[c];
                *reinterpret_cast<uint4 *>(X + 2 * kAtom + off) = lv[c];
            }
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                // D_(i&1) = S_hi E_hi^T + S_hi E_lo^T + S_lo E_hi^T over 8 K-steps of 16; the E
                // image holds per K atom its hi part, then its lo part
                const uint32_t sx = saddr(X), se = saddr(base + kPipeOffE);
                const uint32_t d = tmem + uint32_t(i & 1) * kTcK;
#pragma unroll
                for (uint32_t pr = 0; pr < 3; ++pr)
#pragma unroll
                    for (uint32_t ks = 0; ks < 8; ++ks) {
                        const uint32_t atom = ks >> 2, koff = (ks & 3u) * 32u;
                        const uint32_t a = sx + (pr == 2 ? 2 * kAtom : 0u) + atom * kAtom + koff;
                        const uint32_t b = se + atom * 2 * kAtom + (pr == 1 ? kAtom : 0u) + koff;
                        mma_bf16(d, smem_desc(a), smem_desc(b), kIdescBf16, (pr | ks) ? 1u : 0u);
                    }
                mma_commit(bar0 + 8u * uint32_t(i & 1));
            }
            pending |= 1u << uint32_t(i & 1);
        }
        if (i >= 1) {
            // read-back of slab i - 1 straight to HBM: warp w reads TMEM lane quarter w % 4
            // (32 rows, = two whole 128-byte segments per target value), columns 32 (w / 4) ..
            const uint32_t b = uint32_t((i - 1) & 1);
            if ((pending >> b & 1) && !wait_acc(b)) {
                failed = true;
                break;
            }
            tc_fence_after();
            float2 *g = slab_ptr(i - 1);
            const uint32_t q4 = warp & 3u, g4 = warp >> 2;
            float r[32];
            tmem_ld32(tmem + b * kTcK + ((q4 * 32u) << 16) + 32u * g4, r);
            const uint32_t mo = K.moff[q4 * 32 + lane];
            const uint64_t mg = K.seg_lo[(mo >> lo) & 63] | K.seg_hi[(mo >> (lo + 6)) & 63] | (mo & ((1u << lo) - 1));
#pragma unroll
            for (int q = 0; q < 16; ++q) __stcs(g + (mg | K.jg[16 * g4 + q]), make_float2(r[2 * q], r[2 * q + 1]));
        }
        if (i + 2 < nmine) {
            // slab i's buffer is free once its MMAs have completed: gather slab i + 2 into it
            if (!wait_acc(uint32_t(i & 1))) {
                failed = true;
                break;
            }
            issue_gather(i + 2);
        }
        tc_fence_before();
        __syncthreads();  // accumulator (i - 1) & 1 has been read before MMAs(i + 1) overwrite it
    }
    // timeout path: copies and MMAs in flight finish before the CTA leaves
    cp_async_wait_all();
    for (uint32_t b = 0; b < 2; ++b)
        if (failed && (pending >> b & 1)) mbar_wait_bounded(bar0 + 8u * b, (ph >> b) & 1u);
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

int launch_tc_pipe(const LaunchCtx &c, const DevTc *d_tc, const void *d_images, char *err, size_t errlen)
{
    const size_t smem = kPipeOffCtl + sizeof(TcPipeCtl) + 1024;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaFuncSetAttribute(tc_pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_dev = dev;
    }
    const uint64_t nslabs = 1ull << (c.n - kTcSlabBits);
    uint64_t grid = uint64_t(num_sms());
    if (grid > nslabs) grid = nslabs;
    tc_pipe_kernel<<<(unsigned)grid, kThreads, smem, (cudaStream_t)c.stream>>>(
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
    // 6-qubit BF16 gates in the usual layout (the slab's 4 lowest bits are row bits 0-3): the
    // pipelined kernel
    if (h.mode == QS_TC_BF16X3 && !w7 && h.slab.lo >= 4 && h.mpos[0] == 0 && h.mpos[1] == 1 && h.mpos[2] == 2 &&
        h.mpos[3] == 3)
        return launch_tc_pipe(c, d_tc, d_images, err, errlen);
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
