// k_slab.cu -- the in-cache gate-block kernel (arXiv 2406.14084, Alg. 3 and Sec. V-A) for sm_103a.
//
// Persistent CTAs (one per SM, two slab buffers each) walk over the slabs of the state.  For
// each slab:
//   1. Load: every thread issues 16-byte asynchronous copies (cp.async) of the slab's
//      segments (2^lo contiguous amplitudes each) from HBM into shared memory, one slab ahead
//      of the computation.  (One bulk-copy instruction per 128-byte segment, as issued by a
//      single warp, reached only ~1.3 TB/s on GB300; 16-byte copies from all threads do not
//      have that per-instruction limit.)
//   2. The gate block: a sequence of ops.  OP_STAGE ops run in registers: each thread loads
//      the 2^r amplitudes of one group (r = 5 for complex64, 4 for complex128), applies every
//      sub-op of the stage with compile-time register indices, and writes the group back -- the
//      paper's per-gate loop unrolling taken to the register file, so a stage of m gates costs
//      one shared-memory round trip instead of m.  Ops that cannot run in registers (dense
//      gates on 3+ qubits, wide diagonal tables) run directly on the shared-memory slab.
//   3. Store: 16-byte streaming stores back to the same addresses, optionally through a bit
//      permutation of the slab index (this is how remap passes relabel qubits in place).
// Bits of the state index outside the slab are constant within a CTA's slab, so controls and
// diagonal factors on those qubits are resolved per CTA.
#include <cuda_runtime.h>

#include <cstdio>

#include "dev_common.cuh"
#include "qs_internal.h"

namespace qs {

__device__ int g_qs_device_status;

namespace {

constexpr uint32_t kWaitLimit = 1u << 24;  // mbarrier polls (with backoff) before giving up

struct __align__(16) SlabShared {
    uint64_t seg_lo[64];   // deposit of hi-bit index bits 0..5 into physical positions
    uint64_t seg_hi[64];   // deposit of hi-bit index bits 6..11
    uint16_t inv_lo[256];  // store permutation: source local index of destination bits 0..7
    uint16_t inv_hi[256];  //                                    ... of destination bits 8..15
    DevPass pass;
    unsigned long long full[2];   // TMA load of buffer k has landed
    unsigned long long empty[2];  // buffer k has been stored back and may be refilled
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 64) __nanosleep(128);
    }
    return false;
}

// 1-D bulk copy global -> shared (TMA), completion counted on the mbarrier in bytes.
__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void *src, uint32_t bytes,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void st_stream(uint4 *p, uint4 v)
{
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// ------------------------------------------------------------------ register sub-ops

template <typename C, int RB, int J, bool CTL>
__device__ __forceinline__ void sub_g1_impl(C (&v)[1 << RB], const C *__restrict__ M, uint32_t scm)
{
    const C m00 = M[0], m01 = M[1], m10 = M[2], m11 = M[3];
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) {
        if (e & (1 << J)) continue;
        if (CTL && (uint32_t(e) & scm) != scm) continue;
        const int e1 = e | (1 << J);
        const C a = v[e], b = v[e1];
        v[e] = cmac(m01, b, cmul(m00, a));
        v[e1] = cmac(m11, b, cmul(m10, a));
    }
}

template <typename C, int RB, int J>
__device__ __forceinline__ void sub_g1(C (&v)[1 << RB], const C *__restrict__ M, uint32_t scm)
{
    if (scm == 0) sub_g1_impl<C, RB, J, false>(v, M, 0);
    else sub_g1_impl<C, RB, J, true>(v, M, scm);
}

template <typename C, int RB, int J0, int J1, bool CTL>
__device__ __forceinline__ void sub_g2_impl(C (&v)[1 << RB], const C *__restrict__ M, uint32_t scm)
{
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) {
        if (e & ((1 << J0) | (1 << J1))) continue;
        if (CTL && (uint32_t(e) & scm) != scm) continue;
        const int i0 = e, i1 = e | (1 << J0), i2 = e | (1 << J1), i3 = e | (1 << J0) | (1 << J1);
        const C a0 = v[i0], a1 = v[i1], a2 = v[i2], a3 = v[i3];
        C r[4];
#pragma unroll
        for (int row = 0; row < 4; ++row) {
            C acc = cmul(M[row * 4 + 0], a0);
            acc = cmac(M[row * 4 + 1], a1, acc);
            acc = cmac(M[row * 4 + 2], a2, acc);
            acc = cmac(M[row * 4 + 3], a3, acc);
            r[row] = acc;
        }
        v[i0] = r[0];
        v[i1] = r[1];
        v[i2] = r[2];
        v[i3] = r[3];
    }
}

template <typename C, int RB, int J0, int J1>
__device__ __forceinline__ void sub_g2(C (&v)[1 << RB], const C *__restrict__ M, uint32_t scm)
{
    if (scm == 0) sub_g2_impl<C, RB, J0, J1, false>(v, M, 0);
    else sub_g2_impl<C, RB, J0, J1, true>(v, M, scm);
}

// Phase p on the elements whose bits MASK are all set (MASK is a compile-time constant).
template <typename C, int RB, int MASK, int UNUSED>
__device__ __forceinline__ void sub_phase_mask(C (&v)[1 << RB], C p, bool neg)
{
    if (neg) {
#pragma unroll
        for (int e = 0; e < (1 << RB); ++e)
            if ((e & MASK) == MASK) {
                v[e].x = -v[e].x;
                v[e].y = -v[e].y;
            }
    } else {
#pragma unroll
        for (int e = 0; e < (1 << RB); ++e)
            if ((e & MASK) == MASK) v[e] = cmul(p, v[e]);
    }
}

// 2x2 matrix with real entries (H, RY, ...): half the arithmetic of the complex case.
template <typename C, int RB, int J, bool CTL>
__device__ __forceinline__ void sub_g1r_impl(C (&v)[1 << RB], const C *__restrict__ M, uint32_t scm)
{
    const auto m00 = M[0].x, m01 = M[1].x, m10 = M[2].x, m11 = M[3].x;
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) {
        if (e & (1 << J)) continue;
        if (CTL && (uint32_t(e) & scm) != scm) continue;
        const int e1 = e | (1 << J);
        const C a = v[e], b = v[e1];
        v[e].x = fma(m01, b.x, m00 * a.x);
        v[e].y = fma(m01, b.y, m00 * a.y);
        v[e1].x = fma(m11, b.x, m10 * a.x);
        v[e1].y = fma(m11, b.y, m10 * a.y);
    }
}

template <typename C, int RB, int J>
__device__ __forceinline__ void sub_g1r(C (&v)[1 << RB], const C *__restrict__ M, uint32_t scm)
{
    if (scm == 0) sub_g1r_impl<C, RB, J, false>(v, M, 0);
    else sub_g1r_impl<C, RB, J, true>(v, M, scm);
}

template <typename C, int RB, int J>
__device__ __forceinline__ void sub_x(C (&v)[1 << RB], uint32_t scm)
{
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) {
        if (e & (1 << J)) continue;
        if ((uint32_t(e) & scm) != scm) continue;
        const C t = v[e];
        v[e] = v[e | (1 << J)];
        v[e | (1 << J)] = t;
    }
}

template <typename C, int RB, int J0, int J1>
__device__ __forceinline__ void sub_swap(C (&v)[1 << RB], uint32_t scm)
{
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) {
        // elements with bit J0 = 1, bit J1 = 0 exchange with bit J0 = 0, bit J1 = 1
        if (!(e & (1 << J0)) || (e & (1 << J1))) continue;
        if ((uint32_t(e) & scm) != scm) continue;
        const int f = e ^ ((1 << J0) | (1 << J1));
        const C t = v[e];
        v[e] = v[f];
        v[f] = t;
    }
}

template <typename C, int RB>
__device__ __forceinline__ void apply_sub(C (&v)[1 << RB], const DevSub &s, uint32_t gbase,
                                          uint64_t cta_base, const C *__restrict__ coef)
{
    if ((gbase & s.lcm) != s.lcm || (cta_base & s.ocm) != s.ocm) return;
    const C *__restrict__ M = coef + s.mat;
    const uint32_t scm = s.scm;
    switch (s.type) {
    case SB_G1:
        switch (s.j0) {
        case 0: sub_g1<C, RB, 0>(v, M, scm); break;
        case 1: sub_g1<C, RB, 1>(v, M, scm); break;
        case 2: sub_g1<C, RB, 2>(v, M, scm); break;
        case 3: sub_g1<C, RB, 3>(v, M, scm); break;
        case 4: if (RB > 4) sub_g1<C, RB, (RB > 4 ? 4 : 0)>(v, M, scm); break;
        default: break;
        }
        break;
    case SB_G2:
        switch (s.j0 * 8 + s.j1) {
        case 0 * 8 + 1: sub_g2<C, RB, 0, 1>(v, M, scm); break;
        case 0 * 8 + 2: sub_g2<C, RB, 0, 2>(v, M, scm); break;
        case 0 * 8 + 3: sub_g2<C, RB, 0, 3>(v, M, scm); break;
        case 1 * 8 + 2: sub_g2<C, RB, 1, 2>(v, M, scm); break;
        case 1 * 8 + 3: sub_g2<C, RB, 1, 3>(v, M, scm); break;
        case 2 * 8 + 3: sub_g2<C, RB, 2, 3>(v, M, scm); break;
        case 0 * 8 + 4: if (RB > 4) sub_g2<C, RB, 0, (RB > 4 ? 4 : 1)>(v, M, scm); break;
        case 1 * 8 + 4: if (RB > 4) sub_g2<C, RB, 1, (RB > 4 ? 4 : 2)>(v, M, scm); break;
        case 2 * 8 + 4: if (RB > 4) sub_g2<C, RB, 2, (RB > 4 ? 4 : 3)>(v, M, scm); break;
        case 3 * 8 + 4: if (RB > 4) sub_g2<C, RB, 3, (RB > 4 ? 4 : 0)>(v, M, scm); break;
        default: break;
        }
        break;
    case SB_X:
        switch (s.j0) {
        case 0: sub_x<C, RB, 0>(v, scm); break;
        case 1: sub_x<C, RB, 1>(v, scm); break;
        case 2: sub_x<C, RB, 2>(v, scm); break;
        case 3: sub_x<C, RB, 3>(v, scm); break;
        case 4: if (RB > 4) sub_x<C, RB, (RB > 4 ? 4 : 0)>(v, scm); break;
        default: break;
        }
        break;
    case SB_SWAP:
        switch (s.j0 * 8 + s.j1) {
        case 0 * 8 + 1: sub_swap<C, RB, 0, 1>(v, scm); break;
        case 0 * 8 + 2: sub_swap<C, RB, 0, 2>(v, scm); break;
        case 0 * 8 + 3: sub_swap<C, RB, 0, 3>(v, scm); break;
        case 1 * 8 + 2: sub_swap<C, RB, 1, 2>(v, scm); break;
        case 1 * 8 + 3: sub_swap<C, RB, 1, 3>(v, scm); break;
        case 2 * 8 + 3: sub_swap<C, RB, 2, 3>(v, scm); break;
        case 0 * 8 + 4: if (RB > 4) sub_swap<C, RB, 0, (RB > 4 ? 4 : 1)>(v, scm); break;
        case 1 * 8 + 4: if (RB > 4) sub_swap<C, RB, 1, (RB > 4 ? 4 : 2)>(v, scm); break;
        case 2 * 8 + 4: if (RB > 4) sub_swap<C, RB, 2, (RB > 4 ? 4 : 3)>(v, scm); break;
        case 3 * 8 + 4: if (RB > 4) sub_swap<C, RB, 3, (RB > 4 ? 4 : 0)>(v, scm); break;
        default: break;
        }
        break;
    case SB_PHASE: {
        // Only the elements whose masked register bits are all 1 change.  Masks of 0, 1 or 2
        // register bits (Z/S/T/P, CZ/CP) get compile-time element lists, so no arithmetic is
        // issued for the untouched elements (predicated-off FP64 work still occupies the
        // narrow FP64 pipe).
        const C p = M[0];
        const bool neg = (p.x == -1 && p.y == 0);
        const int pc = __popc(scm);
        if (pc == 0) {
            sub_phase_mask<C, RB, 0, 0>(v, p, neg);
        } else if (pc == 1) {
            switch (__ffs(scm) - 1) {
            case 0: sub_phase_mask<C, RB, 1, 0>(v, p, neg); break;
            case 1: sub_phase_mask<C, RB, 2, 0>(v, p, neg); break;
            case 2: sub_phase_mask<C, RB, 4, 0>(v, p, neg); break;
            case 3: sub_phase_mask<C, RB, 8, 0>(v, p, neg); break;
            case 4: sub_phase_mask<C, RB, (RB > 4 ? 16 : 1), 0>(v, p, neg); break;
            default: break;
            }
        } else if (pc == 2) {
            switch (scm) {
            case 0x03: sub_phase_mask<C, RB, 0x03, 0>(v, p, neg); break;
            case 0x05: sub_phase_mask<C, RB, 0x05, 0>(v, p, neg); break;
            case 0x06: sub_phase_mask<C, RB, 0x06, 0>(v, p, neg); break;
            case 0x09: sub_phase_mask<C, RB, 0x09, 0>(v, p, neg); break;
            case 0x0a: sub_phase_mask<C, RB, 0x0a, 0>(v, p, neg); break;
            case 0x0c: sub_phase_mask<C, RB, 0x0c, 0>(v, p, neg); break;
            case 0x11: sub_phase_mask<C, RB, (RB > 4 ? 0x11 : 0x03), 0>(v, p, neg); break;
            case 0x12: sub_phase_mask<C, RB, (RB > 4 ? 0x12 : 0x03), 0>(v, p, neg); break;
            case 0x14: sub_phase_mask<C, RB, (RB > 4 ? 0x14 : 0x03), 0>(v, p, neg); break;
            case 0x18: sub_phase_mask<C, RB, (RB > 4 ? 0x18 : 0x03), 0>(v, p, neg); break;
            default: break;
            }
        } else {
#pragma unroll
            for (int e = 0; e < (1 << RB); ++e)
                if ((uint32_t(e) & scm) == scm) v[e] = cmul(p, v[e]);
        }
        break;
    }
    case SB_G1R:
        switch (s.j0) {
        case 0: sub_g1r<C, RB, 0>(v, M, scm); break;
        case 1: sub_g1r<C, RB, 1>(v, M, scm); break;
        case 2: sub_g1r<C, RB, 2>(v, M, scm); break;
        case 3: sub_g1r<C, RB, 3>(v, M, scm); break;
        case 4: if (RB > 4) sub_g1r<C, RB, (RB > 4 ? 4 : 0)>(v, M, scm); break;
        default: break;
        }
        break;
    case SB_DIAG: {
        uint32_t hi = 0;
        for (int j = 0; j < s.ndl; ++j) {
            const uint32_t src = s.dl[j];
            const uint32_t bit = (src & 0x80) ? uint32_t((cta_base >> (src & 0x7f)) & 1)
                                              : ((gbase >> src) & 1u);
            hi |= bit << j;
        }
        const C *__restrict__ T = M + (size_t(hi) << RB);
#pragma unroll
        for (int e = 0; e < (1 << RB); ++e) v[e] = cmul(__ldg(&T[e]), v[e]);
        break;
    }
    default: break;
    }
}

template <typename C, int RB>
__device__ __noinline__ void run_stage(C *sm, const DevStage *__restrict__ stg,
                                          const DevSub *__restrict__ subs, const C *__restrict__ coef,
                                          uint64_t cta_base, uint32_t tid, uint32_t nthr)
{
    constexpr int E = 1 << RB;
    const int nrest = stg->nrest;
    const uint32_t ngroups = 1u << nrest;
    const int s0 = stg->sub_begin, s1 = stg->sub_end;
    for (uint32_t g = tid; g < ngroups; g += nthr) {
        uint32_t base = 0;
        for (int j = 0; j < nrest; ++j) base |= ((g >> j) & 1u) << stg->rest[j];
        // off[e] holds swizzled offsets; the swizzle is linear, so one XOR per element
        const uint32_t pb = swz<(sizeof(C) == 8 ? 1 : 2)>(base);
        C v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = sm[pb ^ stg->off[e]];
        for (int s = s0; s < s1; ++s) apply_sub<C, RB>(v, subs[s], base, cta_base, coef);
#pragma unroll
        for (int e = 0; e < E; ++e) sm[pb ^ stg->off[e]] = v[e];
    }
}

// Ops applied directly to the shared-memory slab, kept out of line so that their register
// needs do not compete with the register stage's amplitude array.
template <typename C>
__device__ __noinline__ void run_smem_op(C *sm, int b, const DevOp &op, const C *__restrict__ coef,
                                         uint64_t base, uint32_t tid, uint32_t nthr)
{
    uint32_t toff = 0;
    if (op.type == OP_DIAG)
        for (int j = 0; j < op.nout; ++j) toff |= uint32_t((base >> op.outpos[j]) & 1) << (op.k + j);
    apply_op<C, uint32_t, (sizeof(C) == 8 ? 1 : 2)>(sm, b, op, coef, toff, tid, nthr);
}

// Named barrier 1 among the NT compute threads (the producer warp never joins it).
__device__ __forceinline__ void compute_sync(uint32_t nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// OR of a predicate over the NT compute threads (also a barrier).
__device__ __forceinline__ bool compute_any(bool v, uint32_t nthreads)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(uint32_t(v)), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// ------------------------------------------------------------------ the pass kernel
//
// Double-buffered pipeline per CTA: while slab i is computed in buffer i&1, the 16-byte
// cp.async copies of slab i+1 (issued by every thread, 16 per thread for a 64 KiB slab) land
// in the other buffer.  cp.async.wait_group completes on its own, so no wait can hang.

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename R, int RB, int NT>
__global__ void __launch_bounds__(NT, 1)
    slab_pass_kernel(typename Cx<R>::T *__restrict__ state, const DevPass *__restrict__ d_pass,
                     const DevOp *__restrict__ ops, const DevStage *__restrict__ stages,
                     const DevSub *__restrict__ subs, const typename Cx<R>::T *__restrict__ coef,
                     uint64_t nslabs)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SlabShared &S = *reinterpret_cast<SlabShared *>(smem_raw);
    const uint32_t tid = threadIdx.x;

    if (tid == 0) S.pass = *d_pass;
    __syncthreads();
    const int b = S.pass.b, lo = S.pass.lo, nhi = S.pass.nhi;
    for (uint32_t j = tid; j < 128; j += NT) {
        const uint32_t x = j & 63, sh = (j < 64) ? 0 : 6;
        uint64_t o = 0;
        for (int m = 0; m < 6; ++m)
            if ((x >> m & 1) && int(m + sh) < nhi) o |= 1ull << S.pass.hipos[m + sh];
        if (j < 64) S.seg_lo[x] = o; else S.seg_hi[x] = o;
    }
    if (S.pass.has_perm) {
        for (uint32_t j = tid; j < 512; j += NT) {
            const uint32_t x = j & 255, sh = (j < 256) ? 0 : 8;
            uint32_t src = 0;
            for (int q = 0; q < 8; ++q) {
                if (!(x >> q & 1) || int(q + sh) >= b) continue;
                int from = 0;
                for (int jj = 0; jj < b; ++jj)
                    if (S.pass.perm[jj] == q + sh) from = jj;
                src |= 1u << from;
            }
            if (j < 256) S.inv_lo[x] = (uint16_t)src; else S.inv_hi[x] = (uint16_t)src;
        }
    }
    __syncthreads();

    C *const buf0 = reinterpret_cast<C *>(smem_raw + ((sizeof(SlabShared) + 127) & ~size_t(127)));
    const uint32_t nsl = 1u << b;
    constexpr int kLog16 = (sizeof(C) == 8) ? 1 : 0;  // log2(amplitudes per 16-byte vector)
    const int vps_log = lo - kLog16;
    const uint32_t nvec = 1u << (b - kLog16);
    const int op_begin = S.pass.op_begin, op_end = S.pass.op_end;
    auto slab_base = [&](uint64_t slab) {
        uint64_t base = slab << lo;
        for (int m = 0; m < nhi; ++m) {
            const uint64_t lowm = (1ull << S.pass.hipos[m]) - 1;
            base = ((base & ~lowm) << 1) | (base & lowm);
        }
        return base;
    };
    // 16-byte chunk of the swizzled slab holding vector v (complex64: amplitudes 2v, 2v+1)
    auto chunk_of = [](uint32_t v) -> uint32_t {
        return sizeof(C) == 8 ? (swz<1>(v << 1) >> 1) : swz<2>(v);
    };
    auto issue_load = [&](uint64_t slab, uint32_t k) {
        const C *g = state + slab_base(slab);
        const uint32_t dst = smem_addr(buf0 + size_t(k) * nsl);
        for (uint32_t v = tid; v < nvec; v += NT) {
            const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
            const uint64_t so = S.seg_lo[seg & 63] | S.seg_hi[(seg >> 6) & 63];
            cp_async16(dst + 16u * chunk_of(v), reinterpret_cast<const uint4 *>(g + so) + w);
        }
        cp_async_commit();
    };

    if (blockIdx.x < nslabs) issue_load(blockIdx.x, 0);
    uint32_t i = 0;
    for (uint64_t slab = blockIdx.x; slab < nslabs; slab += gridDim.x, ++i) {
        const uint32_t k = i & 1u;
        const uint64_t next = slab + gridDim.x;
        if (next < nslabs) {
            issue_load(next, k ^ 1u);  // lands while this slab is computed
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const uint64_t base = slab_base(slab);
        C *sm = buf0 + size_t(k) * nsl;
        C *gbase = state + base;
        // the gate block
        for (int o = op_begin; o < op_end; ++o) {
            const DevOp &op = ops[o];
            if ((base & op.ocmask) == op.ocmask) {
                if (op.type == OP_STAGE) run_stage<C, RB>(sm, stages + op.mat, subs, coef, base, tid, NT);
                else run_smem_op<C>(sm, b, op, coef, base, tid, NT);
            }
            __syncthreads();
        }
        // store
        if (!S.pass.has_perm) {
            for (uint32_t v = tid; v < nvec; v += NT) {
                const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
                const uint64_t so = S.seg_lo[seg & 63] | S.seg_hi[(seg >> 6) & 63];
                st_stream(reinterpret_cast<uint4 *>(gbase + so) + w,
                          reinterpret_cast<const uint4 *>(sm)[chunk_of(v)]);
            }
        } else {
            for (uint32_t d = tid; d < nsl; d += NT) {
                const uint32_t src = S.inv_lo[d & 255] | S.inv_hi[(d >> 8) & 255];
                const uint32_t seg = d >> lo, w = d & ((1u << lo) - 1);
                const uint64_t so = S.seg_lo[seg & 63] | S.seg_hi[(seg >> 6) & 63];
                __stcs(gbase + so + w, sm[swz<(sizeof(C) == 8 ? 1 : 2)>(src)]);
            }
        }
        __syncthreads();  // this buffer is reloaded two slabs later
    }
}

// One CTA per SM with NT threads (= 2^(b - RB) register groups for the default slab sizes).
template <typename R, int RB, int NT>
int launch_pass_t(const LaunchCtx &c, const PassArgs &a, const DevPass &h, char *err, size_t errlen)
{
    using C = typename Cx<R>::T;
    const size_t smem = pass_smem_bytes(c.dt, h.b, h.lo);
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaFuncSetAttribute(slab_pass_kernel<R, RB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
        attr_dev = dev;
    }
    const uint64_t nslabs = 1ull << (c.n - h.b);
    uint64_t grid = uint64_t(num_sms());
    if (grid > nslabs) grid = nslabs;
    slab_pass_kernel<R, RB, NT><<<(unsigned)grid, NT, smem, (cudaStream_t)c.stream>>>(
        reinterpret_cast<C *>(c.amp), a.pass, a.ops, a.stages, a.subs,
        reinterpret_cast<const C *>(a.coef), nslabs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "slab pass launch failed: %s", cudaGetErrorString(e));
        return QS_ECUDA;
    }
    return QS_OK;
}

}  // namespace

size_t pass_smem_bytes(qs_dtype dt, int b, int /*lo*/)
{
    const size_t amp = dt == QS_C64 ? 8 : 16;
    return ((sizeof(SlabShared) + 127) & ~size_t(127)) + 2 * (amp << b);  // two slab buffers
}

int max_slab_bits(qs_dtype dt)
{
    int b = 4;
    while (b < kMaxSlabBits && pass_smem_bytes(dt, b + 1, 0) <= 227 * 1024) ++b;
    return b;
}

int launch_pass(const LaunchCtx &c, const PassArgs &a, const DevPass &h, char *err, size_t errlen)
{
    if (c.dt == QS_C64) {
        if (a.stage_bits == kStageBitsC64 - 1)
            return launch_pass_t<float, kStageBitsC64 - 1, 512>(c, a, h, err, errlen);
        return launch_pass_t<float, kStageBitsC64, 256>(c, a, h, err, errlen);
    }
    if (a.stage_bits == kStageBitsC128 - 1)
        return launch_pass_t<double, kStageBitsC128 - 1, 512>(c, a, h, err, errlen);
    return launch_pass_t<double, kStageBitsC128, 256>(c, a, h, err, errlen);
}

// Device address of the status word on the current device (for kernels in other files).
int *device_status_ptr()
{
    static int *ptr[64] = {nullptr};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_qs_device_status) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptr[dev] = static_cast<int *>(p);
    }
    return ptr[dev];
}

int read_device_status(void *stream, int *status)
{
    int v = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyFromSymbolAsync(&v, g_qs_device_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return QS_ECUDA;
    }
    if (v != 0) {
        const int zero = 0;
        cudaMemcpyToSymbolAsync(g_qs_device_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
    }
    *status = v;
    return QS_OK;
}

}  // namespace qs
