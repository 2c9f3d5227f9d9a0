// slab_common.cuh -- device code shared by the slab-pass kernel (k_slab.cu) and the batched
// persistent kernel (k_batch.cu): PTX helpers and the register-stage sub-ops.
#pragma once

#include <cuda_runtime.h>

#include "dev_common.cuh"
#include "df_arith.cuh"
#include "qs_internal.h"

namespace qs {


namespace {

struct __align__(16) SlabShared {
    uint64_t seg_lo[64];   // deposit of hi-bit index bits 0..5 into physical positions
    uint64_t seg_hi[64];   // deposit of hi-bit index bits 6..11
    uint16_t inv_lo[256];  // store permutation: source local index of destination bits 0..7
    uint16_t inv_hi[256];  //                                    ... of destination bits 8..15
    DevPass pass;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void st_stream(uint4 *p, uint4 v)
{
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// ------------------------------------------------------------------ register sub-ops

// Read-only coefficient load in the register type (double-float coefficients: df_arith.cuh).
__device__ __forceinline__ float2 ldgc(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ double2 ldgc(const double2 *p) { return __ldg(p); }

// s * b + a on both parts of a complex amplitude with a real scalar s.  Complex64 uses one packed
// fma.rn.f32x2 (two FP32 FMAs in one instruction); complex128 two FP64 FMAs.
__device__ __forceinline__ float2 rfma(float s, float2 b, float2 a)
{
    float2 d;
    asm("{\n\t.reg .b64 rs, rb, ra, rd;\n\t"
        "mov.b64 rs, {%2, %2};\n\t"
        "mov.b64 rb, {%3, %4};\n\t"
        "mov.b64 ra, {%5, %6};\n\t"
        "fma.rn.f32x2 rd, rs, rb, ra;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(s), "f"(b.x), "f"(b.y), "f"(a.x), "f"(a.y));
    return d;
}
__device__ __forceinline__ double2 rfma(double s, double2 b, double2 a)
{
    return make_double2(::fma(s, b.x, a.x), ::fma(s, b.y, a.y));
}
// s * b on both parts (packed mul.rn.f32x2 for complex64).
__device__ __forceinline__ float2 rmul(float s, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 rs, rb, rd;\n\t"
        "mov.b64 rs, {%2, %2};\n\t"
        "mov.b64 rb, {%3, %4};\n\t"
        "mul.rn.f32x2 rd, rs, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(s), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ double2 rmul(double s, double2 b) { return make_double2(s * b.x, s * b.y); }
// s * b - a on both parts (scalar FMAs: the negation folds into the FMA's operand).
__device__ __forceinline__ float2 rfms(float s, float2 b, float2 a)
{
    return make_float2(fmaf(s, b.x, -a.x), fmaf(s, b.y, -a.y));
}
__device__ __forceinline__ double2 rfms(double s, double2 b, double2 a)
{
    return make_double2(::fma(s, b.x, -a.x), ::fma(s, b.y, -a.y));
}


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
// neg: p = -1 (sign flip); real: p has no imaginary part (two multiplies per element).
template <typename C, int RB, int MASK, int UNUSED>
__device__ __forceinline__ void sub_phase_mask(C (&v)[1 << RB], C p, bool neg, bool real = false)
{
    if (neg) {
#pragma unroll
        for (int e = 0; e < (1 << RB); ++e)
            if ((e & MASK) == MASK) {
                v[e].x = -v[e].x;
                v[e].y = -v[e].y;
            }
    } else if (real) {
#pragma unroll
        for (int e = 0; e < (1 << RB); ++e)
            if ((e & MASK) == MASK) v[e] = rmul(p.x, v[e]);
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
        v[e] = rfma(m01, b, rmul(m00, a));
        v[e1] = rfma(m11, b, rmul(m10, a));
    }
}

template <typename C, int RB, int J>
__device__ __forceinline__ void sub_g1r(C (&v)[1 << RB], const C *__restrict__ M, uint32_t scm)
{
    if (scm == 0) sub_g1r_impl<C, RB, J, false>(v, M, 0);
    else sub_g1r_impl<C, RB, J, true>(v, M, scm);
}

// Real 2x2 with two entries of magnitude 1, uncontrolled: one FMA per real output.
//   K = 0 (SB_G1N):  [[1, x], [y,  1]]: a' = a + x b, b' = y a + b
//   K = 1 (SB_G1NM): [[1, x], [y, -1]]: a' = a + x b, b' = y a - b
//   K = 2 (SB_G1A):  [[x, 1], [1,  y]]: a' = x a + b, b' = a + y b
//   K = 3 (SB_G1AM): [[x, 1], [-1, y]]: a' = x a + b, b' = y b - a
template <typename C, int RB, int J, int K, typename R>
__device__ __forceinline__ void sub_g1n(C (&v)[1 << RB], R x, R y)
{
    if constexpr (sizeof(C) == 8 && K < 2) {
        // complex64, unit diagonal: b' first, then a' from b' (K = 0: a' = (1 - xy) a + x b';
        // K = 1: a' = (1 + xy) a - x b'), so both results overwrite their inputs and no copy
        // through a temporary is needed; |x|, |y| <= 1, so the coefficients stay within 2
        const R c = K == 0 ? fmaf(-x, y, R(1)) : fmaf(x, y, R(1));
        const R xs = K == 0 ? x : -x;
#pragma unroll
        for (int e = 0; e < (1 << RB); ++e) {
            if (e & (1 << J)) continue;
            const int e1 = e | (1 << J);
            v[e1] = K == 0 ? rfma(y, v[e], v[e1]) : rfms(y, v[e], v[e1]);
            v[e] = rfma(xs, v[e1], rmul(c, v[e]));
        }
        return;
    }
#pragma unroll
    for (int e = 0; e < (1 << RB); ++e) {
        if (e & (1 << J)) continue;
        const int e1 = e | (1 << J);
        const C a = v[e], b = v[e1];
        if (K == 0) {
            v[e] = rfma(x, b, a);
            v[e1] = rfma(y, a, b);
        } else if (K == 1) {
            v[e] = rfma(x, b, a);
            v[e1] = rfms(y, a, b);
        } else if (K == 2) {
            v[e] = rfma(x, a, b);
            v[e1] = rfma(y, b, a);
        } else {
            v[e] = rfma(x, a, b);
            v[e1] = rfms(y, b, a);
        }
    }
}

// x, y: the two free entries (real), read ahead with the sub-op's descriptor.
template <typename C, int RB, int K, typename R>
__device__ __forceinline__ void sub_g1n_j(C (&v)[1 << RB], R x, R y, uint32_t j0)
{
    switch (j0) {
    case 0: sub_g1n<C, RB, 0, K>(v, x, y); break;
    case 1: sub_g1n<C, RB, 1, K>(v, x, y); break;
    case 2: sub_g1n<C, RB, 2, K>(v, x, y); break;
    case 3: sub_g1n<C, RB, 3, K>(v, x, y); break;
    case 4: if (RB > 4) sub_g1n<C, RB, (RB > 4 ? 4 : 0), K>(v, x, y); break;
    default: break;
    }
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

// Index of the lowest set bit of i > 0 (folds to a constant in unrolled loops).
__device__ __forceinline__ int lowest_bit(int i) { return __ffs(i) - 1; }

// The first 24 bytes of a DevSub, fetched as one 16-byte and one 8-byte load.
struct SubHead {
    uint32_t w0;   // type | j0 << 8 | j1 << 16 | ndl << 24
    uint32_t scm, lcm, mat;
    uint64_t ocm;
};

__device__ __forceinline__ SubHead load_sub_head(const DevSub *__restrict__ p)
{
    const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
    const unsigned long long o = __ldg(reinterpret_cast<const unsigned long long *>(p) + 2);
    return SubHead{a.x, a.y, a.z, a.w, o};
}

// c0, c1: coef[h.mat] and coef[h.mat + 1], read together with the descriptor one sub-op ahead
// (the pool carries two spare entries past its end).
template <typename C, int RB>
__device__ __forceinline__ void apply_sub(C (&v)[1 << RB], const SubHead &h, const DevSub *__restrict__ sp,
                                          uint32_t gbase, uint64_t cta_base, const C *__restrict__ coef,
                                          C c0, C c1)
{
    if ((gbase & h.lcm) != h.lcm || (cta_base & h.ocm) != h.ocm) return;
    const C *__restrict__ M = coef + h.mat;
    const uint32_t scm = h.scm;
    const uint32_t type = h.w0 & 0xffu, j0 = (h.w0 >> 8) & 0xffu, j1 = (h.w0 >> 16) & 0xffu, ndl = h.w0 >> 24;
    switch (type) {
    case SB_G1:
        switch (j0) {
        case 0: sub_g1<C, RB, 0>(v, M, scm); break;
        case 1: sub_g1<C, RB, 1>(v, M, scm); break;
        case 2: sub_g1<C, RB, 2>(v, M, scm); break;
        case 3: sub_g1<C, RB, 3>(v, M, scm); break;
        case 4: if (RB > 4) sub_g1<C, RB, (RB > 4 ? 4 : 0)>(v, M, scm); break;
        default: break;
        }
        break;
    case SB_G2:
        switch (j0 * 8 + j1) {
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
        switch (j0) {
        case 0: sub_x<C, RB, 0>(v, scm); break;
        case 1: sub_x<C, RB, 1>(v, scm); break;
        case 2: sub_x<C, RB, 2>(v, scm); break;
        case 3: sub_x<C, RB, 3>(v, scm); break;
        case 4: if (RB > 4) sub_x<C, RB, (RB > 4 ? 4 : 0)>(v, scm); break;
        default: break;
        }
        break;
    case SB_SWAP:
        switch (j0 * 8 + j1) {
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
        const C p = c0;
        const bool neg = (p.x == -1 && p.y == 0);
        const int pc = __popc(scm);
        if (pc == 0) {
            sub_phase_mask<C, RB, 0, 0>(v, p, neg, p.y == 0);  // a scalar; real for factored stages
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
        switch (j0) {
        case 0: sub_g1r<C, RB, 0>(v, M, scm); break;
        case 1: sub_g1r<C, RB, 1>(v, M, scm); break;
        case 2: sub_g1r<C, RB, 2>(v, M, scm); break;
        case 3: sub_g1r<C, RB, 3>(v, M, scm); break;
        case 4: if (RB > 4) sub_g1r<C, RB, (RB > 4 ? 4 : 0)>(v, M, scm); break;
        default: break;
        }
        break;
    case SB_G1N: sub_g1n_j<C, RB, 0>(v, c0.x, c1.x, j0); break;
    case SB_G1NM: sub_g1n_j<C, RB, 1>(v, c0.x, c1.x, j0); break;
    case SB_G1A: sub_g1n_j<C, RB, 2>(v, c0.x, c1.x, j0); break;
    case SB_G1AM: sub_g1n_j<C, RB, 3>(v, c0.x, c1.x, j0); break;
    case SB_DIAG: {
        uint32_t hi = 0;
        for (int j = 0; j < int(ndl); ++j) {
            const uint32_t src = sp->dl[j];
            const uint32_t bit = (src & 0x80) ? uint32_t((cta_base >> (src & 0x7f)) & 1)
                                              : ((gbase >> src) & 1u);
            hi |= bit << j;
        }
        const C *__restrict__ T = M + (size_t(hi) << RB);
#pragma unroll
        for (int e = 0; e < (1 << RB); ++e) v[e] = cmul(ldgc(&T[e]), v[e]);
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
    constexpr int SW = sizeof(C) == 8 ? 1 : 2;
    // bytes 0..7: r, nrest, sbits[0..5] (register bits in ascending slab-local order)
    const uint2 hd = __ldg(reinterpret_cast<const uint2 *>(stg));
    const uint2 rng = __ldg(reinterpret_cast<const uint2 *>(&stg->sub_begin));
    const int nrest = (hd.x >> 8) & 0xff;
    uint32_t sb[RB], bo[RB];
#pragma unroll
    for (int j = 0; j < RB; ++j) {
        sb[j] = j < 2 ? (hd.x >> (16 + 8 * j)) & 0xff : (hd.y >> (8 * (j - 2))) & 0xff;
        // the swizzle is linear over GF(2): the offset of register index e is the XOR of the
        // swizzled single-bit offsets of its set bits
        bo[j] = swz<SW>(1u << sb[j]);
    }
    const uint32_t ngroups = 1u << nrest;
    const int s0 = int(rng.x), s1 = int(rng.y);
    for (uint32_t g = tid; g < ngroups; g += nthr) {
        // slab index of the group: g's bits with zeros inserted at the register bits
        uint32_t base = g;
#pragma unroll
        for (int j = 0; j < RB; ++j) {
            const uint32_t low = base & ((1u << sb[j]) - 1u);
            base = ((base ^ low) << 1) | low;
        }
        const uint32_t pb = swz<SW>(base);
        C v[E];
        // element addresses: the address of e is that of e without its lowest set bit, XORed
        // with that bit's offset -- a tree of depth popcount(e), so the loads issue back to back
        {
            uint32_t a[E];
            a[0] = pb;
#pragma unroll
            for (int e = 1; e < E; ++e) a[e] = a[e & (e - 1)] ^ bo[lowest_bit(e)];
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = sm[a[e]];
        }
        if (s0 < s1) {
            SubHead nxt = load_sub_head(subs + s0);
            C n0 = ldgc(coef + nxt.mat), n1 = ldgc(coef + nxt.mat + 1);
            for (int s = s0; s < s1; ++s) {
                const SubHead cur = nxt;
                const C c0 = n0, c1 = n1;
                if (s + 1 < s1) {
                    nxt = load_sub_head(subs + s + 1);
                    n0 = ldgc(coef + nxt.mat);
                    n1 = ldgc(coef + nxt.mat + 1);
                }
                apply_sub<C, RB>(v, cur, subs + s, base, cta_base, coef, c0, c1);
            }
        }
        {
            uint32_t a[E];
            a[0] = pb;
#pragma unroll
            for (int e = 1; e < E; ++e) a[e] = a[e & (e - 1)] ^ bo[lowest_bit(e)];
#pragma unroll
            for (int e = 0; e < E; ++e) sm[a[e]] = v[e];
        }
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

// 16-byte asynchronous global -> shared copies (L2 only, no L1 allocation).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

}  // namespace
}  // namespace qs
