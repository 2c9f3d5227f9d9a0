// dev_common.cuh -- device helpers shared by the gate kernels: complex arithmetic in the
// state precision and the per-op routines that act on an addressable amplitude array (the
// shared-memory slab, or the whole state in global memory).  Each op enumerates its amplitude
// groups by inserting the target bits (0) and local control bits (1) into a group counter, the
// index construction of Eq. 2-3 of arXiv 2406.14084.
#pragma once

#include <cuda_runtime.h>

#include "qs_internal.h"

namespace qs {
namespace {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename C>
__device__ __forceinline__ C cmac(C m, C v, C acc)
{
    acc.x = fma(m.x, v.x, acc.x);
    acc.x = fma(-m.y, v.y, acc.x);
    acc.y = fma(m.x, v.y, acc.y);
    acc.y = fma(m.y, v.x, acc.y);
    return acc;
}

template <typename C>
__device__ __forceinline__ C cmul(C m, C v)
{
    C r;
    r.x = fma(m.x, v.x, -m.y * v.y);
    r.y = fma(m.x, v.y, m.y * v.x);
    return r;
}

template <typename C>
__device__ __forceinline__ C czero()
{
    C z;
    z.x = 0;
    z.y = 0;
    return z;
}

// Insert a zero bit at each of the ascending positions pos[0..n).
template <typename I>
__device__ __forceinline__ I insert_zeros(I g, const uint8_t *pos, int n)
{
    for (int j = 0; j < n; ++j) {
        const I lowm = (I(1) << pos[j]) - 1;
        g = ((g & ~lowm) << 1) | (g & lowm);
    }
    return g;
}

// XOR swizzle of slab-local amplitude indices in shared memory (SW = 0: none, used for the
// state in global memory).  SW = 1 (complex64): bits 1-3 of the index (the 8-byte slot within a
// 128-byte row, pairs kept together for 16-byte copies) are XORed with bits 5-7 and 9-11;
// SW = 2 (complex128): bits 0-2 are XORed with bits 3-5, 6-8 and 9-11.  The map is linear over
// GF(2), so swz(a ^ b) = swz(a) ^ swz(b) for the disjoint bit sets of a group base and offset.
template <int SW, typename I>
__device__ __forceinline__ I swz(I i)
{
    if (SW == 1) return i ^ (((i >> 4) ^ (i >> 8)) & I(0xE));
    if (SW == 2) return i ^ (((i >> 3) ^ (i >> 6) ^ (i >> 9)) & I(7));
    return i;
}

// ------------------------------------------------------------------ ops on an addressable array
// `mem` is either the shared-memory slab (I = uint32_t, nbits = b) or the whole state in global
// memory (I = uint64_t, nbits = n).  Work is split over threads [tid, tid + nthr, ...).

template <typename C, int K, typename I, int SW>
__device__ void op_dense(C *mem, int nbits, const DevOp &op, const C *__restrict__ coef,
                         I tid, I nthr)
{
    constexpr int D = 1 << K;
    const I ngroups = I(1) << (nbits - op.nins);
    I off[D];
#pragma unroll
    for (int l = 0; l < D; ++l) {
        I o = 0;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (l >> j & 1) o |= I(1) << op.t[j];
        off[l] = o;
    }
    const C *__restrict__ M = coef + op.mat;
    const I cm = (I)op.cmask;
    if (K <= 2) {
        C m[D * D];
#pragma unroll
        for (int e = 0; e < D * D; ++e) m[e] = M[e];
        for (I g = tid; g < ngroups; g += nthr) {
            const I i0 = insert_zeros<I>(g, op.ins, op.nins) | cm;
            C v[D];
#pragma unroll
            for (int l = 0; l < D; ++l) v[l] = mem[swz<SW>(i0 | off[l])];
#pragma unroll
            for (int r = 0; r < D; ++r) {
                C acc = czero<C>();
#pragma unroll
                for (int l = 0; l < D; ++l) acc = cmac(m[r * D + l], v[l], acc);
                mem[swz<SW>(i0 | off[r])] = acc;
            }
        }
    } else {
        for (I g = tid; g < ngroups; g += nthr) {
            const I i0 = insert_zeros<I>(g, op.ins, op.nins) | cm;
            C v[D];
#pragma unroll
            for (int l = 0; l < D; ++l) v[l] = mem[swz<SW>(i0 | off[l])];
#pragma unroll 1
            for (int r = 0; r < D; ++r) {
                C acc = czero<C>();
#pragma unroll
                for (int l = 0; l < D; ++l) acc = cmac(__ldg(&M[r * D + l]), v[l], acc);
                mem[swz<SW>(i0 | off[r])] = acc;
            }
        }
    }
}

template <typename C, typename I, int SW>
__device__ void op_diag(C *mem, int nbits, const DevOp &op, const C *__restrict__ table,
                        I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask;
    const int k = op.k;
    for (I g = tid; g < ngroups; g += nthr) {
        const I i = insert_zeros<I>(g, op.ins, op.nins) | cm;
        uint32_t idx = 0;
        for (int j = 0; j < k; ++j) idx |= uint32_t((i >> op.t[j]) & 1) << j;
        mem[swz<SW>(i)] = cmul(__ldg(&table[idx]), mem[swz<SW>(i)]);
    }
}

template <typename C, typename I, int SW>
__device__ void op_permx(C *mem, int nbits, const DevOp &op, I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask, bit = I(1) << op.t[0];
    for (I g = tid; g < ngroups; g += nthr) {
        const I i0 = insert_zeros<I>(g, op.ins, op.nins) | cm;
        const C a = mem[swz<SW>(i0)], b = mem[swz<SW>(i0 | bit)];
        mem[swz<SW>(i0)] = b;
        mem[swz<SW>(i0 | bit)] = a;
    }
}

template <typename C, typename I, int SW>
__device__ void op_swap(C *mem, int nbits, const DevOp &op, I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask, b0 = I(1) << op.t[0], b1 = I(1) << op.t[1];
    for (I g = tid; g < ngroups; g += nthr) {
        const I i0 = insert_zeros<I>(g, op.ins, op.nins) | cm;
        const C a = mem[swz<SW>(i0 | b0)], b = mem[swz<SW>(i0 | b1)];
        mem[swz<SW>(i0 | b0)] = b;
        mem[swz<SW>(i0 | b1)] = a;
    }
}

template <typename C, typename I, int SW>
__device__ void op_phase(C *mem, int nbits, const DevOp &op, const C *__restrict__ coef,
                         I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask;
    const C ph = coef[op.mat];
    for (I g = tid; g < ngroups; g += nthr) {
        const I i = insert_zeros<I>(g, op.ins, op.nins) | cm;
        mem[swz<SW>(i)] = cmul(ph, mem[swz<SW>(i)]);
    }
}

// Dispatch one op.  For DIAG, `table_off` selects the slice fixed by the outer bits.
template <typename C, typename I, int SW>
__device__ __forceinline__ void apply_op(C *mem, int nbits, const DevOp &op,
                                         const C *__restrict__ coef, uint32_t table_off, I tid,
                                         I nthr)
{
    switch (op.type) {
    case OP_DENSE:
        switch (op.k) {
        case 1: op_dense<C, 1, I, SW>(mem, nbits, op, coef, tid, nthr); break;
        case 2: op_dense<C, 2, I, SW>(mem, nbits, op, coef, tid, nthr); break;
        case 3: op_dense<C, 3, I, SW>(mem, nbits, op, coef, tid, nthr); break;
        case 4: op_dense<C, 4, I, SW>(mem, nbits, op, coef, tid, nthr); break;
        case 5: op_dense<C, 5, I, SW>(mem, nbits, op, coef, tid, nthr); break;
        default: break;
        }
        break;
    case OP_DIAG: op_diag<C, I, SW>(mem, nbits, op, coef + op.mat + table_off, tid, nthr); break;
    case OP_PERMX: op_permx<C, I, SW>(mem, nbits, op, tid, nthr); break;
    case OP_SWAP: op_swap<C, I, SW>(mem, nbits, op, tid, nthr); break;
    case OP_PHASE: op_phase<C, I, SW>(mem, nbits, op, coef, tid, nthr); break;
    default: break;
    }
}

}  // namespace
}  // namespace qs
