// op_global.cuh -- the one-op kernel's ops on the whole state in global memory (k_apply.cu).
//
// The same arithmetic as the shared-memory ops of dev_common.cuh, but each thread takes U
// disjoint groups at a time and issues all their loads before the first store, so several
// global loads per thread are in flight.  With one group at a time the gate-by-gate kernel ran
// at 30-50 % of HBM; with four, 1-qubit dense gates reach about 84 % (complex64, 28-33 qubits).
// The slab kernel keeps the one-group form: its operands are in shared memory.
#pragma once

#include "dev_common.cuh"

namespace qs {
namespace {

template <typename C, int K, typename I, int SW>
__device__ void gop_dense(C *mem, int nbits, const DevOp &op, const C *__restrict__ coef,
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
        // U disjoint groups per thread: all their loads are issued before any store
        constexpr int U = K == 1 ? 4 : 2;
        for (I g0 = tid; g0 < ngroups; g0 += I(U) * nthr) {
            I i0[U];
            C v[U][D];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const I g = g0 + I(u) * nthr;
                i0[u] = insert_zeros<I>(g < ngroups ? g : g0, op.ins, op.nins) | cm;
#pragma unroll
                for (int l = 0; l < D; ++l) v[u][l] = mem[swz<SW>(i0[u] | off[l])];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (g0 + I(u) * nthr >= ngroups) break;  // past the end: loaded, never stored
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    C acc = czero<C>();
#pragma unroll
                    for (int l = 0; l < D; ++l) acc = cmac(m[r * D + l], v[u][l], acc);
                    mem[swz<SW>(i0[u] | off[r])] = acc;
                }
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
__device__ void gop_diag(C *mem, int nbits, const DevOp &op, const C *__restrict__ table,
                        I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask;
    const int k = op.k;
    constexpr int U = 4;  // disjoint amplitudes per thread, loads first
    for (I g0 = tid; g0 < ngroups; g0 += I(U) * nthr) {
        I i[U];
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const I g = g0 + I(u) * nthr;
            i[u] = insert_zeros<I>(g < ngroups ? g : g0, op.ins, op.nins) | cm;
            v[u] = mem[swz<SW>(i[u])];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (g0 + I(u) * nthr >= ngroups) break;
            uint32_t idx = 0;
            for (int j = 0; j < k; ++j) idx |= uint32_t((i[u] >> op.t[j]) & 1) << j;
            mem[swz<SW>(i[u])] = cmul(__ldg(&table[idx]), v[u]);
        }
    }
}

template <typename C, typename I, int SW>
__device__ void gop_permx(C *mem, int nbits, const DevOp &op, I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask, bit = I(1) << op.t[0];
    constexpr int U = 4;
    for (I g0 = tid; g0 < ngroups; g0 += I(U) * nthr) {
        I i0[U];
        C a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const I g = g0 + I(u) * nthr;
            i0[u] = insert_zeros<I>(g < ngroups ? g : g0, op.ins, op.nins) | cm;
            a[u] = mem[swz<SW>(i0[u])];
            b[u] = mem[swz<SW>(i0[u] | bit)];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (g0 + I(u) * nthr >= ngroups) break;
            mem[swz<SW>(i0[u])] = b[u];
            mem[swz<SW>(i0[u] | bit)] = a[u];
        }
    }
}

template <typename C, typename I, int SW>
__device__ void gop_swap(C *mem, int nbits, const DevOp &op, I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask, b0 = I(1) << op.t[0], b1 = I(1) << op.t[1];
    constexpr int U = 4;
    for (I g0 = tid; g0 < ngroups; g0 += I(U) * nthr) {
        I i0[U];
        C a[U], b[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const I g = g0 + I(u) * nthr;
            i0[u] = insert_zeros<I>(g < ngroups ? g : g0, op.ins, op.nins) | cm;
            a[u] = mem[swz<SW>(i0[u] | b0)];
            b[u] = mem[swz<SW>(i0[u] | b1)];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (g0 + I(u) * nthr >= ngroups) break;
            mem[swz<SW>(i0[u] | b0)] = b[u];
            mem[swz<SW>(i0[u] | b1)] = a[u];
        }
    }
}

template <typename C, typename I, int SW>
__device__ void gop_phase(C *mem, int nbits, const DevOp &op, const C *__restrict__ coef,
                         I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask;
    const C ph = coef[op.mat];
    constexpr int U = 4;
    for (I g0 = tid; g0 < ngroups; g0 += I(U) * nthr) {
        I i[U];
        C v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const I g = g0 + I(u) * nthr;
            i[u] = insert_zeros<I>(g < ngroups ? g : g0, op.ins, op.nins) | cm;
            v[u] = mem[swz<SW>(i[u])];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (g0 + I(u) * nthr >= ngroups) break;
            mem[swz<SW>(i[u])] = cmul(ph, v[u]);
        }
    }
}

// Dispatch one op.  For DIAG, `table_off` selects the slice fixed by the outer bits.
template <typename C, typename I, int SW>
__device__ __forceinline__ void apply_op_global(C *mem, int nbits, const DevOp &op,
                                         const C *__restrict__ coef, uint32_t table_off, I tid,
                                         I nthr)
{
    switch (op.type) {
    case OP_DENSE:
        switch (op.k) {
        case 1: gop_dense<C, 1, I, SW>(mem, nbits, op, coef, tid, nthr); break;
        case 2: gop_dense<C, 2, I, SW>(mem, nbits, op, coef, tid, nthr); break;
        case 3: gop_dense<C, 3, I, SW>(mem, nbits, op, coef, tid, nthr); break;
        case 4: gop_dense<C, 4, I, SW>(mem, nbits, op, coef, tid, nthr); break;
        case 5: gop_dense<C, 5, I, SW>(mem, nbits, op, coef, tid, nthr); break;
        default: break;
        }
        break;
    case OP_DIAG: gop_diag<C, I, SW>(mem, nbits, op, coef + op.mat + table_off, tid, nthr); break;
    case OP_PERMX: gop_permx<C, I, SW>(mem, nbits, op, tid, nthr); break;
    case OP_SWAP: gop_swap<C, I, SW>(mem, nbits, op, tid, nthr); break;
    case OP_PHASE: gop_phase<C, I, SW>(mem, nbits, op, coef, tid, nthr); break;
    default: break;
    }
}

}  // namespace
}  // namespace qs
