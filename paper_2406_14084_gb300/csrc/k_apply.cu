// k_apply.cu -- gate-application kernels for sm_103a.
//
//  * slab_pass_kernel: the in-cache gate-block kernel (arXiv 2406.14084, Alg. 3 and Sec. V-A).
//    Each CTA owns one slab of 2^b amplitudes at a time (persistent loop over slabs): it loads
//    the slab into shared memory with 16-byte vector loads, applies every op of the gate block
//    there (several amplitude groups per thread, the per-gate unrolling of Sec. V-A), and
//    writes the slab back with 16-byte streaming stores.  A slab is the low `lo` physical bits
//    (one contiguous segment of >= 128 bytes) plus b-lo arbitrary physical bit positions, so a
//    block may use high qubits without a separate swap pass; a store permutation relabels bits
//    inside the slab, which is how remaps (Sec. V-B, Alg. 4) are carried out in place.
//  * unblocked_kernel: one op over the whole state in global memory (gate-by-gate scheme).
//
// Arithmetic: complex multiply-accumulate in the state precision (float or double) with fused
// multiply-adds; no transcendental functions are evaluated on the device.
#include <cuda_runtime.h>

#include <cstdio>

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

// ------------------------------------------------------------------ ops on an addressable array
// `mem` is either the shared-memory slab (I = uint32_t, nbits = b) or the whole state in global
// memory (I = uint64_t, nbits = n).  Work is split over threads [tid, tid + nthr, ...).

template <typename C, int K, typename I>
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
            for (int l = 0; l < D; ++l) v[l] = mem[i0 | off[l]];
#pragma unroll
            for (int r = 0; r < D; ++r) {
                C acc = czero<C>();
#pragma unroll
                for (int l = 0; l < D; ++l) acc = cmac(m[r * D + l], v[l], acc);
                mem[i0 | off[r]] = acc;
            }
        }
    } else {
        for (I g = tid; g < ngroups; g += nthr) {
            const I i0 = insert_zeros<I>(g, op.ins, op.nins) | cm;
            C v[D];
#pragma unroll
            for (int l = 0; l < D; ++l) v[l] = mem[i0 | off[l]];
#pragma unroll 1
            for (int r = 0; r < D; ++r) {
                C acc = czero<C>();
#pragma unroll
                for (int l = 0; l < D; ++l) acc = cmac(__ldg(&M[r * D + l]), v[l], acc);
                mem[i0 | off[r]] = acc;
            }
        }
    }
}

template <typename C, typename I>
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
        mem[i] = cmul(__ldg(&table[idx]), mem[i]);
    }
}

template <typename C, typename I>
__device__ void op_permx(C *mem, int nbits, const DevOp &op, I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask, bit = I(1) << op.t[0];
    for (I g = tid; g < ngroups; g += nthr) {
        const I i0 = insert_zeros<I>(g, op.ins, op.nins) | cm;
        const C a = mem[i0], b = mem[i0 | bit];
        mem[i0] = b;
        mem[i0 | bit] = a;
    }
}

template <typename C, typename I>
__device__ void op_swap(C *mem, int nbits, const DevOp &op, I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask, b0 = I(1) << op.t[0], b1 = I(1) << op.t[1];
    for (I g = tid; g < ngroups; g += nthr) {
        const I i0 = insert_zeros<I>(g, op.ins, op.nins) | cm;
        const C a = mem[i0 | b0], b = mem[i0 | b1];
        mem[i0 | b0] = b;
        mem[i0 | b1] = a;
    }
}

template <typename C, typename I>
__device__ void op_phase(C *mem, int nbits, const DevOp &op, const C *__restrict__ coef,
                         I tid, I nthr)
{
    const I ngroups = I(1) << (nbits - op.nins);
    const I cm = (I)op.cmask;
    const C ph = coef[op.mat];
    for (I g = tid; g < ngroups; g += nthr) {
        const I i = insert_zeros<I>(g, op.ins, op.nins) | cm;
        mem[i] = cmul(ph, mem[i]);
    }
}

// Dispatch one op.  For DIAG, `table_off` selects the slice fixed by the outer bits.
template <typename C, typename I>
__device__ __forceinline__ void apply_op(C *mem, int nbits, const DevOp &op,
                                         const C *__restrict__ coef, uint32_t table_off, I tid,
                                         I nthr)
{
    switch (op.type) {
    case OP_DENSE:
        switch (op.k) {
        case 1: op_dense<C, 1, I>(mem, nbits, op, coef, tid, nthr); break;
        case 2: op_dense<C, 2, I>(mem, nbits, op, coef, tid, nthr); break;
        case 3: op_dense<C, 3, I>(mem, nbits, op, coef, tid, nthr); break;
        case 4: op_dense<C, 4, I>(mem, nbits, op, coef, tid, nthr); break;
        case 5: op_dense<C, 5, I>(mem, nbits, op, coef, tid, nthr); break;
        default: break;
        }
        break;
    case OP_DIAG: op_diag<C, I>(mem, nbits, op, coef + op.mat + table_off, tid, nthr); break;
    case OP_PERMX: op_permx<C, I>(mem, nbits, op, tid, nthr); break;
    case OP_SWAP: op_swap<C, I>(mem, nbits, op, tid, nthr); break;
    case OP_PHASE: op_phase<C, I>(mem, nbits, op, coef, tid, nthr); break;
    default: break;
    }
}

// ------------------------------------------------------------------ slab pass

struct __align__(16) SlabShared {
    uint64_t seg_lo[64];   // deposit of hi-bit index bits 0..5 into physical positions
    uint64_t seg_hi[64];   // deposit of hi-bit index bits 6..11
    uint16_t inv_lo[256];  // store permutation: source local index of destination bits 0..7
    uint16_t inv_hi[256];  //                                    ... of destination bits 8..15
    DevPass pass;
};

__device__ __forceinline__ uint4 ld_stream(const uint4 *p)
{
    uint4 v;
    asm volatile("ld.global.cs.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void st_stream(uint4 *p, uint4 v)
{
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

template <typename R>
__global__ void __launch_bounds__(256, 2) slab_pass_kernel(typename Cx<R>::T *__restrict__ state,
                                                        const DevPass *__restrict__ d_pass,
                                                        const DevOp *__restrict__ ops,
                                                        const typename Cx<R>::T *__restrict__ coef,
                                                        uint64_t nslabs)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SlabShared &S = *reinterpret_cast<SlabShared *>(smem_raw);
    C *sm = reinterpret_cast<C *>(smem_raw + sizeof(SlabShared));
    const uint32_t tid = threadIdx.x, nthr = blockDim.x;

    if (tid == 0) S.pass = *d_pass;
    __syncthreads();
    const int b = S.pass.b, lo = S.pass.lo, nhi = S.pass.nhi;
    // Deposit tables for segment offsets (hi-bit index -> physical offset).
    for (uint32_t j = tid; j < 128; j += nthr) {
        const uint32_t x = j & 63, sh = (j < 64) ? 0 : 6;
        uint64_t o = 0;
        for (int m = 0; m < 6; ++m)
            if ((x >> m & 1) && int(m + sh) < nhi) o |= 1ull << S.pass.hipos[m + sh];
        if (j < 64) S.seg_lo[x] = o; else S.seg_hi[x] = o;
    }
    if (S.pass.has_perm) {
        // destination bit q comes from source bit invp[q]
        for (uint32_t j = tid; j < 512; j += nthr) {
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

    // bit positions occupied by the slab, ascending: 0..lo-1 then hipos
    constexpr int kLog16 = (sizeof(C) == 8) ? 1 : 0;  // log2(amplitudes per 16-byte vector)
    const int vps_log = lo - kLog16;                  // log2(vectors per segment)
    const uint32_t nvec = 1u << (b - kLog16);
    const uint32_t nsl = 1u << b;
    const int op_begin = S.pass.op_begin, op_end = S.pass.op_end;

    for (uint64_t slab = blockIdx.x; slab < nslabs; slab += gridDim.x) {
        uint64_t base = slab << lo;
        for (int m = 0; m < nhi; ++m) {
            const uint64_t lowm = (1ull << S.pass.hipos[m]) - 1;
            base = ((base & ~lowm) << 1) | (base & lowm);
        }
        C *gbase = state + base;
        for (uint32_t v = tid; v < nvec; v += nthr) {
            const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
            const uint64_t so = S.seg_lo[seg & 63] | S.seg_hi[(seg >> 6) & 63];
            reinterpret_cast<uint4 *>(sm)[v] =
                ld_stream(reinterpret_cast<const uint4 *>(gbase + so) + w);
        }
        __syncthreads();
        for (int o = op_begin; o < op_end; ++o) {
            const DevOp &op = ops[o];
            if ((base & op.ocmask) == op.ocmask) {
                uint32_t toff = 0;
                if (op.type == OP_DIAG)
                    for (int j = 0; j < op.nout; ++j)
                        toff |= uint32_t((base >> op.outpos[j]) & 1) << (op.k + j);
                apply_op<C, uint32_t>(sm, b, op, coef, toff, tid, nthr);
            }
            __syncthreads();
        }
        if (!S.pass.has_perm) {
            for (uint32_t v = tid; v < nvec; v += nthr) {
                const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
                const uint64_t so = S.seg_lo[seg & 63] | S.seg_hi[(seg >> 6) & 63];
                st_stream(reinterpret_cast<uint4 *>(gbase + so) + w,
                          reinterpret_cast<const uint4 *>(sm)[v]);
            }
        } else {
            for (uint32_t d = tid; d < nsl; d += nthr) {
                const uint32_t src = S.inv_lo[d & 255] | S.inv_hi[(d >> 8) & 255];
                const uint32_t seg = d >> lo, w = d & ((1u << lo) - 1);
                const uint64_t so = S.seg_lo[seg & 63] | S.seg_hi[(seg >> 6) & 63];
                __stcs(gbase + so + w, sm[src]);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ unblocked

template <typename R>
__global__ void __launch_bounds__(256) unblocked_kernel(typename Cx<R>::T *__restrict__ state, int n,
                                                        const DevOp *__restrict__ d_op,
                                                        const typename Cx<R>::T *__restrict__ coef)
{
    using C = typename Cx<R>::T;
    __shared__ DevOp op;
    if (threadIdx.x == 0) op = *d_op;
    __syncthreads();
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nthr = uint64_t(gridDim.x) * blockDim.x;
    apply_op<C, uint64_t>(state, n, op, coef, 0u, tid, nthr);
}

int g_num_sms = 0;

int num_sms()
{
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

template <typename R>
int launch_pass_t(const LaunchCtx &c, const DevPass *d_pass, const DevPass &h, const DevOp *d_ops,
                  const void *d_coef, int threads, int ctas_per_sm, char *err, size_t errlen)
{
    using C = typename Cx<R>::T;
    const size_t smem = pass_smem_bytes(c.dt, h.b, h.lo);
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(slab_pass_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
        attr_set = true;
    }
    const uint64_t nslabs = 1ull << (c.n - h.b);
    uint64_t grid = uint64_t(num_sms()) * uint64_t(ctas_per_sm > 0 ? ctas_per_sm : 1);
    if (grid > nslabs) grid = nslabs;
    slab_pass_kernel<R><<<(unsigned)grid, threads, smem, (cudaStream_t)c.stream>>>(
        reinterpret_cast<C *>(c.amp), d_pass, d_ops, reinterpret_cast<const C *>(d_coef), nslabs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "slab pass launch failed: %s", cudaGetErrorString(e));
        return QS_ECUDA;
    }
    return QS_OK;
}

template <typename R>
int launch_unblocked_t(const LaunchCtx &c, const DevOp *d_op, const DevOp &h, const void *d_coef,
                       char *err, size_t errlen)
{
    using C = typename Cx<R>::T;
    const uint64_t groups = 1ull << (c.n - h.nins);
    const int threads = 256;
    uint64_t blocks = (groups + threads - 1) / threads;
    const uint64_t cap = uint64_t(num_sms()) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    unblocked_kernel<R><<<(unsigned)blocks, threads, 0, (cudaStream_t)c.stream>>>(
        reinterpret_cast<C *>(c.amp), c.n, d_op, reinterpret_cast<const C *>(d_coef));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "unblocked launch failed: %s", cudaGetErrorString(e));
        return QS_ECUDA;
    }
    return QS_OK;
}

}  // namespace

size_t pass_smem_bytes(qs_dtype dt, int b, int /*lo*/)
{
    const size_t amp = dt == QS_C64 ? 8 : 16;
    return sizeof(SlabShared) + (amp << b);
}

int max_slab_bits(qs_dtype dt)
{
    // largest b with the slab plus bookkeeping inside 227 KiB of shared memory
    int b = 4;
    while (b < kMaxSlabBits && pass_smem_bytes(dt, b + 1, 0) <= 227 * 1024) ++b;
    return b;
}

int launch_pass(const LaunchCtx &c, const DevPass *d_pass, const DevPass &h_pass,
                const DevOp *d_ops, const void *d_coef, int threads, int ctas_per_sm, char *err,
                size_t errlen)
{
    if (c.dt == QS_C64)
        return launch_pass_t<float>(c, d_pass, h_pass, d_ops, d_coef, threads, ctas_per_sm, err,
                                    errlen);
    return launch_pass_t<double>(c, d_pass, h_pass, d_ops, d_coef, threads, ctas_per_sm, err,
                                 errlen);
}

int launch_unblocked(const LaunchCtx &c, const DevOp *d_op, const DevOp &h_op, const void *d_coef,
                     char *err, size_t errlen)
{
    if (c.dt == QS_C64) return launch_unblocked_t<float>(c, d_op, h_op, d_coef, err, errlen);
    return launch_unblocked_t<double>(c, d_op, h_op, d_coef, err, errlen);
}

}  // namespace qs
