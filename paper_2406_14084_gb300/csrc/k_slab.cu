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

#include "slab_common.cuh"

namespace qs {

__device__ int g_qs_device_status;

namespace {

// 16-byte chunks of the largest slab (2^13 complex64 or 2^12 complex128 amplitudes)
constexpr uint32_t kMaxVec = 4096;

// ------------------------------------------------------------------ the pass kernel
//
// Double-buffered pipeline per CTA: while slab i is computed in buffer i&1, the 16-byte
// cp.async copies of slab i+1 (issued by every thread, 16 per thread for a 64 KiB slab) land
// in the other buffer.  cp.async.wait_group completes on its own, so no wait can hang.

// DF (complex128 only): the slab is converted in place to double-float pairs after it lands,
// the register stages compute on the FP32 pipe (df_arith.cuh) with double-float coefficients
// (coef_df), and every amplitude is converted back on its way to HBM.  Only passes made of
// register stages run in this form (the host checks); the state in HBM stays complex128.
template <typename R, int RB, int NT, bool DF = false>
__global__ void __launch_bounds__(NT, 1)
    slab_pass_kernel(typename Cx<R>::T *__restrict__ state, const DevPass *__restrict__ d_pass,
                     const DevOp *__restrict__ ops, const DevStage *__restrict__ stages,
                     const DevSub *__restrict__ subs, const typename Cx<R>::T *__restrict__ coef,
                     const dfc *__restrict__ coef_df, uint64_t nslabs)
{
    using C = typename Cx<R>::T;
    static_assert(!DF || sizeof(C) == sizeof(dfc), "double-float slabs replace complex128 slabs");
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

    // [SlabShared][vector offsets of the slab's 16-byte chunks: kMaxVec x 8 B][buffer 0][buffer 1]
    uint64_t *const voff = reinterpret_cast<uint64_t *>(smem_raw + ((sizeof(SlabShared) + 127) & ~size_t(127)));
    C *const buf0 = reinterpret_cast<C *>(reinterpret_cast<unsigned char *>(voff) + kMaxVec * sizeof(uint64_t));
    const uint32_t nsl = 1u << b;
    constexpr int kLog16 = (sizeof(C) == 8) ? 1 : 0;  // log2(amplitudes per 16-byte vector)
    const int vps_log = lo - kLog16;
    const uint32_t nvec = 1u << (b - kLog16);
    // the global 16-byte-vector offset of chunk v from the slab base is the same for every slab
    // of the pass: computed once here, one shared-memory load per chunk afterwards
    for (uint32_t v = tid; v < nvec; v += NT) {
        const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
        voff[v] = ((S.seg_lo[seg & 63] | S.seg_hi[(seg >> 6) & 63]) >> kLog16) + w;
    }
    __syncthreads();
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
    // chunk_of is linear over GF(2) and NT is a power of two above tid, so the chunk of
    // v = tid + k NT is chunk_of(tid) ^ chunk_of(k NT), the second term a constant per unrolled k
    const uint32_t ct = chunk_of(tid);
    auto issue_load = [&](uint64_t slab, uint32_t k) {
        const uint4 *g = reinterpret_cast<const uint4 *>(state + slab_base(slab));
        const uint32_t dst = smem_addr(buf0 + size_t(k) * nsl);
#pragma unroll
        for (uint32_t j = 0; j < kMaxVec / NT; ++j) {
            const uint32_t v = tid + j * NT;
            if (v >= nvec) break;
            cp_async16(dst + 16u * (ct ^ chunk_of(j * NT)), g + voff[v]);
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
        if (DF) {
            // complex128 -> double-float pairs, each 16-byte slot in place
            dfc *sd = reinterpret_cast<dfc *>(sm);
            for (uint32_t e = tid; e < nsl; e += NT) {
                const C a = sm[e];
                sd[e] = dfc{d2df(a.x), d2df(a.y)};
            }
            __syncthreads();
            for (int o = op_begin; o < op_end; ++o) {
                const DevOp &op = ops[o];
                if ((base & op.ocmask) == op.ocmask) run_stage<dfc, RB>(sd, stages + op.mat, subs, coef_df, base, tid, NT);
                __syncthreads();
            }
        } else {
            // the gate block
            for (int o = op_begin; o < op_end; ++o) {
                const DevOp &op = ops[o];
                if ((base & op.ocmask) == op.ocmask) {
                    if (op.type == OP_STAGE) run_stage<C, RB>(sm, stages + op.mat, subs, coef, base, tid, NT);
                    else run_smem_op<C>(sm, b, op, coef, base, tid, NT);
                }
                __syncthreads();
            }
        }
        // store
        if (!S.pass.has_perm) {
            uint4 *gv = reinterpret_cast<uint4 *>(gbase);
#pragma unroll
            for (uint32_t j = 0; j < kMaxVec / NT; ++j) {
                const uint32_t v = tid + j * NT;
                if (v >= nvec) break;
                const uint32_t slot = ct ^ chunk_of(j * NT);
                if (DF) {
                    const dfc q = reinterpret_cast<const dfc *>(sm)[slot];
                    const double2 d = make_double2(df2d(q.x), df2d(q.y));
                    st_stream(gv + voff[v], *reinterpret_cast<const uint4 *>(&d));
                } else {
                    st_stream(gv + voff[v], reinterpret_cast<const uint4 *>(sm)[slot]);
                }
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
template <typename R, int RB, int NT, bool DF = false>
int launch_pass_t(const LaunchCtx &c, const PassArgs &a, const DevPass &h, char *err, size_t errlen)
{
    using C = typename Cx<R>::T;
    const size_t smem = pass_smem_bytes(c.dt, h.b, h.lo);
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaFuncSetAttribute(slab_pass_kernel<R, RB, NT, DF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
        attr_dev = dev;
    }
    const uint64_t nslabs = 1ull << (c.n - h.b);
    uint64_t grid = uint64_t(num_sms());
    if (grid > nslabs) grid = nslabs;
    slab_pass_kernel<R, RB, NT, DF><<<(unsigned)grid, NT, smem, (cudaStream_t)c.stream>>>(
        reinterpret_cast<C *>(c.amp), a.pass, a.ops, a.stages, a.subs,
        reinterpret_cast<const C *>(a.coef), reinterpret_cast<const dfc *>(a.coef_df), nslabs);
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
    // shared block, chunk-offset table, two slab buffers
    return ((sizeof(SlabShared) + 127) & ~size_t(127)) + kMaxVec * sizeof(uint64_t) + 2 * (amp << b);
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
    if (a.df) {
        if (!a.coef_df) {
            snprintf(err, errlen, "double-float pass without double-float coefficients");
            return QS_EINVAL;
        }
        if (a.stage_bits == kStageBitsC128 - 1)
            return launch_pass_t<double, kStageBitsC128 - 1, 512, true>(c, a, h, err, errlen);
        return launch_pass_t<double, kStageBitsC128, 256, true>(c, a, h, err, errlen);
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
