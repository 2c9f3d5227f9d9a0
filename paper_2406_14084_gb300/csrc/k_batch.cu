// k_batch.cu -- many independent circuits in one persistent launch.
//
// The host concatenates the slab-pass plans of all circuits and lists work items (circuit,
// pass, slab) in dependency rounds: every circuit's pass 0, then every pass 1, and so on.
// Persistent CTAs take items from an atomic queue head in that order.  Before pass p > 0 of a
// circuit may start, all slabs of its pass p-1 must be stored: thread 0 spins, with a bounded
// number of polls, on the circuit's done counter for pass p-1 (acquire loads; producers
// release with a fence before incrementing).  Items are handed out in order and a CTA never
// waits on an item handed out after its own, so the earliest unfinished item can always run.
// Pass 0 initialises |0..0> in shared memory instead of loading the state; the last pass
// accumulates the circuit's Z-string expectation sum_x |a_x|^2 h(x) from the slab in shared
// memory (FP32 partial sums of at most 32 amplitudes, then FP64) and adds it to the
// circuit's result with one FP64 atomic per CTA.
#include <cuda_runtime.h>

#include <cstdio>

#include "slab_common.cuh"

namespace qs {
namespace {

constexpr uint32_t kSpinLimit = 1u << 22;

struct __align__(16) BatchShared {
    uint64_t seg_lo[64], seg_hi[64];
    DevPass pass;
    BatchItem item;
    BatchCirc circ;
    double red[32];
    int go;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename R, int RB, int NT>
__global__ void __launch_bounds__(NT, 1)
    batch_kernel(typename Cx<R>::T *__restrict__ states, BatchArgs a)
{
    using C = typename Cx<R>::T;
    constexpr int SW = sizeof(C) == 8 ? 1 : 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BatchShared &S = *reinterpret_cast<BatchShared *>(smem_raw);
    C *const sm = reinterpret_cast<C *>(smem_raw + ((sizeof(BatchShared) + 127) & ~size_t(127)));
    const uint32_t tid = threadIdx.x;
    const C *coef = reinterpret_cast<const C *>(a.coef);

    while (true) {
        if (tid == 0) {
            const unsigned it = atomicAdd(a.head, 1u);
            S.go = it < a.nitems ? 1 : 0;
            if (S.go) {
                S.item = a.items[it];
                S.circ = a.circs[S.item.circ];
                S.pass = a.passes[S.circ.pass0 + S.item.pass];
                if (S.item.pass > 0) {
                    // wait for every slab of the previous pass of this circuit
                    const unsigned need = 1u << S.circ.nslab_log;
                    const unsigned *cnt = a.done + S.circ.done0 + S.item.pass - 1;
                    uint32_t k = 0;
                    while (ld_acquire(cnt) < need && ++k < kSpinLimit) __nanosleep(128);
                    if (k >= kSpinLimit) {
                        atomicExch(a.status, QS_ETIMEOUT);
                        S.go = 2;  // skip the work; the host reports the timeout
                    }
                    __threadfence();
                }
            }
        }
        __syncthreads();
        const int go = S.go;
        if (go == 0) break;
        const int b = S.pass.b, lo = S.pass.lo, nhi = S.pass.nhi;
        const bool first = S.item.pass == 0, last = S.item.pass == S.circ.npass - 1;
        for (uint32_t j = tid; j < 128; j += NT) {
            const uint32_t x = j & 63, sh = (j < 64) ? 0 : 6;
            uint64_t o = 0;
            for (int m = 0; m < 6; ++m)
                if ((x >> m & 1) && int(m + sh) < nhi) o |= 1ull << S.pass.hipos[m + sh];
            if (j < 64) S.seg_lo[x] = o; else S.seg_hi[x] = o;
        }
        uint64_t base = uint64_t(S.item.slab) << lo;
        for (int m = 0; m < nhi; ++m) {
            const uint64_t lowm = (1ull << S.pass.hipos[m]) - 1;
            base = ((base & ~lowm) << 1) | (base & lowm);
        }
        C *g = states + S.circ.amp_off + base;
        const uint32_t nsl = 1u << b;
        constexpr int kLog16 = (sizeof(C) == 8) ? 1 : 0;
        const int vps_log = lo - kLog16;
        const uint32_t nvec = 1u << (b - kLog16);
        auto chunk_of = [](uint32_t v) -> uint32_t { return sizeof(C) == 8 ? (swz<1>(v << 1) >> 1) : swz<2>(v); };
        __syncthreads();
        if (go == 1) {
            if (first) {
                for (uint32_t i = tid; i < nsl; i += NT) {
                    C z;
                    z.x = (base == 0 && i == 0) ? R(1) : R(0);
                    z.y = R(0);
                    sm[swz<SW>(i)] = z;
                }
            } else {
                const uint32_t dst = smem_addr(sm);
                for (uint32_t v = tid; v < nvec; v += NT) {
                    const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
                    const uint64_t so = S.seg_lo[seg & 63] | S.seg_hi[(seg >> 6) & 63];
                    cp_async16(dst + 16u * chunk_of(v), reinterpret_cast<const uint4 *>(g + so) + w);
                }
                cp_async_commit();
                cp_async_wait<0>();
            }
            __syncthreads();
            for (int o = S.pass.op_begin; o < S.pass.op_end; ++o) {
                const DevOp &op = a.ops[o];
                if ((base & op.ocmask) == op.ocmask) {
                    if (op.type == OP_STAGE) run_stage<C, RB>(sm, a.stages + op.mat, a.subs, coef, base, tid, NT);
                    else run_smem_op<C>(sm, b, op, coef, base, tid, NT);
                }
                __syncthreads();
            }
            if (last) {
                // sum over the slab of |a_x|^2 sum_t c_t (-1)^{popcount(x & z_t)}
                double acc = 0.0;
                R part = 0;
                int cnt = 0;
                const BatchTerm *T = a.terms + S.circ.term0;
                const int nt = S.circ.nterm;
                for (uint32_t i = tid; i < nsl; i += NT) {
                    uint64_t x = base | (i & ((1u << lo) - 1));
                    for (int m = 0; m < nhi; ++m) x |= uint64_t((i >> (lo + m)) & 1u) << S.pass.hipos[m];
                    R h = 0;
                    for (int t = 0; t < nt; ++t) h += (__popcll(x & T[t].zm) & 1) ? -R(T[t].c) : R(T[t].c);
                    const C v = sm[swz<SW>(i)];
                    const R p = v.x * v.x + v.y * v.y;
                    part = fma(p, h, part);
                    if (++cnt == 32) {
                        acc += double(part);
                        part = 0.f;
                        cnt = 0;
                    }
                }
                acc += double(part);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
                if ((tid & 31) == 0) S.red[tid >> 5] = acc;
                __syncthreads();
                if (tid < 32) {
                    double v = tid < NT / 32 ? S.red[tid] : 0.0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                    if (tid == 0) atomicAdd(a.results + S.item.circ, v);
                }
            }
            for (uint32_t v = tid; v < nvec; v += NT) {
                const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
                const uint64_t so = S.seg_lo[seg & 63] | S.seg_hi[(seg >> 6) & 63];
                st_stream(reinterpret_cast<uint4 *>(g + so) + w, reinterpret_cast<const uint4 *>(sm)[chunk_of(v)]);
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(a.done + S.circ.done0 + S.item.pass, 1u);
    }
}

template <typename R, int RB, int NT>
int launch_batch_t(void *states, const BatchArgs &a, int b_max, void *stream, char *err, size_t errlen)
{
    using C = typename Cx<R>::T;
    const size_t smem = ((sizeof(BatchShared) + 127) & ~size_t(127)) + (sizeof(C) << b_max);
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaFuncSetAttribute(batch_kernel<R, RB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_dev = dev;
    }
    unsigned grid = (unsigned)num_sms();
    if (grid > a.nitems) grid = a.nitems > 0 ? a.nitems : 1;
    batch_kernel<R, RB, NT><<<grid, NT, smem, (cudaStream_t)stream>>>(reinterpret_cast<C *>(states), a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "batch launch failed: %s", cudaGetErrorString(e));
        return QS_ECUDA;
    }
    return QS_OK;
}

}  // namespace

int launch_batch(qs_dtype dt, int stage_bits, void *states, const BatchArgs &a, int b_max, void *stream,
                 char *err, size_t errlen)
{
    if (dt == QS_C64) {
        if (stage_bits == kStageBitsC64 - 1)
            return launch_batch_t<float, kStageBitsC64 - 1, 512>(states, a, b_max, stream, err, errlen);
        return launch_batch_t<float, kStageBitsC64, 256>(states, a, b_max, stream, err, errlen);
    }
    if (stage_bits == kStageBitsC128 - 1)
        return launch_batch_t<double, kStageBitsC128 - 1, 512>(states, a, b_max, stream, err, errlen);
    return launch_batch_t<double, kStageBitsC128, 256>(states, a, b_max, stream, err, errlen);
}

}  // namespace qs
