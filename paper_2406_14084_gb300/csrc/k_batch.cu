// k_batch.cu -- many independent circuits in one persistent launch.
//
// The host concatenates the slab-pass plans of all circuits and lists work items (circuit,
// pass, slab) in dependency rounds: every circuit's pass 0, then every pass 1, and so on.
// Persistent CTAs take items from an atomic queue head in that order.  Before pass p > 0 of a
// circuit may start, all slabs of its pass p-1 must be stored (the circuit's done counter for
// pass p-1, read with acquire loads; producers release with a fence before incrementing).
// Each CTA keeps two items: while one is computed, the next one's gather streams into the
// second buffer if its dependency already holds; otherwise thread 0 waits for it (a bounded
// number of polls) only after the current item has been stored and counted.  So a CTA never
// waits on its own work, and the earliest unfinished item in queue order can always run.
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

struct __align__(16) BatchSlot {
    uint64_t seg_lo[64], seg_hi[64];  // gather tables of the item's pass
    DevPass pass;
    BatchItem item;
    BatchCirc circ;
    uint64_t base;                    // slab base index in the circuit's state
    int st;                           // 0 none, 1 ready, 2 dependency wait ran out, 3 not ready yet
    int pad;
};

struct __align__(16) BatchShared {
    BatchSlot slot[2];
    double red[32];
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: the next slab for slot k after slot `from`: the following slab of the same run
// (no queue access; its dependency holds as for the run's first slab), or else the next item
// from the queue, whose dependency (the circuit's previous pass fully stored) is checked once.
__device__ void take_item(BatchShared &S, int k, const BatchArgs &a, int from)
{
    BatchSlot &Z = S.slot[k];
    if (from >= 0) {
        const BatchSlot &P = S.slot[from];
        if (P.st == 1 && P.item.count > 1) {
            Z.item = P.item;
            Z.item.slab += 1;
            Z.item.count -= 1;
            Z.circ = P.circ;
            Z.pass = P.pass;
            Z.st = 1;
            return;
        }
    }
    const unsigned it = atomicAdd(a.head, 1u);
    if (it >= a.nitems) {
        Z.st = 0;
        return;
    }
    Z.item = a.items[it];
    Z.circ = a.circs[Z.item.circ];
    Z.pass = a.passes[Z.circ.pass0 + Z.item.pass];
    Z.st = 1;
    if (Z.item.pass > 0) {
        const unsigned need = 1u << Z.circ.nslab_log;
        if (ld_acquire(a.done + Z.circ.done0 + Z.item.pass - 1) < need) Z.st = 3;
        __threadfence();
    }
}

__device__ void wait_item(BatchShared &S, int k, const BatchArgs &a)
{
    BatchSlot &Z = S.slot[k];
    const unsigned need = 1u << Z.circ.nslab_log;
    const unsigned *cnt = a.done + Z.circ.done0 + Z.item.pass - 1;
    uint32_t n = 0;
    while (ld_acquire(cnt) < need && ++n < kSpinLimit) __nanosleep(128);
    if (n >= kSpinLimit) {
        atomicExch(a.status, QS_ETIMEOUT);
        Z.st = 2;  // skip the work; the host reports the timeout
    } else {
        Z.st = 1;
    }
    __threadfence();
}

// All threads: gather tables and slab base of slot k (its item must be known).
__device__ void prepare_slot(BatchSlot &Z, uint32_t tid, uint32_t nthr)
{
    const int lo = Z.pass.lo, nhi = Z.pass.nhi;
    for (uint32_t j = tid; j < 128; j += nthr) {
        const uint32_t x = j & 63, sh = (j < 64) ? 0 : 6;
        uint64_t o = 0;
        for (int m = 0; m < 6; ++m)
            if ((x >> m & 1) && int(m + sh) < nhi) o |= 1ull << Z.pass.hipos[m + sh];
        if (j < 64) Z.seg_lo[x] = o; else Z.seg_hi[x] = o;
    }
    if (tid == 0) {
        uint64_t base = uint64_t(Z.item.slab) << lo;
        for (int m = 0; m < nhi; ++m) {
            const uint64_t lowm = (1ull << Z.pass.hipos[m]) - 1;
            base = ((base & ~lowm) << 1) | (base & lowm);
        }
        Z.base = base;
    }
}

template <typename C>
__device__ __forceinline__ uint32_t chunk_of(uint32_t v)
{
    return sizeof(C) == 8 ? (swz<1>(v << 1) >> 1) : swz<2>(v);
}

// All threads: issue the 16-byte gather of slot k's slab into buffer `buf` (passes > 0) and
// commit one copy group (empty for pass 0, so that every slot owns exactly one group).
template <typename C>
__device__ void issue_slot_load(const BatchSlot &Z, C *states, C *buf, uint32_t tid, uint32_t nthr)
{
    if (Z.st == 1 && Z.item.pass > 0) {
        constexpr int kLog16 = (sizeof(C) == 8) ? 1 : 0;
        const int vps_log = Z.pass.lo - kLog16;
        const uint32_t nvec = 1u << (Z.pass.b - kLog16);
        const C *g = states + Z.circ.amp_off + Z.base;
        const uint32_t dst = smem_addr(buf);
        for (uint32_t v = tid; v < nvec; v += nthr) {
            const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
            const uint64_t so = Z.seg_lo[seg & 63] | Z.seg_hi[(seg >> 6) & 63];
            cp_async16(dst + 16u * chunk_of<C>(v), reinterpret_cast<const uint4 *>(g + so) + w);
        }
    }
    cp_async_commit();
}

// Each CTA keeps two items in flight: while item i is computed and stored, the gather of the
// item taken after it (when its dependency already holds) streams into the other buffer.  An item
// whose dependency does not hold yet -- for example the next pass of the circuit whose last slab
// is item i itself -- is waited for only after item i has been stored and counted, so a CTA never
// waits on its own work.
template <typename R, int RB, int NT>
__global__ void __launch_bounds__(NT, 1)
    batch_kernel(typename Cx<R>::T *__restrict__ states, BatchArgs a, uint32_t buf_elems)
{
    using C = typename Cx<R>::T;
    constexpr int SW = sizeof(C) == 8 ? 1 : 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BatchShared &S = *reinterpret_cast<BatchShared *>(smem_raw);
    C *const bufs = reinterpret_cast<C *>(smem_raw + ((sizeof(BatchShared) + 127) & ~size_t(127)));
    const uint32_t tid = threadIdx.x;
    const C *coef = reinterpret_cast<const C *>(a.coef);

    int cur = 0;
    if (tid == 0) {
        take_item(S, 0, a, -1);
        if (S.slot[0].st == 3) wait_item(S, 0, a);
    }
    __syncthreads();
    if (S.slot[0].st == 0) return;
    prepare_slot(S.slot[0], tid, NT);
    __syncthreads();
    issue_slot_load<C>(S.slot[0], states, bufs, tid, NT);

    while (true) {
        const int nxt = cur ^ 1;
        BatchSlot &Z = S.slot[cur];
        BatchSlot &Y = S.slot[nxt];
        C *const sm = bufs + size_t(cur) * buf_elems;
        // take the next item; gather it now if its dependency already holds
        if (tid == 0) take_item(S, nxt, a, cur);
        __syncthreads();
        bool prefetched = false;
        if (Y.st == 1) {
            prepare_slot(Y, tid, NT);
            __syncthreads();
            issue_slot_load<C>(Y, states, bufs + size_t(nxt) * buf_elems, tid, NT);
            prefetched = true;
        }
        if (prefetched) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();

        if (Z.st == 1) {
            const int b = Z.pass.b, lo = Z.pass.lo, nhi = Z.pass.nhi;
            const uint64_t base = Z.base;
            const uint32_t nsl = 1u << b;
            const bool first = Z.item.pass == 0, last = Z.item.pass == Z.circ.npass - 1;
            if (first) {
                for (uint32_t i = tid; i < nsl; i += NT) {
                    C z;
                    z.x = (base == 0 && i == 0) ? R(1) : R(0);
                    z.y = R(0);
                    sm[swz<SW>(i)] = z;
                }
                __syncthreads();
            }
            for (int o = Z.pass.op_begin; o < Z.pass.op_end; ++o) {
                const DevOp &op = a.ops[o];
                if ((base & op.ocmask) == op.ocmask) {
                    if (op.type == OP_STAGE) run_stage<C, RB>(sm, a.stages + op.mat, a.subs, coef, base, tid, NT);
                    else run_smem_op<C>(sm, b, op, coef, base, tid, NT);
                }
                __syncthreads();
            }
            if (last) {
                // <psi| sum_t c_t Z_t |psi> over the slab.  With x = base | deposit(i) (base: the
                // bits outside the slab), (-1)^{popcount(x & z_t)} = s_t(base) (-1)^{popcount(i & zl_t)}
                // where zl_t is z_t on the slab's local bits, so the slab contributes
                //   sum_t c_t s_t(base) P^(zl_t),   P^(z) = sum_i |a_i|^2 (-1)^{popcount(i & z)},
                // the Walsh-Hadamard transform of the slab's probabilities, computed in place in
                // shared memory (state precision) in b butterfly stages.
                R *pr = reinterpret_cast<R *>(sm);
                constexpr int kPer = 32;  // slab amplitudes per thread (2^13 / 256, 2^12 / 128 ...)
                R pv[kPer];
#pragma unroll
                for (int k = 0; k < kPer; ++k) {
                    const uint32_t i = tid + uint32_t(k) * NT;
                    if (i < nsl) {
                        const C v = sm[swz<SW>(i)];
                        pv[k] = v.x * v.x + v.y * v.y;
                    }
                }
                __syncthreads();  // every amplitude has been read: the buffer now holds pr[]
#pragma unroll
                for (int k = 0; k < kPer; ++k) {
                    const uint32_t i = tid + uint32_t(k) * NT;
                    if (i < nsl) pr[i] = pv[k];
                }
                for (int j = 0; j < b; ++j) {
                    __syncthreads();
                    const uint32_t low = (1u << j) - 1u;
                    for (uint32_t q = tid; q < nsl / 2; q += NT) {
                        const uint32_t i0 = ((q & ~low) << 1) | (q & low), i1 = i0 | (1u << j);
                        const R u = pr[i0], w = pr[i1];
                        pr[i0] = u + w;
                        pr[i1] = u - w;
                    }
                }
                __syncthreads();
                const BatchTerm *T = a.terms + Z.circ.term0;
                const int nt = Z.circ.nterm;
                double acc = 0.0;
                for (int t = int(tid); t < nt; t += NT) {
                    const uint64_t zm = T[t].zm;
                    uint32_t zl = uint32_t(zm) & ((1u << lo) - 1u);
                    for (int m = 0; m < nhi; ++m) zl |= uint32_t((zm >> Z.pass.hipos[m]) & 1u) << (lo + m);
                    const double sg = (__popcll(base & zm) & 1) ? -T[t].c : T[t].c;
                    acc += sg * double(pr[zl]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
                if ((tid & 31) == 0) S.red[tid >> 5] = acc;
                __syncthreads();
                if (tid < 32) {
                    double v = tid < NT / 32 ? S.red[tid] : 0.0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                    if (tid == 0) atomicAdd(a.results + Z.item.circ, v);
                }
            } else {
                // the final states are not kept (the batch returns expectation values only), so
                // the last pass stores nothing
                constexpr int kLog16 = (sizeof(C) == 8) ? 1 : 0;
                const int vps_log = lo - kLog16;
                const uint32_t nvec = 1u << (b - kLog16);
                C *g = states + Z.circ.amp_off + base;
                for (uint32_t v = tid; v < nvec; v += NT) {
                    const uint32_t seg = v >> vps_log, w = v & ((1u << vps_log) - 1);
                    const uint64_t so = Z.seg_lo[seg & 63] | Z.seg_hi[(seg >> 6) & 63];
                    st_stream(reinterpret_cast<uint4 *>(g + so) + w,
                              reinterpret_cast<const uint4 *>(sm)[chunk_of<C>(v)]);
                }
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) atomicAdd(a.done + Z.circ.done0 + Z.item.pass, 1u);
        // the next item: stop, or wait for its dependency now that this item is counted
        if (Y.st == 0) break;
        if (Y.st == 3) {
            if (tid == 0) wait_item(S, nxt, a);
            __syncthreads();
            prepare_slot(Y, tid, NT);
            __syncthreads();
            issue_slot_load<C>(Y, states, bufs + size_t(nxt) * buf_elems, tid, NT);
        }
        cur = nxt;
    }
    cp_async_wait<0>();
}

template <typename R, int RB, int NT>
int launch_batch_t(void *states, const BatchArgs &a, int b_max, void *stream, char *err, size_t errlen)
{
    using C = typename Cx<R>::T;
    const size_t smem = ((sizeof(BatchShared) + 127) & ~size_t(127)) + 2 * (sizeof(C) << b_max);
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaFuncSetAttribute(batch_kernel<R, RB, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_dev = dev;
    }
    unsigned grid = (unsigned)num_sms();
    if (grid > a.nitems) grid = a.nitems > 0 ? a.nitems : 1;
    if (smem > 227 * 1024) {
        snprintf(err, errlen, "batch slab of %d bits does not fit two buffers in shared memory", b_max);
        return QS_EINVAL;
    }
    batch_kernel<R, RB, NT><<<grid, NT, smem, (cudaStream_t)stream>>>(reinterpret_cast<C *>(states), a,
                                                                       uint32_t(1) << b_max);
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
