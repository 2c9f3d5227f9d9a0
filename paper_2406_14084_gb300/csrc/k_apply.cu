// k_apply.cu -- the gate-by-gate kernel: one op applied to the whole state in global memory
// (the unblocked scheme that arXiv 2406.14084 compares against; also the fallback for an op
// that fits no slab).  Each thread handles amplitude groups g = tid, tid + nthreads, ...
#include <cuda_runtime.h>

#include <cstdio>

#include "op_global.cuh"
#include "qs_internal.h"

namespace qs {
namespace {

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
    apply_op_global<C, uint64_t, 0>(state, n, op, coef, 0u, tid, nthr);
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

int num_sms()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        sms = v > 0 ? v : 1;
    }
    return sms;
}

int launch_unblocked(const LaunchCtx &c, const DevOp *d_op, const DevOp &h_op, const void *d_coef,
                     char *err, size_t errlen)
{
    if (c.dt == QS_C64) return launch_unblocked_t<float>(c, d_op, h_op, d_coef, err, errlen);
    return launch_unblocked_t<double>(c, d_op, h_op, d_coef, err, errlen);
}

}  // namespace qs
