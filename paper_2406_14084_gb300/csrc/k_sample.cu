// k_sample.cu -- measurement sampling in the computational basis (Born rule).
//
// For caller-supplied uniforms u_k in [0, 1) the outcome of shot k is the smallest index x whose
// running weight C(x) = sum_{y <= x} |a_y|^2 exceeds u_k * C(2^n - 1) (inverse transform).  The
// state is cut into blocks of 2^kBlockLog amplitudes:
//   1. block_sums_kernel: one warp per block sums |a|^2 (fixed order: each lane a strided run,
//      then a shuffle tree) in FP64, or for complex64 in float-float pairs (~48 bits);
//   2. scan_chunks_kernel / scan_tops_kernel / add_tops_kernel: exclusive prefix of the block
//      sums (chunks of 1024 in shared memory, then the chunk totals in one block, then the
//      offsets added back), so P[j] is the weight before block j and P[M] the total;
//   3. sample_kernel: one warp per shot finds the block by binary search over P, loads the
//      block's amplitudes at once and finds the index inside it with warp-wide inclusive scans
//      over runs of 32 amplitudes.
#include <cuda_runtime.h>

#include <cstdio>

#include "qs_internal.h"

namespace qs {
namespace {

// 256 amplitudes per block: a shot then reads one block (eight loads per lane, all in flight at
// once) after a binary search over the 2^(n-8) block prefixes, which stay in L2 up to 32 qubits
constexpr int kBlockLog = 8;
constexpr int kLoads = (1 << kBlockLog) / 32;  // amplitudes per lane in one block
constexpr int kChunk = 1024;   // block sums scanned per CTA

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename C>
__device__ __forceinline__ double weight(const C &v)
{
    const double re = (double)v.x, im = (double)v.y;
    return re * re + im * im;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_incl_scan(double v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Float-float (unevaluated hi + lo pair) arithmetic for complex64 block sums, so that the sums
// keep about 48 bits without the FP64 pipe (1/64 of the FP32 rate on this part).  Error-free
// transformations: Knuth's TwoSum and the FMA form of Dekker's TwoProduct; the _rn intrinsics
// keep the compiler from contracting or reordering them.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float bh, float bl)
{
    const float s = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    e = __fadd_rn(e, __fadd_rn(lo, bl));
    hi = __fadd_rn(s, e);  // renormalise (|s| >= |e|)
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// |v|^2 of a complex64 amplitude as a float-float pair (each square is exact as a pair).
__device__ __forceinline__ void ff_weight(const float2 &v, float &hi, float &lo)
{
    const float px = __fmul_rn(v.x, v.x), py = __fmul_rn(v.y, v.y);
    const float ex = __fmaf_rn(v.x, v.x, -px), ey = __fmaf_rn(v.y, v.y, -py);
    hi = px;
    lo = ex;
    ff_add(hi, lo, py, ey);
}

template <typename R>
__global__ void block_sums_kernel(const typename Cx<R>::T *__restrict__ a, uint64_t nblocks, int blog,
                                  double *__restrict__ S)
{
    const uint64_t w = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nblocks) return;
    const uint64_t base = w << blog, len = uint64_t(1) << blog;
    typename Cx<R>::T v[kLoads];
#pragma unroll
    for (int c = 0; c < kLoads; ++c) {
        const uint64_t i = uint64_t(c) * 32 + lane;
        v[c] = i < len ? a[base + i] : typename Cx<R>::T{};
    }
    if constexpr (sizeof(R) == 4) {
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int c = 0; c < kLoads; ++c) {
            float wh, wl;
            ff_weight(v[c], wh, wl);
            ff_add(hi, lo, wh, wl);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o), ol = __shfl_xor_sync(0xffffffffu, lo, o);
            ff_add(hi, lo, oh, ol);
        }
        if (lane == 0) S[w] = (double)hi + (double)lo;
    } else {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < kLoads; ++c) s += weight(v[c]);
        s = warp_sum(s);
        if (lane == 0) S[w] = s;
    }
}

// Exclusive prefix of S within chunks of kChunk; chunk totals to T.
__global__ void __launch_bounds__(kChunk) scan_chunks_kernel(const double *__restrict__ S, uint64_t M,
                                                             double *__restrict__ P, double *__restrict__ T)
{
    __shared__ double wsum[kChunk / 32];
    const uint64_t i = uint64_t(blockIdx.x) * kChunk + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double v = i < M ? S[i] : 0.0;
    const double inc = warp_incl_scan(v, lane);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        const double x = wsum[lane];
        wsum[lane] = warp_incl_scan(x, lane) - x;  // exclusive over warps
    }
    __syncthreads();
    if (i < M) P[i] = wsum[w] + inc - v;
    if (threadIdx.x == kChunk - 1) T[blockIdx.x] = wsum[w] + inc;
}

// Exclusive prefix of the chunk totals (at most kChunk * kChunk chunks, one CTA); T[nt] = total.
__global__ void __launch_bounds__(kChunk) scan_tops_kernel(double *__restrict__ T, int nt)
{
    __shared__ double wsum[kChunk / 32];
    __shared__ double carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0.0;
    __syncthreads();
    for (int base = 0; base < nt; base += kChunk) {
        const int i = base + threadIdx.x;
        const double v = i < nt ? T[i] : 0.0;
        const double inc = warp_incl_scan(v, lane);
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        if (w == 0) {
            const double x = wsum[lane];
            wsum[lane] = warp_incl_scan(x, lane) - x;
        }
        __syncthreads();
        const double c = carry;
        if (i < nt) T[i] = c + wsum[w] + inc - v;
        __syncthreads();
        if (threadIdx.x == kChunk - 1) carry = c + wsum[w] + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) T[nt] = carry;
}

__global__ void add_tops_kernel(double *__restrict__ P, uint64_t M, const double *__restrict__ T)
{
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < M) P[i] += T[i / kChunk];
    if (i == 0) P[M] = T[(M + kChunk - 1) / kChunk];
}

template <typename R>
__global__ void sample_kernel(const typename Cx<R>::T *__restrict__ a, int blog, const double *__restrict__ P,
                              uint64_t M, const double *__restrict__ u, uint64_t shots, uint64_t *__restrict__ out)
{
    const uint64_t k = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= shots) return;
    const double total = P[M];
    const double t = u[k] * total;
    // last block j with P[j] <= t (P is non-decreasing, P[0] = 0); P[j] < total keeps the
    // search off trailing zero-weight blocks even if t reached the total
    uint64_t lo = 0, hi = M - 1;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo + 1) / 2;
        if (P[mid] <= t && P[mid] < total) lo = mid;
        else hi = mid - 1;
    }
    const uint64_t j = lo, base = j << blog, len = uint64_t(1) << blog;
    double w[kLoads];  // the whole block, loaded at once; zero weight past its end (n < 8)
#pragma unroll
    for (int c = 0; c < kLoads; ++c) {
        const uint64_t i = uint64_t(c) * 32 + lane;
        w[c] = i < len ? weight(a[base + i]) : 0.0;
    }
    double run = P[j];
    uint64_t found = ~uint64_t(0), last_nz = base;
#pragma unroll
    for (int c = 0; c < kLoads; ++c) {
        if (found != ~uint64_t(0)) break;  // warp-uniform
        const double inc = warp_incl_scan(w[c], lane);
        const unsigned hit = __ballot_sync(0xffffffffu, run + inc > t);
        const unsigned nz = __ballot_sync(0xffffffffu, w[c] > 0.0);
        if (nz) last_nz = base + uint64_t(c) * 32 + 31 - __clz(nz);
        if (hit) found = base + uint64_t(c) * 32 + __ffs(hit) - 1;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    // rounding can leave t at or past this block's end: the last outcome of positive weight
    if (lane == 0) out[k] = found != ~uint64_t(0) ? found : last_nz;
}

int launched(const char *what, char *err, size_t errlen)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "%s launch failed: %s", what, cudaGetErrorString(e));
        return QS_ECUDA;
    }
    return QS_OK;
}

}  // namespace

size_t sample_scratch_bytes(int n)
{
    const int blog = n < kBlockLog ? n : kBlockLog;
    const uint64_t M = uint64_t(1) << (n - blog);
    const uint64_t nt = (M + kChunk - 1) / kChunk;
    return sizeof(double) * (2 * M + 1 + nt + 1) + 256;
}

size_t sample_total_index(int n)
{
    const int blog = n < kBlockLog ? n : kBlockLog;
    return 2 * (size_t(1) << (n - blog));
}

int launch_sample(const LaunchCtx &c, const double *d_u, uint64_t shots, uint64_t *d_out, void *d_scratch,
                  char *err, size_t errlen)
{
    cudaStream_t st = (cudaStream_t)c.stream;
    const int blog = c.n < kBlockLog ? c.n : kBlockLog;
    const uint64_t M = uint64_t(1) << (c.n - blog);
    const uint64_t nt = (M + kChunk - 1) / kChunk;
    if (nt > uint64_t(kChunk) * kChunk) {
        snprintf(err, errlen, "sample: state too large");
        return QS_EINVAL;
    }
    double *S = static_cast<double *>(d_scratch), *P = S + M, *T = P + M + 1;
    const unsigned wpb = 8;  // warps per 256-thread CTA
    const unsigned g1 = unsigned((M + wpb - 1) / wpb);
    if (c.dt == QS_C64)
        block_sums_kernel<float><<<g1, 256, 0, st>>>((const float2 *)c.amp, M, blog, S);
    else
        block_sums_kernel<double><<<g1, 256, 0, st>>>((const double2 *)c.amp, M, blog, S);
    int rc = launched("sample block sums", err, errlen);
    if (rc) return rc;
    scan_chunks_kernel<<<unsigned(nt), kChunk, 0, st>>>(S, M, P, T);
    scan_tops_kernel<<<1, kChunk, 0, st>>>(T, int(nt));
    add_tops_kernel<<<unsigned((M + 255) / 256), 256, 0, st>>>(P, M, T);
    rc = launched("sample prefix", err, errlen);
    if (rc) return rc;
    if (shots == 0) return QS_OK;
    const unsigned g2 = unsigned((shots + wpb - 1) / wpb);
    if (c.dt == QS_C64)
        sample_kernel<float><<<g2, 256, 0, st>>>((const float2 *)c.amp, blog, P, M, d_u, shots, d_out);
    else
        sample_kernel<double><<<g2, 256, 0, st>>>((const double2 *)c.amp, blog, P, M, d_u, shots, d_out);
    return launched("sample", err, errlen);
}

}  // namespace qs
