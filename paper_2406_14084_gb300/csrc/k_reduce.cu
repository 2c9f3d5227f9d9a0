// k_reduce.cu -- readout reductions over the state vector (one read pass each).
//
//  * norm2:  sum |a_x|^2
//  * probs:  marginal probabilities over a set of physical bit positions
//  * expect: sum_t c_t <psi|P_t|psi> for Pauli strings, grouped by X mask so that one pass
//            serves every term with the same X mask: P|x> = i^{#Y} (-1)^{popcount(x&z)} |x^xm>.
//
// Accumulation: per-thread partial sums (FP64 for complex128; for complex64 at most 32 FP32
// terms are summed before conversion to FP64), warp-shuffle and shared-memory tree per block,
// then a second single-block kernel sums the per-block partials in a fixed order, so results
// are deterministic for a given launch shape.  The per-block partials live in device scratch
// memory owned by the state.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "qs_internal.h"

namespace qs {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocksMax = 4096;
constexpr int kMaxTermsPerGroup = 256;

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of two doubles; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double &a, double &b)
{
    __shared__ double sa[32], sb[32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sa[w] = a; sb[w] = b; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
    }
}

// Each block handles a contiguous range of amplitudes; thread t of the block reads elements
// t, t + T, ... of that range (coalesced).
template <typename R>
__global__ void __launch_bounds__(kRedThreads) norm2_kernel(const typename Cx<R>::T *__restrict__ a,
                                                            uint64_t N, double *__restrict__ part)
{
    const uint64_t per = (N + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = per * blockIdx.x;
    const uint64_t hi = lo + per < N ? lo + per : N;
    double acc = 0.0;
    if (sizeof(R) == 4) {
        float f = 0.f;
        int cnt = 0;
        for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const auto v = a[i];
            f = fmaf((float)v.x, (float)v.x, f);
            f = fmaf((float)v.y, (float)v.y, f);
            if (++cnt == 32) { acc += (double)f; f = 0.f; cnt = 0; }
        }
        acc += (double)f;
    } else {
        for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const auto v = a[i];
            acc = fma((double)v.x, (double)v.x, acc);
            acc = fma((double)v.y, (double)v.y, acc);
        }
    }
    double dummy = 0.0;
    block_sum2(acc, dummy);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// Sum `count` pairs (re, im) laid out as part[i], part[stride + i]; writes out[0], out[1].
__global__ void __launch_bounds__(kRedThreads) finish_kernel(const double *__restrict__ part, int count,
                                                             int stride, double *__restrict__ out)
{
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        a += part[i];
        if (stride) b += part[stride + i];
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

struct TermGroup {
    uint64_t xm;
    int nterms;
    uint64_t zm[kMaxTermsPerGroup];
    double cre[kMaxTermsPerGroup];  // coeff * Re(i^{#Y})
    double cim[kMaxTermsPerGroup];  // coeff * Im(i^{#Y})
};

// sum_x conj(a[x^xm]) a[x] sum_j c_j i^{ny_j} (-1)^{popc(x & zm_j)}
template <typename R>
__global__ void __launch_bounds__(kRedThreads) expect_kernel(const typename Cx<R>::T *__restrict__ a,
                                                             uint64_t N, const TermGroup *__restrict__ grp,
                                                             double *__restrict__ part)
{
    __shared__ uint64_t zm[kMaxTermsPerGroup];
    __shared__ R cre[kMaxTermsPerGroup], cim[kMaxTermsPerGroup];
    const int nt = grp->nterms;
    const uint64_t xm = grp->xm;
    for (int j = threadIdx.x; j < nt; j += blockDim.x) {
        zm[j] = grp->zm[j];
        cre[j] = (R)grp->cre[j];
        cim[j] = (R)grp->cim[j];
    }
    __syncthreads();
    const uint64_t per = (N + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = per * blockIdx.x;
    const uint64_t hi = lo + per < N ? lo + per : N;
    double accr = 0.0, acci = 0.0;
    R fr = 0, fi = 0;
    int cnt = 0;
    for (uint64_t x = lo + threadIdx.x; x < hi; x += blockDim.x) {
        const auto ax = a[x];
        const auto ay = a[x ^ xm];
        // v = conj(ay) * ax
        const R vr = (R)ay.x * (R)ax.x + (R)ay.y * (R)ax.y;
        const R vi = (R)ay.x * (R)ax.y - (R)ay.y * (R)ax.x;
        R er = 0, ei = 0;
        for (int j = 0; j < nt; ++j) {
            const R s = (__popcll(x & zm[j]) & 1) ? R(-1) : R(1);
            er = fma(s, cre[j], er);
            ei = fma(s, cim[j], ei);
        }
        // (er + i ei) * (vr + i vi)
        fr += er * vr - ei * vi;
        fi += er * vi + ei * vr;
        if (sizeof(R) == 4 && ++cnt == 32) {
            accr += (double)fr;
            acci += (double)fi;
            fr = fi = 0;
            cnt = 0;
        }
    }
    accr += (double)fr;
    acci += (double)fi;
    block_sum2(accr, acci);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = accr;
        part[gridDim.x + blockIdx.x] = acci;
    }
}

// Term parities as a linear map.  For a group of Z strings with the same X mask, the sign of term
// t at index x is (-1)^{p_t(x)} with p_t(x) = popcount(x & zm_t) mod 2, linear over GF(2) in x:
// the parity vector p(x) (one bit per term) is the XOR of the columns col[i] of the bits i set
// in x.  With h(x) = sum_t c_t (-1)^{p_t} = sum_t c_t - 2 sum_{t : p_t = 1} c_t, the second sum
// is read from byte tables: tab[b][v] = sum of c_{8b+k} over the set bits k of v.
constexpr int kParityMaxTerms = 128;
constexpr int kParityBytes = kParityMaxTerms / 8;
struct ParityTables {
    uint32_t col[64][kParityMaxTerms / 32];  // parity columns of the physical bits
    double csum_re, csum_im;                 // sum of all coefficients
    int nbytes;                              // table bytes in use
    int incremental;                         // 1: every walked bit touches at most 4 table bytes
    double tre[kParityBytes][256], tim[kParityBytes][256];
    double cb_re[64], cb_im[64];             // sum of the coefficients of the terms containing bit b
    uint32_t bbytes[64];                     // table bytes those terms occupy (4 x 8 bits, 0xff = none)
};

// Each block owns 2^(8 + klog) consecutive amplitudes; thread t visits lo | (gray(i) << 8) | t for
// i = 0 .. 2^klog - 1, so consecutive visits differ in one index bit b and the parity vector
// changes by one column (one XOR per word); the warp's 32 amplitudes stay contiguous.  Only the
// terms containing b change sign, so h(x) is updated rather than recomputed:
//   h_new = h + 2 C_b - 4 S(p & col_b),
// with C_b the sum of their coefficients and S(.) read from the byte tables over the (at most
// four) bytes where col_b is nonzero.  Every 32 visits h is recomputed from all bytes, which
// bounds the rounding drift of the updates.
// Byte b of a parity vector held in NW registers (selects, no local memory).
template <int NW>
__device__ __forceinline__ uint32_t parity_byte(const uint32_t (&Q)[NW], int b)
{
    uint32_t word = Q[0];
#pragma unroll
    for (int w = 1; w < NW; ++w)
        if ((b >> 2) == w) word = Q[w];
    return (word >> (8 * (b & 3))) & 0xffu;
}

template <typename R, int NW, bool CIM>
__global__ void __launch_bounds__(kRedThreads) expect_parity_kernel(const typename Cx<R>::T *__restrict__ a,
                                                                    uint64_t xm, int klog,
                                                                    const ParityTables *__restrict__ pt,
                                                                    double *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    R *tre = reinterpret_cast<R *>(dyn);
    const int nb = pt->nbytes;
    R *tim = tre + nb * 256;
    __shared__ uint32_t col[64][NW];
    __shared__ R cbr[64], cbi[64];
    __shared__ uint32_t bby[64];
    for (int j = threadIdx.x; j < nb * 256; j += blockDim.x) {
        tre[j] = (R)pt->tre[j >> 8][j & 255];
        if (CIM) tim[j] = (R)pt->tim[j >> 8][j & 255];
    }
    for (int j = threadIdx.x; j < 64 * NW; j += blockDim.x) col[j / NW][j % NW] = pt->col[j / NW][j % NW];
    for (int j = threadIdx.x; j < 64; j += blockDim.x) {
        cbr[j] = (R)pt->cb_re[j];
        cbi[j] = (R)pt->cb_im[j];
        bby[j] = pt->bbytes[j];
    }
    __syncthreads();
    const bool inc = pt->incremental != 0;
    const R cre0 = (R)pt->csum_re, cim0 = (R)pt->csum_im;
    const uint64_t lo = uint64_t(blockIdx.x) << (8 + klog);
    const uint64_t x0 = lo | threadIdx.x;
    uint32_t P[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) P[w] = 0;
    for (int i = 0; i < 64; ++i)
        if (x0 >> i & 1)
#pragma unroll
            for (int w = 0; w < NW; ++w) P[w] ^= col[i][w];
    double accr = 0.0, acci = 0.0;
    R fr = 0, fi = 0, er = 0, ei = 0;
    int cnt = 0;
    const uint32_t K = 1u << klog;
    for (uint32_t i = 0; i < K; ++i) {
        int bit = -1;
        if (i) {
            bit = 8 + __ffs(i) - 1;
#pragma unroll
            for (int w = 0; w < NW; ++w) P[w] ^= col[bit][w];
        }
        if (!inc || (i & 31u) == 0) {
            R sr = 0, si = 0;
            for (int b = 0; b < nb; ++b) {
                const uint32_t v = parity_byte<NW>(P, b);
                sr += tre[b * 256 + v];
                if (CIM) si += tim[b * 256 + v];
            }
            er = cre0 - R(2) * sr;
            ei = CIM ? cim0 - R(2) * si : R(0);
        } else {
            uint32_t M[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) M[w] = P[w] & col[bit][w];
            const uint32_t bl = bby[bit];
            R sr = 0, si = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t b = (bl >> (8 * k)) & 0xffu;
                if (b != 0xffu) {
                    const uint32_t v = parity_byte<NW>(M, int(b));
                    sr += tre[b * 256 + v];
                    if (CIM) si += tim[b * 256 + v];
                }
            }
            er += R(2) * cbr[bit] - R(4) * sr;
            if (CIM) ei += R(2) * cbi[bit] - R(4) * si;
        }
        const uint64_t x = x0 | (uint64_t(i ^ (i >> 1)) << 8);
        const auto ax = a[x];
        const auto ay = a[x ^ xm];
        const R vr = (R)ay.x * (R)ax.x + (R)ay.y * (R)ax.y;
        const R vi = (R)ay.x * (R)ax.y - (R)ay.y * (R)ax.x;
        fr += er * vr - ei * vi;
        fi += er * vi + ei * vr;
        if (sizeof(R) == 4 && ++cnt == 32) {
            accr += (double)fr;
            acci += (double)fi;
            fr = fi = 0;
            cnt = 0;
        }
    }
    accr += (double)fr;
    acci += (double)fi;
    block_sum2(accr, acci);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = accr;
        part[gridDim.x + blockIdx.x] = acci;
    }
}

// Marginal probabilities: hist[m] += |a_x|^2 with m gathered from the bits pos[0..nq).
template <typename R>
__global__ void __launch_bounds__(kRedThreads) probs_kernel(const typename Cx<R>::T *__restrict__ a,
                                                            uint64_t N, int nq, uint4 pos_packed0,
                                                            uint4 pos_packed1,
                                                            double *__restrict__ hist)
{
    extern __shared__ double sh[];
    const int M = 1 << nq;
    const bool use_smem = nq <= 11;
    if (use_smem)
        for (int m = threadIdx.x; m < M; m += blockDim.x) sh[m] = 0.0;
    __syncthreads();
    uint8_t pos[32];
    const uint32_t w[8] = {pos_packed0.x, pos_packed0.y, pos_packed0.z, pos_packed0.w,
                           pos_packed1.x, pos_packed1.y, pos_packed1.z, pos_packed1.w};
#pragma unroll
    for (int j = 0; j < 32; ++j) pos[j] = (w[j >> 2] >> (8 * (j & 3))) & 0xff;
    const uint64_t per = (N + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = per * blockIdx.x;
    const uint64_t hi = lo + per < N ? lo + per : N;
    for (uint64_t x = lo + threadIdx.x; x < hi; x += blockDim.x) {
        const auto v = a[x];
        const double p = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        uint32_t m = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j)  // unrolled so that pos[] stays in registers
            if (j < nq) m |= uint32_t((x >> pos[j]) & 1) << j;
        if (use_smem) atomicAdd(&sh[m], p);
        else atomicAdd(&hist[m], p);
    }
    if (use_smem) {
        __syncthreads();
        for (int m = threadIdx.x; m < M; m += blockDim.x)
            if (sh[m] != 0.0) atomicAdd(&hist[m], sh[m]);
    }
}

// Marginals over at most Q qubits (2^Q bins): each thread keeps its bins in registers
// (branch-free select-and-add per bin), then the bins are reduced with warp shuffles and added
// to the global histogram with one FP64 atomic per warp and bin.
template <typename R, int Q>
__global__ void __launch_bounds__(kRedThreads) probs_small_kernel(const typename Cx<R>::T *__restrict__ a,
                                                                  uint64_t N, int nq, uint4 pos_packed0,
                                                                  double *__restrict__ hist)
{
    constexpr int M = 1 << Q;
    uint32_t pos[Q];
    const uint32_t w[4] = {pos_packed0.x, pos_packed0.y, pos_packed0.z, pos_packed0.w};
#pragma unroll
    for (int j = 0; j < Q; ++j) pos[j] = (w[j >> 2] >> (8 * (j & 3))) & 0xff;
    // complex64: FP32 partial sums of at most 32 amplitudes per bin, then FP64 (the FP64 pipe
    // is 1/64 of the FP32 rate on this part); complex128: FP64 throughout
    double acc[M];
    R part[M];
#pragma unroll
    for (int b = 0; b < M; ++b) {
        acc[b] = 0.0;
        part[b] = R(0);
    }
    int cnt = 0;
    const uint64_t per = (N + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = per * blockIdx.x;
    const uint64_t hi = lo + per < N ? lo + per : N;
    for (uint64_t x = lo + threadIdx.x; x < hi; x += blockDim.x) {
        const auto v = a[x];
        const R p = (R)v.x * (R)v.x + (R)v.y * (R)v.y;
        uint32_t m = 0;
#pragma unroll
        for (int j = 0; j < Q; ++j)
            if (j < nq) m |= uint32_t((x >> pos[j]) & 1) << j;
        if (sizeof(R) == 8) {
#pragma unroll
            for (int b = 0; b < M; ++b) acc[b] += (m == uint32_t(b)) ? (double)p : 0.0;
        } else {
#pragma unroll
            for (int b = 0; b < M; ++b) part[b] += (m == uint32_t(b)) ? p : R(0);
            if (++cnt == 32) {
#pragma unroll
                for (int b = 0; b < M; ++b) {
                    acc[b] += (double)part[b];
                    part[b] = R(0);
                }
                cnt = 0;
            }
        }
    }
#pragma unroll
    for (int b = 0; b < M; ++b) acc[b] += (double)part[b];
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int b = 0; b < M; ++b) {
        const double t = warp_sum(acc[b]);
        if (lane == 0 && b < (1 << nq) && t != 0.0) atomicAdd(&hist[b], t);
    }
}

int g_sms = 0;
int reduce_blocks(uint64_t N)
{
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    uint64_t b = uint64_t(g_sms) * 8;
    if (b > kRedBlocksMax) b = kRedBlocksMax;
    const uint64_t need = (N + kRedThreads - 1) / kRedThreads;
    if (b > need) b = need;
    return b < 1 ? 1 : (int)b;
}

int cuda_fail(const char *what, char *err, size_t errlen)
{
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return QS_OK;
    snprintf(err, errlen, "%s: %s", what, cudaGetErrorString(e));
    return QS_ECUDA;
}

}  // namespace

size_t reduce_scratch_bytes()
{
    // partials (2 x blocks) + 2 results + one term group + its parity tables
    return sizeof(double) * (2 * kRedBlocksMax + 8) + sizeof(TermGroup) + 256 + sizeof(ParityTables) + 256;
}

int launch_norm2(const LaunchCtx &c, double *d_scratch, double *h_out, char *err, size_t errlen)
{
    const uint64_t N = 1ull << c.n;
    const int blocks = reduce_blocks(N);
    cudaStream_t st = (cudaStream_t)c.stream;
    double *part = d_scratch, *res = d_scratch + 2 * kRedBlocksMax;
    if (c.dt == QS_C64)
        norm2_kernel<float><<<blocks, kRedThreads, 0, st>>>((const float2 *)c.amp, N, part);
    else
        norm2_kernel<double><<<blocks, kRedThreads, 0, st>>>((const double2 *)c.amp, N, part);
    finish_kernel<<<1, kRedThreads, 0, st>>>(part, blocks, 0, res);
    int rc = cuda_fail("norm2 launch", err, errlen);
    if (rc) return rc;
    double r[2];
    if (cudaMemcpyAsync(r, res, sizeof(r), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_fail("norm2 readback", err, errlen);
    *h_out = r[0];
    return QS_OK;
}

int launch_probs(const LaunchCtx &c, const int *phys_q, int nq, double *d_scratch,
                 size_t scratch_bytes, double *h_out, char *err, size_t errlen)
{
    const uint64_t N = 1ull << c.n;
    const size_t M = size_t(1) << nq;
    if (M * sizeof(double) > scratch_bytes) {
        snprintf(err, errlen, "probs: scratch too small");
        return QS_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)c.stream;
    uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < nq; ++j) w[j >> 2] |= uint32_t(phys_q[j] & 0xff) << (8 * (j & 3));
    uint4 p0 = make_uint4(w[0], w[1], w[2], w[3]), p1 = make_uint4(w[4], w[5], w[6], w[7]);
    if (cudaMemsetAsync(d_scratch, 0, M * sizeof(double), st) != cudaSuccess)
        return cuda_fail("probs memset", err, errlen);
    const int blocks = reduce_blocks(N);
    const size_t smem = nq <= 11 ? M * sizeof(double) : 0;
    if (nq <= 3) {
        if (c.dt == QS_C64)
            probs_small_kernel<float, 3><<<blocks, kRedThreads, 0, st>>>((const float2 *)c.amp, N, nq, p0, d_scratch);
        else
            probs_small_kernel<double, 3><<<blocks, kRedThreads, 0, st>>>((const double2 *)c.amp, N, nq, p0, d_scratch);
    } else if (nq <= 5) {
        if (c.dt == QS_C64)
            probs_small_kernel<float, 5><<<blocks, kRedThreads, 0, st>>>((const float2 *)c.amp, N, nq, p0, d_scratch);
        else
            probs_small_kernel<double, 5><<<blocks, kRedThreads, 0, st>>>((const double2 *)c.amp, N, nq, p0, d_scratch);
    } else if (c.dt == QS_C64) {
        probs_kernel<float><<<blocks, kRedThreads, smem, st>>>((const float2 *)c.amp, N, nq, p0, p1,
                                                               d_scratch);
    } else {
        probs_kernel<double><<<blocks, kRedThreads, smem, st>>>((const double2 *)c.amp, N, nq, p0,
                                                                p1, d_scratch);
    }
    int rc = cuda_fail("probs launch", err, errlen);
    if (rc) return rc;
    if (cudaMemcpyAsync(h_out, d_scratch, M * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_fail("probs readback", err, errlen);
    return QS_OK;
}

namespace {

template <typename R, int NW, bool CIM>
void launch_parity_t(const typename Cx<R>::T *a, uint64_t xm, int klog, const ParityTables *pt, double *part,
                     int nblk, size_t dsm, cudaStream_t st)
{
    static int attr_dev = -1;  // tables of up to 16 bytes x 256 x 2 doubles = 64 KiB
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaFuncSetAttribute(expect_parity_kernel<R, NW, CIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kParityBytes * 256 * 2 * int(sizeof(double)));
        attr_dev = dev;
    }
    expect_parity_kernel<R, NW, CIM><<<nblk, kRedThreads, dsm, st>>>(a, xm, klog, pt, part);
}

template <typename R>
int launch_parity(const typename Cx<R>::T *a, uint64_t xm, int klog, const ParityTables *pt, double *part, int nblk,
                  size_t dsm, int nw, bool cim, cudaStream_t st)
{
    if (nw == 1) {
        if (cim) launch_parity_t<R, 1, true>(a, xm, klog, pt, part, nblk, dsm, st);
        else launch_parity_t<R, 1, false>(a, xm, klog, pt, part, nblk, dsm, st);
    } else if (nw == 2) {
        if (cim) launch_parity_t<R, 2, true>(a, xm, klog, pt, part, nblk, dsm, st);
        else launch_parity_t<R, 2, false>(a, xm, klog, pt, part, nblk, dsm, st);
    } else {
        if (cim) launch_parity_t<R, 4, true>(a, xm, klog, pt, part, nblk, dsm, st);
        else launch_parity_t<R, 4, false>(a, xm, klog, pt, part, nblk, dsm, st);
    }
    return QS_OK;
}

}  // namespace

int launch_expect(const LaunchCtx &c, const uint64_t *xm, const uint64_t *zm, const double *coeff,
                  size_t nterms, double *d_scratch, size_t scratch_bytes, double *h_out, char *err,
                  size_t errlen)
{
    (void)scratch_bytes;
    const uint64_t N = 1ull << c.n;
    cudaStream_t st = (cudaStream_t)c.stream;
    double *part = d_scratch, *res = d_scratch + 2 * kRedBlocksMax;
    TermGroup *dgrp = reinterpret_cast<TermGroup *>(d_scratch + 2 * kRedBlocksMax + 8);
    const int blocks = reduce_blocks(N);
    std::vector<TermGroup> hgv(1);  // host staging; each copy completes before reuse
    TermGroup &hg = hgv[0];
    std::vector<ParityTables> hpt(1);
    ParityTables *dpt = reinterpret_cast<ParityTables *>(
        (reinterpret_cast<uintptr_t>(dgrp) + sizeof(TermGroup) + 255) & ~uintptr_t(255));
    double tot_r = 0.0, tot_i = 0.0;
    std::vector<char> done(nterms, 0);
    for (size_t i = 0; i < nterms; ++i) {
        if (done[i]) continue;
        // gather all not-yet-done terms with this X mask (up to the group capacity)
        hg.xm = xm[i];
        hg.nterms = 0;
        for (size_t j = i; j < nterms && hg.nterms < kMaxTermsPerGroup; ++j) {
            if (done[j] || xm[j] != xm[i]) continue;
            done[j] = 1;
            const int ny = __builtin_popcountll(xm[j] & zm[j]) & 3;
            static const double pr[4] = {1, 0, -1, 0}, pi[4] = {0, 1, 0, -1};
            hg.zm[hg.nterms] = zm[j];
            hg.cre[hg.nterms] = coeff[j] * pr[ny];
            hg.cim[hg.nterms] = coeff[j] * pi[ny];
            hg.nterms++;
        }
        int nblk = blocks;
        int rc_launch = QS_OK;
        if (hg.nterms >= 8 && hg.nterms <= kParityMaxTerms && c.n >= 16) {
            // parity tables (host, FP64), then the Gray-walk kernel
            ParityTables &pt = hpt[0];
            std::memset(&pt, 0, sizeof pt);
            pt.nbytes = (hg.nterms + 7) / 8;
            for (int t = 0; t < hg.nterms; ++t) {
                pt.csum_re += hg.cre[t];
                pt.csum_im += hg.cim[t];
                for (int i = 0; i < 64; ++i)
                    if (hg.zm[t] >> i & 1) pt.col[i][t >> 5] |= 1u << (t & 31);
            }
            for (int b = 0; b < pt.nbytes; ++b)
                for (int v = 0; v < 256; ++v)
                    for (int k = 0; k < 8; ++k) {
                        const int t = 8 * b + k;
                        if ((v >> k & 1) && t < hg.nterms) {
                            pt.tre[b][v] += hg.cre[t];
                            pt.tim[b][v] += hg.cim[t];
                        }
                    }
            // per bit: the coefficient sum of the terms containing it and the table bytes they use
            bool cim = false;
            for (int t = 0; t < hg.nterms; ++t) cim = cim || hg.cim[t] != 0.0;
            pt.incremental = 1;
            for (int i = 0; i < 64; ++i) {
                uint32_t list = 0xffffffffu;
                int nbk = 0;
                for (int t = 0; t < hg.nterms; ++t)
                    if (hg.zm[t] >> i & 1) {
                        pt.cb_re[i] += hg.cre[t];
                        pt.cb_im[i] += hg.cim[t];
                    }
                for (int b = 0; b < pt.nbytes; ++b)
                    if ((pt.col[i][b >> 2] >> (8 * (b & 3))) & 0xffu) {
                        if (nbk < 4) list = (list & ~(0xffu << (8 * nbk))) | (uint32_t(b) << (8 * nbk));
                        ++nbk;
                    }
                if (nbk > 4) pt.incremental = 0;
                pt.bbytes[i] = list;
            }
            if (cudaMemcpyAsync(dpt, &pt, sizeof pt, cudaMemcpyHostToDevice, st) != cudaSuccess)
                return cuda_fail("expect upload", err, errlen);
            const int blog = std::min(12, c.n - 12);
            nblk = 1 << blog;
            const int klog = c.n - blog - 8;
            const size_t dsm = size_t(pt.nbytes) * 256 * 2 * (c.dt == QS_C64 ? sizeof(float) : sizeof(double));
            const int nw = hg.nterms <= 32 ? 1 : hg.nterms <= 64 ? 2 : 4;
            if (c.dt == QS_C64)
                rc_launch = launch_parity<float>((const float2 *)c.amp, hg.xm, klog, dpt, part, nblk, dsm, nw, cim, st);
            else
                rc_launch = launch_parity<double>((const double2 *)c.amp, hg.xm, klog, dpt, part, nblk, dsm, nw, cim, st);
        } else {
            if (cudaMemcpyAsync(dgrp, &hg, sizeof(TermGroup), cudaMemcpyHostToDevice, st) != cudaSuccess)
                return cuda_fail("expect upload", err, errlen);
            if (c.dt == QS_C64)
                expect_kernel<float><<<blocks, kRedThreads, 0, st>>>((const float2 *)c.amp, N, dgrp, part);
            else
                expect_kernel<double><<<blocks, kRedThreads, 0, st>>>((const double2 *)c.amp, N, dgrp,
                                                                      part);
        }
        finish_kernel<<<1, kRedThreads, 0, st>>>(part, nblk, nblk, res);
        int rc = cuda_fail("expect launch", err, errlen);
        if (rc) return rc;
        double r[2];
        if (cudaMemcpyAsync(r, res, sizeof(r), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return cuda_fail("expect readback", err, errlen);
        tot_r += r[0];
        tot_i += r[1];
    }
    h_out[0] = tot_r;
    h_out[1] = tot_i;
    return QS_OK;
}

// ------------------------------------------------------------------ allocation-free probs
// Fixed scratch for qs_probs_noalloc: one histogram of at most 2^kStaticProbsMaxQubits doubles
// (128 KiB).  It is a file-scope device array, so every GPU that loads the library holds it
// until the process exits.  Host code must not pass `g_static_probs_hist` itself to a kernel:
// on the host that name is only a stand-in symbol, not a device address.  Its device address
// is looked up once per device with cudaGetSymbolAddress (static_probs_scratch below).
namespace {

__device__ __align__(256) double g_static_probs_hist[1 << kStaticProbsMaxQubits];

constexpr int kMaxDevices = 64;
double *g_static_probs_ptr[kMaxDevices] = {nullptr};
std::mutex g_static_probs_mu;

// Device address of the fixed histogram on the current device (set up on first use).
int static_probs_scratch(double **out, char *err, size_t errlen)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        snprintf(err, errlen, "probs_noalloc: no usable current device (%s)",
                 e != cudaSuccess ? cudaGetErrorString(e) : "device index out of range");
        return QS_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_static_probs_mu);
    if (!g_static_probs_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_probs_hist);
        if (e != cudaSuccess || !p) {
            snprintf(err, errlen, "probs_noalloc: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
            cudaGetLastError();
            return QS_ECUDA;
        }
        g_static_probs_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_static_probs_ptr[dev];
    return QS_OK;
}

}  // namespace

int launch_probs_static(const LaunchCtx &c, const int *phys_q, int nq, double *h_out, char *err,
                        size_t errlen)
{
    if (nq < 0 || nq > kStaticProbsMaxQubits) {
        snprintf(err, errlen, "probs_noalloc: nq = %d exceeds the fixed scratch of 2^%d bins", nq,
                 kStaticProbsMaxQubits);
        return QS_EINVAL;
    }
    double *hist = nullptr;
    int rc = static_probs_scratch(&hist, err, errlen);
    if (rc) return rc;
    const uint64_t N = 1ull << c.n;
    const size_t M = size_t(1) << nq;
    cudaStream_t st = (cudaStream_t)c.stream;
    uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < nq; ++j) w[j >> 2] |= uint32_t(phys_q[j] & 0xff) << (8 * (j & 3));
    uint4 p0 = make_uint4(w[0], w[1], w[2], w[3]), p1 = make_uint4(w[4], w[5], w[6], w[7]);
    // the array keeps the previous call's histogram: clear the bins this call accumulates into
    if (cudaMemsetAsync(hist, 0, M * sizeof(double), st) != cudaSuccess)
        return cuda_fail("probs_noalloc memset", err, errlen);
    const int blocks = reduce_blocks(N);
    const size_t smem = nq <= 11 ? M * sizeof(double) : 0;
    if (c.dt == QS_C64)
        probs_kernel<float><<<blocks, kRedThreads, smem, st>>>((const float2 *)c.amp, N, nq, p0, p1,
                                                               hist);
    else
        probs_kernel<double><<<blocks, kRedThreads, smem, st>>>((const double2 *)c.amp, N, nq, p0,
                                                                p1, hist);
    rc = cuda_fail("probs_noalloc launch", err, errlen);
    if (rc) return rc;
    if (cudaMemcpyAsync(h_out, hist, M * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_fail("probs_noalloc readback", err, errlen);
    return QS_OK;
}

__global__ void set_one_kernel(void *amp, uint64_t x, int is64)
{
    if (is64) reinterpret_cast<float2 *>(amp)[x] = make_float2(1.f, 0.f);
    else reinterpret_cast<double2 *>(amp)[x] = make_double2(1.0, 0.0);
}

int launch_set_basis(const LaunchCtx &c, uint64_t x, char *err, size_t errlen)
{
    cudaStream_t st = (cudaStream_t)c.stream;
    const size_t bytes = (size_t(1) << c.n) * (c.dt == QS_C64 ? 8 : 16);
    if (cudaMemsetAsync(c.amp, 0, bytes, st) != cudaSuccess)
        return cuda_fail("set_basis memset", err, errlen);
    set_one_kernel<<<1, 1, 0, st>>>(c.amp, x, c.dt == QS_C64 ? 1 : 0);
    return cuda_fail("set_basis launch", err, errlen);
}

}  // namespace qs
