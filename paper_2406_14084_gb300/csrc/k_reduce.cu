// k_reduce.cu -- readout reductions over the state vector (one read pass each).
//
//  * norm2:  sum |a_x|^2
//  * probs:  marginal probabilities over a set of physical bit positions
//  * expect: sum_t c_t <psi|P_t|psi> for Pauli strings, grouped by X mask so that one pass
//            serves every term with the same X mask: P|x> = i^{#Y} (-1)^{popcount(x&z)} |x^xm>.
//            Groups of four or more terms go through 1024-amplitude Walsh-Hadamard tiles, so
//            the pass costs the same whatever the number of terms; smaller groups loop over
//            their terms per amplitude.
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
// t, t + T, ... of that range (coalesced), kUnroll independent loads at a time.
constexpr int kUnroll = 8;
template <typename R>
__global__ void __launch_bounds__(kRedThreads) norm2_kernel(const typename Cx<R>::T *__restrict__ a,
                                                            uint64_t N, double *__restrict__ part)
{
    using T = typename Cx<R>::T;
    const uint64_t per = (N + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = per * blockIdx.x;
    const uint64_t hi = lo + per < N ? lo + per : N;
    double acc = 0.0;
    for (uint64_t x0 = lo + threadIdx.x; x0 < hi; x0 += uint64_t(kUnroll) * blockDim.x) {
        T v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint64_t x = x0 + uint64_t(u) * blockDim.x;
            v[u] = x < hi ? a[x] : T{};
        }
        // complex64: the kUnroll squares are summed in FP32, then added in FP64
        R f = 0;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            f = fma(v[u].x, v[u].x, f);
            f = fma(v[u].y, v[u].y, f);
        }
        acc += (double)f;
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

// Walsh-Hadamard form of one X-mask group.  Write an index as x = (H, L) with L its low 10 bits
// and split each Z mask the same way, z_t = (zh_t, zl_t).  With v(x) = conj(a[x^xm]) a[x],
//   sum_x v(x) sum_t C_t (-1)^{popc(x & z_t)} = sum_H sum_t C_t s_t(H) Vhat_H(zl_t),
// where s_t(H) = (-1)^{popc(H & zh_t)} and Vhat_H is the Walsh-Hadamard transform of v(H, .)
// over the 1024 values of L.  One warp transforms one tile (10 butterfly stages: the bits held
// in a lane's 32 registers, then the five lane bits through shuffles), writes Vhat to shared
// memory and then spends one lookup per term, so the per-amplitude work no longer grows with
// the number of terms.
//   When xm has a bit p >= 10, the tiles with bit p of the index clear are paired with their
// partners H ^ (xm >> 10): the partner's v is conj(v) and its term signs are those of x times
// (-1)^{popc(xm & z_t)}, so one tile pass covers both and every amplitude is read once.  The
// host folds both into four real coefficients per term: re += A Vr + B Vi, im += C Vi + D Vr.
constexpr int kWhtTileLog = 10;
struct WhtTerms {
    uint64_t xm;
    int nterms;
    int pair;
    uint64_t zh[kMaxTermsPerGroup];
    uint32_t zl[kMaxTermsPerGroup];
    double q[4][kMaxTermsPerGroup];
};

// Asks the L2 to fetch [p, p + bytes) (p 16-byte aligned, bytes a multiple of 16); nothing is
// written to the SM and nothing waits for it.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(bytes)
                 : "memory");
}

template <typename R, bool CPLX>
__global__ void __launch_bounds__(kRedThreads) expect_wht_kernel(const typename Cx<R>::T *__restrict__ a, int n,
                                                                 const WhtTerms *__restrict__ wt,
                                                                 double *__restrict__ part)
{
    using T = typename Cx<R>::T;
    constexpr int VL = sizeof(T) == 8 ? 1 : 0;  // complex64: two amplitudes per 16-byte load
    constexpr int NV = 32 >> VL;                // vector loads per lane per tile
    extern __shared__ __align__(16) unsigned char dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    R *wr = reinterpret_cast<R *>(dyn) + (warp << kWhtTileLog) * (CPLX ? 2 : 1);
    R *wi = wr + (1 << kWhtTileLog);
    __shared__ uint64_t zh[kMaxTermsPerGroup];
    __shared__ uint32_t zl[kMaxTermsPerGroup];
    __shared__ R q[4][kMaxTermsPerGroup];
    const int nt = wt->nterms;
    for (int j = threadIdx.x; j < nt; j += blockDim.x) {
        zh[j] = wt->zh[j];
        zl[j] = wt->zl[j];
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k][j] = (R)wt->q[k][j];
    }
    __syncthreads();
    const uint64_t xm = wt->xm, xmh = xm >> kWhtTileLog;
    const uint32_t xml = uint32_t(xm) & ((1u << kWhtTileLog) - 1);
    const bool pair = wt->pair != 0;
    const int p = pair ? 63 - __clzll((long long)xmh) : 0;
    const uint64_t ntiles = 1ull << (n - kWhtTileLog - (pair ? 1 : 0));
    const uint64_t nwarps = uint64_t(gridDim.x) * (blockDim.x >> 5);
    double accr = 0.0, acci = 0.0;
    R fr = 0, fi = 0;
    int cnt = 0;
    for (uint64_t tile = uint64_t(blockIdx.x) * (blockDim.x >> 5) + warp; tile < ntiles; tile += nwarps) {
        const uint64_t H = pair ? ((tile >> p) << (p + 1)) | (tile & ((1ull << p) - 1)) : tile;
        const T *at = a + (H << kWhtTileLog);
        const T *ap = a + ((H ^ xmh) << kWhtTileLog);
        // the warp's next tile moves into L2 while this one is transformed (paired tiles already
        // keep two tiles of loads in flight and ran slower with it: 1.34 -> 1.69 ms at 30 qubits)
        if (!pair && lane == 0 && tile + nwarps < ntiles)
            prefetch_l2_bulk(a + ((tile + nwarps) << kWhtTileLog), uint32_t(sizeof(T)) << kWhtTileLog);
        // element j of the lane sits at L = (j & VL) | lane << VL | (j >> VL) << (5 + VL)
        R vr[32], vi[32];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const uint32_t L0 = (uint32_t(lane) << VL) | (uint32_t(k) << (5 + VL));
            if constexpr (VL != 0) {
                const float4 x = *reinterpret_cast<const float4 *>(at + L0);
                if constexpr (CPLX) {
                    const uint32_t Lp = (L0 ^ xml) & ~1u;
                    float4 y = *reinterpret_cast<const float4 *>(ap + Lp);
                    if (xml & 1u) y = make_float4(y.z, y.w, y.x, y.y);
                    vr[2 * k] = (R)(y.x * x.x + y.y * x.y);
                    vi[2 * k] = (R)(y.x * x.y - y.y * x.x);
                    vr[2 * k + 1] = (R)(y.z * x.z + y.w * x.w);
                    vi[2 * k + 1] = (R)(y.z * x.w - y.w * x.z);
                } else {
                    vr[2 * k] = (R)(x.x * x.x + x.y * x.y);
                    vr[2 * k + 1] = (R)(x.z * x.z + x.w * x.w);
                }
            } else {
                const T x = at[L0];
                if (CPLX) {
                    const T y = ap[L0 ^ xml];
                    vr[k] = (R)(y.x * x.x + y.y * x.y);
                    vi[k] = (R)(y.x * x.y - y.y * x.x);
                } else {
                    vr[k] = (R)(x.x * x.x + x.y * x.y);
                }
            }
        }
        // butterflies over the five register bits ...
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (!(j >> s & 1)) {
                    const int k = j | (1 << s);
                    const R r0 = vr[j], r1 = vr[k];
                    vr[j] = r0 + r1;
                    vr[k] = r0 - r1;
                    if (CPLX) {
                        const R i0 = vi[j], i1 = vi[k];
                        vi[j] = i0 + i1;
                        vi[k] = i0 - i1;
                    }
                }
        // ... and over the five lane bits (the lane with the bit set keeps the difference)
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const R sg = (lane >> s & 1) ? R(-1) : R(1);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                vr[j] = fma(sg, vr[j], __shfl_xor_sync(0xffffffffu, vr[j], 1 << s));
                if (CPLX) vi[j] = fma(sg, vi[j], __shfl_xor_sync(0xffffffffu, vi[j], 1 << s));
            }
        }
        // Vhat(m) sits where v(L = m) was
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const uint32_t L0 = (uint32_t(lane) << VL) | (uint32_t(k) << (5 + VL));
            if constexpr (VL != 0) {
                *reinterpret_cast<float2 *>(wr + L0) = make_float2((float)vr[2 * k], (float)vr[2 * k + 1]);
                if (CPLX) *reinterpret_cast<float2 *>(wi + L0) = make_float2((float)vi[2 * k], (float)vi[2 * k + 1]);
            } else {
                wr[L0] = vr[k];
                if (CPLX) wi[L0] = vi[k];
            }
        }
        __syncwarp();
        for (int t = lane; t < nt; t += 32) {
            const uint32_t m = zl[t];
            const R s = (__popcll(H & zh[t]) & 1) ? R(-1) : R(1);
            const R Vr = wr[m];
            if (CPLX) {
                const R Vi = wi[m];
                fr = fma(s, fma(q[0][t], Vr, q[1][t] * Vi), fr);
                fi = fma(s, fma(q[2][t], Vi, q[3][t] * Vr), fi);
            } else {
                fr = fma(s * q[0][t], Vr, fr);
            }
        }
        __syncwarp();
        if (sizeof(R) == 4 && ++cnt == 8) {
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
    // is 1/64 of the FP32 rate on this part); with at most 8 bins, 32 of those partials are first
    // summed in FP32 (converting every one kept the FP64 pipe 40 % busy on 3-qubit marginals;
    // 32 bins would not fit the second level in registers); complex128: FP64 throughout
    constexpr bool kTwoLevel = M <= 8;
    double acc[M];
    R part[M], part2[M];
#pragma unroll
    for (int b = 0; b < M; ++b) {
        acc[b] = 0.0;
        part[b] = part2[b] = R(0);
    }
    int cnt = 0, cnt2 = 0;
    const uint64_t per = (N + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = per * blockIdx.x;
    const uint64_t hi = lo + per < N ? lo + per : N;
    constexpr int U = 4;  // independent loads in flight per thread
    using T = typename Cx<R>::T;
    for (uint64_t x0 = lo + threadIdx.x; x0 < hi; x0 += uint64_t(U) * blockDim.x) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t x = x0 + uint64_t(u) * blockDim.x;
            v[u] = x < hi ? a[x] : T{};  // past the range: weight 0
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t x = x0 + uint64_t(u) * blockDim.x;
            const R p = (R)v[u].x * (R)v[u].x + (R)v[u].y * (R)v[u].y;
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
            }
        }
        if (sizeof(R) == 4 && (cnt += U) >= 32) {
#pragma unroll
            for (int b = 0; b < M; ++b) {
                part2[b] += part[b];
                part[b] = R(0);
            }
            cnt = 0;
            if (!kTwoLevel || ++cnt2 == 32) {
#pragma unroll
                for (int b = 0; b < M; ++b) {
                    acc[b] += (double)part2[b];
                    part2[b] = R(0);
                }
                cnt2 = 0;
            }
        }
    }
#pragma unroll
    for (int b = 0; b < M; ++b) acc[b] += (double)part[b] + (double)part2[b];
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
    // partials (2 x blocks) + 2 results + one term group + its Walsh-Hadamard term table
    return sizeof(double) * (2 * kRedBlocksMax + 8) + sizeof(TermGroup) + 256 + sizeof(WhtTerms) + 256;
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

template <typename R, bool CPLX>
int launch_wht_t(const typename Cx<R>::T *a, int n, const WhtTerms *wt, uint64_t ntiles, double *part,
                 cudaStream_t st)
{
    const size_t dsm = (size_t(kRedThreads / 32) << kWhtTileLog) * sizeof(R) * (CPLX ? 2 : 1);
    static int attr_dev = -1, per_sm = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaFuncSetAttribute(expect_wht_kernel<R, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(dsm));
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, expect_wht_kernel<R, CPLX>, kRedThreads, dsm) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        attr_dev = dev;
    }
    reduce_blocks(1);  // reads the SM count once
    uint64_t nb = uint64_t(g_sms) * uint64_t(per_sm);
    const uint64_t need = std::max<uint64_t>(1, ntiles / (kRedThreads / 32));
    nb = std::min<uint64_t>(std::min<uint64_t>(nb, need), kRedBlocksMax);
    expect_wht_kernel<R, CPLX><<<int(nb), kRedThreads, dsm, st>>>(a, n, wt, part);
    return int(nb);
}

template <typename R>
int launch_wht(const typename Cx<R>::T *a, int n, const WhtTerms *wt, bool cplx, uint64_t ntiles, double *part,
               cudaStream_t st)
{
    return cplx ? launch_wht_t<R, true>(a, n, wt, ntiles, part, st)
                : launch_wht_t<R, false>(a, n, wt, ntiles, part, st);
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
    std::vector<WhtTerms> hw(1);
    WhtTerms *dpt = reinterpret_cast<WhtTerms *>(
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
        if (hg.nterms >= 4 && c.n >= 16) {
            // Walsh-Hadamard tiles; coefficients folded on the host in FP64
            WhtTerms &w = hw[0];
            w.xm = hg.xm;
            w.nterms = hg.nterms;
            w.pair = (hg.xm >> kWhtTileLog) != 0;
            for (int t = 0; t < hg.nterms; ++t) {
                w.zh[t] = hg.zm[t] >> kWhtTileLog;
                w.zl[t] = uint32_t(hg.zm[t]) & ((1u << kWhtTileLog) - 1);
                const double cr = hg.cre[t], ci = hg.cim[t];
                // partner tile: coefficient times (-1)^{popc(xm & z)}; none without pairing
                const double sg = (__builtin_popcountll(hg.xm & hg.zm[t]) & 1) ? -1.0 : 1.0;
                const double pr = w.pair ? sg * cr : 0.0, pi = w.pair ? sg * ci : 0.0;
                w.q[0][t] = cr + pr;
                w.q[1][t] = pi - ci;
                w.q[2][t] = cr - pr;
                w.q[3][t] = ci + pi;
            }
            if (cudaMemcpyAsync(dpt, &w, sizeof w, cudaMemcpyHostToDevice, st) != cudaSuccess)
                return cuda_fail("expect upload", err, errlen);
            const WhtTerms *dw = dpt;
            const uint64_t ntiles = 1ull << (c.n - kWhtTileLog - w.pair);
            const bool cplx = hg.xm != 0;
            if (c.dt == QS_C64)
                nblk = launch_wht<float>((const float2 *)c.amp, c.n, dw, cplx, ntiles, part, st);
            else
                nblk = launch_wht<double>((const double2 *)c.amp, c.n, dw, cplx, ntiles, part, st);
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
