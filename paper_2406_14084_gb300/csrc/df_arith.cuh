// df_arith.cuh -- double-float arithmetic for the complex128 register stages (optional mode).
//
// GB300 executes FP64 FMAs at about 1/64 of the FP32 rate, so complex128 passes are bound by the
// FP64 pipe.  In this mode a slab of complex128 amplitudes is converted once per pass into
// double-float pairs (value = h + l with two FP32 numbers, about 48 significant bits) and the
// register-stage gates run on the FP32 pipe:
//   two-sum    s + e = a + b exactly              (Knuth: 6 FP32 additions)
//   two-prod   p + e = a * b exactly              (one multiply, one FMA)
//   product and sum of pairs keep the error terms of the high parts and the first-order cross
//   terms and renormalise with a fast two-sum (Dekker), so each operation has a relative error
//   of a few units of 2^-48.
// The state stays complex128 in HBM: the conversions are exact bit manipulations (no FP64
// conversion instructions, which run at the FP64 rate) plus one FP64 addition per real part on
// the way back.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace qs {
namespace {

struct df {
    float h, l;
    df() = default;
    __device__ __forceinline__ df(float a) : h(a), l(0.f) {}
    __device__ __forceinline__ df(float a, float b) : h(a), l(b) {}
};

struct dfc {
    df x, y;
};

__device__ __forceinline__ df df_two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return df(s, (a - (s - bb)) + (b - bb));
}

// |a| >= |b| (or a = 0): s + e = a + b exactly
__device__ __forceinline__ df df_fast_two_sum(float a, float b)
{
    const float s = a + b;
    return df(s, b - (s - a));
}

__device__ __forceinline__ df operator-(df a) { return df(-a.h, -a.l); }

__device__ __forceinline__ df operator+(df a, df b)
{
    const df s = df_two_sum(a.h, b.h);
    return df_fast_two_sum(s.h, s.l + (a.l + b.l));
}

__device__ __forceinline__ df operator*(df a, df b)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df operator*=(df &a, df b) { return a = a * b; }

// a * b + c
__device__ __forceinline__ df fma(df a, df b, df c)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const df s = df_two_sum(p, c.h);
    return df_fast_two_sum(s.h, s.l + (e + c.l));
}

__device__ __forceinline__ bool operator==(df a, float b) { return a.h == b && a.l == 0.f; }

// s * b + a, s * b - a and s * b on both parts of a complex pair with a real scalar s
__device__ __forceinline__ dfc rfma(df s, dfc b, dfc a) { return dfc{fma(s, b.x, a.x), fma(s, b.y, a.y)}; }
__device__ __forceinline__ dfc rfms(df s, dfc b, dfc a) { return dfc{fma(s, b.x, -a.x), fma(s, b.y, -a.y)}; }
__device__ __forceinline__ dfc rmul(df s, dfc b) { return dfc{s * b.x, s * b.y}; }

// Coefficients of this mode are stored as double-float quadruples (h, l of the real part, then
// of the imaginary part): one 16-byte read-only load.
__device__ __forceinline__ dfc ldgc(const dfc *p)
{
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    return dfc{df(q.x, q.y), df(q.z, q.w)};
}

// Exact split of a double into h + l: h keeps the sign, the exponent and the top 23 stored
// mantissa bits (truncation), l = x - h (29 bits, rounded to FP32), then renormalised.
// Magnitudes below 2^-126 become 0 (an absolute error below 1.2e-38); l is dropped below 2^-74.
__device__ __forceinline__ df d2df(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const uint32_t bh = uint32_t(b >> 32), bl = uint32_t(b);
    const int E = int((bh >> 20) & 0x7FFu);
    if (E < 897) return df(0.f, 0.f);
    const uint32_t sgn = bh & 0x80000000u;
    const float h = __uint_as_float(sgn | (uint32_t(E - 896) << 23) | ((bh & 0xFFFFFu) << 3) | (bl >> 29));
    float l = 0.f;
    if (E >= 949) {
        const float scale = __uint_as_float(uint32_t(E - 948) << 23);  // 2^(E - 1075)
        l = __uint_as_float(__float_as_uint(__uint2float_rn(bl & 0x1FFFFFFFu) * scale) | sgn);
    }
    return df_fast_two_sum(h, l);
}

// Exact FP32 -> FP64 by bit manipulation (zero and subnormal FP32 values map to 0).
__device__ __forceinline__ double f2d_bits(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    const unsigned long long bits = (static_cast<unsigned long long>(u & 0x80000000u) << 32) |
                                    (static_cast<unsigned long long>(e + 896u) << 52) |
                                    (static_cast<unsigned long long>(u & 0x7FFFFFu) << 29);
    return __longlong_as_double(static_cast<long long>(bits));
}

__device__ __forceinline__ double df2d(df a) { return f2d_bits(a.h) + f2d_bits(a.l); }

}  // namespace
}  // namespace qs
