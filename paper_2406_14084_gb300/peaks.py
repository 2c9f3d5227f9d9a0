"""Measure the FP32 and FP64 FMA issue rates of the current GPU.

The simulator's slab kernel is bound either by HBM or by the FMA pipe of the state precision,
so the arithmetic roofline needs both rates; GB300 issues FP64 at a small fraction of the FP32
rate.  The probe kernel runs 8 independent FMA chains per thread over a grid of 8 CTAs per SM
and is timed with CUDA events; the result is FMA instructions per second (x2 for flop/s).

    python -m paper_2406_14084_gb300.peaks      # prints one JSON line
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = r'''
#include <cuda_runtime.h>
template <typename T>
__global__ void fma_probe(T *out, int iters, T a, T b)
{
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5,
      x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == T(-1.2345)) out[0] = s;
}
// packed FP32: one fma.rn.f32x2 instruction performs two FMAs
__global__ void fma2_probe(float *out, int iters, float a, float b)
{
    unsigned long long x[8], av, bv;
    float2 t = make_float2(a, a);
    av = *reinterpret_cast<unsigned long long *>(&t);
    t = make_float2(b, b);
    bv = *reinterpret_cast<unsigned long long *>(&t);
    for (int k = 0; k < 8; ++k) {
        float2 s = make_float2(threadIdx.x + k, threadIdx.x - k);
        x[k] = *reinterpret_cast<unsigned long long *>(&s);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(av), "l"(bv));
        }
    }
    float s = 0;
    for (int k = 0; k < 8; ++k) {
        float2 v = *reinterpret_cast<float2 *>(&x[k]);
        s += v.x + v.y;
    }
    if (s == -1.2345f) out[0] = s;
}
extern "C" double probe2(int iters)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void *out = nullptr;
    cudaMalloc(&out, 64);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 256, blocks = sms * 8;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        fma2_probe<<<blocks, threads>>>((float *)out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return double(blocks) * threads * iters * 16.0 * 8.0 * 2.0 / (ms * 1e-3);  // FMAs per second
}
extern "C" double probe(int dbl, int iters)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void *out = nullptr;
    cudaMalloc(&out, 64);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int threads = 256, blocks = sms * 8;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0);
        if (dbl) fma_probe<double><<<blocks, threads>>>((double *)out, iters, 0.999999, 1e-7);
        else fma_probe<float><<<blocks, threads>>>((float *)out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    const double fmas = double(blocks) * threads * iters * 16.0 * 8.0;
    return fmas / (ms * 1e-3);
}
'''


def build() -> str:
    out = os.path.join(HERE, "_build", "libpeaks.so")
    src = os.path.join(HERE, "_build", "peaks_probe.cu")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not os.path.exists(out):
        with open(src, "w") as f:
            f.write(SRC)
        subprocess.run(["nvcc", "-O3", "-shared", "-Xcompiler", "-fPIC", "-gencode",
                        "arch=compute_103a,code=sm_103a", src, "-o", out], check=True)
    return out


def measure() -> dict:
    L = ctypes.CDLL(build())
    L.probe.restype = ctypes.c_double
    L.probe.argtypes = [ctypes.c_int, ctypes.c_int]
    L.probe2.restype = ctypes.c_double
    L.probe2.argtypes = [ctypes.c_int]
    f32 = L.probe(0, 4000)
    f64 = L.probe(1, 200)
    f32x2 = L.probe2(4000)
    return {"fp32_fma_per_s": f32, "fp32x2_fma_per_s": f32x2, "fp64_fma_per_s": f64,
            "fp32_tflops": 2 * f32 / 1e12, "fp32x2_tflops": 2 * f32x2 / 1e12,
            "fp64_tflops": 2 * f64 / 1e12, "ratio_fp32_to_fp64": f32 / f64 if f64 > 0 else None}


if __name__ == "__main__":
    print(json.dumps(measure()))
