// Add-throughput microbenchmark: the measured denominator of the
// de-dispersion roofline.  The de-dispersion is bound by plain 32-bit adds
// (one per channel, DM and sample), so its roofline peak is the rate at
// which an SM retires independent adds.  Each thread runs kChains
// independent dependency chains of one add kind, so that every SM has enough
// independent instructions in flight to keep its pipes busy; inline PTX keeps
// the compiler from folding a chain (integer chains would otherwise collapse
// into one multiply-add).
#include <cuda_runtime.h>

#include <string>

#include "dd_internal.h"

namespace dd {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kIters = 16384;

// Written only when the kernel's `store` argument is non-zero (never by the
// library), which keeps every chain's result live through the assembler.
__device__ float g_peak_sink[256];

// kind 0: FP32 add.rn.f32 of a constant (IEEE rounding forbids folding a
// chain); 1: 32-bit integer adds, half as add.u32 and half as mad.lo.u32
// with a multiplier of 1 known only at run time (the integer ALU and the FMA
// pipe both add 32-bit integers, and the uint8 de-dispersion kernel uses
// both), each chain adding the next chain's current value so that no chain
// reduces to a closed form; 2: packed FP32 pairs add.rn.f32x2 (two adds per
// instruction).
template <int KIND>
__global__ void __launch_bounds__(kThreads) add_peak_kernel(float fb, uint32_t ib, int store) {
    float f[kChains];
    uint32_t u[kChains];
    unsigned long long p[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        f[i] = (float)(threadIdx.x + i);
        u[i] = threadIdx.x * 7u + (uint32_t)i;
        const float lo = (float)i, hi = (float)(i + 1);
        p[i] = ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
    }
    const unsigned long long pb =
        ((unsigned long long)__float_as_uint(fb) << 32) | __float_as_uint(fb);
    const uint32_t one = ib >> 1;  // 1 for the ib passed by the host
#pragma unroll 16
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if (KIND == 0)
                asm volatile("add.rn.f32 %0, %0, %1;" : "+f"(f[i]) : "f"(fb));
            else if (KIND == 1 && (i & 1) == 0)
                asm volatile("add.u32 %0, %0, %1;" : "+r"(u[i]) : "r"(u[(i + 1) % kChains]));
            else if (KIND == 1)
                asm volatile("mad.lo.u32 %0, %1, %2, %0;"
                             : "+r"(u[i])
                             : "r"(u[(i + 1) % kChains]), "r"(one));
            else
                asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(p[i]) : "l"(pb));
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i)
        acc += f[i] + (float)u[i] + __uint_as_float((uint32_t)p[i]);
    if (store)
        g_peak_sink[threadIdx.x & 255] = acc;
}

}  // namespace
}  // namespace dd

extern "C" dd_status dd_add_peak(int kind, int ctas_per_sm, void *stream, double *adds_per_s,
                                 double *ms_out) {
    using dd::fail;
    dd::Range nvtx_range("dd_add_peak");
    if (kind < 0 || kind > 2 || ctas_per_sm < 1 || ctas_per_sm > 8 || !adds_per_s)
        return fail(DD_ERR_INVALID, "kind must be 0..2, ctas_per_sm 1..8, adds_per_s non-NULL");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(DD_ERR_CUDA, "device query failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)(sms * ctas_per_sm);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(DD_ERR_CUDA, "event creation failed");
    float best = -1.0f;
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms up
        cudaEventRecord(e0, s);
        switch (kind) {
        case 0: dd::add_peak_kernel<0><<<grid, dd::kThreads, 0, s>>>(1.0f, 3u, 0); break;
        case 1: dd::add_peak_kernel<1><<<grid, dd::kThreads, 0, s>>>(1.0f, 3u, 0); break;
        default: dd::add_peak_kernel<2><<<grid, dd::kThreads, 0, s>>>(1.0f, 3u, 0); break;
        }
        e = cudaGetLastError();
        cudaEventRecord(e1, s);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (e == cudaSuccess && rep > 0 && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
            best = (best < 0.0f || t < best) ? t : best;
        dd::count_launch();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || best <= 0.0f)
        return fail(DD_ERR_CUDA, std::string("add-peak kernel: ") + cudaGetErrorString(e));
    const double per_inst = kind == 2 ? 2.0 : 1.0;
    const double adds = (double)grid * dd::kThreads * dd::kChains * dd::kIters * per_inst;
    *adds_per_s = adds / (best * 1e-3);
    if (ms_out)
        *ms_out = best;
    return DD_OK;
}
