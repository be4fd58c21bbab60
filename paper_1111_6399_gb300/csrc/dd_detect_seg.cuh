// Boxcar search of one warp's segment of a (DM,t) plane row, shared by the
// detection pass (dd_detect.cu) and the uint8 de-dispersion epilogue
// (dd_kernel.cuh, dd_execute_detect).
//
// A warp owns 32*OWN consecutive start positions s0 .. s0 + 32*OWN - 1 of one
// row: lane l holds samples s0 + l + 32k, k = 0..KH-1 (the owned positions
// plus the tree's reach of 255 samples).  Boxcars are built as a tree,
// B_2w(t) = B_w(t) + B_w(t + w): for w < 32 the second term sits w lanes over
// (one shuffle per sample), for w >= 32 it is w/32 registers further on.  At
// every width each lane keeps its highest boxcar (first on ties: positions
// rise with k); a warp reduction and one 64-bit atomicMax per row and width
// merge the warps, with the key (B << 32) | (2^32 - 1 - t) ordering by B,
// then by smaller t.  Row sums S1, S2 of the owned samples go the same way
// with 64-bit atomics: exact integers for integer-valued planes, FP64
// otherwise.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

namespace dd {
namespace {

constexpr int kMaxLevels = 9;   // widths up to 256
// Registers a lane holds beyond its owned positions: each level w < 32
// looks one k further (5 levels up to w = 16), each level w >= 32 looks w/32
// further (w = 32, 64, 128: 1 + 2 + 4).
constexpr int kReach = 5 + 7;

// Order-preserving map of an FP32 value onto uint32.
__device__ __forceinline__ uint32_t ordered(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// a + b on the FMA pipe (b * one + a, one == 1 at run time): the integer ALU
// pipe is this search's bottleneck.
__device__ __forceinline__ uint32_t add_fma(uint32_t a, uint32_t b, uint32_t one) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(b), "r"(one), "r"(a));
    return r;
}
__device__ __forceinline__ float add_fma(float a, float b, uint32_t) { return a + b; }

// INT: integer-valued plane (exact sums); CHECK: the segment reaches the end
// of the row, so loads and boxcar ends are checked against nsamp (segments
// whose every load lies before nsamp skip the checks); OWN: owned positions
// per lane (at most 32); CG: loads through L2 only (data other CTAs of the
// same kernel wrote).
template <bool INT, bool CHECK, int OWN, bool CG>
__device__ __forceinline__ void detect_segment(const float *__restrict__ x, int64_t nsamp,
                                               int64_t s0, int row, int nlevels, int lane,
                                               uint32_t one, unsigned long long *s1,
                                               unsigned long long *s2,
                                               unsigned long long *keys) {
    static_assert(OWN >= 1 && OWN <= 32, "owned positions per lane");
    constexpr int KH = OWN + kReach;
    using T = typename std::conditional<INT, uint32_t, float>::type;
    // Positions of this lane relative to the end of the row: sample k is
    // valid for width w when 32k + w <= lim.
    const int64_t lim64 = nsamp - s0 - lane;
    const int lim = lim64 > 0x7fffffff ? 0x7fffffff : (int)lim64;
    T z[KH];
    bool bad = false;
    double f1 = 0.0, f2 = 0.0;  // FP64 row sums (float planes)
    uint32_t i1 = 0;            // exact row sums (integer planes): 32 x < 2^21 fits
    uint64_t i2 = 0;
#pragma unroll
    for (int k = 0; k < KH; ++k) {
        float v = 0.0f;
        if (!CHECK || 32 * k < lim)
            v = CG ? __ldcg(x + s0 + lane + 32 * k) : x[s0 + lane + 32 * k];
        if (INT) {
            const uint32_t u = __float2uint_rn(v);
            z[k] = (T)u;
            if (k < OWN) {
                // Only owned samples are checked (each sample of a row is owned
                // by one segment): the samples past the owned windows may be
                // another CTA's unfinished tile in the fused search.
                bad |= !(v >= 0.0f && v < 2097152.0f && (float)u == v);
                i1 += u;
                i2 += (uint64_t)u * u;
            }
        } else {
            z[k] = (T)v;
            if (k < OWN) {
                f1 += (double)v;
                f2 += (double)v * (double)v;
            }
        }
    }

    // Highest boxcar of the current width over this lane's owned positions
    // (first on ties), merged across the warp and into the row's key.
    auto track = [&](int lev, int w) {
        uint32_t bv = 0;
        int bk = -1;
        if (INT && !CHECK && lev <= 5) {
            // Integer boxcars of width <= 32 are below 2^26, so (B << 5) | (31 - k)
            // fits 32 bits: one multiply-add (FMA pipe) and one max per sample
            // give the highest B at its first k.
            const uint32_t by32 = one << 5;  // 32, opaque to the compiler
            uint32_t best = 0;
#pragma unroll
            for (int k = 0; k < OWN; ++k) {
                uint32_t key;
                asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(key) : "r"((uint32_t)z[k]), "r"(by32),
                    "r"(31u - (uint32_t)k));
                best = max(best, key);
            }
            bv = best >> 5;
            bk = 31 - (int)(best & 31u);
        } else {
#pragma unroll
            for (int k = 0; k < OWN; ++k) {
                const uint32_t v = INT ? (uint32_t)z[k] : ordered((float)z[k]);
                if (CHECK) {
                    if (32 * k + w <= lim && (bk < 0 || v > bv)) {
                        bv = v;
                        bk = k;
                    }
                } else if (k == 0 || v > bv) {
                    bv = v;
                    bk = k;
                }
            }
        }
        unsigned long long key = 0;
        if (bk >= 0)
            key = ((unsigned long long)bv << 32) |
                  (0xffffffffull - (uint64_t)(s0 + lane + 32 * bk));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
            key = other > key ? other : key;
        }
        if (lane == 0 && key != 0)
            atomicMax(&keys[(int64_t)row * nlevels + lev], key);
    };
    track(0, 1);
#pragma unroll
    for (int lev = 1; lev < kMaxLevels; ++lev) {
        if (lev >= nlevels)
            break;
        const int w = 1 << (lev - 1);  // B_2w(t) = B_w(t) + B_w(t + w)
        if (w < 32) {
            const int src = (lane + w) & 31;
            const bool wrap = lane + w >= 32;
            T r = __shfl_sync(0xffffffffu, z[0], src);
#pragma unroll
            for (int k = 0; k + 1 < KH; ++k) {
                const T r1 = __shfl_sync(0xffffffffu, z[k + 1], src);
                z[k] = add_fma(z[k], wrap ? r1 : r, one);
                r = r1;
            }
        } else {
            const int m = w / 32;
#pragma unroll
            for (int k = 0; k + m < KH; ++k)
                z[k] = add_fma(z[k], z[k + m], one);
        }
        track(lev, 2 * w);
    }

    if (INT) {
        const bool any_bad = __any_sync(0xffffffffu, bad);
        uint64_t a = i1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            i2 += __shfl_xor_sync(0xffffffffu, i2, o);
        }
        if (lane == 0) {
            atomicAdd(&s1[row], (unsigned long long)a);
            atomicAdd(&s2[row], (unsigned long long)i2);
            if (any_bad)
                atomicOr(&s2[row], 1ull << 63);
        }
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            f1 += __shfl_xor_sync(0xffffffffu, f1, o);
            f2 += __shfl_xor_sync(0xffffffffu, f2, o);
        }
        if (lane == 0) {
            atomicAdd(reinterpret_cast<double *>(&s1[row]), f1);
            atomicAdd(reinterpret_cast<double *>(&s2[row]), f2);
        }
    }
}

}  // namespace
}  // namespace dd
