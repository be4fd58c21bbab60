// Detection on the (DM,t) plane (dd_detect): per DM row, the mean and
// standard deviation of the row and, for boxcar widths w = 1, 2, 4, ...,
// 2^(nlevels-1) (at most 256), the highest boxcar sum and the first sample
// where it starts, turned into S/N = (B - w*mean) / (std*sqrt(w)).
//
// Sec. 4 and Fig. 3 of the paper search the plane for a simulated pulse and
// recover it at its DM and time; this is that search as matched boxcar
// filters (the paper gives no formula, so this is the reading the library
// adopts).  Rows where std is 0 report S/N 0; widths longer than the row
// report t = -1 and S/N -inf.
//
// detect_kernel: one warp owns 1024 consecutive start positions of one row
// (a CTA: 8 warps, 8192 positions).  Lane l holds samples s0 + l + 32k,
// k = 0..KH-1 (the 1024 owned positions plus the 255-sample halo the widest
// boxcar needs, re-read from L2 by the neighbouring warp).  Boxcars are built
// as a tree, B_2w(t) = B_w(t) + B_w(t + w): for w < 32 the second term sits w
// lanes over (one shuffle per sample), for w >= 32 it is w/32 registers
// further on.  At every width each lane keeps its highest boxcar (first on
// ties: positions rise with k); a warp reduction and one 64-bit atomicMax per
// row and width merge the warps, with the key (B << 32) | (2^32 - 1 - t)
// ordering by B, then by smaller t.  Row sums S1, S2 go the same way with
// 64-bit atomics: exact integers for integer-valued planes, FP64 otherwise.
// finalize_kernel then turns the sums and keys into mean, std, S/N and t with
// the same IEEE FP64 operations, in the same order, as the CPU definition.
// The output arrays double as the accumulators, so no scratch is needed.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <type_traits>

#include "dd_internal.h"

namespace {

constexpr int kMaxLevels = 9;   // widths up to 256
constexpr int kOwnK = 32;       // owned positions per lane (1024 per warp)
// Registers per lane: the owned 32 plus the tree's reach: each level w < 32
// looks one k further (5 levels up to w = 16), each level w >= 32 looks w/32
// further (w = 32, 64, 128: 1 + 2 + 4).
constexpr int kKH = kOwnK + 5 + 7;
constexpr int kWarps = 8;

// Order-preserving map of an FP32 value onto uint32.
__device__ __forceinline__ uint32_t ordered(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// One warp's segment.  CHECK: the segment reaches the end of the row, so
// loads and boxcar ends are checked against nsamp; interior segments (every
// boxcar ending before nsamp) skip the checks.
// a + b on the FMA pipe (b * one + a, one == 1 at run time): the integer ALU
// pipe is this kernel's bottleneck.
__device__ __forceinline__ uint32_t add_fma(uint32_t a, uint32_t b, uint32_t one) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(b), "r"(one), "r"(a));
    return r;
}
__device__ __forceinline__ float add_fma(float a, float b, uint32_t) { return a + b; }

template <bool INT, bool CHECK>
__device__ __forceinline__ void detect_segment(const float *__restrict__ x, int64_t nsamp,
                                               int64_t s0, int row, int nlevels, int lane,
                                               uint32_t one, unsigned long long *s1,
                                               unsigned long long *s2,
                                               unsigned long long *keys) {
    using T = typename std::conditional<INT, uint32_t, float>::type;
    // Positions of this lane relative to the end of the row: sample k is
    // valid for width w when 32k + w <= lim.
    const int64_t lim64 = nsamp - s0 - lane;
    const int lim = lim64 > 0x7fffffff ? 0x7fffffff : (int)lim64;
    T z[kKH];
    bool bad = false;
    double f1 = 0.0, f2 = 0.0;  // FP64 row sums (float planes)
    uint32_t i1 = 0;            // exact row sums (integer planes): 32 x < 2^21 fits
    uint64_t i2 = 0;
#pragma unroll
    for (int k = 0; k < kKH; ++k) {
        const float v = (!CHECK || 32 * k < lim) ? x[s0 + lane + 32 * k] : 0.0f;
        if (INT) {
            const uint32_t u = __float2uint_rn(v);
            bad |= !(v >= 0.0f && v < 2097152.0f && (float)u == v);
            z[k] = (T)u;
            if (k < kOwnK) {
                i1 += u;
                i2 += (uint64_t)u * u;
            }
        } else {
            z[k] = (T)v;
            if (k < kOwnK) {
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
            for (int k = 0; k < kOwnK; ++k) {
                uint32_t key;
                asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(key) : "r"((uint32_t)z[k]), "r"(by32),
                    "r"(31u - (uint32_t)k));
                best = max(best, key);
            }
            bv = best >> 5;
            bk = 31 - (int)(best & 31u);
        } else {
#pragma unroll
            for (int k = 0; k < kOwnK; ++k) {
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
            for (int k = 0; k + 1 < kKH; ++k) {
                const T r1 = __shfl_sync(0xffffffffu, z[k + 1], src);
                z[k] = add_fma(z[k], wrap ? r1 : r, one);
                r = r1;
            }
        } else {
            const int m = w / 32;
#pragma unroll
            for (int k = 0; k + m < kKH; ++k)
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

template <bool INT>
__global__ void __launch_bounds__(32 * kWarps, 3) detect_kernel(const float *__restrict__ plane,
                                                                int64_t pitch, int64_t nsamp,
                                                                int groups, int nlevels,
                                                                unsigned long long *s1,
                                                                unsigned long long *s2,
                                                                unsigned long long *keys,
                                                                uint32_t one) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x / groups;
    const int64_t s0 =
        ((int64_t)(blockIdx.x % groups) * kWarps + (threadIdx.x >> 5)) * (32 * kOwnK);
    if (s0 >= nsamp)
        return;
    const float *x = plane + (int64_t)row * pitch;
    if (s0 + 32 * kKH <= nsamp)
        detect_segment<INT, false>(x, nsamp, s0, row, nlevels, lane, one, s1, s2, keys);
    else
        detect_segment<INT, true>(x, nsamp, s0, row, nlevels, lane, one, s1, s2, keys);
}

// One thread per row: sums and keys -> mean, std, S/N, t (in place).
template <bool INT>
__global__ void finalize_kernel(int ndm, int64_t nsamp, int nlevels, double *mean, double *sd,
                                double *snr, int64_t *tpk) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= ndm)
        return;
    const double n = (double)nsamp;
    double s1, s2;
    bool bad = false;
    if (INT) {
        const unsigned long long a = reinterpret_cast<unsigned long long *>(mean)[row];
        const unsigned long long b = reinterpret_cast<unsigned long long *>(sd)[row];
        bad = (b >> 63) != 0;
        s1 = __ull2double_rn(a);
        s2 = __ull2double_rn(b);
    } else {
        s1 = mean[row];
        s2 = sd[row];
    }
    const double m = __ddiv_rn(s1, n);
    double var = __dsub_rn(__ddiv_rn(s2, n), __dmul_rn(m, m));
    if (var < 0.0)
        var = 0.0;
    const double s = __dsqrt_rn(var);
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    mean[row] = bad ? nan : m;
    sd[row] = bad ? nan : s;
    for (int lev = 0; lev < nlevels; ++lev) {
        const int64_t i = (int64_t)row * nlevels + lev;
        const unsigned long long key = reinterpret_cast<unsigned long long *>(snr)[i];
        const double w = (double)(1 << lev);
        if (bad) {
            snr[i] = nan;
            tpk[i] = -1;
        } else if (key == 0) {
            snr[i] = -__longlong_as_double(0x7ff0000000000000ll);  // -inf: no window
            tpk[i] = -1;
        } else {
            const uint32_t v = (uint32_t)(key >> 32);
            const double b = INT ? (double)v : (double)unordered(v);
            tpk[i] = (int64_t)(0xffffffffull - (key & 0xffffffffull));
            snr[i] = s == 0.0 ? 0.0
                              : __ddiv_rn(__dsub_rn(b, __dmul_rn(w, m)),
                                          __dmul_rn(s, __dsqrt_rn(w)));
        }
    }
}

}  // namespace

extern "C" dd_status dd_detect(const float *plane, int64_t pitch, int ndm, int64_t nsamp,
                               int nlevels, int integer_valued, double *mean, double *std_out,
                               double *snr, int64_t *t_peak, void *stream) {
    dd::Range nvtx_range("dd_detect");
    using dd::fail;
    if (ndm < 0 || nsamp < 1 || pitch < nsamp)
        return fail(DD_ERR_INVALID, "need ndm >= 0, nsamp >= 1 and pitch >= nsamp");
    if (nlevels < 1 || nlevels > kMaxLevels)
        return fail(DD_ERR_INVALID, "nlevels must be 1..9 (boxcar widths up to 256)");
    if (nsamp > 0xfffffffeLL || (integer_valued && nsamp > (1LL << 21)))
        return fail(DD_ERR_INVALID, "nsamp too large (2^21 for integer planes)");
    if (ndm == 0)
        return DD_OK;
    if (!plane || !mean || !std_out || !snr || !t_peak || ((uintptr_t)plane & 3u) ||
        ((uintptr_t)mean & 7u) || ((uintptr_t)std_out & 7u) || ((uintptr_t)snr & 7u) ||
        ((uintptr_t)t_peak & 7u))
        return fail(DD_ERR_INVALID, "NULL or misaligned pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(mean, 0, sizeof(double) * ndm, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(std_out, 0, sizeof(double) * ndm, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(snr, 0, sizeof(double) * (size_t)ndm * nlevels, s);
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("detect memset: ") + cudaGetErrorString(e));
    const int64_t per_cta = (int64_t)kWarps * 32 * kOwnK;
    const int64_t groups = (nsamp + per_cta - 1) / per_cta;
    if (groups * ndm > 0x7fffffffLL)
        return fail(DD_ERR_INVALID, "plane too large for one launch");
    const unsigned grid = (unsigned)(groups * ndm);
    auto *s1 = reinterpret_cast<unsigned long long *>(mean);
    auto *s2 = reinterpret_cast<unsigned long long *>(std_out);
    auto *keys = reinterpret_cast<unsigned long long *>(snr);
    if (integer_valued)
        detect_kernel<true><<<grid, 32 * kWarps, 0, s>>>(plane, pitch, nsamp, (int)groups, nlevels,
                                                         s1, s2, keys, 1u);
    else
        detect_kernel<false><<<grid, 32 * kWarps, 0, s>>>(plane, pitch, nsamp, (int)groups,
                                                          nlevels, s1, s2, keys, 1u);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        const unsigned fg = (unsigned)((ndm + 255) / 256);
        if (integer_valued)
            finalize_kernel<true><<<fg, 256, 0, s>>>(ndm, nsamp, nlevels, mean, std_out, snr,
                                                     t_peak);
        else
            finalize_kernel<false><<<fg, 256, 0, s>>>(ndm, nsamp, nlevels, mean, std_out, snr,
                                                      t_peak);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("detect launch: ") + cudaGetErrorString(e));
    dd::count_launch(2);
    return DD_OK;
}
