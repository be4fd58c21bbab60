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
// (a CTA: 8 warps, 8192 positions), searched by detect_segment
// (dd_detect_seg.cuh; the 255-sample halo the widest boxcar needs is re-read
// from L2 by the neighbouring warp).
// finalize_kernel then turns the sums and keys into mean, std, S/N and t with
// the same IEEE FP64 operations, in the same order, as the CPU definition.
// The output arrays double as the accumulators, so no scratch is needed.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <type_traits>

#include "dd_detect_seg.cuh"
#include "dd_internal.h"

namespace {

using dd::detect_segment;
using dd::kMaxLevels;
using dd::unordered;

constexpr int kOwnK = 32;       // owned positions per lane (1024 per warp)
constexpr int kKH = kOwnK + dd::kReach;
constexpr int kWarps = 8;

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
        detect_segment<INT, false, kOwnK, false>(x, nsamp, s0, row, nlevels, lane, one, s1, s2,
                                                 keys);
    else
        detect_segment<INT, true, kOwnK, false>(x, nsamp, s0, row, nlevels, lane, one, s1, s2,
                                                keys);
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

namespace dd {

dd_status detect_begin(int ndm, int nlevels, double *mean, double *sd, double *snr,
                       cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(mean, 0, sizeof(double) * ndm, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(sd, 0, sizeof(double) * ndm, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(snr, 0, sizeof(double) * (size_t)ndm * nlevels, s);
    return e == cudaSuccess ? DD_OK
                            : fail(DD_ERR_CUDA, std::string("detect memset: ") + cudaGetErrorString(e));
}

dd_status detect_finalize_int(int ndm, int64_t nsamp, int nlevels, double *mean, double *sd,
                              double *snr, int64_t *tpk, cudaStream_t s) {
    const unsigned fg = (unsigned)((ndm + 255) / 256);
    finalize_kernel<true><<<fg, 256, 0, s>>>(ndm, nsamp, nlevels, mean, sd, snr, tpk);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("detect finalize: ") + cudaGetErrorString(e));
    count_launch(1);
    return DD_OK;
}

}  // namespace dd
