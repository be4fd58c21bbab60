// Polyphase channeliser (dd_channelise): subband voltages -> finer channels.
//
// The paper's pipeline channelises the received subbands in finer frequency
// before it forms Stokes parameters (Sec. 1) and names the poly-phase filter
// (Sec. 5) without giving the filter or the transform size.  The library's
// reading is the critically sampled polyphase filter bank: per polarisation,
// with x[j] = re + i*im of raw sample j of a subband,
//
//     y_k[n] = sum_{m < M*T} h[m] x[n*M + m] exp(-2 pi i k m / M),   k < M,
//
// for spectra n = 0 .. floor(nraw/M) - T.  Grouping m = t*M + p gives the
// two steps computed here: a T-tap FIR per branch p,
//     z_p[n] = sum_t h[t*M + p] x[(n + t)*M + p],
// then an M-point DFT of z[n] over p.  Channel c = (k + M/2) mod M of subband
// s is written to row s*M + c (the bins of a subband in increasing frequency).
//
// Kernel structure (one CTA = one subband x NSEG segments of consecutive
// spectra, 256 threads):
//  * FIR: thread (p, g) owns branch p of segment g and slides along its
//    spectra in transposed form: each raw sample (one 32-bit word holding
//    Xre, Xim, Yre, Yim) is loaded and converted once, then added with its T
//    weights into the accumulators of the T spectra it belongs to; a
//    spectrum whose last sample arrived is written to shared memory.  A warp
//    loads 32 consecutive branches (128 contiguous bytes) per spectrum.
//  * DFT, four-step M = 16 x M2: pass 1 does a 16-point FFT in registers
//    over p1 (p = M2*p1 + p2) for each (p2, spectrum, polarisation) and
//    multiplies by W_M^(k1*p2); pass 2 does the M2-point FFT over p2 for each
//    k1, giving y[k1 + 16*k2].  Shared memory holds the FFT index as the
//    fastest dimension, so the 32 lanes of a warp always touch 32 different
//    transforms: every shared-memory access is conflict-free.
//  * Packed FP32: the FIR keeps (re, im) pairs and multiplies them by (h, h)
//    with FFMA2, and the FFT's butterflies a +- t run as FADD2 / FFMA2, so a
//    pair of FP32 operations takes one issue slot.
//  * Output: each transform's values go to a shared-memory staging area laid
//    out as [channel][spectrum] -- int8 codes q = clamp(rint(v*scale), -127,
//    127) with v*scale rounded once (FMA into 1.5*2^23), the two
//    polarisations of a spectrum side by side, or FP32 values -- and the CTA
//    then writes channel rows with 16-byte stores (four int8 elements, or one
//    FP32 element, per thread).
//  * Rounds: each round a segment emits RS spectra; the next round's raw
//    words are loaded before the current round's DFT, so they are in flight
//    while it runs.
//  * Occupancy: two CTAs per SM (at most 128 registers per thread; a cap of
//    80 for three CTAs spills and measured 24 % slower on the 16-channel
//    workload).
//
// HBM traffic: each raw word is read once by the segment that uses it (plus
// T-1 words of overlap per segment, served from L2), each output element
// written once.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "dd_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kM1 = 16;        // size of the first DFT pass
constexpr int kMaxRounds = 32;  // rounds per CTA (segment length RS * rounds)

struct PfbArgs {
    const uint8_t *in;   // raw words, rows of in_pitch bytes
    int64_t in_pitch;
    int64_t nblk;        // whole blocks of M raw samples per row
    int64_t nspec;       // spectra per row
    const float *h;      // M*T prototype coefficients
    int T;               // taps (<= the kernel's TI; the rest are zero)
    int nr;              // rounds per CTA
    float scale;         // int8 output: codes = rint(v * scale)
    int ci8;             // 1: int8 elements (4 bytes), 0: FP32 elements (16 bytes)
    int vec;             // int8 rows 16-byte aligned: four elements per store
    uint8_t *out;
    int64_t out_pitch;   // bytes
};

__host__ __device__ constexpr int bitrev(int i, int n) {
    int r = 0;
    for (int b = 1; b < n; b <<= 1) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

// b * W_16^j, W_16 = exp(-2 pi i / 16), j < 8 (cos and sin of multiples of
// pi/8: 1, sqrt(2 + sqrt 2)/2, sqrt 2 / 2, sqrt(2 - sqrt 2)/2).
__device__ __forceinline__ float2 mul_w16(float2 b, int j) {
    constexpr float c1 = 0.923879532511286756f, c2 = 0.707106781186547524f,
                    c3 = 0.382683432365089772f;
    float c = 1.f, s = 0.f;
    switch (j) {
    case 0: return b;
    case 4: return make_float2(b.y, -b.x);  // times -i
    case 1: c = c1; s = c3; break;
    case 2: c = c2; s = c2; break;
    case 3: c = c3; s = c1; break;
    case 5: c = -c3; s = c1; break;
    case 6: c = -c2; s = c2; break;
    case 7: c = -c1; s = c3; break;
    }
    // (b.x + i b.y)(c - i s)
    return make_float2(fmaf(b.x, c, b.y * s), fmaf(b.y, c, -(b.x * s)));
}

__device__ __forceinline__ float2 cmul(float2 b, float2 w) {
    return make_float2(fmaf(b.x, w.x, -(b.y * w.y)), fmaf(b.x, w.y, b.y * w.x));
}

// Packed FP32 pairs (one FADD2 / FFMA2 / FMUL2 per pair): a + b, a - b
// (b * -1 + a, one rounding like a subtraction), h * x + c, h * x.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

// In-register forward DFT of N <= 16 points: radix-2 decimation in time.
// Butterflies a +- t run on packed pairs; t = -i*b is a swap and a sign.
template <int N>
__device__ __forceinline__ void fft_reg(float2 (&v)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int j = bitrev(i, N);
        if (j > i) {
            const float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
#pragma unroll
    for (int len = 2; len <= N; len *= 2) {
#pragma unroll
        for (int i0 = 0; i0 < N; i0 += len) {
#pragma unroll
            for (int k = 0; k < len / 2; ++k) {
                const int tj = k * (16 / len);
                const float2 a = v[i0 + k];
                const float2 b = v[i0 + k + len / 2];
                if (tj == 4) {  // t = -i b = (b.y, -b.x)
                    v[i0 + k] = make_float2(a.x + b.y, a.y - b.x);
                    v[i0 + k + len / 2] = make_float2(a.x - b.y, a.y + b.x);
                } else {
                    const float2 t = mul_w16(b, tj);
                    v[i0 + k] = add2(a, t);
                    v[i0 + k + len / 2] = sub2(a, t);
                }
            }
        }
    }
}

// Four signed bytes (Xre, Xim, Yre, Yim) -> FP32 pairs X, Y, exactly: byte
// b + 128 is placed in the mantissa of 2^23 and 2^23 + 128 is subtracted.
__device__ __forceinline__ void s8x4(uint32_t w, float2 &x, float2 &y) {
    const uint32_t u = w ^ 0x80808080u;
    const float2 off = make_float2(-8388736.0f, -8388736.0f);  // -(2^23 + 128)
    x = add2(make_float2(__uint_as_float(__byte_perm(u, 0x4b000000u, 0x7650)),
                         __uint_as_float(__byte_perm(u, 0x4b000000u, 0x7651))), off);
    y = add2(make_float2(__uint_as_float(__byte_perm(u, 0x4b000000u, 0x7652)),
                         __uint_as_float(__byte_perm(u, 0x4b000000u, 0x7653))), off);
}

// int8 codes (re, im) of v*scale in the low 16 bits: the FMA into 1.5*2^23
// rounds each exact product to the nearest integer (ties to even); clamped
// to [-127, 127]; the low byte of each float's bits is its code in two's
// complement.
__device__ __forceinline__ uint32_t code16(float2 v, float2 scale2) {
    constexpr float magic = 12582912.0f;  // 1.5 * 2^23
    float2 u = __ffma2_rn(v, scale2, make_float2(magic, magic));
    u.x = fminf(fmaxf(u.x, magic - 127.0f), magic + 127.0f);
    u.y = fminf(fmaxf(u.y, magic - 127.0f), magic + 127.0f);
    return __byte_perm(__float_as_uint(u.x), __float_as_uint(u.y), 0x0040);
}

template <int M, int TI>
struct Shape {
    static constexpr int NSEG = kThreads / M;       // segments per CTA
    static constexpr int RS = TI > 8 ? TI : 8;      // spectra per segment per round
    static constexpr int R = NSEG * RS;             // spectra per round
    static constexpr int NF = 2 * R;                // transforms per round
    static constexpr int ZS = NF + 2;               // float2 per branch row (conflict-free STS.128)
    static constexpr int M2 = M / kM1;
    static constexpr int ZBYTES = (M * ZS + M) * 8; // z rows + twiddle table
    // Output staging, [channel][spectrum of the round]: one 4-byte element
    // (int8) or two float2 (FP32) per cell.
    static constexpr int SMEM_CI8 = ZBYTES + M * R * 4;
    static constexpr int SMEM_CF32 = ZBYTES + M * R * 16;
};

template <int M, int TI, bool CI8>
__global__ void __launch_bounds__(kThreads, TI > 8 ? 1 : 2) pfb_kernel(const PfbArgs a) {
    using S = Shape<M, TI>;
    constexpr int NSEG = S::NSEG, RS = S::RS, R = S::R, NF = S::NF, ZS = S::ZS, M2 = S::M2;
    extern __shared__ __align__(16) float2 zsm[];
    float2 *tw = zsm + M * ZS;  // W_M^r, r < M
    uint8_t *stg = reinterpret_cast<uint8_t *>(zsm) + S::ZBYTES;

    const int tid = threadIdx.x;
    const int sub = blockIdx.y;
    const int64_t seg_len = (int64_t)a.nr * RS;
    const int64_t n_cta = (int64_t)blockIdx.x * NSEG * seg_len;

    for (int r = tid; r < M; r += kThreads) {
        float sn, cs;
        sincospif(2.0f * (float)r / (float)M, &sn, &cs);
        tw[r] = make_float2(cs, -sn);
    }

    // ------------------------------ FIR state ------------------------------
    const int p = tid % M;
    const int g = tid / M;
    const int64_t n_first = n_cta + g * seg_len;
    const uint8_t *row = a.in + (int64_t)sub * a.in_pitch + 4 * (int64_t)p;
    float2 hr[TI];  // (h, h): one packed multiplier per tap
#pragma unroll
    for (int t = 0; t < TI; ++t) {
        const float h = t < a.T ? __ldg(a.h + t * M + p) : 0.0f;
        hr[t] = make_float2(h, h);
    }
    // Raw block j of this segment (blocks past the row repeat the last one:
    // they only meet zero taps or spectra that are not stored).
    auto load = [&](int64_t j) -> uint32_t {
        int64_t b = n_first + j;
        b = b < a.nblk ? b : a.nblk - 1;
        return __ldg(reinterpret_cast<const uint32_t *>(row + 4 * M * b));
    };
    float2 ax[TI], ay[TI];  // per spectrum slot: X and Y partial sums
    // Raw block j (j mod TI = J at compile time) into the spectra j - t.
    auto fir = [&](int J, uint32_t w) {
        float2 x, y;
        s8x4(w, x, y);
#pragma unroll
        for (int t = 0; t < TI; ++t) {
            const int slot = ((J - t) % TI + TI) % TI;
            if (t == 0) {
                ax[slot] = __fmul2_rn(hr[0], x);
                ay[slot] = __fmul2_rn(hr[0], y);
            } else {
                ax[slot] = __ffma2_rn(hr[t], x, ax[slot]);
                ay[slot] = __ffma2_rn(hr[t], y, ay[slot]);
            }
        }
    };
    uint32_t xw[RS];
    {
        uint32_t wu[TI - 1];
#pragma unroll
        for (int j = 0; j < TI - 1; ++j)
            wu[j] = load(j);
#pragma unroll
        for (int i = 0; i < RS; ++i)
            xw[i] = load(TI - 1 + i);
#pragma unroll
        for (int j = 0; j < TI - 1; ++j)
            fir(j % TI, wu[j]);
    }
    const float2 scale2 = make_float2(a.scale, a.scale);

    // Value y of transform f (= 2 * spectrum-in-round + polarisation) at bin
    // k, into the staging cell of its channel and spectrum.
    auto stage = [&](int f, int k, float2 y) {
        const int c = (k + M / 2) & (M - 1);
        if constexpr (CI8) {
            reinterpret_cast<uint16_t *>(stg)[(c * R + (f >> 1)) * 2 + (f & 1)] =
                (uint16_t)code16(y, scale2);
        } else {
            reinterpret_cast<float2 *>(stg)[(c * R + (f >> 1)) * 2 + (f & 1)] = y;
        }
    };

    for (int r = 0; r < a.nr; ++r) {
        // FIR: this round's RS raw blocks per segment; spectrum i of the round
        // completes with block TI-1+i and leaves slot i mod TI.
#pragma unroll
        for (int i = 0; i < RS; ++i) {
            fir((TI - 1 + i) % TI, xw[i]);
            const float4 z = make_float4(ax[i % TI].x, ax[i % TI].y, ay[i % TI].x, ay[i % TI].y);
            *reinterpret_cast<float4 *>(&zsm[p * ZS + 2 * (g * RS + i)]) = z;
        }
        if (r + 1 < a.nr) {
#pragma unroll
            for (int i = 0; i < RS; ++i)
                xw[i] = load(TI - 1 + (int64_t)(r + 1) * RS + i);
        }
        __syncthreads();

        // Pass 1: 16-point FFT over p1 for each (p2, transform f).
        for (int u = tid; u < M2 * NF; u += kThreads) {
            const int f = u % NF;
            const int p2 = u / NF;
            float2 v[kM1];
#pragma unroll
            for (int p1 = 0; p1 < kM1; ++p1)
                v[p1] = zsm[(M2 * p1 + p2) * ZS + f];
            fft_reg<kM1>(v);
            if constexpr (M2 == 1) {
#pragma unroll
                for (int k = 0; k < kM1; ++k)
                    stage(f, k, v[k]);
            } else {
#pragma unroll
                for (int k1 = 0; k1 < kM1; ++k1) {
                    const float2 w = tw[(k1 * p2) & (M - 1)];
                    zsm[(M2 * k1 + p2) * ZS + f] = k1 == 0 ? v[0] : cmul(v[k1], w);
                }
            }
        }
        __syncthreads();
        if constexpr (M2 > 1) {
            // Pass 2: M2-point FFT over p2 for each (k1, transform f).
            for (int u = tid; u < kM1 * NF; u += kThreads) {
                const int f = u % NF;
                const int k1 = u / NF;
                float2 v[M2];
#pragma unroll
                for (int p2 = 0; p2 < M2; ++p2)
                    v[p2] = zsm[(M2 * k1 + p2) * ZS + f];
                fft_reg<M2>(v);
#pragma unroll
                for (int k2 = 0; k2 < M2; ++k2)
                    stage(f, k1 + kM1 * k2, v[k2]);
            }
            __syncthreads();
        }

        // Stores: channel rows of the staging area to HBM, 16 bytes per
        // thread (four int8 elements, or one FP32 element).  The next round's
        // FIR writes only z, so no barrier is needed after this phase.
        constexpr int PER = CI8 ? 4 : 1;  // spectra per 16-byte store
        for (int q = tid; q < M * (R / PER); q += kThreads) {
            const int c = q / (R / PER);
            const int rho = (q % (R / PER)) * PER;
            const int64_t n = n_cta + (rho / RS) * seg_len + (int64_t)r * RS + rho % RS;
            uint8_t *orow = a.out + ((int64_t)sub * M + c) * a.out_pitch;
            if constexpr (CI8) {
                const uint4 wv = *reinterpret_cast<const uint4 *>(stg + (c * R + rho) * 4);
                if (a.vec && n + 3 < a.nspec) {
                    __stcs(reinterpret_cast<uint4 *>(orow + 4 * n), wv);
                } else {
                    const uint32_t e[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (n + i < a.nspec)
                            __stcs(reinterpret_cast<unsigned int *>(orow + 4 * (n + i)), e[i]);
                }
            } else {
                const float4 el = *reinterpret_cast<const float4 *>(stg + (c * R + rho) * 16);
                if (n < a.nspec)
                    __stcs(reinterpret_cast<float4 *>(orow + 16 * n), el);
            }
        }
    }
}

template <int M, int TI, bool CI8>
cudaError_t launch(const PfbArgs &a, unsigned gx, unsigned gy, cudaStream_t s) {
    constexpr int smem = CI8 ? Shape<M, TI>::SMEM_CI8 : Shape<M, TI>::SMEM_CF32;
    static unsigned long long attr_set = 0;  // per device
    if (smem > 48 * 1024) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess)
            return e;
        if (dev >= 64 || !((attr_set >> dev) & 1ull)) {
            e = cudaFuncSetAttribute(pfb_kernel<M, TI, CI8>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess)
                return e;
            if (dev < 64)
                attr_set |= 1ull << dev;
        }
    }
    pfb_kernel<M, TI, CI8><<<dim3(gx, gy), kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int M, bool CI8>
cudaError_t launch_t(int ti, const PfbArgs &a, unsigned gx, unsigned gy, cudaStream_t s) {
    switch (ti) {
    case 2: return launch<M, 2, CI8>(a, gx, gy, s);
    case 4: return launch<M, 4, CI8>(a, gx, gy, s);
    case 8: return launch<M, 8, CI8>(a, gx, gy, s);
    case 16: return launch<M, 16, CI8>(a, gx, gy, s);
    }
    return cudaErrorInvalidValue;
}

template <int M>
cudaError_t launch_m(int ti, const PfbArgs &a, unsigned gx, unsigned gy, cudaStream_t s) {
    return a.ci8 ? launch_t<M, true>(ti, a, gx, gy, s) : launch_t<M, false>(ti, a, gx, gy, s);
}

int taps_instantiated(int T) { return T <= 2 ? 2 : T <= 4 ? 4 : T <= 8 ? 8 : 16; }

// Spectra per round of the kernel for (M, T): NSEG * RS.
int64_t spectra_per_round(int M, int T) {
    const int ti = taps_instantiated(T);
    return (int64_t)(kThreads / M) * (ti > 8 ? ti : 8);
}

bool m_ok(int M) { return M == 16 || M == 32 || M == 64 || M == 128 || M == 256; }

}  // namespace

extern "C" int64_t dd_channelise_nspec(int64_t nraw, int nchan_sub, int ntaps) {
    if (nraw < 0 || !m_ok(nchan_sub) || ntaps < 1 || ntaps > 16)
        return -1;
    const int64_t nblk = nraw / nchan_sub;
    return nblk >= ntaps ? nblk - ntaps + 1 : 0;
}

extern "C" dd_status dd_pfb_prototype(int nchan_sub, int ntaps, float *h) {
    using dd::fail;
    if (nchan_sub < 1 || ntaps < 1 || (int64_t)nchan_sub * ntaps < 2 || !h)
        return fail(DD_ERR_INVALID, "pfb_prototype: need nchan_sub >= 1, ntaps >= 1, "
                                    "nchan_sub*ntaps >= 2 and a host array");
    const int64_t L = (int64_t)nchan_sub * ntaps;
    const double pi = 3.14159265358979323846;
    for (int64_t m = 0; m < L; ++m) {
        // sinc with its first zeros one channel spacing from the centre, times
        // a Hamming window over the L taps.
        const double x = ((double)m - (double)(L - 1) / 2.0) / (double)nchan_sub;
        const double sinc = x == 0.0 ? 1.0 : std::sin(pi * x) / (pi * x);
        const double w = 0.54 - 0.46 * std::cos(2.0 * pi * (double)m / (double)(L - 1));
        h[m] = (float)(sinc * w);
    }
    return DD_OK;
}

extern "C" dd_status dd_channelise(const void *volts, int64_t volts_pitch, int nsub,
                                   int64_t nraw, int nchan_sub, int ntaps, const float *coeffs,
                                   int out_kind, float scale, void *out, int64_t out_pitch,
                                   void *stream) {
    dd::Range nvtx_range("dd_channelise");
    using dd::fail;
    const int M = nchan_sub;
    if (!m_ok(M) || ntaps < 1 || ntaps > 16 || nsub < 1 || nsub > 65535 || nraw < 0)
        return fail(DD_ERR_INVALID, "channelise: need nchan_sub in {16,32,64,128,256}, "
                                    "1 <= ntaps <= 16, 1 <= nsub <= 65535, nraw >= 0");
    if (out_kind != DD_PFB_CF32 && out_kind != DD_PFB_CI8)
        return fail(DD_ERR_INVALID, "channelise: out_kind must be DD_PFB_CF32 or DD_PFB_CI8");
    if (out_kind == DD_PFB_CI8 && !(std::isfinite(scale) && scale > 0.0f))
        return fail(DD_ERR_INVALID, "channelise: scale must be finite and > 0");
    const int64_t elem = out_kind == DD_PFB_CI8 ? 4 : 16;
    const int64_t nspec = dd_channelise_nspec(nraw, M, ntaps);
    if (volts_pitch < 4 * nraw || volts_pitch % 4 != 0 || out_pitch < elem * nspec ||
        out_pitch % elem != 0)
        return fail(DD_ERR_INVALID, "channelise: volts_pitch >= 4*nraw (multiple of 4), "
                                    "out_pitch >= element*nspec (multiple of the element: "
                                    "4 bytes int8, 16 bytes FP32)");
    if (nspec == 0)
        return DD_OK;
    if (!volts || !out || !coeffs || ((uintptr_t)volts & 3u) || ((uintptr_t)coeffs & 3u) ||
        ((uintptr_t)out & (uintptr_t)(elem - 1)))
        return fail(DD_ERR_INVALID, "channelise: NULL or misaligned volts/coeffs/out pointer");
    const int64_t per_round = spectra_per_round(M, ntaps);
    int64_t nr = (nspec + per_round - 1) / per_round;
    if (nr > kMaxRounds)
        nr = kMaxRounds;
    const int64_t per_cta = per_round * nr;
    const int64_t gx = (nspec + per_cta - 1) / per_cta;
    if (gx > 0x7fffffffLL)
        return fail(DD_ERR_INVALID, "channelise: too many spectra");
    PfbArgs a;
    a.in = static_cast<const uint8_t *>(volts);
    a.in_pitch = volts_pitch;
    a.nblk = nraw / M;
    a.nspec = nspec;
    a.h = coeffs;
    a.T = ntaps;
    a.nr = (int)nr;
    a.scale = scale;
    a.ci8 = out_kind == DD_PFB_CI8;
    a.vec = ((uintptr_t)out % 16 == 0) && (out_pitch % 16 == 0);
    a.out = static_cast<uint8_t *>(out);
    a.out_pitch = out_pitch;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int ti = taps_instantiated(ntaps);
    cudaError_t e = cudaErrorInvalidValue;
    switch (M) {
    case 16: e = launch_m<16>(ti, a, (unsigned)gx, (unsigned)nsub, s); break;
    case 32: e = launch_m<32>(ti, a, (unsigned)gx, (unsigned)nsub, s); break;
    case 64: e = launch_m<64>(ti, a, (unsigned)gx, (unsigned)nsub, s); break;
    case 128: e = launch_m<128>(ti, a, (unsigned)gx, (unsigned)nsub, s); break;
    case 256: e = launch_m<256>(ti, a, (unsigned)gx, (unsigned)nsub, s); break;
    }
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("channelise launch: ") + cudaGetErrorString(e));
    dd::count_launch(1);
    return DD_OK;
}
