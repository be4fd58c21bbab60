// Brute-force incoherent de-dispersion kernels for sm_103a (GB300).
//
//   out[d][t] = sum_c in[c][t + s(c,d)],   s(c,d) = trunc(dm[d] * dmshift[c])
//
// Design (Sec. 3 of the paper gives the three rules; this is how they map to
// a Blackwell SM):
//  * Accumulators in registers.  A thread owns dm_per_thread trial DMs x 8
//    four-byte words of output time (32 samples for uint8, lane-interleaved so
//    that a warp's shared-memory reads hit 32 consecutive banks).  A CTA owns a
//    rectangle of (DM,t), as in Fig. 2.
//  * The (f,t) data staged next to the SMs.  Per pipeline stage one thread
//    issues one TMA bulk copy (cp.async.bulk, no multicast) per channel row:
//    the 16-byte aligned window [t0 + s(c,dm_min), t0 + T + s(c,dm_max)) of
//    that channel, completing on an mbarrier.  Two stages alternate, so the
//    copy of stage i+1 runs while stage i is summed.  Shifts are arbitrary in
//    bytes, so for 8/16-bit data the stage also holds the window re-aligned
//    by 1..3 bytes (uint8) or 2 bytes (FP16): every shifted 4-byte read is then
//    an aligned, conflict-free LDS.32.
//  * Little shift arithmetic.  One FP32 multiply and one truncation per
//    (channel, DM) per thread, reused for 8 words (32 uint8 samples).
//  * uint8 sums use 16-bit SWAR lanes: for a word x of 4 samples, L1 += x and
//    L2 += (x >> 8) & 0x00ff00ff.  After at most 256 channels
//    L2 = {sum b1, sum b3} and L1 - 256*L2 = {sum b0, sum b2} exactly; these are
//    widened into the FP32 output (exact: every sum < 2^24).  IADD3 folds two
//    channels into one instruction, so a word of 4 samples x 2 channels costs
//    2 LDS + 2 PRMT + 2 IADD3.
//  * FP16/FP32 sums: FP32 partials over blocks of 64 channels, combined into a
//    running sum with TwoSum compensation (error ~1e-7 of sum |in|).
//
// Every wait on an mbarrier is bounded by the global timer; a wait that runs
// out records a timeout in the status word and the CTA leaves after a second
// bounded wait for its own copies.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"

namespace dd {
namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

struct KArgs {
    const uint8_t *in;
    int64_t in_pitch_b;    // bytes between channel rows
    int64_t nsamp_in;      // valid samples per row
    float *out;
    int64_t out_pitch;     // floats between DM rows
    int64_t nsamp_out;
    const float *dmshift;
    const float *dm_sorted;
    const int *perm;
    int nchan;
    int ndm_pad;
    int dm_warps;
    int ntile_d;
    int cstage;
    int wp;                // bytes per phase row
    int *status;
};

struct __align__(16) RowMeta {
    int base;     // smem byte offset of window sample t0 (may precede the row)
    float ds;     // dmshift of the channel (0 for padding rows)
    int bytes;    // bytes fetched into phase 0 (0: padding row, zero filled)
    int pad;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t mb, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx_arrive(uint32_t mb, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mb, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; false if the limit ran out.
__device__ bool mbar_wait(uint32_t mb, uint32_t parity) {
    if (mbar_try(mb, parity))
        return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try(mb, parity)) {
        if (global_ns() - t0 > kWaitLimitNs)
            return false;
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t mb) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(mb)
        : "memory");
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}

__device__ __forceinline__ uint32_t iadd3(uint32_t a, uint32_t b, uint32_t c) {
    return a + b + c;
}

__device__ __forceinline__ int shift_of(float dm, float ds) {
    return __float2int_rz(__fmul_rn(dm, ds));
}

__device__ __forceinline__ float add_f16_lo(uint32_t x, float acc) {
    float r;
    asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %1; add.rn.f32.f16 %0, lo, %2; }"
        : "=f"(r)
        : "r"(x), "f"(acc));
    return r;
}

__device__ __forceinline__ float add_f16_hi(uint32_t x, float acc) {
    float r;
    asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %1; add.rn.f32.f16 %0, hi, %2; }"
        : "=f"(r)
        : "r"(x), "f"(acc));
    return r;
}

__device__ __forceinline__ void record(int *status, int code) {
    atomicCAS(status, kDevOk, code);
}

// ---------------------------------------------------------------------------
// Output stores.  Word k of lane L covers samples t = tw + (4/ELEM)*(L + 32k) ...
// ---------------------------------------------------------------------------
__device__ __forceinline__ void store4(float *row, int64_t t, int64_t n, float4 v, bool accumulate) {
    if (t + 3 < n) {
        float4 *p = reinterpret_cast<float4 *>(row + t);
        if (accumulate) {
            float4 o = *p;
            v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
        }
        *p = v;
    } else {
        float e[4] = {v.x, v.y, v.z, v.w};
        for (int i = 0; i < 4; ++i)
            if (t + i < n)
                row[t + i] = accumulate ? row[t + i] + e[i] : e[i];
    }
}

// ---------------------------------------------------------------------------
// The kernel.  ELEM = bytes per sample (1, 2, 4); DT = DMs per thread.
// ---------------------------------------------------------------------------
template <int ELEM, int DT>
__global__ void __launch_bounds__(512, 1) dedisperse_kernel(const KArgs a) {
    constexpr int NPH = 4 / ELEM;              // phase copies per row
    constexpr int SPW = 4 / ELEM;              // samples per 4-byte word
    constexpr int SPAN = 32 * kWords * SPW;    // samples per warp
    constexpr int FLUSH = (ELEM == 1) ? kSwarChannels : kFloatBlock;

    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int wdi = warp % a.dm_warps;
    const int wti = warp / a.dm_warps;
    const int time_warps = nthreads / 32 / a.dm_warps;
    const int dm_cta = DT * a.dm_warps;
    const int t_cta = SPAN * time_warps;
    const int td = blockIdx.x % a.ntile_d;
    const int64_t t0 = (int64_t)(blockIdx.x / a.ntile_d) * t_cta;

    const int cstage = a.cstage;
    const int wp = a.wp;
    const int row_bytes = NPH * wp;
    const int stage_bytes = cstage * row_bytes;
    RowMeta *meta = reinterpret_cast<RowMeta *>(smem + 2 * stage_bytes);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + 2 * stage_bytes + 2 * cstage * 16);
    const uint32_t mb0 = smem_addr(&mbar[0]);

    // DM range of this CTA (sorted list) and this thread's DMs.
    const int kcta = td * dm_cta;
    const float dm_min = a.dm_sorted[kcta];
    const float dm_max = a.dm_sorted[kcta + dm_cta - 1];
    const int kthr = kcta + wdi * DT;
    float dm[DT];
#pragma unroll
    for (int j = 0; j < DT; ++j)
        dm[j] = a.dm_sorted[kthr + j];
    const int thr_off = ELEM * (wti * SPAN) + 4 * lane;

    if (tid == 0) {
        mbar_init(mb0, 1);
        mbar_init(mb0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int nstage = (a.nchan + cstage - 1) / cstage;

    // Window of channel c fetched by this CTA: [first, first + bytes/ELEM).
    auto window = [&](int c, int64_t *first, int64_t *bytes) {
        const float ds = a.dmshift[c];
        const int64_t smin = shift_of(dm_min, ds);
        const int64_t smax = shift_of(dm_max, ds);
        *first = (t0 + smin) & ~(int64_t)(16 / ELEM - 1);
        int64_t end = t0 + t_cta + smax;
        if (end > a.nsamp_in)
            end = a.nsamp_in;
        *bytes = ((end - *first) * ELEM + 15) & ~(int64_t)15;
    };

    // Producer: row metadata + one bulk copy per channel row of stage st into
    // buffer b, all completing on that buffer's mbarrier.
    auto issue = [&](int st, int b) {
        RowMeta *m = meta + b * cstage;
        uint8_t *buf = smem + b * stage_bytes;
        uint32_t total = 0;
        bool bad = false;
        for (int r = 0; r < cstage; ++r) {
            const int c = st * cstage + r;
            const int rowstart = (int)(buf + r * row_bytes - smem);
            RowMeta rm;
            rm.pad = 0;
            if (c < a.nchan) {
                int64_t first, bytes;
                window(c, &first, &bytes);
                if (bytes > wp - 16) {  // excluded by the host geometry
                    bad = true;
                    bytes = 0;
                }
                rm.base = rowstart + (int)(ELEM * (t0 - first));
                rm.ds = a.dmshift[c];
                rm.bytes = (int)bytes;
            } else {
                rm.base = rowstart;
                rm.ds = 0.0f;
                rm.bytes = 0;
            }
            m[r] = rm;
            total += (uint32_t)rm.bytes;
        }
        if (bad)
            record(a.status, kDevCheck);
        const uint32_t mb = mb0 + 8 * b;
        mbar_expect_tx_arrive(mb, total);
        for (int r = 0; r < cstage; ++r) {
            const int c = st * cstage + r;
            if (c < a.nchan && m[r].bytes > 0) {
                int64_t first, bytes;
                window(c, &first, &bytes);
                const uint8_t *src = a.in + (int64_t)c * a.in_pitch_b + first * ELEM;
                bulk_g2s(smem_addr(buf + r * row_bytes), src, (uint32_t)m[r].bytes, mb);
            }
        }
    };

    if (tid == 0)
        issue(0, 0);

    // Accumulators.
    uint32_t L1[DT][kWords], L2[DT][kWords];  // uint8 SWAR
    float P[DT][kWords][SPW], S[DT][kWords][SPW], C[DT][kWords][SPW];  // floats
#pragma unroll
    for (int j = 0; j < DT; ++j)
#pragma unroll
        for (int k = 0; k < kWords; ++k) {
            L1[j][k] = 0u;
            L2[j][k] = 0u;
#pragma unroll
            for (int e = 0; e < SPW; ++e) {
                P[j][k][e] = 0.f;
                S[j][k][e] = 0.f;
                C[j][k][e] = 0.f;
            }
        }

    int since_flush = 0;
    bool flushed_once = false;
    const int64_t tw = t0 + (int64_t)wti * SPAN;

    auto flush_u8 = [&]() {
#pragma unroll
        for (int j = 0; j < DT; ++j) {
            const int row = a.perm[kthr + j];
#pragma unroll
            for (int k = 0; k < kWords; ++k) {
                const uint32_t lo = L1[j][k] - (L2[j][k] << 8);
                float4 v = make_float4((float)(lo & 0xffffu), (float)(L2[j][k] & 0xffffu),
                                       (float)(lo >> 16), (float)(L2[j][k] >> 16));
                L1[j][k] = 0u;
                L2[j][k] = 0u;
                if (row >= 0) {
                    const int64_t t = tw + 4 * (lane + 32 * k);
                    if (t < a.nsamp_out)
                        store4(a.out + (int64_t)row * a.out_pitch, t, a.nsamp_out, v,
                               flushed_once);
                }
            }
        }
        flushed_once = true;
    };

    auto block_float = [&]() {
#pragma unroll
        for (int j = 0; j < DT; ++j)
#pragma unroll
            for (int k = 0; k < kWords; ++k)
#pragma unroll
                for (int e = 0; e < SPW; ++e) {
                    // TwoSum(S, P): S + P = s + err exactly.
                    const float p = P[j][k][e];
                    const float s = __fadd_rn(S[j][k][e], p);
                    const float bp = __fsub_rn(s, S[j][k][e]);
                    const float err = __fadd_rn(__fsub_rn(S[j][k][e], __fsub_rn(s, bp)),
                                                __fsub_rn(p, bp));
                    C[j][k][e] = __fadd_rn(C[j][k][e], err);
                    S[j][k][e] = s;
                    P[j][k][e] = 0.f;
                }
    };

    for (int st = 0; st < nstage; ++st) {
        const int b = st & 1;
        const uint32_t mb = mb0 + 8 * b;
        uint8_t *buf = smem + b * stage_bytes;
        const RowMeta *m = meta + b * cstage;

        bool failed = !mbar_wait(mb, (st >> 1) & 1);
        if (!failed) {
            // Padding rows: zeros where the threads will read (shift 0).
            for (int r = 0; r < cstage; ++r) {
                if (m[r].bytes == 0) {
                    uint4 *z = reinterpret_cast<uint4 *>(buf + r * row_bytes);
                    const int n16 = (ELEM * t_cta + 16) / 16;
                    for (int g = tid; g < n16; g += nthreads)
                        z[g] = make_uint4(0, 0, 0, 0);
                }
            }
            // Re-aligned copies of each row (phases 1..NPH-1).
            if (NPH > 1) {
                for (int r = 0; r < cstage; ++r) {
                    const int n16 = m[r].bytes >> 4;
                    uint8_t *ph0 = buf + r * row_bytes;
                    for (int g = tid; g < n16; g += nthreads) {
                        const uint4 v = *reinterpret_cast<const uint4 *>(ph0 + 16 * g);
                        const uint32_t nx = *reinterpret_cast<const uint32_t *>(ph0 + 16 * g + 16);
#pragma unroll
                        for (int p = 1; p < NPH; ++p) {
                            const uint32_t sel = (ELEM == 1)
                                                     ? (0x3210u + 0x1111u * (uint32_t)p)
                                                     : 0x5432u;
                            uint4 o;
                            o.x = prmt(v.x, v.y, sel);
                            o.y = prmt(v.y, v.z, sel);
                            o.z = prmt(v.z, v.w, sel);
                            o.w = prmt(v.w, nx, sel);
                            *reinterpret_cast<uint4 *>(ph0 + p * wp + 16 * g) = o;
                        }
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        if (__syncthreads_or(failed)) {
            record(a.status, kDevTimeout);
            mbar_wait(mb, (st >> 1) & 1);  // let this CTA's copies land before leaving
            return;
        }
        if (tid == 0 && st + 1 < nstage)
            issue(st + 1, b ^ 1);

        // Flush / block boundary before this stage if it would overflow.
        if (since_flush + cstage > FLUSH) {
            if (ELEM == 1)
                flush_u8();
            else
                block_float();
            since_flush = 0;
        }
        since_flush += cstage;

        for (int r = 0; r < cstage; r += 2) {
            const RowMeta m0 = m[r];
            const RowMeta m1 = m[r + 1];
            const int B0 = m0.base + thr_off;
            const int B1 = m1.base + thr_off;
#pragma unroll
            for (int j = 0; j < DT; ++j) {
                const int s0 = shift_of(dm[j], m0.ds);
                const int s1 = shift_of(dm[j], m1.ds);
                const int a0 = B0 + ELEM * s0 + (s0 & (NPH - 1)) * (wp - ELEM);
                const int a1 = B1 + ELEM * s1 + (s1 & (NPH - 1)) * (wp - ELEM);
                const uint32_t *p0 = reinterpret_cast<const uint32_t *>(smem + a0);
                const uint32_t *p1 = reinterpret_cast<const uint32_t *>(smem + a1);
                uint32_t x[kWords], y[kWords];
#pragma unroll
                for (int k = 0; k < kWords; ++k) {
                    x[k] = p0[32 * k];
                    y[k] = p1[32 * k];
                }
#pragma unroll
                for (int k = 0; k < kWords; ++k) {
                    if (ELEM == 1) {
                        L1[j][k] = iadd3(L1[j][k], x[k], y[k]);
                        L2[j][k] = iadd3(L2[j][k], prmt(x[k], 0u, 0x4341u),
                                         prmt(y[k], 0u, 0x4341u));
                    } else if (ELEM == 2) {
                        P[j][k][0] = add_f16_lo(y[k], add_f16_lo(x[k], P[j][k][0]));
                        P[j][k][SPW - 1] = add_f16_hi(y[k], add_f16_hi(x[k], P[j][k][SPW - 1]));
                    } else {
                        P[j][k][0] = __fadd_rn(__fadd_rn(P[j][k][0], __uint_as_float(x[k])),
                                               __uint_as_float(y[k]));
                    }
                }
            }
        }
    }

    if (ELEM == 1) {
        flush_u8();
    } else {
        block_float();
#pragma unroll
        for (int j = 0; j < DT; ++j) {
            const int row = a.perm[kthr + j];
            if (row < 0)
                continue;
            float *orow = a.out + (int64_t)row * a.out_pitch;
#pragma unroll
            for (int k = 0; k < kWords; ++k) {
                const int64_t t = tw + SPW * (lane + 32 * k);
                if (SPW == 1) {
                    if (t < a.nsamp_out)
                        orow[t] = __fadd_rn(S[j][k][0], C[j][k][0]);
                } else {
                    if (t + 1 < a.nsamp_out) {
                        *reinterpret_cast<float2 *>(orow + t) =
                            make_float2(__fadd_rn(S[j][k][0], C[j][k][0]),
                                        __fadd_rn(S[j][k][SPW - 1], C[j][k][SPW - 1]));
                    } else if (t < a.nsamp_out) {
                        orow[t] = __fadd_rn(S[j][k][0], C[j][k][0]);
                    }
                }
            }
        }
    }
}

template <int ELEM, int DT>
cudaError_t launch_t(const KArgs &a, const Geometry &g, int64_t ntiles, cudaStream_t s) {
    auto k = dedisperse_kernel<ELEM, DT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem);
    if (e != cudaSuccess)
        return e;
    k<<<(unsigned)ntiles, g.threads, g.smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

dd_status launch_dedisperse(dd_plan_s *p, const Geometry &g, const DevTables &dt, const void *in,
                            dd_dtype dtype, int64_t in_pitch, int64_t nsamp_in, float *out,
                            int64_t out_pitch, int64_t nsamp_out, void *stream) {
    if (nsamp_out == 0)
        return DD_OK;
    KArgs a;
    a.in = static_cast<const uint8_t *>(in);
    a.in_pitch_b = in_pitch * g.elem;
    a.nsamp_in = nsamp_in;
    a.out = out;
    a.out_pitch = out_pitch;
    a.nsamp_out = nsamp_out;
    a.dmshift = dt.dmshift;
    a.dm_sorted = dt.dm_sorted;
    a.perm = dt.perm;
    a.nchan = p->nchan;
    a.ndm_pad = dt.ndm_pad;
    a.dm_warps = g.tiles.dm_warps;
    a.ntile_d = g.ntile_d;
    a.cstage = g.tiles.chan_per_stage;
    a.wp = g.wp;
    a.status = dt.status;
    const int64_t ntile_t = (nsamp_out + g.t_cta - 1) / g.t_cta;
    const int64_t ntiles = ntile_t * g.ntile_d;
    if (ntiles > 0x7fffffffLL)
        return fail(DD_ERR_INVALID, "too many tiles for one launch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaErrorInvalidValue;
    const int dthr = g.tiles.dm_per_thread;
    switch (dtype) {
    case DD_U8:
        e = dthr == 1 ? launch_t<1, 1>(a, g, ntiles, s)
          : dthr == 2 ? launch_t<1, 2>(a, g, ntiles, s) : launch_t<1, 4>(a, g, ntiles, s);
        break;
    case DD_F16:
        e = dthr == 1 ? launch_t<2, 1>(a, g, ntiles, s)
          : dthr == 2 ? launch_t<2, 2>(a, g, ntiles, s) : launch_t<2, 4>(a, g, ntiles, s);
        break;
    case DD_F32:
        e = dthr == 1 ? launch_t<4, 1>(a, g, ntiles, s)
          : dthr == 2 ? launch_t<4, 2>(a, g, ntiles, s) : launch_t<4, 4>(a, g, ntiles, s);
        break;
    }
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    count_launch();
    return DD_OK;
}

}  // namespace dd
