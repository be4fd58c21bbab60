// Front end (dd_frontend): dual-polarisation voltages -> the uint8 filterbank
// rows dd_execute reads.  The paper's pipeline generates Stokes parameters,
// excises RFI and integrates before the dispersion search (Sec. 1) without
// giving formulas; the library's reading, step by step:
//
//   Stokes I of a raw sample (Xre, Xim, Yre, Yim as int8) = Xre^2 + Xim^2 +
//   Yre^2 + Yim^2 (one dp4a of the sample's word with itself);
//   P[c][t] = sum over raw samples t*nint .. t*nint + nint - 1 (exact);
//   RFI excision by niter passes of sigma clipping: pass i takes the exact
//   count, sum P and sum P^2 over the samples the previous pass kept (all of
//   them for the first), then mean, std and thr = floor(mean + k*std) in
//   FP64; the next pass keeps P <= thr;
//   with the last pass's mean, std and thr: P > thr becomes code 128, else
//   code = clamp(rint(128 + ((float)P - (float)mean) * (float)(16/std)), 0,
//   255) in FP32, one IEEE operation at a time; std == 0 gives 128.
//
// Main path, fused_kernel: one thread-block cluster per channel, its cs CTAs
// (1, 2, 4 or 8) each owning m consecutive output samples.  A CTA streams its
// voltages once (each warp reads 32 samples' bytes in 512-byte coalesced
// steps, the 16-byte words of one sample summed over neighbouring lanes),
// keeps P in shared memory, and every clipping pass sums its own P; the
// cluster's partial sums meet in rank 0's shared memory (distributed shared
// memory, hardware cluster barriers), rank 0 derives the statistics and the
// others read them back.  HBM traffic is the compulsory minimum: 4*nint bytes
// of voltages per output sample in, 1 byte of code out.
//
// Fallback for rows whose P does not fit a cluster's shared memory: P in the
// caller's work array and niter + 1 launches -- power_kernel (one thread per
// output sample; P and pass 1's sums), clip_kernel for passes 2..niter and
// quantize_kernel, each block deriving its channel's statistics from the
// exact sums itself.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "dd_internal.h"

namespace {

constexpr int kThreads = 256;

struct Acc {  // exact per-channel sums of one clipping pass
    unsigned long long cnt, s1, s2;
};

struct Stats {
    double mean, sd;
    long long thr;
};

// The FP64 operations of the definition, in order (no contraction).
__device__ __forceinline__ Stats stats_of(const Acc &a, double k) {
    Stats s;
    double var = 0.0;
    s.mean = 0.0;
    if (a.cnt > 0) {
        const double dc = __ull2double_rn(a.cnt);
        s.mean = __ddiv_rn(__ull2double_rn(a.s1), dc);
        var = __dsub_rn(__ddiv_rn(__ull2double_rn(a.s2), dc), __dmul_rn(s.mean, s.mean));
    }
    if (var < 0.0)
        var = 0.0;
    s.sd = __dsqrt_rn(var);
    s.thr = (long long)floor(__dadd_rn(s.mean, __dmul_rn(k, s.sd)));
    return s;
}

// Block sums of (cnt, s1, s2), then one atomic triple per block.  P <= 2^22,
// so a block's P^2 sum stays below 2^62.
__device__ __forceinline__ void block_accumulate(unsigned long long cnt, unsigned long long s1,
                                                 unsigned long long s2, Acc *dst) {
    __shared__ unsigned long long red[3][kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = cnt;
        red[1][threadIdx.x >> 5] = s1;
        red[2][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cnt = s1 = s2 = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            cnt += red[0][w];
            s1 += red[1][w];
            s2 += red[2][w];
        }
        if (cnt != 0) {
            atomicAdd(&dst->cnt, cnt);
            atomicAdd(&dst->s1, s1);
            atomicAdd(&dst->s2, s2);
        }
    }
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads) power_kernel(const uint8_t *__restrict__ volts,
                                                         int64_t pitch, int64_t n, int64_t prow,
                                                         int nint, uint32_t *__restrict__ p_out,
                                                         Acc *acc) {
    const int c = blockIdx.y;
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    uint32_t p = 0;
    if (t < n) {
        const uint8_t *src = volts + (int64_t)c * pitch + 4 * t * nint;
        if (VEC) {
            for (int j = 0; j < nint; j += 4) {
                const uint4 v = *reinterpret_cast<const uint4 *>(src + 4 * j);
                p += (uint32_t)(__dp4a((int)v.x, (int)v.x, 0) + __dp4a((int)v.y, (int)v.y, 0) +
                                __dp4a((int)v.z, (int)v.z, 0) + __dp4a((int)v.w, (int)v.w, 0));
            }
        } else {
            for (int j = 0; j < nint; ++j) {
                const int v = *reinterpret_cast<const int *>(src + 4 * j);
                p += (uint32_t)__dp4a(v, v, 0);
            }
        }
        p_out[(int64_t)c * prow + t] = p;
    }
    block_accumulate(t < n ? 1ull : 0ull, p, (unsigned long long)p * p, &acc[c]);
}

// One clipping pass: sums over the samples at or below the previous pass's
// threshold.
__global__ void __launch_bounds__(kThreads) clip_kernel(const uint32_t *__restrict__ p_in,
                                                        int64_t n, int64_t prow, double k,
                                                        const Acc *prev, Acc *next) {
    const int c = blockIdx.y;
    __shared__ long long sthr;
    if (threadIdx.x == 0)
        sthr = stats_of(prev[c], k).thr;
    __syncthreads();
    const long long thr = sthr;
    const int64_t t = 4 * ((int64_t)blockIdx.x * kThreads + threadIdx.x);
    unsigned long long cnt = 0, s1 = 0, s2 = 0;
    if (t < n) {
        const uint4 q = *reinterpret_cast<const uint4 *>(p_in + (int64_t)c * prow + t);
        const uint32_t v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (t + i < n && (long long)v[i] <= thr) {
                cnt += 1;
                s1 += v[i];
                s2 += (unsigned long long)v[i] * v[i];
            }
        }
    }
    block_accumulate(cnt, s1, s2, &next[c]);
}

__device__ __forceinline__ uint32_t code_of(uint32_t p, long long thr, float m, float s,
                                            bool flat) {
    if (flat || (long long)p > thr)
        return 128u;
    const float d = __fsub_rn(__uint2float_rn(p), m);
    float v = rintf(__fadd_rn(128.0f, __fmul_rn(d, s)));
    v = v < 0.0f ? 0.0f : (v > 255.0f ? 255.0f : v);
    return (uint32_t)v;
}

__global__ void __launch_bounds__(kThreads) quantize_kernel(const uint32_t *__restrict__ p_in,
                                                            int64_t n, int64_t prow, double k,
                                                            const Acc *last, uint8_t *out,
                                                            int64_t out_pitch, double *mean,
                                                            double *sd) {
    const int c = blockIdx.y;
    __shared__ float sm, ss;
    __shared__ long long sthr;
    __shared__ int sflat;
    if (threadIdx.x == 0) {
        const Stats st = stats_of(last[c], k);
        sm = (float)st.mean;
        sflat = st.sd > 0.0 ? 0 : 1;
        ss = st.sd > 0.0 ? (float)__ddiv_rn(16.0, st.sd) : 0.0f;
        sthr = st.thr;
        if (blockIdx.x == 0) {
            mean[c] = st.mean;
            sd[c] = st.sd;
        }
    }
    __syncthreads();
    const float m = sm, s = ss;
    const long long thr = sthr;
    const bool flat = sflat != 0;
    const int64_t t = 4 * ((int64_t)blockIdx.x * kThreads + threadIdx.x);
    if (t >= n)
        return;
    const uint4 q = *reinterpret_cast<const uint4 *>(p_in + (int64_t)c * prow + t);
    uint8_t *dst = out + (int64_t)c * out_pitch + t;
    if (t + 4 <= n) {
        *reinterpret_cast<uint32_t *>(dst) =
            code_of(q.x, thr, m, s, flat) | code_of(q.y, thr, m, s, flat) << 8 |
            code_of(q.z, thr, m, s, flat) << 16 | code_of(q.w, thr, m, s, flat) << 24;
    } else {
        const uint32_t v[4] = {q.x, q.y, q.z, q.w};
        for (int i = 0; t + i < n; ++i)
            dst[i] = (uint8_t)code_of(v[i], thr, m, s, flat);
    }
}

// ---------------------------------------------------------------------------
// Fused cluster kernel.
// ---------------------------------------------------------------------------

constexpr int kFusedThreads = 512;
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int64_t kFusedSmemTarget = 100 * 1024;  // P bytes per CTA aimed for (2 CTAs per SM)
constexpr int64_t kFusedSmemMax = 200 * 1024;     // P bytes per CTA allowed
constexpr int kMaxCluster = 8;

struct Params {
    long long thr;
    float m, s;
    int flat;
    double mean, sd;
};

// Block sums of (cnt, s1, s2) for kFusedThreads threads, left in red[][0] for
// thread 0.  Callers separate uses by a barrier.
__device__ __forceinline__ void fused_block_sum(unsigned long long v[3],
                                                unsigned long long (*red)[kFusedWarps]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
            v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
            red[i][threadIdx.x >> 5] = v[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            unsigned long long a = 0;
#pragma unroll
            for (int w = 0; w < kFusedWarps; ++w)
                a += red[i][w];
            v[i] = a;
        }
    }
}

__device__ __forceinline__ uint32_t fused_power_word(uint4 v) {
    return (uint32_t)(__dp4a((int)v.x, (int)v.x, 0) + __dp4a((int)v.y, (int)v.y, 0) +
                      __dp4a((int)v.z, (int)v.z, 0) + __dp4a((int)v.w, (int)v.w, 0));
}

// Q = nint/4 16-byte words per output sample (1..16); Q = 0: 4-byte loads,
// one thread per sample (nint < 4 or rows not 16-byte aligned).
template <int Q>
__global__ void __launch_bounds__(kFusedThreads) fused_kernel(
    const uint8_t *__restrict__ volts, int64_t pitch, int64_t n, int nint, int m, double k,
    int niter, uint8_t *__restrict__ out, int64_t out_pitch, double *mean_out, double *sd_out) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    const unsigned cs = cluster.num_blocks();
    const int c = blockIdx.x / cs;
    extern __shared__ uint4 fused_smem[];
    uint32_t *P = reinterpret_cast<uint32_t *>(fused_smem);
    __shared__ unsigned long long red[3][kFusedWarps];
    __shared__ unsigned long long part[3];
    __shared__ Params prm;

    const int64_t t0 = (int64_t)rank * m;
    const int len = (int)(n - t0 < 0 ? 0 : (n - t0 < m ? n - t0 : m));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long acc[3] = {0, 0, 0};

    // Pass 1: P = integrated Stokes I, kept in shared memory.
    if (Q > 0) {
        constexpr int QD = Q > 0 ? Q : 1;  // Q, without a zero divisor in the Q = 0 body
        const uint4 *row = reinterpret_cast<const uint4 *>(volts + (int64_t)c * pitch) + t0 * QD;
        constexpr int U = QD >= 8 ? 1 : 2;  // groups of 32 samples in flight per warp
        for (int g0 = warp * 32; g0 < len; g0 += kFusedWarps * 32 * U) {
            uint4 v[U][QD];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int g = g0 + u * kFusedWarps * 32;
#pragma unroll
                for (int j = 0; j < QD; ++j) {
                    const int ci = lane + 32 * j;
                    if (g + ci / QD < len)
                        v[u][j] = __ldcs(row + (int64_t)g * QD + ci);
                    else
                        v[u][j] = make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int g = g0 + u * kFusedWarps * 32;
#pragma unroll
                for (int j = 0; j < QD; ++j) {
                    uint32_t p = fused_power_word(v[u][j]);
#pragma unroll
                    for (int o = QD / 2; o > 0; o >>= 1)
                        p += __shfl_xor_sync(0xffffffffu, p, o);
                    const int sl = g + (32 * j + lane) / QD;
                    if (lane % QD == 0 && sl < len) {
                        P[sl] = p;
                        acc[1] += p;
                        acc[2] += (unsigned long long)p * p;
                    }
                }
            }
        }
    } else {
        const uint8_t *row = volts + (int64_t)c * pitch + 4 * t0 * nint;
        for (int sl = tid; sl < len; sl += kFusedThreads) {
            const int *src = reinterpret_cast<const int *>(row + (int64_t)4 * nint * sl);
            uint32_t p = 0;
            for (int j = 0; j < nint; ++j) {
                const int w = __ldcs(src + j);
                p += (uint32_t)__dp4a(w, w, 0);
            }
            P[sl] = p;
            acc[1] += p;
            acc[2] += (unsigned long long)p * p;
        }
    }
    acc[0] = tid == 0 ? (unsigned long long)len : 0ull;

    long long thr = 0;
    Params pr;
    for (int it = 0; it < niter; ++it) {
        if (it > 0) {
            acc[0] = acc[1] = acc[2] = 0;
            for (int sl = tid; sl < len; sl += kFusedThreads) {
                const uint32_t p = P[sl];
                if ((long long)p <= thr) {
                    acc[0] += 1;
                    acc[1] += p;
                    acc[2] += (unsigned long long)p * p;
                }
            }
        }
        fused_block_sum(acc, red);
        if (tid == 0) {
            part[0] = acc[0];
            part[1] = acc[1];
            part[2] = acc[2];
        }
        cluster.sync();  // every rank's part is written
        if (rank == 0 && tid == 0) {
            Acc a = {0, 0, 0};
            for (unsigned q = 0; q < cs; ++q) {
                const unsigned long long *rp = cluster.map_shared_rank(part, q);
                a.cnt += rp[0];
                a.s1 += rp[1];
                a.s2 += rp[2];
            }
            const Stats st = stats_of(a, k);
            prm.thr = st.thr;
            prm.mean = st.mean;
            prm.sd = st.sd;
            prm.flat = st.sd > 0.0 ? 0 : 1;
            prm.m = (float)st.mean;
            prm.s = st.sd > 0.0 ? (float)__ddiv_rn(16.0, st.sd) : 0.0f;
        }
        cluster.sync();  // rank 0's prm is written; part may be reused after the next sum
        pr = *cluster.map_shared_rank(&prm, 0);
        thr = pr.thr;
    }
    // Rank 0 keeps its shared memory until every rank has read prm.
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    if (rank == 0 && tid == 0) {
        mean_out[c] = pr.mean;
        sd_out[c] = pr.sd;
    }
    const bool flat = pr.flat != 0;
    uint8_t *dst = out + (int64_t)c * out_pitch + t0;
    for (int sl = 4 * tid; sl < len; sl += 4 * kFusedThreads) {
        if (sl + 4 <= len) {
            const uint4 q = *reinterpret_cast<const uint4 *>(P + sl);
            *reinterpret_cast<uint32_t *>(dst + sl) =
                code_of(q.x, thr, pr.m, pr.s, flat) | code_of(q.y, thr, pr.m, pr.s, flat) << 8 |
                code_of(q.z, thr, pr.m, pr.s, flat) << 16 |
                code_of(q.w, thr, pr.m, pr.s, flat) << 24;
        } else {
            for (int i = sl; i < len; ++i)
                dst[i] = (uint8_t)code_of(P[i], thr, pr.m, pr.s, flat);
        }
    }
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Samples per CTA for a cluster of cs CTAs: a multiple of 32 (so every CTA's
// first sample starts a warp group and a 4-byte output word).
int64_t fused_m(int64_t n, int cs) { return ((n + cs - 1) / cs + 31) / 32 * 32; }

template <int Q>
cudaError_t launch_fused_q(int cs, int64_t m, const uint8_t *v, int64_t pitch, int64_t n,
                           int nint, int nchan, double k, int niter, uint8_t *out,
                           int64_t out_pitch, double *mean, double *sd, cudaStream_t s,
                           bool *fits) {
    static unsigned long long attr_set = 0;  // per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev >= 64 || !((attr_set >> dev) & 1ull)) {
        e = cudaFuncSetAttribute(fused_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kFusedSmemMax);
        if (e != cudaSuccess)
            return e;
        if (dev < 64)
            attr_set |= 1ull << dev;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nchan * cs));
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = (size_t)(4 * m);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, fused_kernel<Q>, &cfg);
    if (e != cudaSuccess || clusters < 1) {
        (void)cudaGetLastError();  // not an error of the call: leave it to the fallback path
        *fits = false;
        return cudaSuccess;
    }
    *fits = true;
    return cudaLaunchKernelEx(&cfg, fused_kernel<Q>, v, pitch, n, nint, (int)m, k, niter, out,
                              out_pitch, mean, sd);
}

bool frontend_shape_ok(int nchan, int64_t nsamp_raw, int nint, int niter) {
    return nchan >= 1 && nchan <= 65535 && nsamp_raw >= 0 && nint >= 1 && nint <= 64 &&
           (nint & (nint - 1)) == 0 && niter >= 1 && niter <= 8 &&
           nsamp_raw / nint <= (1LL << 19);
}

// P rows hold a whole number of 16-byte groups.
int64_t p_row(int64_t n) { return (n + 3) / 4 * 4; }

}  // namespace

extern "C" int64_t dd_frontend_work_bytes(int nchan, int64_t nsamp_raw, int nint, int niter) {
    if (!frontend_shape_ok(nchan, nsamp_raw, nint, niter))
        return -1;
    return 4 * (int64_t)nchan * p_row(nsamp_raw / nint) + (int64_t)sizeof(Acc) * niter * nchan;
}

extern "C" dd_status dd_frontend(const void *volts, int64_t volts_pitch, int nchan,
                                 int64_t nsamp_raw, int nint, double k_clip, int niter,
                                 uint8_t *out, int64_t out_pitch, void *work, int64_t work_bytes,
                                 double *mean, double *std_out, void *stream) {
    dd::Range nvtx_range("dd_frontend");
    using dd::fail;
    if (!frontend_shape_ok(nchan, nsamp_raw, nint, niter))
        return fail(DD_ERR_INVALID, "need 1 <= nchan <= 65535, nsamp_raw >= 0, nint a power of "
                                    "two <= 64, 1 <= niter <= 8, nsamp_raw/nint <= 2^19");
    const int64_t n = nsamp_raw / nint;
    if (volts_pitch < 4 * nsamp_raw || volts_pitch % 4 != 0 || out_pitch < n || out_pitch % 16)
        return fail(DD_ERR_INVALID, "volts_pitch >= 4*nsamp_raw (multiple of 4); out_pitch >= "
                                    "nsamp_raw/nint (multiple of 16)");
    // The bound keeps floor(mean + k_clip*std) inside int64 for any P.
    if (!(k_clip > 0.0 && k_clip <= 1e9))
        return fail(DD_ERR_INVALID, "k_clip must be in (0, 1e9]");
    if (!mean || !std_out || ((uintptr_t)mean & 7u) || ((uintptr_t)std_out & 7u))
        return fail(DD_ERR_INVALID, "NULL or misaligned mean/std pointer");
    if (n > 0 && (!volts || !out || !work || ((uintptr_t)volts & 3u) || ((uintptr_t)out & 15u) ||
                  ((uintptr_t)work & 15u)))
        return fail(DD_ERR_INVALID, "NULL or misaligned volts/out/work pointer");
    if (n > 0 && work_bytes < dd_frontend_work_bytes(nchan, nsamp_raw, nint, niter))
        return fail(DD_ERR_INVALID, "work is smaller than dd_frontend_work_bytes");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (n == 0) {  // no output samples: mean and std are 0
        e = cudaMemsetAsync(mean, 0, sizeof(double) * nchan, s);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(std_out, 0, sizeof(double) * nchan, s);
        if (e != cudaSuccess)
            return fail(DD_ERR_CUDA, std::string("frontend memset: ") + cudaGetErrorString(e));
        return DD_OK;
    }
    const uint8_t *v = static_cast<const uint8_t *>(volts);
    const bool vec = nint % 4 == 0 && ((uintptr_t)volts & 15u) == 0 && volts_pitch % 16 == 0;
    int cs = 1;
    while (cs < kMaxCluster && 4 * fused_m(n, cs) > kFusedSmemTarget)
        cs *= 2;
    if (4 * fused_m(n, cs) <= kFusedSmemMax) {
        const int64_t m = fused_m(n, cs);
        bool fits = false;
        const int q = vec ? nint / 4 : 0;
        switch (q) {
#define DD_FE_CASE(QQ)                                                                       \
    case QQ:                                                                                 \
        e = launch_fused_q<QQ>(cs, m, v, volts_pitch, n, nint, nchan, k_clip, niter, out,     \
                               out_pitch, mean, std_out, s, &fits);                          \
        break;
            DD_FE_CASE(0)
            DD_FE_CASE(1)
            DD_FE_CASE(2)
            DD_FE_CASE(4)
            DD_FE_CASE(8)
            DD_FE_CASE(16)
#undef DD_FE_CASE
        default:
            return fail(DD_ERR_INVALID, "frontend: no kernel for this nint");
        }
        if (e != cudaSuccess)
            return fail(DD_ERR_CUDA, std::string("frontend launch: ") + cudaGetErrorString(e));
        if (fits) {
            dd::count_launch(1);
            return DD_OK;
        }
    }
    const int64_t prow = p_row(n);
    auto *p = static_cast<uint32_t *>(work);
    auto *acc = reinterpret_cast<Acc *>(static_cast<uint8_t *>(work) + 4 * nchan * prow);
    e = cudaMemsetAsync(acc, 0, sizeof(Acc) * niter * nchan, s);
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("frontend memset: ") + cudaGetErrorString(e));
    const dim3 g1((unsigned)((n + kThreads - 1) / kThreads), (unsigned)nchan);
    // 16-byte loads need 16-byte aligned rows and whole groups of 4 samples.
    if (vec)
        power_kernel<true><<<g1, kThreads, 0, s>>>(v, volts_pitch, n, prow, nint, p, acc);
    else
        power_kernel<false><<<g1, kThreads, 0, s>>>(v, volts_pitch, n, prow, nint, p, acc);
    e = cudaGetLastError();
    const dim3 g4((unsigned)((n + 4 * kThreads - 1) / (4 * kThreads)), (unsigned)nchan);
    for (int it = 1; it < niter && e == cudaSuccess; ++it) {
        clip_kernel<<<g4, kThreads, 0, s>>>(p, n, prow, k_clip, acc + (int64_t)(it - 1) * nchan,
                                            acc + (int64_t)it * nchan);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        quantize_kernel<<<g4, kThreads, 0, s>>>(p, n, prow, k_clip,
                                                acc + (int64_t)(niter - 1) * nchan, out,
                                                out_pitch, mean, std_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("frontend launch: ") + cudaGetErrorString(e));
    dd::count_launch(niter + 1);
    return DD_OK;
}
