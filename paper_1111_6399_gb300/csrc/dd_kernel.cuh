// Brute-force incoherent de-dispersion kernels for sm_103a (GB300).
//
//   out[d][t] = sum_c in[c][t + s(c,d)],   s(c,d) = trunc(dm[d] * dmshift[c])
//
// Sec. 3 of the paper sets three rules: accumulators in the fastest memory,
// the right (f,t) data always next to the SMs, and few operations for the
// shift.  Their sm_103a form here:
//
//  * Accumulators in registers.  A consumer thread owns dm_per_thread trial
//    DMs x 4 or 8 four-byte words of output time (16 or 32 uint8 samples),
//    lane-interleaved so each shared-memory read of a warp covers 32
//    consecutive banks.  A tile -- one CTA's work item -- is a rectangle of
//    (DM,t) (Fig. 2).
//  * Data next to the SMs.  A producer warp stages each channel's window
//    [t0 + s(c,dm_min), t0 + T + s(c,dm_max)) with TMA bulk copies (no
//    multicast) into a ring of shared-memory stages.  Shifts are arbitrary in
//    bytes while shared-memory words are 4-byte aligned, so for 8/16-bit data
//    every staged row is kept once per byte phase (advanced by 1..3 bytes, or
//    by one FP16 sample): the copy brings phase 0 and builder warps derive the
//    other phases from it in shared memory with byte permutes, so HBM and L2
//    carry each window once.  Every shifted read is then an aligned,
//    conflict-free LDS.32.  Stages pass producer -> builders -> consumers ->
//    producer through raw/full/empty mbarriers, so copies and phase building
//    run ahead of the arithmetic and no CTA-wide barrier sits in the loop.
//  * Shift arithmetic.  The producer computes, per staged channel and DM of
//    the tile, the shared-memory offset of the shifted window (one FP32
//    multiply and one truncation) into a small table; consumers fetch the
//    offsets of a channel pair with one LDS.64.
//  * uint8 sums use 16-bit SWAR lanes: for a word x of 4 samples, L1 += x and
//    L2 += (x >> 8) & 0x00ff00ff.  After at most 256 channels
//    L2 = {sum b1, sum b3} and L1 - 256*L2 = {sum b0, sum b2} exactly; these are
//    widened into the FP32 output (exact: every sum < 2^24).  Per word and two
//    channels: 2 LDS + 1 IADD3 (ALU) + 2 PRMT (ALU) + 2 IMAD (FMA pipe), which
//    balances the integer ALU and FMA pipes.
//  * FP16/FP32 sums: FP32 partials over blocks of 64 channels, combined into a
//    running sum with TwoSum compensation (error ~1e-7 of sum |in|).
//
// Work distribution.  The producer decides which tile the CTA works on and
// tags every stage with it (beam, DM tile, first sample, stage number); the
// builders and consumers follow that stream until a terminating stage.  A
// single-beam launch gives each CTA one tile (blockIdx.x); a batch launch is
// persistent (one CTA per SM) and the producer claims tiles of many beams,
// largest first, from an atomic counter.
//
// Every mbarrier wait is bounded by the global timer; a wait that runs out
// records a timeout in the status word and the thread leaves (the producer
// first waits, again bounded, for the copies it issued).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "dd_detect_seg.cuh"
#include "dd_kargs.h"
#include "dd_internal.h"

namespace dd {
namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

// Stage record written by the producer before it releases a stage.
struct __align__(16) StageMeta {
    int beam;     // -1: no more tiles
    int td;       // DM tile
    int st;       // stage number within the tile
    int nstage;   // stages of the tile
    int64_t t0;   // first output sample of the tile
    int64_t pad;
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

__device__ __forceinline__ void mbar_expect_tx(uint32_t mb, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mb) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
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

// Bounded wait for the completion of the phase with the given parity.  The
// waiting warp backs off with __nanosleep (64 ns doubling to 1 us) so it does
// not take issue slots from the warps that share its scheduler; the global
// timer is read every 16 tries.
__device__ __noinline__ bool mbar_wait_slow(uint32_t mb, uint32_t parity, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    uint32_t ns = 64;
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(mb, parity))
            return true;
        __nanosleep(ns);
        ns = ns < 1024u ? 2u * ns : 1024u;
        if ((i & 15u) == 0 && global_ns() - t0 > limit_ns)
            return false;
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity,
                                          uint64_t limit_ns = kWaitLimitNs) {
    return mbar_try(mb, parity) || mbar_wait_slow(mb, parity, limit_ns);
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

// acc + p on the FMA pipe (p * one + acc with one == 1 at run time).
__device__ __forceinline__ uint32_t imad_acc(uint32_t p, uint32_t one, uint32_t acc) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(p), "r"(one), "r"(acc));
    return r;
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

// Tensor-memory (TMEM) access of one warp: N consecutive 32-bit columns of
// its 32 lanes (thread i: lane i).  The FP16/FP32 consumers keep their
// running sums and compensations there (written and read once per block of
// channels).
template <int N>
__device__ __forceinline__ void tm_ld(uint32_t taddr, uint32_t (&v)[N]) {
    static_assert(N == 4 || N == 8 || N == 16, "TMEM load width");
    if constexpr (N == 4)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                     : "r"(taddr)
                     : "memory");
    else if constexpr (N == 8)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, "
                     "[%8];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                       "=r"(v[6]), "=r"(v[7])
                     : "r"(taddr)
                     : "memory");
    else
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, "
                     "%8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                       "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                       "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                     : "r"(taddr)
                     : "memory");
}

template <int N>
__device__ __forceinline__ void tm_st(uint32_t taddr, const uint32_t (&v)[N]) {
    static_assert(N == 4 || N == 8 || N == 16, "TMEM store width");
    if constexpr (N == 4)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
                     "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
                     : "memory");
    else if constexpr (N == 8)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, "
                     "%8};" ::"r"(taddr),
                     "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                     "r"(v[7])
                     : "memory");
    else
        asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, "
                     "%8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
                     "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                     "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]),
                     "r"(v[13]), "r"(v[14]), "r"(v[15])
                     : "memory");
}

__device__ __forceinline__ void tm_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Registers written by tcgen05.ld hold their values only after
// tcgen05.wait::ld, which the compiler does not know: after each wait the
// loaded registers pass through an empty volatile asm that redefines them, so
// no use of them can be scheduled above the wait.
template <int N>
__device__ __forceinline__ void reg_fence(uint32_t (&v)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i)
        asm volatile("" : "+r"(v[i]));
}

// TMEM columns the FP16/FP32 consumers of a <DT, NW> kernel allocate: per
// warp the running sums S (DT * NW * samples per word) and compensations C
// (DT * NW: one FP32 word, or for FP16 one packed bf16 pair, per output
// word), for up to ceil(max_consumer_warps / 4) warps per lane quarter,
// rounded up to a power of two (at least 32).
DD_HD constexpr int tm_sum_cols(int elem, int dt, int nw) { return dt * nw * (4 / elem) + dt * nw; }
DD_HD constexpr int tm_alloc_cols(int elem, int dt, int nw) {
    const int need = ((max_consumer_warps(dt, nw) + 3) / 4) * tm_sum_cols(elem, dt, nw);
    int c = 32;
    while (c < need)
        c *= 2;
    return c;
}

// Store (first widening of a uint8 SWAR block) or add (later blocks) four
// exact integer sums to out[t..t+3].  Later blocks use fire-and-forget
// vector reductions: the values are integers below 2^24, so FP32 addition is
// exact in any order and the thread does not wait for the old values.
__device__ __forceinline__ void store4(float *row, int64_t t, int64_t n, float4 v,
                                       bool accumulate) {
    if (t + 3 < n) {
        float4 *p = reinterpret_cast<float4 *>(row + t);
        if (accumulate)
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x),
                         "f"(v.y), "f"(v.z), "f"(v.w)
                         : "memory");
        else
            *p = v;
    } else {
        const float e[4] = {v.x, v.y, v.z, v.w};
        for (int i = 0; i < 4; ++i)
            if (t + i < n) {
                if (accumulate)
                    atomicAdd(row + t + i, e[i]);
                else
                    row[t + i] = e[i];
            }
    }
}

__device__ __forceinline__ const BeamArgs &beam_at(const KArgs &a, int i) {
    return a.beams ? a.beams[i] : a.beam0;
}

// Beam owning global tile `tile` (beams are laid out by increasing tile_begin).
__device__ __forceinline__ int beam_of_tile(const KArgs &a, int64_t tile) {
    if (a.beams == nullptr)
        return 0;
    int lo = 0, hi = a.nbeams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.beams[mid].tile_begin <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Fused detection: the boxcar search of dd_detect run on a finished tile of
// the plane (DMs kcta .. kcta + dm_cta - 1, samples t0 .. t0 + 1023) by the
// consumer warps of the CTA that computed it, reading the tile back from L2.
// Boxcar start positions are split so that each is searched once:
//   * [t0, t0 + 768) by tile k itself (every window ends inside the tile);
//   * [t0 - 256, t0) -- windows across the boundary with tile k - 1 -- by
//     whichever of the two tiles finishes second (an atomic counter per
//     boundary: the tile that finds it at 1 searches it; both tiles' values
//     are then final and visible);
//   * the last tile of a row searches [t0, nsamp) whole.
// The sums S1, S2 of the searched positions' samples and the keys go to the
// same accumulators as dd_detect's, so its finalize step completes the
// search.  Returns false if a bounded wait ran out (recorded).
// ---------------------------------------------------------------------------
__device__ __noinline__ bool detect_epilogue(const KArgs &a, int td, int64_t t0, int dm_cta,
                                             int t_cta, int ncw, int warp, int lane, int tid,
                                             uint32_t ep_bar, int *ep_flags) {
    const BeamArgs &B = a.beam0;
    // Every consumer's stores and reductions of the tile are visible before
    // the counters or any search read them.
    __threadfence();
    __syncwarp();
    if (lane == 0)
        mbar_arrive(ep_bar);
    if (!mbar_wait(ep_bar, 0)) {
        record(a.status, kDevTimeout);
        return false;
    }
    const int K = a.det_ntile_t;
    const int k = (int)(t0 / t_cta);
    if (tid == 0) {
        int *cnt = a.det_cnt + (int64_t)td * K;
        __threadfence();
        const int left = k > 0 ? (atomicAdd(&cnt[k], 1) == 1) : 0;
        const int right = k + 1 < K ? (atomicAdd(&cnt[k + 1], 1) == 1) : 0;
        __threadfence();
        ep_flags[0] = left;
        ep_flags[1] = right;
    }
    __syncwarp();
    if (lane == 0)
        mbar_arrive(ep_bar);
    if (!mbar_wait(ep_bar, 1)) {
        record(a.status, kDevTimeout);
        return false;
    }
    const bool left = ep_flags[0] != 0, right = ep_flags[1] != 0;
    const int64_t n = B.nsamp_out;
    const int nl = a.det_nlevels;
    for (int it = warp; it < 3 * dm_cta; it += ncw) {
        const int j = it / 3, part = it % 3;
        const int row = B.perm[td * dm_cta + j];
        if (row < 0 || (part == 1 && !left) || (part == 2 && !right))
            continue;
        const float *x = B.out + (int64_t)row * B.out_pitch;
        if (part == 0 && k + 1 == K) {
            detect_segment<true, true, 32, true>(x, n, t0, row, nl, lane, a.one, a.det_s1,
                                                 a.det_s2, a.det_keys);
        } else if (part == 0) {
            // loads reach 32 * (24 + kReach) samples from t0
            if (t0 + 32 * (24 + kReach) <= n)
                detect_segment<true, false, 24, true>(x, n, t0, row, nl, lane, a.one, a.det_s1,
                                                      a.det_s2, a.det_keys);
            else
                detect_segment<true, true, 24, true>(x, n, t0, row, nl, lane, a.one, a.det_s1,
                                                     a.det_s2, a.det_keys);
        } else {
            const int64_t s0 = part == 1 ? t0 - 256 : t0 + 768;
            detect_segment<true, true, 8, true>(x, n, s0, row, nl, lane, a.one, a.det_s1,
                                                a.det_s2, a.det_keys);
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// The de-dispersion kernel.  ELEM = bytes per sample (1, 2, 4); DT = DMs per
// consumer thread; NW = 4-byte words per DM per consumer thread (4 or 8).
// Warps 0..ncw-1 consume, warp ncw produces, warps ncw+1.. build phases.
// ---------------------------------------------------------------------------
// DET: the uint8 form that also searches the finished plane for pulses
// (fused detection, see detect_epilogue below).
template <int ELEM, int DT, int NW, bool DET = false, int CS = 0>
__global__ void __launch_bounds__(32 * (max_consumer_warps(DT, NW) + 1 + (ELEM < 4 ? kMaxBuilders : 0)), 1)
    dedisperse_kernel(const __grid_constant__ KArgs a) {
    constexpr int NPH = 4 / ELEM;            // phase copies per row
    constexpr bool BUILD = NPH > 1;          // phases 1.. are built in shared memory
    constexpr int SPW = 4 / ELEM;            // samples per 4-byte word
    constexpr int SPAN = 32 * NW * SPW;      // samples per warp
    constexpr int FLUSH = (ELEM == 1) ? kSwarChannels : kFloatBlock;

    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int ncw = a.dm_warps * a.time_warps;  // consumer warps
    const int dm_cta = DT * a.dm_warps;
    const int t_cta = SPAN * a.time_warps;

    const int cstage = CS > 0 ? CS : a.cstage;  // CS: channels per stage fixed at compile time
    const int nst = a.nstages;
    const int stage_bytes = a.stage_bytes;
    const int tab_stride = cstage * dm_cta;  // ints per stage in the offset table
    int *atab = reinterpret_cast<int *>(smem + nst * stage_bytes);
    StageMeta *meta = reinterpret_cast<StageMeta *>(
        smem + nst * stage_bytes + ((nst * tab_stride * 4 + 15) & ~15));
    // Bytes staged for each row of each stage (phase 0), for the builders.
    uint32_t *rowb = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(meta) +
                                                  nst * kStageMetaBytes);
    uint8_t *zero = reinterpret_cast<uint8_t *>(rowb) + (BUILD ? nst * kRowInfoBytes : 0);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(zero + a.zero_bytes);
    const uint32_t full0 = smem_addr(&mbar[0]);
    const uint32_t empty0 = smem_addr(&mbar[nst]);
    const uint32_t raw0 = smem_addr(&mbar[2 * nst]);
    // Fused detection: a barrier of the consumer warps and two flags.
    const uint32_t ep_bar = smem_addr(&mbar[3 * nst]);
    int *ep_flags = reinterpret_cast<int *>(&mbar[3 * nst + 1]);
    // The producer hands a stage to the builders (raw) or, without phases to
    // build, straight to the consumers (full).
    const uint32_t hand0 = BUILD ? raw0 : full0;
    const int nbw = BUILD ? a.builders : 0;
    const int zero_off = (int)(zero - smem);

    for (int i = tid; i < a.zero_bytes / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(zero)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int b = 0; b < nst; ++b) {
            mbar_init(full0 + 8 * b, BUILD ? nbw : 1);
            mbar_init(empty0 + 8 * b, ncw);
            mbar_init(raw0 + 8 * b, 1);
        }
        if (DET || ELEM > 1)
            mbar_init(ep_bar, ncw);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // FP16/FP32: consumer warp 0 allocates the TMEM of the running sums (the
    // address goes to the epilogue slot of shared memory) and frees it at the
    // end.  If another CTA on the SM holds too many columns the allocation
    // waits until it finishes.
    constexpr int TM_COLS = tm_alloc_cols(ELEM, DT, NW);
    uint32_t *tm_slot = reinterpret_cast<uint32_t *>(ep_flags);
    if constexpr (ELEM > 1) {
        static_assert(TM_COLS <= 512, "TMEM columns of the running sums");
        if (warp == 0) {
            asm volatile(
                "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                    smem_addr(tm_slot)),
                "n"(TM_COLS)
                : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
    }
    __syncthreads();

    if (warp == ncw) {
        // ------------------------------ producer ------------------------------
        int64_t g = 0;  // ring position of the next stage
        // g % nst and (g / nst) & 1, advanced with g (no division in the
        // stage loop)
        int gb = 0;
        uint32_t gpar = 0u;
        bool ok = true;
        bool first = true;
        for (;;) {
            int64_t tile;
            if (a.tile_counter) {
                int t = 0;
                if (lane == 0)
                    t = atomicAdd(a.tile_counter, 1);
                tile = __shfl_sync(0xffffffffu, t, 0);
            } else {
                tile = first ? (int64_t)blockIdx.x : a.total_tiles;
            }
            first = false;
            if (tile >= a.total_tiles)
                break;
            const int bi = beam_of_tile(a, tile);
            const BeamArgs &B = beam_at(a, bi);
            const int64_t local = tile - B.tile_begin;
            const int td = (int)(local % B.ntile_d);
            const int64_t t0 = (local / B.ntile_d) * t_cta;
            const int kcta = td * dm_cta;
            const int wp = B.wp;
            const int row_bytes = NPH * wp;
            const int nstage = (B.nchan + cstage - 1) / cstage;
            const float dm_min = B.dm_sorted[kcta];
            const float dm_max = B.dm_sorted[kcta + dm_cta - 1];
            float dmk[2];  // DM columns lane and lane + 32 (dm_cta <= 64, host-checked)
            dmk[0] = B.dm_sorted[kcta + min(lane, dm_cta - 1)];
            dmk[1] = B.dm_sorted[kcta + min(lane + 32, dm_cta - 1)];
            // dmshift of the rows of the next stage (lane r: rows r and r + 32),
            // loaded one stage ahead so the load latency overlaps the empty wait.
            float ds_next[2];
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                ds_next[h] = (lane + 32 * h < cstage && c < B.nchan) ? B.dmshift[c] : 0.0f;
            }
            for (int st = 0; st < nstage; ++st, ++g) {
                const int b = gb;
                const uint32_t par = gpar;
                if (++gb == nst) {
                    gb = 0;
                    gpar ^= 1u;
                }
                const float ds_cur[2] = {ds_next[0], ds_next[1]};
                for (int h = 0; h < 2; ++h) {
                    const int c = (st + 1) * cstage + lane + 32 * h;
                    ds_next[h] = (st + 1 < nstage && lane + 32 * h < cstage && c < B.nchan)
                                     ? B.dmshift[c] : 0.0f;
                }
                if (g >= nst && !mbar_wait(empty0 + 8 * b, par ^ 1u)) {
                    ok = false;
                    break;
                }
                uint8_t *buf = smem + b * stage_bytes;
                int *tab = atab + b * tab_stride;
                uint32_t my_bytes[2] = {0u, 0u};
                int64_t my_first[2] = {0, 0};
                int my_base[2] = {zero_off, zero_off};
                float my_ds[2] = {0.0f, 0.0f};
                bool bad = false;
                // Window of each staged row (lane r holds rows r and r + 32).
                for (int h = 0; h < 2; ++h) {
                    const int r = lane + 32 * h;
                    const int c = st * cstage + r;
                    if (r >= cstage || c >= B.nchan)
                        continue;
                    const float ds = ds_cur[h];
                    const int64_t smin = shift_of(dm_min, ds);
                    const int64_t smax = shift_of(dm_max, ds);
                    const int64_t firsts = (t0 + smin) & ~(int64_t)(16 / ELEM - 1);
                    int64_t end = t0 + t_cta + smax;
                    if (end > B.nsamp_in)
                        end = B.nsamp_in;
                    const int64_t bytes = ((end - firsts) * ELEM + 15) & ~(int64_t)15;
                    if (bytes > wp - 16 || bytes <= 0 || cstage * row_bytes > stage_bytes) {
                        bad = true;  // excluded by the host checks
                        continue;
                    }
                    my_base[h] = (int)(buf + r * row_bytes - smem) + (int)(ELEM * (t0 - firsts));
                    my_ds[h] = ds;
                    my_bytes[h] = (uint32_t)bytes;
                    my_first[h] = firsts;
                }
                if (bad)
                    record(a.status, kDevCheck);
                if (lane == 0) {
                    StageMeta m;
                    m.beam = bi;
                    m.td = td;
                    m.st = st;
                    m.nstage = nstage;
                    m.t0 = t0;
                    m.pad = 0;
                    meta[b] = m;
                }
                // Copies first: the expected byte count is registered without an
                // arrival, the copies are issued, and the offset table is written
                // while they are in flight; the arrival then releases the stage
                // (the phase completes once it and every byte are in).
                uint32_t total = my_bytes[0] + my_bytes[1];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    total += __shfl_xor_sync(0xffffffffu, total, o);
                if (lane == 0)
                    mbar_expect_tx(hand0 + 8 * b, total);
                __syncwarp();
                for (int h = 0; h < 2; ++h) {
                    const int r = lane + 32 * h;
                    if (BUILD && r < cstage)
                        rowb[b * (kRowInfoBytes / 4) + r] = my_bytes[h];
                    if (r >= cstage || my_bytes[h] == 0)
                        continue;
                    const int c = st * cstage + r;
                    const int64_t off = (int64_t)c * B.in_pitch_b + my_first[h] * ELEM;
                    bulk_g2s(smem_addr(buf + r * row_bytes), B.in + off, my_bytes[h], hand0 + 8 * b);
                }
                // Offset table: row r, DM k -> smem offset of the shifted window.
                for (int r = 0; r < cstage; ++r) {
                    const int base = __shfl_sync(0xffffffffu, my_base[r >> 5], r & 31);
                    const float ds = __shfl_sync(0xffffffffu, my_ds[r >> 5], r & 31);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k = lane + 32 * h;
                        if (k < dm_cta) {
                            const int s = shift_of(dmk[h], ds);
                            // pair layout [r/2][k][r%2]: one LDS.64 gives both rows
                            tab[((r >> 1) * dm_cta + k) * 2 + (r & 1)] =
                                base + ELEM * s + (s & (NPH - 1)) * (wp - ELEM);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(hand0 + 8 * b);
            }
            if (!ok)
                break;
        }
        const int64_t real = g;  // stages handed to the consumers
        if (ok) {
            // Terminating stage: tells the consumers there is no further tile.
            const int b = (int)(g % nst);
            const int64_t n = g / nst;
            if (n > 0 && !mbar_wait(empty0 + 8 * b, (uint32_t)((n - 1) & 1))) {
                ok = false;
            } else {
                if (lane == 0) {
                    StageMeta m;
                    m.beam = -1;
                    m.td = m.st = m.nstage = 0;
                    m.t0 = 0;
                    m.pad = 0;
                    meta[b] = m;
                }
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(hand0 + 8 * b);
            }
        }
        if (!ok)
            record(a.status, kDevTimeout);
        // Leave only once the last stages handed over have landed (and,
        // normally, been released by the consumers); bounded.
        for (int64_t q = (real > nst ? real - nst : 0); q < real; ++q) {
            const int b = (int)(q % nst);
            if (!mbar_wait(ok ? empty0 + 8 * b : hand0 + 8 * b, (uint32_t)((q / nst) & 1))) {
                record(a.status, kDevTimeout);
                break;
            }
        }
        return;
    }

    if (BUILD && warp > ncw) {
        // ------------------------------ builders ------------------------------
        // Phase p of a staged row is phase 0 advanced by p bytes (uint8) or by
        // one sample (FP16): word i of phase p takes bytes i*4+p .. i*4+p+3 of
        // phase 0.  Builder w handles rows w, w + nbw, ..., two rows at a time
        // (two independent chains of loads in flight); lane l takes 16-byte
        // chunk j = j0 + l.  Bytes past the copied window only reach samples
        // outside the tile or past nsamp_out.
        const int bw = warp - ncw - 1;
        int b = 0;           // g % nst
        uint32_t par = 0u;   // (g / nst) & 1
        for (;; b = (b + 1 == nst) ? 0 : b + 1, par ^= (b == 0) ? 1u : 0u) {
            if (!mbar_wait(raw0 + 8 * b, par)) {
                record(a.status, kDevTimeout);
                return;
            }
            const int mbeam = meta[b].beam;
            const bool stop = mbeam < 0;
            if (!stop) {
                const int row_bytes = NPH * beam_at(a, mbeam).wp;
                const int wp = row_bytes / NPH;
                uint8_t *buf = smem + b * stage_bytes;
                const uint32_t *nb = rowb + b * (kRowInfoBytes / 4);
                for (int r0 = bw; r0 < cstage; r0 += 2 * nbw) {
                    const int r1 = r0 + nbw;
                    const int n0 = (int)(nb[r0] >> 4);
                    const int n1 = r1 < cstage ? (int)(nb[r1] >> 4) : 0;
                    uint8_t *row0 = buf + r0 * row_bytes;
                    uint8_t *row1 = buf + min(r1, cstage - 1) * row_bytes;
                    const int nmax = max(n0, n1);
                    for (int j0 = 0; j0 < nmax; j0 += 32) {
                        const int j = j0 + lane;
                        // Both rows' loads are issued before any store.  The
                        // word after a chunk lies inside phase 0 of its row
                        // (the copied window ends at least 16 bytes before
                        // phase 1).
                        uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
                        uint32_t x0 = 0, x1 = 0;
                        if (j < n0) {
                            v0 = *reinterpret_cast<const uint4 *>(row0 + 16 * j);
                            x0 = *reinterpret_cast<const uint32_t *>(row0 + 16 * j + 16);
                        }
                        if (j < n1) {
                            v1 = *reinterpret_cast<const uint4 *>(row1 + 16 * j);
                            x1 = *reinterpret_cast<const uint32_t *>(row1 + 16 * j + 16);
                        }
#pragma unroll
                        for (int p = 1; p < NPH; ++p) {
                            const uint32_t sp = (ELEM == 1) ? 0x3210u + 0x1111u * (uint32_t)p : 0x5432u;
                            if (j < n0)
                                *reinterpret_cast<uint4 *>(row0 + p * wp + 16 * j) =
                                    make_uint4(prmt(v0.x, v0.y, sp), prmt(v0.y, v0.z, sp),
                                               prmt(v0.z, v0.w, sp), prmt(v0.w, x0, sp));
                            if (j < n1)
                                *reinterpret_cast<uint4 *>(row1 + p * wp + 16 * j) =
                                    make_uint4(prmt(v1.x, v1.y, sp), prmt(v1.y, v1.z, sp),
                                               prmt(v1.z, v1.w, sp), prmt(v1.w, x1, sp));
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(full0 + 8 * b);
            if (stop)
                return;
        }
    }

    // ------------------------------- consumers --------------------------------
    const int wdi = warp % a.dm_warps;
    const int wti = warp / a.dm_warps;
    const int kw = wdi * DT;  // this thread's first DM column in the offset table
    const int thr_off = ELEM * (wti * SPAN) + 4 * lane;
    const uint32_t one = a.one;

    uint32_t L1[DT][NW], L2[DT][NW];  // uint8 SWAR
    float P[DT][NW][SPW];             // FP16/FP32 block partials
#pragma unroll
    for (int j = 0; j < DT; ++j)
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            L1[j][k] = 0u;
            L2[j][k] = 0u;
#pragma unroll
            for (int e = 0; e < SPW; ++e)
                P[j][k][e] = 0.f;
        }
    // FP16/FP32: the running sums S and compensations C of this thread's
    // outputs live in its TMEM lane (warp w: lane quarter w % 4, columns
    // (w / 4) * tm_sum_cols ..): S of DM j, word k, sample e at column
    // (j*NW + k)*SPW + e, C of DM j, word k at DT*NW*SPW + j*NW + k.  FP16
    // keeps the compensations of a word's two samples as one packed bf16
    // pair: a compensation is a sum of FP32 rounding errors, at most about
    // 64 * 2^-24 |S|, so its 8 significant bits move the result by less than
    // 2^-27 |S|.
    uint32_t tm = 0;
    if constexpr (ELEM > 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tm = *tm_slot + ((uint32_t)(32 * (warp & 3)) << 16) +
             (uint32_t)((warp >> 2) * tm_sum_cols(ELEM, DT, NW));
    }
    bool fresh = true;  // no block of the current tile closed yet

    // Current tile (from the stage records).
    int beam = 0, kthr = 0;
    int64_t tw = 0;
    int tile_td = 0;
    int64_t tile_t0 = 0;
    int since_flush = 0;
    bool flushed_once = false;

    auto flush_u8 = [&]() {
        const BeamArgs &B = beam_at(a, beam);
#pragma unroll
        for (int j = 0; j < DT; ++j) {
            const int row = B.perm[kthr + j];
            float *orow = B.out + (int64_t)row * B.out_pitch;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const uint32_t lo = L1[j][k] - (L2[j][k] << 8);
                // Exact integer -> FP32 for values below 2^23 on the FMA pipe:
                // the bits 0x4b000000 | v are the float 2^23 + v.
                const float4 v = make_float4(
                    __uint_as_float(0x4b000000u | (lo & 0xffffu)) - 8388608.0f,
                    __uint_as_float(0x4b000000u | (L2[j][k] & 0xffffu)) - 8388608.0f,
                    __uint_as_float(0x4b000000u | (lo >> 16)) - 8388608.0f,
                    __uint_as_float(0x4b000000u | (L2[j][k] >> 16)) - 8388608.0f);
                L1[j][k] = 0u;
                L2[j][k] = 0u;
                if (row >= 0) {
                    const int64_t t = tw + 4 * (lane + 32 * k);
                    if (t < B.nsamp_out)
                        store4(orow, t, B.nsamp_out, v, flushed_once);
                }
            }
        }
        flushed_once = true;
    };

    constexpr int NS = ELEM > 1 ? NW * SPW : 4;          // S columns per DM (floats)
    constexpr int CC0 = DT * NW * SPW;                   // first C column
    // Close a block of channels: (S, C) += P by TwoSum, one DM at a time
    // (the first block of a tile sets S = P, C = 0); P is cleared.
    auto block_float = [&]() {
#pragma unroll
        for (int j = 0; j < DT; ++j) {
            uint32_t sv[NS], cv[NW];
            if (fresh) {
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    cv[k] = 0u;
#pragma unroll
                    for (int e = 0; e < SPW; ++e)
                        sv[k * SPW + e] = __float_as_uint(P[j][k][e]);
                }
            } else {
                tm_ld<NS>(tm + (uint32_t)(j * NS), sv);
                tm_ld<NW>(tm + (uint32_t)(CC0 + j * NW), cv);
                tm_wait_ld();
                reg_fence(sv);
                reg_fence(cv);
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    float errs[SPW];
#pragma unroll
                    for (int e = 0; e < SPW; ++e) {
                        // TwoSum(S, P): S + P = s + err exactly.
                        const float S0 = __uint_as_float(sv[k * SPW + e]);
                        const float p = P[j][k][e];
                        const float sum = __fadd_rn(S0, p);
                        const float bp = __fsub_rn(sum, S0);
                        errs[e] = __fadd_rn(__fsub_rn(S0, __fsub_rn(sum, bp)), __fsub_rn(p, bp));
                        sv[k * SPW + e] = __float_as_uint(sum);
                    }
                    if constexpr (ELEM == 2) {
                        __nv_bfloat162 c2 = *reinterpret_cast<__nv_bfloat162 *>(&cv[k]);
                        c2 = __hadd2(c2, __floats2bfloat162_rn(errs[0], errs[SPW - 1]));
                        cv[k] = *reinterpret_cast<uint32_t *>(&c2);
                    } else {
                        cv[k] = __float_as_uint(__fadd_rn(__uint_as_float(cv[k]), errs[0]));
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < NW; ++k)
#pragma unroll
                for (int e = 0; e < SPW; ++e)
                    P[j][k][e] = 0.f;
            tm_st<NS>(tm + (uint32_t)(j * NS), sv);
            tm_st<NW>(tm + (uint32_t)(CC0 + j * NW), cv);
        }
        tm_wait_st();
        fresh = false;
    };

    // The tile's outputs S + C, after its last block.
    auto store_float = [&]() {
        const BeamArgs &B = beam_at(a, beam);
#pragma unroll
        for (int j = 0; j < DT; ++j) {
            uint32_t sv[NS], cv[NW];
            tm_ld<NS>(tm + (uint32_t)(j * NS), sv);
            tm_ld<NW>(tm + (uint32_t)(CC0 + j * NW), cv);
            tm_wait_ld();
            reg_fence(sv);
            reg_fence(cv);
            const int row = B.perm[kthr + j];
            if (row < 0)
                continue;
            float *orow = B.out + (int64_t)row * B.out_pitch;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const int64_t t = tw + SPW * (lane + 32 * k);
                float o[SPW];
#pragma unroll
                for (int e = 0; e < SPW; ++e) {
                    float comp;
                    if constexpr (ELEM == 2) {
                        const __nv_bfloat162 c2 = *reinterpret_cast<const __nv_bfloat162 *>(&cv[k]);
                        comp = e == 0 ? __low2float(c2) : __high2float(c2);
                    } else {
                        comp = __uint_as_float(cv[k]);
                    }
                    o[e] = __fadd_rn(__uint_as_float(sv[k * SPW + e]), comp);
                }
                if (SPW == 1) {
                    if (t < B.nsamp_out)
                        orow[t] = o[0];
                } else if (t + 1 < B.nsamp_out) {
                    *reinterpret_cast<float2 *>(orow + t) = make_float2(o[0], o[SPW - 1]);
                } else if (t < B.nsamp_out) {
                    orow[t] = o[0];
                }
            }
        }
    };

    // One register buffer of words per row (x: row 2q, y: row 2q+1).  Each
    // iteration (channel pair q, DM j) sums its words and, word by word,
    // reloads the buffer with the next iteration's words, so every load is
    // issued one iteration before its use with half the registers of a
    // double buffer.  The next iteration's table offsets are themselves
    // read one iteration earlier still (`on`).
    uint32_t x[NW], y[NW];
    // Offsets of rows 2q, 2q+1 for DM j, in the table of a stage (tb points
    // at this thread's first DM column).
    auto off2 = [&](const int *tb, int q, int j) {
        return *reinterpret_cast<const int2 *>(tb + (q * dm_cta + j) * 2);
    };
    // Offsets of DMs j and j+1 (j even; DT even keeps the int4 16-byte aligned).
    auto off4 = [&](const int *tb, int q, int j) {
        return *reinterpret_cast<const int4 *>(tb + (q * dm_cta + j) * 2);
    };
    int2 hold = make_int2(0, 0);  // DM j+1 half of the last off4
    // Offsets of iteration (q, j) read two iterations ahead: an even j reads
    // the pair (j, j+1) and keeps the odd half for the next iteration.
    auto ahead = [&](const int *tb, int q, int j) {
        if constexpr (DT % 2 == 0) {
            if ((j & 1) == 0) {
                const int4 o = off4(tb, q, j);
                hold = make_int2(o.z, o.w);
                return make_int2(o.x, o.y);
            }
            return hold;
        } else {
            return off2(tb, q, j);
        }
    };
    auto load_words = [&](int2 off) {
        const uint32_t *p0 = reinterpret_cast<const uint32_t *>(smem + off.x + thr_off);
        const uint32_t *p1 = reinterpret_cast<const uint32_t *>(smem + off.y + thr_off);
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            x[k] = p0[32 * k];
            y[k] = p1[32 * k];
        }
    };
    // Sum the words of this iteration into DM j; if `reload`, refill each
    // word from the next iteration's rows (offsets nxt) right after use.
    auto sum_reload = [&](int j, bool reload, int2 nxt) {
        const uint32_t *p0 = reinterpret_cast<const uint32_t *>(smem + nxt.x + thr_off);
        const uint32_t *p1 = reinterpret_cast<const uint32_t *>(smem + nxt.y + thr_off);
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            if (ELEM == 1) {
                L1[j][k] = L1[j][k] + x[k] + y[k];
                if (DT <= 2) {
                    // Fewer DMs per thread leave the ALU pipe room: one IADD3
                    // (measured up to 18 % faster at 2 DMs per thread).
                    L2[j][k] = L2[j][k] + prmt(x[k], 0u, 0x4341u) + prmt(y[k], 0u, 0x4341u);
                } else {
                    L2[j][k] = imad_acc(prmt(x[k], 0u, 0x4341u), one, L2[j][k]);
                    L2[j][k] = imad_acc(prmt(y[k], 0u, 0x4341u), one, L2[j][k]);
                }
            } else if (ELEM == 2) {
                P[j][k][0] = add_f16_lo(y[k], add_f16_lo(x[k], P[j][k][0]));
                P[j][k][SPW - 1] = add_f16_hi(y[k], add_f16_hi(x[k], P[j][k][SPW - 1]));
            } else {
                P[j][k][0] = __fadd_rn(__fadd_rn(P[j][k][0], __uint_as_float(x[k])),
                                       __uint_as_float(y[k]));
            }
            if (reload) {
                x[k] = p0[32 * k];
                y[k] = p1[32 * k];
            }
        }
    };

    // Stages run in ring order.  Within a stage of T = npairs*DT iterations
    // the words of iteration i+1 are loaded during iteration i and the
    // offsets of iteration i+2 are read during iteration i.  When the next
    // stage continues the tile without a widening in between, both reach
    // into it: the consumer waits for that stage at iteration T-2 and
    // releases the current one at T-1, after its last loads from it.
    // Otherwise the next stage starts fresh, so no prefetched buffer is live
    // across a widening.
    const int npairs = cstage / 2;  // >= 2: chan_per_stage is a multiple of 4
    // Pairs whose iterations never reach past the stage (i + 2 < T).
    const int q_plain = npairs - (DT == 1 ? 2 : 1);
    bool prefetched = false;
    int2 on = make_int2(0, 0);  // offsets of the next iteration
    int b = 0;          // g % nst for ring position g
    uint32_t par = 0u;  // (g / nst) & 1
    for (;; par ^= (b + 1 == nst) ? 1u : 0u, b = (b + 1 == nst) ? 0 : b + 1) {
        if (!prefetched && !mbar_wait(full0 + 8 * b, par)) {
            record(a.status, kDevTimeout);
            goto consumers_done;
        }
        const StageMeta m = meta[b];
        if (m.beam < 0)
            break;  // no further tile
        const int *tb = atab + b * tab_stride + 2 * kw;
        if (m.st == 0) {
            beam = m.beam;
            kthr = m.td * dm_cta + kw;
            tw = m.t0 + (int64_t)wti * SPAN;
            tile_td = m.td;
            tile_t0 = m.t0;
            fresh = true;
            since_flush = 0;
            flushed_once = false;
        }
        if (!prefetched) {
            if constexpr (DT % 2 == 0) {
                const int4 o = off4(tb, 0, 0);
                load_words(make_int2(o.x, o.y));
                on = make_int2(o.z, o.w);
            } else {
                load_words(off2(tb, 0, 0));
                on = off2(tb, 1, 0);
            }
        }
        since_flush += cstage;
        const bool last = m.st + 1 == m.nstage;
        // Widen (uint8) or close a compensated block (floats) after this stage
        // if the next one would overflow it.
        const bool widen = !last && since_flush + cstage > FLUSH;
        const bool cross = !last && !widen;
        const int bn = (b + 1 == nst) ? 0 : b + 1;       // (g + 1) % nst
        const uint32_t parn = bn == 0 ? par ^ 1u : par;  // ((g + 1) / nst) & 1
        const int *tbn = atab + bn * tab_stride + 2 * kw;
        // Unrolled by two pairs (measured 2 % faster than the plain loop on
        // the L-band beam at (4,12,1,8,8); unrolling by 4 measured slower),
        // or whole for uint8 with the stage size fixed at compile time
        // (measured 3 % faster than by two on the 4096-channel beam; FP16
        // measured 3 % slower whole).
#pragma unroll((CS > 0 && ELEM == 1) ? CS : 2)
        for (int q = 0; q < q_plain; ++q) {
#pragma unroll
            for (int j = 0; j < DT; ++j) {
                const int2 onn = ahead(tb, q + (j + 2) / DT, (j + 2) % DT);
                sum_reload(j, true, on);
                on = onn;
            }
        }
#pragma unroll(CS > 0 ? CS : 1)
        for (int q = q_plain; q < npairs; ++q) {
#pragma unroll
            for (int j = 0; j < DT; ++j) {
                const int left = (npairs - q) * DT - j;  // iterations left, this one included
                int2 onn = on;
                if (left > 2) {
                    onn = ahead(tb, q + (j + 2) / DT, (j + 2) % DT);
                } else if (cross) {
                    if (left == 2 &&
                        !mbar_wait(full0 + 8 * bn, parn)) {
                        record(a.status, kDevTimeout);
                        goto consumers_done;
                    }
                    onn = ahead(tbn, (2 - left) / DT, (2 - left) % DT);
                }
                if (left == 1) {
                    // Every load from this stage has been issued: release it.
                    __syncwarp();
                    if (lane == 0)
                        mbar_arrive(empty0 + 8 * b);
                }
                sum_reload(j, left > 1 || cross, on);
                on = onn;
            }
        }
        prefetched = cross;
        if (widen) {
            if (ELEM == 1)
                flush_u8();
            else
                block_float();
            since_flush = 0;
        }
        if (last) {
            if (ELEM == 1) {
                flush_u8();
            } else {
                block_float();
                store_float();
            }
            if constexpr (DET) {
                if (!detect_epilogue(a, tile_td, tile_t0, dm_cta, t_cta, ncw, warp, lane, tid,
                                     ep_bar, ep_flags))
                    goto consumers_done;
            }
        }
    }
consumers_done:
    if constexpr (ELEM > 1) {
        // Free the TMEM once every consumer warp is done with it.  The wait is
        // bounded: a warp that gave up on a timeout arrives here too, and if
        // one never does the others still free the columns after the limit.
        tm_wait_st();
        tm_wait_ld();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0)
            mbar_arrive(ep_bar);
        if (!mbar_wait(ep_bar, 0))
            record(a.status, kDevTimeout);
        if (warp == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tm_slot),
                         "n"(TM_COLS)
                         : "memory");
        }
    }
}

template <int ELEM, int DT, int NW, bool DET = false, int CS = 0>
cudaError_t launch_one(const KArgs &a, unsigned grid, int threads, int smem, cudaStream_t s) {
    auto k = dedisperse_kernel<ELEM, DT, NW, DET, CS>;
    // Raise the dynamic shared-memory limit only when a launch needs more than
    // before (so a launch inside a stream capture never changes attributes
    // after an eager launch of the same shape).
    static int configured[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    int &conf = configured[dev & 63];
    if (smem > conf) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess)
            return e;
        conf = smem;
    }
    k<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

// Instantiations for one element size: DMs per thread 1/2/4 x words 4/8.
template <int ELEM>
cudaError_t launch_elem(const KArgs &a, unsigned grid, int threads, int smem, cudaStream_t s,
                        int dthr, int nw) {
    if constexpr (ELEM == 1) {
        if (a.det_s1) {  // fused detection: uint8, 4 DMs x 8 words per thread
            if (nw != 8 || dthr != 4)
                return cudaErrorInvalidValue;
            if (a.cstage == 8)
                return launch_one<1, 4, 8, true, 8>(a, grid, threads, smem, s);
            return launch_one<1, 4, 8, true>(a, grid, threads, smem, s);
        }
    }
    // The tuned shape of each element size at 4 DMs x 8 words also has an
    // instantiation with its stage size fixed, which unrolls the stage loop
    // and resolves its hand-over branches at compile time.
    constexpr int kFixedStage = ELEM == 1 ? 8 : ELEM == 2 ? 12 : 24;
    if (nw == 8 && dthr == 4 && a.cstage == kFixedStage)
        return launch_one<ELEM, 4, 8, false, kFixedStage>(a, grid, threads, smem, s);
    if (nw == 4) {
        switch (dthr) {
        case 1: return launch_one<ELEM, 1, 4>(a, grid, threads, smem, s);
        case 2: return launch_one<ELEM, 2, 4>(a, grid, threads, smem, s);
        case 4: return launch_one<ELEM, 4, 4>(a, grid, threads, smem, s);
        }
    } else if (nw == 8) {
        switch (dthr) {
        case 1: return launch_one<ELEM, 1, 8>(a, grid, threads, smem, s);
        case 2: return launch_one<ELEM, 2, 8>(a, grid, threads, smem, s);
        case 4: return launch_one<ELEM, 4, 8>(a, grid, threads, smem, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace dd
