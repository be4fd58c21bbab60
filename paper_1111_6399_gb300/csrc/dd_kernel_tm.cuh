// De-dispersion of FP16/FP32 input with the shifted windows held in tensor
// memory (TMEM), for sm_103a.
//
//   out[d][t] = sum_c in[c][t + s(c,d)]
//
// With 2- or 4-byte samples the lane-interleaved kernel (dd_kernel.cuh) reads
// one shared-memory word per add, which caps it at 1/2 (FP16) or 1/4 (FP32)
// of the add peak: shared memory delivers 128 bytes per clock per SM.  Here a
// consumer thread owns T consecutive output samples (T = 17 for FP32, 18 for
// FP16) of 4 consecutive trial DMs.  Their windows of channel c overlap: DM
// j needs samples [t + s(c,j), t + s(c,j) + T), so the union for the 4 DMs is
// T + D samples with D = s(c,j0+3) - s(c,j0), instead of 4T.  The thread
// reads that union once from shared memory (a lane stride of 17 words, or 9
// words for FP16, is odd, so the warp's reads are conflict-free), converts
// FP16 to FP32, and writes it to its own TMEM lane with tcgen05.st; each DM's
// slice is then read back with tcgen05.ld at a column offset of s(c,j) -
// s(c,j0), which the instruction takes at run time (registers cannot be
// indexed that way).  Shared-memory reads per add fall from 1 to about 0.56
// on the L-band and low-frequency beams.
//
// Sums follow the library's accumulation order for float input: FP32
// partials P over blocks of 64 channels (packed FP32 pair adds), combined
// into a running sum S with TwoSum compensation C.  S (FP32) and C (a packed
// bf16 pair per two samples) live in TMEM next to the windows, so a thread
// keeps only P and the loaded slices in registers.
//
// CTA: 7 consumer warps (warp w on TMEM lane quarter w % 4, columns
// 256*(w / 4) .. +255: two window buffers of 72 columns, S and C) and one
// producer warp, which stages channel windows with TMA bulk copies (no
// multicast) into an mbarrier ring and writes a table of shifted-window
// offsets, as in dd_kernel.cuh.  Eight warps leave two per SM sub-partition,
// so a thread may hold up to 255 registers: the four slices of a row are
// loaded before one wait.  A tile is 4*dm_warps DMs x 32*T*time_warps
// samples, dm_warps*time_warps = 7.  The
// host admits this shape only when every 4-DM group's shift spread D over
// every channel is at most 72 - T columns.  TMEM (all 512 columns) is
// allocated by consumer warp 0 at the start and freed at the end on every
// path, timeouts included; the host sizes shared memory so that only one CTA
// is resident per SM.
#pragma once

#include "dd_kernel.cuh"

namespace dd {
namespace {

constexpr int kTmThreadsWarps = 9;  // 4 consumers, 1 producer, 4 fillers
constexpr int kTmProducer = 4;      // warp index of the producer
constexpr int kTmDt = 4;            // DMs per consumer thread
constexpr int kTmWin = 72;          // TMEM columns per window buffer
constexpr int kTmBufs = 5;          // window buffers per lane quarter
constexpr int kTmColsAlloc = 512;
constexpr int kMsgLast = 1;         // the row closes its tile
constexpr int kMsgStop = 2;         // no further rows

// A filled window handed from a filler to its consumer: the shift offsets of
// DMs 1..3 relative to DM 0 (TMEM columns), control bits and the tile.
struct __align__(16) RowMsg {
    int d1, d2, d3, ctl;
    int beam, td;
    int64_t t0;
};

__device__ __forceinline__ void tm_st8(uint32_t taddr, const uint32_t (&v)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
        : "memory");
}

__device__ __forceinline__ void tm_st1(uint32_t taddr, uint32_t v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(v)
                 : "memory");
}

__device__ __forceinline__ void tm_st2(uint32_t taddr, uint32_t v0, uint32_t v1) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(v0),
                 "r"(v1)
                 : "memory");
}

__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&v)[16], int o) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr + (uint32_t)o)
        : "memory");
}

__device__ __forceinline__ uint32_t tm_ld1(uint32_t taddr) {
    uint32_t v;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr)
                 : "memory");
    return v;
}

__device__ __forceinline__ void tm_ld2(uint32_t taddr, uint32_t &v0, uint32_t &v1) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                 : "=r"(v0), "=r"(v1)
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tm_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Registers written by tcgen05.ld hold their values only after
// tcgen05.wait::ld.  The compiler does not know that, so after each wait the
// loaded registers pass through an empty volatile asm that "redefines" them:
// every later use depends on it and cannot be scheduled above the wait.
__device__ __forceinline__ void reg_fence(uint32_t &v) { asm volatile("" : "+r"(v)); }

template <int N>
__device__ __forceinline__ void reg_fence(uint32_t (&v)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i)
        asm volatile("" : "+r"(v[i]));
}

__device__ __forceinline__ void tm_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Bounded wait for a fine-grained hand-off (one per row): try_wait lets the
// hardware suspend the warp until the phase completes or a short hint
// expires, so the loop spins without the backoff sleeps of mbar_wait (a
// sleep of 64 ns or more per hand-off would dominate a row's work).  The
// global timer is read every 64 tries; the limit is the kernels' 2 s.
__device__ __noinline__ bool mbar_spin_slow(uint32_t mb, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(mb, parity))
            return true;
        if ((i & 63u) == 0 && global_ns() - t0 > kWaitLimitNs)
            return false;
    }
}

__device__ __forceinline__ bool mbar_spin(uint32_t mb, uint32_t parity) {
    return mbar_try(mb, parity) || mbar_spin_slow(mb, parity);
}

// (a0, a1) += (b0, b1) as one packed FP32 pair add (two IEEE adds, each
// rounded to nearest even).
__device__ __forceinline__ void fadd2(float &a0, float &a1, float b0, float b1) {
    asm("{ .reg .b64 x, y; mov.b64 x, {%0, %1}; mov.b64 y, {%2, %3}; "
        "add.rn.f32x2 x, x, y; mov.b64 {%0, %1}, x; }"
        : "+f"(a0), "+f"(a1)
        : "f"(b0), "f"(b1));
}

// Columns c .. c+17 of a TMEM lane as 9 packed FP32 pairs (64-bit values).
__device__ __forceinline__ void tm_ld18p(uint32_t taddr, uint64_t (&v)[9]) {
    asm volatile(
        "{ .reg .b32 r<18>;\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {r0, r1, r2, r3, r4, r5, r6, r7, r8, r9, r10, "
        "r11, r12, r13, r14, r15}, [%9];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {r16, r17}, [%10];\n\t"
        "mov.b64 %0, {r0, r1}; mov.b64 %1, {r2, r3}; mov.b64 %2, {r4, r5}; "
        "mov.b64 %3, {r6, r7}; mov.b64 %4, {r8, r9}; mov.b64 %5, {r10, r11}; "
        "mov.b64 %6, {r12, r13}; mov.b64 %7, {r14, r15}; mov.b64 %8, {r16, r17}; }"
        : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]), "=l"(v[4]), "=l"(v[5]), "=l"(v[6]),
          "=l"(v[7]), "=l"(v[8])
        : "r"(taddr), "r"(taddr + 16u)
        : "memory");
}

__device__ __forceinline__ void reg_fence(uint64_t &v) { asm volatile("" : "+l"(v)); }

// a += b for packed FP32 pairs (two IEEE adds, each rounded to nearest even).
__device__ __forceinline__ void fadd2p(uint64_t &a, uint64_t b) {
    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(a) : "l"(b));
}

__device__ __forceinline__ float pair_lo(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float pair_hi(uint64_t v) {
    return __uint_as_float((uint32_t)(v >> 32));
}

__device__ __forceinline__ float half_lo(uint32_t w) {
    float f;
    asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %1; cvt.f32.f16 %0, lo; }" : "=f"(f) : "r"(w));
    return f;
}

__device__ __forceinline__ float half_hi(uint32_t w) {
    float f;
    asm("{ .reg .b16 lo, hi; mov.b32 {lo, hi}, %1; cvt.f32.f16 %0, hi; }" : "=f"(f) : "r"(w));
    return f;
}

// ---------------------------------------------------------------------------
// ELEM = 2 (FP16) or 4 (FP32).  Warps 0-3 consume (warp q on TMEM lane
// quarter q), warp 4 produces, warps 5-8 fill (the filler of quarter q is
// warp 8 for q = 0, else warp 4 + q).
// ---------------------------------------------------------------------------
template <int ELEM>
__global__ void __launch_bounds__(32 * kTmThreadsWarps, 1)
    dedisperse_tm_kernel(const __grid_constant__ KArgs a) {
    constexpr int T = ELEM == 4 ? 17 : 18;  // output samples per thread and DM
    constexpr int SPAN = 32 * T;            // samples per warp
    constexpr int NP = (T + 1) / 2;         // FP32 pairs per DM (last one half used for T odd)
    constexpr int SCOL = kTmBufs * kTmWin;  // TMEM column of S
    constexpr int CCOL = SCOL + kTmDt * T;  // TMEM column of C (bf16 pairs)
    static_assert(CCOL + kTmDt * NP <= kTmColsAlloc, "TMEM columns");

    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int dm_cta = kTmDt * a.dm_warps;
    const int t_cta = SPAN * a.time_warps;
    const int cstage = a.cstage;
    const int nst = a.nstages;
    const int stage_bytes = a.stage_bytes;
    const int tab_stride = cstage * dm_cta;
    int *atab = reinterpret_cast<int *>(smem + nst * stage_bytes);
    StageMeta *meta = reinterpret_cast<StageMeta *>(
        smem + nst * stage_bytes + ((nst * tab_stride * 4 + 15) & ~15));
    uint64_t *mbar = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(meta) +
                                                  nst * kStageMetaBytes);
    // Window hand-off, per lane quarter and TMEM buffer: wfull (filler ->
    // consumer) and wempty (consumer -> filler), then the row messages.
    uint64_t *wbar = mbar + 2 * nst;
    RowMsg *msgs = reinterpret_cast<RowMsg *>(wbar + 2 * 4 * kTmBufs);
    uint32_t *tm_slot = reinterpret_cast<uint32_t *>(msgs + 4 * kTmBufs);
    const uint32_t full0 = smem_addr(&mbar[0]);
    const uint32_t empty0 = smem_addr(&mbar[nst]);
    const uint32_t wfull0 = smem_addr(&wbar[0]);
    const uint32_t wempty0 = smem_addr(&wbar[4 * kTmBufs]);

    if (tid == 0) {
        for (int b = 0; b < nst; ++b) {
            mbar_init(full0 + 8 * b, 1);
            mbar_init(empty0 + 8 * b, 4);  // the four fillers
        }
        for (int i = 0; i < 4 * kTmBufs; ++i) {
            mbar_init(wfull0 + 8 * i, 1);
            mbar_init(wempty0 + 8 * i, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_addr(tm_slot)),
            "r"(kTmColsAlloc)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();

    if (warp == kTmProducer) {
        // ------------------------------ producer ------------------------------
        // As in dd_kernel.cuh, with one copy per row (no byte phases) and the
        // offset table laid out [row][DM] so a consumer fetches its 4 DMs with
        // one 16-byte load.
        int64_t g = 0;
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
            const int nstage = (B.nchan + cstage - 1) / cstage;
            const float dm_min = B.dm_sorted[kcta];
            const float dm_max = B.dm_sorted[kcta + dm_cta - 1];
            float dmk[2];
            dmk[0] = B.dm_sorted[kcta + min(lane, dm_cta - 1)];
            dmk[1] = B.dm_sorted[kcta + min(lane + 32, dm_cta - 1)];
            float ds_next[2];
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                ds_next[h] = (c < cstage && c < B.nchan) ? B.dmshift[c] : 0.0f;
            }
            for (int st = 0; st < nstage; ++st, ++g) {
                const int b = (int)(g % nst);
                const int64_t n = g / nst;
                const float ds_cur[2] = {ds_next[0], ds_next[1]};
                for (int h = 0; h < 2; ++h) {
                    const int c = (st + 1) * cstage + lane + 32 * h;
                    ds_next[h] = (st + 1 < nstage && lane + 32 * h < cstage && c < B.nchan)
                                     ? B.dmshift[c] : 0.0f;
                }
                if (n > 0 && !mbar_wait(empty0 + 8 * b, (uint32_t)((n - 1) & 1))) {
                    ok = false;
                    break;
                }
                uint8_t *buf = smem + b * stage_bytes;
                int *tab = atab + b * tab_stride;
                uint32_t my_bytes[2] = {0u, 0u};
                int64_t my_first[2] = {0, 0};
                int my_base[2] = {0, 0};
                float my_ds[2] = {0.0f, 0.0f};
                bool bad = false;
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
                    // The consumers read up to kTmWin samples past a lane's
                    // first one; wp leaves that much room after the copy.
                    if (bytes > wp - kTmWin * ELEM - 16 || bytes <= 0 ||
                        cstage * wp > stage_bytes) {
                        bad = true;  // excluded by the host checks
                        continue;
                    }
                    my_base[h] = (int)(buf + r * wp - smem) + (int)(ELEM * (t0 - firsts));
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
                uint32_t total = my_bytes[0] + my_bytes[1];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    total += __shfl_xor_sync(0xffffffffu, total, o);
                if (lane == 0)
                    mbar_expect_tx(full0 + 8 * b, total);
                __syncwarp();
                for (int h = 0; h < 2; ++h) {
                    const int r = lane + 32 * h;
                    if (r >= cstage || my_bytes[h] == 0)
                        continue;
                    const int c = st * cstage + r;
                    const int64_t off = (int64_t)c * B.in_pitch_b + my_first[h] * ELEM;
                    bulk_g2s(smem_addr(buf + r * wp), B.in + off, my_bytes[h], full0 + 8 * b);
                }
                // Offset table [row][DM]: smem byte offset of sample t0 + s(c,k).
                for (int r = 0; r < cstage; ++r) {
                    const int base = __shfl_sync(0xffffffffu, my_base[r >> 5], r & 31);
                    const float ds = __shfl_sync(0xffffffffu, my_ds[r >> 5], r & 31);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int k = lane + 32 * h;
                        if (k < dm_cta)
                            tab[r * dm_cta + k] = base + ELEM * shift_of(dmk[h], ds);
                    }
                }
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(full0 + 8 * b);
            }
            if (!ok)
                break;
        }
        const int64_t real = g;
        if (ok) {
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
                    mbar_arrive(full0 + 8 * b);
            }
        }
        if (!ok)
            record(a.status, kDevTimeout);
        for (int64_t q = (real > nst ? real - nst : 0); q < real; ++q) {
            const int b = (int)(q % nst);
            if (!mbar_wait(ok ? empty0 + 8 * b : full0 + 8 * b, (uint32_t)((q / nst) & 1))) {
                record(a.status, kDevTimeout);
                break;
            }
        }
        return;
    }


    // ---------------------- consumers and fillers (TMEM) ----------------------
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm_base = *tm_slot;
    const int q = warp & 3;  // TMEM lane quarter
    const uint32_t tm = tm_base + ((uint32_t)(32 * q) << 16);
    const int wdi = q % a.dm_warps;
    const int wti = q / a.dm_warps;
    const int kw = wdi * kTmDt;                  // first DM column of quarter q's threads
    const int lane_t = wti * SPAN + T * lane;    // first sample of this thread in the tile
    const uint32_t my_wfull = wfull0 + 8 * kTmBufs * q;
    const uint32_t my_wempty = wempty0 + 8 * kTmBufs * q;
    RowMsg *my_msgs = msgs + kTmBufs * q;

    if (warp > kTmProducer) {
        // ------------------------------- filler -------------------------------
        // Walks the stages like the consumers of dd_kernel.cuh, and for each row
        // copies the union window of quarter q's 4 DMs from shared memory into
        // the next free TMEM buffer (as FP32), then hands it over with the
        // row's shift offsets.
        int64_t g = 0;
        int bq = 0;          // ring buffer
        uint32_t ph = 0u;    // ring phase
        for (;;) {
            const int slot = (int)(g % nst);
            if (!mbar_wait(full0 + 8 * slot, (uint32_t)((g / nst) & 1))) {
                record(a.status, kDevTimeout);
                break;
            }
            const StageMeta m = meta[slot];
            const int nrows = m.beam < 0 ? 0 : min(cstage, beam_at(a, m.beam).nchan - m.st * cstage);
            for (int r = 0; r <= nrows; ++r) {
                // r == nrows: nothing more in this stage (a terminating stage
                // sends its message here)
                if (r == nrows && m.beam >= 0)
                    break;
                if (!mbar_spin(my_wempty + 8 * bq, ph ^ 1u)) {
                    record(a.status, kDevTimeout);
                    g = -1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                RowMsg msg;
                if (m.beam < 0) {
                    msg.d1 = msg.d2 = msg.d3 = 0;
                    msg.ctl = kMsgStop;
                    msg.beam = msg.td = 0;
                    msg.t0 = 0;
                } else {
                    const int4 o = *reinterpret_cast<const int4 *>(atab + slot * tab_stride +
                                                                   r * dm_cta + kw);
                    const int n = T + (o.w - o.x) / ELEM;
                    const uint32_t tw = tm + (uint32_t)(kTmWin * bq);
                    if constexpr (ELEM == 4) {
                        const uint32_t *p = reinterpret_cast<const uint32_t *>(smem + o.x) + lane_t;
#pragma unroll 1
                        for (int mm = 0; mm < n; mm += 8) {
                            uint32_t v[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                v[i] = p[mm + i];
                            tm_st8(tw + (uint32_t)mm, v);
                        }
                    } else {
                        const int byte0 = o.x + 2 * lane_t;  // lane_t even: uniform phase
                        const uint32_t *p = reinterpret_cast<const uint32_t *>(smem + (byte0 & ~3));
                        const uint32_t sel = (byte0 & 2) ? 0x5432u : 0x3210u;
#pragma unroll 1
                        for (int mm = 0; mm < n; mm += 8) {
                            uint32_t w[5];
#pragma unroll
                            for (int i = 0; i < 5; ++i)
                                w[i] = p[mm / 2 + i];
                            uint32_t v[8];
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const uint32_t h2 = prmt(w[i], w[i + 1], sel);
                                v[2 * i] = __float_as_uint(half_lo(h2));
                                v[2 * i + 1] = __float_as_uint(half_hi(h2));
                            }
                            tm_st8(tw + (uint32_t)mm, v);
                        }
                    }
                    msg.d1 = (o.y - o.x) / ELEM;
                    msg.d2 = (o.z - o.x) / ELEM;
                    msg.d3 = (o.w - o.x) / ELEM;
                    msg.ctl = (m.st + 1 == m.nstage && r + 1 == nrows) ? kMsgLast : 0;
                    msg.beam = m.beam;
                    msg.td = m.td;
                    msg.t0 = m.t0;
                }
                tm_wait_st();
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                if (lane == 0)
                    my_msgs[bq] = msg;
                __syncwarp();
                if (lane == 0)
                    mbar_arrive(my_wfull + 8 * bq);
                if (++bq == kTmBufs) {
                    bq = 0;
                    ph ^= 1u;
                }
                if (m.beam < 0)
                    break;
            }
            if (g < 0 || m.beam < 0)
                break;
            // every shared-memory read of this stage is done: release it
            __syncwarp();
            if (lane == 0)
                mbar_arrive(empty0 + 8 * slot);
            ++g;
        }
    } else {
        // ------------------------------ consumer ------------------------------
        uint64_t P[kTmDt][NP];
#pragma unroll
        for (int j = 0; j < kTmDt; ++j)
#pragma unroll
            for (int i = 0; i < NP; ++i)
                P[j][i] = 0ull;
        // Close a block of channels: S + P by TwoSum into (S, C); on the first
        // block of a tile S = P and C = 0.  P is cleared.
        auto close_block = [&](bool first_block) {
#pragma unroll
            for (int j = 0; j < kTmDt; ++j) {
                const uint32_t ts = tm + (uint32_t)(SCOL + j * T);
                const uint32_t tc = tm + (uint32_t)(CCOL + j * NP);
                uint32_t s[2 * NP];
                uint32_t c[NP];
                if (first_block) {
#pragma unroll
                    for (int i = 0; i < T; ++i)
                        s[i] = __float_as_uint((i & 1) ? pair_hi(P[j][i / 2]) : pair_lo(P[j][i / 2]));
#pragma unroll
                    for (int i = 0; i < NP; ++i)
                        c[i] = 0u;
                } else {
                    uint32_t v[16], w[8];
                    uint32_t s16 = 0u, s17 = 0u, c8x = 0u;
                    tm_ld16(ts, v, 0);
                    if constexpr (T == 17)
                        s16 = tm_ld1(ts + 16u);
                    else
                        tm_ld2(ts + 16u, s16, s17);
                    // C: NP = 9 columns (x8 + x1)
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, "
                        "[%8];"
                        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                          "=r"(w[6]), "=r"(w[7])
                        : "r"(tc)
                        : "memory");
                    c8x = tm_ld1(tc + 8u);
                    tm_wait_ld();
                    reg_fence(v);
                    reg_fence(w);
                    reg_fence(s16);
                    reg_fence(s17);
                    reg_fence(c8x);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        s[i] = v[i];
                    s[16] = s16;
                    if constexpr (T == 18)
                        s[17] = s17;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        c[i] = w[i];
                    c[8] = c8x;
#pragma unroll
                    for (int i = 0; i < T; ++i) {
                        const float S0 = __uint_as_float(s[i]);
                        const float p = (i & 1) ? pair_hi(P[j][i / 2]) : pair_lo(P[j][i / 2]);
                        const float sum = __fadd_rn(S0, p);
                        const float bp = __fsub_rn(sum, S0);
                        const float err = __fadd_rn(__fsub_rn(S0, __fsub_rn(sum, bp)),
                                                    __fsub_rn(p, bp));
                        s[i] = __float_as_uint(sum);
                        // C of samples 2q, 2q+1 as a packed bf16 pair
                        __nv_bfloat162 cc = *reinterpret_cast<__nv_bfloat162 *>(&c[i / 2]);
                        const __nv_bfloat162 e = (i & 1) ? __floats2bfloat162_rn(0.f, err)
                                                         : __floats2bfloat162_rn(err, 0.f);
                        cc = __hadd2(cc, e);
                        c[i / 2] = *reinterpret_cast<uint32_t *>(&cc);
                    }
                }
#pragma unroll
                for (int i = 0; i < NP; ++i)
                    P[j][i] = 0ull;
                uint32_t s8[8], c8[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    s8[i] = s[i];
                    c8[i] = c[i];
                }
                tm_st8(ts, s8);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    s8[i] = s[8 + i];
                tm_st8(ts + 8u, s8);
                if constexpr (T == 17)
                    tm_st1(ts + 16u, s[16]);
                else
                    tm_st2(ts + 16u, s[16], s[17]);
                tm_st8(tc, c8);
                tm_st1(tc + 8u, c[8]);
            }
            tm_wait_st();
        };

        // Store S + C of the tile (after its last block) to the output rows.
        auto store_tile = [&](const BeamArgs &B, int kthr, int64_t t_first) {
#pragma unroll
            for (int j = 0; j < kTmDt; ++j) {
                const int row = B.perm[kthr + j];
                const uint32_t ts = tm + (uint32_t)(SCOL + j * T);
                const uint32_t tc = tm + (uint32_t)(CCOL + j * NP);
                uint32_t s[2 * NP], c[NP];
                uint32_t v[16], w[8];
                uint32_t s16 = 0u, s17 = 0u, c8x = 0u;
                tm_ld16(ts, v, 0);
                if constexpr (T == 17)
                    s16 = tm_ld1(ts + 16u);
                else
                    tm_ld2(ts + 16u, s16, s17);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                    : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                      "=r"(w[6]), "=r"(w[7])
                    : "r"(tc)
                    : "memory");
                c8x = tm_ld1(tc + 8u);
                tm_wait_ld();
                reg_fence(v);
                reg_fence(w);
                reg_fence(s16);
                reg_fence(s17);
                reg_fence(c8x);
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    s[i] = v[i];
                s[16] = s16;
                s[17] = s17;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    c[i] = w[i];
                c[8] = c8x;
                if (row < 0)
                    continue;
                float *orow = B.out + (int64_t)row * B.out_pitch;
#pragma unroll
                for (int i = 0; i < T; ++i) {
                    const __nv_bfloat162 cc = *reinterpret_cast<const __nv_bfloat162 *>(&c[i / 2]);
                    const float comp = (i & 1) ? __high2float(cc) : __low2float(cc);
                    const int64_t t = t_first + i;
                    if (t < B.nsamp_out)
                        orow[t] = __fadd_rn(__uint_as_float(s[i]), comp);
                }
            }
        };


        int bq = 0;
        uint32_t ph = 0u;
        int since = 0;
        bool first_block = true;
        for (;;) {
            if (!mbar_spin(my_wfull + 8 * bq, ph)) {
                record(a.status, kDevTimeout);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const RowMsg msg = my_msgs[bq];
            if (msg.ctl & kMsgStop)
                break;
            const uint32_t tw = tm + (uint32_t)(kTmWin * bq);
            {
                uint64_t v[2][NP];
                tm_ld18p(tw, v[0]);
                tm_ld18p(tw + (uint32_t)msg.d1, v[1]);
                tm_wait_ld();
#pragma unroll
                for (int jj = 0; jj < 2; ++jj)
#pragma unroll
                    for (int i = 0; i < NP; ++i) {
                        reg_fence(v[jj][i]);
                        fadd2p(P[jj][i], v[jj][i]);
                    }
                tm_ld18p(tw + (uint32_t)msg.d2, v[0]);
                tm_ld18p(tw + (uint32_t)msg.d3, v[1]);
                tm_wait_ld();
#pragma unroll
                for (int jj = 0; jj < 2; ++jj)
#pragma unroll
                    for (int i = 0; i < NP; ++i) {
                        reg_fence(v[jj][i]);
                        fadd2p(P[2 + jj][i], v[jj][i]);
                    }
            }
            // the buffer's slices are in registers: hand it back
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                mbar_arrive(my_wempty + 8 * bq);
            if (++bq == kTmBufs) {
                bq = 0;
                ph ^= 1u;
            }
            const bool last = (msg.ctl & kMsgLast) != 0;
            if (++since == kFloatBlock || last) {
                close_block(first_block);
                first_block = false;
                since = 0;
            }
            if (last) {
                store_tile(beam_at(a, msg.beam), msg.td * dm_cta + kw, msg.t0 + lane_t);
                first_block = true;
            }
        }
    }

    // Free TMEM once every warp that touches it is done (also after a
    // timeout: every wait above is bounded).
    tm_wait_st();
    tm_wait_ld();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    asm volatile("bar.sync 1, %0;" ::"n"(32 * (kTmThreadsWarps - 1)) : "memory");
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm_base),
                     "r"(kTmColsAlloc)
                     : "memory");
    }
}

template <int ELEM>
cudaError_t launch_tm(const KArgs &a, unsigned grid, int threads, int smem, cudaStream_t s) {
    auto k = dedisperse_tm_kernel<ELEM>;
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
    if (threads != 32 * kTmThreadsWarps)
        return cudaErrorInvalidValue;
    k<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace
}  // namespace dd
