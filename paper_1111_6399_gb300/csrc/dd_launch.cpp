// Host side of a de-dispersion launch: kernel arguments, the per-dtype kernel
// dispatch and the profiling-event hook.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <functional>
#include <mutex>
#include <queue>
#include <string>
#include <vector>

#include "dd_internal.h"
#include "dd_kargs.h"

namespace dd {
namespace {

thread_local cudaEvent_t g_prof_start = nullptr;
thread_local cudaEvent_t g_prof_stop = nullptr;

// Per-device stream for remainder-DM launches, with the fork and join events.
// One mutex per device keeps each fork / launch / join sequence whole when
// several host threads enqueue at once.
struct SideStream {
    std::mutex mu;
    bool ready = false;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
SideStream g_side[64];

// Cost of a remainder tile relative to a main tile holding as many adds: its
// windows are staged for fewer DMs and its stages hold fewer channels
// (measured 1.33 on the L-band beam: 0.415 ms against 0.312 ms).
constexpr double kTailCost = 1.4;
// Shared memory of an SM available to resident CTAs (228 KB less 1 KB per
// CTA the system reserves).
constexpr int kSmemPerSm = 233472;

int sm_count(int dev) {
    static int cached[64] = {0};
    if (dev < 0 || dev >= 64)
        return 0;
    if (cached[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        cached[dev] = n;
    }
    return cached[dev];
}

int resident(const Geometry &g) { return std::max(1, kSmemPerSm / (g.smem + 1024)); }

// Whether running the remainder DMs as their own launch finishes earlier than
// padding the last DM tile, in units of one main tile's time, with CTAs
// dispatched in launch order (the main launch's first) to `slots` = SMs x
// resident CTAs: padded, ceil(main + ntile_t tiles / slots) rounds; split,
// the main launch's rounds, with the remainder tiles (cost kTailCost times
// their share of a main tile's adds) taking the first free slots from the
// start of its last round on.
bool split_pays(const Geometry &g, const Geometry &gt, int64_t ntile_t, int64_t ntile_t_tail,
                int sms) {
    const int64_t slots = (int64_t)sms * resident(g);
    if (slots <= 0)
        return false;
    const int64_t n_pad = ntile_t * g.ntile_d;
    const int64_t n_main = ntile_t * (g.ntile_d - 1);
    const double t_pad = (double)((n_pad + slots - 1) / slots);
    const int64_t rounds = (n_main + slots - 1) / slots;
    const double c = kTailCost * ((double)gt.dm_cta * gt.t_cta) / ((double)g.dm_cta * g.t_cta);
    // free time of each slot after the main launch: idle ones from the start
    // of the last round, the others from its end
    const int64_t idle = rounds * slots - n_main;
    std::vector<double> free_at((size_t)slots, (double)rounds);
    for (int64_t i = 0; i < idle && i < slots; ++i)
        free_at[(size_t)i] = (double)(rounds > 0 ? rounds - 1 : 0);
    std::priority_queue<double, std::vector<double>, std::greater<double>> q(free_at.begin(),
                                                                             free_at.end());
    double t_split = (double)rounds;
    for (int64_t k = 0; k < ntile_t_tail * gt.ntile_d; ++k) {
        const double t0 = q.top();
        q.pop();
        q.push(t0 + c);
        t_split = std::max(t_split, t0 + c);
    }
    return t_split < t_pad - 0.05;
}

// One launch over DM tiles [0, ntile_d) of geometry g, the sorted DMs from
// d0 on.
cudaError_t enqueue(dd_plan_s *p, const Geometry &g, const DevTables &dt, int d0, int ntile_d,
                    const void *in, dd_dtype dtype, int64_t in_pitch, int64_t nsamp_in,
                    float *out, int64_t out_pitch, int64_t nsamp_out, cudaStream_t s,
                    const DetectTargets *det = nullptr, int *det_cnt = nullptr) {
    KArgs a{};
    BeamArgs &b = a.beam0;
    b.in = static_cast<const uint8_t *>(in);
    b.in_pitch_b = in_pitch * g.elem;
    b.nsamp_in = nsamp_in;
    b.out = out;
    b.out_pitch = out_pitch;
    b.nsamp_out = nsamp_out;
    b.dmshift = dt.dmshift;
    b.dm_sorted = dt.dm_sorted + d0;
    b.perm = dt.perm + d0;
    b.tile_begin = 0;
    b.nchan = p->nchan;
    b.ntile_d = ntile_d;
    b.wp = g.wp;
    a.beams = nullptr;
    a.nbeams = 1;
    a.tile_counter = nullptr;
    a.dm_warps = g.tiles.dm_warps;
    a.time_warps = g.tiles.time_warps;
    a.cstage = g.tiles.chan_per_stage;
    a.nstages = g.nstages;
    a.stage_bytes = g.stage_bytes;
    a.zero_bytes = g.zero_bytes;
    a.builders = g.builders;
    a.one = 1u;
    a.status = dt.status;
    const int64_t ntile_t = (nsamp_out + g.t_cta - 1) / g.t_cta;
    a.total_tiles = ntile_t * ntile_d;
    if (det) {
        a.det_s1 = reinterpret_cast<unsigned long long *>(det->mean);
        a.det_s2 = reinterpret_cast<unsigned long long *>(det->sd);
        a.det_keys = reinterpret_cast<unsigned long long *>(det->snr);
        a.det_cnt = det_cnt;
        a.det_nlevels = det->nlevels;
        a.det_ntile_t = (int)ntile_t;
    }
    const unsigned grid = (unsigned)a.total_tiles;
    const int dthr = g.tiles.dm_per_thread, nw = g.tiles.words_per_thread;
    switch (dtype) {
    case DD_U8: return launch_kernel_u8(a, grid, g.threads, g.smem, s, dthr, nw);
    case DD_F16: return launch_kernel_f16(a, grid, g.threads, g.smem, s, dthr, nw);
    case DD_F32: return launch_kernel_f32(a, grid, g.threads, g.smem, s, dthr, nw);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

dd_status launch_dedisperse_detect(dd_plan_s *p, const Geometry &g, const DevTables &dt,
                                   const void *in, int64_t in_pitch, int64_t nsamp_in,
                                   float *out, int64_t out_pitch, int64_t nsamp_out,
                                   const DetectTargets &det, int *det_cnt, void *stream) {
    if (g.tiles.dm_per_thread != 4 || g.tiles.words_per_thread != 8 || g.tiles.time_warps != 1 ||
        g.t_cta != 1024)
        return fail(DD_ERR_INVALID, "fused detection needs 4 DMs x 8 words per thread and one "
                                    "time warp (1024-sample tiles)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (g_prof_start)
        cudaEventRecord(g_prof_start, s);
    const cudaError_t e = enqueue(p, g, dt, 0, g.ntile_d, in, DD_U8, in_pitch, nsamp_in, out,
                                  out_pitch, nsamp_out, s, &det, det_cnt);
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    if (g_prof_stop)
        cudaEventRecord(g_prof_stop, s);
    count_launch(1);
    return DD_OK;
}

dd_status launch_dedisperse(dd_plan_s *p, const Geometry &g, const DevTables &dt, const void *in,
                            dd_dtype dtype, int64_t in_pitch, int64_t nsamp_in, float *out,
                            int64_t out_pitch, int64_t nsamp_out, void *stream,
                            bool split_tail) {
    if (nsamp_out == 0)
        return DD_OK;
    const int64_t ntile_t = (nsamp_out + g.t_cta - 1) / g.t_cta;
    if (ntile_t * g.ntile_d > 0x7fffffffLL)
        return fail(DD_ERR_INVALID, "too many tiles for one launch");
    bool split = false;
    Geometry gt;
    if (split_tail) {
        dd_status st = tail_geometry(p, dtype, g, &split, &gt);
        if (st != DD_OK)
            return st;
        int dev = 0;
        if (split && cudaGetDevice(&dev) == cudaSuccess)
            split = split_pays(g, gt, ntile_t, (nsamp_out + gt.t_cta - 1) / gt.t_cta,
                               sm_count(dev));
        else
            split = false;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (g_prof_start)
        cudaEventRecord(g_prof_start, s);
    cudaError_t e = cudaSuccess;
    if (!split) {
        e = enqueue(p, g, dt, 0, g.ntile_d, in, dtype, in_pitch, nsamp_in, out, out_pitch,
                    nsamp_out, s);
        if (e != cudaSuccess)
            return fail(DD_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    } else {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess || dev >= 64)
            return fail(DD_ERR_CUDA, "cudaGetDevice failed");
        SideStream &ss = g_side[dev];
        std::lock_guard<std::mutex> lk(ss.mu);
        if (!ss.ready) {
            if (cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming) != cudaSuccess)
                return fail(DD_ERR_CUDA, "remainder stream creation failed");
            ss.ready = true;
        }
        const int d_full = (p->ndm / g.dm_cta) * g.dm_cta;
        // Full DM tiles on the caller's stream; the remainder on the side
        // stream, ordered after everything before it on `s`, and `s` waits
        // for it before anything later.
        e = cudaEventRecord(ss.fork, s);
        if (e == cudaSuccess)
            e = enqueue(p, g, dt, 0, d_full / g.dm_cta, in, dtype, in_pitch, nsamp_in, out,
                        out_pitch, nsamp_out, s);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(ss.s, ss.fork, 0);
        if (e == cudaSuccess)
            e = enqueue(p, gt, dt, d_full, gt.ntile_d, in, dtype, in_pitch, nsamp_in, out,
                        out_pitch, nsamp_out, ss.s);
        if (e == cudaSuccess)
            e = cudaEventRecord(ss.join, ss.s);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(s, ss.join, 0);
        if (e != cudaSuccess)
            return fail(DD_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    }
    if (g_prof_stop)
        cudaEventRecord(g_prof_stop, s);
    count_launch(split ? 2 : 1);
    return DD_OK;
}

}  // namespace dd

extern "C" void dd_profile_events(void *start_event, void *stop_event) {
    dd::g_prof_start = static_cast<cudaEvent_t>(start_event);
    dd::g_prof_stop = static_cast<cudaEvent_t>(stop_event);
}
