// Host side of a de-dispersion launch: kernel arguments, the per-dtype kernel
// dispatch and the profiling-event hook.
#include <cuda_runtime_api.h>

#include <string>

#include "dd_internal.h"
#include "dd_kargs.h"

namespace dd {
namespace {

thread_local cudaEvent_t g_prof_start = nullptr;
thread_local cudaEvent_t g_prof_stop = nullptr;

}  // namespace

dd_status launch_dedisperse(dd_plan_s *p, const Geometry &g, const DevTables &dt, const void *in,
                            dd_dtype dtype, int64_t in_pitch, int64_t nsamp_in, float *out,
                            int64_t out_pitch, int64_t nsamp_out, void *stream) {
    if (nsamp_out == 0)
        return DD_OK;
    KArgs a{};
    BeamArgs &b = a.beam0;
    b.in = static_cast<const uint8_t *>(in);
    b.in_pitch_b = in_pitch * g.elem;
    b.nsamp_in = nsamp_in;
    b.out = out;
    b.out_pitch = out_pitch;
    b.nsamp_out = nsamp_out;
    b.dmshift = dt.dmshift;
    b.dm_sorted = dt.dm_sorted;
    b.perm = dt.perm;
    b.tile_begin = 0;
    b.nchan = p->nchan;
    b.ntile_d = g.ntile_d;
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
    const int64_t ntiles = ntile_t * g.ntile_d;
    if (ntiles > 0x7fffffffLL)
        return fail(DD_ERR_INVALID, "too many tiles for one launch");
    a.total_tiles = ntiles;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (g_prof_start)
        cudaEventRecord(g_prof_start, s);
    const unsigned grid = (unsigned)ntiles;
    const int dthr = g.tiles.dm_per_thread, nw = g.tiles.words_per_thread;
    switch (dtype) {
    case DD_U8: e = launch_kernel_u8(a, grid, g.threads, g.smem, s, dthr, nw); break;
    case DD_F16: e = launch_kernel_f16(a, grid, g.threads, g.smem, s, dthr, nw); break;
    case DD_F32: e = launch_kernel_f32(a, grid, g.threads, g.smem, s, dthr, nw); break;
    }
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    if (g_prof_stop)
        cudaEventRecord(g_prof_stop, s);
    count_launch(1);
    return DD_OK;
}

}  // namespace dd

extern "C" void dd_profile_events(void *start_event, void *stop_event) {
    dd::g_prof_start = static_cast<cudaEvent_t>(start_event);
    dd::g_prof_stop = static_cast<cudaEvent_t>(stop_event);
}
