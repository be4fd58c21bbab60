// Batches: many uneven beams de-dispersed by one persistent launch, captured
// in a CUDA graph.
//
// Each beam keeps its own plan, buffers and geometry (row width in shared
// memory, number of DM tiles); all beams share one tile shape, so one kernel
// instantiation and one shared-memory layout serve the whole batch.  Beam
// descriptors live in device memory in scheduling order -- largest per-tile
// cost (channel count) first -- and the kernel's producer warps claim global
// tile numbers from an atomic counter, so big beams start first and small
// tiles fill the tail.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "dd_internal.h"
#include "dd_kargs.h"

namespace {

using dd::fail;

struct BatchBeam {
    dd_plan_s *plan = nullptr;
    const void *in = nullptr;
    int64_t in_pitch = 0, nsamp_in = 0;
    float *out = nullptr;
    int64_t out_pitch = 0, nsamp_out = 0;
    bool bound = false;
    dd::Geometry g;
    int64_t ntiles = 0;
};

}  // namespace

struct dd_batch_s {
    dd_dtype dtype = DD_U8;
    std::vector<BatchBeam> beams;
    dd_tiles tiles{};
    bool tiles_set = false;
    int dev = -1;
    dd::BeamArgs *d_beams = nullptr;
    int *d_counter = nullptr;
    int *d_status = nullptr;
    dd::KArgs args{};
    unsigned grid = 0;
    int threads = 0, smem = 0;
    int64_t total_tiles = 0;
    bool prepared = false;
    cudaStream_t capture = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::mutex mu;
};

namespace {

bool fits_all(dd_batch_s *b, const dd_tiles &tl) {
    for (auto &bb : b->beams) {
        dd::Geometry g;
        if (dd::make_geometry(bb.plan, b->dtype, tl, &g) != DD_OK)
            return false;
    }
    return true;
}

void drop_graph(dd_batch_s *b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->prepared = false;
}

// Geometry, descriptors and launch shape for the current tiles.
dd_status prepare(dd_batch_s *b) {
    if (b->prepared)
        return DD_OK;
    for (size_t i = 0; i < b->beams.size(); ++i)
        if (!b->beams[i].bound)
            return fail(DD_ERR_INVALID, "beam " + std::to_string(i) + " has no buffers bound");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return fail(DD_ERR_CUDA, "cudaGetDevice failed");
    if (b->dev >= 0 && dev != b->dev)
        return fail(DD_ERR_INVALID, "a batch is bound to the device it was first executed on");
    b->dev = dev;
    if (!b->tiles_set) {
        bool found = false;
        for (const dd_tiles &cand : dd::auto_tiles(b->dtype))
            if (fits_all(b, cand)) {
                b->tiles = cand;
                found = true;
                break;
            }
        if (!found)
            return fail(DD_ERR_INVALID, "no tile shape fits every beam of the batch");
        b->tiles_set = true;
    }
    const int elem = dd::elem_size(b->dtype);
    int64_t stage_max = 0;
    for (auto &bb : b->beams) {
        dd_status st = dd::make_geometry(bb.plan, b->dtype, b->tiles, &bb.g);
        if (st != DD_OK)
            return st;
        stage_max = std::max<int64_t>(stage_max, bb.g.stage_bytes);
        bb.ntiles = (int64_t)bb.g.ntile_d * ((bb.nsamp_out + bb.g.t_cta - 1) / bb.g.t_cta);
    }
    const dd::Geometry &g0 = b->beams[0].g;
    // Shared-memory layout sized for the widest beam.
    auto smem_for = [&](int64_t n) { return dd::ring_smem(g0, stage_max, (int)n); };
    int nst = 4;
    while (nst > 2 && smem_for(nst) > dd::kMaxSmem)
        --nst;
    if (smem_for(nst) > dd::kMaxSmem)
        return fail(DD_ERR_INVALID, "batch tile shape does not fit shared memory");

    // Scheduling order: larger per-tile cost (channels) first.
    std::vector<int> order(b->beams.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return b->beams[x].plan->nchan > b->beams[y].plan->nchan;
    });
    std::vector<dd::BeamArgs> desc(b->beams.size());
    int64_t tile0 = 0;
    for (size_t k = 0; k < order.size(); ++k) {
        BatchBeam &bb = b->beams[order[k]];
        dd::DevTables *dt = nullptr;
        dd_status st = dd::device_tables(bb.plan, &dt);
        if (st != DD_OK)
            return st;
        dd::BeamArgs &d = desc[k];
        d.in = static_cast<const uint8_t *>(bb.in);
        d.in_pitch_b = bb.in_pitch * elem;
        d.nsamp_in = bb.nsamp_in;
        d.out = bb.out;
        d.out_pitch = bb.out_pitch;
        d.nsamp_out = bb.nsamp_out;
        d.dmshift = dt->dmshift;
        d.dm_sorted = dt->dm_sorted;
        d.perm = dt->perm;
        d.tile_begin = tile0;
        d.nchan = bb.plan->nchan;
        d.ntile_d = bb.g.ntile_d;
        d.wp = bb.g.wp;
        d.pad = 0;
        tile0 += bb.ntiles;
    }
    if (!b->d_beams) {
        if (cudaMalloc((void **)&b->d_beams, sizeof(dd::BeamArgs) * b->beams.size()) != cudaSuccess ||
            cudaMalloc((void **)&b->d_counter, sizeof(int)) != cudaSuccess ||
            cudaMalloc((void **)&b->d_status, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            return fail(DD_ERR_NOMEM, "batch descriptor allocation failed");
        }
        cudaMemset(b->d_status, 0, sizeof(int));
    }
    if (cudaMemcpy(b->d_beams, desc.data(), sizeof(dd::BeamArgs) * desc.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(DD_ERR_CUDA, "batch descriptor upload failed");
    if (tile0 > 0x7fffffffLL)
        return fail(DD_ERR_INVALID, "too many tiles in one batch");
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    b->total_tiles = tile0;
    b->grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tile0, nsm > 0 ? nsm : 1));
    b->threads = g0.threads;
    b->smem = (int)smem_for(nst);
    dd::KArgs &a = b->args;
    a = dd::KArgs{};
    a.beams = b->d_beams;
    a.nbeams = (int)b->beams.size();
    a.total_tiles = tile0;
    a.tile_counter = b->d_counter;
    a.dm_warps = b->tiles.dm_warps;
    a.time_warps = b->tiles.time_warps;
    a.cstage = b->tiles.chan_per_stage;
    a.nstages = nst;
    a.stage_bytes = (int)stage_max;
    a.zero_bytes = g0.zero_bytes;
    a.builders = g0.builders;
    a.one = 1u;
    a.status = b->d_status;
    b->prepared = true;
    return DD_OK;
}

// The tile counter reset, then the persistent de-dispersion launch.
dd_status enqueue(dd_batch_s *b, cudaStream_t s, bool count = true) {
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), s);
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("batch counter reset: ") + cudaGetErrorString(e));
    const int dthr = b->tiles.dm_per_thread, nw = b->tiles.words_per_thread;
    switch (b->dtype) {
    case DD_U8: e = dd::launch_kernel_u8(b->args, b->grid, b->threads, b->smem, s, dthr, nw); break;
    case DD_F16: e = dd::launch_kernel_f16(b->args, b->grid, b->threads, b->smem, s, dthr, nw); break;
    case DD_F32: e = dd::launch_kernel_f32(b->args, b->grid, b->threads, b->smem, s, dthr, nw); break;
    }
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("batch kernel launch: ") + cudaGetErrorString(e));
    if (count)
        dd::count_launch(1);
    return DD_OK;
}

}  // namespace

extern "C" {

dd_status dd_batch_create(const dd_plan_t *plans, int nbeams, dd_dtype dtype, dd_batch_t *out) {
    if (!out)
        return fail(DD_ERR_INVALID, "batch_out is NULL");
    *out = nullptr;
    if (!plans || nbeams < 1)
        return fail(DD_ERR_INVALID, "need at least one plan");
    if (dtype != DD_U8 && dtype != DD_F16 && dtype != DD_F32)
        return fail(DD_ERR_INVALID, "unknown dtype");
    for (int i = 0; i < nbeams; ++i)
        if (!plans[i])
            return fail(DD_ERR_INVALID, "NULL plan in batch");
    dd_batch_s *b = new (std::nothrow) dd_batch_s;
    if (!b)
        return fail(DD_ERR_NOMEM, "out of host memory");
    b->dtype = dtype;
    b->beams.resize(nbeams);
    for (int i = 0; i < nbeams; ++i)
        b->beams[i].plan = plans[i];
    *out = b;
    return DD_OK;
}

void dd_batch_destroy(dd_batch_t b) {
    if (!b)
        return;
    if (b->dev >= 0)
        cudaSetDevice(b->dev);
    cudaDeviceSynchronize();
    drop_graph(b);
    cudaFree(b->d_beams);
    cudaFree(b->d_counter);
    cudaFree(b->d_status);
    if (b->capture)
        cudaStreamDestroy(b->capture);
    delete b;
}

dd_status dd_batch_set_io(dd_batch_t b, int beam, const void *in, int64_t in_pitch,
                          int64_t nsamp_in, float *out, int64_t out_pitch, int64_t nsamp_out) {
    if (!b || beam < 0 || beam >= (int)b->beams.size())
        return fail(DD_ERR_INVALID, "bad batch or beam index");
    BatchBeam &bb = b->beams[beam];
    const int64_t elem = dd::elem_size(b->dtype);
    if (nsamp_out < 1 || nsamp_in < nsamp_out + bb.plan->maxshift)
        return fail(DD_ERR_INVALID, "nsamp_out must be >= 1 and nsamp_in >= nsamp_out + maxshift");
    if (in_pitch < nsamp_in || out_pitch < nsamp_out || (in_pitch * elem) % 16 || out_pitch % 4)
        return fail(DD_ERR_INVALID, "pitches must cover a row and be multiples of 16 bytes");
    if (!in || !out || ((uintptr_t)in & 15u) || ((uintptr_t)out & 15u))
        return fail(DD_ERR_INVALID, "in and out must be non-NULL and 16-byte aligned");
    std::lock_guard<std::mutex> lk(b->mu);
    bb.in = in;
    bb.in_pitch = in_pitch;
    bb.nsamp_in = nsamp_in;
    bb.out = out;
    bb.out_pitch = out_pitch;
    bb.nsamp_out = nsamp_out;
    bb.bound = true;
    drop_graph(b);
    return DD_OK;
}

dd_status dd_batch_get_tiles(dd_batch_t b, dd_tiles *t) {
    if (!b || !t)
        return fail(DD_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(b->mu);
    if (!b->tiles_set) {
        for (const dd_tiles &cand : dd::auto_tiles(b->dtype))
            if (fits_all(b, cand)) {
                b->tiles = cand;
                b->tiles_set = true;
                break;
            }
        if (!b->tiles_set)
            return fail(DD_ERR_INVALID, "no tile shape fits every beam of the batch");
    }
    *t = b->tiles;
    return DD_OK;
}

dd_status dd_batch_set_tiles(dd_batch_t b, const dd_tiles *t) {
    if (!b || !t)
        return fail(DD_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(b->mu);
    for (auto &bb : b->beams) {
        dd::Geometry g;
        dd_status st = dd::make_geometry(bb.plan, b->dtype, *t, &g);
        if (st != DD_OK)
            return st;
    }
    b->tiles = *t;
    b->tiles_set = true;
    drop_graph(b);
    return DD_OK;
}

dd_status dd_batch_execute(dd_batch_t b, void *stream) {
    dd::Range nvtx_range("dd_batch_execute");
    if (!b)
        return fail(DD_ERR_INVALID, "batch is NULL");
    std::lock_guard<std::mutex> lk(b->mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!b->exec) {
        dd_status st = prepare(b);
        if (st != DD_OK)
            return st;
        // One eager run first: it sets the kernel attributes outside any capture.
        if ((st = enqueue(b, s)) != DD_OK)
            return st;
        if (!b->capture &&
            cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess)
            return fail(DD_ERR_CUDA, "capture stream creation failed");
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return fail(DD_ERR_CUDA, "stream capture failed to start");
        st = enqueue(b, b->capture, false);
        cudaError_t e = cudaStreamEndCapture(b->capture, &graph);
        if (st != DD_OK)
            return st;
        if (e != cudaSuccess)
            return fail(DD_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return fail(DD_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        return DD_OK;  // this call's work was the eager run
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    dd::count_launch((int)(b->dtype == DD_F32 ? 1 : b->beams.size() + 1));
    return DD_OK;
}

dd_status dd_batch_sync(dd_batch_t b, void *stream) {
    if (!b)
        return fail(DD_ERR_INVALID, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("stream synchronize: ") + cudaGetErrorString(e));
    if (!b->d_status)
        return DD_OK;
    int word = 0;
    if (cudaMemcpy(&word, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(DD_ERR_CUDA, "status read failed");
    if (word != dd::kDevOk) {
        cudaMemset(b->d_status, 0, sizeof(int));
        return word == dd::kDevTimeout ? fail(DD_ERR_TIMEOUT, "a device wait ran out")
                                       : fail(DD_ERR_DEVICE, "kernel recorded a failed check");
    }
    return DD_OK;
}

dd_status dd_batch_autotune(dd_batch_t b, void *stream, int reps, dd_tune_result *results,
                            int max_results, int *n_results) {
    dd::Range nvtx_range("dd_batch_autotune");
    if (!b || reps < 1)
        return fail(DD_ERR_INVALID, "bad batch or reps");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(DD_ERR_CUDA, "event creation failed");
    std::vector<dd_tiles> cands;
    for (int nw : {8, 4})
        for (int dthr : {4, 2, 1})
            for (int dw : {6, 8, 10, 12, 16})
                for (int cs : {8, 12, 16}) {
                    const int wt = 1;
                    if (dw * wt > dd::max_consumer_warps(dthr, nw))
                        continue;
                    cands.push_back(dd_tiles{dthr, dw, wt, cs, nw});
                }
    float best = -1.0f;
    dd_tiles best_t{};
    int n = 0;
    dd_status st = DD_OK;
    std::lock_guard<std::mutex> lk(b->mu);
    for (const dd_tiles &c : cands) {
        float ms = -1.0f;
        if (fits_all(b, c)) {
            drop_graph(b);
            b->tiles = c;
            b->tiles_set = true;
            if ((st = prepare(b)) != DD_OK)
                break;
            if ((st = enqueue(b, s)) != DD_OK)  // warm-up
                break;
            for (int r = 0; r < reps; ++r) {
                cudaEventRecord(e0, s);
                if ((st = enqueue(b, s)) != DD_OK)
                    break;
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    st = fail(DD_ERR_CUDA, "batch autotune synchronize failed");
                    break;
                }
                float t = 0.0f;
                cudaEventElapsedTime(&t, e0, e1);
                ms = (ms < 0.0f || t < ms) ? t : ms;
            }
            if (st != DD_OK)
                break;
            if (ms >= 0.0f && (best < 0.0f || ms < best)) {
                best = ms;
                best_t = c;
            }
        }
        if (results && n < max_results)
            results[n] = dd_tune_result{c, ms};
        ++n;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_results)
        *n_results = n;
    if (st != DD_OK)
        return st;
    if (best < 0.0f)
        return fail(DD_ERR_INVALID, "no candidate tile shape fits every beam");
    drop_graph(b);
    b->tiles = best_t;
    b->tiles_set = true;
    return DD_OK;
}

}  // extern "C"
