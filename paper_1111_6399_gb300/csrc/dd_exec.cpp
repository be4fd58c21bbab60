// Entry points that run the de-dispersion kernel: dd_execute (device
// buffers, asynchronous), dd_execute_host (host buffers, pipelined copies)
// and dd_sync (device status word).
#include <cuda_runtime_api.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dd_internal.h"

namespace {

using dd::fail;

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

using dd::check_layout;

struct HostWorkspace {
    int dev = -1;
    void *in[2] = {nullptr, nullptr};
    float *out[2] = {nullptr, nullptr};
    size_t in_bytes = 0, out_bytes = 0;
    cudaStream_t s[2] = {nullptr, nullptr};
    cudaEvent_t landed[2] = {nullptr, nullptr};   // slot's input block copied in
    cudaEvent_t tail_read[2] = {nullptr, nullptr};  // next slot has read this slot's tail
};

}  // namespace

namespace dd {

dd_status check_layout(dd_plan_s *p, dd_dtype dtype, int64_t in_pitch, int64_t nsamp_in,
                       int64_t out_pitch, int64_t nsamp_out, bool device_rows) {
    if (dtype != DD_U8 && dtype != DD_F16 && dtype != DD_F32)
        return fail(DD_ERR_INVALID, "unknown dtype");
    if (nsamp_out < 0 || nsamp_in < 0)
        return fail(DD_ERR_INVALID, "negative sample count");
    if (nsamp_out > 0 && nsamp_in < nsamp_out + p->maxshift)
        return fail(DD_ERR_INVALID, "nsamp_in must be >= nsamp_out + maxshift (" +
                                        std::to_string(nsamp_out + p->maxshift) + ")");
    if (in_pitch < nsamp_in || out_pitch < nsamp_out)
        return fail(DD_ERR_INVALID, "pitch shorter than a row");
    if (device_rows) {
        const int64_t elem = elem_size(dtype);
        if ((in_pitch * elem) % 16 != 0 || out_pitch % 4 != 0)
            return fail(DD_ERR_INVALID, "row pitches must be multiples of 16 bytes");
    }
    return DD_OK;
}

}  // namespace dd

extern "C" dd_status dd_execute(dd_plan_t p, const void *in, dd_dtype dtype, int64_t in_pitch,
                                int64_t nsamp_in, float *out, int64_t out_pitch,
                                int64_t nsamp_out, void *stream) {
    dd::Range nvtx_range("dd_execute");
    if (!p)
        return fail(DD_ERR_INVALID, "plan is NULL");
    dd_status st = check_layout(p, dtype, in_pitch, nsamp_in, out_pitch, nsamp_out, true);
    if (st != DD_OK)
        return st;
    if (nsamp_out == 0)
        return DD_OK;
    if (!in || !out || !aligned16(in) || !aligned16(out))
        return fail(DD_ERR_INVALID, "in and out must be non-NULL and 16-byte aligned");
    dd::Geometry g;
    if ((st = dd::plan_geometry(p, dtype, &g)) != DD_OK)
        return st;
    dd::DevTables *dt = nullptr;
    if ((st = dd::device_tables(p, &dt)) != DD_OK)
        return st;
    return dd::launch_dedisperse(p, g, *dt, in, dtype, in_pitch, nsamp_in, out, out_pitch,
                                 nsamp_out, stream);
}

extern "C" dd_status dd_sync(dd_plan_t p, void *stream) {
    if (!p)
        return fail(DD_ERR_INVALID, "plan is NULL");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("stream synchronize: ") + cudaGetErrorString(e));
    dd::DevTables *dt = nullptr;
    dd_status st = dd::device_tables(p, &dt);
    if (st != DD_OK)
        return st;
    int word = 0;
    if (cudaMemcpy(&word, dt->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(DD_ERR_CUDA, "status read failed");
    if (word != dd::kDevOk) {
        cudaMemset(dt->status, 0, sizeof(int));
        return word == dd::kDevTimeout
                   ? fail(DD_ERR_TIMEOUT, "a device wait ran out (copy never completed)")
                   : fail(DD_ERR_DEVICE, "kernel recorded a failed internal check");
    }
    return DD_OK;
}

// The host form streams the beam through the GPU in output blocks of B
// samples.  Input block k covers samples [kB, kB + B + S) of every channel;
// its first S samples are the previous block's last S, so they are copied
// device-to-device from the other slot and only B new samples per channel
// cross the host link.  Two slots alternate on two streams, so the input copy
// of block k+1 overlaps the kernel and output copy of block k.
extern "C" dd_status dd_execute_host(dd_plan_t p, const void *in_host, dd_dtype dtype,
                                     int64_t in_pitch, int64_t nsamp_in, float *out_host,
                                     int64_t out_pitch, int64_t nsamp_out) {
    dd::Range nvtx_range("dd_execute_host");
    static std::mutex ws_mu;
    static HostWorkspace ws_by_dev[16];
    if (!p)
        return fail(DD_ERR_INVALID, "plan is NULL");
    dd_status st = check_layout(p, dtype, in_pitch, nsamp_in, out_pitch, nsamp_out, false);
    if (st != DD_OK)
        return st;
    if (nsamp_out == 0)
        return DD_OK;
    if (!in_host || !out_host)
        return fail(DD_ERR_INVALID, "NULL host buffer");
    dd::Geometry g;
    if ((st = dd::plan_geometry(p, dtype, &g)) != DD_OK)
        return st;
    dd::DevTables *dt = nullptr;
    if ((st = dd::device_tables(p, &dt)) != DD_OK)
        return st;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 16)
        return fail(DD_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lk(ws_mu);
    HostWorkspace &ws = ws_by_dev[dev];

    const int64_t elem = dd::elem_size(dtype);
    const int64_t S = p->maxshift;
    // Output blocks: short first and last blocks (the first block's input
    // copy and the last block's output copy overlap no kernel), long middle
    // blocks (each output copy overlaps the next block's kernel).
    std::vector<int64_t> blocks;
    {
        const int64_t mid = std::max<int64_t>(49152, 2 * S);
        const int64_t edge = std::min<int64_t>(16384, std::max<int64_t>(4096, nsamp_out / 8));
        if (nsamp_out <= 2 * edge + mid / 2) {
            for (int64_t t = 0; t < nsamp_out; t += mid)
                blocks.push_back(std::min(mid, nsamp_out - t));
        } else {
            const int64_t rest = nsamp_out - 2 * edge;
            const int64_t m = (rest + mid - 1) / mid;
            blocks.push_back(edge);
            for (int64_t j = 0; j < m; ++j)
                blocks.push_back(rest / m + (j < rest % m ? 1 : 0));
            blocks.push_back(edge);
        }
    }
    const int64_t B = *std::max_element(blocks.begin(), blocks.end());
    const int64_t dpitch_in = ((B + S) * elem + 15) / 16 * 16;   // bytes
    const int64_t dpitch_out = (B + 3) / 4 * 4;                 // floats
    const size_t need_in = (size_t)dpitch_in * p->nchan;
    const size_t need_out = (size_t)dpitch_out * sizeof(float) * p->ndm;
    if (ws.s[0] == nullptr) {
        for (int i = 0; i < 2; ++i) {
            if (cudaStreamCreateWithFlags(&ws.s[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ws.landed[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ws.tail_read[i], cudaEventDisableTiming) != cudaSuccess)
                return fail(DD_ERR_CUDA, "stream/event creation failed");
        }
    }
    if (ws.in_bytes < need_in || ws.out_bytes < need_out) {
        for (int i = 0; i < 2; ++i) {
            cudaFree(ws.in[i]);
            cudaFree(ws.out[i]);
            ws.in[i] = nullptr;
            ws.out[i] = nullptr;
        }
        ws.in_bytes = ws.out_bytes = 0;
        for (int i = 0; i < 2; ++i) {
            if (cudaMalloc(&ws.in[i], need_in) != cudaSuccess ||
                cudaMalloc((void **)&ws.out[i], need_out) != cudaSuccess) {
                cudaGetLastError();
                return fail(DD_ERR_NOMEM, "device workspace allocation failed");
            }
        }
        ws.in_bytes = need_in;
        ws.out_bytes = need_out;
    }
    const uint8_t *src = static_cast<const uint8_t *>(in_host);
    const int64_t hpitch_in = in_pitch * elem;
    const int64_t nblk = (int64_t)blocks.size();
    int64_t t0 = 0, prev_nb = 0;
    for (int64_t k = 0; k < nblk; t0 += blocks[k], prev_nb = blocks[k], ++k) {
        const int i = (int)(k & 1);
        cudaStream_t s = ws.s[i];
        const int64_t nb = blocks[k];
        uint8_t *din = static_cast<uint8_t *>(ws.in[i]);
        cudaError_t e = cudaSuccess;
        if (k >= 2)  // the block after the previous user of this slot read its tail
            e = cudaStreamWaitEvent(s, ws.tail_read[i], 0);
        if (e == cudaSuccess && k == 0) {
            e = cudaMemcpy2DAsync(din, dpitch_in, src, hpitch_in, (size_t)((nb + S) * elem),
                                  p->nchan, cudaMemcpyHostToDevice, s);
        } else if (e == cudaSuccess) {
            e = cudaStreamWaitEvent(s, ws.landed[1 - i], 0);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(din, dpitch_in,
                                      static_cast<uint8_t *>(ws.in[1 - i]) + prev_nb * elem,
                                      dpitch_in, (size_t)(S * elem), p->nchan,
                                      cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaEventRecord(ws.tail_read[1 - i], s);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(din + S * elem, dpitch_in, src + (t0 + S) * elem, hpitch_in,
                                      (size_t)(nb * elem), p->nchan, cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(ws.landed[i], s);
        if (e != cudaSuccess)
            return fail(DD_ERR_CUDA, std::string("input copy: ") + cudaGetErrorString(e));
        st = dd::launch_dedisperse(p, g, *dt, din, dtype, dpitch_in / elem, nb + S,
                                       ws.out[i], dpitch_out, nb, s);
        if (st != DD_OK)
            return st;
        e = cudaMemcpy2DAsync(out_host + t0, (size_t)out_pitch * sizeof(float), ws.out[i],
                              (size_t)dpitch_out * sizeof(float), (size_t)nb * sizeof(float),
                              p->ndm, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess)
            return fail(DD_ERR_CUDA, std::string("output copy: ") + cudaGetErrorString(e));
    }
    for (int i = 0; i < 2; ++i) {
        cudaError_t e = cudaStreamSynchronize(ws.s[i]);
        if (e != cudaSuccess)
            return fail(DD_ERR_CUDA, std::string("synchronize: ") + cudaGetErrorString(e));
    }
    return dd_sync(p, nullptr);
}

// De-dispersion of a uint8 beam with the boxcar search of dd_detect fused
// into the kernel's epilogue: the plane is written to out as by dd_execute,
// and each CTA searches the tile it has just finished while it is in L2.
extern "C" dd_status dd_execute_detect(dd_plan_t p, const void *in, dd_dtype dtype,
                                       int64_t in_pitch, int64_t nsamp_in, float *out,
                                       int64_t out_pitch, int64_t nsamp_out, int nlevels,
                                       double *mean, double *std_out, double *snr,
                                       int64_t *t_peak, void *stream) {
    dd::Range nvtx_range("dd_execute_detect");
    if (!p)
        return fail(DD_ERR_INVALID, "plan is NULL");
    if (dtype != DD_U8)
        return fail(DD_ERR_INVALID, "fused detection takes uint8 input (integer planes)");
    dd_status st = check_layout(p, dtype, in_pitch, nsamp_in, out_pitch, nsamp_out, true);
    if (st != DD_OK)
        return st;
    if (nlevels < 1 || nlevels > 9)
        return fail(DD_ERR_INVALID, "nlevels must be 1..9 (boxcar widths up to 256)");
    if (nsamp_out < 1 || nsamp_out > (1LL << 21))
        return fail(DD_ERR_INVALID, "nsamp_out must be 1 .. 2^21 for an integer search");
    if (!in || !out || !aligned16(in) || !aligned16(out))
        return fail(DD_ERR_INVALID, "in and out must be non-NULL and 16-byte aligned");
    if (!mean || !std_out || !snr || !t_peak || ((uintptr_t)mean & 7u) ||
        ((uintptr_t)std_out & 7u) || ((uintptr_t)snr & 7u) || ((uintptr_t)t_peak & 7u))
        return fail(DD_ERR_INVALID, "NULL or misaligned detection output");
    // Tile shape: the plan's uint8 shape if it has 1024-sample tiles of 4 DMs
    // x 8 words per thread, else the first automatic shape that does.
    dd::Geometry g;
    if ((st = dd::plan_geometry(p, dtype, &g)) != DD_OK)
        return st;
    auto fits = [](const dd::Geometry &x) {
        return x.tiles.dm_per_thread == 4 && x.tiles.words_per_thread == 8 &&
               x.tiles.time_warps == 1 && x.t_cta == 1024;
    };
    if (!fits(g)) {
        bool found = false;
        for (const dd_tiles &cand : dd::auto_tiles(dtype)) {
            dd_tiles t = cand;
            t.time_warps = 1;
            if (t.dm_per_thread == 4 && t.words_per_thread == 8 &&
                dd::make_geometry(p, dtype, t, &g) == DD_OK && fits(g)) {
                found = true;
                break;
            }
        }
        if (!found)
            return fail(DD_ERR_INVALID, "no 1024-sample tile shape fits this plan for fused "
                                        "detection");
    }
    dd::DevTables *dt = nullptr;
    if ((st = dd::device_tables(p, &dt)) != DD_OK)
        return st;
    const int64_t ntile_t = (nsamp_out + g.t_cta - 1) / g.t_cta;
    const int64_t ncnt = ntile_t * g.ntile_d;
    {
        std::lock_guard<std::mutex> lk(p->mu);
        if (dt->det_cnt_n < ncnt) {
            cudaFree(dt->det_cnt);
            dt->det_cnt = nullptr;
            dt->det_cnt_n = 0;
            if (cudaMalloc((void **)&dt->det_cnt, sizeof(int) * (size_t)ncnt) != cudaSuccess) {
                cudaGetLastError();
                return fail(DD_ERR_NOMEM, "detection counter allocation failed");
            }
            dt->det_cnt_n = ncnt;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(dt->det_cnt, 0, sizeof(int) * (size_t)ncnt, s);
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("counter memset: ") + cudaGetErrorString(e));
    if ((st = dd::detect_begin(p->ndm, nlevels, mean, std_out, snr, s)) != DD_OK)
        return st;
    dd::DetectTargets det;
    det.nlevels = nlevels;
    det.mean = mean;
    det.sd = std_out;
    det.snr = snr;
    det.tpk = t_peak;
    if ((st = dd::launch_dedisperse_detect(p, g, *dt, in, in_pitch, nsamp_in, out, out_pitch,
                                           nsamp_out, det, dt->det_cnt, stream)) != DD_OK)
        return st;
    return dd::detect_finalize_int(p->ndm, nsamp_out, nlevels, mean, std_out, snr, t_peak, s);
}

// Candidate tile shapes of the autotuner (validated later by make_geometry).
static std::vector<dd_tiles> tune_candidates(dd_dtype t) {
    std::vector<dd_tiles> out;
    const int dthrs[3] = {1, 2, 4};
    const int nws[2] = {8, 4};
    const int dws[9] = {4, 6, 8, 10, 12, 13, 16, 20, 24};
    const int wts[3] = {1, 2, 4};
    const int css[5] = {4, 8, 12, 16, 24};
    for (int nw : nws)
        for (int dthr : dthrs)
            for (int dw : dws)
                for (int wt : wts) {
                    const int w = dw * wt;
                    if (w > dd::max_consumer_warps(dthr, nw) || w < 8)
                        continue;
                    for (int cs : css) {
                        const int limit = t == DD_U8 ? dd::kSwarChannels : dd::kFloatBlock;
                        if (cs > limit)
                            continue;
                        out.push_back(dd_tiles{dthr, dw, wt, cs, nw});
                    }
                }
    return out;
}

extern "C" dd_status dd_autotune(dd_plan_t p, const void *in, dd_dtype dtype, int64_t in_pitch,
                                 int64_t nsamp_in, float *out, int64_t out_pitch,
                                 int64_t nsamp_out, void *stream, int reps,
                                 dd_tune_result *results, int max_results, int *n_results) {
    dd::Range nvtx_range("dd_autotune");
    if (!p)
        return fail(DD_ERR_INVALID, "plan is NULL");
    dd_status st = check_layout(p, dtype, in_pitch, nsamp_in, out_pitch, nsamp_out, true);
    if (st != DD_OK)
        return st;
    if (nsamp_out == 0 || reps < 1)
        return fail(DD_ERR_INVALID, "autotune needs nsamp_out > 0 and reps >= 1");
    if (!in || !out || !aligned16(in) || !aligned16(out))
        return fail(DD_ERR_INVALID, "in and out must be non-NULL and 16-byte aligned");
    dd::DevTables *dt = nullptr;
    if ((st = dd::device_tables(p, &dt)) != DD_OK)
        return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(DD_ERR_CUDA, "event creation failed");
    float best = -1.0f;
    dd_tiles best_tiles{};
    int n = 0;
    for (const dd_tiles &cand : tune_candidates(dtype)) {
        dd::Geometry g;
        float ms = -1.0f;
        if (dd::make_geometry(p, dtype, cand, &g) == DD_OK) {
            st = dd::launch_dedisperse(p, g, *dt, in, dtype, in_pitch, nsamp_in, out,
                                           out_pitch, nsamp_out, s);  // warm-up
            for (int r = 0; r < reps && st == DD_OK; ++r) {
                cudaEventRecord(e0, s);
                st = dd::launch_dedisperse(p, g, *dt, in, dtype, in_pitch, nsamp_in, out,
                                               out_pitch, nsamp_out, s);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    st = fail(DD_ERR_CUDA, "autotune synchronize failed");
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
                best_tiles = cand;
            }
        }
        if (results && n < max_results)
            results[n] = dd_tune_result{cand, ms};
        ++n;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_results)
        *n_results = n;
    if (st != DD_OK)
        return st;
    if (best < 0.0f)
        return fail(DD_ERR_INVALID, "no candidate tile shape fits this plan");
    if ((st = dd_sync(p, stream)) != DD_OK)
        return st;
    return dd_plan_set_tiles(p, dtype, &best_tiles);
}
