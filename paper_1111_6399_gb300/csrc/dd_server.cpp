// Serving runtime: streams of blocks from many beams, de-dispersed with
// continuous batching.
//
// Each beam keeps the last maxshift samples of every channel on the device
// (its overlap tail).  A block k of B samples is assembled in a device slot
// as [tail | block] (tail copied device-to-device, block copied from pinned
// host staging); the slot's last maxshift samples then become the beam's new
// tail.  A worker thread takes every queued block whose beam is ready (the
// previous block of that beam has been launched, so its tail update is
// ordered before this block's assembly by an event) up to the free slots,
// and launches them together: one persistent de-dispersion launch over all
// their tiles, then the copies of
// the outputs into the callers' buffers.  Batches alternate between two
// streams, so the copies of one batch overlap the kernel of the other.  A
// completion thread watches per-block events, records submit-to-result
// latency and frees slots and staging buffers, which lets the worker admit
// the blocks that arrived meanwhile.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dd_internal.h"
#include "dd_kargs.h"

namespace {

using dd::fail;
using Clock = std::chrono::steady_clock;

struct SrvBeam {
    dd_plan_s *plan = nullptr;
    int64_t B = 0, S = 0;
    void *tail = nullptr;      // device [nchan][tail_pitch] elements
    int64_t tail_pitch = 0;    // elements
    int64_t next_submit = 0;   // index of the next block dd_submit will accept
    int64_t next_launch = 0;   // index of the next block the worker may launch
    bool tail_valid = false;
    cudaEvent_t tail_ready = nullptr;
    dd::Geometry g;
};

enum ReqState { kQueued = 0, kLaunched = 1, kDone = 2, kFailed = 3 };

struct SrvReq {
    int beam = 0;
    int64_t k = 0;
    int staging = -1;
    int slot = -1;
    float *out_host = nullptr;
    int64_t out_pitch = 0;
    Clock::time_point t_submit;
    ReqState state = kQueued;
    cudaEvent_t done = nullptr;
    int64_t first_t = 0, nsamp = 0;
    dd_status err = DD_OK;
};

struct Slot {
    void *in = nullptr;
    float *out = nullptr;
    bool busy = false;
};

struct Lane {  // launch resources of one of the two alternating streams
    cudaStream_t s = nullptr;
    dd::BeamArgs *d_desc = nullptr;
    dd::BeamArgs *h_desc = nullptr;  // pinned
    int *d_counter = nullptr;
    cudaEvent_t done = nullptr;
    // Timing of the last batch on this lane: input copies [t0, t1), kernel
    // [t1, t2), result copies [t2, t3); read when the lane is reused.
    cudaEvent_t t[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t h2d_bytes = 0, d2h_bytes = 0;
    bool accounted = true;  // the last batch's copy statistics are in the server's totals
    bool used = false;
};

// Host threads that copy a submitted block into pinned staging, each a share
// of the channel rows (one host thread's memcpy is far slower than the
// host-to-device link).
class CopyPool {
  public:
    explicit CopyPool(int n) {
        for (int i = 0; i < n; ++i)
            th_.emplace_back([this]() { run(); });
    }
    ~CopyPool() {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : th_)
            t.join();
    }
    // rows [0, n) of `bytes` bytes from src (row pitch sp) to dst (pitch dp);
    // the caller takes one share and waits for the others.
    void copy_rows(uint8_t *dst, int64_t dp, const uint8_t *src, int64_t sp, int64_t n,
                   size_t bytes) {
        const int parts = (int)th_.size() + 1;
        std::unique_lock<std::mutex> lk(mu_);
        job_ = Job{dst, dp, src, sp, n, bytes, parts};
        next_ = 1;
        left_ = parts - 1;
        ++gen_;
        lk.unlock();
        cv_.notify_all();
        part(job_, 0);
        lk.lock();
        cv_done_.wait(lk, [&]() { return left_ == 0; });
    }

  private:
    struct Job {
        uint8_t *dst = nullptr;
        int64_t dp = 0;
        const uint8_t *src = nullptr;
        int64_t sp = 0, n = 0;
        size_t bytes = 0;
        int parts = 1;
    };
    static void part(const Job &j, int k) {
        const int64_t r0 = j.n * k / j.parts, r1 = j.n * (k + 1) / j.parts;
        for (int64_t r = r0; r < r1; ++r)
            std::memcpy(j.dst + r * j.dp, j.src + r * j.sp, j.bytes);
    }
    void run() {
        uint64_t seen = 0;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            cv_.wait(lk, [&]() { return stop_ || (gen_ != seen && next_ < job_.parts); });
            if (stop_)
                return;
            const int k = next_++;
            if (next_ >= job_.parts)
                seen = gen_;
            const Job j = job_;
            lk.unlock();
            part(j, k);
            lk.lock();
            if (--left_ == 0)
                cv_done_.notify_all();
        }
    }
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_, cv_done_;
    Job job_;
    int next_ = 0, left_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};

}  // namespace

struct dd_server_s {
    size_t budget = 0;
    int max_inflight = 0;
    dd_dtype dtype = DD_U8;
    int elem = 1;
    std::vector<SrvBeam> beams;
    bool started = false;
    int dev = 0;
    // device slots and host staging
    std::vector<Slot> slots;
    int64_t in_pitch = 0;      // slot input pitch, elements
    int64_t out_pitch = 0;     // slot output pitch, floats
    size_t in_bytes = 0, out_bytes = 0;
    std::vector<void *> staging;
    std::vector<bool> staging_busy;
    size_t staging_bytes = 0;
    int64_t device_bytes = 0;
    // launch shape
    dd_tiles tiles{};
    int threads = 0, smem = 0, nst = 2, stage_max = 0, zero_bytes = 0, builders = 0, nsm = 1;
    int *d_status = nullptr;
    Lane lanes[2];
    int next_lane = 0;
    // queue, threads, statistics
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<dd_ticket> queued;
    std::deque<dd_ticket> inflight;
    std::map<dd_ticket, SrvReq> reqs;
    dd_ticket next_ticket = 1;
    std::thread worker, completer;
    bool stop = false;
    int64_t window_us = 0;  // how long a partly filled batch waits for more blocks
    bool window_set = false;  // set by the caller (else derived from the block durations)
    int64_t submitted = 0, completed = 0, rejected = 0, batches = 0, batched_blocks = 0;
    std::vector<double> lat_ms;
    CopyPool *pool = nullptr;
    std::mutex submit_mu;  // one staging copy at a time through the pool
    int64_t staged_bytes = 0, h2d_bytes = 0, d2h_bytes = 0;  // copy statistics
    double staged_ms = 0.0, h2d_ms = 0.0, d2h_ms = 0.0, kernel_ms = 0.0;
};

namespace {

size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

void free_all(dd_server_s *v) {
    for (auto &s : v->slots) {
        cudaFree(s.in);
        cudaFree(s.out);
    }
    v->slots.clear();
    for (void *p : v->staging)
        cudaFreeHost(p);
    v->staging.clear();
    for (auto &b : v->beams) {
        cudaFree(b.tail);
        b.tail = nullptr;
        if (b.tail_ready)
            cudaEventDestroy(b.tail_ready);
        b.tail_ready = nullptr;
    }
    for (auto &l : v->lanes) {
        cudaFree(l.d_desc);
        cudaFreeHost(l.h_desc);
        cudaFree(l.d_counter);
        if (l.done)
            cudaEventDestroy(l.done);
        for (cudaEvent_t &ev : l.t)
            if (ev)
                cudaEventDestroy(ev);
        if (l.s)
            cudaStreamDestroy(l.s);
        l = Lane{};
    }
    cudaFree(v->d_status);
    v->d_status = nullptr;
}

// Tile shape, slot layout, device memory within the budget, streams.
dd_status start(dd_server_s *v) {
    if (v->beams.empty())
        return fail(DD_ERR_INVALID, "server has no beams");
    if (cudaGetDevice(&v->dev) != cudaSuccess)
        return fail(DD_ERR_CUDA, "cudaGetDevice failed");
    cudaDeviceGetAttribute(&v->nsm, cudaDevAttrMultiProcessorCount, v->dev);
    if (v->nsm < 1)
        v->nsm = 1;
    bool found = false;
    for (const dd_tiles &cand : dd::auto_tiles(v->dtype)) {
        bool ok = true;
        for (auto &b : v->beams)
            ok = ok && dd::make_geometry(b.plan, v->dtype, cand, &b.g) == DD_OK;
        if (ok) {
            v->tiles = cand;
            found = true;
            break;
        }
    }
    if (!found)
        return fail(DD_ERR_INVALID, "no tile shape fits every beam of the server");
    int64_t nchan_max = 0, ndm_max = 0, B_max = 0, SB_max = 0;
    int64_t stage_max = 0;
    int64_t tails = 0;
    for (auto &b : v->beams) {
        nchan_max = std::max<int64_t>(nchan_max, b.plan->nchan);
        ndm_max = std::max<int64_t>(ndm_max, b.plan->ndm);
        B_max = std::max(B_max, b.B);
        SB_max = std::max(SB_max, b.S + b.B);
        stage_max = std::max<int64_t>(stage_max, b.g.stage_bytes);
        b.tail_pitch = (int64_t)round16((size_t)std::max<int64_t>(b.S, 1) * v->elem) / v->elem;
        tails += (int64_t)b.plan->nchan * b.tail_pitch * v->elem;
    }
    const dd::Geometry &g0 = v->beams[0].g;
    auto smem_for = [&](int64_t n) { return dd::ring_smem(g0, stage_max, (int)n); };
    int nst = 4;
    while (nst > 2 && smem_for(nst) > dd::kMaxSmem)
        --nst;
    if (smem_for(nst) > dd::kMaxSmem)
        return fail(DD_ERR_INVALID, "server tile shape does not fit shared memory");
    v->nst = nst;
    v->smem = (int)smem_for(nst);
    v->threads = g0.threads;
    v->stage_max = (int)stage_max;
    v->zero_bytes = g0.zero_bytes;
    v->builders = g0.builders;

    v->in_pitch = (int64_t)round16((size_t)SB_max * v->elem) / v->elem;
    v->out_pitch = (B_max + 3) / 4 * 4;
    v->in_bytes = (size_t)nchan_max * v->in_pitch * v->elem;
    v->out_bytes = (size_t)ndm_max * v->out_pitch * sizeof(float);
    const size_t slot_bytes = v->in_bytes + v->out_bytes;
    const int64_t room = (int64_t)v->budget - tails;
    const int64_t by_budget = room > 0 ? room / (int64_t)slot_bytes : 0;
    const int nslots = (int)std::min<int64_t>(v->max_inflight, by_budget);
    if (nslots < 1)
        return fail(DD_ERR_NOMEM, "HBM budget too small: tails need " + std::to_string(tails) +
                                      " bytes and one slot " + std::to_string(slot_bytes));
    v->staging_bytes = (size_t)nchan_max * B_max * v->elem;

    bool ok = true;
    for (auto &b : v->beams) {
        ok = ok && cudaMalloc(&b.tail, (size_t)b.plan->nchan * b.tail_pitch * v->elem) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&b.tail_ready, cudaEventDisableTiming) == cudaSuccess;
        dd::DevTables *dt = nullptr;
        ok = ok && dd::device_tables(b.plan, &dt) == DD_OK;
    }
    v->slots.resize(nslots);
    for (auto &s : v->slots) {
        ok = ok && cudaMalloc(&s.in, v->in_bytes) == cudaSuccess;
        ok = ok && cudaMalloc((void **)&s.out, v->out_bytes) == cudaSuccess;
    }
    const int nstaging = 2 * nslots;
    v->staging.assign(nstaging, nullptr);
    v->staging_busy.assign(nstaging, false);
    for (auto &p : v->staging)
        ok = ok && cudaHostAlloc(&p, v->staging_bytes, cudaHostAllocDefault) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&v->d_status, sizeof(int)) == cudaSuccess &&
         cudaMemset(v->d_status, 0, sizeof(int)) == cudaSuccess;
    for (auto &l : v->lanes) {
        ok = ok && cudaStreamCreateWithFlags(&l.s, cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaMalloc((void **)&l.d_desc, sizeof(dd::BeamArgs) * nslots) == cudaSuccess;
        ok = ok && cudaHostAlloc((void **)&l.h_desc, sizeof(dd::BeamArgs) * nslots,
                                 cudaHostAllocDefault) == cudaSuccess;
        ok = ok && cudaMalloc((void **)&l.d_counter, sizeof(int)) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) == cudaSuccess;
        for (cudaEvent_t &ev : l.t)
            ok = ok && cudaEventCreate(&ev) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        free_all(v);
        return fail(DD_ERR_NOMEM, "server device/pinned allocation failed");
    }
    v->device_bytes = tails + (int64_t)slot_bytes * nslots;
    if (!v->window_set) {
        // 1/64 of the shortest block duration, at most 100 ms: far inside the
        // real-time deadline (a block's own duration), long enough for blocks
        // of other beams arriving meanwhile to share a launch.
        double shortest = 1e30;
        for (auto &b : v->beams)
            shortest = std::min(shortest, (double)b.B * b.plan->tsamp);
        v->window_us = (int64_t)std::min(100000.0, shortest * 1e6 / 64.0);
    }
    const unsigned hc = std::thread::hardware_concurrency();
    v->pool = new (std::nothrow) CopyPool((int)std::max(1u, std::min(7u, hc > 1 ? hc / 2 : 1u)));
    v->started = true;
    return DD_OK;
}

// Add the copy statistics of the lane's last (completed) batch to the
// server's totals, once.  Caller holds v->mu.
void account_lane(dd_server_s *v, Lane &l) {
    if (l.accounted)
        return;
    float ms_in = 0.0f, ms_k = 0.0f, ms_out = 0.0f;
    if (cudaEventElapsedTime(&ms_in, l.t[0], l.t[1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms_k, l.t[1], l.t[2]) == cudaSuccess &&
        cudaEventElapsedTime(&ms_out, l.t[2], l.t[3]) == cudaSuccess) {
        v->h2d_bytes += l.h2d_bytes;
        v->d2h_bytes += l.d2h_bytes;
        v->h2d_ms += ms_in;
        v->kernel_ms += ms_k;
        v->d2h_ms += ms_out;
    }
    l.accounted = true;
}

// Launch one batch of (request, slot) pairs on lane l.  Caller holds no lock.
dd_status launch_batch(dd_server_s *v, Lane &l, const std::vector<dd_ticket> &tickets,
                       std::vector<SrvReq *> &rs) {
    cudaStream_t s = l.s;
    const int elem = v->elem;
    cudaError_t e = cudaSuccess;
    if (l.used) {  // descriptors of the previous batch on this lane must be consumed
        e = cudaEventSynchronize(l.done);
        std::lock_guard<std::mutex> lk(v->mu);
        if (e == cudaSuccess)
            account_lane(v, l);
    }
    l.h2d_bytes = l.d2h_bytes = 0;
    if (e == cudaSuccess)
        e = cudaEventRecord(l.t[0], s);
    int64_t tile0 = 0;
    for (size_t i = 0; i < rs.size() && e == cudaSuccess; ++i) {
        SrvReq &r = *rs[i];
        SrvBeam &b = v->beams[r.beam];
        Slot &sl = v->slots[r.slot];
        const int nchan = b.plan->nchan;
        const size_t pitch_b = (size_t)v->in_pitch * elem;
        uint8_t *in = static_cast<uint8_t *>(sl.in);
        // [tail | block]
        if (b.tail_valid) {
            e = cudaStreamWaitEvent(s, b.tail_ready, 0);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(in, pitch_b, b.tail, (size_t)b.tail_pitch * elem,
                                      (size_t)b.S * elem, nchan, cudaMemcpyDeviceToDevice, s);
        } else if (b.S > 0) {
            e = cudaMemset2DAsync(in, pitch_b, 0, (size_t)b.S * elem, nchan, s);
        }
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(in + (size_t)b.S * elem, pitch_b, v->staging[r.staging],
                                  (size_t)b.B * elem, (size_t)b.B * elem, nchan,
                                  cudaMemcpyHostToDevice, s);
        l.h2d_bytes += (int64_t)b.B * elem * nchan;
        // new tail: the last S samples of [tail | block]
        if (e == cudaSuccess && b.S > 0)
            e = cudaMemcpy2DAsync(b.tail, (size_t)b.tail_pitch * elem, in + (size_t)b.B * elem,
                                  pitch_b, (size_t)b.S * elem, nchan, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaEventRecord(b.tail_ready, s);
        b.tail_valid = true;
        dd::DevTables *dt = nullptr;
        dd::device_tables(b.plan, &dt);
        dd::BeamArgs &d = l.h_desc[i];
        d = dd::BeamArgs{};
        d.in = in;
        d.in_pitch_b = (int64_t)pitch_b;
        d.nsamp_in = b.S + b.B;
        d.out = sl.out;
        d.out_pitch = v->out_pitch;
        d.nsamp_out = b.B;
        d.dmshift = dt->dmshift;
        d.dm_sorted = dt->dm_sorted;
        d.perm = dt->perm;
        d.tile_begin = tile0;
        d.nchan = nchan;
        d.ntile_d = b.g.ntile_d;
        d.wp = b.g.wp;
        tile0 += (int64_t)b.g.ntile_d * ((b.B + b.g.t_cta - 1) / b.g.t_cta);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(l.d_desc, l.h_desc, sizeof(dd::BeamArgs) * rs.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(l.d_counter, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = cudaEventRecord(l.t[1], s);
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("server batch staging: ") + cudaGetErrorString(e));
    dd::KArgs a{};
    a.beams = l.d_desc;
    a.nbeams = (int)rs.size();
    a.total_tiles = tile0;
    a.tile_counter = l.d_counter;
    a.dm_warps = v->tiles.dm_warps;
    a.time_warps = v->tiles.time_warps;
    a.cstage = v->tiles.chan_per_stage;
    a.nstages = v->nst;
    a.stage_bytes = v->stage_max;
    a.zero_bytes = v->zero_bytes;
    a.builders = v->builders;
    a.one = 1u;
    a.status = v->d_status;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tile0, v->nsm));
    const int dthr = v->tiles.dm_per_thread, nw = v->tiles.words_per_thread;
    switch (v->dtype) {
    case DD_U8: e = dd::launch_kernel_u8(a, grid, v->threads, v->smem, s, dthr, nw); break;
    case DD_F16: e = dd::launch_kernel_f16(a, grid, v->threads, v->smem, s, dthr, nw); break;
    case DD_F32: e = dd::launch_kernel_f32(a, grid, v->threads, v->smem, s, dthr, nw); break;
    }
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("server kernel launch: ") + cudaGetErrorString(e));
    dd::count_launch(1);
    e = cudaEventRecord(l.t[2], s);
    // results into the callers' buffers
    for (size_t i = 0; i < rs.size() && e == cudaSuccess; ++i) {
        SrvReq &r = *rs[i];
        SrvBeam &b = v->beams[r.beam];
        Slot &sl = v->slots[r.slot];
        const int64_t col0 = r.k == 0 ? b.S : 0;  // block 0: no samples before the stream
        r.first_t = r.k == 0 ? 0 : r.k * b.B - b.S;
        r.nsamp = b.B - col0;
        e = cudaMemcpy2DAsync(r.out_host, (size_t)r.out_pitch * sizeof(float), sl.out + col0,
                              (size_t)v->out_pitch * sizeof(float), (size_t)r.nsamp * sizeof(float),
                              b.plan->ndm, cudaMemcpyDeviceToHost, s);
        l.d2h_bytes += r.nsamp * (int64_t)sizeof(float) * b.plan->ndm;
        if (e == cudaSuccess)
            e = cudaEventRecord(r.done, s);
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(l.t[3], s);
    if (e == cudaSuccess)
        e = cudaEventRecord(l.done, s);
    {
        std::lock_guard<std::mutex> lk(v->mu);
        l.accounted = false;
    }
    l.used = true;
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("server result copy: ") + cudaGetErrorString(e));
    (void)tickets;
    return DD_OK;
}

void worker_main(dd_server_s *v) {
    cudaSetDevice(v->dev);
    std::unique_lock<std::mutex> lk(v->mu);
    while (true) {
        // Blocks whose beam is ready, in submit order, one per beam, up to the free slots.
        std::vector<dd_ticket> pick;
        std::vector<SrvReq *> rs;
        auto collect = [&]() {
            pick.clear();
            rs.clear();
            std::vector<bool> beam_taken(v->beams.size(), false);
            std::vector<int> free_slots;
            for (int i = 0; i < (int)v->slots.size(); ++i)
                if (!v->slots[i].busy)
                    free_slots.push_back(i);
            for (dd_ticket t : v->queued) {
                if (rs.size() >= free_slots.size())
                    break;
                SrvReq &r = v->reqs[t];
                SrvBeam &b = v->beams[r.beam];
                if (beam_taken[r.beam] || r.k != b.next_launch)
                    continue;
                beam_taken[r.beam] = true;
                r.slot = free_slots[rs.size()];
                pick.push_back(t);
                rs.push_back(&r);
            }
            return !rs.empty();
        };
        v->cv_work.wait(lk, [&]() { return v->stop || collect(); });
        if (v->stop && rs.empty())
            break;
        if (v->window_us > 0 && !v->stop) {
            // Let more ready blocks join until the slots are full or the window ends.
            int nfree = 0;
            for (const Slot &sl : v->slots)
                nfree += sl.busy ? 0 : 1;
            const auto until = Clock::now() + std::chrono::microseconds(v->window_us);
            while (!v->stop && (int)rs.size() < nfree &&
                   v->cv_work.wait_until(lk, until) != std::cv_status::timeout)
                collect();
            collect();
            if (rs.empty())
                continue;
        }
        for (size_t i = 0; i < rs.size(); ++i) {
            SrvReq &r = *rs[i];
            v->slots[r.slot].busy = true;
            v->beams[r.beam].next_launch++;
            r.state = kLaunched;
        }
        v->queued.erase(std::remove_if(v->queued.begin(), v->queued.end(),
                                       [&](dd_ticket t) {
                                           return std::find(pick.begin(), pick.end(), t) !=
                                                  pick.end();
                                       }),
                        v->queued.end());
        // The lane whose last batch has finished, else the next in turn.
        int li = v->next_lane;
        if (v->lanes[li].used && cudaEventQuery(v->lanes[li].done) == cudaErrorNotReady &&
            (!v->lanes[li ^ 1].used || cudaEventQuery(v->lanes[li ^ 1].done) != cudaErrorNotReady))
            li ^= 1;
        Lane &l = v->lanes[li];
        v->next_lane = li ^ 1;
        v->batches++;
        v->batched_blocks += (int64_t)rs.size();
        lk.unlock();
        dd_status st = launch_batch(v, l, pick, rs);
        lk.lock();
        for (size_t i = 0; i < rs.size(); ++i) {
            if (st != DD_OK) {
                rs[i]->state = kFailed;
                rs[i]->err = st;
            }
            v->inflight.push_back(pick[i]);
        }
        v->cv_done.notify_all();
    }
}

void completer_main(dd_server_s *v) {
    cudaSetDevice(v->dev);
    std::unique_lock<std::mutex> lk(v->mu);
    while (true) {
        v->cv_done.wait(lk, [&]() { return v->stop || !v->inflight.empty(); });
        if (v->inflight.empty()) {
            if (v->stop)
                break;
            continue;
        }
        bool progress = false;
        for (auto it = v->inflight.begin(); it != v->inflight.end();) {
            SrvReq &r = v->reqs[*it];
            bool finished = r.state == kFailed;
            if (!finished) {
                const cudaError_t q = cudaEventQuery(r.done);
                if (q == cudaSuccess) {
                    r.state = kDone;
                    finished = true;
                } else if (q != cudaErrorNotReady) {
                    r.state = kFailed;
                    r.err = fail(DD_ERR_CUDA, std::string("server block: ") + cudaGetErrorString(q));
                    finished = true;
                }
            }
            if (finished) {
                const double ms =
                    std::chrono::duration<double, std::milli>(Clock::now() - r.t_submit).count();
                if (r.state == kDone)
                    v->lat_ms.push_back(ms);
                v->completed++;
                if (r.slot >= 0)
                    v->slots[r.slot].busy = false;
                if (r.staging >= 0)
                    v->staging_busy[r.staging] = false;
                r.slot = r.staging = -1;
                it = v->inflight.erase(it);
                progress = true;
            } else {
                ++it;
            }
        }
        if (progress) {
            v->cv_work.notify_all();
            v->cv_done.notify_all();
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        }
    }
}

double percentile(std::vector<double> x, double q) {
    if (x.empty())
        return 0.0;
    std::sort(x.begin(), x.end());
    const double pos = q * (double)(x.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < x.size() ? x[i] * (1.0 - f) + x[i + 1] * f : x[i];
}

}  // namespace

extern "C" {

dd_status dd_server_create(size_t hbm_budget_bytes, int max_inflight, dd_dtype dtype,
                           dd_server_t *out) {
    if (!out)
        return fail(DD_ERR_INVALID, "server_out is NULL");
    *out = nullptr;
    if (max_inflight < 1 || hbm_budget_bytes == 0)
        return fail(DD_ERR_INVALID, "need max_inflight >= 1 and a non-zero HBM budget");
    if (dtype != DD_U8 && dtype != DD_F16 && dtype != DD_F32)
        return fail(DD_ERR_INVALID, "unknown dtype");
    dd_server_s *v = new (std::nothrow) dd_server_s;
    if (!v)
        return fail(DD_ERR_NOMEM, "out of host memory");
    v->budget = hbm_budget_bytes;
    v->max_inflight = max_inflight;
    v->dtype = dtype;
    v->elem = dd::elem_size(dtype);
    *out = v;
    return DD_OK;
}

dd_status dd_server_add_beam(dd_server_t v, dd_plan_t plan, int64_t block_nsamp, int *beam_id) {
    if (!v || !plan || !beam_id)
        return fail(DD_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(v->mu);
    if (v->started)
        return fail(DD_ERR_INVALID, "beams must be added before the first dd_submit");
    if (block_nsamp <= plan->maxshift)
        return fail(DD_ERR_INVALID, "block_nsamp must exceed the plan's maxshift (" +
                                        std::to_string(plan->maxshift) + ")");
    SrvBeam b;
    b.plan = plan;
    b.B = block_nsamp;
    b.S = plan->maxshift;
    v->beams.push_back(b);
    *beam_id = (int)v->beams.size() - 1;
    return DD_OK;
}

dd_status dd_submit(dd_server_t v, int beam_id, const void *block_host, int64_t in_pitch,
                    float *out_host, int64_t out_pitch, dd_ticket *ticket) {
    dd::Range nvtx_range("dd_submit");
    if (!v || !block_host || !out_host || !ticket)
        return fail(DD_ERR_INVALID, "NULL argument");
    std::unique_lock<std::mutex> lk(v->mu);
    if (beam_id < 0 || beam_id >= (int)v->beams.size())
        return fail(DD_ERR_INVALID, "unknown beam");
    SrvBeam &b = v->beams[beam_id];
    if (in_pitch < b.B || out_pitch < b.B)
        return fail(DD_ERR_INVALID, "pitches must cover a block (block_nsamp samples)");
    if (!v->started) {
        dd_status st = start(v);
        if (st != DD_OK)
            return st;
        v->worker = std::thread(worker_main, v);
        v->completer = std::thread(completer_main, v);
    }
    int sidx = -1;
    for (int i = 0; i < (int)v->staging.size(); ++i)
        if (!v->staging_busy[i]) {
            sidx = i;
            break;
        }
    if (sidx < 0) {
        v->rejected++;
        return fail(DD_ERR_BUSY, "no staging buffer free (queue full); retry later");
    }
    v->staging_busy[sidx] = true;
    SrvReq r;
    r.beam = beam_id;
    r.k = b.next_submit++;
    r.staging = sidx;
    r.out_host = out_host;
    r.out_pitch = out_pitch;
    r.t_submit = Clock::now();
    const dd_ticket t = v->next_ticket++;
    // Copy the block into pinned staging (outside the lock: the buffer is ours).
    uint8_t *dst = static_cast<uint8_t *>(v->staging[sidx]);
    const int64_t nchan = b.plan->nchan, B = b.B, elem = v->elem;
    CopyPool *pool = v->pool;
    lk.unlock();
    const uint8_t *src = static_cast<const uint8_t *>(block_host);
    const auto c0 = Clock::now();
    if (pool) {
        std::lock_guard<std::mutex> plk(v->submit_mu);
        pool->copy_rows(dst, B * elem, src, in_pitch * elem, nchan, (size_t)(B * elem));
    } else {
        for (int64_t c = 0; c < nchan; ++c)
            std::memcpy(dst + c * B * elem, src + c * in_pitch * elem, (size_t)(B * elem));
    }
    const double copy_ms = std::chrono::duration<double, std::milli>(Clock::now() - c0).count();
    cudaError_t e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming);
    lk.lock();
    v->staged_bytes += nchan * B * elem;
    v->staged_ms += copy_ms;
    if (e != cudaSuccess) {
        v->staging_busy[sidx] = false;
        return fail(DD_ERR_CUDA, "event creation failed");
    }
    v->reqs[t] = r;
    v->queued.push_back(t);
    v->submitted++;
    *ticket = t;
    v->cv_work.notify_all();
    return DD_OK;
}

dd_status dd_poll(dd_server_t v, dd_ticket t, int64_t *first_t, int64_t *nsamp) {
    dd::Range nvtx_range("dd_poll");
    if (!v)
        return fail(DD_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(v->mu);
    auto it = v->reqs.find(t);
    if (it == v->reqs.end())
        return fail(DD_ERR_INVALID, "unknown or already collected ticket");
    SrvReq &r = it->second;
    const bool finished_in_flight = std::find(v->inflight.begin(), v->inflight.end(), t) ==
                                    v->inflight.end();
    if (r.state == kDone || (r.state == kFailed && finished_in_flight)) {
        if (first_t)
            *first_t = r.first_t;
        if (nsamp)
            *nsamp = r.nsamp;
        const dd_status st = r.state == kDone ? DD_OK : r.err;
        cudaEventDestroy(r.done);
        v->reqs.erase(it);
        return st;
    }
    return DD_PENDING;
}

dd_status dd_server_set_batch_window(dd_server_t v, int64_t microseconds) {
    if (!v || microseconds < 0 || microseconds > 10000000)
        return fail(DD_ERR_INVALID, "batch window must be 0..10 s");
    std::lock_guard<std::mutex> lk(v->mu);
    v->window_us = microseconds;
    v->window_set = true;
    return DD_OK;
}

dd_status dd_server_drain(dd_server_t v, int64_t timeout_ms) {
    if (!v)
        return fail(DD_ERR_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(v->mu);
    const bool ok = v->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&]() {
        return v->completed >= v->submitted;
    });
    return ok ? DD_OK : fail(DD_ERR_TIMEOUT, "blocks still in flight after the drain timeout");
}

dd_status dd_server_get_stats(dd_server_t v, dd_server_stats *s) {
    if (!v || !s)
        return fail(DD_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(v->mu);
    s->submitted = v->submitted;
    s->completed = v->completed;
    s->rejected_busy = v->rejected;
    s->batches = v->batches;
    s->p50_ms = percentile(v->lat_ms, 0.50);
    s->p99_ms = percentile(v->lat_ms, 0.99);
    s->max_ms = v->lat_ms.empty() ? 0.0 : *std::max_element(v->lat_ms.begin(), v->lat_ms.end());
    s->mean_batch = v->batches ? (double)v->batched_blocks / (double)v->batches : 0.0;
    s->slots = (int)v->slots.size();
    s->device_bytes = v->device_bytes;
    if (v->completed == v->submitted)  // nothing in flight: count the lanes' last batches
        for (auto &l : v->lanes)
            if (l.used && !l.accounted && cudaEventQuery(l.done) == cudaSuccess)
                account_lane(v, l);
    s->staging_bytes = v->staged_bytes;
    s->staging_ms = v->staged_ms;
    s->h2d_bytes = v->h2d_bytes;
    s->h2d_ms = v->h2d_ms;
    s->d2h_bytes = v->d2h_bytes;
    s->d2h_ms = v->d2h_ms;
    s->kernel_ms = v->kernel_ms;
    s->batch_window_us = v->window_us;
    return DD_OK;
}

dd_status dd_server_destroy(dd_server_t v) {
    if (!v)
        return DD_OK;
    dd_status st = DD_OK;
    if (v->started)
        st = dd_server_drain(v, 60000);
    {
        std::lock_guard<std::mutex> lk(v->mu);
        v->stop = true;
    }
    v->cv_work.notify_all();
    v->cv_done.notify_all();
    if (v->worker.joinable())
        v->worker.join();
    if (v->completer.joinable())
        v->completer.join();
    if (v->started) {
        cudaSetDevice(v->dev);
        cudaDeviceSynchronize();
    }
    for (auto &kv : v->reqs)
        if (kv.second.done)
            cudaEventDestroy(kv.second.done);
    free_all(v);
    delete v->pool;
    delete v;
    return st;
}

}  // extern "C"
