// Host plan of the de-dispersion library: the per-channel FP32 delay table,
// the trial-DM grid, maxshift, tile shapes and their shared-memory geometry.
//
// Sec. 2 of the paper: the cold-plasma law makes the arrival delay grow as
// f^-2 with one free parameter, the DM; a blind search shifts every channel by
// its delay for each trial DM.  The table below is that delay for DM = 1 in
// samples, relative to the highest channel centre, evaluated in FP64 and
// rounded once to FP32.  This file must be compiled with -ffp-contract=off:
// a fused multiply-add in the channel-frequency or delay expression changes
// the rounding of the FP32 table.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <new>

#include "dd_internal.h"

namespace {

thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};

constexpr double kDispersionConst = 4148.808;  // s MHz^2 / (pc cm^-3)

int trunc_product(float dm, float ds) {
    volatile float prod = dm * ds;  // one FP32 multiply, round to nearest even
    return (int)prod;
}

uint64_t geo_key(dd_dtype t, const dd_tiles &tl) {
    return ((uint64_t)t << 60) | ((uint64_t)tl.words_per_thread << 48) |
           ((uint64_t)tl.dm_per_thread << 36) | ((uint64_t)tl.dm_warps << 24) |
           ((uint64_t)tl.time_warps << 12) | (uint64_t)tl.chan_per_stage;
}

bool valid_dtype(dd_dtype t) { return t == DD_U8 || t == DD_F16 || t == DD_F32; }

}  // namespace

namespace dd {

dd_status fail(dd_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

dd_tiles default_tiles(dd_dtype t) {
    switch (t) {
    case DD_U8:  return dd_tiles{4, 12, 1, 8, 8};
    case DD_F16: return dd_tiles{1, 12, 1, 16, 8};
    default:     return dd_tiles{2, 12, 1, 16, 8};
    }
}

std::vector<dd_tiles> auto_tiles(dd_dtype t) {
    const dd_tiles base = default_tiles(t);
    const int max_t_cta = 4096;  // samples per CTA along time
    std::vector<dd_tiles> out;
    for (int dcta = base.dm_per_thread * base.dm_warps; dcta >= 1; dcta /= 2) {
        const int dthr = std::min(base.dm_per_thread, dcta);
        const int wd = dcta / dthr;
        const int nw = base.words_per_thread;
        const int wt = std::max(1, std::min(max_consumer_warps(dthr, nw) / wd,
                                            max_t_cta / warp_span(t, nw)));
        for (int cs = base.chan_per_stage; cs >= 4; cs /= 2)
            out.push_back(dd_tiles{dthr, wd, wt, cs, nw});
    }
    return out;
}

int64_t ring_smem(const Geometry &g, int64_t stage_bytes, int n) {
    const int64_t table = ((int64_t)n * g.tiles.chan_per_stage * g.dm_cta * 4 + 15) / 16 * 16;
    const int64_t rowinfo = g.nph > 1 ? kRowInfoBytes : 0;
    // + 16: the epilogue barrier and flags of fused detection
    return n * stage_bytes + table + n * (kStageMeta + rowinfo) + g.zero_bytes + 24 * (int64_t)n +
           16;
}

dd_status make_geometry(dd_plan_s *p, dd_dtype t, const dd_tiles &tl, Geometry *g) {
    return make_geometry_range(p, t, tl, 0, p->ndm, g);
}

dd_status make_geometry_range(dd_plan_s *p, dd_dtype t, const dd_tiles &tl, int d0, int nd,
                              Geometry *g) {
    if (d0 < 0 || nd < 1 || d0 + nd > p->ndm)
        return fail(DD_ERR_INVALID, "DM range outside the plan");
    if (!valid_dtype(t))
        return fail(DD_ERR_INVALID, "unknown dtype");
    const int dthr = tl.dm_per_thread;
    const int nw = tl.words_per_thread;
    bool ok_dthr = dthr == 1 || dthr == 2 || dthr == 4;
    if (!ok_dthr || (nw != 4 && nw != 8))
        return fail(DD_ERR_INVALID, "tile shape: dm_per_thread must be 1, 2 or 4 and "
                                    "words_per_thread 4 or 8");
    if (tl.dm_warps < 1 || tl.time_warps < 1 ||
        tl.dm_warps * tl.time_warps > max_consumer_warps(dthr, nw))
        return fail(DD_ERR_INVALID, "tile shape: dm_warps*time_warps must be 1.." +
                                        std::to_string(max_consumer_warps(dthr, nw)) +
                                        " for this dm_per_thread and words_per_thread");
    if (tl.chan_per_stage < 4 || tl.chan_per_stage > 64 || (tl.chan_per_stage & 3))
        return fail(DD_ERR_INVALID, "tile shape: chan_per_stage must be a multiple of 4, 4..64");
    const int limit = (t == DD_U8) ? kSwarChannels : kFloatBlock;
    if (tl.chan_per_stage > limit)
        return fail(DD_ERR_INVALID, "tile shape: chan_per_stage must not exceed the "
                                    "accumulation block (256 for uint8, 64 otherwise)");
    // The producer warp writes the offset table for DM columns lane and
    // lane + 32, and the device DM list is padded by 64 entries: at most 64
    // DMs per CTA.
    if (dthr * tl.dm_warps > kMaxDmPerCta)
        return fail(DD_ERR_INVALID, "tile shape: dm_per_thread*dm_warps must be <= 64");
    Geometry r;
    r.tiles = tl;
    r.elem = elem_size(t);
    r.nph = phases(t);
    r.span = warp_span(t, nw);
    r.dm_cta = dthr * tl.dm_warps;
    r.t_cta = r.span * tl.time_warps;
    r.threads = 32 * tl.dm_warps * tl.time_warps;
    r.ntile_d = (nd + r.dm_cta - 1) / r.dm_cta;
    // Widest staged window (bytes) over every DM tile and channel: the CTA at
    // t0 reads samples [t0 + s(c,dm_min), t0 + t_cta + s(c,dm_max)) of channel
    // c, fetched from a 16-byte aligned start.
    int64_t widest = 0;
    for (int td = 0; td < r.ntile_d; ++td) {
        float dmin = p->dm_sorted[(size_t)d0 + (size_t)td * r.dm_cta];
        float dmax = p->dm_sorted[(size_t)d0 +
                                  std::min((size_t)(td + 1) * r.dm_cta, (size_t)nd) - 1];
        for (int c = 0; c < p->nchan; ++c) {
            int64_t smin = trunc_product(dmin, p->dmshift[c]);
            int64_t smax = trunc_product(dmax, p->dmshift[c]);
            int64_t start = (r.elem * smin) & ~(int64_t)15;
            int64_t end = (int64_t)r.elem * (r.t_cta + smax);
            int64_t w = (end - start + 15) & ~(int64_t)15;
            widest = std::max(widest, w);
        }
    }
    const int64_t wp = widest + 16;
    const int64_t zero_bytes = ((int64_t)r.elem * r.t_cta + 16 + 15) / 16 * 16;
    // Per stage: the staged rows (every byte phase), the producer's offset
    // table (one int per staged row and DM of the CTA), a stage record and,
    // with phases to build, the bytes staged per row; then the zero row and
    // three mbarriers per stage.
    const int64_t stage_bytes = (int64_t)tl.chan_per_stage * r.nph * wp;
    r.zero_bytes = (int)zero_bytes;
    auto smem_for = [&](int64_t n) { return ring_smem(r, stage_bytes, (int)n); };
    int nst = 4;
    while (nst > 2 && smem_for(nst) > kMaxSmem)
        --nst;
    const int64_t smem = smem_for(nst);
    if (smem > kMaxSmem)
        return fail(DD_ERR_INVALID, "tile shape: staged window needs " + std::to_string(smem) +
                                        " bytes of shared memory (limit 232448); use fewer "
                                        "channels per stage or fewer DMs per CTA");
    r.wp = (int)wp;
    r.stage_bytes = (int)stage_bytes;
    r.nstages = nst;
    r.zero_bytes = (int)zero_bytes;
    r.smem = (int)smem;
    // Two builder warps: with one, building a stage (about 3 shared-memory
    // ops per staged byte, queued behind the consumers' loads) can take
    // longer than consuming it.
    r.builders = r.nph > 1 ? kMaxBuilders : 0;
    r.threads += 32 * (1 + r.builders);  // producer warp, builder warps
    *g = r;
    return DD_OK;
}

dd_status plan_geometry(dd_plan_s *p, dd_dtype t, Geometry *g) {
    if (!valid_dtype(t))
        return fail(DD_ERR_INVALID, "unknown dtype");
    std::lock_guard<std::mutex> lk(p->mu);
    uint64_t key = geo_key(t, p->tiles[t]);
    auto it = p->geo.find(key);
    if (it != p->geo.end()) {
        *g = it->second;
        return DD_OK;
    }
    Geometry r;
    dd_status st = DD_ERR_INVALID;
    if (p->tiles_auto[t]) {
        for (const dd_tiles &cand : auto_tiles(t)) {
            if ((st = make_geometry(p, t, cand, &r)) == DD_OK) {
                p->tiles[t] = cand;
                break;
            }
        }
        p->tiles_auto[t] = false;
        key = geo_key(t, p->tiles[t]);
    } else {
        st = make_geometry(p, t, p->tiles[t], &r);
    }
    if (st != DD_OK)
        return st;
    p->geo[key] = r;
    *g = r;
    return DD_OK;
}

// The DMs of the last, partly filled DM tile as a launch of their own: a tile
// shape with the same per-thread layout (dm_per_thread, words_per_thread) and
// as many consumer warps, so a tile holds about the same work, but as few DM
// columns as cover the remainder and correspondingly more time.  Used when
// the remainder fills at most half a DM tile (padding it would waste at least
// half of that tile's work); found[0] = false when no such shape fits.
dd_status tail_geometry(dd_plan_s *p, dd_dtype t, const Geometry &g, bool *found,
                        Geometry *tail) {
    *found = false;
    const int rem = p->ndm % g.dm_cta;
    if (rem == 0 || 2 * rem > g.dm_cta || p->ndm < g.dm_cta)
        return DD_OK;
    std::lock_guard<std::mutex> lk(p->mu);
    const uint64_t key = geo_key(t, g.tiles);
    auto it = p->tail_geo.find(key);
    if (it != p->tail_geo.end()) {
        *found = it->second.first;
        *tail = it->second.second;
        return DD_OK;
    }
    const int dthr = g.tiles.dm_per_thread, nw = g.tiles.words_per_thread;
    const int dmw = (rem + dthr - 1) / dthr;
    const int warps = g.tiles.dm_warps * g.tiles.time_warps;
    Geometry best;
    bool have = false;
    // Most time warps first; among shapes that fit, the first with three or
    // more ring stages, else the first that fits at all.
    for (int tw = warps / dmw; tw >= 1 && !(have && best.nstages >= 3); --tw) {
        for (int cs = g.tiles.chan_per_stage; cs >= 4; cs = (cs / 2) & ~3) {
            dd_tiles tl{dthr, dmw, tw, cs, nw};
            Geometry r;
            if (make_geometry_range(p, t, tl, p->ndm - rem, rem, &r) != DD_OK)
                continue;
            if (!have || (best.nstages < 3 && r.nstages >= 3)) {
                best = r;
                have = true;
            }
            if (r.nstages >= 3)
                break;
        }
    }
    p->tail_geo[key] = std::make_pair(have, best);
    *found = have;
    if (have)
        *tail = best;
    return DD_OK;
}

dd_status device_tables(dd_plan_s *p, DevTables **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return fail(DD_ERR_CUDA, "cudaGetDevice failed (no CUDA device?)");
    std::lock_guard<std::mutex> lk(p->mu);
    auto it = p->dev.find(dev);
    if (it != p->dev.end()) {
        *out = &it->second;
        return DD_OK;
    }
    // Pad the sorted DM list to a multiple of 64 (the largest DM tile) with
    // its last value; padding rows are never stored.
    DevTables t;
    t.ndm_pad = (p->ndm + 63) / 64 * 64 + 64;  // covers ceil(ndm/dm_cta)*dm_cta for any dm_cta <= 64
    std::vector<float> dms(t.ndm_pad, p->dm_sorted.back());
    std::vector<int> perm(t.ndm_pad, -1);
    for (int k = 0; k < p->ndm; ++k) {
        dms[k] = p->dm_sorted[k];
        perm[k] = p->order[k];
    }
    bool ok = cudaMalloc((void **)&t.dmshift, sizeof(float) * p->nchan) == cudaSuccess &&
              cudaMalloc((void **)&t.dm_sorted, sizeof(float) * t.ndm_pad) == cudaSuccess &&
              cudaMalloc((void **)&t.perm, sizeof(int) * t.ndm_pad) == cudaSuccess &&
              cudaMalloc((void **)&t.status, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMemcpy(t.dmshift, p->dmshift.data(), sizeof(float) * p->nchan,
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(t.dm_sorted, dms.data(), sizeof(float) * t.ndm_pad,
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(t.perm, perm.data(), sizeof(int) * t.ndm_pad,
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemset(t.status, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaFree(t.dmshift);
        cudaFree(t.dm_sorted);
        cudaFree(t.perm);
        cudaFree(t.status);
        cudaGetLastError();
        return fail(DD_ERR_NOMEM, "device table upload failed");
    }
    auto res = p->dev.emplace(dev, t);
    *out = &res.first->second;
    return DD_OK;
}

}  // namespace dd

extern "C" {

const char *dd_last_error(void) { return g_last_error.c_str(); }

int64_t dd_launch_count(void) { return g_launches.load(); }

dd_status dd_plan(int nchan, double fch1_mhz, double foff_mhz, double tsamp_s,
                  const float *dm_list, int ndm, dd_plan_t *plan_out) {
    dd::Range nvtx_range("dd_plan");
    using dd::fail;
    if (!plan_out)
        return fail(DD_ERR_INVALID, "plan_out is NULL");
    *plan_out = nullptr;
    if (nchan < 1 || ndm < 1 || !dm_list)
        return fail(DD_ERR_INVALID, "need nchan >= 1, ndm >= 1 and a DM list");
    if (!(tsamp_s > 0.0) || !std::isfinite(tsamp_s))
        return fail(DD_ERR_INVALID, "tsamp must be a positive number of seconds");
    if (foff_mhz == 0.0 || !std::isfinite(foff_mhz) || !std::isfinite(fch1_mhz))
        return fail(DD_ERR_INVALID, "foff must be non-zero and finite");
    const double ftop = foff_mhz < 0.0 ? fch1_mhz : fch1_mhz + (double)(nchan - 1) * foff_mhz;
    const double fbot = foff_mhz < 0.0 ? fch1_mhz + (double)(nchan - 1) * foff_mhz : fch1_mhz;
    if (!(fbot > 0.0))
        return fail(DD_ERR_INVALID, "every channel centre frequency must be > 0 MHz");
    for (int d = 0; d < ndm; ++d)
        if (!std::isfinite(dm_list[d]) || dm_list[d] < 0.0f)
            return fail(DD_ERR_INVALID, "trial DMs must be finite and >= 0");

    dd_plan_s *p = new (std::nothrow) dd_plan_s;
    if (!p)
        return fail(DD_ERR_NOMEM, "out of host memory");
    p->nchan = nchan;
    p->ndm = ndm;
    p->fch1 = fch1_mhz;
    p->foff = foff_mhz;
    p->tsamp = tsamp_s;
    p->dmshift.resize(nchan);
    const double inv_top2 = 1.0 / (ftop * ftop);
    for (int c = 0; c < nchan; ++c) {
        const double f = fch1_mhz + (double)c * foff_mhz;
        const double inv_f2 = 1.0 / (f * f);
        p->dmshift[c] = (float)(kDispersionConst * (inv_f2 - inv_top2) / tsamp_s);
    }
    p->dm.assign(dm_list, dm_list + ndm);
    p->order.resize(ndm);
    std::iota(p->order.begin(), p->order.end(), 0);
    std::stable_sort(p->order.begin(), p->order.end(),
                     [&](int a, int b) { return p->dm[a] < p->dm[b]; });
    p->dm_sorted.resize(ndm);
    for (int k = 0; k < ndm; ++k)
        p->dm_sorted[k] = p->dm[p->order[k]];
    // The shift is monotone in DM and in dmshift, so its maximum over the grid
    // is reached at the largest DM; the scan over channels keeps it exact even
    // if the table were not monotone.
    int64_t s = 0;
    for (int c = 0; c < nchan; ++c)
        s = std::max<int64_t>(s, trunc_product(p->dm_sorted.back(), p->dmshift[c]));
    p->maxshift = s;
    for (int t = 0; t < 3; ++t)
        p->tiles[t] = dd::default_tiles((dd_dtype)t);
    *plan_out = p;
    return DD_OK;
}

void dd_plan_destroy(dd_plan_t p) {
    if (!p)
        return;
    int cur = -1;
    cudaGetDevice(&cur);
    for (auto &kv : p->dev) {
        cudaSetDevice(kv.first);
        cudaFree(kv.second.dmshift);
        cudaFree(kv.second.dm_sorted);
        cudaFree(kv.second.perm);
        cudaFree(kv.second.status);
        cudaFree(kv.second.det_cnt);
    }
    if (cur >= 0 && !p->dev.empty())
        cudaSetDevice(cur);
    delete p;
}

int64_t dd_plan_maxshift(dd_plan_t p) { return p ? p->maxshift : -1; }
int dd_plan_nchan(dd_plan_t p) { return p ? p->nchan : -1; }
int dd_plan_ndm(dd_plan_t p) { return p ? p->ndm : -1; }

dd_status dd_plan_dmshift(dd_plan_t p, float *host_out) {
    if (!p || !host_out)
        return dd::fail(DD_ERR_INVALID, "NULL argument");
    std::memcpy(host_out, p->dmshift.data(), sizeof(float) * p->nchan);
    return DD_OK;
}

dd_status dd_plan_get_tiles(dd_plan_t p, dd_dtype t, dd_tiles *out) {
    if (!p || !out || !valid_dtype(t))
        return dd::fail(DD_ERR_INVALID, "NULL argument or unknown dtype");
    dd::Geometry g;
    dd_status st = dd::plan_geometry(p, t, &g);  // resolves an automatic choice
    if (st != DD_OK)
        return st;
    std::lock_guard<std::mutex> lk(p->mu);
    *out = p->tiles[t];
    return DD_OK;
}

dd_status dd_plan_set_tiles(dd_plan_t p, dd_dtype t, const dd_tiles *tl) {
    if (!p || !tl || !valid_dtype(t))
        return dd::fail(DD_ERR_INVALID, "NULL argument or unknown dtype");
    dd::Geometry g;
    dd_status st = dd::make_geometry(p, t, *tl, &g);
    if (st != DD_OK)
        return st;
    std::lock_guard<std::mutex> lk(p->mu);
    p->tiles[t] = *tl;
    p->tiles_auto[t] = false;
    return DD_OK;
}

}  // extern "C"
