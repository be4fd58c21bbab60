// Internal declarations shared by the host plan (dd_plan.cpp) and the CUDA
// translation units of libdd.  Not part of the public ABI (include/dd.h).
#pragma once

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dd.h"

namespace dd {

// Samples covered by one warp along time: 32 lanes x `words` 4-byte words x
// (4 / element size) samples per word.
inline int elem_size(dd_dtype t) { return t == DD_U8 ? 1 : (t == DD_F16 ? 2 : 4); }
inline int warp_span(dd_dtype t, int words) { return 32 * words * (4 / elem_size(t)); }
inline int phases(dd_dtype t) { return 4 / elem_size(t); }

// Channels summed into 16-bit SWAR lanes before they are widened (uint8):
// 256 * 255 = 65280 fits a 16-bit lane.
constexpr int kSwarChannels = 256;
// Channels per compensated block for FP16/FP32 input.
constexpr int kFloatBlock = 64;

constexpr int kMaxSmem = 232448;  // 227 KB dynamic shared memory per CTA
constexpr int kMaxDmPerCta = 64;   // DMs per CTA (offset-table columns, DM padding)
constexpr int kStageMeta = 32;     // bytes of a stage record in shared memory
// Consumer warps per CTA (plus one producer warp), from the registers a
// thread needs: accumulators 2*DT*NW (uint8) + two load buffers 4*NW + ~24.
// 13 warps leave 128 registers a thread (at most 4 warps per SM
// sub-partition), 17 leave 96, 21 leave 85, 25 leave 73.
#ifdef __CUDACC__
#define DD_HD __host__ __device__
#else
#define DD_HD
#endif
DD_HD constexpr int max_consumer_warps(int dm_per_thread, int words) {
    return words >= 8 ? (dm_per_thread >= 4 ? 12 : dm_per_thread == 2 ? 16 : 20)
                      : (dm_per_thread >= 4 ? 20 : 24);
}

// Device status word values (written by kernels, read by dd_sync).
constexpr int kDevOk = 0;
constexpr int kDevTimeout = 1;
constexpr int kDevCheck = 2;

struct DevTables {
    float *dmshift = nullptr;    // [nchan]
    float *dm_sorted = nullptr;  // [ndm_pad]: DMs in ascending order, padded with the last
    int *perm = nullptr;         // [ndm_pad]: output row of sorted DM k, -1 for padding
    int *status = nullptr;       // device status word
    int ndm_pad = 0;
    // Phase-plane scratch of dd_execute (grown on demand).  Uses on different
    // streams are ordered by scratch_done: each use waits for the previous one.
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    void *scratch_done = nullptr;  // cudaEvent_t
};

// Launch geometry derived from a tile shape and the plan's tables.
struct Geometry {
    dd_tiles tiles{};
    int elem = 1, nph = 1, span = 0;
    int dm_cta = 0;       // DMs per CTA
    int t_cta = 0;        // samples per CTA
    int ntile_d = 0;      // DM tiles
    int wp = 0;           // bytes of one phase row in shared memory
    int stage_bytes = 0;  // bytes of one ring stage (chan_per_stage rows, every phase)
    int nstages = 0;      // shared-memory stages in the copy ring
    int zero_bytes = 0;   // zero row read by padding channels
    int smem = 0;         // dynamic shared memory per CTA
    int threads = 0;      // consumer warps + one producer warp
};

}  // namespace dd

struct dd_plan_s {
    int nchan = 0, ndm = 0;
    double fch1 = 0, foff = 0, tsamp = 0;
    int64_t maxshift = 0;
    std::vector<float> dmshift;    // [nchan] FP32 table
    std::vector<float> dm;         // [ndm] caller order
    std::vector<int> order;        // sorted position -> caller index
    std::vector<float> dm_sorted;  // [ndm] ascending
    dd_tiles tiles[3]{};
    bool tiles_auto[3] = {true, true, true};  // resolved by the plan until set
    std::mutex mu;
    std::map<int, dd::DevTables> dev;      // per CUDA device
    std::map<uint64_t, dd::Geometry> geo;  // per (dtype, tiles) key
};

namespace dd {

// Thread-local error message; returns st for chaining.
dd_status fail(dd_status st, const std::string &msg);

// Preferred tile shape for a dtype.
dd_tiles default_tiles(dd_dtype t);

// Tile shapes tried, in order, when the plan picks one itself: the preferred
// shape, then fewer channels per stage, then fewer DMs per CTA (more time
// warps), down to one DM per CTA, which always fits.
std::vector<dd_tiles> auto_tiles(dd_dtype t);

// Validate a tile shape for dtype and compute the launch geometry for the
// plan (shared-memory window bound over every DM tile and channel).
dd_status make_geometry(dd_plan_s *p, dd_dtype t, const dd_tiles &tl, Geometry *g);

// Geometry for the plan's current tile shape, cached.
dd_status plan_geometry(dd_plan_s *p, dd_dtype t, Geometry *g);

// Device tables for the current device, uploaded on first use.
dd_status device_tables(dd_plan_s *p, DevTables **out);

// Bytes of phase-plane scratch for one input (0 for FP32).
int64_t scratch_bytes(dd_dtype dtype, int nchan, int64_t in_pitch_b);

// Launch the phase-plane pre-pass (8/16-bit input) and the de-dispersion
// kernel (dd_kernel.cu) on stream, with caller-provided scratch.
dd_status launch_dedisperse(dd_plan_s *p, const Geometry &g, const DevTables &dt,
                            const void *in, dd_dtype dtype, int64_t in_pitch, int64_t nsamp_in,
                            float *out, int64_t out_pitch, int64_t nsamp_out, void *scratch,
                            void *stream);

// launch_dedisperse with the plan's own per-device scratch (dd_exec.cpp).
dd_status run_with_plan_scratch(dd_plan_s *p, const Geometry &g, DevTables &dt, const void *in,
                                dd_dtype dtype, int64_t in_pitch, int64_t nsamp_in, float *out,
                                int64_t out_pitch, int64_t nsamp_out, void *stream);

void count_launch(int n = 1);

}  // namespace dd
