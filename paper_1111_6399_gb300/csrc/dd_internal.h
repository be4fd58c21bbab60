// Internal declarations shared by the host plan (dd_plan.cpp) and the CUDA
// translation units of libdd.  Not part of the public ABI (include/dd.h).
#pragma once

#include <cuda_runtime_api.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/dd.h"

namespace dd {

// NVTX range over one C-ABI call, named after it, for Nsight timelines (a
// no-op when no tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

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
// Builder warps (8/16-bit input) derive the byte phases 1.. of every staged
// row from phase 0 in shared memory; the producer records the bytes staged
// per row (kRowInfoBytes per stage: one word per row, at most 64 rows).
constexpr int kMaxBuilders = 2;
constexpr int kRowInfoBytes = 256;
// Consumer warps per CTA (plus one producer warp and, for 8/16-bit input, the
// builder warps), from the registers a thread needs: accumulators 2*DT*NW
// (uint8) + two load buffers 4*NW + ~24.  A CTA of at most 16 warps leaves
// 128 registers a thread (at most 4 warps per SM sub-partition), at most 20
// leave 96, at most 24 leave 80, at most 28 leave 72.
#ifdef __CUDACC__
#define DD_HD __host__ __device__
#else
#define DD_HD
#endif
DD_HD constexpr int max_consumer_warps(int dm_per_thread, int words) {
    return words >= 8 ? (dm_per_thread >= 4 ? 13 : dm_per_thread == 2 ? 16 : 20)
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
    int *det_cnt = nullptr;      // tile-boundary counters of fused detection
    int64_t det_cnt_n = 0;
};

// Accumulators of a boxcar search (dd_detect, dd_execute_detect): caller-owned
// output arrays, used as exact sums and keys until the finalize step.
struct DetectTargets {
    int nlevels = 0;
    double *mean = nullptr, *sd = nullptr, *snr = nullptr;
    int64_t *tpk = nullptr;
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
    int builders = 0;     // phase-builder warps (0 for FP32)
    int threads = 0;      // consumer warps + one producer warp + builder warps
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
    // Remainder-DM launch per (dtype, tiles) key: (found, geometry).
    std::map<uint64_t, std::pair<bool, dd::Geometry>> tail_geo;
};

namespace dd {

// Thread-local error message; returns st for chaining.
dd_status fail(dd_status st, const std::string &msg);

// Dynamic shared memory of a ring of n stages of stage_bytes each for a
// geometry: the stages, the offset table, the stage records, the per-row
// byte counts (with phases to build), the zero row and three mbarriers per
// stage, in the order the kernel lays them out, and 16 bytes for the
// epilogue of fused detection.
int64_t ring_smem(const Geometry &g, int64_t stage_bytes, int n);

// Host checks of a beam's layout shared by the entry points that run one
// beam: dtype, sample counts (nsamp_in >= nsamp_out + maxshift), pitches at
// least a row and, for device rows (device_rows), multiples of 16 bytes.
dd_status check_layout(dd_plan_s *p, dd_dtype dtype, int64_t in_pitch, int64_t nsamp_in,
                       int64_t out_pitch, int64_t nsamp_out, bool device_rows);

// Device address of the status word of dd_execute_noalloc's fixed array on
// the current device (looked up once per device; see dd_noalloc.cu).
dd_status noalloc_status_word(int **out);

// Preferred tile shape for a dtype.
dd_tiles default_tiles(dd_dtype t);

// Tile shapes tried, in order, when the plan picks one itself: the preferred
// shape, then fewer channels per stage, then fewer DMs per CTA (more time
// warps), down to one DM per CTA, which always fits.
std::vector<dd_tiles> auto_tiles(dd_dtype t);

// Validate a tile shape for dtype and compute the launch geometry for the
// plan (shared-memory window bound over every DM tile and channel).
dd_status make_geometry(dd_plan_s *p, dd_dtype t, const dd_tiles &tl, Geometry *g);

// The same for the sorted DMs [d0, d0 + nd) only.
dd_status make_geometry_range(dd_plan_s *p, dd_dtype t, const dd_tiles &tl, int d0, int nd,
                              Geometry *g);

// Geometry for the plan's current tile shape, cached.
dd_status plan_geometry(dd_plan_s *p, dd_dtype t, Geometry *g);

// Launch shape for the DMs of the last, partly filled DM tile of geometry g,
// run as a launch of their own (see dd_plan.cpp); cached per tile shape.
dd_status tail_geometry(dd_plan_s *p, dd_dtype t, const Geometry &g, bool *found,
                        Geometry *tail);

// Device tables for the current device, uploaded on first use.
dd_status device_tables(dd_plan_s *p, DevTables **out);

// Launch the de-dispersion kernel (dd_kernel_*.cu) for one beam on stream.
// With split_tail, the DMs of a last DM tile that is at most half full run
// as a second launch with their own tile shape, on a library stream forked
// from and joined back into `stream`, so its CTAs fill the SMs the first
// launch leaves idle in its last wave instead of padding a whole DM tile --
// when a count of the two launches' waves says that finishes earlier.
dd_status launch_dedisperse(dd_plan_s *p, const Geometry &g, const DevTables &dt,
                            const void *in, dd_dtype dtype, int64_t in_pitch, int64_t nsamp_in,
                            float *out, int64_t out_pitch, int64_t nsamp_out, void *stream,
                            bool split_tail = true);

void count_launch(int n = 1);

// Boxcar search accumulators: clear them (dd_detect.cu), and turn them into
// mean, std, S/N and peak t for an integer-valued plane.
dd_status detect_begin(int ndm, int nlevels, double *mean, double *sd, double *snr,
                       cudaStream_t s);
dd_status detect_finalize_int(int ndm, int64_t nsamp, int nlevels, double *mean, double *sd,
                              double *snr, int64_t *tpk, cudaStream_t s);

// One uint8 de-dispersion launch (no remainder split) with the boxcar search
// fused into its epilogue (dd_launch.cpp): g must have 4 DMs x 8 words per
// thread and one time warp (1024-sample tiles); det_cnt holds
// g.ntile_d * ntile_t zeroed ints.
dd_status launch_dedisperse_detect(dd_plan_s *p, const Geometry &g, const DevTables &dt,
                                   const void *in, int64_t in_pitch, int64_t nsamp_in,
                                   float *out, int64_t out_pitch, int64_t nsamp_out,
                                   const DetectTargets &det, int *det_cnt, void *stream);

}  // namespace dd
