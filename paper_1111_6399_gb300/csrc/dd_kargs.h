// Kernel arguments of the de-dispersion kernel and the per-element-size
// launchers (one translation unit each: dd_kernel_u8.cu, _f16.cu, _f32.cu).
#pragma once

#include <cuda_runtime_api.h>

#include <cstdint>

namespace dd {

// One beam: its buffers, plan tables and launch geometry.
struct BeamArgs {
    const uint8_t *in;
    int64_t in_pitch_b;     // bytes between channel rows
    int64_t nsamp_in;       // valid samples per row
    float *out;
    int64_t out_pitch;      // floats between DM rows
    int64_t nsamp_out;
    const float *dmshift;   // [nchan]
    const float *dm_sorted; // [ndm padded by >= 64]
    const int *perm;        // sorted DM -> output row, -1 for padding
    int64_t tile_begin;     // first global tile of this beam
    int nchan;
    int ntile_d;            // DM tiles of this beam
    int wp;                 // bytes per phase row in shared memory
    int pad;
};

// One launch: a single beam (beam0, beams == NULL, one tile per CTA) or a
// batch (beams[], tiles claimed dynamically through tile_counter).
struct KArgs {
    BeamArgs beam0;
    const BeamArgs *beams;
    int nbeams;
    int64_t total_tiles;
    int *tile_counter;      // zeroed before the launch; NULL: tile = blockIdx.x
    int dm_warps;
    int time_warps;
    int cstage;             // channels per ring stage
    int nstages;            // stages in the ring
    int stage_bytes;        // capacity of one ring stage
    int zero_bytes;         // bytes of the zero row (padding channels)
    uint32_t one;           // the constant 1, opaque to the compiler
    int builders;           // phase-builder warps (8/16-bit input; 0 for FP32)
    int *status;
    // Detection fused into the epilogue (uint8 single-beam launches with
    // 1024-sample time tiles; det_s1 == NULL: off): per output row the exact
    // sums S1, S2 and per (row, level) the packed boxcar keys, as dd_detect
    // accumulates them; det_cnt: one counter per (DM tile, time tile),
    // zeroed before the launch, deciding which tile of a neighbouring pair
    // searches the boxcar starts across their boundary.
    unsigned long long *det_s1, *det_s2, *det_keys;
    int *det_cnt;
    int det_nlevels;
    int det_ntile_t;
};

// Launch dedisperse_kernel<elem, dthr, nw> with `threads` threads per CTA.
cudaError_t launch_kernel_u8(const KArgs &a, unsigned grid, int threads, int smem,
                             cudaStream_t s, int dthr, int nw);
cudaError_t launch_kernel_f16(const KArgs &a, unsigned grid, int threads, int smem,
                              cudaStream_t s, int dthr, int nw);
cudaError_t launch_kernel_f32(const KArgs &a, unsigned grid, int threads, int smem,
                              cudaStream_t s, int dthr, int nw);

// Shared-memory bytes of the per-stage metadata record.
constexpr int kStageMetaBytes = 32;

}  // namespace dd
