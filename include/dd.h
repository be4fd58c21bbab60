/*
 * dd.h -- C ABI of the GB300 brute-force incoherent de-dispersion library
 * (libdd.so, built for sm_103a).
 *
 * The operation (ARTEMIS paper, Sec. 2): for every trial dispersion measure
 * d and output sample t,
 *
 *     out[d][t] = sum_{c=0}^{nchan-1} in[c][t + s(c,d)]
 *
 * where each frequency channel of the (f,t) power array is shifted by its
 * cold-plasma dispersion delay before the frequency integration.  The shift
 * rule: dmshift[c] = float(4148.808 * (f_c^-2 - f_top^-2) / tsamp), evaluated
 * in FP64 on the host with f in MHz and tsamp in seconds, rounded once to
 * FP32; s(c,d) = (int)(float(dm[d]) * dmshift[c]) with one FP32 multiply
 * (round to nearest even) and truncation.  f_c = fch1 + c * foff is the
 * centre frequency of channel c and f_top the highest channel centre.
 * Sec. 3 of the paper sets the design rules this library follows on GB300:
 * accumulators in the fastest memory (registers), the (f,t) data staged
 * close to the SMs (shared memory, filled by the TMA), and as little shift
 * arithmetic as possible.
 *
 * Layouts (Sec. 3, Fig. 2: rows of constant frequency, contiguous time):
 *   in  : nchan rows, row c at in + c * in_pitch elements; channel 0 is fch1.
 *         Each row holds at least nsamp_out + maxshift samples.
 *   out : FP32, ndm rows, row d at out + d * out_pitch floats, in the order of
 *         the caller's DM list.  Sample t is the arrival time at f_top.
 * Alignment: in and out 16-byte aligned; in_pitch * element size and
 * out_pitch * 4 multiples of 16 bytes.
 *
 * Accuracy: uint8 input is summed exactly (bit-identical to any exact sum);
 * FP16/FP32 input is summed in FP32 with compensated block accumulation,
 * within 1e-6 * sum_c |in[c][t+s(c,d)]| of the exact sum.
 *
 * Errors: every call returns a dd_status; a negative status leaves no side
 * effect on caller memory, and dd_last_error() gives a message (per thread).
 * Device-side waits are bounded: a wait that runs out records DD_ERR_TIMEOUT
 * in the plan's device status word, which dd_sync() reports.
 *
 * Ownership: the library owns plans, batches and servers (and the device
 * tables inside them); the caller owns every in/out buffer it passes, which
 * must stay valid until the work on the given stream has completed.
 * Streams are passed as void* (a cudaStream_t; NULL is the legacy default
 * stream).  Plans are immutable after creation and may be used from several
 * threads and streams at once; a plan's device tables are uploaded lazily,
 * per device, on its first execution there.
 */
#ifndef DD_H
#define DD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dd_status {
    DD_OK = 0,
    DD_PENDING = 1,         /* dd_poll: the block is still in flight          */
    DD_ERR_INVALID = -1,    /* bad argument, detected before any launch        */
    DD_ERR_CUDA = -2,       /* a CUDA runtime call failed                      */
    DD_ERR_NOMEM = -3,      /* device or pinned-host allocation failed         */
    DD_ERR_BUSY = -4,       /* dd_submit: no slot or HBM budget free right now */
    DD_ERR_TIMEOUT = -5,    /* a bounded device wait ran out                   */
    DD_ERR_DEVICE = -6      /* the kernel recorded an internal check failure   */
} dd_status;

typedef enum dd_dtype { DD_U8 = 0, DD_F16 = 1, DD_F32 = 2 } dd_dtype;

typedef struct dd_plan_s *dd_plan_t;

/* Tile shape of the de-dispersion kernel (chosen by the plan or the autotuner).
 *   dm_per_thread    trial DMs each thread accumulates (register accumulators)
 *   dm_warps         warps of a CTA along the DM axis
 *   time_warps       warps of a CTA along the time axis
 *   chan_per_stage   channels staged in shared memory per pipeline stage
 *                    (a multiple of 4, 4..64)
 *   words_per_thread 4-byte words of output time per DM and thread: 4 or 8
 * A CTA covers dm_per_thread*dm_warps DMs and time_warps*span samples, where
 * span = 32*words_per_thread*(4/element size) samples per warp (1024 for
 * uint8 with 8 words).  Warp limits (dm_warps*time_warps) by register need:
 * 12 for 4 DMs x 8 words, 16 for 2x8, 20 for 1x8 and 4x4, 24 for 2x4 and 1x4;
 * the CTA has one more warp that stages the data.  At most 64 DMs per CTA
 * (dm_per_thread*dm_warps <= 64). */
typedef struct dd_tiles {
    int dm_per_thread;
    int dm_warps;
    int time_warps;
    int chan_per_stage;
    int words_per_thread;
} dd_tiles;

/* --- plan (Sec. 2: the dispersion law and the trial-DM grid) ------------- */

/* Build a plan: the FP64->FP32 dmshift table, the caller's FP32 DM list and
 * maxshift = max_{c,d} s(c,d).  Host-only; no GPU is touched.
 *   nchan >= 1; foff != 0 (MHz, negative for a descending band);
 *   fch1 (MHz) centre of channel 0; every channel centre must be > 0;
 *   tsamp > 0 (seconds); dm_list: ndm >= 1 finite values >= 0, any order
 *   (copied).
 * Returns DD_ERR_INVALID on a bad argument, DD_ERR_NOMEM if out of memory. */
dd_status dd_plan(int nchan, double fch1_mhz, double foff_mhz, double tsamp_s,
                  const float *dm_list, int ndm, dd_plan_t *plan_out);

/* Free a plan and its device tables (NULL is a no-op).  No work using the
 * plan may still be in flight. */
void dd_plan_destroy(dd_plan_t plan);

int64_t dd_plan_maxshift(dd_plan_t plan);   /* -1 on NULL */
int dd_plan_nchan(dd_plan_t plan);          /* -1 on NULL */
int dd_plan_ndm(dd_plan_t plan);            /* -1 on NULL */

/* Copy the FP32 dmshift table (nchan floats) to host memory. */
dd_status dd_plan_dmshift(dd_plan_t plan, float *host_out);

/* Tile shape the plan uses for dtype (default heuristic unless set).  */
dd_status dd_plan_get_tiles(dd_plan_t plan, dd_dtype dtype, dd_tiles *tiles_out);

/* Override the tile shape for dtype (validated: shared-memory fit, supported
 * dm_per_thread).  Not thread-safe against concurrent executions of the plan. */
dd_status dd_plan_set_tiles(dd_plan_t plan, dd_dtype dtype, const dd_tiles *tiles);

/* One autotuner measurement. */
typedef struct dd_tune_result {
    dd_tiles tiles;
    float ms;          /* best of the timed runs; < 0 if the shape was rejected */
} dd_tune_result;

/* Autotuner: time every candidate tile shape for dtype on the caller's
 * buffers (same arguments and rules as dd_execute; out is overwritten), keep
 * the fastest as the plan's shape for dtype, and optionally report each
 * candidate (results may be NULL; at most max_results are written, *n_results
 * receives the number measured).  Each candidate runs `reps` timed
 * executions after one warm-up on stream; the call synchronizes stream.
 * Candidates: DMs per thread 1/2/4 x DM warps x time warps x channels per
 * stage, filtered by the shared-memory fit.  Not thread-safe against
 * concurrent executions of the plan. */
dd_status dd_autotune(dd_plan_t plan, const void *in, dd_dtype dtype, int64_t in_pitch,
                      int64_t nsamp_in, float *out, int64_t out_pitch, int64_t nsamp_out,
                      void *stream, int reps, dd_tune_result *results, int max_results,
                      int *n_results);

/* --- single-beam execution (Sec. 3: the GPU kernel) ---------------------- */

/* De-disperse one beam, asynchronously on stream.
 *   in        device pointer to nchan rows (dtype elements, in_pitch apart)
 *   nsamp_in  valid samples per input row; must be >= nsamp_out + maxshift
 *   out       device pointer to ndm FP32 rows, out_pitch floats apart
 *   nsamp_out output samples per DM (>= 0; 0 is a no-op)
 * Validation (DD_ERR_INVALID, nothing launched): alignment rules above,
 * in_pitch >= nsamp_in, out_pitch >= nsamp_out, nsamp_in large enough.
 * The first call on a device uploads the plan's tables (synchronous copy).
 * When the last DM tile of the plan's tile shape would be at most half full
 * and a count of tile rounds says it finishes earlier, the DMs of that tile
 * run as a second launch on a library-owned stream: it waits for an event
 * recorded on `stream` before the call's work, and `stream` waits for its
 * completion, so every later operation on `stream` sees the whole plane. */
dd_status dd_execute(dd_plan_t plan, const void *in, dd_dtype dtype, int64_t in_pitch,
                     int64_t nsamp_in, float *out, int64_t out_pitch, int64_t nsamp_out,
                     void *stream);

/* End-to-end form on HOST buffers (pinned or pageable): copies the input in
 * time blocks to library-owned device buffers, de-disperses each block and
 * copies the plane back, overlapping copies and kernels on two streams.
 * Synchronous: returns when out_host is complete.  Layouts as dd_execute,
 * with pitches in elements of host rows (no alignment rule on host rows). */
dd_status dd_execute_host(dd_plan_t plan, const void *in_host, dd_dtype dtype,
                          int64_t in_pitch, int64_t nsamp_in, float *out_host,
                          int64_t out_pitch, int64_t nsamp_out);

/* De-disperse one beam like dd_execute, without allocating any device memory.
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc -- code running inside an allocator or memory-pool callback,
 * real-time threads that must not take the driver's allocation locks, hosts
 * that forbid the library from owning device memory.  Everything the kernel
 * needs beyond in and out (the plan's device tables and the status word)
 * lives in one fixed 1 MiB device array inside the library, written with
 * copies and a memset on stream; the call makes no cudaMalloc/cudaFree.  Each
 * GPU that loads the library holds that array until the process exits.
 * Limit: 256 + the tables (4 bytes per channel and 8 per DM, the DM count
 * rounded up to a multiple of 64 plus 64, each part rounded up to 256 bytes)
 * must fit in 1 MiB, e.g. 4096 channels and up to about 128000 DMs; a larger
 * plan returns DD_ERR_INVALID (use dd_execute).  The input size is not
 * limited.  The first call on a device looks up the array's device address.
 * The table copies come from pageable host memory that lives only for the
 * call, so the call may wait for earlier work on stream, and a stream that
 * is being captured is refused with DD_ERR_INVALID.  All calls share the
 * array and a call overwrites what the last one left: calls whose GPU work
 * overlaps (other streams or threads) race and must be serialized by the
 * caller.  Kernel-side failures (a bounded wait that ran out, a failed
 * internal check) are recorded in the array's status word, which
 * dd_sync_noalloc reports. */
dd_status dd_execute_noalloc(dd_plan_t plan, const void *in, dd_dtype dtype, int64_t in_pitch,
                             int64_t nsamp_in, float *out, int64_t out_pitch,
                             int64_t nsamp_out, void *stream);

/* Status of dd_execute_noalloc on the current device, allocating nothing:
 * waits for stream, reads the status word of the fixed array and returns
 * DD_OK, DD_ERR_TIMEOUT (a device wait ran out) or DD_ERR_DEVICE (a failed
 * internal check), clearing the word after a failure.  The word is shared
 * like the rest of the array: it reports every no-alloc call since the last
 * dd_execute_noalloc cleared it. */
dd_status dd_sync_noalloc(void *stream);

/* De-disperse a uint8 beam like dd_execute and search the plane for pulses
 * like dd_detect(plane, out_pitch, ndm, nsamp_out, nlevels, 1, ...), with the
 * search fused into the de-dispersion kernel: each CTA searches the tile of
 * the plane it has just finished while the tile is in L2, instead of a
 * second pass reading the whole plane back from HBM (Sec. 4 / Fig. 3 find the
 * pulse at its DM and time after the search).  The plane is still written to
 * out.  Results are those of dd_detect on the same plane, bit for bit: per
 * output row (caller's DM order) mean[ndm], std_out[ndm] and per (row,
 * level) snr[ndm][nlevels], t_peak[ndm][nlevels] (device arrays, 8-byte
 * aligned).  uint8 input only (integer planes), nlevels 1..9, 1 <= nsamp_out
 * <= 2^21.  Uses one launch (no remainder-DM split) with 1024-sample tiles
 * of 4 DMs x 8 words per thread: the plan's uint8 tile shape when it is one
 * of those, else the first automatic shape that is.  Holds one int of device
 * memory per tile, allocated with the plan on first use.  Asynchronous on
 * stream; DD_ERR_INVALID (nothing launched) for bad arguments. */
dd_status dd_execute_detect(dd_plan_t plan, const void *in, dd_dtype dtype, int64_t in_pitch,
                            int64_t nsamp_in, float *out, int64_t out_pitch, int64_t nsamp_out,
                            int nlevels, double *mean, double *std_out, double *snr,
                            int64_t *t_peak, void *stream);

/* --- input side: corner turn and bit unpacking ---------------------------- */

/* Turn a block of filterbank spectra into the channel rows that dd_execute
 * reads.  The paper's test data are sigproc filterbanks (Sec. 2, Fig. 1):
 * nsamp spectra follow one another, each holding nchan samples of nbits bits
 * (1, 2, 4 or 8), packed in channel order from the lowest bit of each byte
 * (channel c of spectrum t starts at bit (t*nchan + c)*nbits of the block;
 * bit b is bit b%8 of byte b/8).
 *   in:  device pointer to nsamp*nchan*nbits/8 bytes; any alignment.  Input
 *        that is 16-byte aligned, with nchan a multiple of 128 and spectra a
 *        multiple of 16 bytes, takes the faster tiled path.
 *   out: device uint8 [nchan][out_pitch], 16-byte aligned, out_pitch >= nsamp
 *        and a multiple of 16; out[c][t] = the sample (0 .. 2^nbits - 1, not
 *        rescaled).  Columns t >= nsamp are left untouched.
 * nchan*nbits must be a multiple of 8 (whole-byte spectra).  Asynchronous on
 * stream; returns DD_ERR_INVALID (nothing launched) for bad arguments. */
dd_status dd_unpack(const void *in, int nbits, int nchan, int64_t nsamp, uint8_t *out,
                    int64_t out_pitch, void *stream);

/* --- detection: matched boxcar search of the (DM,t) plane ----------------- */

/* Search every DM row of a de-dispersed plane for pulses.  Sec. 4 and Fig. 3
 * of the paper find a simulated pulse at its DM and time; the paper gives no
 * formula, and the library's reading is matched boxcar filters with a per-row
 * noise estimate.  For each row x[0..nsamp):
 *   mean = S1/n, std = sqrt(S2/n - mean^2) (0 if negative), with S1 = sum x,
 *   S2 = sum x^2, n = nsamp;
 *   for each width w = 2^l, l = 0..nlevels-1: the largest boxcar sum
 *   B = x[t] + ... + x[t+w-1] over t = 0..nsamp-w, at its first t, and
 *   snr = (B - w*mean) / (std*sqrt(w)) (0 if std is 0; t = -1 and snr = -inf
 *   if nsamp < w).
 * integer_valued != 0 (planes of uint8 input): every value must be an integer
 * in [0, 2^21) and nsamp <= 2^21; the sums are then exact and the results are
 * identical, bit for bit, to the FP64 CPU definition.  A row holding any other
 * value reports NaN mean, std and S/N.  Otherwise sums are FP32 boxcars and
 * FP64 row sums (order-dependent rounding).
 *   plane: device FP32 [ndm][pitch] (4-byte aligned, pitch >= nsamp).
 *   mean, std: device double [ndm]; snr: device double [ndm][nlevels];
 *   t_peak: device int64 [ndm][nlevels]; all 8-byte aligned, owned by the
 *   caller and overwritten (they also serve as the accumulators).
 * nlevels is 1..9 (widths up to 256).  Asynchronous on stream; bad arguments
 * return DD_ERR_INVALID with nothing launched. */
dd_status dd_detect(const float *plane, int64_t pitch, int ndm, int64_t nsamp, int nlevels,
                    int integer_valued, double *mean, double *std, double *snr, int64_t *t_peak,
                    void *stream);

/* --- front end: voltages -> the uint8 filterbank -------------------------- */

/* Turn channelised dual-polarisation voltages into the uint8 filterbank that
 * dd_execute reads.  Sec. 1 of the paper lists the steps before the
 * dispersion search (Stokes parameters, RFI excision, integration) without
 * formulas; the library's reading:
 *   I[c][r] = Xre^2 + Xim^2 + Yre^2 + Yim^2 of raw sample r (int8 each);
 *   P[c][t] = I[c][t*nint] + ... + I[c][t*nint + nint - 1], t < n =
 *   nsamp_raw / nint (trailing raw samples are dropped);
 *   RFI excision by niter passes of sigma clipping: each pass takes, over
 *   the samples the previous pass kept (all of them for the first), the
 *   exact count, S1 = sum P and S2 = sum P^2, then mean = S1/cnt,
 *   std = sqrt(S2/cnt - mean^2) (0 if negative; both 0 if cnt == 0) and
 *   thr = floor(mean + k_clip*std) in FP64; the next pass keeps P <= thr;
 *   with the last pass's values: P > thr becomes code 128, otherwise
 *   code = clamp(rint(128 + ((float)P - (float)mean) * (float)(16/std)),
 *   0, 255), in FP32 one IEEE operation at a time; std == 0 gives 128.
 *   volts: device int8 [nchan][volts_pitch bytes], raw sample r of channel c
 *          at bytes 4r..4r+3 of the row (Xre, Xim, Yre, Yim); 4-byte aligned,
 *          volts_pitch >= 4*nsamp_raw and a multiple of 4 (16-byte aligned
 *          rows with nint a multiple of 4 take 16-byte loads).
 *   nint:  a power of two, 1..64; n <= 2^19 (the sums of P^2 stay exact).
 *   k_clip: in (0, 1e9]; niter: 1..8 (1 is a single clip with the
 *          statistics of all samples).
 *   out:   device uint8 [nchan][out_pitch], 16-byte aligned, out_pitch >= n
 *          and a multiple of 16; columns >= n are left untouched.
 *   work:  device scratch of work_bytes >= dd_frontend_work_bytes(...),
 *          16-byte aligned, owned by the caller (P and the exact sums; only
 *          rows longer than the fused kernel holds use it).
 *   mean, std: device double [nchan], 8-byte aligned: the last pass's values
 *          (0 when n == 0).
 * Rows of n <= 409600 run in one launch: a thread-block cluster of 1..8 CTAs
 * per channel keeps P in shared memory, so the voltages are read once and
 * nothing else touches HBM but the codes.  Longer rows keep P in work
 * (niter + 1 launches and a memset).  Asynchronous on stream; bad arguments
 * return DD_ERR_INVALID with nothing launched.  The oracle's front end gives
 * the same codes, mean and std bit for bit. */
dd_status dd_frontend(const void *volts, int64_t volts_pitch, int nchan, int64_t nsamp_raw,
                      int nint, double k_clip, int niter, uint8_t *out, int64_t out_pitch,
                      void *work, int64_t work_bytes, double *mean, double *std, void *stream);

/* Bytes of work dd_frontend needs for this shape; -1 if the shape is invalid. */
int64_t dd_frontend_work_bytes(int nchan, int64_t nsamp_raw, int nint, int niter);

/* --- channeliser: subband voltages -> finer channels ----------------------- */

/* Output element kinds of dd_channelise. */
enum {
    DD_PFB_CF32 = 0,  /* four FP32 (Xre, Xim, Yre, Yim): 16 bytes per element   */
    DD_PFB_CI8 = 1    /* four int8 codes (Xre, Xim, Yre, Yim): 4 bytes, the
                         element dd_frontend reads                                */
};

/* Split each subband of dual-polarisation voltages into M finer channels with
 * a critically sampled polyphase filter bank.  The paper channelises the
 * received subbands in finer frequency before forming Stokes parameters
 * (Sec. 1) and names the poly-phase filter (Sec. 5) without giving the
 * filter or the transform size; the library's reading, per polarisation
 * with x[j] = re + i*im of raw sample j:
 *   y_k[n] = sum_{m < M*T} h[m] x[n*M + m] exp(-2 pi i k m / M),  k < M,
 *   for spectra n < nspec = floor(nraw/M) - T + 1 (0 if negative);
 *   channel c = (k + M/2) mod M of subband s goes to row s*M + c, so the
 *   channels of a subband run in increasing frequency; column n.
 *   volts: device int8 [nsub][volts_pitch bytes], raw sample j of subband s
 *          at bytes 4j..4j+3 of the row (Xre, Xim, Yre, Yim); 4-byte aligned,
 *          volts_pitch >= 4*nraw and a multiple of 4.
 *   nchan_sub (M): 16, 32, 64, 128 or 256; ntaps (T): 1..16; nsub: 1..65535.
 *   coeffs: device FP32 [M*T], the prototype filter h (dd_pfb_prototype
 *          gives the windowed-sinc one); 4-byte aligned.
 *   out_kind DD_PFB_CF32: FP32 elements, computed in FP32 (FIR by FMA, a
 *          16 x M/16 four-step FFT with twiddles from sincospif); error
 *          within (T + 6 log2 M + 8) * 2^-23 * sum_m |h[m]| |x| of the
 *          exact value, |x| the sum of the component magnitudes.
 *   out_kind DD_PFB_CI8: int8 codes q = clamp(rint(v * scale), -127, 127),
 *          v the FP32 value above and v*scale rounded once to an integer
 *          (ties to even); scale finite and > 0.  Cells whose exact value
 *          lies within the FP32 error of a rounding boundary may take either
 *          neighbouring code.
 *   out:   device [nsub*M][out_pitch bytes], aligned to its element (4 or 16
 *          bytes), out_pitch >= element * nspec and a multiple of it; columns
 *          >= nspec are left untouched.
 * One launch; each raw word is read from HBM once and each element written
 * once.  Asynchronous on stream; bad arguments return DD_ERR_INVALID with
 * nothing launched; nspec == 0 launches nothing. */
dd_status dd_channelise(const void *volts, int64_t volts_pitch, int nsub, int64_t nraw,
                        int nchan_sub, int ntaps, const float *coeffs, int out_kind, float scale,
                        void *out, int64_t out_pitch, void *stream);

/* Spectra dd_channelise produces per subband: floor(nraw/M) - T + 1, 0 if
 * that is negative, -1 for an invalid M, T or nraw. */
int64_t dd_channelise_nspec(int64_t nraw, int nchan_sub, int ntaps);

/* Host: the windowed-sinc prototype of M*T taps, FP64 rounded once to FP32:
 *   h[m] = sinc((m - (L-1)/2) / M) * (0.54 - 0.46 cos(2 pi m / (L-1))),
 *   sinc(x) = sin(pi x)/(pi x), L = M*T >= 2 (a Hamming-windowed sinc whose
 *   cutoff is half a channel spacing; its sum is about M).
 * h: host float [M*T], owned by the caller.  The paper names no filter. */
dd_status dd_pfb_prototype(int nchan_sub, int ntaps, float *h);

/* --- batches: uneven beams in one persistent launch ------------------------ */

typedef struct dd_batch_s *dd_batch_t;

/* A batch runs many beams -- each with its own plan (nchan, band, DM list)
 * and its own buffers -- in one persistent de-dispersion launch: one CTA per
 * SM claims (beam, DM tile, time tile) work items, largest beams first, from
 * an atomic counter.  The launch (and the reset of the counter before it) is
 * captured once into a CUDA graph and replayed by later
 * dd_batch_execute calls (re-captured after dd_batch_set_io or a tile change).
 * All beams share one tile shape (dd_batch_set_tiles / dd_batch_autotune).
 * plans[i] must outlive the batch; the batch owns its device descriptors and
 * counters. */
dd_status dd_batch_create(const dd_plan_t *plans, int nbeams, dd_dtype dtype,
                          dd_batch_t *batch_out);
void dd_batch_destroy(dd_batch_t batch);

/* Bind beam i's device buffers (layouts and rules as dd_execute). */
dd_status dd_batch_set_io(dd_batch_t batch, int beam, const void *in, int64_t in_pitch,
                          int64_t nsamp_in, float *out, int64_t out_pitch, int64_t nsamp_out);

/* Run every beam of the batch, asynchronously on stream. */
dd_status dd_batch_execute(dd_batch_t batch, void *stream);

dd_status dd_batch_get_tiles(dd_batch_t batch, dd_tiles *tiles_out);
dd_status dd_batch_set_tiles(dd_batch_t batch, const dd_tiles *tiles);

/* Autotuner for the batch: times each candidate tile shape that fits every
 * beam on the bound buffers (outputs are overwritten), keeps the fastest.
 * Same reporting as dd_autotune; synchronizes stream. */
dd_status dd_batch_autotune(dd_batch_t batch, void *stream, int reps, dd_tune_result *results,
                            int max_results, int *n_results);

/* Synchronize stream and report the batch's device status word. */
dd_status dd_batch_sync(dd_batch_t batch, void *stream);

/* --- serving: streaming beams, continuous batching ------------------------- */

typedef struct dd_server_s *dd_server_t;
typedef uint64_t dd_ticket;

typedef struct dd_server_stats {
    int64_t submitted;       /* blocks accepted by dd_submit                   */
    int64_t completed;       /* blocks whose result is in the caller's buffer  */
    int64_t rejected_busy;   /* dd_submit calls that returned DD_ERR_BUSY      */
    int64_t batches;         /* batched launches issued                        */
    double p50_ms, p99_ms, max_ms;  /* submit -> result latency of completed blocks */
    double mean_batch;       /* mean blocks per batched launch                  */
    int slots;               /* device slots (blocks in flight at most)         */
    int64_t device_bytes;    /* device memory held (slots + beam tails)         */
    int64_t staging_bytes;   /* block bytes copied into pinned staging by dd_submit */
    double staging_ms;       /* host time of those copies (wall clock, summed)  */
    int64_t h2d_bytes;       /* block bytes copied host -> device               */
    double h2d_ms;           /* device time of the batches' input phases (the    */
                             /* host-to-device copies and the tail copies)      */
    int64_t d2h_bytes;       /* result bytes copied device -> host              */
    double d2h_ms;           /* device time of the batches' result copies        */
    int64_t batch_window_us; /* batching window in force                        */
    double kernel_ms;        /* device time of the batches' kernel phases (from  */
                             /* the end of the input phase, a wait for SMs the  */
                             /* other lane's kernel holds included)             */
} dd_server_stats;

/* A server de-disperses streams of blocks from many beams (the real-time
 * search of Sec. 1-2).  Every beam keeps the last maxshift samples of each
 * channel on the device (its overlap tail), so block k is processed as
 * [tail | block] and yields the outputs of stream samples
 * [k*B - maxshift, (k+1)*B - maxshift) (block 0: [0, B - maxshift)), B the
 * beam's block length.  A worker thread batches blocks of different beams
 * that are ready (previous block's tail in place) into one persistent launch
 * as device slots free up, while later blocks are being copied in: continuous
 * batching.  Device memory = slots + tails, bounded by hbm_budget_bytes; the
 * number of slots is min(max_inflight, what the budget allows after tails).
 * Blocks wait in pinned host staging (2 x slots buffers); dd_submit returns
 * DD_ERR_BUSY when none is free.  dd_submit copies a block into staging
 * with a few host threads.  A partly filled batch waits up to the batching
 * window for more ready blocks; unless set with dd_server_set_batch_window,
 * the window is 1/64 of the shortest block duration of the server's beams
 * (B * tsamp), at most 100 ms -- 65 ms for blocks of 65536 samples of 64 us. */
dd_status dd_server_create(size_t hbm_budget_bytes, int max_inflight, dd_dtype dtype,
                           dd_server_t *server_out);

/* Register a streaming beam (plan must outlive the server).  block_nsamp B
 * must exceed the plan's maxshift.  Beams must be added before the first
 * dd_submit. */
dd_status dd_server_add_beam(dd_server_t server, dd_plan_t plan, int64_t block_nsamp,
                             int *beam_id_out);

/* Queue the next block of a beam: block_host holds nchan rows of B samples,
 * in_pitch elements apart (copied before return).  out_host receives ndm rows
 * (out_pitch floats apart, >= B) of the block's outputs when dd_poll reports
 * DD_OK; it must stay valid until then (pinned memory lets the copy overlap).
 * DD_ERR_BUSY: no staging buffer free right now (retry later). */
dd_status dd_submit(dd_server_t server, int beam_id, const void *block_host, int64_t in_pitch,
                    float *out_host, int64_t out_pitch, dd_ticket *ticket_out);

/* DD_OK once the block's outputs are in out_host (first_t: stream sample of
 * out row column 0; nsamp: columns written), DD_PENDING while in flight,
 * DD_ERR_INVALID for an unknown or already collected ticket, another error if
 * the block failed.  A ticket is collected by the first DD_OK (or error). */
dd_status dd_poll(dd_server_t server, dd_ticket ticket, int64_t *first_t, int64_t *nsamp);

/* Batching window: when ready blocks fill fewer than the free slots, the
 * worker waits up to `microseconds` for more to arrive before launching
 * (0, the default, launches at once).  Trades latency for larger batches. */
dd_status dd_server_set_batch_window(dd_server_t server, int64_t microseconds);

/* Wait (up to timeout_ms) until every submitted block has completed. */
dd_status dd_server_drain(dd_server_t server, int64_t timeout_ms);

dd_status dd_server_get_stats(dd_server_t server, dd_server_stats *stats_out);

/* Stop the worker threads (after draining in-flight blocks) and free all. */
dd_status dd_server_destroy(dd_server_t server);

/* Synchronize stream and report the plan's device status word (DD_OK,
 * DD_ERR_TIMEOUT or DD_ERR_DEVICE), then clear it. */
dd_status dd_sync(dd_plan_t plan, void *stream);

/* Add-throughput microbenchmark, the measured denominator of the
 * de-dispersion roofline (the method is bound by one 32-bit add per channel,
 * DM and sample).  The paper has no counterpart: it quotes its kernel as a
 * fraction of peak (Sec. 5) without saying how the peak was obtained.
 * Launches ctas_per_sm (1..8) CTAs of 256 threads per SM, each thread running
 * 8 independent chains of one add kind: kind 0 = FP32 add.rn.f32, kind 1 =
 * 32-bit integer adds split between the integer ALU (add.u32) and the FMA
 * pipe (mad.lo.u32 by a run-time 1), kind 2 = packed FP32 pairs
 * (add.rn.f32x2, two adds each).  Times 3 launches after a warm-up with CUDA
 * events on stream and writes the best as adds per second to *adds_per_s and
 * its duration (ms) to *ms_out (may be NULL).  Synchronous; allocates
 * nothing.  Returns DD_ERR_INVALID for a bad kind or CTA count. */
dd_status dd_add_peak(int kind, int ctas_per_sm, void *stream, double *adds_per_s,
                      double *ms_out);

/* Profiling hook: while set (non-NULL), every execution issued from this
 * thread records start_event just before its de-dispersion kernel and
 * stop_event just after it, on the launch stream (cudaEvent_t handles owned
 * by the caller).  Pass NULLs to clear. */
void dd_profile_events(void *start_event, void *stop_event);

/* Self-test of the kernels' bounded waits: one CTA waits, through the same
 * wait routine the de-dispersion kernel uses, on an mbarrier that nothing
 * arrives on, with a limit of limit_ns (1 us .. 2 s).  Returns DD_ERR_TIMEOUT
 * when the wait gave up and reported it as designed (no fault, no hang);
 * synchronizes stream. */
dd_status dd_selftest_wait_timeout(int64_t limit_ns, void *stream);

/* The same wait, recording its timeout in the status word of
 * dd_execute_noalloc's fixed array (reported by dd_sync_noalloc) instead of
 * a word of its own.  Allocates nothing; asynchronous on stream. */
dd_status dd_selftest_noalloc_timeout(int64_t limit_ns, void *stream);

/* Kernel launches made by this process so far (all entry points). */
int64_t dd_launch_count(void);

/* Message for the last non-OK status returned on this thread. */
const char *dd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
