// dd_execute_noalloc: the single-beam de-dispersion with no device
// allocation at all.
//
// Some callers cannot call cudaMalloc: code running inside a custom
// allocator or a memory-pool callback, real-time threads that must not take
// the driver's allocation locks, and hosts that forbid the library from
// owning device memory.  For them this entry point keeps everything the
// kernel needs beyond the caller's input and output -- the plan's device
// tables and the status word -- in one file-scope device array of fixed
// size, and writes it with plain copies and a memset on the caller's stream.
//
// The array is shared by every call in the process: a call overwrites what
// the previous one left there, so calls whose GPU work overlaps (on
// different streams, or from different threads) race and must be serialized
// by the caller.  Each GPU that loads this library holds the array until the
// process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dd_internal.h"

namespace {

constexpr size_t kNoAllocBytes = (size_t)1 << 20;  // 1 MiB

// Device-side scratch of dd_execute_noalloc.  In host code this name is a
// host-side stand-in, not a device address: the address handed to kernels
// comes from cudaGetSymbolAddress (noalloc_base below).
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {nullptr};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the array on the current device, looked up once per
// device (the first call on a device; it must come before any stream capture).
dd_status noalloc_base(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return dd::fail(DD_ERR_CUDA, "cudaGetDevice failed");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return dd::fail(DD_ERR_CUDA, std::string("cudaGetSymbolAddress of the fixed scratch "
                                                     "failed: ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return DD_OK;
}

}  // namespace

namespace dd {

dd_status noalloc_status_word(int **out) {
    void *base = nullptr;
    dd_status st = noalloc_base(&base);
    if (st != DD_OK)
        return st;
    *out = reinterpret_cast<int *>(base);  // the status word sits at offset 0
    return DD_OK;
}

}  // namespace dd

extern "C" dd_status dd_execute_noalloc(dd_plan_t p, const void *in, dd_dtype dtype,
                                        int64_t in_pitch, int64_t nsamp_in, float *out,
                                        int64_t out_pitch, int64_t nsamp_out, void *stream) {
    using dd::fail;
    dd::Range nvtx_range("dd_execute_noalloc");
    if (!p)
        return fail(DD_ERR_INVALID, "plan is NULL");
    dd_status st = dd::check_layout(p, dtype, in_pitch, nsamp_in, out_pitch, nsamp_out, true);
    if (st != DD_OK)
        return st;
    if (nsamp_out == 0)
        return DD_OK;
    if (!in || !out || ((uintptr_t)in & 15u) || ((uintptr_t)out & 15u))
        return fail(DD_ERR_INVALID, "in and out must be non-NULL and 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The table copies below come from pageable host vectors that live only
    // for this call: a stream capture would refuse them (and invalidate the
    // caller's capture), so a capturing stream is turned away up front.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess)
        return fail(DD_ERR_CUDA, "cudaStreamIsCapturing failed");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(DD_ERR_INVALID, "dd_execute_noalloc does not run on a capturing stream");

    // Layout of the fixed array for this call.
    const int ndm_pad = (p->ndm + 63) / 64 * 64 + 64;
    const size_t off_status = 0;
    const size_t off_dmshift = 256;
    const size_t off_dm = off_dmshift + align256(sizeof(float) * (size_t)p->nchan);
    const size_t off_perm = off_dm + align256(sizeof(float) * (size_t)ndm_pad);
    const size_t need = off_perm + align256(sizeof(int) * (size_t)ndm_pad);
    if (need > kNoAllocBytes)
        return fail(DD_ERR_INVALID,
                    "plan too large for dd_execute_noalloc: its tables need " +
                        std::to_string(need) + " bytes of the fixed " +
                        std::to_string(kNoAllocBytes) + "-byte array; use dd_execute");

    dd::Geometry g;
    if ((st = dd::plan_geometry(p, dtype, &g)) != DD_OK)
        return st;
    void *base = nullptr;
    if ((st = noalloc_base(&base)) != DD_OK)
        return st;
    uint8_t *b = static_cast<uint8_t *>(base);

    // Plan tables as the kernels expect them: DMs ascending, padded with the
    // largest; perm maps a sorted position to the caller's row (-1: padding).
    std::vector<float> dms(ndm_pad, p->dm_sorted.back());
    std::vector<int> perm(ndm_pad, -1);
    for (int k = 0; k < p->ndm; ++k) {
        dms[k] = p->dm_sorted[k];
        perm[k] = p->order[k];
    }
    cudaError_t e = cudaMemsetAsync(b + off_status, 0, sizeof(int), s);  // status starts clear
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + off_dmshift, p->dmshift.data(), sizeof(float) * p->nchan,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + off_dm, dms.data(), sizeof(float) * ndm_pad,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + off_perm, perm.data(), sizeof(int) * ndm_pad,
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("table copy: ") + cudaGetErrorString(e));

    dd::DevTables dt;
    dt.dmshift = reinterpret_cast<float *>(b + off_dmshift);
    dt.dm_sorted = reinterpret_cast<float *>(b + off_dm);
    dt.perm = reinterpret_cast<int *>(b + off_perm);
    dt.status = reinterpret_cast<int *>(b + off_status);
    dt.ndm_pad = ndm_pad;
    // One launch: the remainder-DM split needs a library stream and events.
    return dd::launch_dedisperse(p, g, dt, in, dtype, in_pitch, nsamp_in, out, out_pitch,
                                 nsamp_out, stream, false);
}

// Status of the last dd_execute_noalloc on the current device: waits for
// stream, reads the status word of the fixed array into a host int and, if a
// kernel recorded a failure there, clears it.  Allocates nothing.
extern "C" dd_status dd_sync_noalloc(void *stream) {
    using dd::fail;
    dd::Range nvtx_range("dd_sync_noalloc");
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("stream synchronize: ") + cudaGetErrorString(e));
    int *status = nullptr;
    dd_status st = dd::noalloc_status_word(&status);
    if (st != DD_OK)
        return st;
    int word = 0;
    if ((e = cudaMemcpy(&word, status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    if (word == dd::kDevOk)
        return DD_OK;
    if ((e = cudaMemset(status, 0, sizeof(int))) != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("status clear: ") + cudaGetErrorString(e));
    return word == dd::kDevTimeout
               ? fail(DD_ERR_TIMEOUT, "a device wait of dd_execute_noalloc ran out")
               : fail(DD_ERR_DEVICE, "a dd_execute_noalloc kernel recorded a failed check");
}
