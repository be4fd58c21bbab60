// Input side of the search: corner turn and bit unpacking of filterbank
// spectra (dd_unpack).
//
// The paper's test data are sigproc filterbanks (Sec. 2, Fig. 1): spectra
// follow one another in time, each holding nchan samples of nbits bits
// (1, 2, 4 or 8) packed from the lowest bit of each byte.  The de-dispersion
// kernel reads channel rows, so a block of spectra is turned into
// out[c][t] (one byte per sample, value kept).
//
// One CTA handles tiles of 128 channels x 128 spectra (256 for 8-bit input;
// grid x: channel tiles; grid y strides over time tiles).  The tile's bytes are loaded
// row by row (one row = one spectrum's bytes for those channels) with
// coalesced 16-byte loads when every spectrum starts on 16 bytes, byte loads
// otherwise, into shared memory rows padded to an odd number of words.  Then
// each thread reads one 32-bit column word from 4 consecutive rows and builds
// an output word -- 4 consecutive spectra of one channel -- for every channel
// in that column word.  HBM-bound: nchan*nsamp*nbits/8 bytes in,
// nchan*nsamp bytes out.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "dd_internal.h"

namespace {

constexpr int kTileC = 128;  // channels per tile
// Spectra per tile: longer output runs per channel row help 8-bit input
// (measured 4.5 vs 4.1 TB/s on an L-band block); narrower samples run best
// at 128.
__host__ __device__ constexpr int tile_t(int nbits) { return nbits == 8 ? 256 : 128; }

template <int NBITS>
__global__ void __launch_bounds__(256) unpack_kernel(const uint8_t *__restrict__ in,
                                                     int64_t spec_bytes, int nchan, int64_t nsamp,
                                                     uint8_t *__restrict__ out, int64_t out_pitch,
                                                     int64_t ntile_t, int vec) {
    constexpr int kTileT = tile_t(NBITS);
    constexpr int SEG = kTileC * NBITS / 8;  // bytes of one spectrum in a full tile
    constexpr int STRIDE = SEG + 4;          // shared row: an odd number of 4-byte words
    constexpr uint32_t MASK = (1u << NBITS) - 1u;
    __shared__ __align__(16) uint8_t tile[kTileT * STRIDE];

    const int c0 = blockIdx.x * kTileC;
    const int64_t cb0 = (int64_t)c0 * NBITS / 8;  // first byte of the tile in a spectrum
    const int seg = spec_bytes - cb0 < SEG ? (int)(spec_bytes - cb0) : SEG;
    const int nc = nchan - c0 < kTileC ? nchan - c0 : kTileC;
    // 16-byte path: the next tile's loads are issued into registers before
    // the current tile is written out, so they overlap the output phase.
    constexpr int CH = SEG / 16;                         // 16-byte chunks per row
    constexpr int NV = (kTileT * CH + 255) / 256;        // chunks per thread (256 threads)
    uint4 pre[NV];
    auto fetch = [&](int64_t t0n, int rowsn) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int i = threadIdx.x + 256 * v;
            if (i < rowsn * CH)
                pre[v] = *reinterpret_cast<const uint4 *>(in + (t0n + i / CH) * spec_bytes + cb0 +
                                                          16 * (i % CH));
        }
    };
    auto rows_of = [&](int64_t tt) {
        const int64_t left = nsamp - tt * kTileT;
        return left < kTileT ? (int)left : kTileT;
    };
    if (vec && blockIdx.y < ntile_t)
        fetch((int64_t)blockIdx.y * kTileT, rows_of(blockIdx.y));
    for (int64_t tt = blockIdx.y; tt < ntile_t; tt += gridDim.y) {
        const int64_t t0 = tt * kTileT;
        const int rows = rows_of(tt);
        __syncthreads();  // the previous tile has been read
        if (vec) {
            // spec_bytes and cb0 are multiples of 16 and seg == SEG here
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const int i = threadIdx.x + 256 * v;
                if (i < rows * CH) {
                    uint32_t *dst = reinterpret_cast<uint32_t *>(tile + (i / CH) * STRIDE +
                                                                 16 * (i % CH));
                    dst[0] = pre[v].x;
                    dst[1] = pre[v].y;
                    dst[2] = pre[v].z;
                    dst[3] = pre[v].w;
                }
            }
        } else {
            for (int i = threadIdx.x; i < rows * seg; i += blockDim.x) {
                const int r = i / seg, b = i % seg;
                tile[r * STRIDE + b] = in[(t0 + r) * spec_bytes + cb0 + b];
            }
        }
        __syncthreads();
        if (vec && tt + gridDim.y < ntile_t)
            fetch((tt + gridDim.y) * kTileT, rows_of(tt + gridDim.y));
        // Output.  An item is (word q: spectra 4q..4q+3, column word cw: the
        // 32/NBITS channels held in bytes 4cw..4cw+3 of a row).  Lane l takes
        // q = 8*qg + l/4 and cw = 4*cg + l%4, so the 4 rows a warp reads per
        // step fall in 32 different banks and each channel's 8 output words
        // fill one 32-byte sector.  Channel j of the column word comes from
        // byte (j*NBITS)/8 of each of the 4 rows: three byte permutes gather
        // those bytes into one word, and a shift and mask extract the field.
        const int lq = (threadIdx.x & 31) >> 2, lc = threadIdx.x & 3;
        constexpr int NCG = SEG / 16;  // groups of 4 column words
        for (int g = threadIdx.x >> 5; g < (kTileT / 32) * NCG; g += blockDim.x >> 5) {
            const int q = 8 * (g / NCG) + lq;
            const int cw = 4 * (g % NCG) + lc;
            if (4 * q >= rows || cw * (32 / NBITS) >= nc)
                continue;
            const uint32_t *rp = reinterpret_cast<const uint32_t *>(tile + 4 * q * STRIDE) + cw;
            const uint32_t r0 = rp[0], r1 = rp[STRIDE / 4], r2 = rp[2 * (STRIDE / 4)],
                           r3 = rp[3 * (STRIDE / 4)];
            const int64_t t = t0 + 4 * q;
            uint8_t *dst = out + (int64_t)(c0 + cw * (32 / NBITS)) * out_pitch + t;
            const bool whole = t + 4 <= nsamp;
#pragma unroll
            for (int jc = 0; jc < 32 / NBITS; ++jc) {
                if (cw * (32 / NBITS) + jc >= nc)
                    break;
                constexpr uint32_t LANES = MASK * 0x01010101u;
                const uint32_t bj = (uint32_t)(jc * NBITS / 8);
                const uint32_t sel = ((4u + bj) << 4) | bj;
                uint32_t w = __byte_perm(__byte_perm(r0, r1, sel), __byte_perm(r2, r3, sel), 0x5410);
                if (NBITS < 8)
                    w = (w >> ((jc * NBITS) % 8)) & LANES;
                uint8_t *d = dst + (int64_t)jc * out_pitch;
                if (whole) {
                    *reinterpret_cast<uint32_t *>(d) = w;
                } else {
                    for (int k = 0; t + k < nsamp; ++k)
                        d[k] = (uint8_t)(w >> (8 * k));
                }
            }
        }
    }
}

template <int NBITS>
cudaError_t launch_unpack(const uint8_t *in, int64_t spec_bytes, int nchan, int64_t nsamp,
                          uint8_t *out, int64_t out_pitch, int vec, cudaStream_t s) {
    constexpr int kTileT = tile_t(NBITS);
    const int ntc = (nchan + kTileC - 1) / kTileC;
    const int64_t ntt = (nsamp + kTileT - 1) / kTileT;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // about 8 resident CTAs per SM in total
    const int64_t want = std::max<int64_t>(1, (int64_t)nsm * 8 / ntc);
    const unsigned gy = (unsigned)std::min<int64_t>(std::min<int64_t>(ntt, want), 65535);
    unpack_kernel<NBITS><<<dim3((unsigned)ntc, gy), 256, 0, s>>>(in, spec_bytes, nchan, nsamp, out,
                                                                 out_pitch, ntt, vec);
    return cudaGetLastError();
}

}  // namespace

extern "C" dd_status dd_unpack(const void *in, int nbits, int nchan, int64_t nsamp, uint8_t *out,
                               int64_t out_pitch, void *stream) {
    dd::Range nvtx_range("dd_unpack");
    using dd::fail;
    if (nbits != 1 && nbits != 2 && nbits != 4 && nbits != 8)
        return fail(DD_ERR_INVALID, "nbits must be 1, 2, 4 or 8");
    if (nchan < 1 || ((int64_t)nchan * nbits) % 8 != 0)
        return fail(DD_ERR_INVALID, "nchan*nbits must be a positive multiple of 8");
    if (nsamp < 0 || out_pitch < nsamp || out_pitch % 16 != 0)
        return fail(DD_ERR_INVALID, "out_pitch must be >= nsamp and a multiple of 16");
    if (nsamp == 0)
        return DD_OK;
    if (!in || !out || ((uintptr_t)out & 15u))
        return fail(DD_ERR_INVALID, "in must be non-NULL and out non-NULL and 16-byte aligned");
    const int64_t spec_bytes = (int64_t)nchan * nbits / 8;
    // 16-byte loads need every spectrum and every channel tile on 16 bytes
    // and whole tiles across the spectrum.
    const int vec = ((uintptr_t)in & 15u) == 0 && spec_bytes % 16 == 0 &&
                    (nchan % kTileC == 0);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint8_t *src = static_cast<const uint8_t *>(in);
    cudaError_t e = cudaSuccess;
    switch (nbits) {
    case 1: e = launch_unpack<1>(src, spec_bytes, nchan, nsamp, out, out_pitch, vec, s); break;
    case 2: e = launch_unpack<2>(src, spec_bytes, nchan, nsamp, out, out_pitch, vec, s); break;
    case 4: e = launch_unpack<4>(src, spec_bytes, nchan, nsamp, out, out_pitch, vec, s); break;
    default: e = launch_unpack<8>(src, spec_bytes, nchan, nsamp, out, out_pitch, vec, s); break;
    }
    if (e != cudaSuccess)
        return fail(DD_ERR_CUDA, std::string("unpack launch failed: ") + cudaGetErrorString(e));
    dd::count_launch(1);
    return DD_OK;
}
