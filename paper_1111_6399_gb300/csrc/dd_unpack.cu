// Input side of the search: corner turn and bit unpacking of filterbank
// spectra (dd_unpack).
//
// The paper's test data are sigproc filterbanks (Sec. 2, Fig. 1): spectra
// follow one another in time, each holding nchan samples of nbits bits
// (1, 2, 4 or 8) packed from the lowest bit of each byte.  The de-dispersion
// kernel reads channel rows, so a block of spectra is turned into
// out[c][t] (one byte per sample, value kept).
//
// Two kernels.  The tiled kernel takes input whose spectra all start on 16
// bytes, with whole 128-channel tiles; the byte kernel takes anything else.
//
// Tiled kernel: a CTA works on one 128-channel tile of the spectrum and
// strides over 256-spectrum time tiles.
//  * Input: 16-byte asynchronous copies (cp.async) bring each time tile's
//    rows (one row = one spectrum's bytes for those channels) into a ring of
//    shared-memory buffers, NBUF - 1 tiles ahead of the one being turned.
//    Row r sits at r*(SEG + 16) + (r/4)*16 bytes: aligned for the copies,
//    and the 4 rows a warp reads per step fall in 32 different banks.
//  * Corner turn: each thread reads one 32-bit column word from 4
//    consecutive rows and builds, for every channel in that word, an output
//    word of 4 consecutive spectra (three byte permutes, then a shift and a
//    mask for fields below 8 bits).  The words go into a transposed tile
//    out[c][t] in shared memory; word q of row c is stored at q ^ (8 f(c)),
//    which spreads the 4 column words a warp handles per step over distinct
//    banks.
//  * Output: whole rows of the transposed tile leave as 16-byte stores
//    (chunk k of row c read from k ^ (2 f(c))), 256 contiguous bytes of a
//    channel row per half-warp.  Writing rows whole is what lifts the kernel
//    above the byte kernel's 4-byte stores, each of which spread over four
//    channel rows (measured 5.5 against 4.5 TB/s for 8-bit L-band spectra).
//
// Byte kernel: tiles of 128 channels x 128 spectra (256 for 8-bit input)
// loaded byte by byte into shared-memory rows padded to an odd number of
// words; the same corner turn, written straight to global memory.
//
// HBM-bound: nchan*nsamp*nbits/8 bytes in, nchan*nsamp bytes out.
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

// Output word of channel jc of a column word: its field from each of the 4
// rows r0..r3 (4 consecutive spectra), one byte per spectrum.
template <int NBITS>
__device__ __forceinline__ uint32_t turn_word(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3,
                                              int jc) {
    constexpr uint32_t LANES = ((1u << NBITS) - 1u) * 0x01010101u;
    const uint32_t bj = (uint32_t)(jc * NBITS / 8);
    const uint32_t sel = ((4u + bj) << 4) | bj;
    uint32_t w = __byte_perm(__byte_perm(r0, r1, sel), __byte_perm(r2, r3, sel), 0x5410);
    if (NBITS < 8)
        w = (w >> ((jc * NBITS) % 8)) & LANES;
    return w;
}

template <int NBITS>
__global__ void __launch_bounds__(256) unpack_bytes_kernel(const uint8_t *__restrict__ in,
                                                           int64_t spec_bytes, int nchan,
                                                           int64_t nsamp, uint8_t *__restrict__ out,
                                                           int64_t out_pitch, int64_t ntile_t) {
    constexpr int kTileT = tile_t(NBITS);
    constexpr int SEG = kTileC * NBITS / 8;  // bytes of one spectrum in a full tile
    constexpr int STRIDE = SEG + 4;          // shared row: an odd number of 4-byte words
    __shared__ __align__(16) uint8_t tile[kTileT * STRIDE];

    const int c0 = blockIdx.x * kTileC;
    const int64_t cb0 = (int64_t)c0 * NBITS / 8;  // first byte of the tile in a spectrum
    const int seg = spec_bytes - cb0 < SEG ? (int)(spec_bytes - cb0) : SEG;
    const int nc = nchan - c0 < kTileC ? nchan - c0 : kTileC;
    for (int64_t tt = blockIdx.y; tt < ntile_t; tt += gridDim.y) {
        const int64_t t0 = tt * kTileT;
        const int64_t left = nsamp - t0;
        const int rows = left < kTileT ? (int)left : kTileT;
        __syncthreads();  // the previous tile has been read
        for (int i = threadIdx.x; i < rows * seg; i += blockDim.x) {
            const int r = i / seg, b = i % seg;
            tile[r * STRIDE + b] = in[(t0 + r) * spec_bytes + cb0 + b];
        }
        __syncthreads();
        // An item is (word q: spectra 4q..4q+3, column word cw: the 32/NBITS
        // channels held in bytes 4cw..4cw+3 of a row).  Lane l takes
        // q = 8*qg + l/4 and cw = 4*cg + l%4, so the 4 rows a warp reads per
        // step fall in 32 different banks and each channel's 8 output words
        // fill one 32-byte sector.  Channel j of the column word comes from
        // byte (j*NBITS)/8 of each of the 4 rows.
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
                const uint32_t w = turn_word<NBITS>(r0, r1, r2, r3, jc);
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

// Tiled kernel (see the top of the file).  TT spectra per time tile, NBUF
// tile buffers in the input ring, NT threads.
template <int NBITS, int TT, int NBUF, int NT>
__global__ void __launch_bounds__(NT) unpack_tiled_kernel(const uint8_t *__restrict__ in,
                                                           int64_t spec_bytes, int64_t nsamp,
                                                           uint8_t *__restrict__ out,
                                                           int64_t out_pitch, int64_t ntile_t) {
    constexpr int SEG = kTileC * NBITS / 8;        // input bytes of a tile row
    constexpr int P = SEG + 16;                    // input row pitch
    constexpr int BUF = TT * P + (TT / 4) * 16;    // one ring buffer
    constexpr int PO = TT + 16;                    // transposed-tile row pitch
    constexpr int CH = SEG / 16;                   // 16-byte copies per row
    constexpr int S = NBITS == 8 ? 2 : NBITS == 4 ? 3 : NBITS == 2 ? 4 : 5;  // log2(32/NBITS)
    static_assert(TT % 128 == 0, "the word swizzle flips bits 3-4 of a row's word index");
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *turned = smem + NBUF * BUF;
    const int c0 = blockIdx.x * kTileC;
    const int64_t cb0 = (int64_t)c0 * NBITS / 8;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    // f(c): the 4 column words of a warp step hold channels whose rows start
    // 16*cw (8-bit) or 0 (narrower) banks apart; XOR-ing word q with 8 f(c)
    // moves them to 4 distinct groups of 8 banks.
    auto swz = [](int c) {
        const int cw = c >> S;
        return S == 2 ? ((cw >> 1) & 1) : (cw & 3);
    };
    auto rows_of = [&](int64_t tt) {
        const int64_t left = nsamp - tt * TT;
        return left < TT ? (int)left : TT;
    };
    // Copies of time tile tt into buffer b; every thread commits one group
    // per call, also when it has nothing to copy, so group counts agree.
    auto issue = [&](int64_t tt, int b) {
        if (tt < ntile_t) {
            const int rows = rows_of(tt);
            const int64_t t0 = tt * TT;
            for (int i = threadIdx.x; i < rows * CH; i += NT) {
                const int r = i / CH, j = i % CH;
                const uint8_t *src = in + (t0 + r) * spec_bytes + cb0 + 16 * j;
                const uint32_t dst = sbase + (uint32_t)(b * BUF + r * P + (r >> 2) * 16 + 16 * j);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int64_t kstep = gridDim.y;
#pragma unroll
    for (int s = 0; s < NBUF - 1; ++s)
        issue(blockIdx.y + s * kstep, s);
    int b = 0;  // buffer of the current tile
    for (int64_t tt = blockIdx.y; tt < ntile_t; tt += kstep) {
        // The buffer of tile tt + (NBUF-1)*kstep was last read one tile ago.
        issue(tt + (NBUF - 1) * kstep, b == 0 ? NBUF - 1 : b - 1);
        asm volatile("cp.async.wait_group %0;" ::"n"(NBUF - 1) : "memory");
        __syncthreads();  // every thread's copies of tile tt have landed
        const uint8_t *tile = smem + b * BUF;
        const int64_t t0 = tt * TT;
        // Corner turn into the transposed tile (rows past the tile's last
        // spectrum hold stale bytes that no store below reaches).
        const int lq = (threadIdx.x & 31) >> 2, lc = threadIdx.x & 3;
        constexpr int NCG = SEG / 16;
        for (int g = threadIdx.x >> 5; g < (TT / 32) * NCG; g += NT / 32) {
            const int q = 8 * (g / NCG) + lq;
            const int cw = 4 * (g % NCG) + lc;
            const uint32_t *rp =
                reinterpret_cast<const uint32_t *>(tile + 4 * q * P + q * 16) + cw;
            const uint32_t r0 = rp[0], r1 = rp[P / 4], r2 = rp[2 * (P / 4)], r3 = rp[3 * (P / 4)];
#pragma unroll
            for (int jc = 0; jc < 32 / NBITS; ++jc) {
                const int c = cw * (32 / NBITS) + jc;
                reinterpret_cast<uint32_t *>(turned + c * PO)[q ^ (8 * swz(c))] =
                    turn_word<NBITS>(r0, r1, r2, r3, jc);
            }
        }
        __syncthreads();
        // Rows out: CPR 16-byte chunks per row, 32 / CPR rows per warp step.
        constexpr int CPR = TT / 16;
        constexpr int RPW = 32 / CPR;
        const int k = (threadIdx.x & 31) % CPR;
        const int64_t t = t0 + 16 * k;
        for (int c = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / CPR; c < kTileC;
             c += (NT / 32) * RPW) {
            const uint4 v = *reinterpret_cast<const uint4 *>(turned + c * PO + 16 * (k ^ (2 * swz(c))));
            uint8_t *d = out + (int64_t)(c0 + c) * out_pitch + t;
            if (t + 16 <= nsamp) {
                *reinterpret_cast<uint4 *>(d) = v;
            } else if (t < nsamp) {
                for (int e = 0; t + e < nsamp; ++e) {
                    const uint32_t w = e < 4 ? v.x : e < 8 ? v.y : e < 12 ? v.z : v.w;
                    d[e] = (uint8_t)(w >> (8 * (e & 3)));
                }
            }
        }
        __syncthreads();  // the transposed tile and buffer b are free again
        b = b + 1 == NBUF ? 0 : b + 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Tiled-kernel shape per field width: spectra per time tile, ring buffers,
// CTAs per SM, threads (measured best on an L-band block of 147628 spectra
// x 1024 channels: 8-bit 5.65 TB/s at (256, 3, 1, 512 threads), 5.31 with
// 256 threads; 4-bit 5.05 and 1-bit 4.62 TB/s at (256, 2, 2, 512)).
template <int NBITS> struct TiledShape {
    static constexpr int TT = 256;
    static constexpr int NBUF = NBITS == 8 ? 3 : 2;
    static constexpr int CTAS_PER_SM = NBITS == 8 ? 1 : 2;
    static constexpr int THREADS = 512;
    static constexpr int SMEM = NBUF * (TT * (kTileC * NBITS / 8 + 16) + (TT / 4) * 16) +
                                kTileC * (TT + 16);
};

template <int NBITS>
cudaError_t launch_unpack(const uint8_t *in, int64_t spec_bytes, int nchan, int64_t nsamp,
                          uint8_t *out, int64_t out_pitch, bool tiled, cudaStream_t s) {
    const int ntc = (nchan + kTileC - 1) / kTileC;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    if (tiled) {
        using T = TiledShape<NBITS>;
        auto k = unpack_tiled_kernel<NBITS, T::TT, T::NBUF, T::THREADS>;
        static bool configured[64] = {false};
        if (!configured[dev & 63]) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
            if (e != cudaSuccess)
                return e;
            configured[dev & 63] = true;
        }
        const int64_t ntt = (nsamp + T::TT - 1) / T::TT;
        const int64_t want = std::max<int64_t>(1, (int64_t)nsm * T::CTAS_PER_SM / ntc);
        const unsigned gy = (unsigned)std::min<int64_t>(std::min<int64_t>(ntt, want), 65535);
        k<<<dim3((unsigned)ntc, gy), T::THREADS, T::SMEM, s>>>(in, spec_bytes, nsamp, out,
                                                               out_pitch, ntt);
        return cudaGetLastError();
    }
    constexpr int kTileT = tile_t(NBITS);
    const int64_t ntt = (nsamp + kTileT - 1) / kTileT;
    // about 8 resident CTAs per SM in total
    const int64_t want = std::max<int64_t>(1, (int64_t)nsm * 8 / ntc);
    const unsigned gy = (unsigned)std::min<int64_t>(std::min<int64_t>(ntt, want), 65535);
    unpack_bytes_kernel<NBITS><<<dim3((unsigned)ntc, gy), 256, 0, s>>>(in, spec_bytes, nchan, nsamp,
                                                                       out, out_pitch, ntt);
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
    // The tiled kernel's 16-byte copies need every spectrum and every channel
    // tile on 16 bytes, and whole tiles across the spectrum.
    const bool vec = ((uintptr_t)in & 15u) == 0 && spec_bytes % 16 == 0 &&
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
