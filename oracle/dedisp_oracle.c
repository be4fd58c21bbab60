/*
 * Brute-force incoherent de-dispersion: the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library, and the library never
 * calls it.
 *
 * What is computed (Sec. 2 of the ARTEMIS paper): every frequency channel of
 * an (f,t) power array is shifted by the delay that the cold-plasma
 * dispersion law gives for one trial DM, and the shifted channels are summed
 * over frequency.  Doing this for every trial DM of a blind search gives the
 * (DM,t) plane:
 *
 *     out[d][t] = sum_{c=0}^{nchan-1} in[c][t + s(c,d)]
 *
 * The paper names the cold-plasma law (delay growing as f^-2) without
 * writing it out; the integer shift rule used here is the textbook delay
 *     dt(f) = 4148.808 s * DM * (f^-2 - f_top^-2),   f in MHz,
 * expressed in samples, evaluated in FP64 and rounded once to FP32 per
 * channel ("dmshift"), then s(c,d) = trunc(float(DM_d) * dmshift[c]) with a
 * single FP32 multiply.  f_top is the highest channel-centre frequency.
 *
 * Accumulation: uint8 input is summed in FP32 (every partial sum is an
 * integer below 2^24, so the result is exact whatever the order); FP16 and
 * FP32 input is summed in FP64 and returned in FP64.
 *
 * Build this file with -ffp-contract=off: a fused multiply-add in the channel
 * frequency or the delay expression changes the FP32 table.
 * When built with -fopenmp (the "checker" build) the DM loop runs in
 * parallel; every (d,t) sum is independent, so the results are identical.
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>
#include <stdlib.h>

#define ORACLE_KDM 4148.808 /* dispersion constant, s MHz^2 pc^-1 cm^3 */

/* Highest channel-centre frequency of the band (Sec. 2: delays are relative
 * to the top of the band, where the pulse arrives first). */
static double top_frequency(int nchan, double fch1, double foff)
{
    if (foff < 0.0)
        return fch1;
    return fch1 + (double)(nchan - 1) * foff;
}

/* dmshift[c]: delay of channel c relative to f_top for DM = 1, in samples,
 * computed in FP64 and rounded once to FP32. */
int oracle_dmshift(int nchan, double fch1, double foff, double tsamp, float *dmshift)
{
    if (nchan < 1 || !(tsamp > 0.0) || foff == 0.0)
        return -1;
    double ftop = top_frequency(nchan, fch1, foff);
    if (!(ftop > 0.0))
        return -1;
    double inv_top = 1.0 / (ftop * ftop);
    for (int c = 0; c < nchan; ++c) {
        double f = fch1 + (double)c * foff;
        if (!(f > 0.0))
            return -1;
        double inv = 1.0 / (f * f);
        double delay_samples = ORACLE_KDM * (inv - inv_top) / tsamp;
        dmshift[c] = (float)delay_samples;
    }
    return 0;
}

/* s(c,d): one FP32 multiply (round to nearest even), then truncation. */
int oracle_shift(float dm, float dmshift)
{
    float product = dm * dmshift;
    return (int)product;
}

/* maxshift S = max over all (c,d) of s(c,d). */
int64_t oracle_maxshift(int nchan, const float *dmshift, int ndm, const float *dm)
{
    int64_t best = 0;
    for (int d = 0; d < ndm; ++d)
        for (int c = 0; c < nchan; ++c) {
            int s = oracle_shift(dm[d], dmshift[c]);
            if (s > best)
                best = s;
        }
    return best;
}

/* Full (DM,t) plane, uint8 input, FP32 output.
 * in:  nchan rows of in_pitch bytes; row c holds channel c (c = 0 is fch1).
 * out: ndm rows of out_pitch floats; row d holds trial DM dm[d].
 * The caller guarantees every row holds nsamp_out + maxshift samples. */
void oracle_dedisperse_u8(const uint8_t *in, int nchan, int64_t in_pitch,
                          const float *dmshift, const float *dm, int ndm,
                          int64_t nsamp_out, float *out, int64_t out_pitch)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < ndm; ++d) {
        int *s = (int *)malloc(sizeof(int) * (size_t)nchan);
        for (int c = 0; c < nchan; ++c)
            s[c] = oracle_shift(dm[d], dmshift[c]);
        for (int64_t t = 0; t < nsamp_out; ++t) {
            float acc = 0.0f;
            for (int c = 0; c < nchan; ++c)
                acc += (float)in[(int64_t)c * in_pitch + t + s[c]];
            out[(int64_t)d * out_pitch + t] = acc;
        }
        free(s);
    }
}

/* IEEE 754 binary16 -> double, from the bit fields. */
double oracle_half_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int expo = (h >> 10) & 0x1f;
    int mant = h & 0x3ff;
    double v;
    if (expo == 0)
        v = ldexp((double)mant, -24);                 /* zero / subnormal */
    else if (expo == 31)
        v = mant ? NAN : INFINITY;
    else
        v = ldexp((double)(1024 + mant), expo - 25);  /* 1.mant * 2^(e-15) */
    return sign ? -v : v;
}

/* FP16 (bit patterns) or FP32 input, FP64 accumulation and FP64 output.
 * abssum (may be NULL) receives sum_c |in[c][t+s(c,d)]| for each cell, the
 * scale of the FP16/FP32 error bound.
 * elem: 2 for FP16 (uint16 bit patterns), 4 for FP32. in_pitch in elements. */
void oracle_dedisperse_float(const void *in, int elem, int nchan, int64_t in_pitch,
                             const float *dmshift, const float *dm, int ndm,
                             int64_t nsamp_out, double *out, double *abssum,
                             int64_t out_pitch)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < ndm; ++d) {
        int *s = (int *)malloc(sizeof(int) * (size_t)nchan);
        for (int c = 0; c < nchan; ++c)
            s[c] = oracle_shift(dm[d], dmshift[c]);
        for (int64_t t = 0; t < nsamp_out; ++t) {
            double acc = 0.0, aacc = 0.0;
            for (int c = 0; c < nchan; ++c) {
                int64_t i = (int64_t)c * in_pitch + t + s[c];
                double v = elem == 2 ? oracle_half_to_double(((const uint16_t *)in)[i])
                                     : (double)((const float *)in)[i];
                acc += v;
                aacc += fabs(v);
            }
            out[(int64_t)d * out_pitch + t] = acc;
            if (abssum)
                abssum[(int64_t)d * out_pitch + t] = aacc;
        }
        free(s);
    }
}

/* Selected cells only (for full-size workloads): cell i is (d_idx[i], t_idx[i]).
 * elem 1 = uint8 (FP32 sum, returned widened to double), 2 = FP16, 4 = FP32. */
void oracle_dedisperse_cells(const void *in, int elem, int nchan, int64_t in_pitch,
                             const float *dmshift, const float *dm,
                             int64_t ncell, const int32_t *d_idx, const int64_t *t_idx,
                             double *out, double *abssum)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ncell; ++i) {
        int d = d_idx[i];
        int64_t t = t_idx[i];
        if (elem == 1) {
            float acc = 0.0f;
            for (int c = 0; c < nchan; ++c)
                acc += (float)((const uint8_t *)in)[(int64_t)c * in_pitch + t +
                                                    oracle_shift(dm[d], dmshift[c])];
            out[i] = acc;
            if (abssum)
                abssum[i] = acc;
        } else {
            double acc = 0.0, aacc = 0.0;
            for (int c = 0; c < nchan; ++c) {
                int64_t j = (int64_t)c * in_pitch + t + oracle_shift(dm[d], dmshift[c]);
                double v = elem == 2 ? oracle_half_to_double(((const uint16_t *)in)[j])
                                     : (double)((const float *)in)[j];
                acc += v;
                aacc += fabs(v);
            }
            out[i] = acc;
            if (abssum)
                abssum[i] = aacc;
        }
    }
}

/*
 * Input side: corner turn and bit unpacking.  The paper's test data are
 * sigproc filterbanks (Sec. 2, Fig. 1).  A filterbank block in that layout
 * stores nsamp spectra one after another, each holding nchan samples of
 * nbits bits (1, 2, 4 or 8).  Samples
 * are packed in time-then-channel order, filling each byte from its lowest
 * bits: channel c of spectrum t occupies bits (t*nchan + c)*nbits onwards,
 * where bit b is bit (b mod 8) of byte b/8.  nchan*nbits is a multiple of 8,
 * so every spectrum starts on a byte.  The de-dispersion reads channel rows,
 * so the block is turned into out[c][t]; sample values are kept as they are
 * (0 .. 2^nbits - 1).
 */
void oracle_unpack(const uint8_t *in, int nbits, int nchan, int64_t nsamp, uint8_t *out,
                   int64_t out_pitch)
{
    const unsigned mask = (1u << nbits) - 1u;
    for (int64_t t = 0; t < nsamp; ++t)
        for (int c = 0; c < nchan; ++c) {
            const int64_t bit = (t * nchan + c) * (int64_t)nbits;
            out[(int64_t)c * out_pitch + t] = (uint8_t)((in[bit / 8] >> (bit % 8)) & mask);
        }
}

/*
 * Detection on the (DM,t) plane.  Sec. 4 and Fig. 3 of the paper search the
 * plane for a simulated pulse and recover it at its DM and time; the paper
 * gives no detection formula.  Reading adopted here (matched boxcar filters
 * with a per-DM noise estimate):
 *
 *   for each DM row x[0..nsamp):
 *     mean = S1/n and std = sqrt(S2/n - mean^2) (0 if negative), n = nsamp,
 *       S1 = sum x, S2 = sum x^2;
 *     for each width w = 2^l, l = 0..nlevels-1, and t = 0..nsamp-w:
 *       B(t) = sum_{k<w} x[t+k];
 *     peak t = the first t with the largest B(t);
 *     snr = (B(peak) - w*mean) / (std*sqrt(w)), 0 if std == 0;
 *     if nsamp < w there is no window: t = -1, snr = -infinity.
 *
 * Sums over an integer-valued plane (integer_valued != 0; values in
 * [0, 2^21), nsamp <= 2^21) are exact: S1, S2 and B in 64-bit integers,
 * converted to FP64 once.  Otherwise S1, S2 and B are FP64 sums in index
 * order.  Every FP64 step is one IEEE operation (built without contraction).
 */
void oracle_detect(const double *plane, int ndm, int64_t pitch, int64_t nsamp, int nlevels,
                   int integer_valued, double *mean_out, double *std_out, double *snr_out,
                   int64_t *t_out)
{
    const double n = (double)nsamp;
    for (int d = 0; d < ndm; ++d) {
        const double *x = plane + (int64_t)d * pitch;
        double s1, s2;
        if (integer_valued) {
            uint64_t i1 = 0, i2 = 0;
            for (int64_t t = 0; t < nsamp; ++t) {
                const uint64_t v = (uint64_t)x[t];
                i1 += v;
                i2 += v * v;
            }
            s1 = (double)i1;
            s2 = (double)i2;
        } else {
            s1 = 0.0;
            s2 = 0.0;
            for (int64_t t = 0; t < nsamp; ++t) {
                s1 += x[t];
                s2 += x[t] * x[t];
            }
        }
        const double mean = s1 / n;
        double var = s2 / n - mean * mean;
        if (var < 0.0)
            var = 0.0;
        const double sd = sqrt(var);
        mean_out[d] = mean;
        std_out[d] = sd;
        for (int l = 0; l < nlevels; ++l) {
            const int64_t w = (int64_t)1 << l;
            int64_t best_t = -1;
            double best = 0.0;
            for (int64_t t = 0; t + w <= nsamp; ++t) {
                double b;
                if (integer_valued) {
                    uint64_t ib = 0;
                    for (int64_t k = 0; k < w; ++k)
                        ib += (uint64_t)x[t + k];
                    b = (double)ib;
                } else {
                    b = 0.0;
                    for (int64_t k = 0; k < w; ++k)
                        b += x[t + k];
                }
                if (best_t < 0 || b > best) {
                    best = b;
                    best_t = t;
                }
            }
            t_out[(int64_t)d * nlevels + l] = best_t;
            if (best_t < 0)
                snr_out[(int64_t)d * nlevels + l] = -INFINITY;
            else if (sd == 0.0)
                snr_out[(int64_t)d * nlevels + l] = 0.0;
            else
                snr_out[(int64_t)d * nlevels + l] =
                    (best - (double)w * mean) / (sd * sqrt((double)w));
        }
    }
}

/*
 * Front end: dual-polarisation voltages -> the uint8 filterbank the
 * de-dispersion reads.  The paper's pipeline generates Stokes parameters,
 * excises RFI and integrates before the dispersion search (Sec. 1); it gives
 * no formulas, so the steps are:
 *
 *   volts[c][i] = four int8 values (Xre, Xim, Yre, Yim) of raw sample i of
 *   channel c (rows of `pitch` bytes);
 *   Stokes I of a raw sample: Xre^2 + Xim^2 + Yre^2 + Yim^2;
 *   P[c][t] = sum of Stokes I over raw samples t*nint .. t*nint + nint - 1,
 *   t = 0 .. nsamp_raw/nint - 1 (an exact integer);
 *   RFI excision by iterated sigma clipping, per channel: the kept set starts
 *   as every t; each of niter passes takes, over the kept set, cnt, S1 = sum P
 *   and S2 = sum P^2 (exact), then mean = S1/cnt, std = sqrt(S2/cnt - mean^2)
 *   (0 if negative; both 0 if cnt == 0) and thr = floor(mean + k*std) (FP64,
 *   k = k_clip), and the next kept set is {t : P[t] <= thr};
 *   with the last pass's mean, std and thr: P > thr is replaced by the mean
 *   (code 128); otherwise m = (float)mean, s = (float)(16.0 / std),
 *   code = clamp(rint(128 + ((float)P - m) * s), 0, 255) in FP32, one IEEE
 *   operation at a time (round half to even); std == 0 gives 128 everywhere.
 *
 * Outputs the last pass's mean and std per channel (FP64) and out[c][t].
 */
void oracle_frontend(const int8_t *volts, int64_t pitch, int nchan, int64_t nsamp_raw, int nint,
                     double k_clip, int niter, uint8_t *out, int64_t out_pitch, double *mean_out,
                     double *std_out)
{
    const int64_t n = nsamp_raw / nint;
    int64_t *p = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int c = 0; c < nchan; ++c) {
        const int8_t *row = volts + (int64_t)c * pitch;
        for (int64_t t = 0; t < n; ++t) {
            int64_t acc = 0;
            for (int j = 0; j < nint; ++j) {
                const int8_t *v = row + 4 * (t * nint + j);
                acc += (int64_t)v[0] * v[0] + (int64_t)v[1] * v[1] + (int64_t)v[2] * v[2] +
                       (int64_t)v[3] * v[3];
            }
            p[t] = acc;
        }
        int64_t thr = INT64_MAX;
        double mean = 0.0, sd = 0.0;
        for (int it = 0; it < niter; ++it) {
            uint64_t cnt = 0, s1 = 0, s2 = 0;
            for (int64_t t = 0; t < n; ++t) {
                if (p[t] <= thr) {
                    cnt += 1;
                    s1 += (uint64_t)p[t];
                    s2 += (uint64_t)p[t] * (uint64_t)p[t];
                }
            }
            mean = 0.0;
            double var = 0.0;
            if (cnt > 0) {
                mean = (double)s1 / (double)cnt;
                var = (double)s2 / (double)cnt - mean * mean;
            }
            if (var < 0.0)
                var = 0.0;
            sd = sqrt(var);
            thr = (int64_t)floor(mean + k_clip * sd);
        }
        mean_out[c] = mean;
        std_out[c] = sd;
        const float m = (float)mean;
        const float s = sd > 0.0 ? (float)(16.0 / sd) : 0.0f;
        for (int64_t t = 0; t < n; ++t) {
            uint8_t code = 128;
            if (sd > 0.0 && p[t] <= thr) {
                const float d = (float)p[t] - m;
                const float v = rintf(128.0f + d * s);
                code = (uint8_t)(v < 0.0f ? 0.0f : (v > 255.0f ? 255.0f : v));
            }
            out[(int64_t)c * out_pitch + t] = code;
        }
    }
    free(p);
}

/*
 * Polyphase channeliser: subband voltages -> finer frequency channels.  The
 * paper's pipeline channelises the received subbands "in finer frequency"
 * before it generates Stokes parameters (Sec. 1) and names the poly-phase
 * filter (Sec. 5); it gives neither the filter nor the transform size, so the
 * textbook critically sampled polyphase filter bank is used (a window of
 * M*T samples weighted by a prototype low-pass filter, then an M-point DFT,
 * advancing by M samples per spectrum):
 *
 *   volts[s][j] = four int8 (Xre, Xim, Yre, Yim) of raw sample j of subband s
 *   (rows of `pitch` bytes); per polarisation x[j] = re + i*im;
 *   M channels per subband, T taps, prototype h[m], m < M*T;
 *   spectrum n, n = 0 .. floor(nraw/M) - T (none if floor(nraw/M) < T):
 *       y_k[n] = sum_{m=0}^{M*T-1} h[m] * x[n*M + m] * exp(-2 pi i k m / M)
 *   output channel c = (k + M/2) mod M of subband s (row s*M + c): the bins of
 *   a subband in increasing frequency, the most negative bin (k = M/2) first.
 *
 * The sum is evaluated as written, term by term in FP64, with the phase
 * exp(-2 pi i ((k*m) mod M) / M) taken from cos/sin in FP64.
 * oracle_pfb computes the spectra (sub[i], spec[i]) of a list and writes, per
 * listed spectrum, out[i][c][4] = (Xre, Xim, Yre, Yim) of every channel c.
 */
void oracle_pfb(const int8_t *volts, int64_t pitch, int64_t nraw, int M, int T, const double *h,
                int nsel, const int *sub, const int64_t *spec, double *out)
{
    const double twopi = 6.283185307179586476925286766559;
    double *cs = (double *)malloc(sizeof(double) * 2 * (size_t)M);
    for (int r = 0; r < M; ++r) {
        cs[2 * r] = cos(twopi * (double)r / (double)M);
        cs[2 * r + 1] = sin(twopi * (double)r / (double)M);
    }
    const int64_t L = (int64_t)M * T;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < nsel; ++i) {
        const int8_t *row = volts + (int64_t)sub[i] * pitch;
        const int64_t n = spec[i];
        for (int k = 0; k < M; ++k) {
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t m = 0; m < L; ++m) {
                const int8_t *v = row + 4 * (n * M + m);
                const int r = (int)(((int64_t)k * m) % M);
                const double c = cs[2 * r], sn = -cs[2 * r + 1]; /* exp(-i theta) */
                for (int pol = 0; pol < 2; ++pol) {
                    const double re = h[m] * (double)v[2 * pol];
                    const double im = h[m] * (double)v[2 * pol + 1];
                    acc[2 * pol] += re * c - im * sn;
                    acc[2 * pol + 1] += re * sn + im * c;
                }
            }
            const int ch = (k + M / 2) % M;
            for (int e = 0; e < 4; ++e)
                out[((int64_t)i * M + ch) * 4 + e] = acc[e];
        }
    }
    free(cs);
}

/*
 * Requantisation of channelised voltages to int8 (so that the front end can
 * read them): q = clamp(rint(v * scale), -127, 127), round half to even, in
 * FP64.  The clip is symmetric so that negating a voltage negates its code.
 */
void oracle_pfb_quantise(const double *v, int64_t n, double scale, int8_t *q)
{
    for (int64_t i = 0; i < n; ++i) {
        double u = rint(v[i] * scale);
        if (u > 127.0)
            u = 127.0;
        if (u < -127.0)
            u = -127.0;
        q[i] = (int8_t)u;
    }
}

/*
 * Prototype filter of the channeliser, FP64: a Hamming-windowed sinc whose
 * main lobe spans one channel (cutoff at half the channel spacing),
 *     h[m] = sinc((m - (L-1)/2) / M) * (0.54 - 0.46 cos(2 pi m / (L-1))),
 *     sinc(x) = sin(pi x) / (pi x), sinc(0) = 1, L = M*T (L > 1);
 * unnormalised (its centre is near 1, its sum near M).  The paper names no
 * filter; this is the common windowed-sinc design.
 */
int oracle_pfb_prototype(int M, int T, double *h)
{
    const int64_t L = (int64_t)M * T;
    if (M < 1 || T < 1 || L < 2)
        return -1;
    const double pi = 3.141592653589793238462643383280;
    for (int64_t m = 0; m < L; ++m) {
        const double x = ((double)m - (double)(L - 1) / 2.0) / (double)M;
        const double sinc = x == 0.0 ? 1.0 : sin(pi * x) / (pi * x);
        const double w = 0.54 - 0.46 * cos(2.0 * pi * (double)m / (double)(L - 1));
        h[m] = sinc * w;
    }
    return 0;
}
