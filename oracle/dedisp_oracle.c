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
