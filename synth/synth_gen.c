/*
 * Seeded synthetic input generator (counter-based splitmix64).
 *
 * This file holds no arithmetic of the radiative-transfer method: it only
 * turns (seed, stream, counter) into uniform numbers and lays out a synthetic
 * correlated-k table of the shape the paper describes in Sect. 2.3 (a 4-D
 * table over log P, T, wavelength bin and Gauss point, monotone in g).
 *
 * Generator: the splitmix64 output function applied to key + (i+1)*golden,
 * u = (z >> 11) * 2^-53.  Integer-only, so Python (numpy) and C agree bit for
 * bit; synth/__init__.py carries the same definition for scalar draws and a
 * test checks the two against each other.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t synth_stream_key(uint64_t seed, uint64_t stream)
{
    return mix64(seed ^ (stream * GOLDEN));
}

double synth_uniform(uint64_t key, uint64_t i)
{
    return (double)(mix64(key + (i + 1) * GOLDEN) >> 11) * 0x1.0p-53;
}

void synth_uniform_fill(uint64_t key, uint64_t first, int64_t count, double* out)
{
    for (int64_t i = 0; i < count; ++i) out[i] = synth_uniform(key, first + (uint64_t)i);
}

/*
 * k-table [nP][nT][L][G]: for each (iP, iT, l) row draw G uniforms
 * u = synth_uniform(key, ((iP*nT + iT)*L + l)*G + g), sort them ascending over
 * g, map log10(kappa) = lo + (hi - lo) * u and kappa = 10^log10(kappa).
 * Writes float64 to out64 and/or float32 (rounded from the float64 value) to
 * out32; either pointer may be NULL.
 */
void synth_ktable(uint64_t key, int nP, int nT, int L, int G, double lo, double hi,
                  double* out64, float* out32)
{
    const int64_t rows = (int64_t)nP * nT * L;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < rows; ++r) {
        double u[64];
        const int gg = G < 64 ? G : 64;
        for (int g = 0; g < gg; ++g) u[g] = synth_uniform(key, (uint64_t)(r * G + g));
        /* insertion sort, ascending */
        for (int a = 1; a < gg; ++a) {
            double v = u[a];
            int b = a - 1;
            while (b >= 0 && u[b] > v) { u[b + 1] = u[b]; --b; }
            u[b + 1] = v;
        }
        for (int g = 0; g < gg; ++g) {
            double k = pow(10.0, lo + (hi - lo) * u[g]);
            if (out64) out64[r * G + g] = k;
            if (out32) out32[r * G + g] = (float)k;
        }
    }
}
