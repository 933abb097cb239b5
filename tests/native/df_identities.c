/* Exhaustive host check of the exact FP32 identities the double-float generator relies on to
 * skip integer conversions and instructions (phsp_df.cuh, phsp_device.cuh).  Plain C with IEEE
 * single precision, round to nearest, no contraction: the arithmetic of the device code.
 *
 *   1. f32_to_f64_bits_fast: the FP64 high word of an FP32 bit pattern b as
 *      xs + (xs & 0x90000000) + 0x38000000 with xs = b >> 3 (arithmetic) equals the masked form
 *      (((b & 0x7FFFFFFF) >> 3) + 0x38000000) | (b & 0x80000000), for all 2^32 patterns.
 *   2. df_direction: with a = x & ~0xFF and b = (x & 0xFF) + 1/2 as FP32 numbers,
 *      (2^32 - 256) - a, 256 - b and a - 2^31 are exact and equal the conversions of
 *      ~x & ~0xFF, (~x & 0xFF) + 1/2 and (x - 2^31) & ~0xFF, for all 2^32 draws x.
 *   3. The mass gaps: for sorted draws y0 <= y1, FastTwoSum(a1 - a0, b1 - b0) gives the same
 *      pair as FastTwoSum of the converted parts of d = y1 - y0, and the pair sums to d exactly
 *      (all 65536 low-byte pairs against 2048 high parts, and 2^26 random pairs).
 * Prints the number of mismatches of each check and returns nonzero if any check fails. */
#include <stdint.h>
#include <stdio.h>

static void fast_two_sum(float a, float b, float *s, float *e) {
    volatile float sv = a + b;
    volatile float t = sv - a;
    *s = sv;
    *e = b - t;
}

static uint64_t splitmix(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t check_gap(uint32_t y0, uint32_t y1) {
    if (y1 < y0) { uint32_t t = y0; y0 = y1; y1 = t; }
    const float a0 = (float)(y0 & 0xFFFFFF00u), b0 = (float)(y0 & 0xFFu) + 0.5f;
    const float a1 = (float)(y1 & 0xFFFFFF00u), b1 = (float)(y1 & 0xFFu) + 0.5f;
    float s1, e1, s2, e2;
    fast_two_sum(a1 - a0, b1 - b0, &s1, &e1);
    const uint32_t d = y1 - y0;
    fast_two_sum((float)(d & 0xFFFFFF00u), (float)(d & 0xFFu), &s2, &e2);
    const int same = s1 == s2 && e1 == e2 && (double)s1 + (double)e1 == (double)d;
    return same ? 0u : 1u;
}

int main(void) {
    uint64_t bad_word = 0, bad_dir = 0, bad_gap = 0;
    for (uint64_t i = 0; i < (1ull << 32); ++i) {
        const uint32_t v = (uint32_t)i;
        const uint32_t masked = (((v & 0x7FFFFFFFu) >> 3) + 0x38000000u) | (v & 0x80000000u);
        const uint32_t xs = (uint32_t)((int32_t)v >> 3);
        if (xs + (xs & 0x90000000u) + 0x38000000u != masked) ++bad_word;

        const float a = (float)(v & 0xFFFFFF00u), b = (float)(v & 0xFFu) + 0.5f;
        const uint32_t nv = ~v;
        const int32_t c = (int32_t)((v ^ 0x80000000u) & 0xFFFFFF00u);
        if (4294967040.0f - a != (float)(nv & 0xFFFFFF00u) || 256.0f - b != (float)(nv & 0xFFu) + 0.5f ||
            a - 2147483648.0f != (float)c)
            ++bad_dir;
    }
    uint64_t st = 20171115u;
    for (int h = 0; h < 2048; ++h) {
        const uint32_t hi0 = (uint32_t)splitmix(&st) & 0xFFFFFF00u;
        const uint32_t hi1 = (h & 1) ? hi0 : ((uint32_t)splitmix(&st) & 0xFFFFFF00u);
        for (uint32_t l0 = 0; l0 < 256; ++l0)
            for (uint32_t l1 = 0; l1 < 256; ++l1) bad_gap += check_gap(hi0 | l0, hi1 | l1);
    }
    for (int r = 0; r < (1 << 26); ++r) {
        const uint32_t y0 = (uint32_t)splitmix(&st);
        const uint32_t y1 = (r & 1) ? y0 + (uint32_t)(splitmix(&st) & 0xFFFFu) : (uint32_t)splitmix(&st);
        bad_gap += check_gap(y0, y1 < y0 && (r & 1) ? y0 : y1);
    }
    printf("high word %llu, direction parts %llu, gaps %llu\n", (unsigned long long)bad_word,
           (unsigned long long)bad_dir, (unsigned long long)bad_gap);
    return (bad_word || bad_dir || bad_gap) ? 1 : 0;
}
