/*
 * Seeded synthetic UTF-16 workloads.
 *
 * This module only draws input strings; it holds none of the repair or
 * validation arithmetic.  Both the CUDA path and the CPU oracle are fed from
 * these buffers, so it must not know which units are "bad".
 *
 * Random numbers come from xoshiro256** (Blackman and Vigna, "Scrambled
 * linear pseudorandom number generators", 2018), seeded through SplitMix64
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * 2014), both written here from their published definitions.  All integer
 * arithmetic is exact and identical on x86-64 and AArch64; the only libm use
 * is the log-normal length draw (log, sqrt, cos, exp).
 *
 * Unit categories follow the paper's generator description (Section 4: a
 * share of characters are valid surrogate pairs, a share of the remaining
 * units are lone surrogates, half high and half low) with the mix fixed by
 * the workloads this library is measured on:
 *   ASCII 0x20-0x7E, BMP non-surrogate (0x0080-0xD7FF or 0xE000-0xFFFF),
 *   valid pair (high 0xD800-0xDBFF then low 0xDC00-0xDFFF), lone surrogate.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    uint64_t s[4];
} wl_rng;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void rng_seed(wl_rng *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(wl_rng *r) {
    uint64_t *s = r->s;
    const uint64_t result = rotl64(s[1] * 5u, 7) * 9u;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* Uniform integer in [0, m) from the top 32 bits (multiply-shift; the bias is
 * below 2^-32 relative and irrelevant for workload shaping). */
static inline uint32_t rng_below(wl_rng *r, uint32_t m) {
    return (uint32_t)(((rng_next(r) >> 32) * (uint64_t)m) >> 32);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double rng_unit(wl_rng *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

#define BMP_LOW_COUNT 55168u  /* 0x0080 .. 0xD7FF */
#define BMP_HIGH_COUNT 8192u  /* 0xE000 .. 0xFFFF */

static inline uint16_t draw_ascii(wl_rng *r) { return (uint16_t)(0x20u + rng_below(r, 95u)); }

static inline uint16_t draw_bmp(wl_rng *r) {
    uint32_t k = rng_below(r, BMP_LOW_COUNT + BMP_HIGH_COUNT);
    return (uint16_t)(k < BMP_LOW_COUNT ? 0x0080u + k : 0xE000u + (k - BMP_LOW_COUNT));
}

static inline uint16_t draw_high(wl_rng *r) { return (uint16_t)(0xD800u + rng_below(r, 1024u)); }
static inline uint16_t draw_low(wl_rng *r) { return (uint16_t)(0xDC00u + rng_below(r, 1024u)); }

/* Category thresholds on a 32-bit uniform draw, in the order
 * lone | ascii | bmp | pair.  The non-lone shares keep the ratio 70:20:8. */
typedef struct {
    uint64_t lone, ascii, bmp; /* cumulative upper bounds; pair takes the rest */
} mix_thresholds;

static mix_thresholds make_thresholds(double lone_rate, double ascii_w, double bmp_w, double pair_w) {
    const double total = 4294967296.0;
    double rest = 1.0 - lone_rate;
    double wsum = ascii_w + bmp_w + pair_w;
    mix_thresholds t;
    t.lone = (uint64_t)(lone_rate * total);
    t.ascii = t.lone + (uint64_t)(rest * ascii_w / wsum * total);
    t.bmp = t.ascii + (uint64_t)(rest * bmp_w / wsum * total);
    return t;
}

/* Fill out[0..n) with the mix; returns nothing.  A pair drawn with only one
 * position left is replaced by an ASCII (7/9) or BMP (2/9) unit so the length
 * is exact. */
static void fill_mix_rng(uint16_t *out, int64_t n, wl_rng *r, mix_thresholds t) {
    int64_t i = 0;
    while (i < n) {
        uint64_t c = rng_next(r) >> 32;
        if (c < t.lone) {
            out[i++] = (rng_next(r) >> 63) ? draw_low(r) : draw_high(r);
        } else if (c < t.ascii) {
            out[i++] = draw_ascii(r);
        } else if (c < t.bmp) {
            out[i++] = draw_bmp(r);
        } else if (i + 1 < n) {
            out[i++] = draw_high(r);
            out[i++] = draw_low(r);
        } else {
            out[i++] = rng_below(r, 9u) < 7u ? draw_ascii(r) : draw_bmp(r);
        }
    }
}

/* Mixed text: 70% ASCII, 20% BMP non-surrogate, 8% valid pair, scaled by
 * (1 - lone_rate), plus lone surrogates at lone_rate per position. */
void wl_fill_mix(uint16_t *out, int64_t n, uint64_t seed, double lone_rate) {
    wl_rng r;
    rng_seed(&r, seed);
    fill_mix_rng(out, n, &r, make_thresholds(lone_rate, 70.0, 20.0, 8.0));
}

/* The paper's generator shape (Section 4): pair_rate of the characters are
 * valid pairs, lone_rate of the other units are lone surrogates (half high,
 * half low), and the remaining units are ASCII. */
void wl_fill_paper(uint16_t *out, int64_t n, uint64_t seed, double pair_rate, double lone_rate) {
    wl_rng r;
    rng_seed(&r, seed);
    const double total = 4294967296.0;
    uint64_t t_pair = (uint64_t)(pair_rate * total);
    uint64_t t_lone = (uint64_t)(lone_rate * total);
    int64_t i = 0;
    while (i < n) {
        uint64_t c = rng_next(&r) >> 32;
        if (c < t_pair && i + 1 < n) {
            out[i++] = draw_high(&r);
            out[i++] = draw_low(&r);
            continue;
        }
        uint64_t d = rng_next(&r) >> 32;
        if (d < t_lone)
            out[i++] = (rng_next(&r) >> 63) ? draw_low(&r) : draw_high(&r);
        else
            out[i++] = draw_ascii(&r);
    }
}

/* Every unit uniform over the whole surrogate block 0xD800-0xDFFF. */
void wl_fill_uniform_surrogates(uint16_t *out, int64_t n, uint64_t seed) {
    wl_rng r;
    rng_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) out[i] = (uint16_t)(0xD800u + rng_below(&r, 2048u));
}

/* Alternating 0xD800, 0xDC00 with a one-unit phase shift every `period`
 * positions: unit i is 0xDC00 when (i + floor(i / period)) is odd. */
void wl_fill_shifted_alternating(uint16_t *out, int64_t n, int64_t period) {
    for (int64_t i = 0; i < n; ++i) out[i] = ((i + i / period) & 1) ? 0xDC00u : 0xD800u;
}

/* Log-normal lengths floor(exp(mu + sigma*z)), z standard normal by the
 * Box-Muller transform, clipped to [0, clip].  Returns the total. */
int64_t wl_lognormal_lengths(int64_t *len, int64_t count, uint64_t seed, double mu, double sigma,
                             int64_t clip) {
    wl_rng r;
    rng_seed(&r, seed);
    int64_t total = 0;
    for (int64_t s = 0; s < count; ++s) {
        double u1 = rng_unit(&r), u2 = rng_unit(&r);
        double z = sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586 * u2);
        double v = exp(mu + sigma * z);
        int64_t L = v >= (double)clip ? clip : (int64_t)floor(v);
        if (L < 0) L = 0;
        len[s] = L;
        total += L;
    }
    return total;
}

/* Serving request lengths: 80% uniform [16,256], 19% uniform [1024,65536],
 * 1% uniform [1048576,16777216].  Returns the total. */
int64_t wl_request_lengths(int64_t *len, int64_t count, uint64_t seed) {
    wl_rng r;
    rng_seed(&r, seed);
    int64_t total = 0;
    for (int64_t s = 0; s < count; ++s) {
        uint32_t c = rng_below(&r, 100u);
        int64_t L;
        if (c < 80u)
            L = 16 + (int64_t)rng_below(&r, 241u);
        else if (c < 99u)
            L = 1024 + (int64_t)rng_below(&r, 65536u - 1024u + 1u);
        else
            L = 1048576 + (int64_t)rng_below(&r, 16777216u - 1048576u + 1u);
        len[s] = L;
        total += L;
    }
    return total;
}

/* Ragged batch content: string s occupies [offsets[s], offsets[s+1]) and is
 * filled with the mix at lone_rate.  A share `forced` of the non-empty
 * strings is then made to start with a uniform low surrogate or (equally
 * often) end with a uniform high surrogate, so string ends are exercised. */
void wl_fill_ragged(uint16_t *out, const int64_t *offsets, int64_t count, uint64_t seed, double lone_rate,
                    double forced) {
    wl_rng r;
    rng_seed(&r, seed);
    mix_thresholds t = make_thresholds(lone_rate, 70.0, 20.0, 8.0);
    uint64_t t_forced = (uint64_t)(forced * 4294967296.0);
    for (int64_t s = 0; s < count; ++s) {
        int64_t a = offsets[s], b = offsets[s + 1];
        if (b <= a) continue;
        fill_mix_rng(out + a, b - a, &r, t);
        if ((rng_next(&r) >> 32) < t_forced) {
            if (rng_next(&r) >> 63)
                out[a] = draw_low(&r);
            else
                out[b - 1] = draw_high(&r);
        }
    }
}
