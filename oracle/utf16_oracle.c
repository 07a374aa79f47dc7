/*
 * CPU oracle for UTF-16 toWellFormed / isWellFormed.  TEST INFRASTRUCTURE.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this file's library.  The CUDA path never calls it, includes
 * nothing from it and shares no helper with it.
 *
 * Everything here is the plain definition written out as scalar loops:
 *
 *  - Section 1 of the paper: a high surrogate lies in 0xD800-0xDBFF, a low
 *    surrogate in 0xDC00-0xDFFF, and a supplementary code point is encoded as
 *    a high surrogate immediately followed by a low surrogate, decoding to
 *    ((h - 0xD800) << 10) + (l - 0xDC00) + 0x10000.
 *  - Section 1: a high surrogate not followed by a low one, or a low
 *    surrogate not preceded by a high one, is mismatched and is replaced by
 *    U+FFFD; every other unit is kept, so the length does not change.
 *  - Section 3.1 (last paragraph before the example): the units before the
 *    first and after the last are outside the string, so a string that starts
 *    with a low or ends with a high surrogate has that unit replaced.  In a
 *    batch every string is treated on its own; a neighbouring string's units
 *    are outside.
 *  - Section 3.1, second step: the flag illseq(i) = isHigh(in[i-1]) XOR
 *    isLow(in[i]) (the Fig. 3 column of that name), with in[-1] taken as
 *    U+0000 as in the example of Fig. 3.
 *
 * The first-error index (not defined by the paper) is the index of the first
 * unit that repair would replace, or n when there is none; in a batch it is
 * relative to the string's start and equals the length for a clean string.
 *
 * Parity status: pinned (exhaustive enumeration against an independent
 * brute-force matcher, the Fig. 3 worked example, the Section 1 code-point
 * example, closed forms of the adversarial strings and invariants).
 */
#include <stdint.h>

static int is_high(uint16_t u) { return u >= 0xD800 && u <= 0xDBFF; }
static int is_low(uint16_t u) { return u >= 0xDC00 && u <= 0xDFFF; }

/* 1 when in[i] is a mismatched surrogate of the string in[0..n). */
int oracle_unit_is_bad(const uint16_t *in, int64_t n, int64_t i) {
    if (is_high(in[i])) {
        int followed_by_low = (i + 1 < n) && is_low(in[i + 1]);
        return !followed_by_low;
    }
    if (is_low(in[i])) {
        int preceded_by_high = (i > 0) && is_high(in[i - 1]);
        return !preceded_by_high;
    }
    return 0;
}

/* out[i] for i in [lo, hi) of the string in[0..n); out is indexed like in. */
void oracle_to_well_formed_range(const uint16_t *in, int64_t n, int64_t lo, int64_t hi, uint16_t *out) {
    for (int64_t i = lo; i < hi; ++i) out[i] = oracle_unit_is_bad(in, n, i) ? 0xFFFD : in[i];
}

void oracle_to_well_formed(const uint16_t *in, int64_t n, uint16_t *out) {
    oracle_to_well_formed_range(in, n, 0, n, out);
}

/* Index of the first unit that repair replaces, or n. */
int64_t oracle_first_bad(const uint16_t *in, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (oracle_unit_is_bad(in, n, i)) return i;
    return n;
}

/* First-error index restricted to [lo, hi) of the string in[0..n): the first
 * bad i in that range, or hi. */
int64_t oracle_first_bad_range(const uint16_t *in, int64_t n, int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
        if (oracle_unit_is_bad(in, n, i)) return i;
    return hi;
}

/* Batch: string s is in[offsets[s] .. offsets[s+1]).  out is indexed like in;
 * units outside [offsets[0], offsets[count]) are not written. */
void oracle_to_well_formed_batch(const uint16_t *in, const int64_t *offsets, int64_t count, uint16_t *out) {
    for (int64_t s = 0; s < count; ++s) {
        int64_t a = offsets[s], b = offsets[s + 1];
        oracle_to_well_formed(in + a, b - a, out + a);
    }
}

/* Batch first-error index, relative to each string's start (length if clean). */
void oracle_first_bad_batch(const uint16_t *in, const int64_t *offsets, int64_t count, int64_t *first_bad) {
    for (int64_t s = 0; s < count; ++s) {
        int64_t a = offsets[s], b = offsets[s + 1];
        first_bad[s] = oracle_first_bad(in + a, b - a);
    }
}

/* Section 3.1 step two: illseq(i) = isHigh(in[i-1]) XOR isLow(in[i]). */
void oracle_illseq(const uint16_t *in, int64_t n, uint8_t *flags) {
    for (int64_t i = 0; i < n; ++i) {
        uint16_t lookback = i > 0 ? in[i - 1] : 0x0000;
        flags[i] = (uint8_t)(is_high(lookback) ^ is_low(in[i]));
    }
}

/* Section 1: the code point of the surrogate pair (h, l). */
uint32_t oracle_code_point(uint16_t h, uint16_t l) {
    return (((uint32_t)h - 0xD800u) << 10) + ((uint32_t)l - 0xDC00u) + 0x10000u;
}
