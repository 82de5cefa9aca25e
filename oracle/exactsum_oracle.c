/*
 * exactsum_oracle.c -- plain, slow CPU exact sum.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library
 * is checked against.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load it.  It shares no code, header, table or helper with
 * the CUDA library, and the library never calls it.
 *
 * What it computes is the plain definition of the problem (Section 1, the
 * problem statement): S = x_1 + ... + x_n exactly, then one rounding of S to
 * the requested format.
 *
 *  - Representation: the dense fixed-point number of Section 2 (a sign and
 *    enough integer and fraction bits that every partial sum is exact),
 *    stored as one two's-complement integer in units of the input format's
 *    smallest subnormal, 32 bits per limb.  Each element is added into it
 *    one at a time with ordinary carry propagation.
 *  - Per-element decode (Section 1 / Section 2 number format): IEEE 754
 *    binary64, binary32 and bfloat16, subnormals included; the paper's own
 *    format formula has no subnormals and a garbled bias, so the IEEE
 *    definition is used.
 *  - Rounding (Section 3 step 7, Section 5 step 5): locate the most
 *    significant non-zero bit, keep the target precision, and round the
 *    dropped bits by the mode: to nearest with ties to even (always
 *    faithful in the sense of Section 1), toward zero, up or down.
 *  - NaN / infinity / signed-zero rules (the paper is silent):
 *      any NaN, or both +Inf and -Inf         -> quiet NaN (sign +)
 *      else any +Inf -> +Inf; else any -Inf   -> -Inf
 *      exact sum zero, n >= 1: every input -0 -> -0; every input +0 -> +0;
 *                              otherwise -0 under round-down, else +0
 *      n == 0                                 -> +0
 *    Overflow of the rounded finite sum follows IEEE 754 for each mode.
 *
 * Threads: the input is cut into contiguous pieces, one per thread; each
 * thread builds its own fixed-point sum and the pieces' sums are added at
 * the end (integer addition is associative, so this changes nothing).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_F64 = 0, OR_F32 = 1, OR_BF16 = 2 };
enum { OR_RNE = 0, OR_RTZ = 1, OR_RUP = 2, OR_RDOWN = 3 };

/* 96 limbs = 3072 bits: the largest term is below 2^2099 units (FP64), and
 * n < 2^63 terms add at most 63 more bits, plus a sign bit. */
#define OR_LIMBS 96

typedef struct {
    int frac_bits;  /* t: stored fraction bits */
    int exp_bits;   /* l: exponent bits */
    int bias;
    int unit_exp;   /* log2 of the smallest subnormal: 1 - bias - t */
    int width;      /* bytes per element */
} or_format;

static or_format or_fmt(int dtype) {
    or_format f;
    if (dtype == OR_F64) { f.frac_bits = 52; f.exp_bits = 11; f.bias = 1023; f.width = 8; }
    else if (dtype == OR_F32) { f.frac_bits = 23; f.exp_bits = 8; f.bias = 127; f.width = 4; }
    else { f.frac_bits = 7; f.exp_bits = 8; f.bias = 127; f.width = 2; }
    f.unit_exp = 1 - f.bias - f.frac_bits;
    return f;
}

typedef struct { uint32_t limb[OR_LIMBS]; } or_big; /* two's complement */

typedef struct {
    or_big sum;
    int has_nan, has_pinf, has_ninf;
    int all_pos_zero, all_neg_zero; /* vacuously true for no elements */
} or_partial;

static uint64_t or_load(const void* x, int64_t i, int width) {
    if (width == 8) { uint64_t v; memcpy(&v, (const char*)x + 8 * i, 8); return v; }
    if (width == 4) { uint32_t v; memcpy(&v, (const char*)x + 4 * i, 4); return v; }
    uint16_t v; memcpy(&v, (const char*)x + 2 * i, 2); return v;
}

/* sum += m * 2^p  (m < 2^64, p >= 0) */
static void or_add_shifted(or_big* a, uint64_t m, int p) {
    int limb = p / 32, off = p % 32;
    /* m << off spans at most three limbs */
    uint64_t lo = (m << off) & 0xffffffffu;
    uint64_t mid = (off == 0) ? (m >> 32) & 0xffffffffu : (m >> (32 - off)) & 0xffffffffu;
    uint64_t hi = (off == 0) ? 0 : (m >> (64 - off));
    uint64_t add[3] = {lo, mid, hi};
    uint64_t carry = 0;
    for (int k = limb; k < OR_LIMBS; k++) {
        uint64_t t = (uint64_t)a->limb[k] + carry + (k - limb < 3 ? add[k - limb] : 0);
        a->limb[k] = (uint32_t)t;
        carry = t >> 32;
        if (k - limb >= 2 && carry == 0) break;
    }
}

/* sum -= m * 2^p */
static void or_sub_shifted(or_big* a, uint64_t m, int p) {
    int limb = p / 32, off = p % 32;
    uint64_t lo = (m << off) & 0xffffffffu;
    uint64_t mid = (off == 0) ? (m >> 32) & 0xffffffffu : (m >> (32 - off)) & 0xffffffffu;
    uint64_t hi = (off == 0) ? 0 : (m >> (64 - off));
    uint64_t sub[3] = {lo, mid, hi};
    uint64_t borrow = 0;
    for (int k = limb; k < OR_LIMBS; k++) {
        uint64_t s = (k - limb < 3 ? sub[k - limb] : 0) + borrow;
        uint64_t cur = a->limb[k];
        a->limb[k] = (uint32_t)(cur - s);
        borrow = (cur < s) ? 1 : 0;
        if (k - limb >= 2 && borrow == 0) break;
    }
}

static void or_big_add(or_big* a, const or_big* b) {
    uint64_t carry = 0;
    for (int k = 0; k < OR_LIMBS; k++) {
        uint64_t t = (uint64_t)a->limb[k] + b->limb[k] + carry;
        a->limb[k] = (uint32_t)t;
        carry = t >> 32;
    }
}

static void or_partial_init(or_partial* s) {
    memset(s, 0, sizeof(*s));
    s->all_pos_zero = 1;
    s->all_neg_zero = 1;
}

/* Add elements [begin, end) of x into s, one by one. */
static void or_accumulate(or_partial* s, const void* x, int64_t begin, int64_t end, int dtype) {
    or_format f = or_fmt(dtype);
    const int sign_shift = 8 * f.width - 1;
    const uint64_t exp_all_ones = (1u << f.exp_bits) - 1;
    for (int64_t i = begin; i < end; i++) {
        uint64_t bits = or_load(x, i, f.width);
        int sign = (int)((bits >> sign_shift) & 1);
        uint64_t E = (bits >> f.frac_bits) & exp_all_ones;
        uint64_t F = bits & (((uint64_t)1 << f.frac_bits) - 1);
        uint64_t magnitude_bits = bits & ~((uint64_t)1 << sign_shift);
        if (!(sign == 0 && magnitude_bits == 0)) s->all_pos_zero = 0;
        if (!(sign == 1 && magnitude_bits == 0)) s->all_neg_zero = 0;
        if (E == exp_all_ones) {
            if (F != 0) s->has_nan = 1;
            else if (sign) s->has_ninf = 1;
            else s->has_pinf = 1;
            continue;
        }
        /* x = (-1)^sign * m * 2^p * 2^unit_exp */
        uint64_t m = (E == 0) ? F : (F | ((uint64_t)1 << f.frac_bits));
        int p = (E == 0) ? 0 : (int)E - 1;
        if (m == 0) continue;
        if (sign) or_sub_shifted(&s->sum, m, p);
        else or_add_shifted(&s->sum, m, p);
    }
}

typedef struct {
    const void* x;
    int64_t begin, end;
    int dtype;
    or_partial part;
} or_job;

static void* or_worker(void* arg) {
    or_job* j = (or_job*)arg;
    or_partial_init(&j->part);
    or_accumulate(&j->part, j->x, j->begin, j->end, j->dtype);
    return NULL;
}

/* ---- rounding of the exact integer ---- */

static int or_is_negative(const or_big* a) { return (a->limb[OR_LIMBS - 1] >> 31) & 1; }

static void or_negate(or_big* a) {
    uint64_t carry = 1;
    for (int k = 0; k < OR_LIMBS; k++) {
        uint64_t t = (uint64_t)(uint32_t)~a->limb[k] + carry;
        a->limb[k] = (uint32_t)t;
        carry = t >> 32;
    }
}

static int or_bit(const or_big* a, int i) {
    if (i < 0 || i >= 32 * OR_LIMBS) return 0;
    return (a->limb[i / 32] >> (i % 32)) & 1;
}

/* number of significant bits of a non-negative big integer (0 for zero) */
static int or_bitlen(const or_big* a) {
    for (int k = OR_LIMBS - 1; k >= 0; k--) {
        if (a->limb[k]) {
            int b = 31;
            while (!((a->limb[k] >> b) & 1)) b--;
            return 32 * k + b + 1;
        }
    }
    return 0;
}

/* bits [lo, lo + count) of a as an integer, count <= 64 */
static uint64_t or_bits(const or_big* a, int lo, int count) {
    uint64_t v = 0;
    for (int i = count - 1; i >= 0; i--) v = (v << 1) | (uint64_t)or_bit(a, lo + i);
    return v;
}

static int or_any_below(const or_big* a, int i) {
    for (int k = 0; k < i; k++)
        if (or_bit(a, k)) return 1;
    return 0;
}

static uint64_t or_encode(int out, int sign, uint64_t biased_exp, uint64_t frac) {
    or_format f = or_fmt(out);
    return ((uint64_t)sign << (8 * f.width - 1)) | (biased_exp << f.frac_bits) | frac;
}

static uint64_t or_inf(int out, int sign) {
    or_format f = or_fmt(out);
    return or_encode(out, sign, ((uint64_t)1 << f.exp_bits) - 1, 0);
}

static uint64_t or_max_finite(int out, int sign) {
    or_format f = or_fmt(out);
    return or_encode(out, sign, ((uint64_t)1 << f.exp_bits) - 2, ((uint64_t)1 << f.frac_bits) - 1);
}

static uint64_t or_quiet_nan(int out) {
    or_format f = or_fmt(out);
    return or_encode(out, 0, ((uint64_t)1 << f.exp_bits) - 1, (uint64_t)1 << (f.frac_bits - 1));
}

/* Round (-1)^sign * M * 2^unit_exp into format `out` under `mode`. */
static uint64_t or_round(const or_big* M, int sign, int unit_exp, int out, int mode) {
    or_format f = or_fmt(out);
    const int P = f.frac_bits + 1;       /* precision */
    const int emin = 1 - f.bias;         /* exponent of the smallest normal */
    const int emax = f.bias;             /* exponent of the largest finite */
    int L = or_bitlen(M);
    /* exponent of the leading bit, and of the last kept bit (the quantum) */
    int e = L - 1 + unit_exp;
    int qexp = (e > emin ? e : emin) - (P - 1);
    int shift = qexp - unit_exp;         /* low bits of M that are dropped */
    uint64_t q;
    int inexact = 0, round_up = 0;
    if (shift <= 0) {
        q = or_bits(M, 0, L) << (-shift); /* exact: L <= P here */
    } else {
        q = or_bits(M, shift, L - shift > 0 ? L - shift : 0);
        int half = or_bit(M, shift - 1);
        int sticky = or_any_below(M, shift - 1);
        inexact = half || sticky;
        if (mode == OR_RNE) round_up = half && (sticky || (q & 1));
        else if (mode == OR_RTZ) round_up = 0;
        else if (mode == OR_RUP) round_up = inexact && !sign;
        else round_up = inexact && sign;
    }
    q += (uint64_t)round_up;
    if (q == ((uint64_t)1 << P)) { q >>= 1; qexp += 1; }
    if (qexp + (P - 1) > emax) { /* overflow */
        int to_inf;
        if (mode == OR_RNE) to_inf = 1;
        else if (mode == OR_RTZ) to_inf = 0;
        else if (mode == OR_RUP) to_inf = !sign;
        else to_inf = sign;
        return to_inf ? or_inf(out, sign) : or_max_finite(out, sign);
    }
    if (q < ((uint64_t)1 << (P - 1))) /* subnormal (qexp == emin - (P - 1)) */
        return or_encode(out, sign, 0, q);
    return or_encode(out, sign, (uint64_t)(qexp + (P - 1) + f.bias), q - ((uint64_t)1 << (P - 1)));
}

static void or_store(void* result, uint64_t bits, int out) {
    or_format f = or_fmt(out);
    if (f.width == 8) memcpy(result, &bits, 8);
    else if (f.width == 4) { uint32_t v = (uint32_t)bits; memcpy(result, &v, 4); }
    else { uint16_t v = (uint16_t)bits; memcpy(result, &v, 2); }
}

static uint64_t or_finish(or_partial* s, int64_t n, int in, int out, int mode) {
    if (n == 0) return 0; /* +0 */
    if (s->has_nan || (s->has_pinf && s->has_ninf)) return or_quiet_nan(out);
    if (s->has_pinf) return or_inf(out, 0);
    if (s->has_ninf) return or_inf(out, 1);
    int sign = or_is_negative(&s->sum);
    or_big M = s->sum;
    if (sign) or_negate(&M);
    if (or_bitlen(&M) == 0) {
        or_format f = or_fmt(out);
        uint64_t neg_zero = (uint64_t)1 << (8 * f.width - 1);
        if (s->all_neg_zero) return neg_zero;
        if (s->all_pos_zero) return 0;
        return mode == OR_RDOWN ? neg_zero : 0;
    }
    return or_round(&M, sign, or_fmt(in).unit_exp, out, mode);
}

/*
 * Exact sum of n elements of `x` (dtype `in`), rounded to `out` under
 * `mode`; the result's bits are stored at `result` (2, 4 or 8 bytes).
 * Returns 0, or -1 for a bad argument.  `threads` <= 0 means one thread.
 */
int oracle_sum(const void* x, int64_t n, int in, int out, int mode, int threads, void* result) {
    if (in < 0 || in > 2 || out < 0 || out > 2 || mode < 0 || mode > 3 || n < 0) return -1;
    if (n > 0 && !x) return -1;
    if (threads < 1) threads = 1;
    if ((int64_t)threads > n) threads = n > 0 ? (int)n : 1;
    or_job* jobs = (or_job*)calloc((size_t)threads, sizeof(or_job));
    pthread_t* tids = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tids) { free(jobs); free(tids); return -1; }
    for (int t = 0; t < threads; t++) {
        jobs[t].x = x;
        jobs[t].begin = n * t / threads;
        jobs[t].end = n * (t + 1) / threads;
        jobs[t].dtype = in;
    }
    int* joined = (int*)calloc((size_t)threads, sizeof(int));
    for (int t = 1; t < threads; t++) {
        /* a thread that cannot be started runs inline instead */
        if (joined && pthread_create(&tids[t], NULL, or_worker, &jobs[t]) == 0) joined[t] = 1;
        else or_worker(&jobs[t]);
    }
    or_worker(&jobs[0]);
    for (int t = 1; t < threads; t++)
        if (joined && joined[t]) pthread_join(tids[t], NULL);
    free(joined);
    or_partial total;
    or_partial_init(&total);
    for (int t = 0; t < threads; t++) {
        or_big_add(&total.sum, &jobs[t].part.sum);
        total.has_nan |= jobs[t].part.has_nan;
        total.has_pinf |= jobs[t].part.has_pinf;
        total.has_ninf |= jobs[t].part.has_ninf;
        total.all_pos_zero &= jobs[t].part.all_pos_zero;
        total.all_neg_zero &= jobs[t].part.all_neg_zero;
    }
    uint64_t bits = or_finish(&total, n, in, out, mode);
    or_store(result, bits, out);
    free(jobs);
    free(tids);
    return 0;
}

/*
 * Segmented form: results[s] = exact sum of x[offsets[s] .. offsets[s+1]),
 * rounded; results is an array of S elements of format `out`.
 * Returns 0, or -1 for a bad argument (including decreasing offsets).
 */
int oracle_segmented_sum(const void* x, const int64_t* offsets, int64_t S, int in, int out,
                         int mode, int threads, void* results) {
    if (S < 0 || (S > 0 && (!offsets || !results))) return -1;
    int width = or_fmt(out).width;
    int in_width = or_fmt(in).width;
    for (int64_t s = 0; s < S; s++) {
        if (offsets[s + 1] < offsets[s] || offsets[s] < 0) return -1;
        const char* base = (const char*)x + (size_t)offsets[s] * (size_t)in_width;
        int rc = oracle_sum(base, offsets[s + 1] - offsets[s], in, out, mode, threads,
                            (char*)results + (size_t)s * (size_t)width);
        if (rc) return rc;
    }
    return 0;
}

/*
 * The exact sum itself, for tests that check a value rather than its
 * rounding: writes the two's-complement limbs (OR_LIMBS little-endian
 * 32-bit words, in units of the input format's smallest subnormal) to
 * `limbs_out`.  Returns the number of limbs, or -1.  Non-finite inputs are
 * skipped.
 */
int oracle_exact_limbs(const void* x, int64_t n, int in, uint32_t* limbs_out) {
    if (in < 0 || in > 2 || n < 0 || !limbs_out) return -1;
    or_partial s;
    or_partial_init(&s);
    or_accumulate(&s, x, 0, n, in);
    memcpy(limbs_out, s.sum.limb, sizeof(s.sum.limb));
    return OR_LIMBS;
}

/* Round an exact value given as sign-magnitude limbs (units 2^unit_exp). */
int oracle_round_limbs(const uint32_t* magnitude, int nlimbs, int sign, int unit_exp, int out,
                       int mode, void* result) {
    if (nlimbs < 0 || nlimbs > OR_LIMBS || out < 0 || out > 2 || mode < 0 || mode > 3) return -1;
    or_big M;
    memset(&M, 0, sizeof(M));
    memcpy(M.limb, magnitude, (size_t)nlimbs * 4);
    if (M.limb[OR_LIMBS - 1] >> 31) return -1;
    uint64_t bits;
    if (or_bitlen(&M) == 0) {
        or_format f = or_fmt(out);
        bits = sign ? (uint64_t)1 << (8 * f.width - 1) : 0;
    } else {
        bits = or_round(&M, sign, unit_exp, out, mode);
    }
    or_store(result, bits, out);
    return 0;
}
