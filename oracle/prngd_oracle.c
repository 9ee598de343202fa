/*
 * PRNGD oracle: test infrastructure only.
 *
 * Plain, slow, exact CPU implementation of the extended-precision uniform generator of
 * V. Demchik and A. Gulov, "Increasing precision of uniform pseudorandom number generators"
 * (arXiv:1401.8230), Section 2. It exists to check the CUDA library and to time a CPU
 * baseline. Only the tests, the package's smoke check and the benchmark's CPU-baseline leg
 * may load it. It shares no code, header or constant table with the CUDA path.
 *
 * Everything is integer arithmetic (unsigned __int128 for the exact rational step), except
 * where a form's definition is itself a floating-point operation sequence (form (a) and the
 * FP32 pair of form (c)); those use the host's IEEE-754 doubles and floats. Build without
 * -ffast-math and with -ffp-contract=off.
 *
 * Notation (Section 2): base draws x1 = a0 + u1*k and x2 = b0 + u2*k, with integers
 * u1, u2 in [0, 2^w - 1] and k = 2^-w.
 *
 * Parity: every function here is pinned by the CPU tests (closed forms, brute force over all
 * pairs at small w, published generator test vectors, exact rational arithmetic in Python).
 * Nothing is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORC_OK 0
#define ORC_EINVAL 1

/* ------------------------------------------------------------------------------------------
 * Base generators. The paper does not name a base generator (it asks only for independent,
 * uniform, statistically good draws, Section 2, last paragraph). This library uses
 * Marsaglia's xorshift128, one per stream, seeded from splitmix64.
 * ---------------------------------------------------------------------------------------- */

/* splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014): the state advances by the odd constant GAMMA (2^64 / golden ratio), and each
 * output is the state passed through a bijective 64-bit finaliser (xor-shift / multiply
 * rounds; the multipliers are Stafford's "Mix13" variant used by that paper). */
static const uint64_t SM64_GAMMA = 0x9E3779B97F4A7C15ull;

static uint64_t sm64_finalise(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Output number i (i = 0, 1, ...) of the splitmix64 sequence whose initial state is `seed`. */
uint64_t orc_splitmix64_output(uint64_t seed, uint64_t i) {
    uint64_t state = seed;
    /* The state after i+1 advances, written as the repeated addition it is. */
    state += (i + 1) * SM64_GAMMA;
    return sm64_finalise(state);
}

/* Seeding of stream `stream` from (seed, stream id): the stream takes splitmix64 outputs
 * 2*stream and 2*stream+1 and splits each into two 32-bit words (low word first):
 * (x, y, z, w) = (lo o_{2s}, hi o_{2s}, lo o_{2s+1}, hi o_{2s+1}). The finaliser maps only 0
 * to 0, and the two inputs differ by GAMMA, so the state is never all-zero. */
void orc_stream_seed(uint64_t seed, uint64_t stream, uint32_t st[4]) {
    uint64_t o0 = orc_splitmix64_output(seed, 2 * stream);
    uint64_t o1 = orc_splitmix64_output(seed, 2 * stream + 1);
    st[0] = (uint32_t)o0;
    st[1] = (uint32_t)(o0 >> 32);
    st[2] = (uint32_t)o1;
    st[3] = (uint32_t)(o1 >> 32);
}

/* Marsaglia, "Xorshift RNGs", J. Stat. Softw. 8(14), 2003: the 128-bit xor128 generator,
 * state (x, y, z, w), shift triple (11, 8, 19). Returns the new w. */
uint32_t orc_xorshift128_next(uint32_t st[4]) {
    uint32_t t = st[0] ^ (st[0] << 11);
    st[0] = st[1];
    st[1] = st[2];
    st[2] = st[3];
    st[3] = st[3] ^ (st[3] >> 19) ^ (t ^ (t >> 8));
    return st[3];
}

/* A w-bit base draw u in [0, 2^w - 1]: the top w bits of the next 32-bit output. This is
 * the integer numerator of the base PRN x = u * 2^-w, exact in FP32 for w <= 24. */
uint32_t orc_draw(uint32_t st[4], int w) {
    uint32_t r = orc_xorshift128_next(st);
    return (w == 32) ? r : (r >> (32 - w));
}

/* The state after `draws` more draws: the generator stepped that many times. */
void orc_skip(uint32_t st[4], uint64_t draws) {
    for (uint64_t i = 0; i < draws; ++i) orc_xorshift128_next(st);
}

/* First `count` raw 32-bit outputs of one stream. */
void orc_stream_raw(uint64_t seed, uint64_t stream, uint64_t count, uint32_t* out) {
    uint32_t st[4];
    orc_stream_seed(seed, stream, st);
    for (uint64_t i = 0; i < count; ++i) out[i] = orc_xorshift128_next(st);
}

/* L'Ecuyer's MRG32k3a ("Good parameters and implementations for combined multiple recursive
 * random number generators", Operations Research 47(1), 1999), one of the generators Section 2
 * recommends: two order-3 recurrences
 *     x1_n = (1403580 x1_{n-2} - 810728 x1_{n-3}) mod m1,   m1 = 2^32 - 209,
 *     x2_n = (527612 x2_{n-1} - 1370589 x2_{n-3}) mod m2,   m2 = 2^32 - 22853,
 * combined as z_n = (x1_n - x2_n) mod m1, with z = 0 reported as m1 (so z is in [1, m1]).
 * State st = (x1_{n-3}, x1_{n-2}, x1_{n-1}, x2_{n-3}, x2_{n-2}, x2_{n-1}). Exact 64-bit integer
 * arithmetic. Returns z. */
#define ORC_MRG_M1 4294967087ull
#define ORC_MRG_M2 4294944443ull
uint32_t orc_mrg32k3a_next(uint32_t st[6]) {
    int64_t p1 = (int64_t)(1403580ll * st[1]) - (int64_t)(810728ll * st[0]);
    p1 %= (int64_t)ORC_MRG_M1;
    if (p1 < 0) p1 += (int64_t)ORC_MRG_M1;
    int64_t p2 = (int64_t)(527612ll * st[5]) - (int64_t)(1370589ll * st[3]);
    p2 %= (int64_t)ORC_MRG_M2;
    if (p2 < 0) p2 += (int64_t)ORC_MRG_M2;
    st[0] = st[1];
    st[1] = st[2];
    st[2] = (uint32_t)p1;
    st[3] = st[4];
    st[4] = st[5];
    st[5] = (uint32_t)p2;
    int64_t z = p1 - p2;
    if (z <= 0) z += (int64_t)ORC_MRG_M1;
    return (uint32_t)z;
}

/* MRG32k3a stream seeding (the paper is silent): stream s takes splitmix64 outputs 3s, 3s+1 and
 * 3s+2 of `seed`, split into six 32-bit words w0..w5 (low word first); x1 state = w0..w2 mod m1,
 * x2 state = w3..w5 mod m2; a component that comes out all zero gets 1 as its first word. */
void orc_mrg_stream_seed(uint64_t seed, uint64_t stream, uint32_t st[6]) {
    uint32_t w[6];
    for (int i = 0; i < 3; ++i) {
        uint64_t o = orc_splitmix64_output(seed, 3 * stream + (uint64_t)i);
        w[2 * i] = (uint32_t)o;
        w[2 * i + 1] = (uint32_t)(o >> 32);
    }
    for (int i = 0; i < 3; ++i) {
        st[i] = (uint32_t)(w[i] % ORC_MRG_M1);
        st[3 + i] = (uint32_t)(w[3 + i] % ORC_MRG_M2);
    }
    if (!st[0] && !st[1] && !st[2]) st[0] = 1;
    if (!st[3] && !st[4] && !st[5]) st[3] = 1;
}

/* ------------------------------------------------------------------------------------------
 * The method, Section 2.
 * ---------------------------------------------------------------------------------------- */

/* Discrete accept-reject rule (Section 2, after Fig. 1): x1 is discrete with step k, so the
 * rejection region of Eq. (3) reduces to its two end points; a pair with x1 = a0 (u1 = 0) or
 * x1 = a (u1 = 2^w - 1) is dropped. Returns 1 if the pair is accepted. */
int orc_accept(uint32_t u1, int w) {
    uint64_t top = (w == 32) ? 0xFFFFFFFFull : ((1ull << w) - 1);
    return (u1 != 0) && ((uint64_t)u1 != top);
}

/* D_w = (2^w - 1)^2, the common denominator of Eq. (4) once both sides are scaled by 2^(2w). */
uint64_t orc_denominator(int w) {
    uint64_t m = (w == 32) ? 0xFFFFFFFFull : ((1ull << w) - 1);
    return m * m;
}

/* Numerator of Eq. (4) scaled by 2^(2w). With x1 = a0 + u1 k, x2 = b0 + u2 k and
 * a - a0 = b - b0 = (2^w - 1) k, Eq. (4) reads
 *     z' = (u1 k + u2 k^2 - (2^w - 1) k^2) / ((2^w - 1) k (1 - k)),
 * and multiplying both parts by 2^(2w) gives z' = n / D_w with
 *     n = u1 2^w + u2 - (2^w - 1).
 * The offsets a0 and b0 cancel. For an accepted pair n is in [1, D_w - 1]. */
uint64_t orc_numerator(uint32_t u1, uint32_t u2, int w) {
    uint64_t m = (w == 32) ? 0xFFFFFFFFull : ((1ull << w) - 1);
    return ((uint64_t)u1 << w) + (uint64_t)u2 - m;
}

/* Bit length of a nonzero integer. */
static int bitlen_u64(uint64_t v) {
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

/* Round-to-nearest-even of num/den (1 <= num, 1 <= den < 2^64, num/den >= 2^-1000 and
 * < 2^1000), from the definition: find the 53-bit integer part q of num*2^s/den, then compare
 * the remainder with den/2. Returns the IEEE-754 double. */
double orc_rn_ratio(uint64_t num, uint64_t den) {
    /* s with num*2^s/den in [2^52, 2^53): start from the bit lengths and correct by one. */
    int s = 52 + bitlen_u64(den) - bitlen_u64(num);
    u128 q, r;
    for (;;) {
        u128 scaled = (s >= 0) ? ((u128)num << s) : 0;
        u128 d = (u128)den;
        if (s < 0) {
            /* num/den >= 2^53 would need a right shift; not used by this library. */
            return NAN;
        }
        q = scaled / d;
        r = scaled % d;
        if (q >= ((u128)1 << 53)) {
            --s;
            continue;
        }
        if (q < ((u128)1 << 52)) {
            ++s;
            continue;
        }
        break;
    }
    /* Round half to even on the remainder: compare 2r with den. */
    u128 twice_r = r * 2;
    if (twice_r > (u128)den || (twice_r == (u128)den && (q & 1))) q += 1;
    /* q <= 2^53, so (double)q is exact; the scaling by 2^-s is exact (normal range). */
    return ldexp((double)(uint64_t)q, -s);
}

/* Bit length of a nonzero 128-bit integer. */
static int bitlen_u128(u128 v) {
    uint64_t hi = (uint64_t)(v >> 64);
    return hi ? 64 + bitlen_u64(hi) : bitlen_u64((uint64_t)v);
}

/* Round-to-nearest-even of (num/den) * 2^-e for 0 <= num < 2^128, 1 <= den < 2^64 and
 * num/den < 2^64, from the same definition as orc_rn_ratio: the 53-bit integer part q of
 * num*2^s/den, then the remainder against den/2. Returns 0.0 for num = 0. */
static double rn_ratio128(u128 num, uint64_t den, int e) {
    if (num == 0) return 0.0;
    int s = 52 + bitlen_u64(den) - bitlen_u128(num);
    u128 q, r, d;
    for (;;) {
        if (s >= 0) {
            d = (u128)den;
            q = (num << s) / d; /* num * 2^s < 2^54 den < 2^118: no overflow */
            r = (num << s) % d;
        } else {
            if (-s > 63) return NAN; /* num/den >= 2^116: not used by this library */
            d = (u128)den << (-s);
            q = num / d;
            r = num % d;
        }
        if (q >= ((u128)1 << 53)) {
            --s;
            continue;
        }
        if (q < ((u128)1 << 52)) {
            ++s;
            continue;
        }
        break;
    }
    u128 twice_r = r * 2;
    if (twice_r > d || (twice_r == d && (q & 1))) q += 1;
    return ldexp((double)(uint64_t)q, -s - e);
}

/* Form (b): the correctly rounded double nearest to z' = n / D_w. */
double orc_value_rn(uint64_t n, int w) { return orc_rn_ratio(n, orc_denominator(w)); }

/* C_w = RN(1 / D_w), the compile-time constant of the final scale ("most of Z is computed
 * during compilation", Algorithm 1's note). */
double orc_scale_constant(int w) { return orc_rn_ratio(1, orc_denominator(w)); }

/* Form (a): the FP64 operation sequence RN(RN(n) * C_w): one correctly rounded unsigned
 * 64-bit to double conversion, then one double multiply. */
double orc_value_form_a(uint64_t n, int w) {
    volatile double dn = (double)n; /* C conversion, IEEE round-to-nearest */
    volatile double c = orc_scale_constant(w);
    volatile double prod = dn * c;
    return prod;
}

/* Form (c): an FP32 pair (hi, lo) with hi = RN32(d) and lo = RN32(d - hi), where d is the
 * form-(b) value. d - hi is exact in double. */
void orc_value_form_c(uint64_t n, int w, float* hi, float* lo) {
    double d = orc_value_rn(n, w);
    volatile float h = (float)d;
    volatile double rest = d - (double)h;
    *hi = h;
    *lo = (float)rest;
}

/* Statistics of one output, exact integers: t = floor(2^32 z'), bin = floor(2^16 z') = t >> 16,
 * and the fixed-point powers p2 = floor(t^2 / 2^32), p3 = floor(p2 t / 2^32),
 * p4 = floor(p3 t / 2^32). out = {t, bin, p2, p3, p4}. */
void orc_stat_terms(uint64_t n, int w, uint64_t out[5]) {
    uint64_t d = orc_denominator(w);
    uint64_t t = (uint64_t)(((u128)n << 32) / d);
    uint64_t p2 = (t * t) >> 32;
    uint64_t p3 = (p2 * t) >> 32;
    uint64_t p4 = (p3 * t) >> 32;
    out[0] = t;
    out[1] = t >> 16;
    out[2] = p2;
    out[3] = p3;
    out[4] = p4;
}

/* Next accepted n of a stream, with pair semantics: each attempt takes two consecutive draws
 * (x1 first, then x2; Algorithm 1 draws r1 before r2). A rejected pair is dropped whole and
 * the next pair is taken ("take next pair (x1, x2)", Section 2). *rejects counts dropped pairs. */
uint64_t orc_next_n(uint32_t st[4], int w, uint64_t* rejects) {
    for (;;) {
        uint32_t u1 = orc_draw(st, w);
        uint32_t u2 = orc_draw(st, w);
        if (orc_accept(u1, w)) return orc_numerator(u1, u2, w);
        ++*rejects;
    }
}

/* Output forms, matching the library's numbering. */
#define ORC_FORM_A 0 /* double, FP64 conversion sequence */
#define ORC_FORM_B 1 /* double, correctly rounded */
#define ORC_FORM_C 2 /* float pair (hi, lo) */
#define ORC_FORM_N 3 /* the integer numerators n themselves (uint64) */
#define ORC_FORM_L 4 /* double, Algorithm 1's literal FP64 evaluation */

static int form_ok(int form) { return form >= 0 && form <= 4; }

/* Modes, bit flags (0: the map of Eq. (4) and pair rejects).
 * ORC_MODE_EQ5: the map of Eq. (5), which for one base generator on [0, 1 - k] is Eq. (6):
 *   x1 = a0 + k and x2 = b0 go to 0, x1 = a - k and x2 = b go to 1 - k'. With x1 = a0 + u1 k,
 *   x2 = b0 + u2 k and a - a0 = b - b0 = (2^w - 1) k, Eq. (5) reads
 *       z' = (1 - k^2) ((u1 - 1) + u2 k) / ((2^w - 3) + (2^w - 1) k),
 *   and scaling both parts by 2^w gives z' = (1 - k^2) m / (D_w - 2) with m = n - 1 =
 *   (u1 - 1) 2^w + u2 in [0, D_w - 2]: the range is [0, 1 - k^2].
 * ORC_MODE_ONE_MINUS: output 1 - z' instead of z' (Section 2: the usual way to exclude 0).
 * ORC_MODE_SINGLE: Algorithm 1's reject loop, which redraws only r1 until it is accepted and
 *   then draws r2 once; the default drops the whole pair ("take next pair", Section 2). */
#define ORC_MODE_EQ5 1
#define ORC_MODE_ONE_MINUS 2
#define ORC_MODE_SINGLE 4

static int mode_ok(int mode) { return mode >= 0 && mode <= 7; }

/* Next accepted attempt (u1, u2) of a stream under the mode's reject rule. */
static void next_attempt(uint32_t st[4], int w, int mode, uint64_t* rejects, uint32_t* u1,
                         uint32_t* u2) {
    if (mode & ORC_MODE_SINGLE) {
        for (;;) {
            *u1 = orc_draw(st, w);
            if (orc_accept(*u1, w)) break;
            ++*rejects;
        }
        *u2 = orc_draw(st, w);
        return;
    }
    for (;;) {
        *u1 = orc_draw(st, w);
        *u2 = orc_draw(st, w);
        if (orc_accept(*u1, w)) return;
        ++*rejects;
    }
}

/* The exact output value of an accepted attempt with numerator n (Eq. (4)) under the mode's
 * map, rounded to nearest: Eq. (4) is n / D_w and its complement (D_w - n) / D_w; Eq. (5) is
 * (2^2w - 1) m / ((D_w - 2) 2^2w) and its complement ((D_w - 2) 2^2w - (2^2w - 1) m) /
 * ((D_w - 2) 2^2w), both exact integer ratios (u128). */
static double value_mode_rn(uint64_t n, int w, int mode) {
    uint64_t d = orc_denominator(w);
    if (!(mode & ORC_MODE_EQ5)) return rn_ratio128((mode & ORC_MODE_ONE_MINUS) ? d - n : n, d, 0);
    uint64_t m = n - 1, e = d - 2;
    u128 p = ((u128)1 << (2 * w)) - 1;
    u128 num = p * m;
    if (mode & ORC_MODE_ONE_MINUS) num = ((u128)e << (2 * w)) - num;
    return rn_ratio128(num, e, 2 * w);
}

/* Form (a) under a mode: the FP64 conversion sequence RN(RN(x) * C) of the map's integer
 * numerator x and the compile-time constant C (Eq. (4): x = n, C = RN(1 / D_w); Eq. (5):
 * x = m, C = RN((1 - k^2) / (D_w - 2))), then 1 - z as one more FP64 subtraction. */
static double value_mode_form_a(uint64_t n, int w, int mode) {
    volatile double z;
    if (mode & ORC_MODE_EQ5) {
        uint64_t e = orc_denominator(w) - 2;
        volatile double c = rn_ratio128(((u128)1 << (2 * w)) - 1, e, 2 * w);
        volatile double x = (double)(n - 1);
        z = x * c;
    } else {
        z = orc_value_form_a(n, w);
    }
    if (mode & ORC_MODE_ONE_MINUS) z = 1.0 - z;
    return z;
}

/* Form L: Algorithm 1 evaluated literally in FP64, one IEEE operation at a time (round to
 * nearest even, no contraction), with the base PRNs R1 = u1 k and R2 = u2 k of one generator
 * on [min, max] = [0, 1 - k] (exact doubles). Eq. (4) as Algorithm 1 writes it:
 *     Z = (R1 + k R2 - (min + k max)) / ((max - min) (1 - k)),
 * the constants min + k max and (max - min)(1 - k) folded once ("computed during
 * compilation"). Eq. (5) through its one-generator form Eq. (6):
 *     Z = (1 - k^2) (trunc[R1 / k] + R2 - 1) / (trunc[1 / k] - 2 - k).
 * Then 1 - Z for ORC_MODE_ONE_MINUS. */
static double value_mode_form_l(uint32_t u1, uint32_t u2, int w, int mode) {
    volatile double k = ldexp(1.0, -w);
    volatile double r1 = ldexp((double)u1, -w), r2 = ldexp((double)u2, -w);
    volatile double mn = 0.0, mx = 1.0 - k;
    volatile double z;
    if (mode & ORC_MODE_EQ5) {
        volatile double t = trunc(r1 / k);
        volatile double s1 = t + r2;
        volatile double s2 = s1 - 1.0;
        volatile double kk = k * k;
        volatile double c3 = 1.0 - kk;
        volatile double num = c3 * s2;
        volatile double t1 = trunc(1.0 / k);
        volatile double d1 = t1 - 2.0;
        volatile double den = d1 - k;
        z = num / den;
    } else {
        volatile double kmx = k * mx;
        volatile double c1 = mn + kmx;
        volatile double span = mx - mn;
        volatile double onek = 1.0 - k;
        volatile double c2 = span * onek;
        volatile double kr2 = k * r2;
        volatile double a = r1 + kr2;
        volatile double b = a - c1;
        z = b / c2;
    }
    if (mode & ORC_MODE_ONE_MINUS) z = 1.0 - z;
    return z;
}

/* One output of form `form` for the accepted attempt (u1, u2) under `mode`, written to
 * element i of `out` (double, double, 2 floats, uint64, double). */
static void put_output(uint32_t u1, uint32_t u2, int w, int form, int mode, void* out, uint64_t i) {
    uint64_t n = orc_numerator(u1, u2, w);
    switch (form) {
        case ORC_FORM_A: ((double*)out)[i] = value_mode_form_a(n, w, mode); break;
        case ORC_FORM_B: ((double*)out)[i] = value_mode_rn(n, w, mode); break;
        case ORC_FORM_C: {
            double d = value_mode_rn(n, w, mode);
            volatile float h = (float)d;
            volatile double rest = d - (double)h;
            ((float*)out)[2 * i] = h;
            ((float*)out)[2 * i + 1] = (float)rest;
            break;
        }
        case ORC_FORM_L: ((double*)out)[i] = value_mode_form_l(u1, u2, w, mode); break;
        default: ((uint64_t*)out)[i] = n; break;
    }
}

/* Continue one stream from state `st` for `count` outputs. `out` receives count elements of
 * the form's type. */
static void fill_from_state(uint32_t st[4], int w, int form, int mode, uint64_t count, void* out,
                            uint64_t* rejects) {
    for (uint64_t i = 0; i < count; ++i) {
        uint32_t u1, u2;
        next_attempt(st, w, mode, rejects, &u1, &u2);
        put_output(u1, u2, w, form, mode, out, i);
    }
}

static size_t form_bytes(int form) { return (form == ORC_FORM_C) ? 8 : 8; }

/* Stream-major fill: out[j * per_stream + i] is output i of stream first_stream + j, each
 * stream freshly seeded from (seed, stream id). rejects (nullable) gets one count per stream. */
int orc_fill_mode(uint64_t seed, uint64_t first_stream, uint64_t n_streams, uint64_t per_stream,
                  int w, int form, int mode, void* out, uint64_t* rejects) {
    if (w < 2 || w > 32 || !form_ok(form) || !mode_ok(mode) || (!out && n_streams && per_stream))
        return ORC_EINVAL;
    for (uint64_t j = 0; j < n_streams; ++j) {
        uint32_t st[4];
        uint64_t rj = 0;
        orc_stream_seed(seed, first_stream + j, st);
        fill_from_state(st, w, form, mode, per_stream,
                        (char*)out + j * per_stream * form_bytes(form), &rj);
        if (rejects) rejects[j] = rj;
    }
    return ORC_OK;
}

int orc_fill(uint64_t seed, uint64_t first_stream, uint64_t n_streams, uint64_t per_stream,
             int w, int form, void* out, uint64_t* rejects) {
    return orc_fill_mode(seed, first_stream, n_streams, per_stream, w, form, 0, out, rejects);
}

/* One stream continued from a given state; the state is updated in place. */
int orc_fill_state_mode(uint32_t st[4], uint64_t count, int w, int form, int mode, void* out,
                        uint64_t* rejects) {
    if (w < 2 || w > 32 || !form_ok(form) || !mode_ok(mode)) return ORC_EINVAL;
    uint64_t r = 0;
    fill_from_state(st, w, form, mode, count, out, &r);
    if (rejects) *rejects = r;
    return ORC_OK;
}

int orc_fill_state(uint32_t st[4], uint64_t count, int w, int form, void* out,
                   uint64_t* rejects) {
    return orc_fill_state_mode(st, count, w, form, 0, out, rejects);
}

/* Fused statistics over streams first_stream .. first_stream + n_streams - 1, per_stream
 * outputs each, no values stored: hist[bin] += 1 for 65536 bins, and the four sums
 * S1 = sum t, S2 = sum p2, S3 = sum p3, S4 = sum p4 as 128-bit integers, stored as
 * sums[2p] = low word, sums[2p+1] = high word. Results are accumulated into hist and sums
 * (the caller zeroes them). rejects (nullable) gets one count per stream. */
int orc_stats(uint64_t seed, uint64_t first_stream, uint64_t n_streams, uint64_t per_stream,
              int w, uint64_t* hist, uint64_t* sums, uint64_t* rejects) {
    if (w < 2 || w > 32 || !hist || !sums) return ORC_EINVAL;
    u128 acc[4];
    for (int p = 0; p < 4; ++p) acc[p] = ((u128)sums[2 * p + 1] << 64) | sums[2 * p];
    for (uint64_t j = 0; j < n_streams; ++j) {
        uint32_t st[4];
        uint64_t rj = 0;
        orc_stream_seed(seed, first_stream + j, st);
        for (uint64_t i = 0; i < per_stream; ++i) {
            uint64_t terms[5];
            orc_stat_terms(orc_next_n(st, w, &rj), w, terms);
            hist[terms[1]] += 1;
            acc[0] += terms[0];
            acc[1] += terms[2];
            acc[2] += terms[3];
            acc[3] += terms[4];
        }
        if (rejects) rejects[j] = rj;
    }
    for (int p = 0; p < 4; ++p) {
        sums[2 * p] = (uint64_t)acc[p];
        sums[2 * p + 1] = (uint64_t)(acc[p] >> 64);
    }
    return ORC_OK;
}

/* Every pair (u1, u2) of w-bit draws, u1-major: accept[i] in {0,1} and n[i] (0 if rejected).
 * For brute-force checks of the accept-reject rule and of Eq. (4) at small w. */
int orc_enumerate_pairs(int w, uint8_t* accept, uint64_t* n) {
    if (w < 1 || w > 14) return ORC_EINVAL;
    uint64_t side = 1ull << w;
    for (uint64_t u1 = 0; u1 < side; ++u1)
        for (uint64_t u2 = 0; u2 < side; ++u2) {
            uint64_t i = u1 * side + u2;
            accept[i] = (uint8_t)orc_accept((uint32_t)u1, w);
            n[i] = accept[i] ? orc_numerator((uint32_t)u1, (uint32_t)u2, w) : 0;
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------
 * The method over MRG32k3a draws. The base PRN of the method is a grid of M points with step
 * k = 1/M; MRG32k3a's z in [1, m1] is read as the draw u = z - 1 on the grid of M = m1 points.
 * Everything of Section 2 then holds with 2^w replaced by M: accept u1 not in {0, M - 1},
 * z' = n / D with n = u1 M + u2 - (M - 1) and D = (M - 1)^2 (< 2^64).
 * ---------------------------------------------------------------------------------------- */
uint64_t orc_mrg_denominator(void) { return (ORC_MRG_M1 - 1) * (ORC_MRG_M1 - 1); }

/* Stream-major fill (forms A, B, C, N) with the pair rule, as orc_fill. */
int orc_fill_mrg(uint64_t seed, uint64_t first_stream, uint64_t n_streams, uint64_t per_stream, int form,
                 void* out, uint64_t* rejects) {
    if (form < 0 || form > 3 || (!out && n_streams && per_stream)) return ORC_EINVAL;
    const uint64_t M = ORC_MRG_M1, D = orc_mrg_denominator();
    volatile double c = orc_rn_ratio(1, D);
    for (uint64_t j = 0; j < n_streams; ++j) {
        uint32_t st[6];
        uint64_t rj = 0;
        orc_mrg_stream_seed(seed, first_stream + j, st);
        for (uint64_t i = 0; i < per_stream; ++i) {
            uint64_t u1, u2;
            for (;;) {
                u1 = orc_mrg32k3a_next(st) - 1u;
                u2 = orc_mrg32k3a_next(st) - 1u;
                if (u1 != 0 && u1 != M - 1) break;
                ++rj;
            }
            const uint64_t n = u1 * M + u2 - (M - 1);
            const uint64_t k = j * per_stream + i;
            switch (form) {
                case ORC_FORM_A: {
                    volatile double dn = (double)n;
                    ((double*)out)[k] = dn * c;
                    break;
                }
                case ORC_FORM_B: ((double*)out)[k] = orc_rn_ratio(n, D); break;
                case ORC_FORM_C: {
                    double d = orc_rn_ratio(n, D);
                    volatile float h = (float)d;
                    volatile double rest = d - (double)h;
                    ((float*)out)[2 * k] = h;
                    ((float*)out)[2 * k + 1] = (float)rest;
                    break;
                }
                default: ((uint64_t*)out)[k] = n; break;
            }
        }
        if (rejects) rejects[j] = rj;
    }
    return ORC_OK;
}

/* Per-element helpers over arrays (for checks over many n at once). */
void orc_values_rn(const uint64_t* n, uint64_t count, int w, double* out) {
    for (uint64_t i = 0; i < count; ++i) out[i] = orc_value_rn(n[i], w);
}
void orc_values_form_a(const uint64_t* n, uint64_t count, int w, double* out) {
    for (uint64_t i = 0; i < count; ++i) out[i] = orc_value_form_a(n[i], w);
}
void orc_values_form_c(const uint64_t* n, uint64_t count, int w, float* out) {
    for (uint64_t i = 0; i < count; ++i) orc_value_form_c(n[i], w, &out[2 * i], &out[2 * i + 1]);
}
void orc_values_stat_terms(const uint64_t* n, uint64_t count, int w, uint64_t* out) {
    for (uint64_t i = 0; i < count; ++i) orc_stat_terms(n[i], w, &out[5 * i]);
}

/* Output of each accepted attempt (u1[i], u2[i]) in form `form` under `mode` (the reject bit
 * is ignored: the attempts are given). */
int orc_values_mode(const uint32_t* u1, const uint32_t* u2, uint64_t count, int w, int form,
                    int mode, void* out) {
    if (w < 2 || w > 32 || !form_ok(form) || !mode_ok(mode)) return ORC_EINVAL;
    for (uint64_t i = 0; i < count; ++i) put_output(u1[i], u2[i], w, form, mode, out, i);
    return ORC_OK;
}
