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

/* First `count` raw 32-bit outputs of one stream. */
void orc_stream_raw(uint64_t seed, uint64_t stream, uint64_t count, uint32_t* out) {
    uint32_t st[4];
    orc_stream_seed(seed, stream, st);
    for (uint64_t i = 0; i < count; ++i) out[i] = orc_xorshift128_next(st);
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

static int form_ok(int form) { return form >= 0 && form <= 3; }

/* Continue one stream from state `st` for `count` outputs. `out` receives count elements of
 * the form's type (double, double, 2 floats, uint64). */
static void fill_from_state(uint32_t st[4], int w, int form, uint64_t count, void* out,
                            uint64_t* rejects) {
    for (uint64_t i = 0; i < count; ++i) {
        uint64_t n = orc_next_n(st, w, rejects);
        switch (form) {
            case ORC_FORM_A: ((double*)out)[i] = orc_value_form_a(n, w); break;
            case ORC_FORM_B: ((double*)out)[i] = orc_value_rn(n, w); break;
            case ORC_FORM_C: {
                float h, l;
                orc_value_form_c(n, w, &h, &l);
                ((float*)out)[2 * i] = h;
                ((float*)out)[2 * i + 1] = l;
                break;
            }
            default: ((uint64_t*)out)[i] = n; break;
        }
    }
}

static size_t form_bytes(int form) { return (form == ORC_FORM_C) ? 8 : 8; }

/* Stream-major fill: out[j * per_stream + i] is output i of stream first_stream + j, each
 * stream freshly seeded from (seed, stream id). rejects (nullable) gets one count per stream. */
int orc_fill(uint64_t seed, uint64_t first_stream, uint64_t n_streams, uint64_t per_stream,
             int w, int form, void* out, uint64_t* rejects) {
    if (w < 2 || w > 32 || !form_ok(form) || (!out && n_streams && per_stream)) return ORC_EINVAL;
    for (uint64_t j = 0; j < n_streams; ++j) {
        uint32_t st[4];
        uint64_t rj = 0;
        orc_stream_seed(seed, first_stream + j, st);
        fill_from_state(st, w, form, per_stream, (char*)out + j * per_stream * form_bytes(form),
                        &rj);
        if (rejects) rejects[j] = rj;
    }
    return ORC_OK;
}

/* One stream continued from a given state; the state is updated in place. */
int orc_fill_state(uint32_t st[4], uint64_t count, int w, int form, void* out,
                   uint64_t* rejects) {
    if (w < 2 || w > 32 || !form_ok(form)) return ORC_EINVAL;
    uint64_t r = 0;
    fill_from_state(st, w, form, count, out, &r);
    if (rejects) *rejects = r;
    return ORC_OK;
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
