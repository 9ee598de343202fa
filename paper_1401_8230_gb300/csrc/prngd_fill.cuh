// prngd_fill.cuh -- the fill kernels: one xorshift128 stream per thread, state in registers,
// outputs produced in order (Algorithm 1 per output, pair semantics for rejects), staged per
// warp in shared memory and written with 2D TMA tiled stores (cp.async.bulk.tensor) or, when
// the output cannot be described by a tensor map, with coalesced scalar stores.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "prngd_math.cuh"

namespace prngd {

constexpr int kChunk = 16;         // outputs per stream per staged tile (128 bytes per row)
constexpr int kTileBytes = 32 * kChunk * 8;  // one warp: 32 streams x 16 outputs x 8 bytes

enum Form : int { kFormA = 0, kFormB = 1, kFormC = 2, kFormL = 4, kFormAF = 8 };
// Form A takes RN(n) by the u64 -> f64 conversion instruction (its definition: the conversion
// and the final scale are its FP64 steps) unless MAP has kMapCvt (PRNG_MODE_BALANCED): then by
// integer rounding, the same bits with the ALU pipe's help, since FP64 issue is scarce.
// kFormAF forces the conversion instruction under either MAP.

// Map bits (template parameter MAP of the per-output code): the map of Eq. 5 (one generator:
// Eq. 6) instead of Eq. 4, and 1 - z instead of z. MAP = 0 is Eq. 4.
constexpr int kMapEq5 = 1;
constexpr int kMapOneMinus = 2;
// Not a map: PRNG_MODE_BALANCED, the same values by a route that shares the work between the
// integer and FP64 pipes (form B: 3 of 4 outputs rounded by the FP64 conversion, see
// cvt_group_mask; form A: n converted with integer operations).
constexpr int kMapCvt = 4;

struct FillParams {
  uint4* state;         // n_streams xorshift states (x, y, z, w)
  uint64_t n_streams;
  uint64_t per_stream;
  uint64_t* out;        // stream-major, 8 bytes per output
  uint64_t* rejects;    // nullable, per stream
  DivConst dc;          // exact-division constants of D
  double scale;         // C_w = RN(1/D) for form A
  int w;                // draw precision
  uint32_t one;         // always 1; a run-time multiplier keeps the adds below on the FMA pipe
  uint32_t single;      // 1: Algorithm 1's reject loop (only r1 is redrawn); 0: the pair rule
  uint32_t keep_lines;  // 1: rows do not start on 128-byte lines; tensor stores ask L2 to keep
                        // their lines (evict_last) until the neighbouring store completes them
  DivConst ec;          // exact-division constants of D - 2 (Eq. 5)
  double scale5;        // RN((1 - k^2) / (D - 2)), form A under Eq. 5
  double k;             // 2^-w (form L)
  double l1, l2;        // form L constants: Eq. 4: min + k max and (max - min)(1 - k);
                        // Eq. 6: 1 - k^2 and trunc(1/k) - 2 - k
};

// ------------------------------------------------------------------------ per-output work
// Rejects, in order (Section 2 and Algorithm 1): the pair rule drops (u1, u2) and takes the
// next two draws; Algorithm 1's rule redraws only r1, so the pair's second draw is the next
// r1 candidate and one more draw follows as r2.
template <int W>
__device__ __forceinline__ void take_accepted(uint32_t& u1, uint32_t& u2, XorShift128& st, uint32_t& rej, int w,
                                              uint32_t top, uint32_t single) {
  while (!accepted(u1, top)) {
    ++rej;
    if (single) {
      u1 = u2;
      u2 = draw<W>(st, w);
    } else {
      u1 = draw<W>(st, w);
      u2 = draw<W>(st, w);
    }
  }
}

// Exactly rounded output bits (forms B and C) of an accepted pair at w = 32 or 24 under a map,
// from compile-time constants only. Eq. 4's complement is Eq. 4 of the complemented draws.
template <int W, int FORM, int MAP>
__device__ __forceinline__ uint64_t exact_bc(uint32_t u1, uint32_t u2) {
  constexpr uint32_t top = (W == 32) ? 0xFFFFFFFFu : ((1u << W) - 1u);
  if constexpr ((MAP & kMapEq5) != 0) {
    const uint64_t bits = eq5_bits_exact<W>(u1, u2, (MAP & kMapOneMinus) != 0);
    if constexpr (FORM == kFormC) return bits ? f32pair_from_bits(bits) : 0ull;  // z' = 0 is a pair of zeros
    return bits;
  } else {
    const uint32_t a1 = (MAP & kMapOneMinus) ? top - u1 : u1, a2 = (MAP & kMapOneMinus) ? top - u2 : u2;
    const uint64_t bits = rn_bits_exact(numerator(a1, a2, W), divconst_for<W>());
    return FORM == kFormC ? f32pair_from_bits(bits) : bits;
  }
}

// Form L: Algorithm 1 evaluated literally in FP64 with the base PRNs R1 = u1 k and R2 = u2 k
// (exact): Eq. 4 as (R1 + k R2 - (min + k max)) / ((max - min)(1 - k)); Eq. 5 through its
// one-generator form Eq. 6, (1 - k^2)(trunc[R1/k] + R2 - 1) / (trunc[1/k] - 2 - k), where
// trunc[R1/k] = u1. One IEEE operation at a time; the constants come folded from the host.
template <int MAP>
__device__ __forceinline__ uint64_t form_l_bits(uint32_t u1, uint32_t u2, const FillParams& p) {
  const double r2 = __dmul_rn((double)u2, p.k);
  double z;
  if constexpr ((MAP & kMapEq5) != 0) {
    const double s1 = __dadd_rn((double)u1, r2);
    z = __ddiv_rn(__dmul_rn(p.l1, __dsub_rn(s1, 1.0)), p.l2);
  } else {
    const double a = __dadd_rn(__dmul_rn((double)u1, p.k), __dmul_rn(p.k, r2));
    z = __ddiv_rn(__dsub_rn(a, p.l1), p.l2);
  }
  if constexpr ((MAP & kMapOneMinus) != 0) z = __dsub_rn(1.0, z);
  return (uint64_t)__double_as_longlong(z);
}

// The output of an accepted pair, exactly as each form defines it, under a map.
template <int W, int FORM, int MAP>
__device__ __forceinline__ uint64_t convert_exact(uint32_t u1, uint32_t u2, const FillParams& p) {
  const int w = W > 0 ? W : p.w;
  if constexpr (FORM == kFormL) {
    return form_l_bits<MAP>(u1, u2, p);
  } else if constexpr (FORM == kFormA || FORM == kFormAF) {
    constexpr bool kIntRound = FORM == kFormA && (MAP & kMapCvt) != 0;
    double z;
    if constexpr ((MAP & kMapEq5) != 0) {
      const uint64_t m = ((uint64_t)(u1 - 1u) << w) + u2;  // 0 for the pair mapped to z' = 0
      const double rm = kIntRound ? __longlong_as_double((long long)(m ? u64_to_f64_bits(m) : 0ull))
                                  : __ull2double_rn(m);
      z = __dmul_rn(rm, p.scale5);  // RN(RN(m) C5)
    } else {
      const uint64_t n = numerator(u1, u2, w);
      const double rn = kIntRound ? __longlong_as_double((long long)u64_to_f64_bits(n)) : __ull2double_rn(n);
      z = __dmul_rn(rn, p.scale);  // RN(RN(n) C_w)
    }
    if constexpr ((MAP & kMapOneMinus) != 0) z = __dsub_rn(1.0, z);
    return (uint64_t)__double_as_longlong(z);
  } else if constexpr (W == 32 || W == 24) {
    return exact_bc<W, FORM, MAP>(u1, u2);
  } else {
    const uint32_t top = (w == 32) ? 0xFFFFFFFFu : ((1u << w) - 1u);
    uint64_t bits;
    if constexpr ((MAP & kMapEq5) != 0) {
      bits = eq5_bits_exact_w(u1, u2, w, p.ec, (MAP & kMapOneMinus) != 0);
      if constexpr (FORM == kFormC) return bits ? f32pair_from_bits(bits) : 0ull;
      return bits;
    } else {
      const uint32_t a1 = (MAP & kMapOneMinus) ? top - u1 : u1, a2 = (MAP & kMapOneMinus) ? top - u2 : u2;
      bits = rn_bits_exact(numerator(a1, a2, w), p.dc);
    }
    return FORM == kFormC ? f32pair_from_bits(bits) : bits;
  }
}

// The slow path of one output: redraw rejected attempts in order, then convert exactly. Only
// entered for a reject (probability 2^(1-w)), for small values (probability ~2^-10) and for
// the rare values near a rounding boundary of the fast paths.
template <int W, int FORM, int MAP = 0>
__device__ __forceinline__ uint64_t slow_output(uint32_t u1, uint32_t u2, XorShift128& st, uint32_t& rej,
                                                const FillParams& p) {
  const uint32_t top = (p.w == 32) ? 0xFFFFFFFFu : ((1u << p.w) - 1u);
  take_accepted<W>(u1, u2, st, rej, p.w, top, p.single);
  return convert_exact<W, FORM, MAP>(u1, u2, p);
}

// One output of a stream, in order. Returns the 8 output bytes.
template <int W, int FORM, int MAP = 0>
__device__ __forceinline__ uint64_t next_output(XorShift128& st, uint32_t& rej, const FillParams& p) {
  const uint32_t u1 = draw<W>(st, p.w);
  const uint32_t u2 = draw<W>(st, p.w);
  if constexpr (FORM == kFormA || FORM == kFormAF || FORM == kFormL) {
    const uint32_t top = (W == 32) ? 0xFFFFFFFFu : (W > 0 ? ((1u << W) - 1u) : ((1u << p.w) - 1u));
    if (__builtin_expect(accepted(u1, top), 1)) return convert_exact<W, FORM, MAP>(u1, u2, p);
    return slow_output<W, FORM, MAP>(u1, u2, st, rej, p);
  } else if constexpr (W != 32 && W != 24) {
    return slow_output<W, FORM, MAP>(u1, u2, st, rej, p);
  } else {
    constexpr bool kComp = (MAP & kMapOneMinus) != 0;
    constexpr uint32_t top = (W == 32) ? 0xFFFFFFFFu : ((1u << W) - 1u);
    const uint32_t a1 = kComp ? top - u1 : u1, a2 = kComp ? top - u2 : u2;  // 1 - z: complemented draws
    uint64_t bits;
    if constexpr ((MAP & kMapEq5) != 0) {
      if constexpr (W == 32) {
        const uint64_t Y = fast32_eq5_Y(a1, a2);
        if (!__builtin_expect(fast32_eq5_ok(a1, Y), 1)) return slow_output<W, FORM, MAP>(u1, u2, st, rej, p);
        bits = fast32_eq5_bits(a1, a2, Y, kComp ? 1u : 0u);
      } else {
        const uint64_t K = fast24_eq5_K(a1, a2);
        if (__builtin_expect(fast24_eq5_ok(a1, K), 1)) bits = fast24_eq5_bits(a1, a2, K, kComp ? 0x10000u : 0u);
        else if (medium24_eq5_ok(a1, a2)) bits = medium24_eq5_bits(a1, a2, kComp ? 1u : 0u);
        else return slow_output<W, FORM, MAP>(u1, u2, st, rej, p);
      }
    } else if constexpr (W == 32) {
      const uint64_t X = fast32_X(a1, a2);
      if (!__builtin_expect(fast32_ok(a1, X), 1)) return slow_output<W, FORM, MAP>(u1, u2, st, rej, p);
      bits = fast32_bits(a1, a2, X);
    } else {
      const uint64_t K = fast24_K(a1, a2);
      if (!__builtin_expect(fast24_ok(a1, K), 1)) return slow_output<W, FORM, MAP>(u1, u2, st, rej, p);
      bits = fast24_bits(a1, a2, K);
    }
    return FORM == kFormC ? f32pair_from_bits(bits) : bits;
  }
}

// ------------------------------------------------------------------------ pair fast path
// Four consecutive draws in place: each state word is replaced once, so after the block
// (x, y, z, w) is again the state in its usual order and the four draws are its words.
__device__ __forceinline__ uint32_t xs_word(uint32_t a, uint32_t w) {
  const uint32_t t = a ^ (a << 11);
  return w ^ (w >> 19) ^ (t ^ (t >> 8));
}
__device__ __forceinline__ void xs_block4(XorShift128& s) {
  s.x = xs_word(s.x, s.w);
  s.y = xs_word(s.y, s.x);
  s.z = xs_word(s.z, s.y);
  s.w = xs_word(s.w, s.z);
}

// ~u as u * (-1) - 1, a multiply-add by the run-time -1 (`neg_one` = 0 - FillParams::one), so
// that the complement of the 1 - z map runs on the FMA pipe instead of adding an ALU operation
// per draw to the pipe that bounds the pair path.
__device__ __forceinline__ uint32_t complement_fma(uint32_t u, uint32_t neg_one) {
  uint32_t c;
  asm("mad.lo.u32 %0, %1, %2, -1;" : "=r"(c) : "r"(u), "r"(neg_one));
  return c;
}

// The w = 32 fast paths written out as PTX (Eq. 4: fast32_ok / fast32_bits; Eq. 5:
// fast32_eq5_ok / fast32_eq5_bits) in two steps: the 64-bit I = floor(V 2^64) and the check,
// then the rounding of I to the output's bits (bits_from_I_int or bits_from_I_cvt). The adds
// that need no carry are multiply-adds by the run-time constant `one`, so that they run on the
// FMA pipe beside the ALU work of the draws. X = K1 u1 + 2 u2 + C0 and
// I = A 2^32 + 2A + u2 + (X >> 32) + PLUS: Eq. 4 with (K1, C0, PLUS) = (3, -1, 1), X = 2B + 3A;
// Eq. 5 with (4, -4, 0 or 1), X = 4A + 2 u2. The check is 1 when 2^22 <= A <= 2^32 - 4 and the
// low word of X is below LIM; I is meaningless otherwise.
// The wide multiply-adds form K1 u1 + 2 u2 = X - C0 with no 64-bit constant, and C0 is added to
// the low word alone, which gives X's low word exactly. Its high word is X's whenever X's low
// word is below 2^32 + C0, which the check (LIM <= 2^32 - 64 for Eq. 5, 2^32 - 8 for Eq. 4)
// ensures. (Measured on the bulk fill against C0 as the 64-bit addend of the first multiply-add,
// Gsamples/s: integer-only form B 676 -> 708, balanced 732 -> 751, form C 563 -> 571, Eq. 5
// 679 -> 707 and 733 -> 755, 1 - z 645 -> 670.)
//
// Both outputs of a pair (draws x, y and z, w), with one check for the two.
template <int K1, int C0, int PLUS, unsigned LIM>
__device__ __forceinline__ uint32_t fast32_pair_I_ptx_t(uint32_t x, uint32_t y, uint32_t z, uint32_t w, uint32_t one,
                                                        uint64_t& Ia, uint64_t& Ib) {
  uint32_t ok;
  asm("{\n\t"
      ".reg .u64 Ya, Xa, Pa, Ja, Yb, Xb, Pb, Jb;\n\t"
      ".reg .u32 xla, fa, aa, Aa, ga, ila, iha, xlb, fb, ab, Ab, gb, ilb, ihb;\n\t"
      ".reg .pred p1, p2, p3, p4;\n\t"
      "mul.wide.u32 Ya, %4, 2;\n\t"
      "mad.wide.u32 Xa, %3, %9, Ya;\n\t"         // X of output a, less C0
      "mov.b64 {xla, fa}, Xa;\n\t"
      "mad.lo.u32 xla, xla, %7, %8;\n\t"
      "mul.wide.u32 Yb, %6, 2;\n\t"
      "mad.wide.u32 Xb, %5, %9, Yb;\n\t"         // X of output b, less C0
      "mov.b64 {xlb, fb}, Xb;\n\t"
      "mad.lo.u32 xlb, xlb, %7, %8;\n\t"
      "mad.lo.u32 aa, %3, %7, -4194305;\n\t"
      "mad.lo.u32 ab, %5, %7, -4194305;\n\t"
      "setp.lt.u32 p1, aa, 0xFFBFFFFD;\n\t"      // both A in [2^22, 2^32 - 4], both low words of X
      "setp.lt.and.u32 p2, xla, %11, p1;\n\t"    // below LIM
      "setp.lt.and.u32 p3, ab, 0xFFBFFFFD, p2;\n\t"
      "setp.lt.and.u32 p4, xlb, %11, p3;\n\t"
      "selp.u32 %0, 1, 0, p4;\n\t"
      "mad.lo.u32 Aa, %3, %7, -1;\n\t"
      "mov.b64 Pa, {%4, Aa};\n\t"
      "mad.wide.u32 Ja, Aa, 2, Pa;\n\t"
      "mad.lo.u32 ga, fa, %7, %10;\n\t"
      "mov.b64 {ila, iha}, Ja;\n\t"
      "add.cc.u32 ila, ila, ga;\n\t"
      "addc.u32 iha, iha, 0;\n\t"
      "mov.b64 %1, {ila, iha};\n\t"
      "mad.lo.u32 Ab, %5, %7, -1;\n\t"
      "mov.b64 Pb, {%6, Ab};\n\t"
      "mad.wide.u32 Jb, Ab, 2, Pb;\n\t"
      "mad.lo.u32 gb, fb, %7, %10;\n\t"
      "mov.b64 {ilb, ihb}, Jb;\n\t"
      "add.cc.u32 ilb, ilb, gb;\n\t"
      "addc.u32 ihb, ihb, 0;\n\t"
      "mov.b64 %2, {ilb, ihb};\n\t"
      "}"
      : "=r"(ok), "=l"(Ia), "=l"(Ib)
      : "r"(x), "r"(y), "r"(z), "r"(w), "r"(one), "n"(C0), "n"(K1), "n"(PLUS), "n"(LIM));
  return ok;
}

// One output.
template <int K1, int C0, int PLUS, unsigned LIM>
__device__ __forceinline__ uint64_t fast32_I_ptx_t(uint32_t u1, uint32_t u2, uint32_t one, uint32_t& ok) {
  uint64_t I;
  asm("{\n\t"
      ".reg .u64 Y, X, P, Ip;\n\t"
      ".reg .u32 xlo, f, a, A, g, ilo, ihi;\n\t"
      ".reg .pred p1, p2;\n\t"
      "mul.wide.u32 Y, %3, 2;\n\t"
      "mad.wide.u32 X, %2, %6, Y;\n\t"
      "mov.b64 {xlo, f}, X;\n\t"
      "mad.lo.u32 xlo, xlo, %4, %5;\n\t"
      "mad.lo.u32 a, %2, %4, -4194305;\n\t"
      "setp.lt.u32 p1, a, 0xFFBFFFFD;\n\t"
      "setp.lt.and.u32 p2, xlo, %8, p1;\n\t"
      "selp.u32 %1, 1, 0, p2;\n\t"
      "mad.lo.u32 A, %2, %4, -1;\n\t"
      "mov.b64 P, {%3, A};\n\t"
      "mad.wide.u32 Ip, A, 2, P;\n\t"
      "mad.lo.u32 g, f, %4, %7;\n\t"
      "mov.b64 {ilo, ihi}, Ip;\n\t"
      "add.cc.u32 ilo, ilo, g;\n\t"
      "addc.u32 ihi, ihi, 0;\n\t"
      "mov.b64 %0, {ilo, ihi};\n\t"
      "}"
      : "=l"(I), "=r"(ok)
      : "r"(u1), "r"(u2), "r"(one), "n"(C0), "n"(K1), "n"(PLUS), "n"(LIM));
  return I;
}

// RN(I 2^-64) as the output's bits, for I in [2^54, 2^64) with the exact value strictly
// between I and I + 1, by integer operations (ALU and FMA pipes): p = the top bit of I, then
// the mantissa (I + 2^(p - 53)) >> (p - 52) with the exponent (p + 990) << 20 added to its
// high word (the implicit bit adds one more).
__device__ __forceinline__ uint64_t bits_from_I_int(uint64_t I, uint32_t one) {
  uint32_t lo, hi;
  asm("{\n\t"
      ".reg .u32 ilo, ihi, q, s, rb, jlo, jhi, s1, mhi, e;\n\t"
      "mov.b64 {ilo, ihi}, %2;\n\t"
      "bfind.u32 q, ihi;\n\t"
      "mad.lo.u32 s, q, %3, -21;\n\t"
      "shl.b32 rb, 1, s;\n\t"
      "add.cc.u32 jlo, ilo, rb;\n\t"             // J = I + 2^s
      "addc.u32 jhi, ihi, 0;\n\t"
      "mad.lo.u32 s1, q, %3, -20;\n\t"
      "shf.r.wrap.b32 %1, jlo, jhi, s1;\n\t"
      "shr.u32 mhi, jhi, s1;\n\t"
      "mad.lo.u32 e, q, 0x100000, 0x3DE00000;\n\t"
      "mad.lo.u32 %0, mhi, %3, e;\n\t"
      "}"
      : "=r"(hi), "=r"(lo)
      : "l"(I), "r"(one));
  return ((uint64_t)hi << 32) | lo;
}

// The same by the u64 -> f64 conversion instruction (FP64 pipe), then 2^-64 as an exponent
// subtraction. I has at least 55 bits, so the rounding point lies above bit 1 and the halfway
// point below it is even; I | 1 therefore rounds as the exact value does, never as a tie.
__device__ __forceinline__ uint64_t bits_from_I_cvt(uint64_t I, uint32_t one) {
  uint32_t lo, hi;
  asm("{\n\t"
      ".reg .u64 J;\n\t"
      ".reg .f64 d;\n\t"
      ".reg .u32 dhi;\n\t"
      "or.b64 J, %2, 1;\n\t"
      "cvt.rn.f64.u64 d, J;\n\t"
      "mov.b64 {%1, dhi}, d;\n\t"
      "mad.lo.u32 %0, dhi, %3, -67108864;\n\t"   // exponent - 64
      "}"
      : "=r"(hi), "=r"(lo)
      : "l"(I), "r"(one));
  return ((uint64_t)hi << 32) | lo;
}

// I and the check of both outputs of a pair: one combined check when either output takes the
// conversion route (measured best there), two separate ones on the integer route (1% faster
// there); callers pass `joint` as a constant.
template <int K1, int C0, int PLUS, unsigned LIM>
__device__ __forceinline__ uint32_t fast32_I_pair(uint32_t x, uint32_t y, uint32_t z, uint32_t w, uint32_t one,
                                                  bool joint, uint64_t& Ia, uint64_t& Ib) {
  if (joint) return fast32_pair_I_ptx_t<K1, C0, PLUS, LIM>(x, y, z, w, one, Ia, Ib);
  uint32_t ok0, ok1;
  Ia = fast32_I_ptx_t<K1, C0, PLUS, LIM>(x, y, one, ok0);
  Ib = fast32_I_ptx_t<K1, C0, PLUS, LIM>(z, w, one, ok1);
  return ok0 & ok1;
}

// Which outputs of a 4-output group (bit i: output i) the pair paths (w = 32 and 24, forms B
// and C, every map) round by the conversion instruction: form C all of them,
// form B 3 in 4 when MAP has kMapCvt and none otherwise (form B is integer-only by default). The ALU pipe bounds
// these kernels and the FP64 pipe is otherwise idle. Measured on the bulk fill (Gsamples/s,
// none / 1 in 2 / 3 in 4 / all):
//   form B: Eq. 4 669 / 696 / 720 / 595, Eq. 5 664 / 704 / 724 / 596, Eq. 5 and 1 - z
//           624 / 668 / 688 / 594, w = 24 646 / 681 / 696 / 593 (7 in 8 at Eq. 4: 667);
//   form C: Eq. 4 504 / 528 / 539 / 563, Eq. 5 464 / 478 / 492 / 506, w = 24 497 / 515 / 525 / 544
// (form C spends more ALU work per output on the float pair, so the FP64 pipe has room for all).
template <int FORM, int W = 32, int MAP = 0>
__device__ __forceinline__ constexpr uint32_t cvt_group_mask() {
  return FORM == kFormC ? 0xFu : ((FORM == kFormB && (MAP & kMapCvt)) ? 0xEu : 0x0u);
}

// The w = 24 fast path of fast24_ok / fast24_bits as PTX, from the raw 32-bit words (the draws
// are their top 24 bits). With A = u1 - 1 and B = u2 + 1,
// K = (3A + 2B) 2^24 + (4A + 3B) = A (3 2^24 + 4) + B (2 2^24 + 3) (a wide multiply and a wide
// multiply-add; below 2^51), and I = A 2^40 + (2A + B) 2^16 + (K >> 32) is one more wide
// multiply-add, (2A + B) 2^16 added to the word pair {K >> 32, A 2^8}; rounded as at w = 32.
// The check is 1 when 2^14 <= A <= 2^24 - 3 and the low word of K is below 2^32 - 16.
// (Measured on the bulk w = 24 fill with two checks a pair: 652 -> 663 Gsamples/s
// integer-only, 705 -> 710 balanced, against c1 = 3 u1 + 2 u2 - 1, c2 = 4 u1 + 3 u2 - 1 by four
// multiply-adds; folding the constants into a 64-bit addend instead lost 3 %.)
__device__ __forceinline__ uint64_t fast24_I_ptx(uint32_t x, uint32_t y, uint32_t one, uint32_t& ok) {
  uint64_t I;
  asm("{\n\t"
      ".reg .u64 K, P;\n\t"
      ".reg .u32 A, B, klo, khi, a, d, a8;\n\t"
      ".reg .pred p1, p2;\n\t"
      "shr.u32 A, %2, 8;\n\t"
      "shr.u32 B, %3, 8;\n\t"
      "mad.lo.u32 A, A, %4, -1;\n\t"
      "mad.lo.u32 B, B, %4, 1;\n\t"
      "mul.wide.u32 K, B, 33554435;\n\t"
      "mad.wide.u32 K, A, 50331652, K;\n\t"
      "mov.b64 {klo, khi}, K;\n\t"
      "mad.lo.u32 a, A, %4, -16384;\n\t"
      "setp.lt.u32 p1, a, 0xFFBFFE;\n\t"
      "setp.lt.and.u32 p2, klo, 0xFFFFFFF0, p1;\n\t"
      "selp.u32 %1, 1, 0, p2;\n\t"
      "mad.lo.u32 d, A, 2, B;\n\t"
      "shl.b32 a8, A, 8;\n\t"
      "mov.b64 P, {khi, a8};\n\t"
      "mad.wide.u32 %0, d, 65536, P;\n\t"
      "}"
      : "=l"(I), "=r"(ok)
      : "r"(x), "r"(y), "r"(one));
  return I;
}

// Both outputs of a pair (draws x, y and z, w) with one check for the two (measured on the bulk
// w = 24 fill, Gsamples/s: integer-only 667 against 662 with two checks, balanced 723 against
// 709, form C 566 against 552; PRNGD_W24_JOINT=0 builds the two-check form).
#ifndef PRNGD_W24_JOINT
#define PRNGD_W24_JOINT 1
#endif
__device__ __forceinline__ uint32_t fast24_pair_I_ptx(uint32_t x, uint32_t y, uint32_t z, uint32_t w, uint32_t one,
                                                      uint64_t& Ia, uint64_t& Ib) {
  uint32_t ok;
  asm("{\n\t"
      ".reg .u64 Ka, Pa, Kb, Pb;\n\t"
      ".reg .u32 Aa, Ba, kla, kha, aa, da, a8a, Ab, Bb, klb, khb, ab, db, a8b;\n\t"
      ".reg .pred p1, p2, p3, p4;\n\t"
      "shr.u32 Aa, %3, 8;\n\t"
      "shr.u32 Ba, %4, 8;\n\t"
      "shr.u32 Ab, %5, 8;\n\t"
      "shr.u32 Bb, %6, 8;\n\t"
      "mad.lo.u32 Aa, Aa, %7, -1;\n\t"
      "mad.lo.u32 Ba, Ba, %7, 1;\n\t"
      "mad.lo.u32 Ab, Ab, %7, -1;\n\t"
      "mad.lo.u32 Bb, Bb, %7, 1;\n\t"
      "mul.wide.u32 Ka, Ba, 33554435;\n\t"
      "mad.wide.u32 Ka, Aa, 50331652, Ka;\n\t"
      "mov.b64 {kla, kha}, Ka;\n\t"
      "mul.wide.u32 Kb, Bb, 33554435;\n\t"
      "mad.wide.u32 Kb, Ab, 50331652, Kb;\n\t"
      "mov.b64 {klb, khb}, Kb;\n\t"
      "mad.lo.u32 aa, Aa, %7, -16384;\n\t"
      "mad.lo.u32 ab, Ab, %7, -16384;\n\t"
      "setp.lt.u32 p1, aa, 0xFFBFFE;\n\t"
      "setp.lt.and.u32 p2, kla, 0xFFFFFFF0, p1;\n\t"
      "setp.lt.and.u32 p3, ab, 0xFFBFFE, p2;\n\t"
      "setp.lt.and.u32 p4, klb, 0xFFFFFFF0, p3;\n\t"
      "selp.u32 %0, 1, 0, p4;\n\t"
      "mad.lo.u32 da, Aa, 2, Ba;\n\t"
      "shl.b32 a8a, Aa, 8;\n\t"
      "mov.b64 Pa, {kha, a8a};\n\t"
      "mad.wide.u32 %1, da, 65536, Pa;\n\t"
      "mad.lo.u32 db, Ab, 2, Bb;\n\t"
      "shl.b32 a8b, Ab, 8;\n\t"
      "mov.b64 Pb, {khb, a8b};\n\t"
      "mad.wide.u32 %2, db, 65536, Pb;\n\t"
      "}"
      : "=r"(ok), "=l"(Ia), "=l"(Ib)
      : "r"(x), "r"(y), "r"(z), "r"(w), "r"(one));
  return ok;
}

struct PairOut {
  uint64_t v0, v1;
  uint32_t x, y, z, w, rej;
};

// Exact replay of two outputs (w = 32 or 24). (x, y, z, w) is the state after the pair's 4-draw
// block; it is rewound 4 steps to the block's start, then the two outputs are redrawn with
// in-order rejects (pair rule, or Algorithm 1's when `single`) and converted exactly.
template <int FORM, int W, int MAP = 0>
__device__ __noinline__ PairOut slow_pair(uint32_t x, uint32_t y, uint32_t z, uint32_t w, uint32_t rej,
                                          uint32_t single) {
  constexpr int wbits = W;
  XorShift128 st{x, y, z, w};
  xs_prev(st);
  xs_prev(st);
  xs_prev(st);
  xs_prev(st);
  const uint32_t top = (wbits == 32) ? 0xFFFFFFFFu : ((1u << wbits) - 1u);
  uint64_t v[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    uint32_t u1 = draw<0>(st, wbits), u2 = draw<0>(st, wbits);
    take_accepted<0>(u1, u2, st, rej, wbits, top, single);
    v[k] = exact_bc<W, FORM, MAP>(u1, u2);
  }
  return PairOut{v[0], v[1], st.x, st.y, st.z, st.w, rej};
}

// The output of an accepted pair by the fastest valid path, with the pair path's own code: at
// w = 32 and w = 24 (forms B and C) the fast path (PTX where the pair path uses PTX), then the
// medium path for small values, else the exact conversion.
// cvt: round the fast path's value by the conversion instruction (as the pair path does for the
// outputs cvt_group_mask selects).
template <int W, int FORM, int MAP>
__device__ __forceinline__ uint64_t convert_accepted(uint32_t u1, uint32_t u2, const FillParams& p,
                                                     bool cvt = false) {
  if constexpr ((W == 32 || W == 24) && (FORM == kFormB || FORM == kFormC)) {
    constexpr bool kComp = (MAP & kMapOneMinus) != 0;
    constexpr uint32_t top = (W == 32) ? 0xFFFFFFFFu : 0xFFFFFFu;
    const uint32_t a1 = kComp ? top - u1 : u1, a2 = kComp ? top - u2 : u2;
    uint64_t bits;
    if constexpr (W == 32 && (MAP & kMapEq5) != 0) {
      uint32_t ok;
      const uint64_t I = fast32_I_ptx_t<4, -4, kComp ? 1 : 0, 0xFFFFFFC0u>(a1, a2, p.one, ok);
      bits = cvt ? bits_from_I_cvt(I, p.one) : bits_from_I_int(I, p.one);
      if (!ok) {
        if (medium32_eq5_ok(a1, a2)) bits = medium32_eq5_bits(a1, a2, fast32_eq5_Y(a1, a2), kComp ? 1u : 0u);
        else return convert_exact<W, FORM, MAP>(u1, u2, p);
      }
    } else if constexpr (W == 32) {
      uint32_t ok;
      const uint64_t I = fast32_I_ptx_t<3, -1, 1, 0xFFFFFFF8u>(a1, a2, p.one, ok);
      bits = cvt ? bits_from_I_cvt(I, p.one) : bits_from_I_int(I, p.one);
      if (!ok) {
        const uint64_t X = fast32_X(a1, a2);
        if (medium32_ok(a1, X, a2)) bits = medium32_bits(a1, a2, X);
        else return convert_exact<W, FORM, MAP>(u1, u2, p);
      }
    } else if constexpr ((MAP & kMapEq5) != 0) {
      const uint64_t K = fast24_eq5_K(a1, a2);
      if (fast24_eq5_ok(a1, K)) {
        const uint64_t I = fast24_eq5_I(a1, a2, K, kComp ? 0x10000u : 0u);
        bits = cvt ? bits_from_I_cvt(I, p.one) : bits_from_I_int(I, p.one);
      } else if (medium24_eq5_ok(a1, a2)) {
        bits = medium24_eq5_bits(a1, a2, kComp ? 1u : 0u);
      } else {
        return convert_exact<W, FORM, MAP>(u1, u2, p);
      }
    } else {
      uint32_t ok;
      const uint64_t I = fast24_I_ptx(a1 << 8, a2 << 8, p.one, ok);  // raw words: the draws in their top 24 bits
      bits = cvt ? bits_from_I_cvt(I, p.one) : bits_from_I_int(I, p.one);
      if (!ok) {
        const uint64_t K = fast24_K(a1, a2);
        if (medium24_ok(a1, K, a2)) bits = medium24_bits(a1, a2, K);
        else return convert_exact<W, FORM, MAP>(u1, u2, p);
      }
    }
    return FORM == kFormC ? f32pair_from_bits(bits) : bits;  // the fast and medium values are not 0
  } else {
    return convert_exact<W, FORM, MAP>(u1, u2, p);
  }
}

// Two outputs of a w = 32 or w = 24 stream (forms B and C) from one 4-draw block, with one
// branch for the pair. A small value takes the inline medium path; a reject or a value near
// a rounding boundary replays the pair exactly from the block's starting state.
// ca, cb: round output a / b by the conversion instruction (w = 32, Eq. 4; see
// cvt_group_mask); callers pass constants.
template <int W, int FORM, int MAP = 0>
__device__ __forceinline__ void next_pair(XorShift128& st, uint32_t& rej, const FillParams& p, uint64_t& v0,
                                          uint64_t& v1, bool ca = false, bool cb = false) {
  xs_block4(st);
  // 1 - z: the arithmetic runs on the complemented draws (the state itself is not changed);
  // complementing the 32-bit word complements its top w bits.
  constexpr bool kComp = (MAP & kMapOneMinus) != 0;
  const uint32_t neg_one = 0u - p.one;
  const uint32_t dx = kComp ? complement_fma(st.x, neg_one) : st.x, dy = kComp ? complement_fma(st.y, neg_one) : st.y;
  const uint32_t dz = kComp ? complement_fma(st.z, neg_one) : st.z, dw = kComp ? complement_fma(st.w, neg_one) : st.w;
  uint32_t ok;
  if constexpr ((MAP & kMapEq5) != 0) {
    // Eq. 5. Small values take the inline medium path (w = 32 and 24); rejects and boundary
    // values replay the pair exactly.
    if constexpr (W == 32) {
      uint64_t Ia, Ib;
      ok = fast32_I_pair<4, -4, kComp ? 1 : 0, 0xFFFFFFC0u>(dx, dy, dz, dw, p.one, ca || cb, Ia, Ib);
      v0 = ca ? bits_from_I_cvt(Ia, p.one) : bits_from_I_int(Ia, p.one);
      v1 = cb ? bits_from_I_cvt(Ib, p.one) : bits_from_I_int(Ib, p.one);
    } else {
      const uint32_t u1a = dx >> 8, u2a = dy >> 8, u1b = dz >> 8, u2b = dw >> 8;
      const uint64_t Ka = fast24_eq5_K(u1a, u2a), Kb = fast24_eq5_K(u1b, u2b);
      ok = fast24_eq5_ok(u1a, Ka) & fast24_eq5_ok(u1b, Kb);
      const uint64_t Ia = fast24_eq5_I(u1a, u2a, Ka, kComp ? 0x10000u : 0u);
      const uint64_t Ib = fast24_eq5_I(u1b, u2b, Kb, kComp ? 0x10000u : 0u);
      v0 = ca ? bits_from_I_cvt(Ia, p.one) : bits_from_I_int(Ia, p.one);
      v1 = cb ? bits_from_I_cvt(Ib, p.one) : bits_from_I_int(Ib, p.one);
    }
    if (__builtin_expect(ok == 0, 0)) {
      bool replay = false;
      if constexpr (W == 32) {
        const uint64_t Ya = fast32_eq5_Y(dx, dy), Yb = fast32_eq5_Y(dz, dw);
        if (!fast32_eq5_ok(dx, Ya)) {
          if (medium32_eq5_ok(dx, dy)) v0 = medium32_eq5_bits(dx, dy, Ya, kComp ? 1u : 0u); else replay = true;
        }
        if (!fast32_eq5_ok(dz, Yb)) {
          if (medium32_eq5_ok(dz, dw)) v1 = medium32_eq5_bits(dz, dw, Yb, kComp ? 1u : 0u); else replay = true;
        }
      } else {
        const uint32_t u1a = dx >> 8, u2a = dy >> 8, u1b = dz >> 8, u2b = dw >> 8;
        if (!fast24_eq5_ok(u1a, fast24_eq5_K(u1a, u2a))) {
          if (medium24_eq5_ok(u1a, u2a)) v0 = medium24_eq5_bits(u1a, u2a, kComp ? 1u : 0u); else replay = true;
        }
        if (!fast24_eq5_ok(u1b, fast24_eq5_K(u1b, u2b))) {
          if (medium24_eq5_ok(u1b, u2b)) v1 = medium24_eq5_bits(u1b, u2b, kComp ? 1u : 0u); else replay = true;
        }
      }
      if (replay) {
        const PairOut o = slow_pair<kFormB, W, MAP>(st.x, st.y, st.z, st.w, rej, p.single);
        v0 = o.v0;
        v1 = o.v1;
        rej = o.rej;
        st = XorShift128{o.x, o.y, o.z, o.w};
      }
    }
    if (FORM == kFormC) {
      v0 = v0 ? f32pair_from_bits(v0) : 0ull;  // z' = 0 is a pair of zeros
      v1 = v1 ? f32pair_from_bits(v1) : 0ull;
    }
    return;
  }
  if constexpr (W == 32) {
    uint64_t Ia, Ib;
    ok = fast32_I_pair<3, -1, 1, 0xFFFFFFF8u>(dx, dy, dz, dw, p.one, ca || cb, Ia, Ib);
    v0 = ca ? bits_from_I_cvt(Ia, p.one) : bits_from_I_int(Ia, p.one);
    v1 = cb ? bits_from_I_cvt(Ib, p.one) : bits_from_I_int(Ib, p.one);
  } else {
    uint64_t Ia, Ib;
#if PRNGD_W24_JOINT
    ok = fast24_pair_I_ptx(dx, dy, dz, dw, p.one, Ia, Ib);
#else
    uint32_t ok0, ok1;
    Ia = fast24_I_ptx(dx, dy, p.one, ok0);
    Ib = fast24_I_ptx(dz, dw, p.one, ok1);
    ok = ok0 & ok1;
#endif
    v0 = ca ? bits_from_I_cvt(Ia, p.one) : bits_from_I_int(Ia, p.one);
    v1 = cb ? bits_from_I_cvt(Ib, p.one) : bits_from_I_int(Ib, p.one);
  }
  if (__builtin_expect(ok == 0, 0)) {
    // Almost always a small value (A < 2^22 at w = 32): the inline medium path. Rejects and
    // values near a rounding boundary replay the pair exactly.
    bool replay = false;
    if constexpr (W == 32) {
      const uint64_t Xa = fast32_X(dx, dy), Xb = fast32_X(dz, dw);
      if (!fast32_ok(dx, Xa)) {
        if (medium32_ok(dx, Xa, dy)) v0 = medium32_bits(dx, dy, Xa); else replay = true;
      }
      if (!fast32_ok(dz, Xb)) {
        if (medium32_ok(dz, Xb, dw)) v1 = medium32_bits(dz, dw, Xb); else replay = true;
      }
    } else {
      const uint32_t u1a = dx >> 8, u2a = dy >> 8, u1b = dz >> 8, u2b = dw >> 8;
      const uint64_t Ka = fast24_K(u1a, u2a), Kb = fast24_K(u1b, u2b);
      if (!fast24_ok(u1a, Ka)) {
        if (medium24_ok(u1a, Ka, u2a)) v0 = medium24_bits(u1a, u2a, Ka); else replay = true;
      }
      if (!fast24_ok(u1b, Kb)) {
        if (medium24_ok(u1b, Kb, u2b)) v1 = medium24_bits(u1b, u2b, Kb); else replay = true;
      }
    }
    if (replay) {
      const PairOut o = slow_pair<kFormB, W, MAP>(st.x, st.y, st.z, st.w, rej, p.single);
      v0 = o.v0;
      v1 = o.v1;
      rej = o.rej;
      st = XorShift128{o.x, o.y, o.z, o.w};
    }
  }
  if (FORM == kFormC) {
    v0 = f32pair_from_bits(v0);
    v1 = f32pair_from_bits(v1);
  }
}

// ------------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(map),
               "r"(src), "r"(x), "r"(y)
               : "memory");
}
// The same with an L2 evict_last policy: a box whose rows start inside a 128-byte line leaves
// the line's other part to the neighbouring box, and under the default policy the part written
// first can leave L2 before the line is whole (measured on rows 16, 32, 64 or 96 bytes into a
// line: 1.55 ms per 2^30 outputs against 1.43 aligned; 1.44-1.47 with this policy, whose cost on
// aligned rows is 0.4 %).
__device__ __forceinline__ void tma_store_2d_keep(const CUtensorMap* map, uint32_t src, int x, int y) {
  asm volatile("{\n\t"
               ".reg .b64 pol;\n\t"
               "createpolicy.fractional.L2::evict_last.b64 pol, 1.0;\n\t"
               "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%2, %3}], [%1], pol;\n\t"
               "}" ::"l"(map), "r"(src), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint64_t a, uint64_t b) {
  asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b) : "memory");
}

// ------------------------------------------------------------------------ kernels
// TMA path. Warp g owns streams 32g .. 32g+31 (lane = row of the tile). Per chunk of 16
// outputs each lane computes its 16 outputs in registers, writes them as 8 x 16-byte pieces
// into the warp's tile with the 128-byte swizzle (piece c of row r at r*128 + ((c ^ (r & 7))
// * 16)), and lane 0 issues one 2D bulk tensor store of the 32 x 16 box. Rows past n_streams
// and columns past per_stream fall outside the tensor and are not written. NBUF tiles per
// warp let the next chunk's staging proceed while the previous store still reads shared memory.
// SHIFT: rows start 16 bytes into a 32-byte sector (every row, as per_stream is a multiple of 4),
// and the map starts 2 outputs into each row, on a sector boundary, with the rows' own pitch:
// each lane makes its row's first two outputs first, keeps them in registers while the rest of
// the row goes out in whole sectors, and writes them with one 16-byte store at the end.
template <int W, int FORM, int NBUF, int MAP = 0, bool SHIFT = false>
__global__ void __launch_bounds__(256, 4) fill_tma_kernel(const FillParams p,
                                                       const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base = (smem_addr(smem_raw) + 1023u) & ~1023u;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint64_t warp_global = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (warp_global * 32 >= p.n_streams) return;  // the whole warp is past the last stream
  const uint64_t stream = warp_global * 32 + lane;
  const bool active = stream < p.n_streams;
  uint4 s4 = active ? p.state[stream] : make_uint4(1u, 2u, 3u, 4u);
  XorShift128 st{s4.x, s4.y, s4.z, s4.w};
  uint32_t rej = 0;
  const uint32_t tile0 = base + (uint32_t)warp * NBUF * kTileBytes;
  const uint32_t row_off = (uint32_t)lane * 128u;
  const uint32_t sw = (uint32_t)(lane & 7);
  const int y0 = (int)(warp_global * 32);
  uint64_t head0 = 0, head1 = 0;
  if constexpr (SHIFT) {
    if constexpr ((W == 32 || W == 24) && (FORM == kFormB || FORM == kFormC)) {
      next_pair<W, FORM, MAP>(st, rej, p, head0, head1, cvt_group_mask<FORM, W, MAP>() & 1u,
                              (cvt_group_mask<FORM, W, MAP>() >> 1) & 1u);
    } else {
      head0 = next_output<W, FORM, MAP>(st, rej, p);
      head1 = next_output<W, FORM, MAP>(st, rej, p);
    }
  }
  const uint64_t span = p.per_stream - (SHIFT ? 2u : 0u);  // outputs the map covers per row
  uint32_t chunk_idx = 0;
  for (uint64_t x0 = 0; x0 < span; x0 += kChunk, ++chunk_idx) {
    uint64_t v[kChunk];
    const uint64_t left = span - x0;
    if (left >= (uint64_t)kChunk) {
      if constexpr ((W == 32 || W == 24) && (FORM == kFormB || FORM == kFormC)) {
#pragma unroll
        for (int j = 0; j < kChunk; j += 2)
          next_pair<W, FORM, MAP>(st, rej, p, v[j], v[j + 1], (cvt_group_mask<FORM, W, MAP>() >> (j & 3)) & 1u,
                                  (cvt_group_mask<FORM, W, MAP>() >> ((j + 1) & 3)) & 1u);
      } else if constexpr (FORM == kFormA && W == 32 && (MAP & kMapCvt) != 0) {
        // balanced form A: one output in eight still converts on the FP64 pipe (kFormAF), which
        // the integer rounding leaves idle: measured 446 against 425 Gsamples/s for none (one in
        // two: 352, in four: 401). Not at w = 24, where n < 2^53 converts exactly and cheaply
        // (517 against 460).
#pragma unroll
        for (int j = 0; j < kChunk; ++j)
          v[j] = (j % 8 == 0) ? next_output<W, kFormAF, MAP>(st, rej, p) : next_output<W, FORM, MAP>(st, rej, p);
      } else {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) v[j] = next_output<W, FORM, MAP>(st, rej, p);
      }
    } else {
#pragma unroll
      for (int j = 0; j < kChunk; ++j) v[j] = (j < (int)left) ? next_output<W, FORM, MAP>(st, rej, p) : 0ull;
    }
    const uint32_t tile = tile0 + (chunk_idx % NBUF) * kTileBytes;
    if (lane == 0) bulk_wait_read<NBUF - 1>();
    __syncwarp();
    // piece c at row + ((c ^ sw) << 4) = (row | (sw << 4)) ^ (c << 4): bits 4..6 of a row's
    // address are zero (1024-byte aligned tiles, 128-byte rows), so one xor per store
    const uint32_t rowb = (tile + row_off) | (sw << 4);
#pragma unroll
    for (int c = 0; c < kChunk / 2; ++c) st_shared_v2(rowb ^ ((uint32_t)c << 4), v[2 * c], v[2 * c + 1]);
    fence_async_shared();
    __syncwarp();
    if (lane == 0) {
      if (SHIFT || p.keep_lines)
        tma_store_2d_keep(&tmap, tile, (int)x0, y0);
      else
        tma_store_2d(&tmap, tile, (int)x0, y0);
      bulk_commit();
    }
  }
  if (lane == 0) bulk_wait_all();
  if (active) {
    if constexpr (SHIFT) *(ulonglong2*)(p.out + stream * p.per_stream) = make_ulonglong2(head0, head1);
    p.state[stream] = make_uint4(st.x, st.y, st.z, st.w);
    if (p.rejects) p.rejects[stream] = rej;
  }
}

// Generic store path (any alignment, any per_stream): the warp stages its 32 x 16 tile with a
// padded row pitch of 17 words and writes it back row by row, 16 lanes per row, so each store
// instruction covers two 128-byte row segments.
template <int W, int FORM, int MAP = 0>
__global__ void __launch_bounds__(256) fill_plain_kernel(const FillParams p) {
  __shared__ uint64_t tiles[8][32 * (kChunk + 1)];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const uint64_t warp_global = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const uint64_t stream = warp_global * 32 + lane;
  const bool active = stream < p.n_streams;
  uint4 s4 = active ? p.state[stream] : make_uint4(1u, 2u, 3u, 4u);
  XorShift128 st{s4.x, s4.y, s4.z, s4.w};
  uint32_t rej = 0;
  uint64_t* tile = tiles[warp];
  for (uint64_t x0 = 0; x0 < p.per_stream; x0 += kChunk) {
    const uint64_t left = p.per_stream - x0;
    const int cnt = left >= (uint64_t)kChunk ? kChunk : (int)left;
#pragma unroll
    for (int j = 0; j < kChunk; ++j)
      if (j < cnt) tile[lane * (kChunk + 1) + j] = next_output<W, FORM, MAP>(st, rej, p);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kChunk; ++i) {
      const int idx = i * 32 + lane;
      const int row = idx / kChunk, col = idx % kChunk;
      const uint64_t s = warp_global * 32 + row;
      if (col < cnt && s < p.n_streams) p.out[s * p.per_stream + x0 + col] = tile[row * (kChunk + 1) + col];
    }
    __syncwarp();
  }
  if (active) {
    p.state[stream] = make_uint4(st.x, st.y, st.z, st.w);
    if (p.rejects) p.rejects[stream] = rej;
  }
}

}  // namespace prngd
