/*
 * prngd.h -- C ABI of the GB300 PRNGD library (libprngd.so).
 *
 * Bulk generation of extended-precision uniform variates by the construction of
 * V. Demchik and A. Gulov, "Increasing precision of uniform pseudorandom number generators"
 * (arXiv:1401.8230), Section 2: two w-bit base draws x1, x2 are combined as z = x1 + k x2 with
 * k = 2^-w (Eq. 1); a pair whose x1 lies on a range end is rejected and the next pair of the
 * same stream is taken (the discrete accept-reject rule after Fig. 1); the accepted z is
 * mapped onto the unit interval by Eq. 4, z' = (z - (a0 + k b)) / (a - a0 - k (b - b0)).
 *
 * With base draws x1 = a0 + u1 k, x2 = b0 + u2 k (integers u1, u2 in [0, 2^w - 1]) Eq. 4 is
 * exactly z' = n / D with n = u1 2^w + u2 - (2^w - 1) and D = (2^w - 1)^2, for any offsets
 * a0, b0; accepted outputs are the D - 1 equally spaced points 1/D .. (D-1)/D.
 *
 * Streams: stream s is Marsaglia's xorshift128 seeded from splitmix64 outputs 2s and 2s+1 of
 * the sequence started at `seed`; a w-bit draw is the top w bits of a 32-bit output. Attempt
 * j of a stream uses draws 2j (x1) and 2j+1 (x2). Every call continues each stream from its
 * device-resident state, so a stream's output sequence never depends on launch shapes.
 *
 * Conventions for every entry point:
 *  - Return value: PRNG_OK (0) or one of the PRNG_E* codes below. No exception crosses the ABI.
 *    prng_last_error() gives a message for the calling thread's most recent failure.
 *  - "device pointer" means memory the caller allocated on the current CUDA device
 *    (cudaMalloc, a torch tensor, ...). The caller owns it; the library never frees it.
 *  - `cuda_stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Device work is enqueued on it and the call returns without synchronising, unless the
 *    entry point says otherwise.
 *  - A handle is not thread-safe: calls on one handle must come from one thread at a time,
 *    and two fills on one handle must not overlap on the GPU (they continue the same state).
 */
#ifndef PRNGD_H
#define PRNGD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define PRNG_OK 0
#define PRNG_EINVAL 1   /* bad argument: null pointer, w out of [2, 32], zero streams,     */
                        /* ranges that break the step condition, unknown form, ...         */
#define PRNG_ENOMEM 2   /* a device or pinned-host allocation failed                       */
#define PRNG_ECUDA 3    /* a CUDA runtime call or kernel launch failed (see prng_last_error) */
#define PRNG_ETIMEOUT 4 /* a bounded device or host wait gave up                           */
#define PRNG_EBUSY 5    /* admission refused: the queue or the memory budget is full        */
#define PRNG_ENOTFOUND 6 /* unknown ticket                                                  */

/* Output forms. All three are functions of the same accepted n; each output is 8 bytes. */
#define PRNG_FORM_A_FP64 0    /* double RN(RN(n) * C_w), C_w = RN(1/D): the FP64 sequence   */
                              /* (u64 -> f64 conversion, multiply); at most 1 ulp from      */
                              /* RN(n/D) (see PRNG_MODE_BALANCED)                            */
#define PRNG_FORM_B_INTBITS 1 /* double RN(n/D), correctly rounded, built with integer ops  */
                              /* only (see PRNG_MODE_BALANCED)                          */
#define PRNG_FORM_C_F32PAIR 2 /* two floats (hi, lo): hi = RN32(d), lo = RN32(d - hi), with */
                              /* d the form-B value; stored interleaved hi, lo; the exact    */
                              /* sum hi + lo is within 8.5 ulp64 of n/D (prng_fill_f32pair)  */
#define PRNG_FORM_L_ALGO1 4   /* double: Algorithm 1's Z evaluated literally in FP64, one IEEE */
                              /* operation at a time (prng_fill_mode only)                    */

/* Modes of prng_fill_mode, bit flags (0 = the map of Eq. 4 with pair rejects). */
#define PRNG_MODE_EQ5 1             /* the map of Eq. 5 (one generator: Eq. 6): z' = (1 - k^2) */
                                    /* (n - 1)/(D - 2), range [0, 1 - k^2] with k = 2^-w        */
#define PRNG_MODE_ONE_MINUS 2       /* output 1 - z' instead of z' (Section 2: excludes zero)  */
#define PRNG_MODE_SINGLE_REDRAW 4   /* Algorithm 1's reject loop: redraw only r1, then draw r2  */
#define PRNG_MODE_BALANCED 8        /* forms A and B: the same bits by a route that shares the  */
                                    /* work between the integer and FP64 pipes                  */

typedef struct prng_ctx* prng_t;

/* Base generators of a handle's streams. */
#define PRNG_GEN_XORSHIFT128 0 /* Marsaglia's xor128 (prng_create): every entry point            */
#define PRNG_GEN_MRG32K3A 1    /* L'Ecuyer's MRG32k3a (prng_create_mrg32k3a): the fills only     */

/* Human-readable message for the calling thread's last failed call ("" if none). */
const char* prng_last_error(void);

/* Library version as major*10000 + minor*100 + patch. */
int prng_version(void);

/*
 * prng_create -- allocate and seed `n_streams` streams on the current CUDA device.
 * Section 2 (Eq. 1, Eq. 4): w is the precision of one base draw (2 <= w <= 32) and
 * [a0, a], [b0, b] are the ranges of x1 and x2. The discrete accept-reject rule assumes both
 * are grids of step k = 2^-w, so a - a0 and b - b0 must both equal exactly (2^w - 1) 2^-w;
 * any a0, b0 satisfying this give the same outputs (the offsets cancel in Eq. 4).
 * Streams 0 .. n_streams-1 of `seed` are seeded on the device; the call synchronises.
 * Errors: PRNG_EINVAL (out == NULL, n_streams == 0 or > 2^32, w outside [2, 32], ranges with
 * another step), PRNG_ENOMEM, PRNG_ECUDA. On error *out is set to NULL.
 */
int prng_create(prng_t* out, uint64_t seed, uint64_t n_streams, int w, double a0, double a,
                double b0, double b);

/*
 * prng_create_mrg32k3a -- streams of L'Ecuyer's MRG32k3a (Operations Research 47(1), 1999), one
 * of the base generators Section 2 recommends. Its output z in [1, m1] (m1 = 2^32 - 209) is the
 * draw u = z - 1 on a grid of M = m1 points with step k = 1/M, and Section 2 holds with 2^w
 * replaced by M: u1 in {0, M - 1} is rejected (pair rule) and z' = n/D with
 * n = u1 M + u2 - (M - 1), D = (M - 1)^2. Stream s is seeded from splitmix64 outputs 3s, 3s+1
 * and 3s+2 of `seed` (six 32-bit words, low first, reduced modulo m1 and m2; an all-zero
 * component gets 1 as its first word). 32 bytes of device state per stream.
 * Such a handle takes prng_fill_f64, prng_fill_f32pair, prng_fill_mode (forms A, B, C; mode 0 or
 * PRNG_MODE_BALANCED),
 * prng_fill_f64_host(_noalloc) and prng_state_*; the entry points built on xorshift128's
 * structure (fused statistics, batches, serving, skip, split) answer PRNG_EINVAL.
 * Errors: PRNG_EINVAL (out == NULL, n_streams == 0 or > 2^32), PRNG_ENOMEM, PRNG_ECUDA.
 */
int prng_create_mrg32k3a(prng_t* out, uint64_t seed, uint64_t n_streams);

/* PRNG_GEN_* of a handle's streams; -1 for NULL. */
int prng_generator(prng_t h);

/* Release the handle and its device memory (synchronises the device first). NULL is a no-op. */
int prng_destroy(prng_t h);

/* Number of streams and w of a handle (either pointer may be NULL). */
int prng_get_info(prng_t h, uint64_t* n_streams, int* w);

/*
 * prng_fill_f64 -- per_stream outputs of every stream, as doubles, stream-major:
 * d_out[s * per_stream + i] is output i of stream s in this call (Algorithm 1 per output;
 * accept-reject as in Section 2, pair semantics). form is PRNG_FORM_A_FP64 or
 * PRNG_FORM_B_INTBITS. d_out: device pointer to n_streams * per_stream doubles (8-byte
 * aligned; 16-byte alignment and an even per_stream select the TMA store path).
 * d_rejects (nullable): device pointer to n_streams uint64, set to the number of rejected
 * pairs each stream consumed in this call (8-byte aligned). per_stream == 0 is a no-op.
 * n_streams * per_stream may not exceed 2^60 outputs (every byte offset fits in 64 bits).
 * Errors: PRNG_EINVAL (null handle or d_out, misaligned d_out or d_rejects, bad form, more
 * than 2^60 outputs), PRNG_ECUDA.
 */
int prng_fill_f64(prng_t h, double* d_out, uint64_t per_stream, int form, uint64_t* d_rejects,
                  void* cuda_stream);

/*
 * prng_fill_f32pair -- as prng_fill_f64 with form C: d_out holds 2 * n_streams * per_stream
 * floats, element 2*(s*per_stream+i) = hi and 2*(s*per_stream+i)+1 = lo of output i of
 * stream s, with hi = RN32(d), lo = RN32(d - hi) and d = RN(n/D).
 * Error bound: |hi + lo - n/D| < 8.5 ulp(n/D), ulp(V) = 2^(floor(log2 V) - 52). d is within
 * half an ulp of n/D. If |d - hi| is half an FP32 ulp of d it is a power of two and lo is
 * exact; otherwise |d - hi| lies a binade lower, where an FP32 ulp is 16 FP64 ulps, so lo's
 * rounding adds at most 8. hi + lo (at most 48 significant bits) is a double at most 8
 * steps from d. Measured on 2^30 outputs at w = 32: 8 steps, error up to 8.4999 ulp.
 */
int prng_fill_f32pair(prng_t h, float* d_out, uint64_t per_stream, uint64_t* d_rejects,
                      void* cuda_stream);

/*
 * prng_fill_mode -- as prng_fill_f64 / prng_fill_f32pair, for any form and mode.
 * form: PRNG_FORM_A_FP64, PRNG_FORM_B_INTBITS, PRNG_FORM_C_F32PAIR (2 floats per output) or
 * PRNG_FORM_L_ALGO1. mode: an OR of PRNG_MODE_* bits.
 *  - PRNG_MODE_EQ5 (Section 2, Eq. 5 and Eq. 6): x1 = a0 + k, x2 = b0 map to 0 and
 *    x1 = a - k, x2 = b to 1 - k^2; the output is (1 - k^2) m / (D - 2) with
 *    m = (u1 - 1) 2^w + u2. Form B is its correctly rounded double, form A RN(RN(m) C5) with
 *    C5 = RN((1 - k^2)/(D - 2)), form L Eq. 6 in FP64. At w = 32 the top value rounds to 1.0.
 *  - PRNG_MODE_ONE_MINUS (Section 2): 1 - z'. Form B: the correctly rounded 1 - z' (under
 *    Eq. 4 it equals z' of the complemented draws); forms A and L: one more FP64 subtraction.
 *  - PRNG_MODE_SINGLE_REDRAW (Algorithm 1): a rejected r1 is redrawn alone and r2 is drawn
 *    after the accepted r1; d_rejects then counts redrawn r1 values.
 *  - PRNG_MODE_BALANCED: the same values by a faster route that balances the integer and
 *    FP64 pipes. Form B builds the correctly rounded double with integer instructions only;
 *    with this bit, 3 of every 4 outputs of a row (w = 32 and 24) take I = floor(V 2^64) to
 *    double by the u64 -> f64 conversion instead (as RN(I | 1), the same rounding). Form A
 *    takes RN(n) by the conversion instruction; with this bit, by integer rounding (exact, the
 *    same double) for 7 of every 8 outputs at w = 32 and all at other w. No effect on forms C
 *    (which always rounds on the FP64 pipe; it has no integer-only definition) and L.
 * Form L with PRNG_MODE_SINGLE_REDRAW is Algorithm 1 as printed. mode = 0 and forms A, B, C
 * give exactly the outputs of prng_fill_f64 / prng_fill_f32pair. The streams advance as the
 * reject rule consumes draws. d_out: device memory, 8-byte aligned; the fast (TMA) path needs
 * 16-byte alignment and an even per_stream.
 * Errors: PRNG_EINVAL (null handle or d_out, misaligned d_out or d_rejects, unknown form or
 * mode bits, more than 2^60 outputs), PRNG_ECUDA.
 */
int prng_fill_mode(prng_t h, void* d_out, uint64_t per_stream, int form, int mode, uint64_t* d_rejects,
                   void* cuda_stream);

/*
 * prng_skip -- advance every stream of the handle by `draws` base draws (2 per attempt under
 * the pair rule), as if that many draws had been made and discarded. xorshift128 is linear
 * over GF(2), so the jump is g(T) applied to each state with g = x^draws mod P, P the
 * characteristic polynomial of the generator's step T: the cost does not depend on `draws`.
 * Asynchronous on cuda_stream. Errors: PRNG_EINVAL (null handle), PRNG_ECUDA.
 */
int prng_skip(prng_t h, uint64_t draws, void* cuda_stream);

/*
 * prng_fill_split -- the outputs of prng_fill_mode (same values, same reject counts, same
 * state afterwards), computed with each stream cut into `segments` pieces that run in
 * parallel, so that a few long streams fill the GPU. Under the pair rule (Section 2) attempt a
 * of a stream always uses draws 2a and 2a + 1, so piece j starts from the state jumped ahead by
 * 2 j (per_stream / segments) draws; the outputs it owns are shifted back by the rejects of the
 * pieces before it (rare: 2/2^w per attempt), which the call resolves on the device.
 * segments: a power of two (<= 2^23) dividing per_stream, or 0 to let the library choose
 * (1 means no split). The single-redraw rule of Algorithm 1 has no fixed attempt boundaries and
 * is refused. Scratch (28 bytes per piece) is kept with the handle.
 * Errors: PRNG_EINVAL (as prng_fill_mode; PRNG_MODE_SINGLE_REDRAW; bad segments),
 * PRNG_ENOMEM, PRNG_ECUDA.
 */
int prng_fill_split(prng_t h, void* d_out, uint64_t per_stream, int form, int mode, uint32_t segments,
                    uint64_t* d_rejects, void* cuda_stream);

/*
 * prng_convert_pairs -- the method's conversion (Section 2: Eq. 4, or Eq. 5 / 1 - z by `mode`)
 * applied to given w-bit base draws, with the same device code as the fills: output i is the
 * form-`form` value (A, B, C or L) of the pair (d_u1[i], d_u2[i]) (values taken modulo 2^w).
 * A pair whose u1 is rejected (0 or 2^w - 1) gives all-ones bits (a NaN); the reject rule bit of
 * `mode` is ignored (there is no stream to redraw from). For callers with their own base draws,
 * and for testing the conversions on chosen inputs. No handle; asynchronous on cuda_stream.
 * At w = 32 under Eq. 4 (forms B and C) pair i is rounded by the route the fills use for output
 * i mod 4 of a row (integer normalisation or the u64 -> f64 conversion instruction); both give
 * the same bits.
 * d_u1, d_u2: device arrays of n uint32 (4-byte aligned); d_out: device array of n 8-byte
 * outputs (8-byte aligned).
 * Errors: PRNG_EINVAL (w outside [2, 32], unknown form or mode bits, null or misaligned
 * pointers), PRNG_ECUDA.
 */
int prng_convert_pairs(int w, int form, int mode, const uint32_t* d_u1, const uint32_t* d_u2, uint64_t n,
                       uint64_t* d_out, void* cuda_stream);

/*
 * prng_fill_f64_host -- end-to-end fill into HOST memory: the same values as prng_fill_f64
 * (the streams advance identically) into `host_out` (n_streams * per_stream doubles). The
 * values are generated on the device in slices (two 256 MiB staging buffers kept with the
 * handle) and copied back by the copy engines, the next slice being generated while the
 * previous one is copied; a pinned host_out is copied into directly at the host link's rate.
 * The call synchronises. host_rejects (nullable, host memory) receives per-stream reject counts.
 * Errors: PRNG_EINVAL, PRNG_ENOMEM (staging buffers), PRNG_ECUDA.
 */
int prng_fill_f64_host(prng_t h, double* host_out, uint64_t per_stream, int form,
                       uint64_t* host_rejects);

/*
 * prng_fill_f64_host_noalloc -- the paper has no counterpart; this is a library convenience.
 * Same values, reject counts and stream advance as prng_fill_f64_host, but the call
 * allocates nothing: no cudaMalloc, no cudaFree, no pinned buffers, no streams. It is for
 * callers that cannot allocate device memory when they need numbers. Examples: a process
 * whose GPU memory already belongs to another allocator (a framework pool that reserved the
 * device), a service that fixes its footprint at start-up and must not fail with
 * out-of-memory later, or a loop that cannot afford the device-wide synchronisation that
 * cudaMalloc/cudaFree may cause. (prng_create still allocates the stream state, once.)
 * Device staging is a fixed array inside the library of PRNG_NOALLOC_VALUE_BYTES +
 * 8 * PRNG_NOALLOC_MAX_SLICE_STREAMS bytes (17 MiB); every GPU that loads the library holds
 * it until the process exits.
 * Work runs on `cuda_stream` (NULL = legacy default stream) in slices that fit the array,
 * one after another; the call synchronises that stream before returning. It orders itself
 * after nothing else: earlier asynchronous work on this handle queued on another stream
 * (a prng_fill_* or prng_fused_stats that is still running) must be complete or ordered
 * before `cuda_stream` by the caller (an event wait, or a synchronise), or this call reads
 * stream states that are still being updated. prng_fill_f64_host needs no such care: it
 * synchronises the device first. The first call on a
 * device looks up the array's device address (once per device); make that first call
 * before any stream capture.
 * All calls share the one array, and it keeps the last call's contents. Calls that overlap
 * on the GPU (two host threads, or two streams, on the same device) race on it and give
 * wrong results; serialise them.
 * Limits: per_stream <= PRNG_NOALLOC_VALUE_BYTES / 8 (2^21 outputs per stream); larger
 * values return PRNG_EINVAL with the limit in prng_last_error().
 * Errors: PRNG_EINVAL, PRNG_ECUDA.
 */
#define PRNG_NOALLOC_VALUE_BYTES ((size_t)16 << 20)
#define PRNG_NOALLOC_MAX_SLICE_STREAMS ((uint64_t)1 << 17)
int prng_fill_f64_host_noalloc(prng_t h, double* host_out, uint64_t per_stream, int form,
                               uint64_t* host_rejects, void* cuda_stream);

/*
 * prng_fused_stats -- generate per_stream outputs of every stream (advancing the streams
 * exactly as a fill would) and reduce them without storing any value: a 65536-bin
 * histogram of floor(2^16 z') and the four sums S1 = sum t, S2 = sum p2, S3 = sum p3,
 * S4 = sum p4 with t = floor(2^32 z'), p2 = floor(t^2 / 2^32), p3 = floor(p2 t / 2^32),
 * p4 = floor(p3 t / 2^32). z' = n/D exactly (no rounding), so all results are exact
 * integers independent of summation order; the p-th moment estimate is S_p / (N 2^32).
 * d_hist: device pointer to 65536 uint64, d_sums: device pointer to 8 uint64 (S_p as a
 * 128-bit integer, low word at 2(p-1), high word at 2(p-1)+1). Both are ACCUMULATED into
 * (zero them first for a fresh result). d_rejects as for prng_fill_f64.
 * Errors: PRNG_EINVAL (null pointers), PRNG_ENOMEM (scratch), PRNG_ECUDA.
 */
int prng_fused_stats(prng_t h, uint64_t per_stream, uint64_t* d_hist, uint64_t* d_sums,
                     uint64_t* d_rejects, void* cuda_stream);

/*
 * prng_stats_merge -- add one fused-statistics result into an accumulator, on the host:
 * hist_in (65536 counts) and sums_in (S1..S4 as 128-bit (low, high) pairs, the layout
 * prng_fused_stats leaves) into hist_acc and sums_acc of the same layout, each count and each
 * 128-bit sum exactly (with the carry into the high word). Results of replicas that ran on
 * disjoint stream ranges (one process per GPU) merge into the statistics of all their
 * streams, in any order. All four pointers are host memory; no device work.
 * Errors: PRNG_EINVAL (null pointer).
 */
int prng_stats_merge(const uint64_t* hist_in, const uint64_t* sums_in, uint64_t* hist_acc, uint64_t* sums_acc);

/*
 * Batched requests. Many fill requests of uneven length run in one persistent launch over a
 * device work queue (a counter over items of 32 rows), replayed from a CUDA graph captured
 * once per launch shape. Each request's output is a stream-major block of rows, row j being
 * one stream's outputs in order (Section 2's construction per output, as in the fills):
 *
 *  PRNG_REQ_FRESH:    rows are streams first_stream + j of `seed` (seeded as in prng_create),
 *                     `chunk` outputs each (even; 0 means 1024), the last row shorter;
 *                     ceil(length / chunk) streams. Stateless: the same request always gives
 *                     the same output.
 *  PRNG_REQ_RESIDENT: rows continue the handle's streams first_stream .. first_stream +
 *                     n_streams - 1 (device-resident state, advanced by the call). Row length
 *                     per = 16 * ceil(length / (16 * n_streams)); row j holds
 *                     min(per, max(0, length - j * per)) outputs (trailing rows may be empty:
 *                     their streams do not advance).
 *
 * The outputs never depend on the launch shape, on the batch a request is in, or on the
 * other requests of the batch. d_out: device pointer, 16-byte aligned, 8 * length bytes
 * (form C: interleaved float pairs). d_rejects (nullable, device): one reject count per row.
 * Rate: rows are written in 128-byte segments, so d_out should be 128-byte aligned and a
 * fresh request's chunk a multiple of 16; rows that start 16 bytes off a 32-byte sector
 * boundary write partial sectors and run at about 0.6 of the full rate.
 */
#define PRNG_REQ_FRESH 0
#define PRNG_REQ_RESIDENT 1
#define PRNG_MAX_BATCH_REQUESTS 4096

typedef struct prng_request {
  int32_t kind;          /* PRNG_REQ_FRESH or PRNG_REQ_RESIDENT */
  int32_t form;          /* PRNG_FORM_A_FP64, PRNG_FORM_B_INTBITS, PRNG_FORM_C_F32PAIR or
                            PRNG_FORM_L_ALGO1 */
  uint64_t length;       /* outputs, 1 .. 2^60 */
  uint64_t seed;         /* FRESH: seed of the request's streams */
  uint64_t first_stream; /* FRESH: first stream id; RESIDENT: first stream of the handle */
  uint64_t n_streams;    /* RESIDENT: streams of the handle to continue (FRESH: ignored) */
  uint32_t chunk;        /* FRESH: outputs per stream, even (0 = 1024); RESIDENT: ignored */
  uint32_t mode;         /* PRNG_MODE_* bits as for prng_fill_mode (0: Eq. 4, pair rejects) */
  void* d_out;           /* device pointer, 16-byte aligned */
  uint64_t* d_rejects;   /* nullable device pointer, 8-byte aligned, one count per row */
} prng_request;

/*
 * prng_submit -- enqueue a batch of 1 .. PRNG_MAX_BATCH_REQUESTS requests on `cuda_stream`
 * and return a ticket. The call copies the descriptors, so `reqs` may be reused at once.
 * Resident requests of one batch must not share streams; batches on different CUDA streams
 * that use the same resident streams must be ordered by the caller.
 * Errors: PRNG_EINVAL (bad request, overlapping resident ranges, n out of range),
 * PRNG_EBUSY (all 32 batch slots still in flight: poll or wait, then retry), PRNG_ENOMEM,
 * PRNG_ECUDA.
 */
int prng_submit(prng_t h, const prng_request* reqs, int n, uint64_t* ticket, void* cuda_stream);

/* prng_poll -- *done = 1 if the batch of `ticket` has finished on the device, else 0.
 * Non-blocking. Errors: PRNG_ENOTFOUND (a ticket this handle never issued), PRNG_ECUDA. */
int prng_poll(prng_t h, uint64_t ticket, int* done);

/* prng_wait -- block (polling) until the batch of `ticket` has finished, at most timeout_s
 * seconds. Errors: PRNG_ETIMEOUT, PRNG_ENOTFOUND, PRNG_ECUDA. */
int prng_wait(prng_t h, uint64_t ticket, double timeout_s);

/* Launch shape of the batch kernel: warps per block (1..8), blocks per SM (1..16), items
 * (32 rows of one request) taken per counter increment (1..64), and outputs per chunk (16 or
 * 32): how many outputs each thread makes for its row before the warp writes them with
 * tensor stores (32: two stores of 32 x 16 boxes; it applies to batches whose requests all use
 * mode 0 or all form B with exactly PRNG_MODE_BALANCED, the others use 16). Changing the shape
 * never changes outputs; set_shape waits for in-flight batches and re-captures the graphs on
 * next use. Errors: PRNG_EINVAL (a value out of range), PRNG_ENOMEM, PRNG_ECUDA. */
int prng_batch_get_shape(prng_t h, int* warps_per_block, int* blocks_per_sm, int* items_per_ticket,
                         int* outputs_per_chunk);
int prng_batch_set_shape(prng_t h, int warps_per_block, int blocks_per_sm, int items_per_ticket,
                         int outputs_per_chunk);

/*
 * prng_batch_autotune -- pick the batch launch shape for requests of `form` with lengths in
 * [length_lo, length_hi]. If table_path names a table with a line for this (GPU name, w,
 * form, length range) and force == 0, that shape is applied without measuring. Otherwise
 * every candidate (4 or 8 warps per block x 2, 3, 4, 6 or 8 blocks per SM x 1, 4 or 8 items
 * per ticket x 16 or 32 outputs per chunk) is timed on a synthetic batch of 256 fresh requests
 * with log-uniform lengths in the range (at most 2^30 outputs, in an 8 GiB scratch buffer the
 * call allocates and frees), the fastest is applied and, if table_path is not NULL, appended to
 * the table as "<key> <warps> <blocks> <items> <outputs per chunk> <ms>". Outputs never depend
 * on the shape.
 * The chosen shape and its time (ms; -1 when read from the table) are returned through the
 * nullable pointers. Errors: PRNG_EINVAL, PRNG_ENOMEM, PRNG_ECUDA.
 */
int prng_batch_autotune(prng_t h, int form, uint64_t length_lo, uint64_t length_hi, const char* table_path,
                        int force, int* warps_per_block, int* blocks_per_sm, int* items_per_ticket,
                        int* outputs_per_chunk, double* best_ms);

/*
 * Serving loop. A server keeps per-client generator state resident on the device and runs
 * client fill requests with continuous batching. The paper has no serving layer; each
 * request is the method of Section 2 applied to the client's streams.
 *
 * Clients: client c owns the handle's streams [c S, (c+1) S) (S = streams_per_client, which
 * must divide the handle's stream count). A request of `length` outputs from client c is the
 * resident request (see prng_request) over the first n = min(S, ceil(length /
 * min_per_stream)) of the client's streams. A client's requests run one at a time in
 * admission order, so a result is fixed by the client's history and the request alone,
 * never by what else is in flight.
 *
 * Admission: prng_server_submit takes output memory from a device pool of pool_bytes
 * (allocated once by prng_server_create) and returns PRNG_EBUSY when it does not fit;
 * the caller retries after releasing finished requests.
 * Batching: prng_server_step harvests finished batches and launches the admitted requests of
 * idle clients as batches, one per lane: requests of up to 2^20 outputs, up to 2^24, up to
 * 2^26, and longer. Up to 8 batches of a lane are on the device at once, each on a CUDA stream of its
 * own (lanes of shorter requests at higher stream priority), so work admitted while other
 * batches run overlaps with them. The server's batches take one item (32 rows) per warp and
 * then end their blocks, which frees SM slots item by item for the other lanes.
 * Results stay in the pool until prng_server_release; prng_server_poll gives the device
 * pointer, prng_server_read copies them to the host.
 * A server is not thread-safe. Errors as for the batch calls; PRNG_ENOTFOUND for an unknown
 * request id.
 */
typedef struct prng_server* prng_server_t;

int prng_server_create(prng_server_t* out, prng_t h, uint64_t streams_per_client,
                       uint64_t min_per_stream, size_t pool_bytes);
int prng_server_destroy(prng_server_t s);
int prng_server_submit(prng_server_t s, uint64_t client, uint64_t length, int form, uint64_t* id);
/* As prng_server_submit, with the request's PRNG_MODE_* bits (prng_server_submit: mode 0). */
int prng_server_submit_mode(prng_server_t s, uint64_t client, uint64_t length, int form, uint32_t mode,
                            uint64_t* id);
int prng_server_step(prng_server_t s);
int prng_server_poll(prng_server_t s, uint64_t id, int* done, void** d_out);
int prng_server_read(prng_server_t s, uint64_t id, void* host_dst, size_t bytes);
int prng_server_release(prng_server_t s, uint64_t id);
/* Withdraw a request that has not been launched yet: its pool memory is freed, its id is
 * forgotten, and the client's streams do not advance (its later requests continue from the
 * state the earlier ones left). A request already on the device, or finished, cannot be
 * withdrawn: PRNG_EBUSY (wait for it, then release it). Errors: PRNG_EINVAL, PRNG_ENOTFOUND,
 * PRNG_EBUSY. */
int prng_server_cancel(prng_server_t s, uint64_t id);
/* Step until nothing is waiting or running, at most timeout_s seconds (PRNG_ETIMEOUT). */
int prng_server_drain(prng_server_t s, double timeout_s);
int prng_server_info(prng_server_t s, uint64_t* n_clients, uint64_t* batches, uint64_t* completed,
                     uint64_t* samples, size_t* pool_used);

/*
 * prng_server_run_trace -- replay an arrival trace in real time: item i arrives t seconds
 * after the call starts (items sorted by t), is admitted when the pool has room (in arrival
 * order within each lane, and always after its client's earlier arrivals, so a small request
 * does not wait for the memory of a large one), runs, and is released as soon as it finishes. latency (nullable, n doubles) gets
 * finish time minus arrival time per item; makespan (nullable) the total wall time.
 * Errors: PRNG_ETIMEOUT after timeout_s seconds, and those of the calls above.
 */
typedef struct prng_trace_item {
  double t;         /* arrival time, seconds from the start of the replay */
  uint64_t client;
  uint64_t length;  /* outputs */
  int32_t form;
  uint32_t mode;    /* PRNG_MODE_* bits */
} prng_trace_item;
int prng_server_run_trace(prng_server_t s, const prng_trace_item* items, uint64_t n, double* latency,
                          double* makespan, double timeout_s);

/*
 * State checkpoint: each stream's state is 16 bytes (xorshift128 words x, y, z, w).
 * prng_state_bytes gives n_streams * 16 (32 for MRG32k3a streams). save copies the device state into host_buf and
 * restore copies it back; both synchronise. A fill after restore reproduces the outputs
 * that followed the save, bit for bit.
 * Errors: PRNG_EINVAL (null pointers, bytes != prng_state_bytes), PRNG_ECUDA.
 */
size_t prng_state_bytes(prng_t h);
int prng_state_save(prng_t h, void* host_buf, size_t bytes);
int prng_state_restore(prng_t h, const void* host_buf, size_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* PRNGD_H */
