/* A C caller of the library through include/prngd.h alone: no Python, no torch, and no CUDA
 * runtime call of its own. Without arguments it checks the argument errors that need no GPU;
 * with --gpu it also makes a handle, fills host memory (prng_fill_f64_host), compares every
 * output and reject count with the C oracle (whose function it declares below), and checks
 * that a state save / restore repeats a fill bit for bit. Built and run by test_abi.py and
 * test_gpu_abi_c.py. Prints "bad <count>" and exits non-zero on any failure. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "prngd.h"

/* the oracle (oracle/prngd_oracle.c, linked into this test program only) */
int orc_fill(uint64_t seed, uint64_t first_stream, uint64_t n_streams, uint64_t per_stream, int w, int form,
             void* out, uint64_t* rejects);

static int bad = 0;

static void check(int ok, const char* what) {
  if (!ok) {
    ++bad;
    printf("FAILED: %s (last error: %s)\n", what, prng_last_error());
  }
}

static double step_of(int w) { return (ldexp(1.0, w) - 1.0) * ldexp(1.0, -w); } /* (2^w - 1) 2^-w */

static void host_checks(void) {
  prng_t h = NULL;
  const double s = step_of(32);
  check(prng_version() >= 100, "prng_version");
  check(prng_create(NULL, 1, 64, 32, 0.0, s, 0.0, s) == PRNG_EINVAL, "create: null out");
  check(prng_create(&h, 1, 64, 1, 0.0, step_of(1), 0.0, step_of(1)) == PRNG_EINVAL && h == NULL, "create: w = 1");
  check(strstr(prng_last_error(), "outside") != NULL, "create: message names the range");
  check(prng_create(&h, 1, 64, 33, 0.0, s, 0.0, s) == PRNG_EINVAL, "create: w = 33");
  check(prng_create(&h, 1, 0, 32, 0.0, s, 0.0, s) == PRNG_EINVAL, "create: zero streams");
  check(prng_create(&h, 1, 64, 32, 0.0, 1.0, 0.0, s) == PRNG_EINVAL, "create: step of x1 is not 2^-32");
  check(prng_create(&h, 1, 64, 32, 0.0, s, NAN, s) == PRNG_EINVAL, "create: NaN range");
  check(prng_fill_f64(NULL, NULL, 16, PRNG_FORM_B_INTBITS, NULL, NULL) == PRNG_EINVAL, "fill: null handle");
  check(prng_fill_f64_host(NULL, NULL, 16, PRNG_FORM_B_INTBITS, NULL) == PRNG_EINVAL, "host fill: null handle");
  check(prng_state_bytes(NULL) == 0, "state bytes of NULL");
  check(prng_generator(NULL) == -1, "generator of NULL");
  check(prng_destroy(NULL) == PRNG_OK, "destroy NULL");
}

static void gpu_checks(void) {
  const uint64_t seed = 1, ns = 64, per = 1000;
  const int w = 32;
  const double s = step_of(w);
  prng_t h = NULL;
  check(prng_create(&h, seed, ns, w, 0.25, 0.25 + s, -3.0, -3.0 + s) == PRNG_OK, "create");
  if (!h) return;
  double* got = malloc(ns * per * 8);
  double* want = malloc(ns * per * 8);
  double* again = malloc(ns * per * 8);
  uint64_t* rej = malloc(ns * 8);
  uint64_t* want_rej = malloc(ns * 8);
  const size_t sb = prng_state_bytes(h);
  unsigned char* st = malloc(sb);
  check(sb == ns * 16, "state bytes");
  check(prng_fill_f64_host(h, got, per, PRNG_FORM_B_INTBITS, rej) == PRNG_OK, "host fill");
  check(orc_fill(seed, 0, ns, per, w, 1 /* form B */, want, want_rej) == 0, "oracle fill");
  check(memcmp(got, want, ns * per * 8) == 0, "host fill equals the oracle, word for word");
  check(memcmp(rej, want_rej, ns * 8) == 0, "reject counts equal the oracle's");
  /* checkpoint, fill, restore, fill again: the same outputs */
  check(prng_state_save(h, st, sb) == PRNG_OK, "state save");
  check(prng_fill_f64_host(h, got, per, PRNG_FORM_A_FP64, NULL) == PRNG_OK, "second fill");
  check(prng_state_restore(h, st, sb) == PRNG_OK, "state restore");
  check(prng_fill_f64_host(h, again, per, PRNG_FORM_A_FP64, NULL) == PRNG_OK, "fill after restore");
  check(memcmp(got, again, ns * per * 8) == 0, "restore repeats the fill");
  check(prng_state_save(h, st, sb - 1) == PRNG_EINVAL, "state save with a wrong size");
  check(prng_destroy(h) == PRNG_OK, "destroy");
  free(got);
  free(want);
  free(again);
  free(rej);
  free(want_rej);
  free(st);
}

int main(int argc, char** argv) {
  host_checks();
  if (argc > 1 && strcmp(argv[1], "--gpu") == 0) gpu_checks();
  printf("bad %d\n", bad);
  return bad ? 1 : 0;
}
