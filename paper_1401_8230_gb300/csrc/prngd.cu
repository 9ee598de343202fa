// prngd.cu -- host side of the C ABI declared in include/prngd.h: handle management,
// argument checking, tensor-map encoding and kernel dispatch for the fill paths.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <string>

#include "prngd.h"
#include "prngd_fill.cuh"
#include "prngd_internal.h"
#include "prngd_launch.h"

using prngd::DivConst;
using prngd::FillParams;

namespace prngd {
// Seed streams [0, n) of `seed`.
__global__ void seed_kernel(uint4* state, uint64_t n, uint64_t seed) {
  const uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const XorShift128 x = seed_stream(seed, s);
  state[s] = make_uint4(x.x, x.y, x.z, x.w);
}
}  // namespace prngd

namespace prngd_host {

thread_local char g_err[512];

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

DivConst make_divconst(int w) {
  const uint64_t m = (w == 32) ? 0xFFFFFFFFull : ((1ull << w) - 1);
  const uint64_t D = m * m;
  DivConst dc;
  dc.sh = 64 - 2 * w;
  dc.d_norm = D << dc.sh;
  const unsigned __int128 all = ~(unsigned __int128)0;
  dc.v = (uint64_t)(all / dc.d_norm - ((unsigned __int128)1 << 64));
  return dc;
}

// Division constants of E = D - 2, the denominator of Eq. 5 (E is normalised by its own shift).
DivConst make_divconst_eq5(int w) {
  const uint64_t m = (w == 32) ? 0xFFFFFFFFull : ((1ull << w) - 1);
  const uint64_t e = m * m - 2;
  DivConst dc;
  dc.sh = prngd::clz64(e);
  dc.d_norm = e << dc.sh;
  const unsigned __int128 all = ~(unsigned __int128)0;
  dc.v = (uint64_t)(all / dc.d_norm - ((unsigned __int128)1 << 64));
  return dc;
}

// The constants the map kernels take: C5 = RN((2^2w - 1) / ((D - 2) 2^2w)) for form A under
// Eq. 5, and form L's folded constants, each one IEEE double operation as Algorithm 1 (Eq. 4)
// or Eq. 6 writes them (volatile: no contraction, one rounding per operation).
void set_mode_constants(FillParams& p, int w, int mode) {
  p.single = (mode & PRNG_MODE_SINGLE_REDRAW) ? 1u : 0u;
  p.ec = make_divconst_eq5(w);
  const int s2 = 2 * w;
  const uint64_t num = (s2 == 64) ? ~0ull : ((1ull << s2) - 1);  // 2^2w - 1 (< 2^64)
  const uint64_t c5 = prngd::rn_bits_ratio128(0, num, p.ec, s2);
  memcpy(&p.scale5, &c5, 8);
  volatile double k = std::ldexp(1.0, -w);
  p.k = k;
  if (mode & PRNG_MODE_EQ5) {
    volatile double kk = k * k;
    volatile double c3 = 1.0 - kk;
    volatile double t1 = std::trunc(1.0 / k);
    volatile double d1 = t1 - 2.0;
    volatile double den = d1 - k;
    p.l1 = c3;
    p.l2 = den;
  } else {
    volatile double mn = 0.0, mx = 1.0 - k;
    volatile double kmx = k * mx;
    volatile double c1 = mn + kmx;
    volatile double span = mx - mn;
    volatile double onek = 1.0 - k;
    volatile double c2 = span * onek;
    p.l1 = c1;
    p.l2 = c2;
  }
}

double scale_constant(const DivConst& dc) {
  const uint64_t bits = prngd::rn_bits_exact(1, dc);  // RN(1/D)
  double d;
  memcpy(&d, &bits, 8);
  return d;
}

// ----------------------------------------------------------------- tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Looked up once per process (the driver entry point is the same for every device); the
// initialisation of a function-local static is thread-safe.
static EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    cudaGetLastError();
    return nullptr;
  }();
  return fn;
}

// 2D map over a stream-major array of 8-byte outputs: dim0 = outputs per stream (contiguous),
// dim1 = streams; box = box_x outputs x box_y streams, rows of box_x * 8 bytes swizzled in
// 128-byte (box_x = 16) or 64-byte (box_x = 8) mode.
// pitch: bytes from one stream's row to the next (0: per_stream * 8).
bool encode_out_map_box(CUtensorMap* map, void* out, uint64_t n_streams, uint64_t per_stream, uint32_t box_x,
                        uint32_t box_y, uint64_t pitch) {
  EncodeTiledFn fn = encode_fn();
  if (!pitch) pitch = per_stream * 8;
  if (!fn || (box_x != 16 && box_x != 8) || box_y == 0 || box_y > 256) return false;
  if (((uintptr_t)out & 15) || (per_stream & 1) || per_stream == 0 || per_stream >= (1ull << 31) ||
      n_streams >= (1ull << 31) || (pitch & 15) || pitch < per_stream * 8)
    return false;
  cuuint64_t gdim[2] = {per_stream, n_streams};
  cuuint64_t gstride[1] = {pitch};
  cuuint32_t box[2] = {box_x, box_y};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, out, gdim, gstride, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, box_x == 16 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// The fills' map: box = 16 outputs x 32 streams with the 128-byte swizzle.
bool encode_out_map(CUtensorMap* map, void* out, uint64_t n_streams, uint64_t per_stream) {
  return encode_out_map_box(map, out, n_streams, per_stream, (uint32_t)prngd::kChunk, 32, 0);
}

// ----------------------------------------------------------------- fill dispatch
constexpr int kWarpsPerBlock = 8;
constexpr int kNbuf = 1;  // one tile per warp: 4 blocks of 8 warps fit per SM (registers and shared memory)
constexpr size_t kTmaSmem = (size_t)kWarpsPerBlock * kNbuf * prngd::kTileBytes + 1024;

template <int W, int FORM, int MAP = 0>
static cudaError_t launch_w_form(const FillParams& p, const CUtensorMap* map, cudaStream_t s, bool shift) {
  const uint64_t warps = (p.n_streams + 31) / 32;
  const unsigned blocks = (unsigned)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock);
  if (map && shift) {
    auto k = prngd::fill_tma_kernel<W, FORM, kNbuf, MAP, true>;
    static std::atomic<uint64_t> attr{0};
    const cudaError_t e = prngd::smem_limit_once(k, (int)kTmaSmem, attr);
    if (e != cudaSuccess) return e;
    k<<<blocks, kWarpsPerBlock * 32, kTmaSmem, s>>>(p, *map);
  } else if (map) {
    auto k = prngd::fill_tma_kernel<W, FORM, kNbuf, MAP>;
    static std::atomic<uint64_t> attr{0};
    const cudaError_t e = prngd::smem_limit_once(k, (int)kTmaSmem, attr);
    if (e != cudaSuccess) return e;
    k<<<blocks, kWarpsPerBlock * 32, kTmaSmem, s>>>(p, *map);
  } else {
    prngd::fill_plain_kernel<W, FORM, MAP><<<blocks, kWarpsPerBlock * 32, 0, s>>>(p);
  }
  return cudaGetLastError();
}

template <int FORM, int MAP = 0>
static cudaError_t launch_form(const FillParams& p, const CUtensorMap* map, cudaStream_t s, bool shift) {
  if (p.w == 32) return launch_w_form<32, FORM, MAP>(p, map, s, shift);
  if (p.w == 24) return launch_w_form<24, FORM, MAP>(p, map, s, shift);
  return launch_w_form<0, FORM, MAP>(p, map, s, shift);
}

// Host memory the device can address (pinned / registered); its device-side address in *dev.
bool device_mapped_host(const void* p, void** dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
  if (dev) *dev = a.devicePointer;
  return true;
}

int require_xorshift(prng_ctx* h, const char* what) {
  if (h->gen != PRNG_GEN_XORSHIFT128)
    return fail(PRNG_EINVAL, "%s is available for xorshift128 streams only", what);
  return PRNG_OK;
}

int launch_fill(prng_ctx* h, uint4* state, uint64_t n_streams, void* out, uint64_t per_stream, int form,
                uint64_t* rejects, cudaStream_t s, bool allow_tma, int mode) {
  if (h->gen == PRNG_GEN_MRG32K3A)
    return launch_fill_mrg(h, state, n_streams, out, per_stream, form, rejects, s, allow_tma, mode);
  if (n_streams == 0 || per_stream == 0) return PRNG_OK;
  if (allow_tma && device_mapped_host(out, nullptr)) allow_tma = false;  // host memory: plain stores only
  FillParams p;
  p.state = state;
  p.n_streams = n_streams;
  p.per_stream = per_stream;
  p.out = (uint64_t*)out;
  p.rejects = rejects;
  p.dc = h->dc;
  p.scale = h->scale;
  p.w = h->w;
  p.one = 1;
  // rows that do not all start on a 128-byte line: the tensor stores keep their lines in L2
  p.keep_lines = (((uintptr_t)out & 127) != 0 || ((per_stream * 8) & 127) != 0) ? 1u : 0u;
  set_mode_constants(p, h->w, mode);
  CUtensorMap map;
  const CUtensorMap* mp = (allow_tma && encode_out_map(&map, out, n_streams, per_stream)) ? &map : nullptr;
  cudaError_t e;
  // Fast kernels: w = 32 / 24, forms B and C, TMA stores; everything else: the generic ones,
  // which have no conversion route (the same values by integer rounding).
  const bool fast = mp && (h->w == 32 || h->w == 24) &&
                    (form == PRNG_FORM_B_INTBITS || form == PRNG_FORM_C_F32PAIR);
  int map_bits = map_bits_of(form, mode);
  if (!fast && form != PRNG_FORM_A_FP64) map_bits &= ~prngd::kMapCvt;  // form B's route: pair kernels only
  const bool balanced_a = form == PRNG_FORM_A_FP64 && map_bits == prngd::kMapCvt;
  const bool generic_map = (map_bits || form == PRNG_FORM_L_ALGO1) && !fast && !balanced_a;
  // Rows that all start 16 bytes into a 32-byte sector: every tensor store would begin and end in
  // half a sector. The kernels of the plain forms and of the fast maps then take a map that
  // starts 2 outputs into each row (fill_tma_kernel's SHIFT); the generic map kernels keep theirs.
  bool shift = false;
  if (mp && !generic_map && ((uintptr_t)out & 31) == 16 && (per_stream & 3) == 0 && per_stream > 2) {
    CUtensorMap smap;
    if (encode_out_map_box(&smap, (uint64_t*)out + 2, n_streams, per_stream - 2, (uint32_t)prngd::kChunk, 32,
                           per_stream * 8)) {
      map = smap;
      shift = true;
    }
  }
  if (balanced_a) {  // balanced form A under Eq. 4
    e = launch_form<prngd::kFormA, prngd::kMapCvt>(p, mp, s, shift);
    if (e != cudaSuccess) return fail(PRNG_ECUDA, "fill launch: %s", cudaGetErrorString(e));
    return PRNG_OK;
  }
  if (map_bits || form == PRNG_FORM_L_ALGO1) {
    e = fast ? launch_fill_map_fast(p, form, map_bits, mp, s, shift) : launch_fill_map(p, form, map_bits, mp, s);
    if (e != cudaSuccess) return fail(PRNG_ECUDA, "fill launch: %s", cudaGetErrorString(e));
    return PRNG_OK;
  }
  switch (form) {
    case PRNG_FORM_A_FP64: e = launch_form<prngd::kFormA>(p, mp, s, shift); break;
    case PRNG_FORM_B_INTBITS: e = launch_form<prngd::kFormB>(p, mp, s, shift); break;
    case PRNG_FORM_C_F32PAIR: e = launch_form<prngd::kFormC>(p, mp, s, shift); break;
    default: return fail(PRNG_EINVAL, "unknown form %d", form);
  }
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "fill launch: %s", cudaGetErrorString(e));
  return PRNG_OK;
}

int check_fill_extent(prng_ctx* h, uint64_t per_stream, const void* d_rejects) {
  if ((uintptr_t)d_rejects & 7) return fail(PRNG_EINVAL, "d_rejects must be 8-byte aligned");
  if (per_stream > kMaxOutputs / h->n_streams)
    return fail(PRNG_EINVAL, "n_streams * per_stream exceeds 2^60 outputs");
  return PRNG_OK;
}

int check_handle_device(prng_ctx* h) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev != h->device) return fail(PRNG_EINVAL, "handle lives on device %d, current device is %d", h->device, dev);
  return PRNG_OK;
}

}  // namespace prngd_host

using namespace prngd_host;

extern "C" {

const char* prng_last_error(void) { return g_err; }

int prng_version(void) { return 100; }

int prng_create(prng_t* out, uint64_t seed, uint64_t n_streams, int w, double a0, double a, double b0, double b) {
  g_err[0] = 0;
  if (!out) return fail(PRNG_EINVAL, "out is NULL");
  *out = nullptr;
  if (w < 2 || w > 32) return fail(PRNG_EINVAL, "w = %d is outside [2, 32]", w);
  if (n_streams == 0 || n_streams > (1ull << 32)) return fail(PRNG_EINVAL, "n_streams must be in [1, 2^32]");
  if (!std::isfinite(a0) || !std::isfinite(a) || !std::isfinite(b0) || !std::isfinite(b))
    return fail(PRNG_EINVAL, "ranges must be finite");
  // Discrete rule of Section 2: x1 and x2 are grids of step k = 2^-w with 2^w points each.
  const double step = std::ldexp((double)((w == 32) ? 0xFFFFFFFFull : ((1ull << w) - 1)), -w);
  if (a - a0 != step || a0 + step != a || b - b0 != step || b0 + step != b)
    return fail(PRNG_EINVAL, "ranges must satisfy a - a0 = b - b0 = (2^w - 1) 2^-w exactly");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  prng_ctx* h = new prng_ctx();
  h->device = dev;
  h->seed = seed;
  h->n_streams = n_streams;
  h->w = w;
  h->dc = make_divconst(w);
  h->scale = scale_constant(h->dc);
  e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete h;
    return fail(PRNG_ECUDA, "device attributes: %s", cudaGetErrorString(e));
  }
  e = cudaMalloc(&h->d_state, n_streams * sizeof(uint4));
  if (e != cudaSuccess) {
    delete h;
    cudaGetLastError();
    return fail(PRNG_ENOMEM, "cudaMalloc(state, %llu bytes): %s", (unsigned long long)(n_streams * 16),
                cudaGetErrorString(e));
  }
  const unsigned blocks = (unsigned)((n_streams + 255) / 256);
  prngd::seed_kernel<<<blocks, 256>>>(h->d_state, n_streams, seed);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  if (e != cudaSuccess) {
    cudaFree(h->d_state);
    delete h;
    return fail(PRNG_ECUDA, "seeding: %s", cudaGetErrorString(e));
  }
  *out = h;
  return PRNG_OK;
}

int prng_destroy(prng_t h) {
  if (!h) return PRNG_OK;
  cudaDeviceSynchronize();
  release_batch(h);
  release_aux(h);
  release_split(h);
  cudaFree(h->d_state);
  delete h;
  return PRNG_OK;
}

int prng_get_info(prng_t h, uint64_t* n_streams, int* w) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  if (n_streams) *n_streams = h->n_streams;
  if (w) *w = h->w;
  return PRNG_OK;
}

int prng_fill_f64(prng_t h, double* d_out, uint64_t per_stream, int form, uint64_t* d_rejects, void* cuda_stream) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  if (form != PRNG_FORM_A_FP64 && form != PRNG_FORM_B_INTBITS)
    return fail(PRNG_EINVAL, "prng_fill_f64 takes form A (0) or B (1), got %d", form);
  if (per_stream == 0) return PRNG_OK;
  if (!d_out) return fail(PRNG_EINVAL, "d_out is NULL");
  if ((uintptr_t)d_out & 7) return fail(PRNG_EINVAL, "d_out must be 8-byte aligned");
  int rc = check_fill_extent(h, per_stream, d_rejects);
  if (!rc) rc = check_handle_device(h);
  if (rc) return rc;
  return launch_fill(h, h->d_state, h->n_streams, d_out, per_stream, form, d_rejects, (cudaStream_t)cuda_stream,
                     true);
}

int prng_fill_f32pair(prng_t h, float* d_out, uint64_t per_stream, uint64_t* d_rejects, void* cuda_stream) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  if (per_stream == 0) return PRNG_OK;
  if (!d_out) return fail(PRNG_EINVAL, "d_out is NULL");
  if ((uintptr_t)d_out & 7) return fail(PRNG_EINVAL, "d_out must be 8-byte aligned");
  int rc = check_fill_extent(h, per_stream, d_rejects);
  if (!rc) rc = check_handle_device(h);
  if (rc) return rc;
  return launch_fill(h, h->d_state, h->n_streams, d_out, per_stream, PRNG_FORM_C_F32PAIR, d_rejects,
                     (cudaStream_t)cuda_stream, true);
}

int prng_fill_mode(prng_t h, void* d_out, uint64_t per_stream, int form, int mode, uint64_t* d_rejects,
                   void* cuda_stream) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  if (form != PRNG_FORM_A_FP64 && form != PRNG_FORM_B_INTBITS && form != PRNG_FORM_C_F32PAIR &&
      form != PRNG_FORM_L_ALGO1)
    return fail(PRNG_EINVAL, "unknown form %d", form);
  if (mode & ~kAllModes) return fail(PRNG_EINVAL, "unknown mode bits 0x%x", (unsigned)mode);
  if (per_stream == 0) return PRNG_OK;
  if (!d_out) return fail(PRNG_EINVAL, "d_out is NULL");
  if ((uintptr_t)d_out & 7) return fail(PRNG_EINVAL, "d_out must be 8-byte aligned");
  int rc = check_fill_extent(h, per_stream, d_rejects);
  if (!rc) rc = check_handle_device(h);
  if (rc) return rc;
  return launch_fill(h, h->d_state, h->n_streams, d_out, per_stream, form, d_rejects, (cudaStream_t)cuda_stream,
                     true, mode);
}

size_t prng_state_bytes(prng_t h) {
  return h ? (size_t)h->n_streams * (h->gen == PRNG_GEN_MRG32K3A ? 32 : 16) : 0;
}

int prng_state_save(prng_t h, void* host_buf, size_t bytes) {
  if (!h || !host_buf) return fail(PRNG_EINVAL, "null argument");
  if (bytes != prng_state_bytes(h)) return fail(PRNG_EINVAL, "bytes must be prng_state_bytes(h)");
  cudaError_t e = cudaMemcpy(host_buf, h->d_state, bytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "state save: %s", cudaGetErrorString(e));
  return PRNG_OK;
}

int prng_state_restore(prng_t h, const void* host_buf, size_t bytes) {
  if (!h || !host_buf) return fail(PRNG_EINVAL, "null argument");
  if (bytes != prng_state_bytes(h)) return fail(PRNG_EINVAL, "bytes must be prng_state_bytes(h)");
  cudaError_t e = cudaMemcpy(h->d_state, host_buf, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "state restore: %s", cudaGetErrorString(e));
  return PRNG_OK;
}

int prng_fill_f64_host(prng_t h, double* host_out, uint64_t per_stream, int form, uint64_t* host_rejects) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  if (form != PRNG_FORM_A_FP64 && form != PRNG_FORM_B_INTBITS)
    return fail(PRNG_EINVAL, "prng_fill_f64_host takes form A (0) or B (1), got %d", form);
  if (per_stream == 0) return PRNG_OK;
  if (!host_out) return fail(PRNG_EINVAL, "host_out is NULL");
  int rc = check_fill_extent(h, per_stream, nullptr);
  if (!rc) rc = check_handle_device(h);
  if (rc) return rc;
  return host_fill(h, host_out, per_stream, form, host_rejects);
}

}  // extern "C"
