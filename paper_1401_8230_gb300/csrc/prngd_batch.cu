// prngd_batch.cu -- host side of the batched path: request validation, descriptor staging in
// pinned memory, one persistent launch per batch replayed from a captured CUDA graph, tickets
// and the launch-shape autotuner.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <numeric>
#include <vector>

#include "prngd.h"
#include "prngd_batch.cuh"
#include "prngd_internal.h"

namespace prngd_host {

static constexpr int kSlots = 32;

struct BatchSlot {
  prngd::BatchDesc* h_desc = nullptr;  // pinned
  CUtensorMap* h_maps = nullptr;       // pinned, one per descriptor
  CUtensorMap* d_maps = nullptr;
  uint32_t* h_meta = nullptr;          // pinned: n_req, then the item prefix
  prngd::BatchDesc* d_desc = nullptr;
  uint32_t* d_meta = nullptr;
  unsigned long long* d_ticket = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t exec[6] = {};  // by kernel (kind + 2): any mode, mixed forms, A, B, C, B with FP64 rounding
  int cfg_version[6] = {-1, -1, -1, -1, -1, -1};  // launch shape each graph was captured with
  uint64_t ticket = 0;      // ticket of the batch last launched from this slot
};

struct BatchEngine {
  int max_req = 0;
  BatchSlot slot[kSlots];
  cudaStream_t capture_stream = nullptr;
  uint64_t next_ticket = 1;
  int next_slot = 0;
  BatchShape shape;
  int cfg_version = 0;
};

void release_batch(prng_ctx* h) {
  BatchEngine* b = h->batch;
  if (!b) return;
  for (auto& s : b->slot) {
    for (auto& x : s.exec)
      if (x) cudaGraphExecDestroy(x);
    if (s.done) cudaEventDestroy(s.done);
    cudaFreeHost(s.h_desc);
    cudaFreeHost(s.h_maps);
    cudaFree(s.d_maps);
    cudaFreeHost(s.h_meta);
    cudaFree(s.d_desc);
    cudaFree(s.d_meta);
    cudaFree(s.d_ticket);
  }
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
  h->batch = nullptr;
}

static int ensure_engine(prng_ctx* h) {
  if (h->batch) return PRNG_OK;
  BatchEngine* b = new BatchEngine();
  b->max_req = PRNG_MAX_BATCH_REQUESTS;
  b->shape = default_batch_shape(h->num_sms);
  h->batch = b;
  cudaError_t e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
  for (auto& s : b->slot) {
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_desc, sizeof(prngd::BatchDesc) * b->max_req);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_meta, sizeof(uint32_t) * (b->max_req + 2));
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_maps, sizeof(CUtensorMap) * b->max_req);
    if (e == cudaSuccess) e = cudaMalloc(&s.d_maps, sizeof(CUtensorMap) * b->max_req);
    if (e == cudaSuccess) e = cudaMalloc(&s.d_desc, sizeof(prngd::BatchDesc) * b->max_req);
    if (e == cudaSuccess) e = cudaMalloc(&s.d_meta, sizeof(uint32_t) * (b->max_req + 2));
    if (e == cudaSuccess) e = cudaMalloc(&s.d_ticket, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    release_batch(h);
    cudaGetLastError();
    return fail(PRNG_ENOMEM, "batch engine allocation: %s", cudaGetErrorString(e));
  }
  return PRNG_OK;
}

// 8 warps x 3 blocks (all resident at the kernel's register count) taking 4 items per ticket,
// 16 outputs per chunk: the fastest untuned shape on the batched workload with aligned outputs.
BatchShape default_batch_shape(int num_sms) {
  BatchShape s;
  s.warps_per_block = 8;
  s.blocks_per_sm = 3;
  s.items_per_ticket = 4;
  s.outputs_per_chunk = prngd::kChunk;
  (void)num_sms;
  return s;
}

template <int W, int FORM_ALL>
static cudaError_t launch_batch_wf(const prngd::BatchParams& p, const BatchShape& sh, unsigned blocks, int max_req,
                                   cudaStream_t s) {
  if (sh.outputs_per_chunk == 2 * prngd::kChunk)
    return prngd::launch_batch_kernel<W, FORM_ALL, 2 * prngd::kChunk>(p, sh.warps_per_block, blocks, max_req, s);
  return prngd::launch_batch_kernel<W, FORM_ALL>(p, sh.warps_per_block, blocks, max_req, s);
}

template <int W>
static cudaError_t launch_batch_w(const prngd::BatchParams& p, const BatchShape& sh, unsigned blocks, int max_req,
                                  int form_all, cudaStream_t s) {
  switch (form_all) {
    case prngd::kAnyMode: return launch_batch_any_mode_w<W>(p, sh, blocks, max_req, s);
    case prngd::kFormBBalanced: return launch_batch_wf<W, prngd::kFormBBalanced>(p, sh, blocks, max_req, s);
    case prngd::kFormA: return launch_batch_wf<W, prngd::kFormA>(p, sh, blocks, max_req, s);
    case prngd::kFormB: return launch_batch_wf<W, prngd::kFormB>(p, sh, blocks, max_req, s);
    case prngd::kFormC: return launch_batch_wf<W, prngd::kFormC>(p, sh, blocks, max_req, s);
    default: return launch_batch_wf<W, -1>(p, sh, blocks, max_req, s);
  }
}

// A launch: reset the item counter, run the kernel. The descriptors and item prefix are
// copied before it (sized to the batch) by submit(). A graph captures it with the persistent
// grid (blocks = 0: the shape's blocks per SM on every SM, shared memory for the largest
// batch); a capped launch passes its own grid and request count.
static cudaError_t enqueue_batch(prng_ctx* h, BatchSlot& sl, int form_all, cudaStream_t s, unsigned blocks = 0,
                                 int max_req = PRNG_MAX_BATCH_REQUESTS, uint32_t items_per_warp = 0, int warps = 0) {
  BatchEngine* b = h->batch;
  prngd::BatchParams p;
  p.desc = sl.d_desc;
  p.maps = sl.d_maps;
  p.meta = sl.d_meta;
  p.ticket = sl.d_ticket;
  p.state = h->d_state;
  p.dc = h->dc;
  p.scale = h->scale;
  p.w = h->w;
  p.one = 1;
  p.items_per_ticket = (uint32_t)b->shape.items_per_ticket;
  p.items_per_warp = items_per_warp;
  if (!blocks) blocks = (unsigned)(h->num_sms * b->shape.blocks_per_sm);
  prngd::FillParams f4, f5;  // the map constants (Eq. 5 division, form A and form L factors)
  set_mode_constants(f4, h->w, 0);
  set_mode_constants(f5, h->w, PRNG_MODE_EQ5);
  p.ec = f4.ec;
  p.scale5 = f4.scale5;
  p.k = f4.k;
  p.l1_eq4 = f4.l1;
  p.l2_eq4 = f4.l2;
  p.l1_eq5 = f5.l1;
  p.l2_eq5 = f5.l2;
  cudaError_t e = cudaMemsetAsync(sl.d_ticket, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  BatchShape sh = b->shape;
  if (warps) sh.warps_per_block = warps;
  if (h->w == 32) return launch_batch_w<32>(p, sh, blocks, max_req, form_all, s);
  if (h->w == 24) return launch_batch_w<24>(p, sh, blocks, max_req, form_all, s);
  return launch_batch_w<0>(p, sh, blocks, max_req, form_all, s);
}

// Capture the slot's reset + launch once per launch shape.
static int ensure_graph(prng_ctx* h, BatchSlot& sl, int form_all) {
  BatchEngine* b = h->batch;
  const int g_i = form_all + 2;  // any mode -> 0, mixed forms -> 1, A -> 2, B -> 3, C -> 4, B rounded -> 5
  if (sl.exec[g_i] && sl.cfg_version[g_i] == b->cfg_version) return PRNG_OK;
  if (sl.exec[g_i]) {
    cudaGraphExecDestroy(sl.exec[g_i]);
    sl.exec[g_i] = nullptr;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "begin capture: %s", cudaGetErrorString(e));
  cudaError_t e2 = enqueue_batch(h, sl, form_all, b->capture_stream);
  e = cudaStreamEndCapture(b->capture_stream, &g);
  if (e2 != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(PRNG_ECUDA, "batch capture: %s", cudaGetErrorString(e2 != cudaSuccess ? e2 : e));
  }
  e = cudaGraphInstantiate(&sl.exec[g_i], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  sl.cfg_version[g_i] = b->cfg_version;
  return PRNG_OK;
}

// Row layout of one request (see prng_request in prngd.h).
static int describe(prng_ctx* h, const prng_request& r, prngd::BatchDesc& d) {
  if (r.form != PRNG_FORM_A_FP64 && r.form != PRNG_FORM_B_INTBITS && r.form != PRNG_FORM_C_F32PAIR &&
      r.form != PRNG_FORM_L_ALGO1)
    return fail(PRNG_EINVAL, "request form %d", r.form);
  if (r.mode & ~(uint32_t)kAllModes) return fail(PRNG_EINVAL, "request mode %u", r.mode);
  d.mode = (uint16_t)r.mode;
  if (r.length == 0) return fail(PRNG_EINVAL, "request length 0");
  if (r.length > kMaxOutputs) return fail(PRNG_EINVAL, "request length exceeds 2^60 outputs");
  if (!r.d_out || ((uintptr_t)r.d_out & 15)) return fail(PRNG_EINVAL, "request d_out must be 16-byte aligned");
  if ((uintptr_t)r.d_rejects & 7) return fail(PRNG_EINVAL, "request d_rejects must be 8-byte aligned");
  d.length = r.length;
  d.out = (uint64_t*)r.d_out;
  d.rejects = r.d_rejects;
  d.form = r.form;
  if (r.kind == PRNG_REQ_FRESH) {
    const uint64_t chunk = r.chunk ? r.chunk : 1024;
    if (chunk & 1) return fail(PRNG_EINVAL, "request chunk must be even");
    const uint64_t rows = (r.length + chunk - 1) / chunk;
    if (rows > 0xFFFFFFFFull) return fail(PRNG_EINVAL, "request needs too many streams");
    d.seed = r.seed;
    d.first_stream = r.first_stream;
    d.per_stream = chunk;
    d.n_rows = (uint32_t)rows;
    d.resident = 0;
    d.full_rows = (uint32_t)(r.length / chunk);
  } else if (r.kind == PRNG_REQ_RESIDENT) {
    if (r.n_streams == 0 || r.first_stream >= h->n_streams || r.n_streams > h->n_streams - r.first_stream)
      return fail(PRNG_EINVAL, "resident request streams [%llu, +%llu) outside the handle's %llu streams",
                  (unsigned long long)r.first_stream, (unsigned long long)r.n_streams,
                  (unsigned long long)h->n_streams);
    // Rows of a multiple of 16 outputs: with a 128-byte aligned d_out every row starts on a
    // 128-byte line, so each 16-output row segment is written as four whole 32-byte sectors.
    const uint64_t sixteenths = (r.length + 16 * r.n_streams - 1) / (16 * r.n_streams);
    if (16 * sixteenths >= 0xFFFFFFFFull)
      return fail(PRNG_EINVAL, "resident request rows must hold fewer than 2^32 outputs");
    d.seed = 0;
    d.first_stream = r.first_stream;
    d.per_stream = 16 * sixteenths;
    d.n_rows = (uint32_t)r.n_streams;
    d.resident = 1;
    d.full_rows = (uint32_t)std::min<uint64_t>(r.length / d.per_stream, r.n_streams);
  } else {
    return fail(PRNG_EINVAL, "request kind %d", r.kind);
  }
  return PRNG_OK;
}

int submit(prng_ctx* h, const prng_request* reqs, int n, uint64_t* ticket, cudaStream_t s) {
  return submit_capped(h, reqs, n, ticket, s, 0);
}

int submit_capped(prng_ctx* h, const prng_request* reqs, int n, uint64_t* ticket, cudaStream_t s,
                  uint32_t items_per_warp, int warps) {
  if (n <= 0 || n > PRNG_MAX_BATCH_REQUESTS)
    return fail(PRNG_EINVAL, "a batch holds 1 .. %d requests", PRNG_MAX_BATCH_REQUESTS);
  std::vector<prngd::BatchDesc> d(n);
  std::vector<std::pair<uint64_t, uint64_t>> ranges;
  for (int i = 0; i < n; ++i) {
    int rc = describe(h, reqs[i], d[i]);
    if (rc) return rc;
    if (d[i].resident) ranges.push_back({d[i].first_stream, d[i].first_stream + d[i].n_rows});
  }
  std::sort(ranges.begin(), ranges.end());
  for (size_t i = 1; i < ranges.size(); ++i)
    if (ranges[i].first < ranges[i - 1].second)
      return fail(PRNG_EINVAL, "two resident requests of one batch use the same streams");
  int rc = ensure_engine(h);
  if (rc) return rc;
  BatchEngine* b = h->batch;
  // a free slot: its previous batch has finished (or it was never used)
  BatchSlot* sl = nullptr;
  for (int k = 0; k < kSlots && !sl; ++k) {
    BatchSlot& c = b->slot[(b->next_slot + k) % kSlots];
    if (c.ticket == 0 || cudaEventQuery(c.done) == cudaSuccess) {
      sl = &c;
      b->next_slot = (b->next_slot + k + 1) % kSlots;
    }
  }
  cudaGetLastError();
  if (!sl) return fail(PRNG_EBUSY, "all %d batch slots are in flight", kSlots);
  // longest rows first, so the long items start early
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return d[a].per_stream > d[c].per_stream; });
  uint64_t acc = 0;
  sl->h_meta[0] = (uint32_t)n;
  for (int i = 0; i < n; ++i) {
    sl->h_desc[i] = d[order[i]];
    sl->h_meta[1 + i] = (uint32_t)acc;
    acc += (d[order[i]].n_rows + 31) / 32;
    if (acc >= 0xFFFFFFFFull) return fail(PRNG_EINVAL, "a batch holds fewer than 2^37 rows");
  }
  sl->h_meta[1 + n] = (uint32_t)acc;
  for (int i = 0; i < n; ++i) {  // 2D maps of the full rows; a request without one uses plain stores
    prngd::BatchDesc& q = sl->h_desc[i];
    // rows that all start 16 bytes into a 32-byte sector: the map covers outputs 2 .. per_stream - 1
    // of each row, so that every tensor store writes whole sectors (batch_item_full)
    q.shift = (((uintptr_t)q.out & 31) == 16 && (q.per_stream & 3) == 0 && q.per_stream > 2) ? 1 : 0;
    const bool mapped =
        q.shift ? encode_out_map_box(&sl->h_maps[i], q.out + 2, q.full_rows, q.per_stream - 2,
                                     (uint32_t)prngd::kChunk, 32, q.per_stream * 8)
                : encode_out_map(&sl->h_maps[i], q.out, q.full_rows, q.per_stream);
    if (q.full_rows < 32 || !mapped) q.full_rows = 0;
  }
  // kernel: one form, mode 0 -> a single-form kernel; form B with exactly PRNG_MODE_BALANCED
  // -> its single-form kernel; forms A, B, C, mode 0 -> the mixed-form kernel; otherwise the
  // any-mode kernel
  int form_all = d[0].form;
  for (int i = 1; i < n && form_all >= 0; ++i)
    if (d[i].form != form_all) form_all = -1;
  bool all_b_round = true;  // every request form B with exactly PRNG_MODE_BALANCED
  for (int i = 0; i < n; ++i)
    all_b_round = all_b_round && d[i].form == PRNG_FORM_B_INTBITS && d[i].mode == PRNG_MODE_BALANCED;
  for (int i = 0; i < n; ++i)
    if (d[i].mode || d[i].form == PRNG_FORM_L_ALGO1) form_all = prngd::kAnyMode;
  if (all_b_round) form_all = prngd::kFormBBalanced;
  if (!items_per_warp) {
    rc = ensure_graph(h, *sl, form_all);
    if (rc) return rc;
  }
  cudaError_t e = cudaMemcpyAsync(sl->d_desc, sl->h_desc, sizeof(prngd::BatchDesc) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl->d_maps, sl->h_maps, sizeof(CUtensorMap) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(sl->d_meta, sl->h_meta, sizeof(uint32_t) * (n + 2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    if (items_per_warp) {
      const int wpb = (warps >= 1 && warps <= 8) ? warps : b->shape.warps_per_block;
      const uint64_t per_block = (uint64_t)wpb * items_per_warp;
      const uint64_t blocks = (acc + per_block - 1) / per_block;
      e = enqueue_batch(h, *sl, form_all, s, (unsigned)std::max<uint64_t>(1, blocks), n, items_per_warp, wpb);
    } else {
      e = cudaGraphLaunch(sl->exec[form_all + 2], s);
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(sl->done, s);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "batch launch: %s", cudaGetErrorString(e));
  sl->ticket = b->next_ticket++;
  *ticket = sl->ticket;
  return PRNG_OK;
}

int poll(prng_ctx* h, uint64_t ticket, int* done) {
  BatchEngine* b = h->batch;
  if (!b || ticket == 0 || ticket >= b->next_ticket) return fail(PRNG_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
  for (auto& s : b->slot) {
    if (s.ticket == ticket) {
      cudaError_t e = cudaEventQuery(s.done);
      if (e == cudaSuccess) {
        *done = 1;
      } else if (e == cudaErrorNotReady) {
        *done = 0;
        cudaGetLastError();
      } else {
        return fail(PRNG_ECUDA, "poll: %s", cudaGetErrorString(e));
      }
      return PRNG_OK;
    }
  }
  *done = 1;  // the slot has been reused since, so this batch finished before
  return PRNG_OK;
}

int set_batch_shape(prng_ctx* h, const BatchShape& sh) {
  int rc = ensure_engine(h);
  if (rc) return rc;
  if (sh.warps_per_block < 1 || sh.warps_per_block > 8 || sh.blocks_per_sm < 1 || sh.blocks_per_sm > 16 ||
      sh.items_per_ticket < 1 || sh.items_per_ticket > 64 ||
      (sh.outputs_per_chunk != prngd::kChunk && sh.outputs_per_chunk != 2 * prngd::kChunk))
    return fail(PRNG_EINVAL, "batch shape out of range");
  for (auto& s : h->batch->slot)
    if (s.ticket && cudaEventSynchronize(s.done) != cudaSuccess) return fail(PRNG_ECUDA, "sync before reshape");
  h->batch->shape = sh;
  h->batch->cfg_version++;
  return PRNG_OK;
}

int get_batch_shape(prng_ctx* h, BatchShape* sh) {
  int rc = ensure_engine(h);
  if (rc) return rc;
  *sh = h->batch->shape;
  return PRNG_OK;
}

// ----------------------------------------------------------------- autotuner
// Times each candidate launch shape on a synthetic batch of fresh requests whose lengths are
// log-uniform in [lo, hi] (deterministic, at most 2^30 outputs in total, 256-byte aligned
// outputs) and keeps the fastest.
// Results are cached in a text table, one line per key:
// "<key> <warps> <blocks> <items> <outputs per chunk> <ms>".
static std::string tune_key(prng_ctx* h, int form, uint64_t lo, uint64_t hi) {
  cudaDeviceProp pr;
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&pr, h->device) == cudaSuccess) name = pr.name;
  for (char& c : name)
    if (c == ' ') c = '_';
  char buf[256];
  snprintf(buf, sizeof(buf), "%s|w=%d|form=%d|len=%llu-%llu", name.c_str(), h->w, form, (unsigned long long)lo,
           (unsigned long long)hi);
  return buf;
}

static bool table_lookup(const char* path, const std::string& key, BatchShape* sh) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char k[256];
  int a, b, c, d;
  double ms;
  bool found = false;
  while (fscanf(f, "%255s %d %d %d %d %lf", k, &a, &b, &c, &d, &ms) == 6)
    if (key == k) {
      *sh = BatchShape{a, b, c, d};
      found = true;
    }
  fclose(f);
  return found;
}

// Outputs reserved for a request of L outputs in the tuning scratch: each request starts on a
// 256-byte boundary, as separately allocated outputs would.
static uint64_t slot_of(uint64_t L) { return (L + 31) & ~31ull; }

int autotune(prng_ctx* h, int form, uint64_t lo, uint64_t hi, const char* path, int force, BatchShape* best_out,
             double* best_ms) {
  if (lo == 0 || hi < lo) return fail(PRNG_EINVAL, "length range");
  const std::string key = tune_key(h, form, lo, hi);
  BatchShape found;
  if (!force && table_lookup(path, key, &found)) {
    int rc = set_batch_shape(h, found);
    if (rc) return rc;
    *best_out = found;
    if (best_ms) *best_ms = -1;
    return PRNG_OK;
  }
  // synthetic batch
  const int n = 256;
  std::vector<uint64_t> len(n);
  uint64_t total = 0, z = 0x2545F4914F6CDD1Dull;
  for (int i = 0; i < n; ++i) {
    z = z * 6364136223846793005ull + 1442695040888963407ull;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    len[i] = (uint64_t)std::exp(std::log((double)lo) + u * (std::log((double)hi) - std::log((double)lo)));
    if (len[i] < lo) len[i] = lo;
    total += slot_of(len[i]);
  }
  const uint64_t cap = 1ull << 30;  // about 2 ms per trial at full speed: long enough that tails do not decide
  if (total > cap) {
    const double f = (double)cap / total;
    total = 0;
    for (auto& L : len) {
      L = std::max<uint64_t>(1, (uint64_t)(L * f));
      total += slot_of(L);
    }
  }
  uint64_t* scratch = nullptr;
  cudaError_t e = cudaMalloc(&scratch, total * 8 + 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(PRNG_ENOMEM, "autotune scratch: %s", cudaGetErrorString(e));
  }
  std::vector<prng_request> reqs(n);
  uint64_t off = 0, first = 0;
  for (int i = 0; i < n; ++i) {
    prng_request& r = reqs[i];
    r = prng_request{};
    r.kind = PRNG_REQ_FRESH;
    r.form = form;
    r.length = len[i];
    r.seed = 1000 + i;
    r.first_stream = first;
    r.d_out = scratch + off;
    first += (len[i] + 1023) / 1024;
    off += slot_of(len[i]);
  }
  cudaStream_t st;
  cudaEvent_t a, b;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int W[] = {4, 8}, B[] = {2, 3, 4, 6, 8}, I[] = {1, 4, 8}, C[] = {prngd::kChunk, 2 * prngd::kChunk};
  BatchShape best = default_batch_shape(h->num_sms);
  double best_t = 1e30;
  int rc = PRNG_OK;
  for (int cv : C)
  for (int wv : W)
    for (int bv : B)
      for (int iv : I) {
        if (rc) break;
        rc = set_batch_shape(h, BatchShape{wv, bv, iv, cv});
        uint64_t t = 0;
        if (!rc) rc = submit(h, reqs.data(), n, &t, st);  // warm-up (captures the graph)
        if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(PRNG_ECUDA, "autotune sync");
        float times[3];
        for (int k = 0; k < 3 && !rc; ++k) {
          cudaEventRecord(a, st);
          rc = submit(h, reqs.data(), n, &t, st);
          cudaEventRecord(b, st);
          if (!rc && cudaEventSynchronize(b) != cudaSuccess) rc = fail(PRNG_ECUDA, "autotune sync");
          if (!rc) cudaEventElapsedTime(&times[k], a, b);
        }
        if (rc) break;
        std::sort(times, times + 3);
        if (times[1] < best_t) {
          best_t = times[1];
          best = BatchShape{wv, bv, iv, cv};
        }
      }
  cudaStreamSynchronize(st);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaStreamDestroy(st);
  cudaFree(scratch);
  if (rc) return rc;
  rc = set_batch_shape(h, best);
  if (rc) return rc;
  if (path) {
    FILE* f = fopen(path, "a");
    if (f) {
      fprintf(f, "%s %d %d %d %d %.6f\n", key.c_str(), best.warps_per_block, best.blocks_per_sm, best.items_per_ticket,
              best.outputs_per_chunk, best_t);
      fclose(f);
    }
  }
  *best_out = best;
  if (best_ms) *best_ms = best_t;
  return PRNG_OK;
}

}  // namespace prngd_host

using namespace prngd_host;

extern "C" {

int prng_submit(prng_t h, const prng_request* reqs, int n, uint64_t* ticket, void* cuda_stream) {
  if (!h || !reqs || !ticket) return fail(PRNG_EINVAL, "null argument");
  int rc = require_xorshift(h, "prng_submit");
  if (!rc) rc = check_handle_device(h);
  if (rc) return rc;
  return submit(h, reqs, n, ticket, (cudaStream_t)cuda_stream);
}

int prng_poll(prng_t h, uint64_t ticket, int* done) {
  if (!h || !done) return fail(PRNG_EINVAL, "null argument");
  return poll(h, ticket, done);
}

int prng_wait(prng_t h, uint64_t ticket, double timeout_s) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    int done = 0;
    int rc = poll(h, ticket, &done);
    if (rc) return rc;
    if (done) return PRNG_OK;
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > timeout_s)
      return fail(PRNG_ETIMEOUT, "ticket %llu not done after %.3f s", (unsigned long long)ticket, timeout_s);
  }
}

int prng_batch_get_shape(prng_t h, int* warps_per_block, int* blocks_per_sm, int* items_per_ticket,
                         int* outputs_per_chunk) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  BatchShape sh;
  int rc = get_batch_shape(h, &sh);
  if (rc) return rc;
  if (warps_per_block) *warps_per_block = sh.warps_per_block;
  if (blocks_per_sm) *blocks_per_sm = sh.blocks_per_sm;
  if (items_per_ticket) *items_per_ticket = sh.items_per_ticket;
  if (outputs_per_chunk) *outputs_per_chunk = sh.outputs_per_chunk;
  return PRNG_OK;
}

int prng_batch_autotune(prng_t h, int form, uint64_t length_lo, uint64_t length_hi, const char* table_path,
                        int force, int* warps_per_block, int* blocks_per_sm, int* items_per_ticket,
                        int* outputs_per_chunk, double* best_ms) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  if (form != PRNG_FORM_A_FP64 && form != PRNG_FORM_B_INTBITS && form != PRNG_FORM_C_F32PAIR)
    return fail(PRNG_EINVAL, "form %d", form);
  int rc = check_handle_device(h);
  if (rc) return rc;
  BatchShape sh;
  rc = autotune(h, form, length_lo, length_hi, table_path, force, &sh, best_ms);
  if (rc) return rc;
  if (warps_per_block) *warps_per_block = sh.warps_per_block;
  if (blocks_per_sm) *blocks_per_sm = sh.blocks_per_sm;
  if (items_per_ticket) *items_per_ticket = sh.items_per_ticket;
  if (outputs_per_chunk) *outputs_per_chunk = sh.outputs_per_chunk;
  return PRNG_OK;
}

int prng_batch_set_shape(prng_t h, int warps_per_block, int blocks_per_sm, int items_per_ticket,
                         int outputs_per_chunk) {
  if (!h) return fail(PRNG_EINVAL, "null handle");
  BatchShape sh{warps_per_block, blocks_per_sm, items_per_ticket, outputs_per_chunk};
  return set_batch_shape(h, sh);
}

}  // extern "C"
