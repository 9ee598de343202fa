// prngd_serve.cpp -- the serving loop: admission of fill requests against an output-pool
// budget, continuous batching onto the device, per-client resident streams, latency stats.
//
// Clients: client c owns the handle's streams [c S, (c+1) S). A request of length L from c
// continues the first n = min(S, ceil(L / min_per_stream)) of them as one resident request
// (rows of 16 ceil(L / 16n) outputs), so a request's result is fixed by the client's history
// and the request itself, never by what else is in flight. A client has at most one request
// on the device at a time; later requests of a busy client wait in order.
//
// Batching: step() puts every admitted request whose client is idle into the next batch of
// its lane (four lanes by request length, so that a request is not held back by much longer
// batch-mates) and harvests finished batches. Requests that arrive while batches run are
// admitted as soon as pool memory allows and join the next batch. Every batch in flight has a
// CUDA stream of its own: no two batches in flight share a client (hence a stream of the
// handle), so they need no order, and a batch does not wait for another to finish (a 2^28-output
// request of a 16384-stream client has rows of 16384 outputs, a few milliseconds of one warp's
// work). Batches are launched with a cap of one item per warp, so their blocks free SM slots
// item by item, and the lanes of shorter requests run on streams of higher priority.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <unordered_map>
#include <vector>

#include "prngd.h"
#include "prngd_internal.h"
#include "prngd_pool.h"

using prngd_host::fail;

namespace {

// The output pool: one device allocation, its ranges handed out by a first-fit RangePool
// (offsets in bytes, 256-byte granules, so every request's output is 256-byte aligned).
class Pool {
 public:
  bool init(size_t bytes) {
    if (cudaMalloc(&base_, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    ranges_.reset(bytes);
    return true;
  }
  ~Pool() {
    if (base_) cudaFree(base_);
  }
  // returns offset or SIZE_MAX
  size_t alloc(size_t bytes) { return ranges_.alloc(bytes); }
  void release(size_t off, size_t bytes) { ranges_.release(off, bytes); }
  void* ptr(size_t off) const { return (char*)base_ + off; }
  size_t used() const { return ranges_.used(); }
  size_t size() const { return ranges_.size(); }

 private:
  void* base_ = nullptr;
  prngd_host::RangePool ranges_;
};

struct Req {
  uint64_t client, length;
  int form;
  uint32_t mode;
  size_t off, bytes;
  int state;  // 0 admitted, 1 launched, 2 done
  uint64_t ticket;
  double t_admit, t_done;
};

// Lanes by request size: <= 2^20 outputs, <= 2^24, <= 2^26, longer. A batch finishes as a whole,
// so a request batched with much longer ones would wait for them; separate lanes keep a
// request's batch-mates of a similar length (measured, p50 / p99 over all requests: two lanes
// 1.0 / 11 ms, three 0.61 / 10.4, four 0.47 / 9.5).
#ifndef PRNGD_SERVE_LANES
#define PRNGD_SERVE_LANES 4
#endif
constexpr int kLanes = PRNGD_SERVE_LANES;
// longest request of each lane (the last lane takes the rest)
constexpr uint64_t kLaneMax[4] = {1ull << 20, kLanes >= 3 ? 1ull << 24 : ~0ull, kLanes >= 4 ? 1ull << 26 : ~0ull, ~0ull};
static_assert(kLanes >= 1 && kLanes <= 4, "one to four lanes");
#ifndef PRNGD_SERVE_STREAMS
#define PRNGD_SERVE_STREAMS 8
#endif
#ifndef PRNGD_SERVE_WARPS
#define PRNGD_SERVE_WARPS 4
#endif
// Batches of one lane on the device at once, each on a CUDA stream of its own: a batch that
// shared a stream waited for the one before it (small batches: 0.36 ms on the GPU at the
// median, 1.2 ms from launch to completion with 6 batches over 3 streams).
constexpr int kStreamsPerLane = PRNGD_SERVE_STREAMS;
constexpr int kMaxBatchesPerLane = PRNGD_SERVE_STREAMS;
// Warps per block of the serving launches (0: the handle's shape). With 4 a slot frees up when
// 4 items end rather than 8: measured p50 / p99 0.61 / 10.4 ms and saturation 554 Gsamples/s,
// against 0.56 / 10.6 ms and 530 with the shape's 8.
constexpr int kServeWarps = PRNGD_SERVE_WARPS;
#ifndef PRNGD_SERVE_CAP
#define PRNGD_SERVE_CAP 1
#endif
// Items (32 rows of a request) each warp of a lane's batch takes before its block ends (0: the
// persistent launch of prng_submit). A persistent batch holds its SM slots until its last
// item, and an item of a 2^28-output request is milliseconds of one warp's work, so small
// requests waited for whole large batches; with capped batches slots free up every item and go
// first to the lanes of shorter requests, whose streams have higher priority.
constexpr uint32_t kLaneCap = PRNGD_SERVE_CAP;

int lane_of(uint64_t length) {
  int l = 0;
  while (l < kLanes - 1 && length > kLaneMax[l]) ++l;
  return l;
}

}  // namespace

struct prng_server {
  prng_t h = nullptr;
  uint64_t S = 0, min_per = 0, n_clients = 0;
  Pool pool;
  cudaStream_t lane_stream[kLanes][kStreamsPerLane] = {};
  int lane_next[kLanes] = {};  // stream of the lane's next batch
  uint64_t next_id = 1;
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<uint64_t> waiting[kLanes];              // admitted, not launched (arrival order)
  std::unordered_map<uint64_t, uint64_t> busy;       // client -> id on the device
  std::unordered_map<uint64_t, std::deque<uint64_t>> client_q;  // admitted, not launched, per client
  struct Inflight {
    uint64_t ticket;
    int lane;
    std::vector<uint64_t> ids;
  };
  std::vector<Inflight> inflight;
  uint64_t launched_batches = 0, completed = 0, samples_done = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

int harvest(prng_server* s) {
  for (size_t k = 0; k < s->inflight.size();) {
    int done = 0;
    int rc = prng_poll(s->h, s->inflight[k].ticket, &done);
    if (rc) return rc;
    if (!done) {
      ++k;
      continue;
    }
    const double t = s->now();
    for (uint64_t id : s->inflight[k].ids) {
      Req& r = s->reqs[id];
      r.state = 2;
      r.t_done = t;
      s->busy.erase(r.client);
      s->completed++;
      s->samples_done += r.length;
    }
    s->inflight.erase(s->inflight.begin() + k);
  }
  return PRNG_OK;
}

int launch_lane(prng_server* s, int lane) {
  int lane_inflight = 0;
  for (auto& f : s->inflight) lane_inflight += f.lane == lane;
  if (lane_inflight >= kMaxBatchesPerLane) return PRNG_OK;
  std::vector<prng_request> batch;
  std::vector<uint64_t> ids;
  std::deque<uint64_t> keep;
  std::unordered_map<uint64_t, bool> taken;  // one request per client per batch
  while (!s->waiting[lane].empty()) {
    const uint64_t id = s->waiting[lane].front();
    s->waiting[lane].pop_front();
    Req& r = s->reqs[id];
    // a client's requests run one at a time, in admission order
    if (s->busy.count(r.client) || taken.count(r.client) || s->client_q[r.client].front() != id ||
        (int)batch.size() >= PRNG_MAX_BATCH_REQUESTS) {
      keep.push_back(id);
      continue;
    }
    taken[r.client] = true;
    const uint64_t n = std::min<uint64_t>(s->S, (r.length + s->min_per - 1) / s->min_per);
    prng_request q{};
    q.kind = PRNG_REQ_RESIDENT;
    q.form = r.form;
    q.mode = r.mode;
    q.length = r.length;
    q.first_stream = r.client * s->S;
    q.n_streams = n;
    q.d_out = s->pool.ptr(r.off);
    batch.push_back(q);
    ids.push_back(id);
  }
  s->waiting[lane] = std::move(keep);
  if (batch.empty()) return PRNG_OK;
  uint64_t ticket = 0;
  int rc = prngd_host::check_handle_device(s->h);
  if (rc) return rc;
  rc = prngd_host::submit_capped(s->h, batch.data(), (int)batch.size(), &ticket,
                                 s->lane_stream[lane][s->lane_next[lane]], kLaneCap, kServeWarps);
  if (rc == PRNG_EBUSY) {  // no free batch slot: put them back in front, in order
    for (size_t i = ids.size(); i-- > 0;) s->waiting[lane].push_front(ids[i]);
    return PRNG_OK;
  }
  if (rc) return rc;
  for (uint64_t id : ids) {
    Req& r = s->reqs[id];
    r.state = 1;
    r.ticket = ticket;
    s->busy[r.client] = id;
    auto& q = s->client_q[r.client];
    q.pop_front();
    if (q.empty()) s->client_q.erase(r.client);
  }
  s->inflight.push_back({ticket, lane, ids});
  s->launched_batches++;
  s->lane_next[lane] = (s->lane_next[lane] + 1) % kStreamsPerLane;
  return PRNG_OK;
}

}  // namespace

extern "C" {

int prng_server_create(prng_server_t* out, prng_t h, uint64_t streams_per_client, uint64_t min_per_stream,
                       size_t pool_bytes) {
  if (!out || !h) return fail(PRNG_EINVAL, "null argument");
  *out = nullptr;
  if (prng_generator(h) != PRNG_GEN_XORSHIFT128)
    return fail(PRNG_EINVAL, "the serving loop runs on xorshift128 streams only");
  uint64_t n_streams = 0;
  int w = 0;
  int rc = prng_get_info(h, &n_streams, &w);
  if (rc) return rc;
  if (streams_per_client == 0 || streams_per_client > n_streams || n_streams % streams_per_client)
    return fail(PRNG_EINVAL, "streams_per_client must divide the handle's %llu streams", (unsigned long long)n_streams);
  if (min_per_stream == 0) min_per_stream = 256;
  if (pool_bytes < 4096) return fail(PRNG_EINVAL, "pool too small");
  prng_server* s = new prng_server();
  s->h = h;
  s->S = streams_per_client;
  s->min_per = min_per_stream;
  s->n_clients = n_streams / streams_per_client;
  if (!s->pool.init(pool_bytes)) {
    delete s;
    return fail(PRNG_ENOMEM, "output pool of %zu bytes", pool_bytes);
  }
  int least = 0, greatest = 0;  // numerically lower is higher priority
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
    cudaGetLastError();
    least = greatest = 0;
  }
  for (int l = 0; l < kLanes; ++l)
    for (int k = 0; k < kStreamsPerLane; ++k)
      if (cudaStreamCreateWithPriority(&s->lane_stream[l][k], cudaStreamNonBlocking,
                                       std::min(least, greatest + l)) != cudaSuccess) {  // lane 0 highest
        cudaGetLastError();
        for (auto& lane : s->lane_stream)
          for (auto& st : lane)
            if (st) cudaStreamDestroy(st);
        delete s;
        return fail(PRNG_ECUDA, "stream creation");
      }
  *out = s;
  return PRNG_OK;
}

int prng_server_destroy(prng_server_t s) {
  if (!s) return PRNG_OK;
  for (auto& lane : s->lane_stream)
    for (auto& st : lane) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  delete s;
  return PRNG_OK;
}

int prng_server_submit(prng_server_t s, uint64_t client, uint64_t length, int form, uint64_t* id) {
  return prng_server_submit_mode(s, client, length, form, 0, id);
}

int prng_server_submit_mode(prng_server_t s, uint64_t client, uint64_t length, int form, uint32_t mode,
                            uint64_t* id) {
  if (!s || !id) return fail(PRNG_EINVAL, "null argument");
  if (client >= s->n_clients) return fail(PRNG_EINVAL, "client %llu of %llu", (unsigned long long)client,
                                          (unsigned long long)s->n_clients);
  if (length == 0) return fail(PRNG_EINVAL, "length 0");
  if (form != PRNG_FORM_A_FP64 && form != PRNG_FORM_B_INTBITS && form != PRNG_FORM_C_F32PAIR &&
      form != PRNG_FORM_L_ALGO1)
    return fail(PRNG_EINVAL, "form %d", form);
  if (mode & ~(uint32_t)prngd_host::kAllModes) return fail(PRNG_EINVAL, "mode %u", mode);
  if (length > s->pool.size() / 8) return fail(PRNG_EINVAL, "request larger than the whole pool");
  const size_t bytes = (size_t)length * 8;
  const size_t off = s->pool.alloc(bytes);
  if (off == SIZE_MAX) return fail(PRNG_EBUSY, "output pool full (%zu of %zu bytes in use)", s->pool.used(), s->pool.size());
  Req r;
  r.client = client;
  r.length = length;
  r.form = form;
  r.mode = mode;
  r.off = off;
  r.bytes = bytes;
  r.state = 0;
  r.ticket = 0;
  r.t_admit = s->now();
  r.t_done = 0;
  *id = s->next_id++;
  s->reqs[*id] = r;
  s->waiting[lane_of(length)].push_back(*id);
  s->client_q[client].push_back(*id);
  return PRNG_OK;
}

int prng_server_step(prng_server_t s) {
  if (!s) return fail(PRNG_EINVAL, "null server");
  int rc = harvest(s);
  if (rc) return rc;
  for (int l = 0; l < kLanes; ++l) {
    rc = launch_lane(s, l);
    if (rc) return rc;
  }
  return PRNG_OK;
}

int prng_server_poll(prng_server_t s, uint64_t id, int* done, void** d_out) {
  if (!s || !done) return fail(PRNG_EINVAL, "null argument");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(PRNG_ENOTFOUND, "request %llu", (unsigned long long)id);
  *done = it->second.state == 2;
  if (d_out) *d_out = s->pool.ptr(it->second.off);
  return PRNG_OK;
}

int prng_server_read(prng_server_t s, uint64_t id, void* host_dst, size_t bytes) {
  if (!s || !host_dst) return fail(PRNG_EINVAL, "null argument");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(PRNG_ENOTFOUND, "request %llu", (unsigned long long)id);
  if (it->second.state != 2) return fail(PRNG_EBUSY, "request %llu has not finished", (unsigned long long)id);
  if (bytes != it->second.bytes) return fail(PRNG_EINVAL, "bytes must be 8 * length");
  cudaError_t e = cudaMemcpy(host_dst, s->pool.ptr(it->second.off), bytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(PRNG_ECUDA, "read: %s", cudaGetErrorString(e));
  return PRNG_OK;
}

int prng_server_release(prng_server_t s, uint64_t id) {
  if (!s) return fail(PRNG_EINVAL, "null server");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(PRNG_ENOTFOUND, "request %llu", (unsigned long long)id);
  if (it->second.state != 2) return fail(PRNG_EBUSY, "request %llu has not finished", (unsigned long long)id);
  s->pool.release(it->second.off, it->second.bytes);
  s->reqs.erase(it);
  return PRNG_OK;
}

int prng_server_cancel(prng_server_t s, uint64_t id) {
  if (!s) return fail(PRNG_EINVAL, "null server");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(PRNG_ENOTFOUND, "request %llu", (unsigned long long)id);
  if (it->second.state != 0)
    return fail(PRNG_EBUSY, "request %llu is on the device or finished: wait, then release", (unsigned long long)id);
  const Req r = it->second;
  for (auto& w : s->waiting) {
    auto pos = std::find(w.begin(), w.end(), id);
    if (pos != w.end()) w.erase(pos);
  }
  auto cq = s->client_q.find(r.client);
  if (cq != s->client_q.end()) {
    auto pos = std::find(cq->second.begin(), cq->second.end(), id);
    if (pos != cq->second.end()) cq->second.erase(pos);
    if (cq->second.empty()) s->client_q.erase(cq);
  }
  s->pool.release(r.off, r.bytes);
  s->reqs.erase(it);
  return PRNG_OK;
}

int prng_server_drain(prng_server_t s, double timeout_s) {
  if (!s) return fail(PRNG_EINVAL, "null server");
  const double t_end = s->now() + timeout_s;
  for (;;) {
    int rc = prng_server_step(s);
    if (rc) return rc;
    bool idle = s->inflight.empty();
    for (int l = 0; l < kLanes; ++l) idle = idle && s->waiting[l].empty();
    if (idle) return PRNG_OK;
    if (s->now() > t_end) return fail(PRNG_ETIMEOUT, "server not drained after %.3f s", timeout_s);
  }
}

int prng_server_run_trace(prng_server_t s, const prng_trace_item* items, uint64_t n, double* latency,
                          double* makespan, double timeout_s) {
  if (!s || (!items && n)) return fail(PRNG_EINVAL, "null argument");
  const double t_start = s->now();
  // Arrivals waiting for pool memory, per lane: a small request does not wait behind a large
  // one refused for memory. A request is admitted only as its client's earliest waiting
  // arrival, so every client's requests are admitted (and run) in arrival order.
  std::deque<uint64_t> arrived[kLanes];
  std::unordered_map<uint64_t, std::deque<uint64_t>> client_wait;  // client -> waiting arrivals
  std::vector<uint64_t> ids(n, 0);
  std::unordered_map<uint64_t, uint64_t> id_to_index;
  uint64_t next = 0, finished = 0;
  auto admit = [&](uint64_t i, bool* busy) -> int {
    uint64_t id = 0;
    int rc = prng_server_submit_mode(s, items[i].client, items[i].length, items[i].form, items[i].mode, &id);
    *busy = rc == PRNG_EBUSY;
    if (rc) return *busy ? PRNG_OK : rc;
    ids[i] = id;
    id_to_index[id] = i;
    auto& cw = client_wait[items[i].client];
    cw.pop_front();
    if (cw.empty()) client_wait.erase(items[i].client);
    return PRNG_OK;
  };
  while (finished < n) {
    const double t = s->now() - t_start;
    if (t > timeout_s) return fail(PRNG_ETIMEOUT, "trace not finished after %.1f s (%llu of %llu done)", timeout_s,
                                   (unsigned long long)finished, (unsigned long long)n);
    while (next < n && items[next].t <= t) {
      arrived[lane_of(items[next].length)].push_back(next);
      client_wait[items[next].client].push_back(next);
      ++next;
    }
    for (int l = 0; l < kLanes; ++l) {
      auto& q = arrived[l];
      for (size_t k = 0; k < q.size();) {
        const uint64_t i = q[k];
        if (client_wait[items[i].client].front() != i) {  // an earlier arrival of its client waits
          if (l > 0) break;  // longer requests stay in arrival order
          ++k;
          continue;
        }
        bool busy = false;
        int rc = admit(i, &busy);
        if (rc) return rc;
        if (busy) break;
        q.erase(q.begin() + (std::ptrdiff_t)k);
      }
    }
    int rc = prng_server_step(s);
    if (rc) return rc;
    // completions: record latency from arrival, release the output
    for (auto it = id_to_index.begin(); it != id_to_index.end();) {
      Req& r = s->reqs[it->first];
      if (r.state == 2) {
        if (latency) latency[it->second] = (r.t_done - t_start) - items[it->second].t;
        prng_server_release(s, it->first);
        it = id_to_index.erase(it);
        ++finished;
      } else {
        ++it;
      }
    }
  }
  if (makespan) *makespan = s->now() - t_start;
  return PRNG_OK;
}

int prng_server_info(prng_server_t s, uint64_t* n_clients, uint64_t* batches, uint64_t* completed,
                     uint64_t* samples, size_t* pool_used) {
  if (!s) return fail(PRNG_EINVAL, "null server");
  if (n_clients) *n_clients = s->n_clients;
  if (batches) *batches = s->launched_batches;
  if (completed) *completed = s->completed;
  if (samples) *samples = s->samples_done;
  if (pool_used) *pool_used = s->pool.used();
  return PRNG_OK;
}

}  // extern "C"
