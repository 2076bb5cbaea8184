// Serving loop: continuous batching of independent RVEA runs.
//
// A client of the library's own C ABI (rvea_init_ex, rvea_autotune,
// rvea_step_batch, rvea_population, rvea_objectives): requests (a run
// configuration and a generation budget) queue on the host; between steps
// the loop admits queued requests in arrival order while their workspaces
// fit the device arena (the HBM budget, owned by the caller); every step
// runs one generation of every live run, packed into batched launches of up
// to 320 runs; a run whose budget is spent leaves the batch and waits, on
// the device, until its result is fetched, which returns its memory.
// Requests that arrive while others are on the GPU therefore join at the
// next step, and each run's result is the bits it gets alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <new>
#include <vector>

#include "../../include/rvea.h"
#include "nvtx_range.h"

namespace {

constexpr int kBatchMax = 320;   // runs per batched launch (rvea_step_batch)
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over [0, size) with coalescing of free neighbours.
class Arena {
 public:
  explicit Arena(size_t size) { free_[0] = size; }
  // offset of a block of `bytes`, or SIZE_MAX
  size_t alloc(size_t bytes) {
    bytes = align_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      used_ += bytes;
      return off;
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;   // offset -> size
  size_t used_ = 0;
};

struct Request {
  int64_t id;
  rvea_config cfg;
  int generations;
};

struct Live {
  int64_t id;
  rvea_run *run;
  size_t off, bytes;
  int left;   // generations still to run
};

}  // namespace

struct rvea_server {
  uint8_t *arena_base = nullptr;
  size_t arena_bytes = 0;
  Arena arena;
  int max_live = 0;
  int tune = 1;
  int64_t next_id = 1;
  std::list<Request> queue;
  std::vector<Live> live;
  std::map<int64_t, Live> done;        // budget spent, result not fetched yet
  std::map<int64_t, rvea_status> failed;   // admission failed, error not fetched yet
  std::vector<int64_t> done_unpolled;
  long long gens_run = 0;
  cudaStream_t init_stream = nullptr;   // admissions' initialisation and tuning
  cudaEvent_t init_done = nullptr;      // the last admission's work, for the step stream
  int head_skips = 0;                   // steps the queue's head has been passed over
  explicit rvea_server(size_t bytes) : arena(bytes) {}
};

namespace {
constexpr int kBackfillLookahead = 64;   // queued requests an admission round looks at
constexpr int kHeadSkipsMax = 32;        // steps a waiting head can be passed over
}  // namespace

extern "C" {

rvea_status rvea_server_create(void *dev_arena, size_t arena_bytes, int max_live, int autotune,
                               rvea_server **out) {
  if (!dev_arena || !out || arena_bytes < kAlign || max_live < 1 ||
      (reinterpret_cast<uintptr_t>(dev_arena) & (kAlign - 1)))
    return RVEA_ERR_ARG;
  rvea_server *s = new (std::nothrow) rvea_server(arena_bytes);
  if (!s) return RVEA_ERR_NOMEM;
  s->arena_base = static_cast<uint8_t *>(dev_arena);
  s->arena_bytes = arena_bytes;
  s->max_live = max_live;
  s->tune = autotune ? 1 : 0;
  *out = s;
  return RVEA_OK;
}

rvea_status rvea_server_submit(rvea_server *s, const rvea_config *cfg, int generations,
                               int64_t *id_out) {
  if (!s || !cfg || generations < 1 || cfg->neuro) return RVEA_ERR_ARG;
  // an invalid configuration, or one whose workspace can never fit the
  // arena, is refused at once (it would otherwise block the queue's head)
  const size_t need = rvea_workspace_bytes_ex(cfg);
  if (need == 0) return RVEA_ERR_ARG;
  if (align_up(need) > s->arena_bytes) return RVEA_ERR_NOMEM;
  Request r;
  r.id = s->next_id++;
  r.cfg = *cfg;
  r.generations = generations;
  s->queue.push_back(r);
  if (id_out) *id_out = r.id;
  return RVEA_OK;
}

rvea_status rvea_server_step(rvea_server *s, void *cuda_stream, rvea_server_stats *stats) {
  if (!s) return RVEA_ERR_ARG;
  const rvea::NvtxRange nr("rvea server step", (int64_t)s->live.size());
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // one generation of every live run, enqueued first: the GPU works on it
  // while the host admits new requests below
  std::vector<rvea_run *> runs;
  runs.reserve(s->live.size());
  for (const Live &l : s->live) runs.push_back(l.run);
  for (size_t a = 0; a < runs.size(); a += kBatchMax) {
    const int n = (int)std::min<size_t>(kBatchMax, runs.size() - a);
    const rvea_status sr = rvea_step_batch(runs.data() + a, n, cuda_stream);
    if (sr != RVEA_OK) return sr;
  }
  s->gens_run += (long long)runs.size();
  // runs whose budget is spent leave the batch
  std::vector<Live> keep;
  keep.reserve(s->live.size());
  for (Live &l : s->live) {
    if (--l.left > 0) {
      keep.push_back(l);
    } else {
      s->done[l.id] = l;
      s->done_unpolled.push_back(l.id);
    }
  }
  s->live.swap(keep);
  // admission on the server's own stream (initialisation and tuning
  // synchronise that stream, not the step's): in arrival order, and past a
  // head that does not fit yet (backfill) unless the head has waited
  // kHeadSkipsMax steps already
  int admitted = 0;
  bool head_passed = false;
  // the admission stream and its event, made at the first admission (a
  // server can be created and fed requests without a device)
  bool have_stream = s->init_stream != nullptr;
  if (!have_stream && !s->queue.empty()) {
    have_stream = cudaStreamCreateWithFlags(&s->init_stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&s->init_done, cudaEventDisableTiming) == cudaSuccess;
    if (!have_stream) {
      cudaGetLastError();
      if (s->init_stream) cudaStreamDestroy(s->init_stream);
      s->init_stream = nullptr;
      s->init_done = nullptr;
    }
  }
  int looked = 0;
  for (auto it = s->queue.begin();
       it != s->queue.end() && (int)s->live.size() < s->max_live && looked < kBackfillLookahead;
       ++looked) {
    const Request q = *it;
    const size_t bytes = rvea_workspace_bytes_ex(&q.cfg);
    const size_t off = s->arena.alloc(bytes);
    if (off == SIZE_MAX) {
      if (it == s->queue.begin()) {
        head_passed = true;
        if (s->head_skips >= kHeadSkipsMax) break;   // let the arena drain for the head
      }
      ++it;
      continue;
    }
    rvea_run *run = nullptr;
    rvea_status sa = have_stream
                         ? rvea_init_ex(&q.cfg, s->arena_base + off, bytes, s->init_stream, &run)
                         : RVEA_ERR_CUDA;
    if (sa == RVEA_OK && s->tune) sa = rvea_autotune(run, s->init_stream, 1, nullptr);
    const bool was_head = it == s->queue.begin();
    it = s->queue.erase(it);
    if (was_head) s->head_skips = 0;
    if (sa != RVEA_OK) {
      // the request ends here: poll reports its id, fetch returns this error
      if (run) rvea_free(run);
      s->arena.release(off, bytes);
      s->failed[q.id] = sa;
      s->done_unpolled.push_back(q.id);
      continue;
    }
    s->live.push_back(Live{q.id, run, off, bytes, q.generations});
    ++admitted;
  }
  if (head_passed && !s->queue.empty()) ++s->head_skips;
  if (admitted > 0) {
    // the next step's launches on the step stream follow the new runs' set-up
    if (cudaEventRecord(s->init_done, s->init_stream) != cudaSuccess ||
        cudaStreamWaitEvent(st, s->init_done, 0) != cudaSuccess)
      return RVEA_ERR_CUDA;
  }
  if (stats) {
    stats->live = (int)s->live.size();
    stats->queued = (int)s->queue.size();
    stats->finished = (int)(s->done.size() + s->failed.size());
    stats->admitted = admitted;
    stats->arena_used = s->arena.used();
    stats->generations = s->gens_run;
  }
  return RVEA_OK;
}

rvea_status rvea_server_poll(rvea_server *s, int64_t *ids, int cap, int *n_out) {
  if (!s || !n_out || cap < 0 || (cap > 0 && !ids)) return RVEA_ERR_ARG;
  const int n = std::min<int>(cap, (int)s->done_unpolled.size());
  for (int q = 0; q < n; ++q) ids[q] = s->done_unpolled[q];
  s->done_unpolled.erase(s->done_unpolled.begin(), s->done_unpolled.begin() + n);
  *n_out = n;
  return RVEA_OK;
}

rvea_status rvea_server_fetch(rvea_server *s, int64_t id, float *X, float *F, uint8_t *valid,
                              void *cuda_stream) {
  if (!s) return RVEA_ERR_ARG;
  const auto fit = s->failed.find(id);
  if (fit != s->failed.end()) {   // admission failed: its error, once
    const rvea_status st = fit->second;
    s->failed.erase(fit);
    return st;
  }
  auto it = s->done.find(id);
  if (it == s->done.end()) return RVEA_ERR_STATE;
  Live l = it->second;
  rvea_status st = RVEA_OK;
  if (X) st = rvea_population(l.run, X, valid, cuda_stream);
  if (st == RVEA_OK && F) st = rvea_objectives(l.run, F, valid, cuda_stream);
  if (st != RVEA_OK) return st;
  // the copies read the run's memory: let them land before it is reused
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess)
    return RVEA_ERR_CUDA;
  st = rvea_sync_status(l.run);
  rvea_free(l.run);
  s->arena.release(l.off, l.bytes);
  s->done.erase(it);
  return st;
}

void rvea_server_free(rvea_server *s) {
  if (!s) return;
  for (Live &l : s->live) rvea_free(l.run);
  for (auto &kv : s->done) rvea_free(kv.second.run);
  if (s->init_done) cudaEventDestroy(s->init_done);
  if (s->init_stream) cudaStreamDestroy(s->init_stream);
  delete s;
}

}  // extern "C"
