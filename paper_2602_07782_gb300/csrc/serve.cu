// Serving loop: continuous batching of packing requests on one GPU.
//
// A server owns a device-memory budget split into L lanes.  A lane is a
// packing context (its slice of the budget as arena, its graphs) with its
// own stream and pinned staging.  Requests are queued as they are submitted;
// a worker thread forms a batch for every idle lane from the head of the
// queue (arrival order, as many as the lane's arena admits, up to a request
// cap), stages the inputs in pinned memory and launches the batch on the
// lane's stream.  Batches of different lanes run on the device at the same
// time, so requests that arrive while others are on the GPU start as soon as
// a lane is free.  A host function enqueued behind each batch marks the lane
// finished; the worker then hands every request its status, scale and
// placements, and the lane takes the next batch.  Each request gets exactly
// the result it would get alone: batching never changes a result.
//
// No thread waits on the device without a bound: the worker sleeps on a
// condition variable with a short timeout, waiters use tabi_wait's timeout,
// and shutdown gives in-flight batches a bounded time before it gives up on
// them (TABI_ERR_TIMEOUT).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "context.h"

using namespace tabi;

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

struct Ticket {
  tabi_request req{};  // the caller's request (host pointers)
  size_t est = 0;      // arena bytes the request may need
  int64_t t_submit = 0, t_start = 0, t_done = 0;
  int32_t status = TABI_PENDING, k = 0;
  int64_t quality[3] = {-1, -1, -1};  // overlap, gutter, outside texels (-1: unchecked)
  bool done = false;
};

struct Lane {
  tabi_ctx *ctx = nullptr;
  cudaStream_t st = nullptr;
  char *stage = nullptr;  // pinned: the batch's inputs and placements
  size_t stage_bytes = 0;
  size_t budget = 0;      // arena bytes
  std::vector<tabi_request> reqs;  // the staged copies of the batch
  std::vector<uint64_t> ids;
  InFlight fl;
  std::atomic<int> finished{0};  // set by the host function behind the batch
  bool busy = false;
};

}  // namespace

struct tabi_server {
  tabi_server_config cfg{};
  tabi_params params{};
  char *arena = nullptr;
  std::vector<std::unique_ptr<Lane>> lanes;
  std::mutex mu;
  std::condition_variable wake;  // the worker: a submission, a finished lane, shutdown
  std::condition_variable done;  // waiters: a finished request
  std::deque<uint64_t> queue;    // submitted, not yet launched, in arrival order
  std::unordered_map<uint64_t, Ticket> tickets;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  tabi_server_stats stats{};
  int64_t t0 = 0;
};

namespace {

void CUDART_CB lane_finished(void *arg) {
  // runs on a CUDA driver thread: no CUDA calls and no locks here
  auto *pair = static_cast<std::pair<tabi_server *, Lane *> *>(arg);
  pair->second->finished.store(1);
  pair->first->wake.notify_one();
  delete pair;
}

// The host walks a request's vertex loops (request_bytes) before any device
// check runs, so the offsets are checked here first: they start at 0, end
// at n_verts and give every chart at least three vertices (so they never
// decrease and never pass n_verts).
bool offsets_valid(const tabi_request &r) {
  if (r.offsets[0] != 0 || r.offsets[r.n_charts] != (uint32_t)r.n_verts) return false;
  for (int c = 0; c < r.n_charts; ++c)
    if (r.offsets[c + 1] < r.offsets[c] || r.offsets[c + 1] - r.offsets[c] < 3 ||
        r.offsets[c + 1] > (uint32_t)r.n_verts)
      return false;
  return true;
}

// Arena bytes a request may need at fan-out F: the per-chart arrays, and
// the envelope pools of one wave of F candidates at most as large as at
// k = 1024 (column words, their chart indices, row words; each at most the
// summed AABB extent plus the gutters).
size_t request_bytes(const tabi_request &r, int F, int gutter) {
  int64_t ext = 0;
  for (int c = 0; c < r.n_charts; ++c) {
    int32_t mnx = 0x7fffffff, mny = 0x7fffffff, mxx = -0x7fffffff - 1, mxy = -0x7fffffff - 1;
    for (uint32_t v = r.offsets[c]; v < r.offsets[c + 1]; ++v) {
      mnx = std::min(mnx, r.verts[2 * v]);
      mxx = std::max(mxx, r.verts[2 * v]);
      mny = std::min(mny, r.verts[2 * v + 1]);
      mxy = std::max(mxy, r.verts[2 * v + 1]);
    }
    ext += ((int64_t)mxx - mnx + 255) / 256 + ((int64_t)mxy - mny + 255) / 256 + 2;
  }
  const size_t per_cand = 3 * 4 * ((size_t)ext + (size_t)r.n_charts * (2 * (size_t)gutter + 2) + 4);
  return tabi_arena_bytes(r.n_charts, r.n_verts, r.atlas_w, r.atlas_h, ext, gutter) -
         (size_t)kScales * per_cand + (size_t)F * per_cand;
}

bool ensure_stage(Lane &ln, size_t bytes) {
  if (ln.stage_bytes >= bytes) return true;
  if (ln.stage) cudaFreeHost(ln.stage);
  ln.stage = nullptr;
  ln.stage_bytes = 0;
  const size_t want = std::max(bytes + bytes / 2, (size_t)64 << 20);
  if (cudaMallocHost(&ln.stage, want) != cudaSuccess) return false;
  ln.stage_bytes = want;
  return true;
}

void finish_ticket(tabi_server *s, uint64_t id, int32_t status, int32_t k) {
  Ticket &t = s->tickets[id];
  t.status = status;
  t.k = k;
  t.t_done = now_ns() - s->t0;
  t.done = true;
}

// Hand a finished lane's results to its requests (lock held).
void finish_lane(tabi_server *s, Lane &ln) {
  const int R = (int)ln.ids.size();
  batch_finish(ln.ctx, ln.reqs.data(), R, ln.fl, nullptr);
  if (ln.fl.checked) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ln.ctx->cev[0], ln.ctx->cev[1]) == cudaSuccess)
      s->stats.check_ns += (int64_t)(ms * 1e6f);
  }
  for (int i = 0; i < R; ++i) {
    const tabi_request &r = ln.reqs[i];
    Ticket &t = s->tickets[ln.ids[i]];
    if (r.status == TABI_OK)
      memcpy(t.req.out, r.out, sizeof(tabi_placement) * (size_t)r.n_charts);
    if (r.status == TABI_OK && ln.fl.checked) {
      batch_quality(ln.ctx, ln.fl, i, t.quality);
      if (t.quality[0] >= 0) {
        s->stats.checked += 1;
        s->stats.check_violations += (t.quality[0] | t.quality[1] | t.quality[2]) != 0;
      }
    }
    finish_ticket(s, ln.ids[i], r.status, r.scale_k);
  }
  s->stats.completed += R;
  ln.ids.clear();
  ln.reqs.clear();
  ln.busy = false;
  ln.finished.store(0);
  s->done.notify_all();
}

// Form and launch a batch on an idle lane from the head of the queue (lock
// held).  Returns false if the queue is empty.
bool launch_lane(tabi_server *s, Lane &ln) {
  if (s->queue.empty()) return false;
  size_t used = 0, stage = 0;
  ln.ids.clear();
  while (!s->queue.empty() && (int)ln.ids.size() < s->cfg.max_batch) {
    const Ticket &t = s->tickets[s->queue.front()];
    if (!ln.ids.empty() && used + t.est > ln.budget) break;  // arrival order: the head waits
    used += t.est;
    stage += align16(4 * ((size_t)t.req.n_charts + 1)) + align16(8 * (size_t)t.req.n_verts) +
             align16(sizeof(tabi_placement) * (size_t)t.req.n_charts);
    ln.ids.push_back(s->queue.front());
    s->queue.pop_front();
  }
  const int64_t t_start = now_ns() - s->t0;
  if (!ensure_stage(ln, stage)) {
    for (uint64_t id : ln.ids) finish_ticket(s, id, TABI_ERR_CUDA, 0);
    ln.ids.clear();
    s->done.notify_all();
    return true;
  }
  // inputs into pinned staging; the batch reads them from there and writes
  // its placements back there
  ln.reqs.assign(ln.ids.size(), tabi_request{});
  char *p = ln.stage;
  for (size_t i = 0; i < ln.ids.size(); ++i) {
    Ticket &t = s->tickets[ln.ids[i]];
    t.t_start = t_start;
    const tabi_request &r = t.req;
    tabi_request &q = ln.reqs[i];
    q = r;
    memcpy(p, r.offsets, 4 * ((size_t)r.n_charts + 1));
    q.offsets = reinterpret_cast<const uint32_t *>(p);
    p += align16(4 * ((size_t)r.n_charts + 1));
    memcpy(p, r.verts, 8 * (size_t)r.n_verts);
    q.verts = reinterpret_cast<const int32_t *>(p);
    p += align16(8 * (size_t)r.n_verts);
    q.out = reinterpret_cast<tabi_placement *>(p);
    p += align16(sizeof(tabi_placement) * (size_t)r.n_charts);
  }
  tabi_status st = batch_launch(ln.ctx, &s->params, ln.reqs.data(), (int)ln.reqs.size(), ln.st, true, nullptr,
                                nullptr, ln.fl, s->cfg.check != 0);
  if (st == TABI_OK) {
    auto *arg = new std::pair<tabi_server *, Lane *>(s, &ln);
    if (cudaLaunchHostFunc(ln.st, lane_finished, arg) != cudaSuccess) {
      delete arg;
      st = TABI_ERR_CUDA;
    }
  }
  if (st != TABI_OK) {
    // nothing in flight to wait for: the whole batch gets the error
    cudaStreamSynchronize(ln.st);
    for (uint64_t id : ln.ids) finish_ticket(s, id, st, 0);
    ln.ids.clear();
    ln.reqs.clear();
    s->done.notify_all();
    return true;
  }
  ln.busy = true;
  s->stats.batches += 1;
  s->stats.launched += (int64_t)ln.ids.size();
  s->stats.max_batch = std::max<int64_t>(s->stats.max_batch, (int64_t)ln.ids.size());
  return true;
}

void worker_main(tabi_server *s) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  int64_t stop_deadline = 0;
  while (true) {
    bool any_busy = false;
    for (auto &ln : s->lanes) {
      if (ln->busy && ln->finished.load()) finish_lane(s, *ln);
      any_busy |= ln->busy;
    }
    if (!s->stop)
      for (auto &ln : s->lanes)
        if (!ln->busy && launch_lane(s, *ln)) any_busy |= ln->busy;
    if (s->stop) {
      // queued requests are not started; in-flight batches get a bounded time
      while (!s->queue.empty()) {
        finish_ticket(s, s->queue.front(), TABI_ERR_BUSY, 0);
        s->queue.pop_front();
      }
      s->done.notify_all();
      if (!any_busy) break;
      if (!stop_deadline) stop_deadline = now_ns() + 60LL * 1000 * 1000 * 1000;
      if (now_ns() > stop_deadline) {
        for (auto &ln : s->lanes)
          if (ln->busy)
            for (uint64_t id : ln->ids) finish_ticket(s, id, TABI_ERR_TIMEOUT, 0);
        s->done.notify_all();
        break;
      }
    }
    // a lost wake-up costs at most the timeout
    s->wake.wait_for(lk, std::chrono::microseconds(any_busy ? 200 : 2000));
  }
}

tabi_status take_result(tabi_server *s, uint64_t ticket, tabi_result *res) {
  auto it = s->tickets.find(ticket);
  const Ticket &t = it->second;
  if (res) {
    res->status = t.status;
    res->scale_k = t.k;
    res->t_submit_ns = t.t_submit;
    res->t_start_ns = t.t_start;
    res->t_done_ns = t.t_done;
    res->overlap_texels = t.quality[0];
    res->gutter_texels = t.quality[1];
    res->outside_texels = t.quality[2];
  }
  s->tickets.erase(it);
  return TABI_OK;
}

}  // namespace

extern "C" {

void tabi_server_config_default(tabi_server_config *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->device = 0;
  c->arena_bytes = (size_t)8 << 30;
  c->lanes = 4;
  c->max_batch = 64;
  c->check = 1;
  tabi_params_default(&c->params);
  c->params.scale_fanout = 8;
}

tabi_status tabi_server_create(tabi_server **out, const tabi_server_config *cfg) {
  if (!out || !cfg) return TABI_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->lanes < 1 || cfg->lanes > 64 || cfg->max_batch < 1 || cfg->max_batch > TABI_MAX_BATCH ||
      cfg->arena_bytes < ((size_t)cfg->lanes << 24) || cfg->params.scale_fanout < 1 ||
      cfg->params.scale_fanout > kScales || cfg->params.version != TABI_PARAMS_VERSION || cfg->check < 0 ||
      cfg->check > 1)
    return TABI_ERR_INVALID_ARG;
  if (cudaSetDevice(cfg->device) != cudaSuccess) return TABI_ERR_INVALID_ARG;
  auto *s = new tabi_server();
  s->cfg = *cfg;
  s->params = cfg->params;
  s->t0 = now_ns();
  const size_t per = (cfg->arena_bytes / (size_t)cfg->lanes) & ~(size_t)255;
  bool ok = cudaMalloc(&s->arena, per * (size_t)cfg->lanes) == cudaSuccess;
  for (int i = 0; ok && i < cfg->lanes; ++i) {
    auto ln = std::make_unique<Lane>();
    ln->budget = per;
    ok = tabi_ctx_create(&ln->ctx, cfg->device, s->arena + per * (size_t)i, per) == TABI_OK &&
         cudaStreamCreateWithFlags(&ln->st, cudaStreamNonBlocking) == cudaSuccess && ensure_stage(*ln, 0);
    s->lanes.push_back(std::move(ln));
  }
  if (!ok) {
    for (auto &ln : s->lanes) {
      if (ln->ctx) tabi_ctx_destroy(ln->ctx);
      if (ln->st) cudaStreamDestroy(ln->st);
      if (ln->stage) cudaFreeHost(ln->stage);
    }
    if (s->arena) cudaFree(s->arena);
    delete s;
    return TABI_ERR_CUDA;
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return TABI_OK;
}

void tabi_server_destroy(tabi_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
  }
  s->wake.notify_one();
  s->worker.join();
  cudaSetDevice(s->cfg.device);
  // The worker gave in-flight batches up to 60 s; whatever still runs gets
  // the rest of a 60 s budget here, polled, never an unbounded wait.  A lane
  // whose stream is still busy after that keeps its context, staging and
  // the shared arena allocated (freeing memory a running kernel may still
  // touch is never safe); everything else is released.
  const int64_t deadline = now_ns() + 60LL * 1000 * 1000 * 1000;
  bool leak = false;
  for (auto &ln : s->lanes) {
    cudaError_t q = cudaStreamQuery(ln->st);
    while (q == cudaErrorNotReady && now_ns() < deadline) {
      std::this_thread::sleep_for(std::chrono::microseconds(500));
      q = cudaStreamQuery(ln->st);
    }
    if (q == cudaErrorNotReady) {
      leak = true;
      continue;
    }
    tabi_ctx_destroy(ln->ctx);
    cudaStreamDestroy(ln->st);
    if (ln->stage) cudaFreeHost(ln->stage);
  }
  if (!leak) cudaFree(s->arena);
  delete s;
}

tabi_status tabi_submit(tabi_server *s, const tabi_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return TABI_ERR_INVALID_ARG;
  *ticket = 0;
  Ticket t;
  t.req = *req;
  t.t_submit = now_ns() - s->t0;
  bool reject = false;
  int32_t why = TABI_ERR_INVALID_ARG;
  if (req->n_charts < 1 || req->n_charts > TABI_MAX_CHARTS || req->n_verts < 3 || !req->offsets ||
      !req->verts || !req->out || !offsets_valid(*req)) {
    reject = true;
  } else {
    t.est = request_bytes(*req, s->params.scale_fanout, s->params.gutter);
    if (t.est > s->lanes[0]->budget) {
      reject = true;
      why = TABI_ERR_OOM;
    }
  }
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stop) return TABI_ERR_BUSY;
  const uint64_t id = s->next_id++;
  s->tickets.emplace(id, t);
  s->stats.submitted += 1;
  *ticket = id;
  if (reject) {
    finish_ticket(s, id, why, 0);
    s->done.notify_all();
    return TABI_OK;
  }
  s->queue.push_back(id);
  s->wake.notify_one();
  return TABI_OK;
}

tabi_status tabi_poll(tabi_server *s, uint64_t ticket, tabi_result *res) {
  if (!s) return TABI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return TABI_ERR_INVALID_ARG;
  if (!it->second.done) return TABI_PENDING;
  return take_result(s, ticket, res);
}

tabi_status tabi_wait(tabi_server *s, uint64_t ticket, int32_t timeout_ms, tabi_result *res) {
  if (!s || timeout_ms < 0) return TABI_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->tickets.find(ticket) == s->tickets.end()) return TABI_ERR_INVALID_ARG;
  const bool ok = s->done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
    auto it = s->tickets.find(ticket);
    return it == s->tickets.end() || it->second.done;
  });
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return TABI_ERR_INVALID_ARG;  // taken by another waiter
  if (!ok) return TABI_ERR_TIMEOUT;
  return take_result(s, ticket, res);
}

tabi_status tabi_server_get_stats(tabi_server *s, tabi_server_stats *out) {
  if (!s || !out) return TABI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->stats;
  out->queued = (int64_t)s->queue.size();
  int64_t busy = 0;
  for (auto &ln : s->lanes) busy += ln->busy;
  out->busy_lanes = busy;
  return TABI_OK;
}

}  // extern "C"
