// Continuous batching across streams.
//
// A server runs pushes of many streams concurrently on one GPU: `slots` worker
// threads, each of which takes the oldest queued request whose stream is not
// already running and whose memory fits, and runs push_microbatch on that
// stream's own CUDA stream — so micro-batches of different streams overlap on
// the device while each stream's batches still run one at a time, in the
// order they were submitted.  Admission by memory: a request may start only if
// the device bytes of every stream the server has seen, plus what the running
// requests may still allocate, plus what this push may allocate, stay within
// memory_budget_bytes; otherwise it waits for a running request to finish
// (a request that alone exceeds the budget is failed with LMS_ENOMEM rather
// than waiting forever).  Requests arriving while others run are admitted as
// soon as a slot and memory free up.  The paper has no counterpart: it runs
// one query's micro-batches one after another.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/lmstream.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket;
  lms_stream* s;
  lms_batch b;
  uint64_t reserve;  // bytes the push may allocate
};

struct Done {
  lms_status status;
  double start_ms, end_ms;  // since the server started
  int slot;
};

}  // namespace

struct lms_server {
  lms_server_config cfg{};
  lms_server_ops ops{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req> queue;
  std::unordered_set<lms_stream*> running;
  std::unordered_map<lms_stream*, uint64_t> held;  // last known device bytes per stream
  std::map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  uint64_t reserved = 0;  // sum of running requests' reserves
  bool stop = false;
  std::vector<std::thread> workers;
  Clock::time_point t0 = Clock::now();
  lms_server_stats st{};
  int active = 0;
};

namespace {

uint64_t held_total(const lms_server* sv) {
  uint64_t t = 0;
  for (const auto& kv : sv->held) t += kv.second;
  return t;
}

void worker(lms_server* sv, int slot) {
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    // the oldest request whose stream is idle (and has no older request
    // queued) and whose memory fits
    auto pick = sv->queue.end(), blocked = sv->queue.end();
    const uint64_t budget = sv->cfg.memory_budget_bytes;
    for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it) {
      if (sv->running.count(it->s)) continue;
      bool older = false;
      for (auto jt = sv->queue.begin(); jt != it && !older; ++jt) older = jt->s == it->s;
      if (older) continue;
      if (budget && held_total(sv) + sv->reserved + it->reserve > budget) {
        if (blocked == sv->queue.end()) blocked = it;
        continue;
      }
      pick = it;
      break;
    }
    if (pick == sv->queue.end()) {
      if (blocked != sv->queue.end()) {
        if (sv->running.empty()) {  // nothing running can free memory: it never fits
          sv->done[blocked->ticket] = Done{LMS_ENOMEM, 0.0, 0.0, slot};
          sv->queue.erase(blocked);
          sv->cv_done.notify_all();
          continue;
        }
        ++sv->st.memory_waits;
      }
      if (sv->stop && sv->queue.empty()) return;
      sv->cv_work.wait(lk);
      continue;
    }
    Req r = *pick;
    sv->queue.erase(pick);
    sv->running.insert(r.s);
    sv->reserved += r.reserve;
    ++sv->active;
    sv->st.max_concurrent = std::max<int64_t>(sv->st.max_concurrent, sv->active);
    const double start = std::chrono::duration<double, std::milli>(Clock::now() - sv->t0).count();
    lk.unlock();
    const lms_status status = sv->ops.push(sv->ops.ctx, r.s, &r.b);
    uint64_t now_bytes = 0;
    sv->ops.device_bytes(sv->ops.ctx, r.s, &now_bytes);
    lk.lock();
    const double end = std::chrono::duration<double, std::milli>(Clock::now() - sv->t0).count();
    --sv->active;
    sv->reserved -= r.reserve;
    sv->running.erase(r.s);
    sv->held[r.s] = now_bytes;
    sv->st.completed += 1;
    sv->st.busy_ms += end - start;
    sv->st.peak_bytes = std::max<uint64_t>(sv->st.peak_bytes, held_total(sv) + sv->reserved);
    sv->done[r.ticket] = Done{status, start, end, slot};
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

namespace {
lms_status engine_push(void*, lms_stream* s, const lms_batch* b) { return push_microbatch(s, b); }
lms_status engine_push_bytes(void*, lms_stream* s, int64_t n, int32_t host, uint64_t* out) {
  return lms_stream_push_bytes(s, n, host, out);
}
lms_status engine_device_bytes(void*, lms_stream* s, uint64_t* out) {
  return lms_stream_device_bytes(s, out);
}
}  // namespace

lms_status lms_server_create(const lms_server_config* cfg, lms_server** out) {
  const lms_server_ops ops{nullptr, engine_push, engine_push_bytes, engine_device_bytes};
  return lms_server_create_ops(cfg, &ops, out);
}

lms_status lms_server_create_ops(const lms_server_config* cfg, const lms_server_ops* ops,
                                 lms_server** out) {
  if (!cfg || !out || !ops || !ops->push || !ops->push_bytes || !ops->device_bytes ||
      cfg->slots < 1 || cfg->slots > 64)
    return LMS_EINVAL;
  lms_server* sv = new lms_server();
  sv->cfg = *cfg;
  sv->ops = *ops;
  for (int i = 0; i < cfg->slots; ++i) sv->workers.emplace_back(worker, sv, i);
  *out = sv;
  return LMS_OK;
}

lms_status lms_server_submit(lms_server* sv, lms_stream* s, const lms_batch* b,
                             uint64_t* ticket) {
  if (!sv || !s || !b || !ticket) return LMS_EINVAL;
  uint64_t reserve = 0;
  lms_status r =
      sv->ops.push_bytes(sv->ops.ctx, s, b->n_rows, b->memory == LMS_MEM_HOST ? 1 : 0, &reserve);
  if (r != LMS_OK) return r;
  uint64_t held = 0;
  sv->ops.device_bytes(sv->ops.ctx, s, &held);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return LMS_ECLOSED;
  if (!sv->held.count(s)) sv->held[s] = held;
  const uint64_t t = sv->next_ticket++;
  sv->queue.push_back(Req{t, s, *b, reserve});
  sv->st.submitted += 1;
  *ticket = t;
  sv->cv_work.notify_all();
  return LMS_OK;
}

lms_status lms_server_wait(lms_server* sv, uint64_t ticket, int32_t timeout_ms,
                           lms_status* result, double* start_ms, double* end_ms) {
  if (!sv || !result) return LMS_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  if (ticket == 0 || ticket >= sv->next_ticket) return LMS_EINVAL;
  auto ready = [&] { return sv->done.count(ticket) != 0; };
  if (timeout_ms < 0) {
    sv->cv_done.wait(lk, ready);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return LMS_ETIMEDOUT;
  }
  const Done d = sv->done[ticket];
  sv->done.erase(ticket);
  *result = d.status;
  if (start_ms) *start_ms = d.start_ms;
  if (end_ms) *end_ms = d.end_ms;
  return LMS_OK;
}

lms_status lms_server_forget(lms_server* sv, lms_stream* s) {
  if (!sv || !s) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->running.count(s)) return LMS_EAGAIN;
  for (const Req& r : sv->queue)
    if (r.s == s) return LMS_EAGAIN;
  sv->held.erase(s);
  sv->cv_work.notify_all();
  return LMS_OK;
}

lms_status lms_server_get_stats(lms_server* sv, lms_server_stats* out) {
  if (!sv || !out) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->st;
  out->queued = (int64_t)sv->queue.size();
  out->held_bytes = held_total(sv);
  return LMS_OK;
}

lms_status lms_server_destroy(lms_server* sv) {
  if (!sv) return LMS_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv_work.notify_all();
  }
  for (std::thread& t : sv->workers) t.join();
  delete sv;
  return LMS_OK;
}

}  // extern "C"
