// The serving loop: dynamic micro-batching over an arrival process on a
// virtual clock whose processing steps are real (the backend runs each
// admitted micro-batch and reports how long it took).
//
// Alg. 1 (ConstructMicroBatch) decides when the buffered datasets form a
// micro-batch; here a dataset is one poll tick of arrivals, as in Section
// III-C where new data is collected every polling period.  With the latency
// bound of the serving setting as its target, the analytic policy is Alg. 1
// with Eq. 5; the learned policy is Alg. 1 with a predictor of the processing
// time installed in place of Eq. 5's bytes / AvgThPut term.  Two fixed
// policies (a fixed number of events; a fixed trigger period) are the
// baselines.  Admission by memory (not in the paper) caps a batch at what the
// backend says it can hold; datasets that do not fit stay buffered and are
// offered again.
//
// Per-event latency = completion time of the batch - arrival time of the
// event (Eq. 4 applied to each event).  Event j of a tick [t0, t0 + w) with n
// events arrives at t0 + (j + 0.5) w / n, so each processed piece of a tick
// contributes latencies in arithmetic progression; quantiles are the exact
// order statistics of that multiset.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <limits>
#include <vector>

#include "../../include/lmstream.h"

namespace {

struct Piece {
  double t0, w;
  int64_t n_total, jb, je, first;
  bool fed;  // already offered to Alg. 1
};

// Latencies A - (j + 0.5) d for j in [jb, je).
struct Seg {
  double A, d;
  int64_t jb, je;
};

int64_t count_le(const Seg& s, double v) {
  // A - (j + 0.5) d <= v  <=>  j >= (A - v) / d - 0.5
  const double x = (s.A - v) / s.d - 0.5;
  if (x <= (double)s.jb) return s.je - s.jb;
  if (x > (double)(s.je - 1)) return 0;
  const int64_t jmin = (int64_t)std::ceil(x);
  return s.je - std::min(s.je, std::max(s.jb, jmin));
}

double seg_min(const Seg& s) { return s.A - ((double)(s.je - 1) + 0.5) * s.d; }
double seg_max(const Seg& s) { return s.A - ((double)s.jb + 0.5) * s.d; }

// k-th smallest latency (1-based) over all segments, by bisection on the value.
double kth(const std::vector<Seg>& segs, int64_t k) {
  double lo = std::numeric_limits<double>::infinity(), hi = -lo;
  for (const Seg& s : segs) {
    lo = std::min(lo, seg_min(s));
    hi = std::max(hi, seg_max(s));
  }
  if (!(lo <= hi)) return 0.0;
  auto cnt = [&](double v) {
    int64_t c = 0;
    for (const Seg& s : segs) c += count_le(s, v);
    return c;
  };
  if (cnt(lo) >= k) return lo;
  for (int it = 0; it < 200 && hi > lo; ++it) {
    const double mid = lo + 0.5 * (hi - lo);
    if (mid <= lo || mid >= hi) break;
    if (cnt(mid) >= k) hi = mid;
    else lo = mid;
  }
  return hi;
}

}  // namespace

extern "C" lms_status lms_serve_run(const lms_serve_config* cfg, const int64_t* tick_counts,
                                    int64_t n_ticks, const lms_serve_backend* be,
                                    lms_proc_predictor pred, void* pred_ctx,
                                    lms_batch_observer observe, lms_serve_result* out,
                                    lms_serve_batch* log, size_t log_cap, size_t* n_log) {
  if (!cfg || !be || !be->process || !out || n_ticks < 0 || (n_ticks > 0 && !tick_counts))
    return LMS_EINVAL;
  const int policy = cfg->policy;
  if (policy < LMS_POLICY_FIXED_SIZE || policy > LMS_POLICY_LEARNED) return LMS_EINVAL;
  if (!(cfg->poll_ms > 0) || !(cfg->latency_bound_ms > 0) || cfg->bytes_per_event < 0)
    return LMS_EINVAL;
  if (policy == LMS_POLICY_FIXED_SIZE && cfg->fixed_rows <= 0) return LMS_EINVAL;
  if (policy == LMS_POLICY_FIXED_TRIGGER && !(cfg->trigger_ms > 0)) return LMS_EINVAL;
  if (policy == LMS_POLICY_LEARNED && !pred) return LMS_EINVAL;
  const double qhi = cfg->quantile_hi > 0 ? cfg->quantile_hi : 0.99;
  if (qhi > 1.0) return LMS_EINVAL;
  int64_t offered = 0;
  for (int64_t t = 0; t < n_ticks; ++t) {
    if (tick_counts[t] < 0) return LMS_EINVAL;
    offered += tick_counts[t];
  }
  const double poll = cfg->poll_ms, bound = cfg->latency_bound_ms, bpe = cfg->bytes_per_event;

  lms_admission* adm = nullptr;
  if (policy == LMS_POLICY_ANALYTIC || policy == LMS_POLICY_LEARNED) {
    adm = lms_admission_create(bound, cfg->admit_rule, poll);
    if (!adm) return LMS_EINVAL;
    if (policy == LMS_POLICY_LEARNED) lms_admission_set_predictor(adm, pred, pred_ctx);
  }

  std::deque<Piece> pending;
  int64_t pend_events = 0, tick = 0, first = 0;
  double now = 0.0, next_fire = cfg->trigger_ms;
  std::vector<Seg> segs;
  int64_t processed = 0, batches = 0, over = 0, max_backlog = 0;
  double busy = 0.0, end = 0.0, decide_total = 0.0, observe_total = 0.0;
  // p_hi <= bound  <=>  at most offered - ceil(qhi * offered) events exceed it
  const int64_t k_hi_total = offered > 0 ? (int64_t)std::ceil(qhi * (double)offered) : 0;
  const int64_t allowed_over = offered - k_hi_total;
  size_t nl = 0;
  bool completed = true;
  lms_status status = LMS_OK;
  std::vector<double> arr, bytes;
  std::vector<lms_serve_chunk> chunks;
  double arrive_total = 0.0;

  for (;;) {
    while (tick < n_ticks && (double)(tick + 1) * poll <= now + 1e-9) {
      const int64_t c = tick_counts[tick];
      if (c > 0) {
        pending.push_back({(double)tick * poll, poll, c, 0, c, first, false});
        if (be->arrive) {
          const auto a0 = std::chrono::steady_clock::now();
          const lms_serve_chunk tc{(double)tick * poll, poll, c, 0, c, first};
          const int32_t ar = be->arrive(be->ctx, &tc);
          arrive_total += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a0).count();
          if (ar < 0) {
            status = LMS_EDEVICE;
            break;
          }
        }
        pend_events += c;
        first += c;
      }
      ++tick;
    }
    if (status != LMS_OK) break;
    const bool all_arrived = tick == n_ticks;
    max_backlog = std::max(max_backlog, pend_events);
    if (pending.empty()) {
      if (all_arrived) break;
      now = (double)(tick + 1) * poll;
      continue;
    }
    const auto d0 = std::chrono::steady_clock::now();
    int64_t take = 0;
    bool via_alg1 = false, forced = false;
    double est = 0.0;
    if (policy == LMS_POLICY_FIXED_SIZE) {
      if (pend_events >= cfg->fixed_rows) take = cfg->fixed_rows;
      else if (all_arrived) take = pend_events, forced = true;
    } else if (policy == LMS_POLICY_FIXED_TRIGGER) {
      if (now >= next_fire - 1e-9 || all_arrived) {
        forced = now < next_fire - 1e-9;
        take = pend_events;
        next_fire = (std::floor(now / cfg->trigger_ms + 1e-9) + 1.0) * cfg->trigger_ms;
      }
    } else {
      arr.clear();
      bytes.clear();
      for (Piece& p : pending) {
        if (p.fed) continue;
        arr.push_back(p.t0 + ((double)p.jb + 0.5) * p.w / (double)p.n_total);
        bytes.push_back((double)(p.je - p.jb) * bpe);
        p.fed = true;
      }
      int32_t nadm = 0;
      const int32_t r = lms_admission_poll(adm, now, arr.data(), bytes.data(), (int32_t)arr.size(),
                                           &est, &nadm);
      if (r < 0) {
        status = r;
        break;
      }
      if (r == 1) {
        take = pend_events;
        via_alg1 = true;
      } else if (all_arrived) {
        take = pend_events;
        forced = true;
      }
    }
    if (take > 0 && be->admissible_rows) {
      const int64_t cap = be->admissible_rows(be->ctx);
      if (cap == 0) {
        status = LMS_ENOMEM;
        break;
      }
      if (cap > 0 && take > cap) {
        take = cap;
        forced = true;
      }
    }
    double decide_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - d0).count();
    decide_total += decide_ms;
    if (cfg->add_decide_time) now += decide_ms;
    if (take == 0) {
      double nxt = tick < n_ticks ? (double)(tick + 1) * poll : now + poll;
      if (policy == LMS_POLICY_FIXED_TRIGGER && next_fire > now) nxt = std::min(nxt, next_fire);
      now = std::max(now, nxt);
      continue;
    }
    // cut the batch from the head of the queue, splitting one tick if needed
    chunks.clear();
    int64_t left = take, earliest_j = -1;
    double earliest = 0.0;
    bool split = false;
    while (left > 0) {
      Piece& p = pending.front();
      const int64_t m = p.je - p.jb;
      const int64_t use = std::min(m, left);
      chunks.push_back({p.t0, p.w, p.n_total, p.jb, p.jb + use, p.first});
      if (earliest_j < 0) {
        earliest_j = p.jb;
        earliest = p.t0 + ((double)p.jb + 0.5) * p.w / (double)p.n_total;
      }
      left -= use;
      if (use == m) {
        pending.pop_front();
      } else {
        p.jb += use;
        p.fed = false;  // the rest is offered again
        split = true;
      }
    }
    pend_events -= take;
    if (via_alg1 && !pending.empty()) {
      // memory admission kept only a prefix of what Alg. 1 admitted: the rest
      // is offered again at the next poll
      for (Piece& p : pending) p.fed = false;
      const lms_serve_chunk& lc = chunks.back();
      const double last_b = split ? (double)(lc.j_end - lc.j_begin) * bpe : 0.0;
      lms_admission_truncate(adm, (int32_t)chunks.size(), last_b);
    }
    lms_serve_batch rec{};
    rec.admit_ms = now;
    rec.est_ms = est;
    rec.decide_ms = decide_ms;
    rec.n_events = take;
    rec.n_chunks = (int32_t)chunks.size();
    rec.forced = forced ? 1 : 0;
    const double proc = be->process(be->ctx, chunks.data(), (int32_t)chunks.size(), take, &rec);
    if (!(proc >= 0)) {
      status = LMS_EDEVICE;
      break;
    }
    if (via_alg1) lms_admission_complete(adm, proc);
    now += proc;
    busy += proc;
    end = now;
    rec.proc_ms = proc;
    rec.maxlat_ms = now - earliest;
    for (const lms_serve_chunk& c : chunks) {
      Seg s{now - c.t0_ms, c.width_ms / (double)c.n_total, c.j_begin, c.j_end};
      over += (s.je - s.jb) - count_le(s, bound);
      segs.push_back(s);
    }
    processed += take;
    ++batches;
    if (log && nl < log_cap) log[nl] = rec;
    ++nl;
    if (observe) {
      const double ob = observe(pred_ctx, &rec);
      observe_total += ob;
      if (cfg->add_decide_time && ob > 0) now += ob;
    }
    if (cfg->stop_when_missed && over > allowed_over) {
      completed = false;
      break;
    }
  }
  if (adm) lms_admission_destroy(adm);
  if (status != LMS_OK) return status;
  if (processed < offered) completed = false;

  lms_serve_result r{};
  r.offered_events = offered;
  r.processed_events = processed;
  r.batches = batches;
  r.completed = completed ? 1 : 0;
  r.arrival_span_ms = (double)n_ticks * poll;
  r.end_ms = end;
  r.busy_ms = busy;
  r.max_backlog_events = max_backlog;
  r.decide_ms = decide_total;
  r.observe_ms = observe_total;
  r.arrive_ms = arrive_total;
  if (processed > 0) {
    r.p50_ms = kth(segs, (int64_t)std::ceil(0.5 * (double)processed));
    r.p_hi_ms = kth(segs, std::max<int64_t>(1, (int64_t)std::ceil(qhi * (double)processed)));
    double sum = 0.0, mx = -std::numeric_limits<double>::infinity();
    for (const Seg& s : segs) {
      const double n = (double)(s.je - s.jb);
      const double sj = 0.5 * (double)(s.jb + s.je - 1) * n;  // sum of j
      sum += n * s.A - s.d * (sj + 0.5 * n);
      mx = std::max(mx, seg_max(s));
    }
    r.mean_ms = sum / (double)processed;
    r.max_ms = mx;
  }
  r.met_bound = (completed && processed > 0 && r.p_hi_ms <= bound) ? 1 : 0;
  r.events_per_s = r.arrival_span_ms > 0 ? (double)processed / (r.arrival_span_ms * 1e-3) : 0.0;
  *out = r;
  if (n_log) *n_log = nl;
  return LMS_OK;
}
