// TEST INFRASTRUCTURE ONLY — the CPU oracle for windowed group-by aggregation.
//
// This file is the plain, slow, obviously-correct definition of what the
// engine's data-parallel hot path computes for one micro-batch stream query
// (filter -> project -> window assignment -> group-by aggregate -> emit closed
// windows).  It is used only by the tests, by `__graft_entry__.smoke()` and by
// the CPU-baseline leg of `bench.py`; the product path never links or calls it.
// It shares no code, header or constant table with the CUDA engine.
//
// Paper: LMStream (micro-batch stream processing meets GPU).  The paper runs
// its queries inside Spark and does not define window or aggregate semantics
// itself (Table III lists the queries: windows "[range R slide S]", AVG/SUM,
// GROUPBY, WHERE).  The semantics written out here are the textbook event-time
// ones, in this order, for every event in arrival order:
//   1. filter: `column OP constant`; integer columns compare as int64, the
//      float32 value column compares as double (IEEE comparison).
//   2. windows: with K = size/slide, the event at time ts belongs to the K
//      windows [s, s+size) with s = (floor(ts/slide) - k) * slide, k = 0..K-1
//      (true floor, also for negative ts).  Tumbling windows are K = 1
//      (SlideTime = 0 in Table I of the paper means "tumbling").
//   3. lateness: a window whose end s+size is <= the watermark of the previous
//      micro-batch has already been emitted; the event is not added to it.
//      An event none of whose windows is still open counts as a late row.
//   4. aggregate per (window start, key): count += 1, sum += value (int64 for
//      int32 values, sequential double for float32 values), min/max by value;
//      float min/max follow IEEE-754 totalOrder (-0.0 < +0.0).
//   5. after the micro-batch: watermark = max(watermark, max ts of all rows of
//      the batch, filtered or not, - allowed_lateness); a caller may raise the
//      batch's max ts to a floor (oracle_push_floor: when the stream holds one
//      key shard of a micro-batch, the max is the whole batch's).  Every group whose
//      window end is <= watermark is emitted, in (window start, key) order, with
//      avg = (double)sum / count, and deleted.  End of stream emits everything.
//   6. post-aggregation (Table III: LR2S's HAVING, CM1's ORDER BY, the
//      multi-column GROUP BY of LR2S), per query and optional:
//      * GROUP BY a subset of the key's packed fields: the group key is
//        key & group_mask (the bits of the selected fields);
//      * HAVING agg OP c: an emitted row is kept iff (double)agg OP c (the
//        same IEEE comparison as the filter), agg one of count, sum, min,
//        max, avg;
//      * ORDER BY agg: the rows of each window come out sorted by the
//        aggregate's value (ascending, or descending), equal values in key
//        order (a stable sort of the key-ordered rows).
// Parity pins for this file live in tests/test_oracle_pins.py (brute force per
// window on tiny streams, invariants, special cases that reduce to numpy
// group-by routines, hand-worked fixtures).

#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <algorithm>
#include <map>
#include <utility>
#include <vector>

// One emitted row.  The layout is the oracle's own (the Python side reads it
// through a numpy structured dtype declared next to the loader).
struct OracleRow {
  int64_t window_start;
  int64_t window_end;
  int64_t count;
  int64_t sum_i;
  double sum_f;
  double avg;
  int32_t min_i;
  int32_t max_i;
  float min_f;
  float max_f;
  uint32_t key;
  uint32_t pad;
};

namespace {

enum { COL_TS = 0, COL_KEY = 1, COL_VALUE = 2, COL_TYPE = 3 };
enum { OP_NONE = 0, OP_EQ = 1, OP_NE = 2, OP_LT = 3, OP_LE = 4, OP_GT = 5, OP_GE = 6 };

struct OracleQuery {
  int filter_col = COL_TS;
  int filter_op = OP_NONE;
  int64_t filter_i = 0;
  double filter_f = 0.0;
  int64_t size = 1;
  int64_t slide = 1;
  uint32_t group_mask = 0xffffffffu;
  int having_agg = 0, having_op = OP_NONE;
  double having_value = 0.0;
  int order_agg = 0, order_desc = 0;
  // Per (window start, key) group.
  struct Agg {
    int64_t count = 0;
    int64_t sum_i = 0;
    double sum_f = 0.0;
    int32_t min_i = 0, max_i = 0;
    float min_f = 0.0f, max_f = 0.0f;
  };
  std::map<std::pair<int64_t, uint32_t>, Agg> groups;
  std::vector<OracleRow> out;
  int64_t late_rows = 0;
};

}  // namespace

namespace {

// Mathematical floor of a / b for b > 0 (C++ division truncates toward zero).
int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) q -= 1;
  return q;
}

// IEEE-754 totalOrder "a < b" for non-NaN floats: a negative sign orders
// first (so -0.0 < +0.0); equal signs order by magnitude, reversed when
// negative.
bool total_less(float a, float b) {
  uint32_t ba, bb;
  std::memcpy(&ba, &a, 4);
  std::memcpy(&bb, &b, 4);
  bool na = (ba >> 31) != 0, nb = (bb >> 31) != 0;
  if (na != nb) return na;
  uint32_t ma = ba & 0x7fffffffu, mb = bb & 0x7fffffffu;
  return na ? (ma > mb) : (ma < mb);
}

bool compare_i(int op, int64_t x, int64_t c) {
  switch (op) {
    case OP_EQ: return x == c;
    case OP_NE: return x != c;
    case OP_LT: return x < c;
    case OP_LE: return x <= c;
    case OP_GT: return x > c;
    case OP_GE: return x >= c;
    default: return true;
  }
}

bool compare_f(int op, double x, double c) {
  switch (op) {
    case OP_EQ: return x == c;
    case OP_NE: return x != c;
    case OP_LT: return x < c;
    case OP_LE: return x <= c;
    case OP_GT: return x > c;
    case OP_GE: return x >= c;
    default: return true;
  }
}

struct Oracle {
  int value_is_float = 0;
  int64_t lateness = 0;
  bool have_wm = false;
  int64_t wm = 0;
  std::vector<OracleQuery> queries;
};

// The value of aggregate `agg` (1 count, 2 sum, 3 min, 4 max, 5 avg) of a row.
double agg_value(const Oracle& o, const OracleRow& r, int agg) {
  switch (agg) {
    case 1: return (double)r.count;
    case 2: return o.value_is_float ? r.sum_f : (double)r.sum_i;
    case 3: return o.value_is_float ? (double)r.min_f : (double)r.min_i;
    case 4: return o.value_is_float ? (double)r.max_f : (double)r.max_i;
    default: return r.avg;
  }
}

// Sorts the rows of one window, out[from ..], by the ORDER BY aggregate.
void order_window(const Oracle& o, const OracleQuery& q, std::vector<OracleRow>& out,
                  size_t from) {
  std::stable_sort(out.begin() + (long)from, out.end(),
                   [&](const OracleRow& x, const OracleRow& y) {
                     const double a = agg_value(o, x, q.order_agg), b = agg_value(o, y, q.order_agg);
                     return q.order_desc ? a > b : a < b;
                   });
}

void emit_closed(Oracle& o, OracleQuery& q, bool all) {
  size_t win_from = q.out.size();
  int64_t win_start = 0;
  bool have_win = false;
  auto it = q.groups.begin();
  while (it != q.groups.end()) {
    int64_t start = it->first.first;
    if (!all && !(start + q.size <= o.wm)) break;  // map order = (start, key)
    const OracleQuery::Agg& a = it->second;
    OracleRow r;
    std::memset(&r, 0, sizeof(r));
    r.window_start = start;
    r.window_end = start + q.size;
    r.key = it->first.second;
    r.count = a.count;
    if (o.value_is_float) {
      r.sum_f = a.sum_f;
      r.min_f = a.min_f;
      r.max_f = a.max_f;
      r.avg = a.sum_f / (double)a.count;
    } else {
      r.sum_i = a.sum_i;
      r.min_i = a.min_i;
      r.max_i = a.max_i;
      r.avg = (double)a.sum_i / (double)a.count;
    }
    it = q.groups.erase(it);
    if (q.having_agg && !compare_f(q.having_op, agg_value(o, r, q.having_agg), q.having_value))
      continue;
    if (q.order_agg && (!have_win || start != win_start)) {
      if (have_win) order_window(o, q, q.out, win_from);
      win_from = q.out.size();
      win_start = start;
      have_win = true;
    }
    q.out.push_back(r);
  }
  if (q.order_agg && have_win) order_window(o, q, q.out, win_from);
}

}  // namespace

extern "C" {

void* oracle_open(int value_is_float, int64_t allowed_lateness) {
  Oracle* o = new Oracle();
  o->value_is_float = value_is_float;
  o->lateness = allowed_lateness;
  return o;
}

void oracle_close(void* h) { delete static_cast<Oracle*>(h); }

int oracle_add_query(void* h, int filter_col, int filter_op, int64_t filter_i,
                     double filter_f, int64_t size, int64_t slide) {
  Oracle* o = static_cast<Oracle*>(h);
  if (slide <= 0 || size <= 0 || size % slide != 0) return -1;
  OracleQuery q;
  q.filter_col = filter_col;
  q.filter_op = filter_op;
  q.filter_i = filter_i;
  q.filter_f = filter_f;
  q.size = size;
  q.slide = slide;
  o->queries.push_back(std::move(q));
  return (int)o->queries.size() - 1;
}

// Feeds one micro-batch, event by event, then advances the watermark and emits.
// `value` points at int32 or float32 values; `type` may be NULL.  ts_floor is
// INT64_MIN, or a lower bound of the batch's max event time: the max over a
// micro-batch whose rows were split by key over several streams, each of
// which must advance the watermark the whole batch advances.
int oracle_push_floor(void* h, int64_t n, const int64_t* ts, const uint32_t* key,
                      const void* value, const uint8_t* type, int eos, int64_t ts_floor) {
  Oracle* o = static_cast<Oracle*>(h);
  const int32_t* vi = static_cast<const int32_t*>(value);
  const float* vf = static_cast<const float*>(value);
  for (OracleQuery& q : o->queries) {
    const int64_t K = q.size / q.slide;
    for (int64_t e = 0; e < n; ++e) {
      // 1. filter
      bool pass;
      switch (q.filter_col) {
        case COL_TS: pass = compare_i(q.filter_op, ts[e], q.filter_i); break;
        case COL_KEY: pass = compare_i(q.filter_op, (int64_t)key[e], q.filter_i); break;
        case COL_TYPE:
          pass = compare_i(q.filter_op, type ? (int64_t)type[e] : 0, q.filter_i);
          break;
        default:
          pass = o->value_is_float ? compare_f(q.filter_op, (double)vf[e], q.filter_f)
                                   : compare_i(q.filter_op, (int64_t)vi[e], q.filter_i);
      }
      if (!pass) continue;
      // 2-4. every window containing ts that is still open
      const int64_t w0 = floor_div(ts[e], q.slide);
      const uint32_t gk = key[e] & q.group_mask;
      bool any_open = false;
      for (int64_t k = 0; k < K; ++k) {
        const int64_t start = (w0 - k) * q.slide;
        if (o->have_wm && start + q.size <= o->wm) continue;  // already emitted
        any_open = true;
        OracleQuery::Agg& a = q.groups[std::make_pair(start, gk)];
        if (o->value_is_float) {
          const float v = vf[e];
          if (a.count == 0) {
            a.min_f = v;
            a.max_f = v;
          } else {
            if (total_less(v, a.min_f)) a.min_f = v;
            if (total_less(a.max_f, v)) a.max_f = v;
          }
          a.sum_f += (double)v;
        } else {
          const int32_t v = vi[e];
          if (a.count == 0) {
            a.min_i = v;
            a.max_i = v;
          } else {
            if (v < a.min_i) a.min_i = v;
            if (v > a.max_i) a.max_i = v;
          }
          a.sum_i += (int64_t)v;
        }
        a.count += 1;
      }
      if (!any_open) q.late_rows += 1;
    }
  }
  // 5. watermark over every arriving row (and the floor), then emission
  if (n > 0 || ts_floor != INT64_MIN) {
    int64_t mx = ts_floor;
    for (int64_t e = 0; e < n; ++e)
      if (ts[e] > mx) mx = ts[e];
    const int64_t cand = mx - o->lateness;
    if (!o->have_wm || cand > o->wm) o->wm = cand;
    o->have_wm = true;
  }
  for (OracleQuery& q : o->queries) {
    if (eos)
      emit_closed(*o, q, true);
    else if (o->have_wm)
      emit_closed(*o, q, false);
  }
  return 0;
}

int oracle_push(void* h, int64_t n, const int64_t* ts, const uint32_t* key,
                const void* value, const uint8_t* type, int eos) {
  return oracle_push_floor(h, n, ts, key, value, type, eos, INT64_MIN);
}

// Post-aggregation of query qid (see item 6 above): group_mask, HAVING (agg
// 0 = none) and ORDER BY (agg 0 = none).  Must precede the first push.
int oracle_set_post(void* h, int qid, uint32_t group_mask, int having_agg, int having_op,
                    double having_value, int order_agg, int order_desc) {
  Oracle* o = static_cast<Oracle*>(h);
  if (qid < 0 || qid >= (int)o->queries.size() || having_agg < 0 || having_agg > 5 ||
      order_agg < 0 || order_agg > 5)
    return -1;
  OracleQuery& q = o->queries[qid];
  q.group_mask = group_mask;
  q.having_agg = having_agg;
  q.having_op = having_op;
  q.having_value = having_value;
  q.order_agg = order_agg;
  q.order_desc = order_desc;
  return 0;
}

int64_t oracle_pending_rows(void* h, int qid) {
  Oracle* o = static_cast<Oracle*>(h);
  return (int64_t)o->queries[qid].out.size();
}

// Moves up to `cap` emitted rows (oldest first) into `dst`; returns the count.
int64_t oracle_take_rows(void* h, int qid, OracleRow* dst, int64_t cap) {
  Oracle* o = static_cast<Oracle*>(h);
  std::vector<OracleRow>& v = o->queries[qid].out;
  int64_t m = (int64_t)v.size() < cap ? (int64_t)v.size() : cap;
  if (m > 0) std::memcpy(dst, v.data(), (size_t)m * sizeof(OracleRow));
  v.erase(v.begin(), v.begin() + m);
  return m;
}

int64_t oracle_late_rows(void* h, int qid) {
  return static_cast<Oracle*>(h)->queries[qid].late_rows;
}

int64_t oracle_open_groups(void* h, int qid) {
  return (int64_t)static_cast<Oracle*>(h)->queries[qid].groups.size();
}

int64_t oracle_row_size(void) { return (int64_t)sizeof(OracleRow); }

}  // extern "C"
