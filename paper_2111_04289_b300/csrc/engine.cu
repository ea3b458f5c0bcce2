// Host engine behind the C ABI of include/lmstream.h.
//
// One lms_stream owns: the registered queries with their device window state
// (partial-group and state arrays), the scratch shared by the per-query
// pipelines, the device result buffers, device input buffers for host pushes,
// and a CUDA stream (its own, or the caller's).  push_microbatch enqueues the
// whole hot path for the batch — H2D (host input), fused K1, watermark, and per
// query sort/reduce, window enumeration + emission and carry — and then
// synchronises once, reads the control blocks back and, only if a device-side
// capacity check failed, grows the buffer and re-runs the emission.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lmstream.h"
#include "../../include/lmstream_testing.h"
#include "lms_internal.h"

namespace lms {

void set_float_filter(QueryDev* d) {
  const double c = d->filter_f;
  const float f = (float)c;
  float lo = f, hi = f;
  if ((double)f > c) lo = std::nextafter(f, -INFINITY);
  else if ((double)f < c) hi = std::nextafter(f, INFINITY);
  d->filter_lo = lo;
  d->filter_hi = hi;
  d->filter_exact = (lo == hi) ? 1 : 0;
}

void udiv_constants(unsigned long long d, unsigned long long* magic, int* sh1, int* sh2) {
  int l = 0;
  while (l < 64 && (1ull << l) < d) ++l;  // l = ceil(log2 d)
  const unsigned __int128 two64 = (unsigned __int128)1 << 64;
  const unsigned __int128 num = two64 * (((unsigned __int128)1 << l) - d);
  *magic = (unsigned long long)(num / d + 1);
  *sh1 = l < 1 ? l : 1;
  *sh2 = l > 1 ? l - 1 : 0;
}
}  // namespace lms

using namespace lms;

namespace {

long long floor_div_h(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

struct QueryHost {
  lms_query_spec spec{};
  long long size = 0, slide = 0;
  int k = 1;
  QueryDev dev{};
  unsigned long long cap = 0;  // group capacity of parts/state
  ResultRowDev* rows = nullptr;
  ResultRowDev* rows_tmp = nullptr;   // scratch rows of HAVING / ORDER BY (same capacity)
  unsigned long long rows_cap = 0;
  unsigned long long rows_read = 0;   // rows already handed out by poll
  unsigned long long row_base = 0;    // rows in the device buffer (mirror)
  unsigned long long carried = 0;     // groups carried into the next batch (mirror)
  unsigned long long n_state = 0;
  unsigned long long late_rows = 0, range_rows = 0;
  unsigned long long rows_emitted = 0;
  double sort_ms = 0, emit_count_ms = 0, emit_write_ms = 0;  // with enable_timing
  bool hidden = false;  // a side of a join (its rows feed the join, not the caller)
};

struct JoinHost {
  lms_join_spec spec{};
  int ql = 0, qr = 0;  // the side queries
  JCtl* jc = nullptr;
  JoinRowDev* rows = nullptr;
  unsigned long long cap = 0, row_base = 0, rows_read = 0, rows_emitted = 0;
};

}  // namespace

namespace {
struct GraphSlot {  // captured tail of a push
  cudaGraphExec_t exec = nullptr;
  unsigned long long gen = 0;
  int timing = 0;
  int launches = 0;
};
}  // namespace

struct lms_stream {
  lms_stream_config cfg{};
  unsigned long long gen = 0;  // bumped by every device allocation (pointers change)
  unsigned long long gen_prev = ~0ull;
  bool graph_ok = true;
  GraphSlot graphs[1];
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int sms = 148;
  std::mutex mu;
  std::string err;
  lms_status latched = LMS_OK;
  bool eos_seen = false;
  bool origin_set = false;
  long long origin_ts = 0;
  SCtl* sctl = nullptr;
  QCtl* qctl = nullptr;  // device array [kMaxQueries]
  std::vector<QueryHost> qs;
  std::vector<JoinHost> joins;
  Scratch scr{};
  unsigned long long in_cap = 0;
  long long* in_ts = nullptr;
  unsigned* in_key = nullptr;
  unsigned* in_val = nullptr;
  unsigned char* in_type = nullptr;
  unsigned long long dev_bytes = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  // ingest ring (lms_ingest / lms_push_ingested): rows [ring_head, ring_tail)
  // (absolute counters; row r lives at r mod ring_cap) in device memory, and
  // in pinned host memory for rows the library copied on the host
  cudaStream_t ist = nullptr;           // side stream of the ring's host-to-device copies
  unsigned long long ring_cap = 0, ring_head = 0, ring_tail = 0;
  long long* r_ts = nullptr;
  unsigned* r_key = nullptr;
  unsigned* r_val = nullptr;
  unsigned char* r_type = nullptr;
  long long* h_ts = nullptr;
  unsigned* h_key = nullptr;
  unsigned* h_val = nullptr;
  unsigned char* h_type = nullptr;
  unsigned long long pinned_bytes = 0;
  struct Copy {
    unsigned long long end;  // rows before this absolute index are copied once ev completes
    cudaEvent_t ev;
  };
  std::deque<Copy> copies;
  std::vector<cudaEvent_t> free_events;
  long long ring_first_ts = 0;          // ts of the first row ever ingested
  bool ring_first_set = false;
  cudaEvent_t ev[8] = {};
  cudaEvent_t tev[2] = {};  // around the fused pass while the autotuner samples
  cudaEvent_t qev[kMaxQueries][6] = {};  // E1, E2, sort/reduce
  lms_stats stats{};
  long long wm = LLONG_MIN;
  // watermark hint for the next push (lms_stream_set_batch_max_ts)
  long long ts_hint = 0;
  bool ts_hint_set = false;
  // fused-pass variant chooser installed by lms_stream_set_variant_chooser
  lms_variant_chooser vc = nullptr;
  lms_variant_observer vo = nullptr;
  void* vctx = nullptr;
};

namespace {

lms_status fail(lms_stream* s, lms_status code, const std::string& msg) {
  s->err = msg;
  return code;
}

lms_status cuda_fail(lms_stream* s, cudaError_t e, const char* what) {
  s->err = std::string(what) + ": " + cudaGetErrorString(e);
  s->latched = LMS_ECUDA;
  return LMS_ECUDA;
}

#define LMS_CK(call)                                    \
  do {                                                  \
    cudaError_t e__ = (call);                           \
    if (e__ != cudaSuccess) return cuda_fail(s, e__, #call); \
  } while (0)

lms_status dalloc(lms_stream* s, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (s->cfg.state_cap_bytes && s->dev_bytes + bytes > s->cfg.state_cap_bytes)
    return fail(s, LMS_ENOMEM, "device memory cap (state_cap_bytes) exceeded");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(s, LMS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  s->dev_bytes += bytes;
  s->allocs.emplace_back(*p, bytes);
  s->gen += 1;
  return LMS_OK;
}

void dfree(lms_stream* s, void* p) {
  if (!p) return;
  for (size_t i = 0; i < s->allocs.size(); ++i) {
    if (s->allocs[i].first == p) {
      s->dev_bytes -= s->allocs[i].second;
      s->allocs.erase(s->allocs.begin() + (long)i);
      break;
    }
  }
  cudaFree(p);
}

template <class T>
lms_status dgrow(lms_stream* s, T** p, unsigned long long old_n, unsigned long long new_n,
                 unsigned long long keep_n) {
  void* np = nullptr;
  lms_status r = dalloc(s, &np, new_n * sizeof(T));
  if (r != LMS_OK) return r;
  if (*p && keep_n) {
    cudaError_t e = cudaMemcpyAsync(np, *p, keep_n * sizeof(T), cudaMemcpyDeviceToDevice, s->st);
    if (e != cudaSuccess) return cuda_fail(s, e, "cudaMemcpyAsync(grow)");
  }
  if (*p) {
    cudaStreamSynchronize(s->st);
    dfree(s, *p);
  }
  (void)old_n;
  *p = static_cast<T*>(np);
  return LMS_OK;
}



unsigned long long round_cap(unsigned long long need) {
  unsigned long long c = 1ull << 12;
  while (c < need) c <<= 1;
  return c;
}

// Makes every group buffer hold `need` groups (parts keep their carried prefix).
lms_status ensure_group_capacity(lms_stream* s, unsigned long long need) {
  if (need >= (1ull << 32) - 1)
    return fail(s, LMS_EINVAL, "batch too large: more than 2^32-2 groups per query");
  for (QueryHost& q : s->qs) {
    if (q.cap >= need) continue;
    const unsigned long long nc = round_cap(need);
    lms_status r;
    if ((r = dgrow(s, &q.dev.parts, q.cap, nc, q.carried)) != LMS_OK) return r;
    if ((r = dgrow(s, &q.dev.pkeys, q.cap, nc, q.carried)) != LMS_OK) return r;
    if ((r = dgrow(s, &q.dev.state, q.cap, nc, 0)) != LMS_OK) return r;
    q.cap = nc;
    q.dev.parts_cap = nc;
  }
  Scratch& sc = s->scr;
  if (sc.cap < need) {
    const unsigned long long nc = round_cap(need);
    lms_status r;
    if ((r = dgrow(s, &sc.keysA, sc.cap, nc, 0)) != LMS_OK) return r;
    if ((r = dgrow(s, &sc.keysB, sc.cap, nc, 0)) != LMS_OK) return r;
    if ((r = dgrow(s, &sc.valsA, sc.cap, nc, 0)) != LMS_OK) return r;
    if ((r = dgrow(s, &sc.valsB, sc.cap, nc, 0)) != LMS_OK) return r;
    if ((r = dgrow(s, &sc.blk_id, sc.cap, nc + 1, 0)) != LMS_OK) return r;
    if ((r = dgrow(s, &sc.blk_begin, sc.cap, nc + 1, 0)) != LMS_OK) return r;
    sc.cap = nc;
    sc.blk_cap = nc;
  }
  return LMS_OK;
}

lms_status ensure_items(lms_stream* s, unsigned long long need) {
  Scratch& sc = s->scr;
  if (sc.item_cap >= need) return LMS_OK;
  const unsigned long long nc = round_cap(need);
  lms_status r;
  if ((r = dgrow(s, &sc.item_c, sc.item_cap, nc, 0)) != LMS_OK) return r;
  if ((r = dgrow(s, &sc.item_j, sc.item_cap, nc, 0)) != LMS_OK) return r;
  if ((r = dgrow(s, &sc.item_stat, sc.item_cap, nc, 0)) != LMS_OK) return r;
  if ((r = dgrow(s, &sc.unit_off, sc.item_cap * kMaxItemWindows, nc * kMaxItemWindows, 0)) != LMS_OK)
    return r;
  if ((r = dgrow(s, &sc.unit_bnd, sc.item_cap * kUnitBnd, nc * kUnitBnd, 0)) != LMS_OK) return r;
  sc.item_cap = nc;
  return LMS_OK;
}

lms_status ensure_rows(lms_stream* s, QueryHost& q, unsigned long long need) {
  if (q.rows_cap >= need) return LMS_OK;
  const unsigned long long nc = round_cap(need + need / 4);
  lms_status r = dgrow(s, &q.rows, q.rows_cap, nc, q.row_base);
  if (r != LMS_OK) return r;
  if (q.dev.having_agg || q.dev.order_agg) {
    if ((r = dgrow(s, &q.rows_tmp, q.rows_cap, nc, 0)) != LMS_OK) return r;
  }
  q.rows_cap = nc;
  return LMS_OK;
}

lms_status ensure_input(lms_stream* s, unsigned long long n) {
  if (s->in_cap >= n) return LMS_OK;
  const unsigned long long nc = round_cap(n);
  lms_status r;
  if ((r = dgrow(s, &s->in_ts, s->in_cap, nc, 0)) != LMS_OK) return r;
  if ((r = dgrow(s, &s->in_key, s->in_cap, nc, 0)) != LMS_OK) return r;
  if ((r = dgrow(s, &s->in_val, s->in_cap, nc, 0)) != LMS_OK) return r;
  if (s->cfg.has_type && (r = dgrow(s, &s->in_type, s->in_cap, nc, 0)) != LMS_OK) return r;
  s->in_cap = nc;
  return LMS_OK;
}

void set_origin(lms_stream* s, long long origin) {
  s->origin_ts = origin;
  s->origin_set = true;
  for (QueryHost& q : s->qs) {
    const long long op = floor_div_h(origin, q.slide);
    q.dev.origin_pane = op;
    q.dev.base = op * q.slide;
    q.dev.ts_off = (unsigned long long)kPaneBias * (unsigned long long)q.slide -
                   (unsigned long long)q.dev.base;
    q.dev.u_limit = 0xffffffffull * (unsigned long long)q.slide;
  }
}

lms_status read_ctls(lms_stream* s, QCtl* h) {
  LMS_CK(cudaMemcpyAsync(h, s->qctl, sizeof(QCtl) * s->qs.size(), cudaMemcpyDeviceToHost, s->st));
  LMS_CK(cudaStreamSynchronize(s->st));
  return LMS_OK;
}

// The fused pass's variant (tile of 1024 or 2048 events, with or without warp
// aggregation of equal group keys) for a batch of n rows: the configured one,
// or the autotuner's.  Below 2^15 rows variant 1 is used; above, each size
// class (log2 n) first runs every variant kTuneSamples times (timed with CUDA
// events) and then keeps the fastest per row.  Results do not depend on it.
// The table is shared by every stream of the process and keyed by (value type,
// number of queries, size class); the first timed pass of each variant in a
// class only warms it up and is not counted.
constexpr int kTuneSamples = 2;

struct Tune {
  double ms_per_row[5] = {0, 0, 0, 0, 0};
  int samples[5] = {0, 0, 0, 0, 0};  // -1: warm-up pending
  int choice = 0;
};
std::mutex g_tune_mu;
Tune g_tune[2][kMaxQueries + 1][48];

Tune& tune_slot(const lms_stream* s, long long n) {
  int b = 0;
  while ((1ll << (b + 1)) <= n && b < 47) ++b;
  return g_tune[s->cfg.value_type == LMS_VALUE_FLOAT32 ? 1 : 0][s->qs.size()][b];
}

int pick_k1_variant(lms_stream* s, long long n, bool* tuning) {
  *tuning = false;
  if (s->vc) {
    const int v = s->vc(s->vctx, n, (int32_t)s->qs.size());
    return (v >= 1 && v <= 4) ? v : 1;
  }
  if (s->cfg.k1_variant >= 1 && s->cfg.k1_variant <= 4) return s->cfg.k1_variant;
  if (n < (1ll << 15)) return 1;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  Tune& t = tune_slot(s, n);
  if (t.choice) return t.choice;
  *tuning = true;
  int v = 1;
  for (int k = 2; k <= 4; ++k)
    if (t.samples[k] < t.samples[v]) v = k;
  return v;
}

void record_k1_sample(lms_stream* s, long long n, int variant, float ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  Tune& t = tune_slot(s, n);
  s->stats.autotune_samples += 1;
  if (t.choice) return;
  if (t.samples[variant] == 0 && t.ms_per_row[variant] == 0.0) {
    t.ms_per_row[variant] = -1.0;  // the warm-up pass: not counted
    return;
  }
  if (t.ms_per_row[variant] < 0) t.ms_per_row[variant] = 0.0;
  t.ms_per_row[variant] += (double)ms / (double)n;
  t.samples[variant] += 1;
  for (int k = 1; k <= 4; ++k)
    if (t.samples[k] < kTuneSamples) return;
  int best = 1;
  for (int k = 2; k <= 4; ++k)
    if (t.ms_per_row[k] / t.samples[k] < t.ms_per_row[best] / t.samples[best]) best = k;
  t.choice = best;
}

}  // namespace

extern "C" {

int32_t lms_k1_tuned_variant(int32_t value_type, int32_t n_queries, int64_t rows) {
  if (n_queries < 1 || n_queries > kMaxQueries || rows < (1ll << 15)) return 1;
  int b = 0;
  while ((1ll << (b + 1)) <= rows && b < 47) ++b;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune[value_type == LMS_VALUE_FLOAT32 ? 1 : 0][n_queries][b].choice;
}

uint64_t lms_udiv_invariant(uint64_t n, uint64_t d) {
  if (d == 0) return 0;
  unsigned long long m;
  int sh1, sh2;
  udiv_constants(d, &m, &sh1, &sh2);
  const unsigned long long t = (unsigned long long)(((unsigned __int128)m * n) >> 64);
  return (t + ((n - t) >> sh1)) >> sh2;
}

lms_status stream_open(const lms_stream_config* cfg, lms_stream** out) {
  if (!cfg || !out) return LMS_EINVAL;
  if (cfg->value_type != LMS_VALUE_INT32 && cfg->value_type != LMS_VALUE_FLOAT32) return LMS_EINVAL;
  if (cfg->allowed_lateness_ms < 0 || cfg->max_batch_rows < 0) return LMS_EINVAL;
  if (cfg->graph_mode < LMS_GRAPH_DEFAULT || cfg->graph_mode > LMS_GRAPH_ON) return LMS_EINVAL;
  {
    unsigned bits = 0;
    for (int f = 0; f < 4; ++f) bits += (cfg->key_fields >> (8 * f)) & 0xffu;
    if (bits > 32) return LMS_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return LMS_ECUDA;
  }
  lms_stream* s = new lms_stream();
  s->cfg = *cfg;
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    delete s;
    return LMS_ECUDA;
  }
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, cfg->device);
  if (cfg->cuda_stream) {
    s->st = static_cast<cudaStream_t>(cfg->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return LMS_ECUDA;
    }
    s->own_stream = true;
  }
  void* p = nullptr;
  if (dalloc(s, &p, sizeof(SCtl)) != LMS_OK) {
    stream_close(s);
    return LMS_ENOMEM;
  }
  s->sctl = static_cast<SCtl*>(p);
  if (dalloc(s, &p, sizeof(QCtl) * kMaxQueries) != LMS_OK) {
    stream_close(s);
    return LMS_ENOMEM;
  }
  s->qctl = static_cast<QCtl*>(p);
  SCtl h{};
  h.batch_max_ts = LLONG_MIN;
  cudaMemcpy(s->sctl, &h, sizeof(h), cudaMemcpyHostToDevice);
  if (dalloc(s, &p, sizeof(unsigned) * (256 * kGrid + 256)) != LMS_OK ||
      (s->scr.hist = static_cast<unsigned*>(p), dalloc(s, &p, sizeof(unsigned long long) * (kGrid + 1))) != LMS_OK) {
    stream_close(s);
    return LMS_ENOMEM;
  }
  s->scr.chunk = static_cast<unsigned long long*>(p);
  for (int i = 0; i < 8; ++i) cudaEventCreate(&s->ev[i]);
  for (int i = 0; i < 2; ++i) cudaEventCreate(&s->tev[i]);
  for (int i = 0; i < kMaxQueries; ++i)
    for (int j = 0; j < 6; ++j) cudaEventCreate(&s->qev[i][j]);
  s->stats.watermark = LLONG_MIN;
  if (cudaGetLastError() != cudaSuccess) {
    stream_close(s);
    return LMS_ECUDA;
  }
  *out = s;
  return LMS_OK;
}

}  // extern "C"

namespace {

lms_status register_query(lms_stream* s, const lms_query_spec* q, bool hidden, int32_t* query_id) {
  if (s->stats.batches > 0) return fail(s, LMS_EINVAL, "queries must be registered before the first push");
  if ((int)s->qs.size() >= kMaxQueries) return fail(s, LMS_EINVAL, "at most 8 queries per stream");
  const long long size = q->window_size_ms;
  const long long slide = q->window_slide_ms == 0 ? size : q->window_slide_ms;
  if (size <= 0 || slide <= 0 || size % slide != 0 || size / slide > kMaxRuns ||
      slide >= (1ll << 31))
    return fail(s, LMS_EINVAL, "window: need size > 0, size % slide == 0, size/slide <= 4096, slide < 2^31");
  if (q->filter_col < LMS_COL_TS || q->filter_col > LMS_COL_TYPE || q->filter_op < LMS_OP_NONE ||
      q->filter_op > LMS_OP_GE)
    return fail(s, LMS_EINVAL, "filter: bad column or operator");
  if (q->having_agg < 0 || q->having_agg > LMS_POST_AVG || q->having_op < LMS_OP_NONE ||
      q->having_op > LMS_OP_GE || q->order_agg < 0 || q->order_agg > LMS_POST_AVG)
    return fail(s, LMS_EINVAL, "HAVING / ORDER BY: bad aggregate or operator");
  // GROUP BY fields: the mask of the selected fields' bits
  unsigned key_mask = 0xffffffffu;
  if (q->group_fields) {
    const unsigned kf = s->cfg.key_fields;
    unsigned shift = 0;
    key_mask = 0u;
    for (int f = 0; f < 4; ++f) {
      const unsigned w = (kf >> (8 * f)) & 0xffu;
      if ((q->group_fields >> f) & 1u) {
        if (w == 0) return fail(s, LMS_EINVAL, "GROUP BY: field not declared in key_fields");
        key_mask |= (w >= 32 ? 0xffffffffu : ((1u << w) - 1u)) << shift;
      }
      shift += w;
    }
    if (q->group_fields >> 4) return fail(s, LMS_EINVAL, "GROUP BY: at most four key fields");
  }
  QueryHost h;
  h.spec = *q;
  h.size = size;
  h.slide = slide;
  h.k = (int)(size / slide);
  QueryDev& d = h.dev;
  d.filter_col = q->filter_col;
  d.filter_op = q->filter_op;
  d.filter_i = q->filter_i;
  d.filter_f = q->filter_f;
  set_float_filter(&d);
  d.slide = (unsigned long long)slide;
  udiv_constants(d.slide, &d.magic, &d.sh1, &d.sh2);
  d.size = size;
  d.k = h.k;
  set_block_shape(&d);
  d.key_mask = key_mask;
  d.having_agg = q->having_agg;
  d.having_op = q->having_op;
  d.having_value = q->having_value;
  d.order_agg = q->order_agg;
  d.order_desc = q->order_desc ? 1 : 0;
  d.agg_mask = q->agg_mask ? q->agg_mask : LMS_AGG_ALL;
  d.qid = (int)s->qs.size();
  d.value_is_float = s->cfg.value_type == LMS_VALUE_FLOAT32;
  d.ctl = s->qctl + d.qid;
  QCtl c{};
  c.and_mask = ~0ull;
  c.cursor = 0;
  if (cudaMemcpy(d.ctl, &c, sizeof(c), cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_fail(s, cudaGetLastError(), "cudaMemcpy(ctl)");
  h.hidden = hidden;
  s->qs.push_back(h);
  *query_id = d.qid;
  return LMS_OK;
}

lms_status ensure_join_rows(lms_stream* s, JoinHost& j, unsigned long long need) {
  if (j.cap >= need) return LMS_OK;
  const unsigned long long nc = round_cap(need + need / 4);
  lms_status r = dgrow(s, &j.rows, j.cap, nc, j.row_base);
  if (r != LMS_OK) return r;
  j.cap = nc;
  return LMS_OK;
}

JoinArgs join_args(lms_stream* s, int i) {
  JoinHost& j = s->joins[i];
  JoinArgs a{};
  a.lrows = s->qs[j.ql].rows;
  a.lc = s->qs[j.ql].dev.ctl;
  a.rrows = s->qs[j.qr].rows;
  a.rc = s->qs[j.qr].dev.ctl;
  a.out = j.rows;
  a.cap = j.cap;
  a.jc = j.jc;
  a.jid = i;
  return a;
}

}  // namespace

extern "C" {

lms_status query_register(lms_stream* s, const lms_query_spec* q, int32_t* query_id) {
  if (!s || !q || !query_id) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  return register_query(s, q, false, query_id);
}

lms_status lms_join_register(lms_stream* s, const lms_join_spec* j, int32_t* join_id) {
  if (!s || !j || !join_id) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stats.batches > 0) return fail(s, LMS_EINVAL, "joins must be registered before the first push");
  if (s->joins.size() >= 4) return fail(s, LMS_EINVAL, "at most 4 joins per stream");
  if ((int)s->qs.size() + 2 > kMaxQueries)
    return fail(s, LMS_EINVAL, "a join needs two of the stream's 8 query slots");
  lms_query_spec side{};
  side.window_size_ms = j->window_size_ms;
  side.window_slide_ms = j->window_slide_ms;
  side.agg_mask = LMS_AGG_COUNT | LMS_AGG_SUM;
  JoinHost jh;
  jh.spec = *j;
  lms_status r;
  side.filter_col = j->left_col;
  side.filter_op = j->left_op;
  side.filter_i = j->left_i;
  side.filter_f = j->left_f;
  if ((r = register_query(s, &side, true, &jh.ql)) != LMS_OK) return r;
  side.filter_col = j->right_col;
  side.filter_op = j->right_op;
  side.filter_i = j->right_i;
  side.filter_f = j->right_f;
  if ((r = register_query(s, &side, true, &jh.qr)) != LMS_OK) {
    s->qs.pop_back();
    return r;
  }
  void* p = nullptr;
  if ((r = dalloc(s, &p, sizeof(JCtl))) != LMS_OK) return r;
  jh.jc = static_cast<JCtl*>(p);
  const JCtl z{};
  if (cudaMemcpy(jh.jc, &z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_fail(s, cudaGetLastError(), "cudaMemcpy(join ctl)");
  s->joins.push_back(jh);
  if ((r = ensure_join_rows(s, s->joins.back(), 4096)) != LMS_OK) return r;
  *join_id = (int32_t)s->joins.size() - 1;
  return LMS_OK;
}

lms_status lms_join_poll(lms_stream* s, int32_t join_id, lms_join_row* out, size_t cap,
                         size_t* n_out) {
  if (!s || !n_out || (cap && !out)) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->latched != LMS_OK) return s->latched;
  if (join_id < 0 || join_id >= (int)s->joins.size()) return fail(s, LMS_EINVAL, "bad join id");
  JoinHost& j = s->joins[join_id];
  const unsigned long long avail = j.row_base - j.rows_read;
  if (avail == 0) return LMS_EAGAIN;
  const unsigned long long m = std::min<unsigned long long>(avail, cap);
  if (m) {
    LMS_CK(cudaMemcpyAsync(out, j.rows + j.rows_read, m * sizeof(lms_join_row),
                           cudaMemcpyDeviceToHost, s->st));
    LMS_CK(cudaStreamSynchronize(s->st));
  }
  j.rows_read += m;
  if (j.rows_read == j.row_base) {
    j.rows_read = 0;
    j.row_base = 0;
    const unsigned long long zero = 0;
    LMS_CK(cudaMemcpyAsync(&j.jc->row_base, &zero, sizeof(zero), cudaMemcpyHostToDevice, s->st));
    LMS_CK(cudaStreamSynchronize(s->st));
  }
  *n_out = (size_t)m;
  return LMS_OK;
}

}  // extern "C"

namespace {

// One contiguous piece of a micro-batch's columns in device memory.
struct InSeg {
  const long long* ts;
  const unsigned* key;
  const void* val;
  const unsigned char* typ;
  long long n;
};

// Copies `bytes` on the host, with up to 8 threads for large copies.
void par_memcpy(void* dst, const void* src, size_t bytes) {
  constexpr size_t kPiece = 16u << 20;
  if (bytes < 2 * kPiece) {
    std::memcpy(dst, src, bytes);
    return;
  }
  const size_t hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nt = std::min<size_t>(std::min<size_t>(8, hw), bytes / kPiece);
  const size_t per = (bytes + nt - 1) / nt;
  std::vector<std::thread> th;
  for (size_t t = 1; t < nt; ++t) {
    const size_t a = t * per;
    if (a >= bytes) break;
    const size_t len = std::min(per, bytes - a);
    th.emplace_back([=] { std::memcpy(static_cast<char*>(dst) + a, static_cast<const char*>(src) + a, len); });
  }
  std::memcpy(dst, src, std::min(per, bytes));
  for (std::thread& x : th) x.join();
}

// Grows the ingest ring to at least `need` rows: new device and pinned
// rings, the rows held moved to their front (after every copy in flight).
lms_status ensure_ring(lms_stream* s, unsigned long long need) {
  if (s->ring_cap >= need) return LMS_OK;
  const unsigned long long nc = round_cap(need + need / 2);
  LMS_CK(cudaStreamSynchronize(s->ist));
  LMS_CK(cudaStreamSynchronize(s->st));
  void *d_ts, *d_key, *d_val, *d_type = nullptr;
  lms_status r;
  if ((r = dalloc(s, &d_ts, nc * 8)) != LMS_OK || (r = dalloc(s, &d_key, nc * 4)) != LMS_OK ||
      (r = dalloc(s, &d_val, nc * 4)) != LMS_OK ||
      (s->cfg.has_type && (r = dalloc(s, &d_type, nc)) != LMS_OK))
    return r;
  void *p_ts = nullptr, *p_key = nullptr, *p_val = nullptr, *p_type = nullptr;
  if (cudaHostAlloc(&p_ts, nc * 8, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&p_key, nc * 4, cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&p_val, nc * 4, cudaHostAllocDefault) != cudaSuccess ||
      (s->cfg.has_type && cudaHostAlloc(&p_type, nc, cudaHostAllocDefault) != cudaSuccess)) {
    cudaGetLastError();
    cudaFreeHost(p_ts);
    cudaFreeHost(p_key);
    cudaFreeHost(p_val);
    cudaFreeHost(p_type);
    return fail(s, LMS_ENOMEM, "cudaHostAlloc: pinned ingest ring");
  }
  // move the rows held, [head, tail), to rows [0, tail - head) of the new ring
  const unsigned long long held = s->ring_tail - s->ring_head;
  for (unsigned long long done = 0; done < held;) {
    const unsigned long long pos = (s->ring_head + done) % s->ring_cap;
    const unsigned long long m = std::min(held - done, s->ring_cap - pos);
    LMS_CK(cudaMemcpyAsync(static_cast<long long*>(d_ts) + done, s->r_ts + pos, m * 8,
                           cudaMemcpyDeviceToDevice, s->st));
    LMS_CK(cudaMemcpyAsync(static_cast<unsigned*>(d_key) + done, s->r_key + pos, m * 4,
                           cudaMemcpyDeviceToDevice, s->st));
    LMS_CK(cudaMemcpyAsync(static_cast<unsigned*>(d_val) + done, s->r_val + pos, m * 4,
                           cudaMemcpyDeviceToDevice, s->st));
    if (d_type)
      LMS_CK(cudaMemcpyAsync(static_cast<unsigned char*>(d_type) + done, s->r_type + pos, m,
                             cudaMemcpyDeviceToDevice, s->st));
    done += m;
  }
  LMS_CK(cudaStreamSynchronize(s->st));
  dfree(s, s->r_ts);
  dfree(s, s->r_key);
  dfree(s, s->r_val);
  dfree(s, s->r_type);
  cudaFreeHost(s->h_ts);
  cudaFreeHost(s->h_key);
  cudaFreeHost(s->h_val);
  cudaFreeHost(s->h_type);
  s->r_ts = static_cast<long long*>(d_ts);
  s->r_key = static_cast<unsigned*>(d_key);
  s->r_val = static_cast<unsigned*>(d_val);
  s->r_type = static_cast<unsigned char*>(d_type);
  s->h_ts = static_cast<long long*>(p_ts);
  s->h_key = static_cast<unsigned*>(p_key);
  s->h_val = static_cast<unsigned*>(p_val);
  s->h_type = static_cast<unsigned char*>(p_type);
  s->pinned_bytes = nc * (8 + 4 + 4 + (s->cfg.has_type ? 1 : 0));
  for (const lms_stream::Copy& c : s->copies) s->free_events.push_back(c.ev);
  s->copies.clear();
  s->ring_tail = held;
  s->ring_head = 0;
  s->ring_cap = nc;
  return LMS_OK;
}

// Sets the event-time origin from the first row of the first pushed batch.
void origin_from(lms_stream* s, bool have_row, long long first_ts) {
  if (s->origin_set) return;
  if (s->cfg.origin_ts != LMS_ORIGIN_AUTO) set_origin(s, s->cfg.origin_ts);
  else set_origin(s, have_row ? first_ts : 0);
}

// The hot path of one micro-batch of n rows whose columns are the device
// segments seg[0 .. nseg) (their copy, if any, is already enqueued on s->st
// after s->ev[0]); group buffers must hold the carried groups plus n.
lms_status run_batch(lms_stream* s, const InSeg* seg, int nseg, long long n, int eos,
                     std::chrono::steady_clock::time_point t0) {
  const bool timing = s->cfg.enable_timing != 0;
  lms_status r = LMS_OK;
  if (timing) LMS_CK(cudaEventRecord(s->ev[5], s->st));
  int launches = 0;
  int variant = 1;
  bool tuning = false, timed_k1 = false;
  QCtl* ctls[kMaxQueries];
  const int nq = (int)s->qs.size();
  for (int i = 0; i < nq; ++i) ctls[i] = s->qs[i].dev.ctl;
  LMS_CK(launch_batch_begin(s->sctl, ctls, nq, s->ts_hint_set ? s->ts_hint : LLONG_MIN, s->st));
  s->ts_hint_set = false;
  ++launches;
  if (timing) LMS_CK(cudaEventRecord(s->ev[1], s->st));
  if (n > 0) {
    variant = pick_k1_variant(s, n, &tuning);
    timed_k1 = tuning || s->vo != nullptr;
    if (timed_k1) LMS_CK(cudaEventRecord(s->tev[0], s->st));
    for (int g = 0; g < nseg; ++g) {  // one fused pass per contiguous piece of the batch
      if (seg[g].n == 0) continue;
      K1Args a{};
      a.ts = seg[g].ts;
      a.key = seg[g].key;
      a.value = seg[g].val;
      a.type = seg[g].typ;
      a.n = seg[g].n;
      a.nq = nq;
      a.value_is_float = s->cfg.value_type == LMS_VALUE_FLOAT32;
      a.sctl = s->sctl;
      for (int i = 0; i < nq; ++i) a.q[i] = s->qs[i].dev;
      const long long ntiles = (a.n + k1_tile_events(variant) - 1) / k1_tile_events(variant);
      const int grid = (int)std::min<long long>(ntiles, k1_max_grid(s->cfg.device, variant, 0));
      LMS_CK(launch_k1(a, variant, grid, s->st));
      ++launches;
      ++s->stats.k1_launches;
    }
    if (timed_k1) LMS_CK(cudaEventRecord(s->tev[1], s->st));
    s->stats.k1_tile_events = (uint64_t)k1_tile_events(variant);
  }
  if (timing) LMS_CK(cudaEventRecord(s->ev[2], s->st));
  std::vector<QueryDev> qd(nq);
  for (int i = 0; i < nq; ++i) qd[i] = s->qs[i].dev;
  // emission needs item and row buffers; make sure something exists
  if ((r = ensure_items(s, 1024)) != LMS_OK) return r;
  for (QueryHost& q : s->qs)
    if ((r = ensure_rows(s, q, q.row_base + 4096)) != LMS_OK) return r;
  for (JoinHost& j : s->joins)
    if ((r = ensure_join_rows(s, j, j.row_base + 4096)) != LMS_OK) return r;
  // (Timing events inside the tail are recorded as external event nodes so that
  // a replayed graph still records them.)
  // The rest of the batch's work — watermark, then per query (back to back:
  // they share the scratch) sort/reduce into the window state, pane index,
  // emission of closed windows, carry of open panes — reads every size on the
  // device, so it is the same launch sequence for every batch until a buffer
  // is reallocated: it is captured once into a CUDA graph and replayed.
  auto enqueue_tail = [&](int* nl) -> cudaError_t {
    cudaError_t e = launch_watermark(s->sctl, qd.data(), nq, s->cfg.allowed_lateness_ms, eos, s->st);
    ++*nl;
    for (int i = 0; i < nq && e == cudaSuccess; ++i) {
      QueryHost& q = s->qs[i];
      if (timing && (e = record_event(s->qev[i][4], s->st)) != cudaSuccess) break;
      if ((e = launch_sort_reduce(qd[i], s->scr, s->st, nl)) != cudaSuccess) break;
      if (timing && (e = record_event(s->qev[i][5], s->st)) != cudaSuccess) break;
      if ((e = launch_block_index(q.dev, s->scr, s->st, nl)) != cudaSuccess) break;
      if ((e = launch_emit(q.dev, s->scr, q.rows, q.rows_cap, s->sms, s->st, nl,
                           timing ? s->qev[i] : nullptr)) != cudaSuccess)
        break;
      if ((e = launch_post(q.dev, s->scr, q.rows, q.rows_tmp, s->sms, s->st, nl)) != cudaSuccess)
        break;
      e = launch_trim(q.dev, s->scr, s->sms, s->st, nl);
    }
    for (size_t i = 0; i < s->joins.size() && e == cudaSuccess; ++i)
      e = launch_join(join_args(s, (int)i), s->scr, true, s->st, nl);
    if (e == cudaSuccess && timing) e = record_event(s->ev[4], s->st);
    return e;
  };
  // Replay only once the buffers are stable (the previous push saw the same
  // ones), and not for the one-off end-of-stream push; the first launches of
  // a stream also run plainly, so one-time kernel set-up never happens inside
  // a capture.
  const bool stable = s->gen == s->gen_prev;
  s->gen_prev = s->gen;
  GraphSlot& g = s->graphs[0];
  bool use_graph = s->cfg.graph_mode != LMS_GRAPH_OFF && stable && !eos && s->graph_ok;
  if (use_graph && (!g.exec || g.gen != s->gen || g.timing != (int)timing)) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    if (cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();  // this stream cannot be captured (e.g. a legacy stream)
      s->graph_ok = false;
      use_graph = false;
    } else {
      cudaGraph_t graph = nullptr;
      int nl = 0;
      const cudaError_t ce = enqueue_tail(&nl);
      const cudaError_t ee = cudaStreamEndCapture(s->st, &graph);
      LMS_CK(ce);
      LMS_CK(ee);
      const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      LMS_CK(ie);
      g.gen = s->gen;
      g.timing = (int)timing;
      g.launches = nl;
      s->stats.graph_captures += 1;
    }
  }
  if (use_graph) {
    LMS_CK(cudaGraphLaunch(g.exec, s->st));
    launches += g.launches;
    s->stats.graph_launches += 1;
  } else {
    LMS_CK(enqueue_tail(&launches));
  }
  std::vector<QCtl> hc(nq);
  if ((r = read_ctls(s, hc.data())) != LMS_OK) return r;
  if (timed_k1) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->tev[0], s->tev[1]) == cudaSuccess) {
      if (tuning) record_k1_sample(s, n, variant, ms);
      if (s->vo) s->vo(s->vctx, n, variant, (double)ms);
    }
    cudaGetLastError();
  }
  // retry emission for queries whose buffers were too small
  bool retried = false;
  for (int i = 0; i < nq; ++i) {
    QueryHost& q = s->qs[i];
    for (int attempt = 0; (hc[i].err & kErrNeedRetry) && attempt < 4; ++attempt) {
      if (hc[i].err & kErrItemOverflow) {
        if ((r = ensure_items(s, hc[i].n_items)) != LMS_OK) return r;
      }
      if (hc[i].err & kErrRowsOverflow) {
        if ((r = ensure_rows(s, q, hc[i].row_base + hc[i].rows_batch)) != LMS_OK) return r;
      }
      LMS_CK(launch_block_index(q.dev, s->scr, s->st, &launches));
      LMS_CK(launch_emit(q.dev, s->scr, q.rows, q.rows_cap, s->sms, s->st, &launches,
                         nullptr));
      LMS_CK(launch_post(q.dev, s->scr, q.rows, q.rows_tmp, s->sms, s->st, &launches));
      LMS_CK(launch_trim(q.dev, s->scr, s->sms, s->st, &launches));
      if ((r = read_ctls(s, hc.data())) != LMS_OK) return r;
      retried = true;
    }
    if (hc[i].err & kErrNeedRetry)
      return fail(s, LMS_ENOMEM, "emission buffers could not be grown enough");
    if (hc[i].err & kErrOrderBy)
      return fail(s, LMS_EINVAL, "ORDER BY: a window holds more than LMS_ORDER_MAX_ROWS rows");
    if (hc[i].err & (kErrPartsOverflow | kErrProbe)) {
      s->latched = LMS_EDEVICE;
      return fail(s, LMS_EDEVICE, "internal device error flag raised by a kernel");
    }
  }
  // joins whose sides were retried, or whose row buffer was too small
  for (size_t i = 0; i < s->joins.size(); ++i) {
    JoinHost& j = s->joins[i];
    for (int attempt = 0;; ++attempt) {
      JCtl jh{};
      LMS_CK(cudaMemcpyAsync(&jh, j.jc, sizeof(jh), cudaMemcpyDeviceToHost, s->st));
      LMS_CK(cudaStreamSynchronize(s->st));
      if (!(jh.err & kJoinPendingBit)) {
        j.rows_emitted += jh.rows_batch;
        j.row_base = jh.row_base;
        break;
      }
      if (attempt >= 4) return fail(s, LMS_ENOMEM, "join rows: the buffer could not be grown enough");
      if (jh.err & kJoinOverflowBit) {
        if ((r = ensure_join_rows(s, j, jh.row_base + jh.rows_batch)) != LMS_OK) return r;
      }
      LMS_CK(launch_join(join_args(s, (int)i), s->scr, false, s->st, &launches));
    }
  }
  if (!s->joins.empty() && (r = read_ctls(s, hc.data())) != LMS_OK) return r;
  SCtl hs{};
  LMS_CK(cudaMemcpyAsync(&hs, s->sctl, sizeof(hs), cudaMemcpyDeviceToHost, s->st));
  LMS_CK(cudaStreamSynchronize(s->st));
  if (hs.wm_valid) s->wm = hs.wm;
  unsigned long long late = 0, range = 0, rows = 0, groups = 0;
  for (int i = 0; i < nq; ++i) {
    QueryHost& q = s->qs[i];
    s->stats.partials += hc[i].parts_at_sort - q.carried;
    s->stats.groups_built += hc[i].n_state;
    q.rows_emitted += hc[i].rows_batch;
    q.row_base = hc[i].row_base;
    q.carried = hc[i].carried;
    q.n_state = hc[i].n_state;
    q.late_rows = hc[i].late_rows;
    q.range_rows = hc[i].range_rows;
    late += q.late_rows;
    range += q.range_rows;
    if (!q.hidden) rows += q.rows_emitted;
    groups += q.carried;
  }
  if (timing) {
    float a = 0, bms = 0, all = 0, sort_ms = 0;
    for (int i = 0; i < nq; ++i) {
      float x = 0;
      cudaEventElapsedTime(&x, s->qev[i][4], s->qev[i][5]);
      sort_ms += x;
      s->qs[i].sort_ms += x;
    }
    cudaEventElapsedTime(&a, s->ev[0], s->ev[5]);
    cudaEventElapsedTime(&bms, s->ev[1], s->ev[2]);
    cudaEventElapsedTime(&all, s->ev[2], s->ev[4]);
    cudaGetLastError();  // a failed timing read must not poison later calls
    s->stats.h2d_ms += a;
    s->stats.k1_ms += bms;
    s->stats.sort_ms += sort_ms;
    s->stats.emit_ms += all - sort_ms;
    if (!retried) {
      for (int i = 0; i < nq; ++i) {
        float e1 = 0, e2 = 0;
        cudaEventElapsedTime(&e1, s->qev[i][0], s->qev[i][1]);
        cudaEventElapsedTime(&e2, s->qev[i][2], s->qev[i][3]);
        s->qs[i].emit_count_ms += e1;
        s->qs[i].emit_write_ms += e2;
        s->stats.e1_ms += e1;
        s->stats.e2_ms += e2;
      }
      cudaGetLastError();
    }
  }
  s->stats.batches += 1;
  s->stats.events += (unsigned long long)n;
  s->stats.late_rows = late;
  s->stats.range_rows = range;
  s->stats.rows_emitted = rows;
  s->stats.state_groups = groups;
  s->stats.watermark = s->wm;
  s->stats.kernel_launches += (unsigned long long)launches;
  s->stats.last_batch_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (eos) s->eos_seen = true;
  return LMS_OK;
}

}  // namespace

extern "C" {

lms_status push_microbatch(lms_stream* s, const lms_batch* b) {
  if (!s || !b) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->latched != LMS_OK) return s->latched;
  if (s->eos_seen) return fail(s, LMS_ECLOSED, "stream already ended");
  if (s->qs.empty()) return fail(s, LMS_EINVAL, "no query registered");
  const long long n = b->n_rows;
  if (n < 0) return fail(s, LMS_EINVAL, "n_rows < 0");
  if (n > 0 && (!b->ts || !b->key || !b->value || (s->cfg.has_type && !b->type)))
    return fail(s, LMS_EINVAL, "missing column pointer");
  if (b->memory != LMS_MEM_HOST && b->memory != LMS_MEM_DEVICE)
    return fail(s, LMS_EINVAL, "bad memory kind");
  if (s->ring_tail != s->ring_head)
    return fail(s, LMS_EINVAL, "ingested rows pending: push them with lms_push_ingested first");
  const auto t0 = std::chrono::steady_clock::now();
  LMS_CK(cudaSetDevice(s->cfg.device));
  const int eos = (b->flags & LMS_BATCH_EOS) ? 1 : 0;
  if (!s->origin_set) {
    long long first = 0;
    if (n > 0 && s->cfg.origin_ts == LMS_ORIGIN_AUTO) {
      if (b->memory == LMS_MEM_HOST) first = (long long)b->ts[0];
      else {
        LMS_CK(cudaMemcpyAsync(&first, b->ts, sizeof(long long), cudaMemcpyDeviceToHost, s->st));
        LMS_CK(cudaStreamSynchronize(s->st));
      }
    }
    origin_from(s, n > 0, first);
  }
  // capacities: parts hold the carried groups plus at most one group per row
  unsigned long long need = 0;
  for (QueryHost& q : s->qs) need = std::max(need, q.carried + (unsigned long long)n);
  lms_status r = ensure_group_capacity(s, need + 1);
  if (r != LMS_OK) return r;
  const bool timing = s->cfg.enable_timing != 0;
  InSeg seg{reinterpret_cast<const long long*>(b->ts), b->key, b->value,
            s->cfg.has_type ? b->type : nullptr, n};
  if (timing) LMS_CK(cudaEventRecord(s->ev[0], s->st));
  if (n > 0 && b->memory == LMS_MEM_HOST) {
    if ((r = ensure_input(s, (unsigned long long)n)) != LMS_OK) return r;
    LMS_CK(cudaMemcpyAsync(s->in_ts, b->ts, n * 8, cudaMemcpyHostToDevice, s->st));
    LMS_CK(cudaMemcpyAsync(s->in_key, b->key, n * 4, cudaMemcpyHostToDevice, s->st));
    LMS_CK(cudaMemcpyAsync(s->in_val, b->value, n * 4, cudaMemcpyHostToDevice, s->st));
    if (seg.typ) LMS_CK(cudaMemcpyAsync(s->in_type, b->type, n, cudaMemcpyHostToDevice, s->st));
    seg = InSeg{s->in_ts, s->in_key, s->in_val, seg.typ ? s->in_type : nullptr, n};
  }
  return run_batch(s, &seg, 1, n, eos, t0);
}

lms_status lms_ingest(lms_stream* s, const lms_batch* b) {
  if (!s || !b) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->latched != LMS_OK) return s->latched;
  if (s->eos_seen) return fail(s, LMS_ECLOSED, "stream already ended");
  if (s->qs.empty()) return fail(s, LMS_EINVAL, "no query registered");
  const long long n = b->n_rows;
  if (n < 0) return fail(s, LMS_EINVAL, "n_rows < 0");
  if (b->memory != LMS_MEM_HOST) return fail(s, LMS_EINVAL, "lms_ingest takes host columns");
  if (n == 0) return LMS_OK;
  if (!b->ts || !b->key || !b->value || (s->cfg.has_type && !b->type))
    return fail(s, LMS_EINVAL, "missing column pointer");
  LMS_CK(cudaSetDevice(s->cfg.device));
  if (!s->ist) LMS_CK(cudaStreamCreateWithFlags(&s->ist, cudaStreamNonBlocking));
  lms_status r = ensure_ring(s, s->ring_tail - s->ring_head + (unsigned long long)n);
  if (r != LMS_OK) return r;
  if (!s->ring_first_set) {
    s->ring_first_ts = (long long)b->ts[0];
    s->ring_first_set = true;
  }
  const bool stable = (b->flags & LMS_INGEST_STABLE) != 0;
  const bool typ = s->cfg.has_type;
  unsigned long long pos = s->ring_tail % s->ring_cap, done = 0;
  while (done < (unsigned long long)n) {
    const unsigned long long m = std::min((unsigned long long)n - done, s->ring_cap - pos);
    const void* src_ts = b->ts + done;
    const void* src_key = b->key + done;
    const void* src_val = static_cast<const unsigned*>(b->value) + done;
    const void* src_type = typ ? b->type + done : nullptr;
    if (!stable) {  // into the library's pinned ring first: the caller may reuse its buffers
      par_memcpy(s->h_ts + pos, src_ts, m * 8);
      par_memcpy(s->h_key + pos, src_key, m * 4);
      par_memcpy(s->h_val + pos, src_val, m * 4);
      if (typ) par_memcpy(s->h_type + pos, src_type, m);
      src_ts = s->h_ts + pos;
      src_key = s->h_key + pos;
      src_val = s->h_val + pos;
      src_type = typ ? s->h_type + pos : nullptr;
    }
    LMS_CK(cudaMemcpyAsync(s->r_ts + pos, src_ts, m * 8, cudaMemcpyHostToDevice, s->ist));
    LMS_CK(cudaMemcpyAsync(s->r_key + pos, src_key, m * 4, cudaMemcpyHostToDevice, s->ist));
    LMS_CK(cudaMemcpyAsync(s->r_val + pos, src_val, m * 4, cudaMemcpyHostToDevice, s->ist));
    if (typ) LMS_CK(cudaMemcpyAsync(s->r_type + pos, src_type, m, cudaMemcpyHostToDevice, s->ist));
    done += m;
    pos = 0;
  }
  cudaEvent_t ev = nullptr;
  if (!s->free_events.empty()) {
    ev = s->free_events.back();
    s->free_events.pop_back();
  } else {
    LMS_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  LMS_CK(cudaEventRecord(ev, s->ist));
  s->ring_tail += (unsigned long long)n;
  s->copies.push_back({s->ring_tail, ev});
  return LMS_OK;
}

lms_status lms_push_ingested(lms_stream* s, int64_t n_rows, uint32_t flags) {
  if (!s) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->latched != LMS_OK) return s->latched;
  if (s->eos_seen) return fail(s, LMS_ECLOSED, "stream already ended");
  if (s->qs.empty()) return fail(s, LMS_EINVAL, "no query registered");
  if (n_rows < 0 || (unsigned long long)n_rows > s->ring_tail - s->ring_head)
    return fail(s, LMS_EINVAL, "n_rows exceeds the rows ingested and not yet pushed");
  const auto t0 = std::chrono::steady_clock::now();
  LMS_CK(cudaSetDevice(s->cfg.device));
  const long long n = n_rows;
  const int eos = (flags & LMS_BATCH_EOS) ? 1 : 0;
  origin_from(s, s->ring_first_set, s->ring_first_ts);
  unsigned long long need = 0;
  for (QueryHost& q : s->qs) need = std::max(need, q.carried + (unsigned long long)n);
  lms_status r = ensure_group_capacity(s, need + 1);
  if (r != LMS_OK) return r;
  if (s->cfg.enable_timing) LMS_CK(cudaEventRecord(s->ev[0], s->st));
  InSeg seg[2];
  int nseg = 0;
  if (n > 0) {
    // the compute stream waits for the copies of the batch's rows
    const unsigned long long end = s->ring_head + (unsigned long long)n;
    for (const lms_stream::Copy& c : s->copies) {
      LMS_CK(cudaStreamWaitEvent(s->st, c.ev, 0));
      if (c.end >= end) break;
    }
    const unsigned long long pos = s->ring_head % s->ring_cap;
    const unsigned long long m = std::min((unsigned long long)n, s->ring_cap - pos);
    const bool typ = s->cfg.has_type;
    seg[nseg++] = InSeg{s->r_ts + pos, s->r_key + pos, s->r_val + pos, typ ? s->r_type + pos : nullptr,
                        (long long)m};
    if ((unsigned long long)n > m)
      seg[nseg++] = InSeg{s->r_ts, s->r_key, s->r_val, typ ? s->r_type : nullptr, n - (long long)m};
  }
  r = run_batch(s, seg, nseg, n, eos, t0);
  if (r == LMS_OK) {
    s->ring_head += (unsigned long long)n;
    while (!s->copies.empty() && s->copies.front().end <= s->ring_head) {
      s->free_events.push_back(s->copies.front().ev);
      s->copies.pop_front();
    }
  }
  return r;
}

lms_status lms_ingest_pending(lms_stream* s, int64_t* n_rows) {
  if (!s || !n_rows) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *n_rows = (int64_t)(s->ring_tail - s->ring_head);
  return LMS_OK;
}

lms_status poll_results(lms_stream* s, int32_t query_id, lms_result_row* out, size_t cap,
                        size_t* n_out, int32_t timeout_ms) {
  (void)timeout_ms;  // results are complete when push_microbatch returns
  if (!s || !n_out || (cap && !out)) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->latched != LMS_OK) return s->latched;
  if (query_id < 0 || query_id >= (int)s->qs.size() || s->qs[query_id].hidden)
    return fail(s, LMS_EINVAL, "bad query id");
  QueryHost& q = s->qs[query_id];
  const unsigned long long avail = q.row_base - q.rows_read;
  if (avail == 0) return LMS_EAGAIN;
  const unsigned long long m = std::min<unsigned long long>(avail, cap);
  if (m) {
    LMS_CK(cudaMemcpyAsync(out, q.rows + q.rows_read, m * sizeof(lms_result_row),
                           cudaMemcpyDeviceToHost, s->st));
    LMS_CK(cudaStreamSynchronize(s->st));
  }
  q.rows_read += m;
  if (q.rows_read == q.row_base) {
    q.rows_read = 0;
    q.row_base = 0;
    const unsigned long long zero = 0;
    LMS_CK(cudaMemcpyAsync(&q.dev.ctl->row_base, &zero, sizeof(zero), cudaMemcpyHostToDevice,
                           s->st));
    LMS_CK(cudaStreamSynchronize(s->st));
  }
  *n_out = (size_t)m;
  return LMS_OK;
}

lms_status lms_results_device(lms_stream* s, int32_t query_id, const lms_result_row** rows,
                              size_t* n) {
  if (!s || !rows || !n) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (query_id < 0 || query_id >= (int)s->qs.size() || s->qs[query_id].hidden)
    return fail(s, LMS_EINVAL, "bad query id");
  QueryHost& q = s->qs[query_id];
  *rows = reinterpret_cast<const lms_result_row*>(q.rows + q.rows_read);
  *n = (size_t)(q.row_base - q.rows_read);
  return LMS_OK;
}

lms_status lms_results_discard(lms_stream* s, int32_t query_id) {
  if (!s) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (query_id < 0 || query_id >= (int)s->qs.size() || s->qs[query_id].hidden)
    return fail(s, LMS_EINVAL, "bad query id");
  QueryHost& q = s->qs[query_id];
  q.rows_read = 0;
  q.row_base = 0;
  const unsigned long long zero = 0;
  LMS_CK(cudaMemcpyAsync(&q.dev.ctl->row_base, &zero, sizeof(zero), cudaMemcpyHostToDevice, s->st));
  LMS_CK(cudaStreamSynchronize(s->st));
  return LMS_OK;
}

lms_status lms_stream_set_variant_chooser(lms_stream* s, lms_variant_chooser choose,
                                          lms_variant_observer observe, void* ctx) {
  if (!s) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->vc = choose;
  s->vo = observe;
  s->vctx = ctx;
  return LMS_OK;
}

lms_status lms_stream_stats(lms_stream* s, lms_stats* out) {
  if (!s || !out) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  unsigned long long pending = 0;
  for (QueryHost& q : s->qs) pending += q.row_base - q.rows_read;
  out->rows_pending = pending;
  out->device_bytes = s->dev_bytes;
  return LMS_OK;
}

lms_status lms_stream_reserve(lms_stream* s, int64_t n_rows, int32_t host_input) {
  if (!s || n_rows < 0) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->latched != LMS_OK) return s->latched;
  if (s->qs.empty()) return fail(s, LMS_EINVAL, "no query registered");
  LMS_CK(cudaSetDevice(s->cfg.device));
  unsigned long long need = 0;
  for (QueryHost& q : s->qs) need = std::max(need, q.carried + (unsigned long long)n_rows);
  lms_status r = ensure_group_capacity(s, need + 1);
  if (r == LMS_OK && host_input == 1) r = ensure_input(s, (unsigned long long)n_rows);
  if (r == LMS_OK && host_input == 2) {
    if (!s->ist) LMS_CK(cudaStreamCreateWithFlags(&s->ist, cudaStreamNonBlocking));
    r = ensure_ring(s, (unsigned long long)n_rows);
  }
  if (r == LMS_OK) LMS_CK(cudaStreamSynchronize(s->st));
  return r;
}

lms_status lms_stream_push_bytes(lms_stream* s, int64_t n_rows, int32_t host_input,
                                 uint64_t* bytes) {
  if (!s || n_rows < 0 || !bytes) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  unsigned long long need = 0, total = 0;
  for (const QueryHost& q : s->qs) need = std::max(need, q.carried + (unsigned long long)n_rows);
  need += 1;
  const unsigned long long nc = round_cap(need);
  for (const QueryHost& q : s->qs)
    if (q.cap < need) total += nc * (2 * sizeof(Grp) + 8);
  if (s->scr.cap < need) total += nc * (8 + 8 + 4 + 4) + (nc + 1) * (4 + 8);
  if (host_input && s->in_cap < (unsigned long long)n_rows) {
    const unsigned long long ic = round_cap((unsigned long long)n_rows);
    total += ic * (8 + 4 + 4 + (s->cfg.has_type ? 1 : 0));
  }
  // emission buffers a first push allocates (later growth follows the rows
  // a batch emits and is not predicted here)
  if (s->scr.item_cap == 0) total += 1024ull * (8 + 4 + 8 + 8 * kMaxItemWindows + 4 * kUnitBnd);
  for (const QueryHost& q : s->qs)
    if (q.rows_cap == 0) total += round_cap(4096 + 4096 / 4) * sizeof(lms_result_row);
  *bytes = total;
  return LMS_OK;
}

lms_status lms_stream_device_bytes(lms_stream* s, uint64_t* bytes) {
  if (!s || !bytes) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *bytes = s->dev_bytes;
  return LMS_OK;
}

lms_status lms_stream_admissible_rows(lms_stream* s, int32_t host_input, int64_t* n_out) {
  if (!s || !n_out) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  const unsigned long long cap = s->cfg.state_cap_bytes;
  if (cap == 0) {
    *n_out = -1;
    return LMS_OK;
  }
  // bytes per group of capacity: parts + pkeys + state per query; the shared
  // sort keys/values and pane index; the input copy of a host push
  const unsigned long long nq = s->qs.size();
  const unsigned long long per_q = sizeof(Grp) + 8 + sizeof(Grp);
  const unsigned long long per_scr = 8 + 8 + 4 + 4 + 4 + 8;
  const unsigned long long per_in = host_input ? (8 + 4 + 4 + (s->cfg.has_type ? 1 : 0)) : 0;
  unsigned long long carried = 0, qcap = 0;
  for (const QueryHost& q : s->qs) {
    carried = std::max(carried, q.carried);
    qcap = std::max(qcap, q.cap);
  }
  const unsigned long long grown = nq * qcap * per_q + s->scr.cap * per_scr + 16 +
                                   s->in_cap * (8 + 4 + 4 + (s->cfg.has_type ? 1 : 0));
  const unsigned long long other = s->dev_bytes > grown ? s->dev_bytes - grown : 0;
  // keep room for result rows, window lists and merge scratch growing
  const unsigned long long reserve = std::max<unsigned long long>(cap / 16, 64ull << 20);
  long long best = 0;
  for (unsigned long long c = 1ull << 12; c <= (1ull << 34); c <<= 1) {
    const unsigned long long total = other + nq * c * per_q + c * per_scr + 16 + c * per_in;
    // a buffer is grown by allocating the new one before freeing the old
    const unsigned long long peak = total + c * sizeof(Grp);
    if (peak + reserve > cap) break;
    if (c > carried + 1) best = std::max<long long>(best, (long long)(c - carried - 1));
  }
  *n_out = best;
  return LMS_OK;
}

lms_status lms_query_stats(lms_stream* s, int32_t query_id, lms_query_stats_t* out) {
  if (!s || !out) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (query_id < 0 || query_id >= (int)s->qs.size() || s->qs[query_id].hidden)
    return fail(s, LMS_EINVAL, "bad query id");
  const QueryHost& q = s->qs[query_id];
  out->sort_ms = q.sort_ms;
  out->emit_count_ms = q.emit_count_ms;
  out->emit_write_ms = q.emit_write_ms;
  out->rows_emitted = q.rows_emitted;
  out->state_groups = q.carried;
  return LMS_OK;
}

lms_status lms_stream_set_batch_max_ts(lms_stream* s, int64_t ts) {
  if (!s) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->ts_hint = (long long)ts;
  s->ts_hint_set = true;
  return LMS_OK;
}

lms_status lms_stream_set_origin(lms_stream* s, int64_t origin_ts) {
  if (!s) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->origin_set || s->stats.batches > 0 || s->ring_first_set)
    return fail(s, LMS_EINVAL, "the event-time origin is already set");
  s->cfg.origin_ts = (long long)origin_ts;
  return LMS_OK;
}

const char* lms_last_error(lms_stream* s) { return s ? s->err.c_str() : "null stream"; }

lms_status stream_close(lms_stream* s) {
  if (!s) return LMS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    cudaSetDevice(s->cfg.device);
    if (s->st) cudaStreamSynchronize(s->st);
    if (s->ist) cudaStreamSynchronize(s->ist);
    for (const lms_stream::Copy& c : s->copies) cudaEventDestroy(c.ev);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    cudaFreeHost(s->h_ts);
    cudaFreeHost(s->h_key);
    cudaFreeHost(s->h_val);
    cudaFreeHost(s->h_type);
    if (s->ist) cudaStreamDestroy(s->ist);
    for (auto& a : s->allocs) cudaFree(a.first);
    s->allocs.clear();
    for (GraphSlot& g : s->graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    for (int i = 0; i < 8; ++i)
      if (s->ev[i]) cudaEventDestroy(s->ev[i]);
    for (int i = 0; i < 2; ++i)
      if (s->tev[i]) cudaEventDestroy(s->tev[i]);
    for (int i = 0; i < kMaxQueries; ++i)
      for (int j = 0; j < 6; ++j)
        if (s->qev[i][j]) cudaEventDestroy(s->qev[i][j]);
    if (s->own_stream && s->st) cudaStreamDestroy(s->st);
  }
  delete s;
  return LMS_OK;
}

}  // extern "C"

// ---- snapshot / resume -------------------------------------------------------

namespace {

constexpr char kSnapMagic[8] = {'L', 'M', 'S', 'S', 'N', 'A', 'P', '\0'};
constexpr uint32_t kSnapVersion = 1;

struct SnapHead {
  char magic[8];
  uint32_t version;
  uint32_t cfg_bytes, spec_bytes, join_spec_bytes, ctl_bytes, jctl_bytes, grp_bytes, row_bytes;
  uint32_t nq, nj;
  int32_t origin_set, eos_seen;
  int64_t origin_ts, wm;
  SCtl sctl;
  lms_stats stats;
  lms_stream_config cfg;
};
struct SnapQuery {
  lms_query_spec spec;
  int32_t hidden, pad;
  QCtl ctl;
  uint64_t groups, rows, rows_emitted;
};
struct SnapJoin {
  lms_join_spec spec;
  int32_t ql, qr;
  JCtl ctl;
  uint64_t rows, rows_emitted;
};

// Bounded writer/reader over a host buffer.
struct SnapOut {
  unsigned char* p;
  size_t cap, off;
  unsigned char* take(size_t n) {
    unsigned char* r = (p && off + n <= cap) ? p + off : nullptr;
    off += n;
    return r;
  }
};
struct SnapIn {
  const unsigned char* p;
  size_t size, off;
  const unsigned char* take(size_t n) {
    if (n > size - off) return nullptr;
    const unsigned char* r = p + off;
    off += n;
    return r;
  }
};

}  // namespace

extern "C" {

lms_status lms_stream_snapshot(lms_stream* s, void* buf, size_t cap, size_t* size) {
  if (!s || !size) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->latched != LMS_OK) return s->latched;
  if (s->ring_tail != s->ring_head)
    return fail(s, LMS_EINVAL, "snapshot: ingested rows are pending");
  LMS_CK(cudaSetDevice(s->cfg.device));
  const int nq = (int)s->qs.size(), nj = (int)s->joins.size();
  std::vector<QCtl> hc((size_t)nq);
  std::vector<JCtl> jc((size_t)nj);
  SCtl hs{};
  if (nq) LMS_CK(cudaMemcpyAsync(hc.data(), s->qctl, sizeof(QCtl) * nq, cudaMemcpyDeviceToHost, s->st));
  for (int j = 0; j < nj; ++j)
    LMS_CK(cudaMemcpyAsync(&jc[j], s->joins[j].jc, sizeof(JCtl), cudaMemcpyDeviceToHost, s->st));
  LMS_CK(cudaMemcpyAsync(&hs, s->sctl, sizeof(hs), cudaMemcpyDeviceToHost, s->st));
  LMS_CK(cudaStreamSynchronize(s->st));
  size_t need = sizeof(SnapHead);
  for (int i = 0; i < nq; ++i)
    need += sizeof(SnapQuery) + hc[i].carried * sizeof(Grp) +
            (s->qs[i].row_base - s->qs[i].rows_read) * sizeof(ResultRowDev);
  for (int j = 0; j < nj; ++j)
    need += sizeof(SnapJoin) + (s->joins[j].row_base - s->joins[j].rows_read) * sizeof(JoinRowDev);
  *size = need;
  if (!buf) return LMS_OK;
  if (cap < need) return fail(s, LMS_EINVAL, "snapshot: buffer too small");
  SnapOut o{static_cast<unsigned char*>(buf), cap, 0};
  SnapHead h{};
  std::memcpy(h.magic, kSnapMagic, sizeof(kSnapMagic));
  h.version = kSnapVersion;
  h.cfg_bytes = sizeof(lms_stream_config);
  h.spec_bytes = sizeof(lms_query_spec);
  h.join_spec_bytes = sizeof(lms_join_spec);
  h.ctl_bytes = sizeof(QCtl);
  h.jctl_bytes = sizeof(JCtl);
  h.grp_bytes = sizeof(Grp);
  h.row_bytes = sizeof(ResultRowDev);
  h.nq = (uint32_t)nq;
  h.nj = (uint32_t)nj;
  h.origin_set = s->origin_set ? 1 : 0;
  h.eos_seen = s->eos_seen ? 1 : 0;
  h.origin_ts = s->origin_ts;
  h.wm = s->wm;
  h.sctl = hs;
  h.stats = s->stats;
  h.cfg = s->cfg;
  h.cfg.cuda_stream = nullptr;
  std::memcpy(o.take(sizeof(h)), &h, sizeof(h));
  for (int i = 0; i < nq; ++i) {
    const QueryHost& q = s->qs[i];
    SnapQuery sq{};
    sq.spec = q.spec;
    sq.hidden = q.hidden ? 1 : 0;
    sq.ctl = hc[i];
    sq.groups = hc[i].carried;
    sq.rows = q.row_base - q.rows_read;
    sq.rows_emitted = q.rows_emitted;
    sq.ctl.row_base = sq.rows;
    std::memcpy(o.take(sizeof(sq)), &sq, sizeof(sq));
    if (sq.groups)
      LMS_CK(cudaMemcpyAsync(o.take(sq.groups * sizeof(Grp)), q.dev.parts, sq.groups * sizeof(Grp),
                             cudaMemcpyDeviceToHost, s->st));
    if (sq.rows)
      LMS_CK(cudaMemcpyAsync(o.take(sq.rows * sizeof(ResultRowDev)), q.rows + q.rows_read,
                             sq.rows * sizeof(ResultRowDev), cudaMemcpyDeviceToHost, s->st));
  }
  for (int j = 0; j < nj; ++j) {
    const JoinHost& jh = s->joins[j];
    SnapJoin sj{};
    sj.spec = jh.spec;
    sj.ql = jh.ql;
    sj.qr = jh.qr;
    sj.ctl = jc[j];
    sj.rows = jh.row_base - jh.rows_read;
    sj.rows_emitted = jh.rows_emitted;
    sj.ctl.row_base = sj.rows;
    std::memcpy(o.take(sizeof(sj)), &sj, sizeof(sj));
    if (sj.rows)
      LMS_CK(cudaMemcpyAsync(o.take(sj.rows * sizeof(JoinRowDev)), jh.rows + jh.rows_read,
                             sj.rows * sizeof(JoinRowDev), cudaMemcpyDeviceToHost, s->st));
  }
  LMS_CK(cudaStreamSynchronize(s->st));
  return LMS_OK;
}

lms_status lms_stream_get_config(lms_stream* s, lms_stream_config* out) {
  if (!s || !out) return LMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->cfg;
  if (s->origin_set) out->origin_ts = s->origin_ts;
  out->cuda_stream = s->st;
  return LMS_OK;
}

lms_status lms_stream_restore(const void* buf, size_t size, int32_t device, lms_stream** out) {
  if (!buf || !out) return LMS_EINVAL;
  *out = nullptr;
  SnapIn in{static_cast<const unsigned char*>(buf), size, 0};
  const unsigned char* hp = in.take(sizeof(SnapHead));
  if (!hp) return LMS_EINVAL;
  SnapHead h;
  std::memcpy(&h, hp, sizeof(h));
  if (std::memcmp(h.magic, kSnapMagic, sizeof(kSnapMagic)) != 0 || h.version != kSnapVersion ||
      h.cfg_bytes != sizeof(lms_stream_config) || h.spec_bytes != sizeof(lms_query_spec) ||
      h.join_spec_bytes != sizeof(lms_join_spec) || h.ctl_bytes != sizeof(QCtl) ||
      h.jctl_bytes != sizeof(JCtl) || h.grp_bytes != sizeof(Grp) ||
      h.row_bytes != sizeof(ResultRowDev) || h.nq > (uint32_t)kMaxQueries || h.nj > 4)
    return LMS_EINVAL;
  // walk the buffer once to find every record (and check that it is complete)
  std::vector<SnapQuery> sq(h.nq);
  std::vector<const unsigned char*> q_groups(h.nq), q_rows(h.nq);
  for (uint32_t i = 0; i < h.nq; ++i) {
    const unsigned char* p = in.take(sizeof(SnapQuery));
    if (!p) return LMS_EINVAL;
    std::memcpy(&sq[i], p, sizeof(SnapQuery));
    if (sq[i].groups > (1ull << 40) || sq[i].rows > (1ull << 40)) return LMS_EINVAL;
    q_groups[i] = in.take(sq[i].groups * sizeof(Grp));
    q_rows[i] = in.take(sq[i].rows * sizeof(ResultRowDev));
    if ((sq[i].groups && !q_groups[i]) || (sq[i].rows && !q_rows[i])) return LMS_EINVAL;
  }
  std::vector<SnapJoin> sj(h.nj);
  std::vector<const unsigned char*> j_rows(h.nj);
  for (uint32_t j = 0; j < h.nj; ++j) {
    const unsigned char* p = in.take(sizeof(SnapJoin));
    if (!p) return LMS_EINVAL;
    std::memcpy(&sj[j], p, sizeof(SnapJoin));
    if (sj[j].rows > (1ull << 40) || sj[j].ql < 0 || sj[j].qr != sj[j].ql + 1 ||
        sj[j].qr >= (int32_t)h.nq)
      return LMS_EINVAL;
    j_rows[j] = in.take(sj[j].rows * sizeof(JoinRowDev));
    if (sj[j].rows && !j_rows[j]) return LMS_EINVAL;
  }
  if (in.off != size) return LMS_EINVAL;
  lms_stream_config cfg = h.cfg;
  cfg.cuda_stream = nullptr;
  if (device >= 0) cfg.device = device;
  lms_stream* s = nullptr;
  lms_status r = stream_open(&cfg, &s);
  if (r != LMS_OK) return r;
  auto bail = [&](lms_status code) {
    stream_close(s);
    return code;
  };
  // registrations in their original order: a join's two hidden side queries
  // are consecutive and created by registering the join
  for (uint32_t i = 0; i < h.nq; ++i) {
    int jfound = -1;
    for (uint32_t j = 0; j < h.nj; ++j)
      if (sj[j].ql == (int32_t)i) jfound = (int)j;
    int32_t id = -1;
    if (jfound >= 0) {
      if (!sq[i].hidden || !sq[i + 1].hidden) return bail(LMS_EINVAL);
      if ((r = lms_join_register(s, &sj[jfound].spec, &id)) != LMS_OK) return bail(r);
      if (id != jfound || s->joins[id].ql != (int)i) return bail(LMS_EINVAL);
      ++i;
    } else {
      if (sq[i].hidden) return bail(LMS_EINVAL);
      if ((r = query_register(s, &sq[i].spec, &id)) != LMS_OK) return bail(r);
      if (id != (int32_t)i) return bail(LMS_EINVAL);
    }
  }
  if ((int)s->joins.size() != (int)h.nj) return bail(LMS_EINVAL);
  // (s is not visible to any other thread yet; the copies below run on s->st,
  // after the registrations' own copies have completed)
  if (cudaSetDevice(s->cfg.device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return bail(LMS_ECUDA);
  if (h.origin_set) set_origin(s, h.origin_ts);
  s->eos_seen = h.eos_seen != 0;
  s->wm = h.wm;
  unsigned long long need = 0;
  for (uint32_t i = 0; i < h.nq; ++i) need = std::max<unsigned long long>(need, sq[i].groups);
  if ((r = ensure_group_capacity(s, need + 1)) != LMS_OK) return bail(r);
  std::vector<unsigned long long> gk;
  for (uint32_t i = 0; i < h.nq; ++i) {
    QueryHost& q = s->qs[i];
    const SnapQuery& x = sq[i];
    if ((r = ensure_rows(s, q, x.rows + 4096)) != LMS_OK) return bail(r);
    if (x.groups) {
      gk.resize(x.groups);
      for (unsigned long long g = 0; g < x.groups; ++g)
        std::memcpy(&gk[g], q_groups[i] + g * sizeof(Grp), sizeof(unsigned long long));
      if (cudaMemcpyAsync(q.dev.parts, q_groups[i], x.groups * sizeof(Grp),
                          cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
          cudaMemcpyAsync(q.dev.pkeys, gk.data(), x.groups * 8, cudaMemcpyHostToDevice,
                          s->st) != cudaSuccess)
        return bail(LMS_ECUDA);
    }
    if (x.rows && cudaMemcpyAsync(q.rows, q_rows[i], x.rows * sizeof(ResultRowDev),
                                  cudaMemcpyHostToDevice, s->st) != cudaSuccess)
      return bail(LMS_ECUDA);
    QCtl c = x.ctl;
    c.err = 0u;
    if (cudaMemcpyAsync(q.dev.ctl, &c, sizeof(c), cudaMemcpyHostToDevice, s->st) != cudaSuccess)
      return bail(LMS_ECUDA);
    q.row_base = x.rows;
    q.rows_read = 0;
    q.carried = x.groups;
    q.n_state = c.n_state;
    q.late_rows = c.late_rows;
    q.range_rows = c.range_rows;
    q.rows_emitted = x.rows_emitted;
  }
  for (uint32_t j = 0; j < h.nj; ++j) {
    JoinHost& jh = s->joins[j];
    const SnapJoin& x = sj[j];
    if ((r = ensure_join_rows(s, jh, x.rows + 4096)) != LMS_OK) return bail(r);
    if (x.rows && cudaMemcpyAsync(jh.rows, j_rows[j], x.rows * sizeof(JoinRowDev),
                                  cudaMemcpyHostToDevice, s->st) != cudaSuccess)
      return bail(LMS_ECUDA);
    JCtl c = x.ctl;
    c.err = 0u;
    if (cudaMemcpyAsync(jh.jc, &c, sizeof(c), cudaMemcpyHostToDevice, s->st) != cudaSuccess)
      return bail(LMS_ECUDA);
    jh.row_base = x.rows;
    jh.rows_read = 0;
    jh.rows_emitted = x.rows_emitted;
  }
  SCtl sc = h.sctl;
  sc.batch_max_ts = LLONG_MIN;
  if (cudaMemcpyAsync(s->sctl, &sc, sizeof(sc), cudaMemcpyHostToDevice, s->st) != cudaSuccess)
    return bail(LMS_ECUDA);
  s->stats = h.stats;
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return bail(LMS_ECUDA);
  *out = s;
  return LMS_OK;
}

}  // extern "C"
