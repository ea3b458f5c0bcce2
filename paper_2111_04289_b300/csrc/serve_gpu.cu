// The engine as the serving loop's backend.
//
// Each admitted micro-batch is cut from the synthetic load: the key and value
// columns are a slice of a pool drawn once at creation (consecutive events
// take consecutive pool entries), and a kernel writes the batch's ts column
// for the ticks the loop admitted — all outside the measured time.  In host
// mode the columns live in pinned host memory and the batch is processed as a
// serving client would: one push_microbatch from those host buffers (the
// host-to-device copy is inside the measured time) followed by poll_results of
// every emitted row into pinned host memory.  In device mode the columns are
// already in HBM (push reads them in place) and the rows are still polled to
// the host.  In ingest mode the columns are in pinned host memory too, but
// every tick is handed to lms_ingest when it arrives (its ts written into a
// pinned ts pool indexed like the key/value pool), so its host-to-device copy
// runs on the stream's side stream while the data waits for admission; each
// micro-batch is then lms_push_ingested + polls.  The processing time is the
// wall time of push + polls.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/lmstream.h"
#include "lms_internal.h"

using namespace lms;

namespace {
constexpr long long kPool = 1ll << 26;  // distinct events of the load before it repeats
}

struct lms_serve_gpu {
  lms_stream* s = nullptr;
  int nq = 0;
  int dev = 0;
  int sms = 148;
  bool device_input = false;
  bool ingest = false;
  long long* ts_pool = nullptr;   // ingest mode: pinned ts of event c at c mod kPool
  long long* m_ts_pool = nullptr; // its device-side address
  long long ingested = 0, pushed = 0;
  cudaStream_t gen_st = nullptr;
  unsigned long long seed = 0;
  unsigned n_keys = 0;
  double* d_cdf = nullptr;
  long long max_rows = 0;
  // columns: ts [max_rows]; key / value pool [kPool + max_rows]
  long long* ts = nullptr;
  unsigned* key = nullptr;
  float* val = nullptr;
  long long* m_ts = nullptr;  // device-side address of ts (mapped, in host mode)
  GenChunk* h_chunks = nullptr;  // pinned staging of the chunk table
  GenChunk* d_chunks = nullptr;
  int chunk_cap = 0;
  lms_result_row* h_rows = nullptr;
  size_t rows_cap = 0;
  unsigned long long rows_polled = 0;
  bool keep_rows = false;
  std::vector<std::vector<lms_result_row>> kept;  // per query, when keep_rows
};

namespace {

void free_col(lms_serve_gpu* g, void* p) {
  if (!p) return;
  if (g->device_input) cudaFree(p);
  else cudaFreeHost(p);
}

void destroy(lms_serve_gpu* g) {
  if (!g) return;
  if (g->s) stream_close(g->s);
  cudaSetDevice(g->dev);
  if (g->gen_st) cudaStreamDestroy(g->gen_st);
  cudaFree(g->d_cdf);
  cudaFree(g->d_chunks);
  free_col(g, g->ts);
  free_col(g, g->key);
  free_col(g, g->val);
  cudaFreeHost(g->ts_pool);
  cudaFreeHost(g->h_chunks);
  cudaFreeHost(g->h_rows);
  delete g;
}

// Writes the batch's ts column; returns the pool offset of its first event.
lms_status make_batch(lms_serve_gpu* g, const lms_serve_chunk* chunks, int32_t n_chunks,
                      int64_t n_events, long long* pool_off) {
  if (n_events > g->max_rows || n_chunks <= 0) return LMS_EINVAL;
  if (cudaSetDevice(g->dev) != cudaSuccess) return LMS_ECUDA;
  if (n_chunks > g->chunk_cap) {
    cudaFree(g->d_chunks);
    cudaFreeHost(g->h_chunks);
    g->d_chunks = nullptr;
    g->h_chunks = nullptr;
    g->chunk_cap = 0;
    const int cap = n_chunks * 2;
    if (cudaMalloc(&g->d_chunks, sizeof(GenChunk) * cap) != cudaSuccess ||
        cudaHostAlloc(&g->h_chunks, sizeof(GenChunk) * cap, cudaHostAllocDefault) != cudaSuccess)
      return LMS_ENOMEM;
    g->chunk_cap = cap;
  }
  long long off = 0;
  for (int i = 0; i < n_chunks; ++i) {
    const lms_serve_chunk& c = chunks[i];
    // the batch's events must be consecutive in the stream
    if (i > 0 && c.first_event + c.j_begin != chunks[i - 1].first_event + chunks[i - 1].j_end)
      return LMS_EINVAL;
    g->h_chunks[i] = {c.t0_ms, c.width_ms, c.n_total, c.j_begin, c.first_event, off};
    off += c.j_end - c.j_begin;
  }
  if (off != n_events) return LMS_EINVAL;
  *pool_off = (chunks[0].first_event + chunks[0].j_begin) % kPool;
  if (cudaMemcpyAsync(g->d_chunks, g->h_chunks, sizeof(GenChunk) * n_chunks,
                      cudaMemcpyHostToDevice, g->gen_st) != cudaSuccess ||
      launch_gen_ts(g->d_chunks, n_chunks, n_events, g->m_ts, g->sms, g->gen_st) != cudaSuccess ||
      cudaStreamSynchronize(g->gen_st) != cudaSuccess)
    return LMS_ECUDA;
  return LMS_OK;
}

// Ingest mode: a tick became visible; its ts go to the ts pool (not measured)
// and its rows to lms_ingest.
int32_t arrive(void* ctx, const lms_serve_chunk* t) {
  lms_serve_gpu* g = static_cast<lms_serve_gpu*>(ctx);
  const long long n = t->j_end - t->j_begin;
  // rows ingested and not pushed must keep their ts pool slots
  if (n <= 0 || n > g->max_rows || g->ingested + n - g->pushed > kPool) return -1;
  const long long pos = (t->first_event + t->j_begin) % kPool;
  if (cudaSetDevice(g->dev) != cudaSuccess) return -1;
  g->h_chunks[0] = {t->t0_ms, t->width_ms, t->n_total, t->j_begin, t->first_event, 0};
  if (cudaMemcpyAsync(g->d_chunks, g->h_chunks, sizeof(GenChunk), cudaMemcpyHostToDevice,
                      g->gen_st) != cudaSuccess ||
      launch_gen_ts(g->d_chunks, 1, n, g->m_ts_pool + pos, g->sms, g->gen_st) != cudaSuccess ||
      cudaStreamSynchronize(g->gen_st) != cudaSuccess)
    return -1;
  lms_batch b{};
  b.n_rows = n;
  b.ts = reinterpret_cast<const int64_t*>(g->ts_pool + pos);
  b.key = g->key + pos;
  b.value = g->val + pos;
  b.memory = LMS_MEM_HOST;
  b.flags = LMS_INGEST_STABLE;
  if (lms_ingest(g->s, &b) != LMS_OK) return -1;
  g->ingested += n;
  return 0;
}

double process(void* ctx, const lms_serve_chunk* chunks, int32_t n_chunks, int64_t n_events,
               lms_serve_batch* rec) {
  lms_serve_gpu* g = static_cast<lms_serve_gpu*>(ctx);
  long long off = 0;
  // make the batch (not measured; in ingest mode its rows are already ingested)
  if (!g->ingest && make_batch(g, chunks, n_chunks, n_events, &off) != LMS_OK) return -1.0;
  lms_stats before{}, after{};
  lms_stream_stats(g->s, &before);
  // process it as a client would: push, then poll every row to the host
  const auto t0 = std::chrono::steady_clock::now();
  if (g->ingest) {
    if (lms_push_ingested(g->s, n_events, 0u) != LMS_OK) return -1.0;
    g->pushed += n_events;
  } else {
    lms_batch b{};
    b.n_rows = n_events;
    b.ts = reinterpret_cast<const int64_t*>(g->ts);
    b.key = g->key + off;
    b.value = g->val + off;
    b.memory = g->device_input ? LMS_MEM_DEVICE : LMS_MEM_HOST;
    if (push_microbatch(g->s, &b) != LMS_OK) return -1.0;
  }
  unsigned long long rows = 0;
  for (int q = 0; q < g->nq; ++q) {
    for (;;) {
      size_t got = 0;
      const lms_status st = poll_results(g->s, q, g->h_rows, g->rows_cap, &got, 0);
      if (st == LMS_EAGAIN) break;
      if (st != LMS_OK) return -1.0;
      rows += got;
      if (g->keep_rows) g->kept[q].insert(g->kept[q].end(), g->h_rows, g->h_rows + got);
    }
  }
  const double ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  lms_stream_stats(g->s, &after);
  g->rows_polled += rows;
  rec->h2d_ms = after.h2d_ms - before.h2d_ms;
  rec->k1_ms = after.k1_ms - before.k1_ms;
  rec->sort_ms = after.sort_ms - before.sort_ms;
  rec->emit_ms = after.emit_ms - before.emit_ms;
  rec->state_groups_before = before.state_groups;
  rec->rows_out = rows;
  return ms;
}

int64_t admissible(void* ctx) {
  lms_serve_gpu* g = static_cast<lms_serve_gpu*>(ctx);
  int64_t n = -1;
  if (lms_stream_admissible_rows(g->s, g->device_input ? 0 : 1, &n) != LMS_OK) return 0;
  if (n < 0 || n > g->max_rows) n = g->max_rows;
  return n;
}

cudaError_t alloc_col(lms_serve_gpu* g, void** p, size_t bytes) {
  if (g->device_input) return cudaMalloc(p, bytes);
  return cudaHostAlloc(p, bytes, cudaHostAllocMapped);
}

}  // namespace

extern "C" {

lms_status lms_serve_gpu_create(const lms_stream_config* cfg, const lms_query_spec* qs,
                                int32_t nq, uint64_t seed, uint32_t n_keys, double zipf_s,
                                int64_t max_batch_rows, int32_t flags, lms_serve_gpu** out) {
  if (!cfg || !qs || nq < 1 || !out || n_keys < 1 || !(zipf_s > 0) || max_batch_rows < 1 ||
      max_batch_rows > kPool || cfg->value_type != LMS_VALUE_FLOAT32 || cfg->has_type)
    return LMS_EINVAL;
  lms_serve_gpu* g = new lms_serve_gpu();
  g->dev = cfg->device;
  g->seed = seed;
  g->n_keys = n_keys;
  g->max_rows = max_batch_rows;
  g->nq = nq;
  g->keep_rows = (flags & LMS_SERVE_KEEP_ROWS) != 0;
  g->device_input = (flags & LMS_SERVE_DEVICE_INPUT) != 0;
  g->ingest = !g->device_input && (flags & LMS_SERVE_INGEST) != 0;
  g->kept.resize(nq);
  lms_status r = stream_open(cfg, &g->s);
  if (r != LMS_OK) {
    g->s = nullptr;
    destroy(g);
    return r;
  }
  for (int i = 0; i < nq; ++i) {
    int32_t id = 0;
    if ((r = query_register(g->s, &qs[i], &id)) != LMS_OK) {
      destroy(g);
      return r;
    }
  }
  cudaSetDevice(g->dev);
  cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->dev);
  // Zipf CDF over ranks 1..n_keys (rank r -> key r - 1)
  std::vector<double> cdf(n_keys);
  double acc = 0.0;
  for (uint32_t i = 0; i < n_keys; ++i) {
    acc += std::pow((double)(i + 1), -zipf_s);
    cdf[i] = acc;
  }
  for (uint32_t i = 0; i < n_keys; ++i) cdf[i] /= acc;
  cdf[n_keys - 1] = 1.0;
  g->rows_cap = 1u << 22;
  const size_t n = (size_t)max_batch_rows, np = (size_t)(kPool + max_batch_rows);
  if (cudaStreamCreateWithFlags(&g->gen_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&g->d_cdf, sizeof(double) * n_keys) != cudaSuccess ||
      cudaMemcpy(g->d_cdf, cdf.data(), sizeof(double) * n_keys, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      alloc_col(g, (void**)&g->ts, 8 * n) != cudaSuccess ||
      alloc_col(g, (void**)&g->key, 4 * np) != cudaSuccess ||
      alloc_col(g, (void**)&g->val, 4 * np) != cudaSuccess ||
      (g->ingest && cudaHostAlloc((void**)&g->ts_pool, 8 * np, cudaHostAllocMapped) != cudaSuccess) ||
      cudaHostAlloc(&g->h_rows, sizeof(lms_result_row) * g->rows_cap, cudaHostAllocDefault) !=
          cudaSuccess) {
    cudaGetLastError();
    destroy(g);
    return LMS_ENOMEM;
  }
  unsigned* m_key = g->key;
  float* m_val = g->val;
  g->m_ts = g->ts;
  if (!g->device_input &&
      (cudaHostGetDevicePointer((void**)&g->m_ts, g->ts, 0) != cudaSuccess ||
       cudaHostGetDevicePointer((void**)&m_key, g->key, 0) != cudaSuccess ||
       cudaHostGetDevicePointer((void**)&m_val, g->val, 0) != cudaSuccess ||
       (g->ingest && cudaHostGetDevicePointer((void**)&g->m_ts_pool, g->ts_pool, 0) != cudaSuccess))) {
    cudaGetLastError();
    destroy(g);
    return LMS_ECUDA;
  }
  if (launch_gen_pool(seed, g->d_cdf, n_keys, kPool, (long long)np, m_key, m_val, g->sms,
                      g->gen_st) != cudaSuccess ||
      cudaStreamSynchronize(g->gen_st) != cudaSuccess) {
    destroy(g);
    return LMS_ECUDA;
  }
  // Warm-up outside any measurement: a throwaway stream with the same queries
  // runs a small batch (loads every kernel), then the serving stream's
  // buffers are sized for the largest batch its memory cap admits.
  {
    lms_stream_config wc = *cfg;
    wc.state_cap_bytes = 0;
    wc.cuda_stream = nullptr;
    lms_stream* w = nullptr;
    lms_status wr = stream_open(&wc, &w);
    for (int i = 0; wr == LMS_OK && i < nq; ++i) {
      int32_t id = 0;
      wr = query_register(w, &qs[i], &id);
    }
    const int64_t wn = max_batch_rows < 65536 ? max_batch_rows : 65536;
    lms_serve_chunk c{0.0, 10.0, wn, 0, wn, 0};
    long long off = 0;
    if (wr == LMS_OK) wr = make_batch(g, &c, 1, wn, &off);
    for (int rep = 0; wr == LMS_OK && rep < 2; ++rep) {
      lms_batch b{};
      b.n_rows = wn;
      b.ts = reinterpret_cast<const int64_t*>(g->ts);
      b.key = g->key;
      b.value = g->val;
      b.memory = g->device_input ? LMS_MEM_DEVICE : LMS_MEM_HOST;
      b.flags = rep == 1 ? LMS_BATCH_EOS : 0u;
      wr = push_microbatch(w, &b);
    }
    if (w) stream_close(w);
    // let the autotuner settle every size class a batch can have, so that no
    // measured batch runs a variant under trial
    for (int c = 15; wr == LMS_OK && cfg->k1_variant == 0 && (1ll << c) <= max_batch_rows; ++c) {
      const int64_t rows = 1ll << c;
      if (lms_k1_tuned_variant(cfg->value_type, nq, rows) != 0) continue;
      lms_stream* t = nullptr;
      wr = stream_open(&wc, &t);
      for (int i = 0; wr == LMS_OK && i < nq; ++i) {
        int32_t id = 0;
        wr = query_register(t, &qs[i], &id);
      }
      for (int rep = 0; wr == LMS_OK && rep < 16 && lms_k1_tuned_variant(cfg->value_type, nq, rows) == 0;
           ++rep) {
        lms_serve_chunk tc{(double)rep * 100.0, 100.0, rows, 0, rows, (int64_t)rep * rows};
        long long toff = 0;
        if ((wr = make_batch(g, &tc, 1, rows, &toff)) != LMS_OK) break;
        lms_batch b{};
        b.n_rows = rows;
        b.ts = reinterpret_cast<const int64_t*>(g->ts);
        b.key = g->key + toff;
        b.value = g->val + toff;
        b.memory = g->device_input ? LMS_MEM_DEVICE : LMS_MEM_HOST;
        wr = push_microbatch(t, &b);
        for (int q = 0; wr == LMS_OK && q < nq; ++q) wr = lms_results_discard(t, q);
      }
      if (t) stream_close(t);
    }
    int64_t adm = -1;
    if (wr == LMS_OK) wr = lms_stream_admissible_rows(g->s, g->device_input ? 0 : 1, &adm);
    const int64_t res = (adm < 0 || adm > max_batch_rows) ? max_batch_rows : adm;
    if (wr == LMS_OK) wr = lms_stream_reserve(g->s, res, g->device_input ? 0 : g->ingest ? 2 : 1);
    // the chunk table of one tick (arrive() in ingest mode)
    if (wr == LMS_OK && g->chunk_cap < 1) {
      if (cudaMalloc(&g->d_chunks, sizeof(GenChunk) * 2) != cudaSuccess ||
          cudaHostAlloc(&g->h_chunks, sizeof(GenChunk) * 2, cudaHostAllocDefault) != cudaSuccess)
        wr = LMS_ENOMEM;
      else
        g->chunk_cap = 2;
    }
    if (wr != LMS_OK) {
      destroy(g);
      return wr;
    }
  }
  *out = g;
  return LMS_OK;
}

lms_status lms_serve_gpu_backend(lms_serve_gpu* g, lms_serve_backend* out) {
  if (!g || !out) return LMS_EINVAL;
  out->ctx = g;
  out->process = process;
  out->admissible_rows = admissible;
  out->arrive = g->ingest ? arrive : nullptr;
  return LMS_OK;
}

lms_stream* lms_serve_gpu_stream(lms_serve_gpu* g) { return g ? g->s : nullptr; }

int32_t lms_serve_gpu_device_input(const lms_serve_gpu* g) {
  return (g && g->device_input) ? 1 : 0;
}

lms_status lms_serve_gpu_prefill(lms_serve_gpu* g, double t0_ms, double span_ms,
                                 int32_t n_batches, int64_t events_per_batch) {
  if (!g || n_batches < 1 || events_per_batch < 1 || events_per_batch > g->max_rows ||
      !(span_ms > 0))
    return LMS_EINVAL;
  if (cudaSetDevice(g->dev) != cudaSuccess) return LMS_ECUDA;
  const double w = span_ms / n_batches;
  for (int b = 0; b < n_batches; ++b) {
    const long long first = (long long)b * events_per_batch;
    g->h_chunks[0] = {t0_ms + b * w, w, events_per_batch, 0, first, 0};
    if (cudaMemcpyAsync(g->d_chunks, g->h_chunks, sizeof(GenChunk), cudaMemcpyHostToDevice,
                        g->gen_st) != cudaSuccess ||
        launch_gen_ts(g->d_chunks, 1, events_per_batch, g->m_ts, g->sms, g->gen_st) !=
            cudaSuccess ||
        cudaStreamSynchronize(g->gen_st) != cudaSuccess)
      return LMS_ECUDA;
    const long long off = first % kPool;
    lms_batch bt{};
    bt.n_rows = events_per_batch;
    bt.ts = reinterpret_cast<const int64_t*>(g->ts);
    bt.key = g->key + off;
    bt.value = g->val + off;
    bt.memory = g->device_input ? LMS_MEM_DEVICE : LMS_MEM_HOST;
    lms_status r = push_microbatch(g->s, &bt);
    if (r != LMS_OK) return r;
    for (int q = 0; q < g->nq; ++q)
      if ((r = lms_results_discard(g->s, q)) != LMS_OK) return r;
  }
  return LMS_OK;
}

lms_status lms_serve_gpu_generate(lms_serve_gpu* g, const lms_serve_chunk* chunks,
                                  int32_t n_chunks, int64_t n_events, int64_t* ts,
                                  uint32_t* key, float* value) {
  if (!g || !chunks || n_events < 0 || (n_events > 0 && (!ts || !key || !value)))
    return LMS_EINVAL;
  long long off = 0;
  const lms_status r = make_batch(g, chunks, n_chunks, n_events, &off);
  if (r != LMS_OK) return r;
  const cudaMemcpyKind k = g->device_input ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  if (cudaMemcpy(ts, g->ts, 8 * (size_t)n_events, k) != cudaSuccess ||
      cudaMemcpy(key, g->key + off, 4 * (size_t)n_events, k) != cudaSuccess ||
      cudaMemcpy(value, g->val + off, 4 * (size_t)n_events, k) != cudaSuccess)
    return LMS_ECUDA;
  return LMS_OK;
}

lms_status lms_serve_gpu_kept_rows(lms_serve_gpu* g, int32_t query_id, lms_result_row* out,
                                   size_t cap, size_t* n_out) {
  if (!g || !n_out || query_id < 0 || query_id >= g->nq || (cap && !out)) return LMS_EINVAL;
  const std::vector<lms_result_row>& v = g->kept[query_id];
  if (!out) {
    *n_out = v.size();
    return LMS_OK;
  }
  const size_t m = v.size() < cap ? v.size() : cap;
  std::memcpy(out, v.data(), m * sizeof(lms_result_row));
  *n_out = m;
  return LMS_OK;
}

void lms_serve_gpu_destroy(lms_serve_gpu* g) { destroy(g); }

}  // extern "C"
