// The engine as the serving loop's backend.
//
// Each admitted micro-batch is made by the synthetic load generator (a kernel
// that writes the batch's columns straight into pinned host memory, outside
// the measured time), then processed the way a serving client would: one
// push_microbatch from those host buffers (the host-to-device copy is inside
// the measured time) followed by poll_results of every emitted row into a
// pinned host buffer.  The processing time is the wall time of push + polls.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/lmstream.h"
#include "lms_internal.h"

using namespace lms;

struct lms_serve_gpu {
  lms_stream* s = nullptr;
  int nq = 0;
  int dev = 0;
  int sms = 148;
  cudaStream_t gen_st = nullptr;
  unsigned long long seed = 0;
  unsigned n_keys = 0;
  double* d_cdf = nullptr;
  long long max_rows = 0;
  long long* h_ts = nullptr;  // pinned, mapped
  unsigned* h_key = nullptr;
  float* h_val = nullptr;
  long long* m_ts = nullptr;  // their device-side addresses
  unsigned* m_key = nullptr;
  float* m_val = nullptr;
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

void destroy(lms_serve_gpu* g) {
  if (!g) return;
  if (g->s) stream_close(g->s);
  cudaSetDevice(g->dev);
  if (g->gen_st) cudaStreamDestroy(g->gen_st);
  cudaFree(g->d_cdf);
  cudaFree(g->d_chunks);
  cudaFreeHost(g->h_ts);
  cudaFreeHost(g->h_key);
  cudaFreeHost(g->h_val);
  cudaFreeHost(g->h_chunks);
  cudaFreeHost(g->h_rows);
  delete g;
}

// Writes the batch made of chunks[0 .. n_chunks) into the pinned columns.
lms_status make_batch(lms_serve_gpu* g, const lms_serve_chunk* chunks, int32_t n_chunks,
                      int64_t n_events) {
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
    g->h_chunks[i] = {c.t0_ms, c.width_ms, c.n_total, c.j_begin, c.first_event, off};
    off += c.j_end - c.j_begin;
  }
  if (off != n_events) return LMS_EINVAL;
  if (cudaMemcpyAsync(g->d_chunks, g->h_chunks, sizeof(GenChunk) * n_chunks,
                      cudaMemcpyHostToDevice, g->gen_st) != cudaSuccess ||
      launch_gen_serving(g->d_chunks, n_chunks, n_events, g->seed, g->d_cdf, g->n_keys, g->m_ts,
                         g->m_key, g->m_val, g->sms, g->gen_st) != cudaSuccess ||
      cudaStreamSynchronize(g->gen_st) != cudaSuccess)
    return LMS_ECUDA;
  return LMS_OK;
}

double process(void* ctx, const lms_serve_chunk* chunks, int32_t n_chunks, int64_t n_events,
               lms_serve_batch* rec) {
  lms_serve_gpu* g = static_cast<lms_serve_gpu*>(ctx);
  // make the batch (not measured)
  if (make_batch(g, chunks, n_chunks, n_events) != LMS_OK) return -1.0;
  lms_stats before{}, after{};
  lms_stream_stats(g->s, &before);
  // process it as a client would: push from host memory, poll every row back
  const auto t0 = std::chrono::steady_clock::now();
  lms_batch b{};
  b.n_rows = n_events;
  b.ts = reinterpret_cast<const int64_t*>(g->h_ts);
  b.key = g->h_key;
  b.value = g->h_val;
  b.memory = LMS_MEM_HOST;
  if (push_microbatch(g->s, &b) != LMS_OK) return -1.0;
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
  if (lms_stream_admissible_rows(g->s, 1, &n) != LMS_OK) return 0;
  if (n < 0 || n > g->max_rows) n = g->max_rows;
  return n;
}

}  // namespace

extern "C" {

lms_status lms_serve_gpu_create(const lms_stream_config* cfg, const lms_query_spec* qs,
                                int32_t nq, uint64_t seed, uint32_t n_keys, double zipf_s,
                                int64_t max_batch_rows, int32_t keep_rows,
                                lms_serve_gpu** out) {
  if (!cfg || !qs || nq < 1 || !out || n_keys < 1 || !(zipf_s > 0) || max_batch_rows < 1 ||
      cfg->value_type != LMS_VALUE_FLOAT32 || cfg->has_type)
    return LMS_EINVAL;
  lms_serve_gpu* g = new lms_serve_gpu();
  g->dev = cfg->device;
  g->seed = seed;
  g->n_keys = n_keys;
  g->max_rows = max_batch_rows;
  g->nq = nq;
  g->keep_rows = keep_rows != 0;
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
  const size_t n = (size_t)max_batch_rows;
  if (cudaStreamCreateWithFlags(&g->gen_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&g->d_cdf, sizeof(double) * n_keys) != cudaSuccess ||
      cudaMemcpy(g->d_cdf, cdf.data(), sizeof(double) * n_keys, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaHostAlloc(&g->h_ts, 8 * n, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&g->h_key, 4 * n, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&g->h_val, 4 * n, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&g->h_rows, sizeof(lms_result_row) * g->rows_cap, cudaHostAllocDefault) !=
          cudaSuccess ||
      cudaHostGetDevicePointer((void**)&g->m_ts, g->h_ts, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&g->m_key, g->h_key, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&g->m_val, g->h_val, 0) != cudaSuccess) {
    cudaGetLastError();
    destroy(g);
    return LMS_ENOMEM;
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
    if (wr == LMS_OK) wr = make_batch(g, &c, 1, wn);
    for (int rep = 0; wr == LMS_OK && rep < 2; ++rep) {
      lms_batch b{};
      b.n_rows = wn;
      b.ts = reinterpret_cast<const int64_t*>(g->h_ts);
      b.key = g->h_key;
      b.value = g->h_val;
      b.memory = LMS_MEM_HOST;
      b.flags = rep == 1 ? LMS_BATCH_EOS : 0u;
      wr = push_microbatch(w, &b);
    }
    if (w) stream_close(w);
    int64_t adm = -1;
    if (wr == LMS_OK) wr = lms_stream_admissible_rows(g->s, 1, &adm);
    const int64_t res = (adm < 0 || adm > max_batch_rows) ? max_batch_rows : adm;
    if (wr == LMS_OK) wr = lms_stream_reserve(g->s, res, 1);
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
  return LMS_OK;
}

lms_stream* lms_serve_gpu_stream(lms_serve_gpu* g) { return g ? g->s : nullptr; }

lms_status lms_serve_gpu_generate(lms_serve_gpu* g, const lms_serve_chunk* chunks,
                                  int32_t n_chunks, int64_t n_events, int64_t* ts,
                                  uint32_t* key, float* value) {
  if (!g || !chunks || n_events < 0 || (n_events > 0 && (!ts || !key || !value)))
    return LMS_EINVAL;
  const lms_status r = make_batch(g, chunks, n_chunks, n_events);
  if (r != LMS_OK) return r;
  std::memcpy(ts, g->h_ts, 8 * (size_t)n_events);
  std::memcpy(key, g->h_key, 4 * (size_t)n_events);
  std::memcpy(value, g->h_val, 4 * (size_t)n_events);
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
