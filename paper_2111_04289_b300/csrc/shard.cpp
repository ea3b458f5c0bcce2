// Key-hash sharding of a host micro-batch over G per-device streams: the
// "Shuffling" operation of Table II done on the host before the copy to the
// device.  A window group (window, key) is built from the rows of its key
// only, so each key is owned by exactly one shard; the one quantity every
// shard needs from the whole batch is its max event time (the watermark
// input of Section II-A's event-time windows), returned here as the hint the
// shards are given (lms_stream_set_batch_max_ts).
//
// The split is a stable counting sort by shard: per-thread histograms over
// contiguous row ranges, an exclusive scan over (shard, thread), then each
// thread scatters its range.  Rows of one shard keep their input order.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <thread>
#include <vector>

#include "../../include/lmstream.h"

namespace {

inline uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

inline uint32_t shard_of(uint32_t key, uint32_t mask, uint32_t g) {
  return (uint32_t)(((uint64_t)fmix32(key & mask) * (uint64_t)g) >> 32);
}

template <class F>
void run_threads(int nt, F f) {
  if (nt == 1) {
    f(0);
    return;
  }
  std::vector<std::thread> th;
  th.reserve((size_t)nt);
  for (int t = 0; t < nt; ++t) th.emplace_back(f, t);
  for (auto& x : th) x.join();
}

}  // namespace

extern "C" {

uint32_t lms_shard_of(uint32_t key, uint32_t key_mask, int32_t n_shards) {
  return n_shards < 1 ? 0u : shard_of(key, key_mask, (uint32_t)n_shards);
}

lms_status lms_shard_split(const lms_batch* in, uint32_t key_mask, int32_t n_shards,
                           int64_t* ts_out, uint32_t* key_out, uint32_t* value_out,
                           uint8_t* type_out, int64_t* offsets, int64_t* max_ts) {
  if (!in || !offsets || n_shards < 1 || in->n_rows < 0) return LMS_EINVAL;
  if (in->memory != LMS_MEM_HOST) return LMS_EINVAL;
  const long long n = in->n_rows;
  if (n > 0 && (!in->ts || !in->key || !in->value || !ts_out || !key_out || !value_out))
    return LMS_EINVAL;
  if (n > 0 && in->type && !type_out) return LMS_EINVAL;
  const uint32_t G = (uint32_t)n_shards;
  const int nt = n >= (1ll << 20) ? (int)std::min<unsigned>(8u, std::max(1u, std::thread::hardware_concurrency())) : 1;
  std::vector<long long> lo((size_t)nt + 1);
  for (int t = 0; t <= nt; ++t) lo[(size_t)t] = n * t / nt;
  // hist[t * G + g]: rows of thread t's range that go to shard g
  std::vector<long long> hist((size_t)nt * G, 0);
  std::vector<long long> tmax((size_t)nt, LLONG_MIN);
  const int64_t* ts = in->ts;
  const uint32_t* key = in->key;
  const uint32_t* val = static_cast<const uint32_t*>(in->value);
  const uint8_t* typ = in->type;
  run_threads(nt, [&](int t) {
    long long* h = hist.data() + (size_t)t * G;
    long long mx = LLONG_MIN;
    for (long long i = lo[(size_t)t]; i < lo[(size_t)t + 1]; ++i) {
      h[shard_of(key[i], key_mask, G)] += 1;
      mx = std::max<long long>(mx, ts[i]);
    }
    tmax[(size_t)t] = mx;
  });
  // exclusive scan in (shard, thread) order: start of thread t's rows of shard g
  long long acc = 0;
  for (uint32_t g = 0; g < G; ++g) {
    offsets[g] = acc;
    for (int t = 0; t < nt; ++t) {
      long long& h = hist[(size_t)t * G + g];
      const long long c = h;
      h = acc;
      acc += c;
    }
  }
  offsets[G] = acc;
  run_threads(nt, [&](int t) {
    long long* pos = hist.data() + (size_t)t * G;
    for (long long i = lo[(size_t)t]; i < lo[(size_t)t + 1]; ++i) {
      const long long o = pos[shard_of(key[i], key_mask, G)]++;
      ts_out[o] = ts[i];
      key_out[o] = key[i];
      value_out[o] = val[i];
      if (typ) type_out[o] = typ[i];
    }
  });
  if (max_ts) {
    long long mx = LLONG_MIN;
    for (long long m : tmax) mx = std::max(mx, m);
    *max_ts = mx;
  }
  return LMS_OK;
}

}  // extern "C"
