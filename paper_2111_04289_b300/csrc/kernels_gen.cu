// Synthetic load generator for the serving backend (input data only: none of
// the method's arithmetic).  Events of the large float stream: key Zipf(s) over
// n_keys keys by inverse CDF, value float32 lognormal(0, 1) by the Box-Muller
// transform, both drawn once for a pool of event counters (random bits from
// SplitMix64 — Steele, Lea & Flood, 2014 — on the counter); event c of the
// stream takes the pool's entry c mod pool, so every event depends only on the
// seed and its stream-wide index.  ts = floor(arrival ms) is written per batch
// for the arrival ticks the serving loop admitted.
#include "lms_internal.h"

namespace lms {

namespace {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// uniform double in (0, 1)
__device__ __forceinline__ double unit(unsigned long long bits) {
  return ((double)(bits >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

// Key and value of event counters i mod pool, for i in [0, n): the pool of
// columns the batches are sliced from (its tail repeats its head, so every
// batch of up to n - pool consecutive counters is one contiguous slice).
__global__ void k_gen_pool(unsigned long long seed, const double* __restrict__ cdf,
                           unsigned n_keys, long long pool, long long n,
                           unsigned* __restrict__ key, float* __restrict__ value) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long ctr = (unsigned long long)(i % pool);
    const unsigned long long b0 = splitmix64(seed ^ (ctr * 0xD1B54A32D192ED03ull));
    const unsigned long long b1 = splitmix64(b0);
    const unsigned long long b2 = splitmix64(b1);
    // key: first rank whose CDF reaches u
    const double u = unit(b0);
    unsigned a = 0, b = n_keys - 1;
    while (a < b) {
      const unsigned m = (a + b) >> 1;
      if (cdf[m] >= u) b = m;
      else a = m + 1;
    }
    const double z = sqrt(-2.0 * log(unit(b1))) * cospi(2.0 * unit(b2));
    key[i] = a;
    value[i] = (float)exp(z);
  }
}

// ts = floor(arrival ms) of the batch's events (chunks in event order).
__global__ void k_gen_ts(const GenChunk* __restrict__ chunks, int n_chunks, long long n,
                         long long* __restrict__ ts) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    int lo = 0, hi = n_chunks - 1;  // last chunk with offset <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunks[mid].offset <= e) lo = mid;
      else hi = mid - 1;
    }
    const GenChunk c = chunks[lo];
    const long long j = c.j_begin + (e - c.offset);
    ts[e] = (long long)floor(c.t0_ms + ((double)j + 0.5) * c.width_ms / (double)c.n_total);
  }
}

}  // namespace

cudaError_t launch_gen_pool(unsigned long long seed, const double* cdf, unsigned n_keys,
                            long long pool, long long n, unsigned* key, float* value, int sms,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gen_pool<<<8 * sms, 256, 0, st>>>(seed, cdf, n_keys, pool, n, key, value);
  return cudaGetLastError();
}

cudaError_t launch_gen_ts(const GenChunk* chunks, int n_chunks, long long n, long long* ts,
                          int sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = (n + 255) / 256;
  const int grid = (int)(blocks < 8LL * sms ? blocks : 8LL * sms);
  k_gen_ts<<<grid, 256, 0, st>>>(chunks, n_chunks, n, ts);
  return cudaGetLastError();
}

}  // namespace lms
