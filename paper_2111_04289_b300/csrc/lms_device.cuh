// Device helpers shared by the kernels of the engine.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lms_internal.h"

namespace lms {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kEmpty = ~0ull;

// q = n / d for the constants of udiv_constants(d): t = mulhi(m, n),
// q = (t + ((n - t) >> sh1)) >> sh2   (Granlund & Montgomery 1994, Fig. 4.1).
__device__ __forceinline__ unsigned long long udiv_inv(unsigned long long n, unsigned long long m,
                                                       int sh1, int sh2) {
  unsigned long long t = __umul64hi(m, n);
  return (t + ((n - t) >> sh1)) >> sh2;
}

// Group keys (see lms_internal.h): block-major, then key, then the pane's
// position in its block of 2^lb panes.
__device__ __forceinline__ unsigned long long make_gkey(unsigned long long pane_rel, unsigned key,
                                                        int lb) {
  const unsigned long long lo = (1ull << lb) - 1ull;
  return ((pane_rel >> lb) << (32 + lb)) | ((unsigned long long)key << lb) | (pane_rel & lo);
}
__device__ __forceinline__ unsigned gkey_key(unsigned long long g, int lb) {
  return (unsigned)(g >> lb);
}
__device__ __forceinline__ unsigned long long gkey_pane(unsigned long long g, int lb) {
  return ((g >> (32 + lb)) << lb) | (g & ((1ull << lb) - 1ull));
}
__device__ __forceinline__ unsigned long long gkey_block(unsigned long long g, int lb) {
  return g >> (32 + lb);
}

// Order-preserving uint32 images of int32 and float32 values, so that
// unsigned atomicMin/atomicMax implement min/max.  The float image orders by
// IEEE-754 totalOrder (-0.0 < +0.0).
__device__ __forceinline__ unsigned enc_i32(int v) { return (unsigned)v ^ 0x80000000u; }
__device__ __forceinline__ int dec_i32(unsigned u) { return (int)(u ^ 0x80000000u); }
__device__ __forceinline__ unsigned enc_f32(float f) {
  unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ unsigned dec_f32_bits(unsigned u) {
  return (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
}

// Multiplicative (Fibonacci) hash of a 64-bit group key to `bits` bits.
__device__ __forceinline__ unsigned hash_slot(unsigned long long g, int bits) {
  return (unsigned)((g * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

__device__ __forceinline__ bool filter_pass_i(int op, long long x, long long c) {
  switch (op) {
    case 1: return x == c;
    case 2: return x != c;
    case 3: return x < c;
    case 4: return x <= c;
    case 5: return x > c;
    case 6: return x >= c;
    default: return true;
  }
}
__device__ __forceinline__ bool filter_pass_f(int op, double x, double c) {
  switch (op) {
    case 1: return x == c;
    case 2: return x != c;
    case 3: return x < c;
    case 4: return x <= c;
    case 5: return x > c;
    case 6: return x >= c;
    default: return true;
  }
}

// `(double)v OP c` for a float32 v, decided in float32 (see QueryDev).
__device__ __forceinline__ bool filter_pass_f32(int op, float v, float lo, float hi, int exact) {
  switch (op) {
    case 1: return exact && v == lo;
    case 2: return !(exact && v == lo);
    case 3: return v < hi;
    case 4: return v <= lo;
    case 5: return v > lo;
    case 6: return v >= hi;
    default: return true;
  }
}

__device__ __forceinline__ Grp load_grp(const Grp* p) {
  const uint4 a = reinterpret_cast<const uint4*>(p)[0];
  const uint4 b = reinterpret_cast<const uint4*>(p)[1];
  Grp g;
  g.gkey = ((unsigned long long)a.y << 32) | a.x;
  g.cnt = (long long)(((unsigned long long)a.w << 32) | a.z);
  g.sum = ((unsigned long long)b.y << 32) | b.x;
  g.mn = b.z;
  g.mx = b.w;
  return g;
}
// One 32-byte vector load of a group record (records are 32-byte aligned):
// one load instruction per random gather instead of two.  For kernels that
// do not write the records they read.
__device__ __forceinline__ Grp load_grp_v(const Grp* p) {
  unsigned long long a, b, c, d;
  asm("ld.global.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
  Grp g;
  g.gkey = a;
  g.cnt = (long long)b;
  g.sum = c;
  g.mn = (unsigned)d;
  g.mx = (unsigned)(d >> 32);
  return g;
}
__device__ __forceinline__ void store_grp(Grp* p, unsigned long long gkey, long long cnt,
                                          unsigned long long sum, unsigned mn, unsigned mx) {
  uint4* q = reinterpret_cast<uint4*>(p);
  q[0] = make_uint4((unsigned)gkey, (unsigned)(gkey >> 32), (unsigned)cnt,
                    (unsigned)((unsigned long long)cnt >> 32));
  q[1] = make_uint4((unsigned)sum, (unsigned)(sum >> 32), mn, mx);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Inclusive warp scan of 64-bit values.
__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long n = __shfl_up_sync(kFull, v, o);
    if ((int)lane_id() >= o) v += n;
  }
  return v;
}

// Exclusive block scan of one 64-bit value per thread; returns the prefix and
// writes the block total to *total.  `tmp` needs blockDim/32 + 1 entries.
// Must be called by all threads of the block.
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v,
                                                              unsigned long long* tmp,
                                                              unsigned long long* total) {
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long inc = warp_incl_scan(v);
  if (lane_id() == 31) tmp[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned long long x = (int)lane_id() < nw ? tmp[lane_id()] : 0ull;
    unsigned long long xi = warp_incl_scan(x);
    if ((int)lane_id() < nw) tmp[lane_id()] = xi - x;
    if (lane_id() == 31) tmp[32] = xi;
  }
  __syncthreads();
  unsigned long long r = tmp[w] + inc - v;
  *total = tmp[32];
  __syncthreads();
  return r;
}

// ---- segmented scans (reduce-by-key) -------------------------------------

struct SegAgg {  // (run started here?, aggregate since the run's head)
  unsigned f;
  long long cnt;
  unsigned long long sum;
  unsigned mn, mx;
};

template <bool FLOAT>
__device__ __forceinline__ SegAgg seg_combine(const SegAgg& x, const SegAgg& y) {
  if (y.f) return y;  // y's run starts inside y: x does not reach past it
  SegAgg r;
  r.f = x.f;
  r.cnt = x.cnt + y.cnt;
  r.sum = FLOAT ? (unsigned long long)__double_as_longlong(__longlong_as_double((long long)x.sum) +
                                                           __longlong_as_double((long long)y.sum))
                : x.sum + y.sum;
  r.mn = min(x.mn, y.mn);
  r.mx = max(x.mx, y.mx);
  return r;
}

__device__ __forceinline__ SegAgg seg_identity() {
  SegAgg r;
  r.f = 0;
  r.cnt = 0;
  r.sum = 0ull;  // +0.0 for doubles
  r.mn = 0xffffffffu;
  r.mx = 0u;
  return r;
}

__device__ __forceinline__ SegAgg seg_shfl_up(const SegAgg& v, int d) {
  SegAgg r;
  r.f = __shfl_up_sync(kFull, v.f, d);
  r.cnt = __shfl_up_sync(kFull, v.cnt, d);
  r.sum = __shfl_up_sync(kFull, v.sum, d);
  r.mn = __shfl_up_sync(kFull, v.mn, d);
  r.mx = __shfl_up_sync(kFull, v.mx, d);
  return r;
}

__device__ __forceinline__ SegAgg seg_shfl_idx(const SegAgg& v, int src) {
  SegAgg r;
  r.f = __shfl_sync(kFull, v.f, src);
  r.cnt = __shfl_sync(kFull, v.cnt, src);
  r.sum = __shfl_sync(kFull, v.sum, src);
  r.mn = __shfl_sync(kFull, v.mn, src);
  r.mx = __shfl_sync(kFull, v.mx, src);
  return r;
}

// Exclusive segmented scan of the warp totals wt[0 .. nw) (nw <= 32), done by
// warp 0 with shuffles, starting from *carry: wt[j] becomes what precedes warp
// j and *carry what precedes the next tile.  Every thread of the block calls
// it between two barriers; only warp 0 works.
template <bool FLOAT>
__device__ __forceinline__ void seg_scan_warp_totals(SegAgg* wt, int nw, SegAgg* carry) {
  if (threadIdx.x >= 32) return;
  const int lane = (int)threadIdx.x;
  SegAgg incl = lane < nw ? wt[lane] : seg_identity();
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const SegAgg o = seg_shfl_up(incl, d);
    if (lane >= d) incl = seg_combine<FLOAT>(o, incl);
  }
  const SegAgg ex = seg_shfl_up(incl, 1);
  const SegAgg tot = seg_shfl_idx(incl, nw - 1);
  const SegAgg c = *carry;
  __syncwarp();
  if (lane < nw) wt[lane] = lane == 0 ? c : seg_combine<FLOAT>(c, ex);
  if (lane == 0) *carry = seg_combine<FLOAT>(c, tot);
}

// Contiguous chunk [lo, hi) of n items owned by chunk c of g chunks.
__device__ __forceinline__ void chunk_range(unsigned long long n, int c, int g,
                                            unsigned long long* lo, unsigned long long* hi) {
  unsigned long long per = (n + g - 1) / g;
  per = (per + 255ull) & ~255ull;
  unsigned long long a = per * (unsigned long long)c;
  unsigned long long b = a + per;
  *lo = a < n ? a : n;
  *hi = b < n ? b : n;
}

}  // namespace lms
