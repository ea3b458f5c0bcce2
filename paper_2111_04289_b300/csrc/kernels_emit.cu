// Watermark, window enumeration, window assembly from panes, row emission and
// the carry of still-open panes into the next micro-batch.
//
// After a micro-batch the watermark is max(previous, max ts of the batch -
// allowed lateness); every window whose end is <= the watermark closes (the
// paper's per-micro-batch output step, Section III-A; window semantics as in
// the public header).  A window of K panes is assembled from the sorted
// window state: its panes are K contiguous, key-sorted runs of the state, so
// a CTA merges the runs (merge path) into the window's key-sorted list in
// shared memory and emits one row per distinct key, in key order.  A CTA
// handles a range of consecutive windows and carries the list from window to
// window (drop the pane that left, merge in the pane that entered).  Windows
// larger than shared memory are merged in global scratch.  Rows of all closed
// windows are written in (window_start, key) order; each range finds its row
// offset by a decoupled look-back over the ranges before it.
#include <climits>

#include "lms_device.cuh"

namespace lms {
namespace {

constexpr int kEmitThreads = 512;
constexpr unsigned kWwStage = 512;  // window ids of a range staged for the count pass
constexpr size_t kEmitSmemMax = 224 * 1024;  // dynamic shared memory of the emit kernel (static: ~2.3 KB)
// Largest window (entries) merged in shared memory for windows of k panes:
// two padded buffers (17 slots per 16 entries) plus two (k+1)-entry boundary
// arrays must fit in kEmitSmemMax.
inline unsigned emit_cap(int k) {
  const size_t avail = kEmitSmemMax - 2ull * (k + 2) * sizeof(unsigned) - 64;
  const size_t padded = avail / (2 * sizeof(unsigned long long));
  return (unsigned)(((padded - 1) * 16 / 17) & ~size_t(15));
}
inline size_t emit_smem(int k) {
  const unsigned cap = emit_cap(k);
  return 2ull * (cap + (cap >> 4) + 1) * sizeof(unsigned long long) +
         2ull * (k + 2) * sizeof(unsigned);
}

__device__ __forceinline__ long long floor_div_ll(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

__global__ void k_batch_begin(SCtl* sc, QCtl* c0, QCtl* c1, QCtl* c2, QCtl* c3, QCtl* c4,
                              QCtl* c5, QCtl* c6, QCtl* c7) {
  if (threadIdx.x != 0) return;
  sc->batch_max_ts = LLONG_MIN;
  QCtl* cs[8] = {c0, c1, c2, c3, c4, c5, c6, c7};
  for (int i = 0; i < 8; ++i)
    if (cs[i]) cs[i]->err = 0u;
}

struct WmArgs {
  int nq;
  int eos;
  long long lateness;
  QCtl* ctl[kMaxQueries];
  long long size[kMaxQueries];
  long long slide[kMaxQueries];
  long long origin_pane[kMaxQueries];
};

__global__ void k_watermark(SCtl* sc, const WmArgs a) {
  if (threadIdx.x != 0) return;
  const long long mx = sc->batch_max_ts;
  if (mx != LLONG_MIN) {
    const long long cand = mx - a.lateness;
    if (!sc->wm_valid || cand > sc->wm) sc->wm = cand;
    sc->wm_valid = 1;
  }
  for (int q = 0; q < a.nq; ++q) {
    QCtl* c = a.ctl[q];
    long long hi;
    if (a.eos) {
      hi = LLONG_MAX / 4;
    } else if (!sc->wm_valid) {
      hi = c->cursor - 1;
    } else {
      // last window w (absolute) with w*slide + size <= wm
      const long long wabs = floor_div_ll(sc->wm - a.size[q], a.slide[q]);
      long long d = wabs - a.origin_pane[q];
      if (d > (1ll << 40)) d = 1ll << 40;
      if (d < -(1ll << 40)) d = -(1ll << 40);
      hi = d + kPaneBias;
    }
    if (hi < c->cursor - 1) hi = c->cursor - 1;
    c->w_hi = hi;
  }
}

__global__ void k_emit_begin(QCtl* c) {
  if (threadIdx.x != 0) return;
  c->pool_used = 0ull;
  c->pool_need = 0ull;
  c->big_windows = 0ull;
  c->rows_batch = 0ull;
  c->n_windows = 0ull;
  c->win_ticket = 0ull;
  c->err &= ~kErrNeedRetry;
}

// Windows anchored at pane j: those whose first present pane is pane j.
__device__ __forceinline__ void anchored_range(const QueryDev& q, const Scratch& s,
                                               const QCtl* c, unsigned long long j, long long* lo,
                                               long long* hi) {
  const long long p = (long long)s.pane_id[j];
  long long a = p - q.k + 1;
  if (j > 0) {
    const long long prev = (long long)s.pane_id[j - 1] + 1;
    a = prev > a ? prev : a;
  }
  a = c->cursor > a ? c->cursor : a;
  const long long b = p < c->w_hi ? p : c->w_hi;
  *lo = a;
  *hi = b;
}

__global__ void __launch_bounds__(256) k_win_count(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  unsigned long long lo, hi;
  chunk_range(c->n_panes, blockIdx.x, gridDim.x, &lo, &hi);
  unsigned long long cnt = 0;
  for (unsigned long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
    long long a, b;
    anchored_range(q, s, c, j, &a, &b);
    if (b >= a) cnt += (unsigned long long)(b - a + 1);
  }
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  block_excl_scan(cnt, tmp, &tot);
  if (threadIdx.x == 0) s.chunk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_win_scan(const QueryDev q, const Scratch s) {
  __shared__ unsigned long long tmp[33];
  const unsigned long long v = (int)threadIdx.x < kGrid ? s.chunk[threadIdx.x] : 0ull;
  unsigned long long tot;
  const unsigned long long r = block_excl_scan(v, tmp, &tot);
  if ((int)threadIdx.x < kGrid) s.chunk[threadIdx.x] = r;
  if (threadIdx.x == 0) {
    q.ctl->n_windows = tot;
    if (tot > s.win_cap) atomicOr(&q.ctl->err, kErrWinOverflow);
  }
}

__global__ void __launch_bounds__(256) k_win_write(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  if (c->n_windows > s.win_cap) return;
  const unsigned long long P = c->n_panes;
  unsigned long long lo, hi;
  chunk_range(P, blockIdx.x, gridDim.x, &lo, &hi);
  __shared__ unsigned long long tmp[33];
  unsigned long long out = s.chunk[blockIdx.x];
  for (unsigned long long j0 = lo; j0 < hi; j0 += blockDim.x) {
    const unsigned long long j = j0 + threadIdx.x;
    long long a = 0, b = -1;
    if (j < hi) anchored_range(q, s, c, j, &a, &b);
    const unsigned long long cnt = b >= a ? (unsigned long long)(b - a + 1) : 0ull;
    unsigned long long tot;
    const unsigned long long r = block_excl_scan(cnt, tmp, &tot);
    unsigned long long j1 = j + 1;
    for (unsigned long long t = 0; t < cnt; ++t) {
      const long long w = a + (long long)t;
      while (j1 < P && (long long)s.pane_id[j1] < w + q.k) ++j1;
      const unsigned long long o = out + r + t;
      s.win_w[o] = w;
      s.win_j0[o] = (unsigned)j;
      s.win_j1[o] = (unsigned)j1;
      s.win_stat[o] = 0ull;
    }
    out += tot;
  }
}

// Index of element i in a merge buffer.  Shared buffers are padded by one
// slot per 16 elements so that threads writing consecutive chunks do not all
// hit the same bank; global scratch is not padded.
template <bool PAD>
__device__ __forceinline__ unsigned pix(unsigned i) { return PAD ? i + (i >> 4) : i; }

// Pairwise merge rounds of `nr` sorted runs of A (boundaries bc[0..nr],
// bc[nr] = len), ping-ponging with B.  Values are distinct.  Returns the
// buffer holding the fully merged sequence.  All threads must call.  Each
// round gives every thread one chunk of about len / blockDim outputs.
template <bool PAD>
__device__ unsigned long long* merge_runs(unsigned long long* A, unsigned long long* B,
                                          unsigned* bc, unsigned* bn, int nr, unsigned len) {
  const unsigned chunk = max(4u, (len + blockDim.x - 1) / blockDim.x);
  while (nr > 1) {
    const int np = (nr + 1) >> 1;
    for (unsigned ch = threadIdx.x; ch * chunk < len; ch += blockDim.x) {
      unsigned o = ch * chunk;
      const unsigned oe = min(len, o + chunk);
      // pair m holding output position o: largest m with bc[2m] <= o
      int lo = 0, hi = np - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bc[2 * mid] <= o) lo = mid; else hi = mid - 1;
      }
      int m = lo;
      while (o < oe) {
        const unsigned s0 = bc[2 * m];
        const unsigned s1 = bc[min(2 * m + 1, nr)];
        const unsigned s2 = bc[min(2 * m + 2, nr)];
        const unsigned la = s1 - s0, lb = s2 - s1, diag = o - s0;
        unsigned a = diag > lb ? diag - lb : 0u, b = min(diag, la);
        while (a < b) {
          const unsigned mid = (a + b) >> 1;
          if (A[pix<PAD>(s0 + mid)] < A[pix<PAD>(s1 + diag - 1u - mid)]) a = mid + 1u;
          else b = mid;
        }
        unsigned i = a, k = diag - a;
        const unsigned stop = min(oe, s2);
        unsigned long long va = i < la ? A[pix<PAD>(s0 + i)] : ~0ull;
        unsigned long long vb = k < lb ? A[pix<PAD>(s1 + k)] : ~0ull;
        while (o < stop) {
          if (k >= lb || (i < la && va < vb)) {
            B[pix<PAD>(o++)] = va;
            ++i;
            va = i < la ? A[pix<PAD>(s0 + i)] : ~0ull;
          } else {
            B[pix<PAD>(o++)] = vb;
            ++k;
            vb = k < lb ? A[pix<PAD>(s1 + k)] : ~0ull;
          }
        }
        ++m;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t <= np; t += blockDim.x) bn[t] = t < np ? bc[2 * t] : len;
    __syncthreads();
    unsigned long long* tA = A; A = B; B = tA;
    unsigned* tb = bc; bc = bn; bn = tb;
    nr = np;
  }
  return A;
}

// 1/n as a double, to about 2^-47 relative, for 3 <= n < 2^24 with n not a
// power of two, using no FP64 arithmetic (the FP64 pipe of this part is
// narrow): r0 = RN(1/n) in float, e = 1 - n r0 by FMA, 1/n = r0 (1 + e + e^2
// ...) ~ r0 + RN(r0 e); the two floats are summed into one double with integer
// operations.  |r0 e| <= 2^-24 r0 and r0's mantissa is neither all zeros nor
// all ones, so the sum stays in r0's binade (a carry into the exponent field
// still gives the right bits).
__device__ __forceinline__ double recip_small(unsigned n) {
  const float nf = (float)n;  // exact below 2^24
  const float r0 = __frcp_rn(nf);
  const float rl = r0 * fmaf(-nf, r0, 1.0f);
  const unsigned b0 = __float_as_uint(r0), b1 = __float_as_uint(rl);
  const int e0 = (int)((b0 >> 23) & 0xffu);
  long long m = (long long)(b0 & 0x7fffffu) << 29;  // mantissa field of the double
  if (rl != 0.0f) {
    const int sh = (int)((b1 >> 23) & 0xffu) - e0 + 29;  // rl's unit in the field's units
    const long long m1 = (long long)((b1 & 0x7fffffu) | 0x800000u);
    const long long c = sh >= 0 ? (m1 << sh) : (sh > -40 ? (m1 >> -sh) : 0ll);
    m += (b1 >> 31) ? -c : c;
  }
  return __longlong_as_double(((long long)(e0 + 896) << 52) + m);
}

template <bool FLOAT>
__device__ __forceinline__ void write_row(const QueryDev& q, ResultRowDev* out, long long wstart,
                                          unsigned key, long long cnt, unsigned long long sbits,
                                          unsigned mn, unsigned mx) {
  // avg = sum / count; counts of 1 and powers of two need no division (the
  // product with an exact power of two is the correctly rounded quotient).
  const double sd = FLOAT ? __longlong_as_double((long long)sbits) : (double)(long long)sbits;
  double avg;
  if (cnt == 1) {
    avg = sd;
  } else if ((cnt & (cnt - 1)) == 0) {
    const int e = __ffsll(cnt) - 1;
    avg = sd * __longlong_as_double((long long)(1023 - e) << 52);
  } else if (FLOAT && cnt < (1ll << 24)) {
    // float sums are checked to 1e-9 relative: one FP64 multiply by a
    // reciprocal good to 2^-47
    avg = sd * recip_small((unsigned)cnt);
  } else if (FLOAT) {
    // larger counts: float32 reciprocal refined by two corrections with exact
    // FMA remainders
    const double n = (double)cnt;
    const double r = (double)__frcp_rn((float)cnt);
    const double q0 = sd * r;
    const double q1 = fma(fma(-q0, n, sd), r, q0);
    avg = fma(fma(-q1, n, sd), r, q1);
  } else {
    avg = sd / (double)cnt;  // int sums: exact division (bit-exact rows)
  }
  unsigned mnv = 0u, mxv = 0u;
  if (q.agg_mask & 4u) mnv = FLOAT ? dec_f32_bits(mn) : (unsigned)dec_i32(mn);
  if (q.agg_mask & 8u) mxv = FLOAT ? dec_f32_bits(mx) : (unsigned)dec_i32(mx);
  // rows are written once and read only by the host: streaming stores, so
  // that they do not displace the state groups the next windows gather
  uint4* o = reinterpret_cast<uint4*>(out);
  __stcs(o, make_uint4((unsigned)wstart, (unsigned)((unsigned long long)wstart >> 32),
                       (unsigned)cnt, (unsigned)((unsigned long long)cnt >> 32)));
  const unsigned long long ab = (unsigned long long)__double_as_longlong(avg);
  __stcs(o + 1,
         make_uint4((unsigned)sbits, (unsigned)(sbits >> 32), (unsigned)ab, (unsigned)(ab >> 32)));
  __stcs(o + 2, make_uint4(key, mnv, mxv, (unsigned)q.qid));
}

// Exclusive scan of one count per thread over the block; returns the prefix
// and writes the block total to *total.  wt holds 33 counters.
__device__ __forceinline__ unsigned block_scan_u32(unsigned v, unsigned* wt, unsigned* total) {
  const unsigned lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, inc, o);
    if ((int)lane >= o) inc += y;
  }
  if (lane == 31) wt[w] = inc;
  __syncthreads();
  if (w == 0) {
    const unsigned x = lane < nw ? wt[lane] : 0u;
    unsigned wi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, wi, o);
      if ((int)lane >= o) wi += y;
    }
    if (lane < nw) wt[lane] = wi - x;
    if (lane == 31) wt[32] = wi;
  }
  __syncthreads();
  const unsigned r = wt[w] + inc - v;
  *total = wt[32];
  __syncthreads();
  return r;
}

// Heads (first entries of a key) in this thread's contiguous chunk of S[0..len).
template <bool PAD>
__device__ __forceinline__ unsigned chunk_heads(const unsigned long long* S, unsigned len,
                                                unsigned a, unsigned b) {
  unsigned h = 0;
  unsigned prev = a > 0 ? (unsigned)(S[pix<PAD>(a - 1)] >> 32) : 0u;
  for (unsigned i = a; i < b; ++i) {
    const unsigned k = (unsigned)(S[pix<PAD>(i)] >> 32);
    h += (i == 0 || k != prev) ? 1u : 0u;
    prev = k;
  }
  return h;
}

// Distinct keys of the merged window S[0..len), in key order: their number.
template <bool PAD>
__device__ __forceinline__ unsigned long long count_distinct(const unsigned long long* S,
                                                             unsigned len, unsigned* wt) {
  const unsigned per = (len + blockDim.x - 1) / blockDim.x;
  const unsigned a = min(len, threadIdx.x * per), b = min(len, a + per);
  unsigned tot;
  block_scan_u32(chunk_heads<PAD>(S, len, a, b), wt, &tot);
  return tot;
}

// One row per distinct key of the merged window S[0..len) (entries key << 32 |
// state index, key-sorted), written from out[0] in key order; returns the
// number of rows.  First the position of every key's first entry goes to
// hp[rank] (hp: len + 1 words of scratch not aliasing S); then thread t takes
// rows t, t + blockDim, ...: it combines the key's groups (one per pane that
// holds the key) and writes the row, so a warp's rows are consecutive and its
// stores coalesce.  Ends with a barrier (hp may be reused).
template <bool FLOAT, bool PAD>
__device__ unsigned write_distinct(const QueryDev& q, const unsigned long long* S, unsigned len,
                                   long long wstart, ResultRowDev* out, unsigned* hp,
                                   unsigned* wt) {
  const unsigned per = (len + blockDim.x - 1) / blockDim.x;
  const unsigned a = min(len, threadIdx.x * per), b = min(len, a + per);
  unsigned nrows;
  unsigned r = block_scan_u32(chunk_heads<PAD>(S, len, a, b), wt, &nrows);
  unsigned prev = a > 0 ? (unsigned)(S[pix<PAD>(a - 1)] >> 32) : 0u;
  for (unsigned i = a; i < b; ++i) {
    const unsigned k = (unsigned)(S[pix<PAD>(i)] >> 32);
    if (i == 0 || k != prev) hp[r++] = i;
    prev = k;
  }
  if (threadIdx.x == 0) hp[nrows] = len;
  __syncthreads();
  // Every load is issued unconditionally (an exhausted row re-reads its last
  // entry) so that a row's gathers are in flight together.
  const Grp* st = q.state;
  for (unsigned row = threadIdx.x; row < nrows; row += blockDim.x) {
    const unsigned e0 = hp[row], e1 = hp[row + 1];
    const unsigned long long x0 = S[pix<PAD>(e0)];
    const Grp g0 = load_grp_v(st + (x0 & 0xffffffffull));
    long long cnt = g0.cnt;
    unsigned long long isum = g0.sum;
    double fsum = __longlong_as_double((long long)g0.sum);
    unsigned mn = g0.mn, mx = g0.mx;
    for (unsigned e = e0 + 1; e < e1; e += 2) {  // the key's other panes, two loads in flight
      const bool two = e + 1 < e1;
      const unsigned long long x1 = S[pix<PAD>(e)], x2 = S[pix<PAD>(two ? e + 1 : e)];
      const Grp g1 = load_grp_v(st + (x1 & 0xffffffffull));
      const Grp g2 = load_grp_v(st + (x2 & 0xffffffffull));
      cnt += g1.cnt;
      mn = min(mn, g1.mn);
      mx = max(mx, g1.mx);
      if (FLOAT) fsum += __longlong_as_double((long long)g1.sum);
      else isum += g1.sum;
      if (two) {
        cnt += g2.cnt;
        mn = min(mn, g2.mn);
        mx = max(mx, g2.mx);
        if (FLOAT) fsum += __longlong_as_double((long long)g2.sum);
        else isum += g2.sum;
      }
    }
    const unsigned long long sb = FLOAT ? (unsigned long long)__double_as_longlong(fsum) : isum;
    write_row<FLOAT>(q, out + row, wstart, (unsigned)(x0 >> 32), cnt, sb, mn, mx);
  }
  __syncthreads();
  return nrows;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Decoupled look-back over the window ranges before `ri` (ranges are taken in
// ticket order, so every predecessor is already running or done).  Publishes
// this range's row count, waits (bounded, ~4 s) for the predecessors' counts
// and returns the exclusive prefix, or ~0 after setting kErrLookback.
__device__ unsigned long long range_lookback(unsigned long long* stat, unsigned long long ri,
                                             unsigned long long n, QCtl* c) {
  constexpr unsigned long long kAgg = 1ull << 62, kPre = 2ull << 62, kVal = kAgg - 1;
  volatile unsigned long long* vs = stat;
  if (ri == 0) {
    vs[0] = kPre | n;
    return 0ull;
  }
  vs[ri] = kAgg | n;
  unsigned long long acc = 0;
  long long p = (long long)ri - 1;
  const unsigned long long t0 = global_ns();
  unsigned spins = 0;
  while (p >= 0) {
    const unsigned long long v = vs[p];
    if ((v >> 62) == 0) {
      if ((++spins & 255u) == 0 && global_ns() - t0 > 4000000000ull) {
        atomicOr(&c->err, kErrLookback);
        return ~0ull;
      }
      __nanosleep(128);
      continue;
    }
    acc += v & kVal;
    if ((v >> 62) == 2) break;
    --p;
  }
  __threadfence();
  vs[ri] = kPre | (acc + n);
  return acc;
}

// Copies state entries [g0, g1) as (key << 32 | state index) to T[base ..].
__device__ __forceinline__ void load_runs(const QueryDev& q, unsigned long long* T, unsigned base,
                                          unsigned long long g0, unsigned long long g1) {
  for (unsigned long long g = g0 + threadIdx.x; g < g1; g += blockDim.x)
    T[pix<true>(base + (unsigned)(g - g0))] = ((q.state[g].gkey & 0xffffffffull) << 32) | g;
}

// Keeps the entries of L[0..n) whose state index is >= lo, in order, in T.
// Returns their number.  All threads must call.
__device__ unsigned compact_list(const unsigned long long* L, unsigned n, unsigned long long lo,
                                 unsigned long long* T, unsigned* wt) {
  const unsigned per = (n + blockDim.x - 1) / blockDim.x;
  const unsigned a = min(n, threadIdx.x * per), b = min(n, a + per);
  unsigned keep = 0;
  for (unsigned i = a; i < b; ++i) keep += (L[pix<true>(i)] & 0xffffffffull) >= lo ? 1u : 0u;
  // exclusive scan of `keep` over the block
  const unsigned lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned inc = keep;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, inc, o);
    if ((int)lane >= o) inc += y;
  }
  if (lane == 31) wt[w] = inc;
  __syncthreads();
  if (w == 0) {
    const unsigned x = lane < nw ? wt[lane] : 0u;
    unsigned wi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, wi, o);
      if ((int)lane >= o) wi += y;
    }
    if (lane < nw) wt[lane] = wi - x;
    if (lane == 31) wt[32] = wi;
  }
  __syncthreads();
  unsigned o = wt[w] + inc - keep;
  const unsigned total = wt[32];
  for (unsigned i = a; i < b; ++i) {
    const unsigned long long x = L[pix<true>(i)];
    if ((x & 0xffffffffull) >= lo) T[pix<true>(o++)] = x;
  }
  __syncthreads();
  return total;
}

struct EmitSmem {
  unsigned long long* L;  // key-sorted list of the current window
  unsigned long long* T;  // the other buffer
  unsigned* bnd0;
  unsigned* bnd1;
  unsigned* wt;
};

// Rows of windows [wa, wb): counted (WRITE=false) or written from out[0]
// (WRITE=true).  Consecutive windows share most of their panes, so the
// window's key-sorted list is carried from one window to the next: entries of
// panes that left are dropped and the runs of panes that entered are merged
// in.  Windows of one pane need no list; windows above `cap` entries are
// merged in global scratch on their own.
template <bool FLOAT, bool WRITE>
__device__ unsigned long long run_range(const QueryDev& q, const Scratch& s, QCtl* c,
                                        unsigned long long wa, unsigned long long wb,
                                        unsigned cap, EmitSmem& m, ResultRowDev* out,
                                        unsigned long long* s_off) {
  const int tid = threadIdx.x;
  unsigned long long acc = 0;
  bool have = false;
  unsigned cj0 = 0, cj1 = 0, n = 0;
  unsigned long long cb1 = 0;  // state index where the carried list's last pane ends
  // the next window's id, panes and state range are loaded one window ahead
  long long nw_ = 0;
  unsigned nj0 = 0, nj1 = 0;
  unsigned long long nb0 = 0, nb1 = 0;
  if (wa < wb) {
    nw_ = s.win_w[wa];
    nj0 = s.win_j0[wa];
    nj1 = s.win_j1[wa];
    nb0 = s.pane_begin[nj0];
    nb1 = s.pane_begin[nj1];
  }
  for (unsigned long long wi = wa; wi < wb; ++wi) {
    const long long w = nw_;
    const unsigned j0 = nj0, j1 = nj1;
    const unsigned long long b0 = nb0, b1 = nb1;
    if (wi + 1 < wb) {
      nw_ = s.win_w[wi + 1];
      nj0 = s.win_j0[wi + 1];
      nj1 = s.win_j1[wi + 1];
    }
    const unsigned len = (unsigned)(b1 - b0);
    const int nr = (int)(j1 - j0);
    const long long wstart = (w - kPaneBias) * (long long)q.slide + q.base;
    if (nr == 1) {  // one pane: its run is already unique and key-sorted
      if (WRITE) {
        for (unsigned i = tid; i < len; i += blockDim.x) {
          const Grp g = load_grp(q.state + b0 + i);
          write_row<FLOAT>(q, out + acc + i, wstart, (unsigned)g.gkey, g.cnt, g.sum, g.mn, g.mx);
        }
      }
      acc += len;
      have = false;
      if (wi + 1 < wb) {
        nb0 = s.pane_begin[nj0];
        nb1 = s.pane_begin[nj1];
      }
      continue;
    }
    if (len > cap) {  // global-scratch merge of this window alone
      have = false;
      if (tid == 0) {
        unsigned long long off = atomicAdd(&c->pool_used, 2ull * len);
        if (off + 2ull * len > s.pool_cap) {
          atomicOr(&c->err, kErrPoolOverflow);
          off = ~0ull;
        } else {
          atomicAdd(&c->big_windows, 1ull);
        }
        *s_off = off;
      }
      __syncthreads();
      const unsigned long long off = *s_off;
      __syncthreads();
      if (off == ~0ull) {  // the host grows the scratch and runs the emission again
        if (wi + 1 < wb) {
          nb0 = s.pane_begin[nj0];
          nb1 = s.pane_begin[nj1];
        }
        continue;
      }
      unsigned long long* A = s.pool + off;
      unsigned long long* B = A + len;
      for (unsigned i = tid; i < len; i += blockDim.x)
        A[i] = ((q.state[b0 + i].gkey & 0xffffffffull) << 32) | (b0 + i);
      for (int r = tid; r <= nr; r += blockDim.x)
        m.bnd0[r] = (unsigned)(s.pane_begin[j0 + r] - b0);
      __syncthreads();
      const unsigned long long* S = merge_runs<false>(A, B, m.bnd0, m.bnd1, nr, len);
      unsigned* hp = reinterpret_cast<unsigned*>(S == A ? B : A);  // len u64 free: >= len + 1 words
      if (WRITE) acc += write_distinct<FLOAT, false>(q, S, len, wstart, out + acc, hp, m.wt);
      else acc += count_distinct<false>(S, len, m.wt);
      __syncthreads();
      if (wi + 1 < wb) {
        nb0 = s.pane_begin[nj0];
        nb1 = s.pane_begin[nj1];
      }
      continue;
    }
    // shared-memory list of this window
    if (have && j0 < cj1) {
      // drop the panes that left (their state indices are below b0) ...
      unsigned nk = n;
      if (j0 > cj0) {
        nk = compact_list(m.L, n, b0, m.T, m.wt);
        unsigned long long* t = m.L; m.L = m.T; m.T = t;
      }
      // ... then merge in the runs of the panes that entered
      if (j1 > cj1) {
        const unsigned long long g0 = cb1;  // = pane_begin[cj1]
        load_runs(q, m.L, nk, g0, b1);  // behind the kept entries
        const int add = (int)(j1 - cj1);
        if (tid == 0) m.bnd0[0] = 0u;
        for (int r = tid; r <= add; r += blockDim.x)
          m.bnd0[1 + r] = nk + (unsigned)((r == 0 ? g0 : r == add ? b1 : s.pane_begin[cj1 + r]) - g0);
        __syncthreads();
        unsigned long long* S = merge_runs<true>(m.L, m.T, m.bnd0, m.bnd1, add + 1, len);
        if (S != m.L) { m.T = m.L; m.L = S; }
      }
    } else {  // full build: merge the window's runs
      load_runs(q, m.T, 0u, b0, b1);
      for (int r = tid; r <= nr; r += blockDim.x)
        m.bnd0[r] = (unsigned)(s.pane_begin[j0 + r] - b0);
      __syncthreads();
      unsigned long long* S = merge_runs<true>(m.T, m.L, m.bnd0, m.bnd1, nr, len);
      if (S != m.L) { m.T = m.L; m.L = S; }
    }
    have = true;
    cj0 = j0;
    cj1 = j1;
    cb1 = b1;
    n = len;
    if (wi + 1 < wb) {  // the next window's state range (its panes have arrived by now)
      nb0 = s.pane_begin[nj0];
      nb1 = s.pane_begin[nj1];
    }
    __syncthreads();
    // the other buffer is free until the next window: it holds the key heads
    if (WRITE)
      acc += write_distinct<FLOAT, true>(q, m.L, len, wstart, out + acc,
                                         reinterpret_cast<unsigned*>(m.T), m.wt);
    else acc += count_distinct<true>(m.L, len, m.wt);
  }
  __syncthreads();
  return acc;
}

// Rows of windows [wa, wb) without assembling them.  A window's rows are its
// distinct keys; the group of key k in pane P is the first occurrence of k in
// exactly the windows whose ids lie in [max(prev + 1, P - K + 1), P], prev the
// last earlier pane holding k.  The CTA sweeps the range's panes in order
// (pane by pane; keys within a pane are distinct) with a shared table of
// (last pane, key) — entries older than any window still ahead are reused —
// and adds, per group, the number of the range's windows in that id
// interval.  Returns ~0 if the table overflowed (the caller then counts by
// assembling the windows).
__device__ unsigned long long count_range(const QueryDev& q, const Scratch& s, QCtl* c,
                                          unsigned long long wa, unsigned long long wb,
                                          unsigned cap, unsigned long long* tab, unsigned tab_n,
                                          unsigned* s_fail) {
  if (threadIdx.x == 0) *s_fail = 0u;
  __syncthreads();
  // global merge scratch the range's windows above `cap` entries will need
  // (so that one retry can size the scratch for the whole emission)
  unsigned long long need = 0;
  unsigned big = 0;
  for (unsigned long long wi = wa + threadIdx.x; wi < wb; wi += blockDim.x) {
    const unsigned long long len = s.pane_begin[s.win_j1[wi]] - s.pane_begin[s.win_j0[wi]];
    if (s.win_j1[wi] - s.win_j0[wi] > 1 && len > cap) need += 2ull * len;
    if (2ull * len > tab_n) big = 1u;  // a window's keys might not fit the table
  }
  if (need) atomicAdd(&c->pool_need, need);
  if (big) atomicOr(s_fail, 1u);
  __syncthreads();
  if (*s_fail) return ~0ull;  // count by assembling the windows instead
  for (unsigned i = threadIdx.x; i < tab_n; i += blockDim.x) tab[i] = 0ull;  // pane ids are >= 1
  const unsigned j_begin = s.win_j0[wa], j_end = s.win_j1[wb - 1];
  const long long w_first = s.win_w[wa], w_last = s.win_w[wb - 1];
  const long long* ww = s.win_w + wa;
  const unsigned nw = (unsigned)(wb - wa);
  // the range's window ids: consecutive (counts by arithmetic), else searched
  // in shared memory when they fit, else in global memory
  __shared__ unsigned s_ww[kWwStage];
  const bool contig = w_last - w_first + 1 == (long long)nw;
  const bool staged = !contig && nw <= kWwStage && w_last - w_first < (1ll << 32);
  if (staged)
    for (unsigned i = threadIdx.x; i < nw; i += blockDim.x) s_ww[i] = (unsigned)(ww[i] - w_first);
  __syncthreads();
  unsigned long long total = 0;
  // one group (key of pane P): update the key's last pane in the table and add
  // the range's windows in which this group is the key's first occurrence
  auto group = [&](unsigned key, long long P) {
    const unsigned long long nv = ((unsigned long long)P << 32) | key;
    long long prev = LLONG_MIN;
    unsigned h = (unsigned)(((unsigned long long)(key * 0x9E3779B1u) * tab_n) >> 32);
    unsigned stale = 0xffffffffu;
    unsigned long long stale_v = 0ull;
    bool done = false;
    for (unsigned probe = 0; probe < 256u && !done; ++probe) {
      const unsigned long long e = *((volatile unsigned long long*)&tab[h]);
      if (e != 0ull && (unsigned)e == key) {  // the key's entry: update its pane
        if (atomicCAS(&tab[h], e, nv) == e) {
          prev = (long long)(e >> 32);
          done = true;
        }
        continue;  // changed under us: look again
      }
      if (e == 0ull) {  // the key is absent: take the first stale slot seen, else this one
        if (stale != 0xffffffffu) {
          if (atomicCAS(&tab[stale], stale_v, nv) == stale_v) {
            done = true;
          } else {
            stale = 0xffffffffu;  // taken meanwhile: start over
            h = (unsigned)(((unsigned long long)(key * 0x9E3779B1u) * tab_n) >> 32);
          }
        } else if (atomicCAS(&tab[h], 0ull, nv) == 0ull) {
          done = true;
        }
        continue;
      }
      if (stale == 0xffffffffu && (long long)(e >> 32) < P - q.k + 1) {
        stale = h;  // no window still to come can contain that entry's pane
        stale_v = e;
      }
      h = h + 1 == tab_n ? 0u : h + 1;
    }
    if (!done) {
      atomicOr(s_fail, 1u);
      return;
    }
    long long lo = prev == LLONG_MIN ? P - q.k + 1 : max(prev + 1, P - q.k + 1);
    long long hi = P;
    lo = max(lo, w_first);
    hi = min(hi, w_last);
    if (lo > hi) return;
    if (contig) {
      total += (unsigned long long)(hi - lo + 1);
      return;
    }
    if (staged) {  // ids relative to w_first (their span is below 2^32)
      const unsigned rl = (unsigned)(lo - w_first), rh = (unsigned)(hi - w_first);
      unsigned a = 0, b = nw;  // first window with id >= lo
      while (a < b) {
        const unsigned m = (a + b) >> 1;
        if (s_ww[m] < rl) a = m + 1;
        else b = m;
      }
      unsigned c = a, d = nw;  // first window with id > hi
      while (c < d) {
        const unsigned m = (c + d) >> 1;
        if (s_ww[m] <= rh) c = m + 1;
        else d = m;
      }
      total += c - a;
      return;
    }
    unsigned a = 0, b = nw;  // first window with id >= lo
    while (a < b) {
      const unsigned m = (a + b) >> 1;
      if (ww[m] < lo) a = m + 1;
      else b = m;
    }
    unsigned c = a, d = nw;  // first window with id > hi
    while (c < d) {
      const unsigned m = (c + d) >> 1;
      if (ww[m] <= hi) c = m + 1;
      else d = m;
    }
    total += c - a;
  };
  // Panes in order, one barrier per pane (its table updates before the next
  // pane's lookups).  The next pane's bounds and this thread's first two keys
  // of it are loaded while the current pane is processed.
  const Grp* st = q.state;
  const unsigned bd = blockDim.x;
  long long nP = 0;
  unsigned long long ng0 = 0, ng1 = 0;
  unsigned nk0 = 0, nk1 = 0;
  auto fetch = [&](unsigned jj) {
    nP = (long long)s.pane_id[jj];
    ng0 = s.pane_begin[jj];
    ng1 = s.pane_begin[jj + 1];
    const unsigned long long ga = ng0 + threadIdx.x, gb = ga + bd;
    nk0 = ga < ng1 ? (unsigned)st[ga].gkey : 0u;
    nk1 = gb < ng1 ? (unsigned)st[gb].gkey : 0u;
  };
  if (j_begin < j_end) fetch(j_begin);
  for (unsigned j = j_begin; j < j_end; ++j) {
    const long long P = nP;
    const unsigned long long g0 = ng0, g1 = ng1;
    const unsigned k0 = nk0, k1 = nk1;
    if (j + 1 < j_end) fetch(j + 1);
    const unsigned long long ga = g0 + threadIdx.x;
    if (ga < g1) group(k0, P);
    if (ga + bd < g1) group(k1, P);
    for (unsigned long long g = ga + 2ull * bd; g < g1; g += bd) group((unsigned)st[g].gkey, P);
    __syncthreads();
  }
  __shared__ unsigned long long ctmp[33];
  unsigned long long tot;
  block_excl_scan(total, ctmp, &tot);
  return *s_fail ? ~0ull : tot;
}

// Assembles the closed windows.  CTAs take ranges of consecutive windows in
// ticket order; for each range: count its rows (pass 1), find the range's row
// offset by the look-back, then write its rows (pass 2) in (window, key) order.
// Dynamic shared memory: two padded list buffers of `cap` entries, then two
// run-boundary arrays of k + 2 entries.
template <bool FLOAT>
__global__ void __launch_bounds__(kEmitThreads, 1)
    k_emit(const QueryDev q, const Scratch s, ResultRowDev* rows, unsigned cap,
           unsigned long long rows_cap) {
  extern __shared__ __align__(16) unsigned long long esm[];
  const unsigned padded = cap + (cap >> 4) + 1;
  __shared__ unsigned wt[33];
  __shared__ unsigned long long s_ri, s_off;
  __shared__ unsigned s_fail;
  EmitSmem m;
  m.L = esm;
  m.T = esm + padded;
  m.bnd0 = reinterpret_cast<unsigned*>(esm + 2ull * padded);
  m.bnd1 = m.bnd0 + (q.k + 2);
  m.wt = wt;
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long W = c->n_windows;
  const unsigned long long per = (W + 4ull * gridDim.x - 1) / (4ull * gridDim.x);
  const unsigned long long NR = per ? (W + per - 1) / per : 0;
  const unsigned long long row_base = c->row_base;
  while (true) {
    if (threadIdx.x == 0) s_ri = atomicAdd(&c->win_ticket, 1ull);
    __syncthreads();
    const unsigned long long ri = s_ri;
    __syncthreads();
    if (ri >= NR) break;
    const unsigned long long wa = ri * per, wb = min(W, wa + per);
    // the range's row count: by the pane sweep, else by assembling the windows
    unsigned long long n = count_range(q, s, c, wa, wb, cap, esm, 2u * padded, &s_fail);
    __syncthreads();
    if (n == ~0ull) n = run_range<FLOAT, false>(q, s, c, wa, wb, cap, m, nullptr, &s_off);
    if (threadIdx.x == 0) {
      const unsigned long long off = range_lookback(s.win_stat, ri, n, c);
      s_off = off;
      if (off != ~0ull) {
        if (ri == NR - 1) c->rows_batch = off + n;
        if (row_base + off + n > rows_cap) atomicOr(&c->err, kErrRowsOverflow);
      }
    }
    __syncthreads();
    const unsigned long long off = s_off;
    __syncthreads();
    if (off != ~0ull && row_base + off + n <= rows_cap && !(c->err & kErrPoolOverflow))
      run_range<FLOAT, true>(q, s, c, wa, wb, cap, m, rows + row_base + off, &s_off);
  }
}

// ---- carry the panes that stay open into the next batch's partial arrays --

__global__ void k_trim_prep(const QueryDev q, const Scratch s) {
  if (threadIdx.x != 0) return;
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  c->row_base += c->rows_batch;
  if (c->w_hi >= c->cursor) c->cursor = c->w_hi + 1;
  // first pane that stays open: pane id > w_hi
  const unsigned long long P = c->n_panes;
  unsigned long long lo = 0, hi = P;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if ((long long)s.pane_id[mid] <= c->w_hi) lo = mid + 1; else hi = mid;
  }
  const unsigned long long from = lo < P ? s.pane_begin[lo] : c->n_state;
  c->trim_from = from;
  c->carried = c->n_state - from;
  c->n_parts = c->carried;
  c->or_mask = 0ull;
  c->and_mask = ~0ull;
}

__global__ void __launch_bounds__(256) k_trim_copy(const QueryDev q) {
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long from = c->trim_from, n = c->carried;
  unsigned long long o_acc = 0ull, a_acc = ~0ull;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const Grp g = load_grp(q.state + from + i);
    store_grp(q.parts + i, g.gkey, g.cnt, g.sum, g.mn, g.mx);
    q.pkeys[i] = g.gkey;
    o_acc |= g.gkey;
    a_acc &= g.gkey;
  }
  const unsigned olo = __reduce_or_sync(kFull, (unsigned)o_acc);
  const unsigned ohi = __reduce_or_sync(kFull, (unsigned)(o_acc >> 32));
  const unsigned alo = __reduce_and_sync(kFull, (unsigned)a_acc);
  const unsigned ahi = __reduce_and_sync(kFull, (unsigned)(a_acc >> 32));
  if (lane_id() == 0) {
    const unsigned long long o = ((unsigned long long)ohi << 32) | olo;
    const unsigned long long a = ((unsigned long long)ahi << 32) | alo;
    if (o) atomicOr(&c->or_mask, o);
    if (a != ~0ull) atomicAnd(&c->and_mask, a);
  }
}

template <bool FLOAT>
cudaError_t launch_emit_t(const QueryDev& q, const Scratch& s, ResultRowDev* rows, int grid,
                          size_t smem, unsigned long long rows_cap, cudaStream_t st) {
  // once per process (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(
      k_emit<FLOAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEmitSmemMax);
  if (attr != cudaSuccess) return attr;
  k_emit<FLOAT><<<grid, kEmitThreads, smem, st>>>(q, s, rows, smem ? emit_cap(q.k) : 0u,
                                                 rows_cap);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_begin(SCtl* sctl, QCtl* const* ctls, int nq, cudaStream_t st) {
  QCtl* c[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int i = 0; i < nq && i < 8; ++i) c[i] = ctls[i];
  k_batch_begin<<<1, 32, 0, st>>>(sctl, c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7]);
  return cudaGetLastError();
}

cudaError_t launch_watermark(SCtl* sctl, const QueryDev* qs, int nq, long long lateness, int eos,
                             cudaStream_t st) {
  WmArgs a;
  a.nq = nq;
  a.eos = eos;
  a.lateness = lateness;
  for (int i = 0; i < nq; ++i) {
    a.ctl[i] = qs[i].ctl;
    a.size[i] = qs[i].size;
    a.slide[i] = (long long)qs[i].slide;
    a.origin_pane[i] = qs[i].origin_pane;
  }
  k_watermark<<<1, 32, 0, st>>>(sctl, a);
  return cudaGetLastError();
}

// ev4 (optional): events recorded before/after E1 and before/after E2.
cudaError_t launch_emit(const QueryDev& q, const Scratch& s, ResultRowDev* rows,
                        unsigned long long rows_cap, int sms, cudaStream_t st, int* launches,
                        cudaEvent_t* ev4) {
  k_emit_begin<<<1, 32, 0, st>>>(q.ctl);
  k_win_count<<<kGrid, 256, 0, st>>>(q, s);
  k_win_scan<<<1, 1024, 0, st>>>(q, s);
  k_win_write<<<kGrid, 256, 0, st>>>(q, s);
  // Tumbling windows (one pane each) need no merge buffers.
  const size_t smem = q.k > 1 ? emit_smem(q.k) : 0;
  const int grid = q.k > 1 ? sms : 4 * sms;
  if (ev4) {
    record_event(ev4[0], st);
    record_event(ev4[1], st);
    record_event(ev4[2], st);
  }
  cudaError_t e = q.value_is_float ? launch_emit_t<true>(q, s, rows, grid, smem, rows_cap, st)
                                   : launch_emit_t<false>(q, s, rows, grid, smem, rows_cap, st);
  if (ev4) record_event(ev4[3], st);
  if (launches) *launches += 5;
  return e;
}

cudaError_t launch_trim(const QueryDev& q, const Scratch& s, int sms, cudaStream_t st,
                        int* launches) {
  k_trim_prep<<<1, 32, 0, st>>>(q, s);
  k_trim_copy<<<2 * sms, 256, 0, st>>>(q);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

}  // namespace lms
