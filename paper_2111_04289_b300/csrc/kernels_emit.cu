// Watermark, emission items, window assembly and row emission, and the carry
// of still-open panes into the next micro-batch.
//
// After a micro-batch the watermark is max(previous, max ts of the batch -
// allowed lateness); every window whose end is <= the watermark closes (the
// paper's per-micro-batch output step, Section III-A; window semantics as in
// the public header).  Rows of all closed windows are written in
// (window_start, key) order.
//
// The window state is sorted by (block, key, pane) with blocks of B >= K panes
// (lms_internal.h).  Closed windows are emitted by "items": an item is a run
// of up to 64 consecutive window ids that start in one block b, so every
// window of the item covers panes of blocks b and b + 1 only.  Both blocks
// are key-major runs of the state; the CTA that takes an item merges the two
// runs by key (merge path, chunks of 1024 entries through shared memory) and
// gives each distinct key to one thread.  The thread walks the key's groups
// (in pane order) once to find the windows of the item that hold the key (a
// 64-bit mask), and the warp's ballots over the masks give every row its rank
// among the window's keys, so the rows of one window and one warp land at
// consecutive positions; then the thread combines, for each of its windows,
// the groups whose pane lies in the window and writes the row.  Each group is
// read by the threads of at most two items (instead of once per window that
// holds it), and no per-window key list is built.
//
// An item's row count is found first (the same merge; each group is the key's
// first group in the windows between its previous pane + 1 and its own pane,
// added to a difference array over the item's windows), then the item's row
// offset comes from a decoupled look-back over the items before it.
#include <climits>

#include "lms_device.cuh"

namespace lms {
namespace {

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
  c->rows_batch = 0ull;
  c->n_items = 0ull;
  c->item_ticket = 0ull;
  c->err &= ~kErrNeedRetry;
}

// ---- emission items ----------------------------------------------------------

// Items anchored at block index j: the window chunks c (windows [c*nw, c*nw +
// nw)) whose windows touch block blk_id[j] but not block blk_id[j - 1],
// clipped to the windows this batch closes, [cursor, w_hi].  A window w covers
// panes [w, w + K - 1], so it touches block P iff P*B - K + 1 <= w <= P*B + B - 1.
__device__ __forceinline__ void block_items(const QueryDev& q, const Scratch& s, const QCtl* c,
                                            unsigned long long j, long long* lo, long long* hi) {
  *lo = 1;
  *hi = 0;
  if (c->w_hi < c->cursor) return;
  const long long B = 1ll << q.lb, NW = q.nw;
  const long long P = (long long)s.blk_id[j];
  long long a = P * B - q.k + 1;
  a = (a < 0 ? 0 : a) / NW;
  long long b = (P * B + B - 1) / NW;
  if (j > 0) {
    const long long prev = ((long long)s.blk_id[j - 1] * B + B - 1) / NW + 1;
    a = a > prev ? a : prev;
  }
  const long long cl = c->cursor / NW, ch = c->w_hi / NW;
  *lo = a > cl ? a : cl;
  *hi = b < ch ? b : ch;
}

__global__ void __launch_bounds__(256) k_item_count(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  unsigned long long lo, hi;
  chunk_range(c->n_blocks, blockIdx.x, gridDim.x, &lo, &hi);
  unsigned long long cnt = 0;
  for (unsigned long long j = lo + threadIdx.x; j < hi; j += blockDim.x) {
    long long a, b;
    block_items(q, s, c, j, &a, &b);
    if (b >= a) cnt += (unsigned long long)(b - a + 1);
  }
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  block_excl_scan(cnt, tmp, &tot);
  if (threadIdx.x == 0) s.chunk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_item_scan(const QueryDev q, const Scratch s) {
  __shared__ unsigned long long tmp[33];
  const unsigned long long v = (int)threadIdx.x < kGrid ? s.chunk[threadIdx.x] : 0ull;
  unsigned long long tot;
  const unsigned long long r = block_excl_scan(v, tmp, &tot);
  if ((int)threadIdx.x < kGrid) s.chunk[threadIdx.x] = r;
  if (threadIdx.x == 0) {
    q.ctl->n_items = tot;
    if (tot > s.item_cap) atomicOr(&q.ctl->err, kErrItemOverflow);
  }
}

__global__ void __launch_bounds__(256) k_item_write(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  if (c->n_items > s.item_cap) return;
  unsigned long long lo, hi;
  chunk_range(c->n_blocks, blockIdx.x, gridDim.x, &lo, &hi);
  __shared__ unsigned long long tmp[33];
  unsigned long long out = s.chunk[blockIdx.x];
  for (unsigned long long j0 = lo; j0 < hi; j0 += blockDim.x) {
    const unsigned long long j = j0 + threadIdx.x;
    long long a = 1, b = 0;
    if (j < hi) block_items(q, s, c, j, &a, &b);
    const unsigned long long cnt = b >= a ? (unsigned long long)(b - a + 1) : 0ull;
    unsigned long long tot;
    const unsigned long long r = block_excl_scan(cnt, tmp, &tot);
    for (unsigned long long t = 0; t < cnt; ++t) {
      s.item_c[out + r + t] = (unsigned long long)(a + (long long)t);
      s.item_j[out + r + t] = (unsigned)j;
      s.item_stat[out + r + t] = 0ull;
    }
    out += tot;
  }
}

// ---- rows --------------------------------------------------------------------

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
    // FMA remainders; a non-finite sum (a group holding Inf or NaN) has no
    // remainder to correct (Inf - Inf would turn the quotient into NaN)
    const double n = (double)cnt;
    const double r = (double)__frcp_rn((float)cnt);
    const double q0 = sd * r;
    if (!isfinite(sd)) {
      avg = q0;
    } else {
      const double q1 = fma(fma(-q0, n, sd), r, q0);
      avg = fma(fma(-q1, n, sd), r, q1);
    }
  } else {
    avg = sd / (double)cnt;  // int sums: exact division (bit-exact rows)
  }
  unsigned mnv = 0u, mxv = 0u;
  if (q.agg_mask & 4u) mnv = FLOAT ? dec_f32_bits(mn) : (unsigned)dec_i32(mn);
  if (q.agg_mask & 8u) mxv = FLOAT ? dec_f32_bits(mx) : (unsigned)dec_i32(mx);
  // rows are written once and read only by the host: streaming stores, so
  // that they do not displace the state groups the next items read
  uint4* o = reinterpret_cast<uint4*>(out);
  __stcs(o, make_uint4((unsigned)wstart, (unsigned)((unsigned long long)wstart >> 32),
                       (unsigned)cnt, (unsigned)((unsigned long long)cnt >> 32)));
  const unsigned long long ab = (unsigned long long)__double_as_longlong(avg);
  __stcs(o + 1,
         make_uint4((unsigned)sbits, (unsigned)(sbits >> 32), (unsigned)ab, (unsigned)(ab >> 32)));
  __stcs(o + 2, make_uint4(key, mnv, mxv, (unsigned)q.qid));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Decoupled look-back over the items before `ri` (items are taken in ticket
// order, so every predecessor is already running or done).  Publishes this
// item's row count, waits (bounded by limit_ns) for the predecessors' counts
// and returns the exclusive prefix, or ~0 after setting kErrLookback.
__device__ unsigned long long item_lookback(unsigned long long* stat, unsigned long long ri,
                                            unsigned long long n, QCtl* c,
                                            unsigned long long limit_ns) {
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
      if ((++spins & 63u) == 0 && global_ns() - t0 > limit_ns) {
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

// ---- assembly of an item's windows -------------------------------------------

constexpr int kEmT = 256;              // threads per CTA
constexpr int kEmE = 4;                // merged entries per thread and chunk
constexpr int kEmC = kEmT * kEmE;      // merged entries per chunk
constexpr int kEmWarps = kEmT / 32;

struct EmSmem {
  unsigned long long ga[kEmC];         // the chunk's gkeys from run A (block b)
  unsigned long long gb[kEmC];         // ... and from run B (block b + 1)
  unsigned hk[kEmC + 1];               // distinct keys starting in the chunk (heads)
  unsigned hia[kEmC + 1];              // their first A / B entries (relative to the runs)
  unsigned hib[kEmC + 1];
  unsigned long long split[kEmT + 1];  // merge-path A counts at chunk starts
  long long cnt[kMaxItemWindows + 2];  // difference array, then rows per window
  unsigned long long woff[kMaxItemWindows + 1];  // rows of the item before window i
  unsigned wc[kEmWarps][kMaxItemWindows];        // per-warp rows of a round, then their offsets
  unsigned long long run[kMaxItemWindows];       // rows of window i written by earlier rounds
  unsigned tkey[kEmT];                 // each thread's last merged entry of the chunk
  unsigned long long tpane[kEmT];
  unsigned long long tmp[33];
  unsigned carry_key;                  // the previous chunk's last entry
  unsigned long long carry_pane;
  int carry_valid;
  unsigned nh;
  unsigned long long ri, off, total;
};

struct Item {
  const Grp* A;               // run A: block b, key-major (may be empty)
  unsigned long long na;
  const Grp* Bv;              // run B: block b + 1 (empty if the item's windows do not reach it)
  unsigned long long nb;
  long long wlo, whi;         // the item's closed windows (relative ids, inclusive)
};

__device__ __forceinline__ Item load_item(const QueryDev& q, const Scratch& s, const QCtl* c,
                                          unsigned long long ii) {
  Item it;
  const long long cc = (long long)s.item_c[ii];
  const unsigned long long ja = s.item_j[ii];
  const unsigned long long nblk = c->n_blocks;
  const long long w0 = cc * q.nw;
  const unsigned long long b = (unsigned long long)w0 >> q.lb;
  it.wlo = w0 > c->cursor ? w0 : c->cursor;
  it.whi = w0 + q.nw - 1 < c->w_hi ? w0 + q.nw - 1 : c->w_hi;
  unsigned long long jb = ja;
  it.A = q.state;
  it.na = 0;
  if (ja < nblk && s.blk_id[ja] == b) {
    const unsigned long long a0 = s.blk_begin[ja];
    it.A = q.state + a0;
    it.na = s.blk_begin[ja + 1] - a0;
    jb = ja + 1;
  }
  it.Bv = q.state;
  it.nb = 0;
  const long long last_pane = it.whi + q.k - 1;
  if (q.k > 1 && jb < nblk && s.blk_id[jb] == b + 1 &&
      last_pane >= (long long)((b + 1) << q.lb)) {
    const unsigned long long b0 = s.blk_begin[jb];
    it.Bv = q.state + b0;
    it.nb = s.blk_begin[jb + 1] - b0;
  }
  return it;
}

// Merge order of the two runs: by key; on equal keys run A first.  Number of
// A entries among the first d merged entries (merge path, global memory).
__device__ unsigned long long merge_split_g(const Item& it, unsigned long long d, int lb) {
  unsigned long long lo = d > it.nb ? d - it.nb : 0ull, hi = d < it.na ? d : it.na;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if (gkey_key(it.A[mid].gkey, lb) <= gkey_key(it.Bv[d - 1 - mid].gkey, lb)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The same within a chunk staged in shared memory.
__device__ __forceinline__ unsigned merge_split_s(const unsigned long long* ga, unsigned la,
                                                  const unsigned long long* gb, unsigned lbn,
                                                  unsigned d, int lb) {
  unsigned lo = d > lbn ? d - lbn : 0u, hi = d < la ? d : la;
  while (lo < hi) {
    const unsigned mid = (lo + hi) >> 1;
    if (gkey_key(ga[mid], lb) <= gkey_key(gb[d - 1 - mid], lb)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Windows of the item [wlo, whi] that contain pane p, as bits relative to wlo.
__device__ __forceinline__ unsigned long long pane_windows(long long p, int k, long long wlo,
                                                           long long whi) {
  long long lo = p - k + 1, hi = p;
  lo = lo > wlo ? lo : wlo;
  hi = hi < whi ? hi : whi;
  if (lo > hi) return 0ull;
  const int width = (int)(hi - lo + 1);
  const unsigned long long m = width >= 64 ? ~0ull : ((1ull << width) - 1ull);
  return m << (int)(lo - wlo);
}

// One merged chunk of an item: thread t receives entries t*E .. t*E + E - 1
// of the chunk (key, pane, and the positions in A and B before the entry).
struct Merged {
  unsigned key[kEmE];
  unsigned long long pane[kEmE];
  unsigned ia[kEmE], ib[kEmE];
  int n;
};

// Walks chunk by chunk over the merged runs of the item, calling
// f(chunk_len, merged) with every thread's entries after a barrier that made
// each thread's last entry visible in sm.tkey / sm.tpane; sm.carry_* holds the
// previous chunk's last entry.  f must end with a barrier.
template <class F>
__device__ void for_merged_chunks(const QueryDev& q, const Item& it, EmSmem& sm, F f) {
  const int tid = threadIdx.x;
  const int lb = q.lb;
  const unsigned long long L = it.na + it.nb;
  const unsigned long long nch = (L + kEmC - 1) / kEmC;
  if (tid == 0) sm.carry_valid = 0;
  for (unsigned long long k0 = 0; k0 < nch; k0 += kEmT) {
    const unsigned long long kn = nch - k0 < (unsigned long long)kEmT ? nch - k0 : kEmT;
    __syncthreads();  // the previous batch of chunks no longer reads sm.split
    for (unsigned long long t = tid; t <= kn; t += kEmT) {
      const unsigned long long d = (k0 + t) * kEmC;
      sm.split[t] = merge_split_g(it, d < L ? d : L, lb);
    }
    __syncthreads();
    for (unsigned long long kk = 0; kk < kn; ++kk) {
      const unsigned long long d0 = (k0 + kk) * kEmC;
      const unsigned long long d1 = d0 + kEmC < L ? d0 + kEmC : L;
      const unsigned long long a0 = sm.split[kk], a1 = sm.split[kk + 1];
      const unsigned long long b0 = d0 - a0, b1 = d1 - a1;
      const unsigned la = (unsigned)(a1 - a0), lbn = (unsigned)(b1 - b0);
      for (unsigned i = tid; i < la; i += kEmT) sm.ga[i] = it.A[a0 + i].gkey;
      for (unsigned i = tid; i < lbn; i += kEmT) sm.gb[i] = it.Bv[b0 + i].gkey;
      __syncthreads();
      Merged m;
      m.n = 0;
      const unsigned len = la + lbn, d = (unsigned)tid * kEmE;
      if (d < len) {
        unsigned i = merge_split_s(sm.ga, la, sm.gb, lbn, d, lb), j = d - i;
#pragma unroll
        for (int e = 0; e < kEmE; ++e) {
          if (d + e < len) {
            const bool ta = j >= lbn || (i < la && gkey_key(sm.ga[i], lb) <= gkey_key(sm.gb[j], lb));
            const unsigned long long g = ta ? sm.ga[i] : sm.gb[j];
            m.key[e] = gkey_key(g, lb);
            m.pane[e] = gkey_pane(g, lb);
            m.ia[e] = (unsigned)(a0 + i);
            m.ib[e] = (unsigned)(b0 + j);
            if (ta) ++i; else ++j;
            m.n = e + 1;
          }
        }
        sm.tkey[tid] = m.key[m.n - 1];
        sm.tpane[tid] = m.pane[m.n - 1];
      }
      __syncthreads();
      f(len, m);
      // f ended with a barrier: the chunk's last entry becomes the carry
      if (len > 0 && (unsigned)tid == (len - 1) / kEmE) {
        sm.carry_key = m.key[m.n - 1];
        sm.carry_pane = m.pane[m.n - 1];
        sm.carry_valid = 1;
      }
    }
  }
  __syncthreads();
}

// The entry before merged entry e of this thread (key, pane), if any.
__device__ __forceinline__ bool prev_entry(const EmSmem& sm, const Merged& m, int e, unsigned* key,
                                           unsigned long long* pane) {
  if (e > 0) {
    *key = m.key[e - 1];
    *pane = m.pane[e - 1];
    return true;
  }
  if (threadIdx.x > 0) {
    *key = sm.tkey[threadIdx.x - 1];
    *pane = sm.tpane[threadIdx.x - 1];
    return true;
  }
  *key = sm.carry_key;
  *pane = sm.carry_pane;
  return sm.carry_valid != 0;
}

// Rows of each window of the item: a group is its key's first group in the
// windows from max(previous pane of the key + 1, pane - K + 1) to its pane.
__device__ void count_item(const QueryDev& q, const Item& it, EmSmem& sm) {
  const int nw = (int)(it.whi - it.wlo + 1);
  for (int i = threadIdx.x; i <= nw; i += kEmT) sm.cnt[i] = 0;
  if (q.k == 1) {  // tumbling: one window, one pane, unique keys
    __syncthreads();
    if (threadIdx.x == 0) sm.cnt[0] = (long long)it.na;
  } else {
    for_merged_chunks(q, it, sm, [&](unsigned, const Merged& m) {
      for (int e = 0; e < m.n; ++e) {
        unsigned pk;
        unsigned long long pp;
        long long lo = (long long)m.pane[e] - q.k + 1;
        if (prev_entry(sm, m, e, &pk, &pp) && pk == m.key[e]) {
          const long long after = (long long)pp + 1;
          lo = lo > after ? lo : after;
        }
        long long hi = (long long)m.pane[e];
        lo = lo > it.wlo ? lo : it.wlo;
        hi = hi < it.whi ? hi : it.whi;
        if (lo <= hi) {
          atomicAdd(reinterpret_cast<unsigned long long*>(&sm.cnt[lo - it.wlo]), 1ull);
          atomicAdd(reinterpret_cast<unsigned long long*>(&sm.cnt[hi - it.wlo + 1]), ~0ull);
        }
      }
      __syncthreads();
    });
    if (threadIdx.x == 0) {
      long long acc = 0;
      for (int i = 0; i < nw; ++i) {
        acc += sm.cnt[i];
        sm.cnt[i] = acc;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long acc = 0;
    for (int i = 0; i < nw; ++i) {
      sm.woff[i] = acc;
      acc += (unsigned long long)sm.cnt[i];
    }
    sm.total = acc;
  }
  __syncthreads();
}

// End (exclusive) of the run of key k in g[from, n): galloping, then binary search.
__device__ unsigned long long run_end(const Grp* g, unsigned long long from, unsigned long long n,
                                      unsigned k, int lb) {
  if (from >= n || gkey_key(g[from].gkey, lb) != k) return from;
  unsigned long long lo = from, step = 1;  // key(lo) == k
  while (lo + step < n && gkey_key(g[lo + step].gkey, lb) == k) {
    lo += step;
    step <<= 1;
  }
  unsigned long long hi = lo + step < n ? lo + step : n;
  while (hi - lo > 1) {
    const unsigned long long mid = lo + ((hi - lo) >> 1);
    if (gkey_key(g[mid].gkey, lb) == k) lo = mid;
    else hi = mid;
  }
  return hi;
}

// Writes the item's rows from out[0]: rows of window i from out[woff[i]], in
// key order.
template <bool FLOAT>
__device__ void write_item(const QueryDev& q, const Item& it, EmSmem& sm, ResultRowDev* out) {
  const int tid = threadIdx.x, w = tid >> 5;
  const unsigned lane = lane_id(), lt = (1u << lane) - 1u;
  const int lb = q.lb, K = q.k;
  const int nw = (int)(it.whi - it.wlo + 1);
  if (K == 1) {  // tumbling: the rows are the pane's groups, in key order
    const long long wstart = (it.wlo - kPaneBias) * (long long)q.slide + q.base;
    for (unsigned long long i = tid; i < it.na; i += kEmT) {
      const Grp g = load_grp_v(it.A + i);
      write_row<FLOAT>(q, out + i, wstart, gkey_key(g.gkey, lb), g.cnt, g.sum, g.mn, g.mx);
    }
    __syncthreads();
    return;
  }
  for (int i = tid; i < nw; i += kEmT) sm.run[i] = 0ull;
  for_merged_chunks(q, it, sm, [&](unsigned len, const Merged& m) {
    // heads: the entries that start a key
    unsigned nh_t = 0;
    bool head[kEmE];
#pragma unroll
    for (int e = 0; e < kEmE; ++e) {
      head[e] = false;
      if (e < m.n) {
        unsigned pk;
        unsigned long long pp;
        head[e] = !(prev_entry(sm, m, e, &pk, &pp) && pk == m.key[e]);
        nh_t += head[e] ? 1u : 0u;
      }
    }
    unsigned long long htot;
    unsigned long long hpos = block_excl_scan((unsigned long long)nh_t, sm.tmp, &htot);
#pragma unroll
    for (int e = 0; e < kEmE; ++e) {
      if (head[e]) {
        sm.hk[hpos] = m.key[e];
        sm.hia[hpos] = m.ia[e];
        sm.hib[hpos] = m.ib[e];
        ++hpos;
      }
    }
    (void)len;
    __syncthreads();
    const unsigned nh = (unsigned)htot;
    if (tid == 0 && nh > 0) {  // the last key may continue past the chunk
      const unsigned k = sm.hk[nh - 1];
      sm.hia[nh] = (unsigned)run_end(it.A, sm.hia[nh - 1], it.na, k, lb);
      sm.hib[nh] = (unsigned)run_end(it.Bv, sm.hib[nh - 1], it.nb, k, lb);
    }
    __syncthreads();
    for (unsigned r0 = 0; r0 < nh; r0 += kEmT) {
      const unsigned h = r0 + (unsigned)tid;
      const bool valid = h < nh;
      unsigned key = 0u, ia = 0u, na_k = 0u, ib = 0u, nb_k = 0u;
      unsigned long long mask = 0ull;
      if (valid) {
        key = sm.hk[h];
        ia = sm.hia[h];
        ib = sm.hib[h];
        na_k = sm.hia[h + 1] - ia;
        nb_k = sm.hib[h + 1] - ib;
        for (unsigned e = 0; e < na_k; ++e)
          mask |= pane_windows((long long)gkey_pane(it.A[ia + e].gkey, lb), K, it.wlo, it.whi);
        for (unsigned e = 0; e < nb_k; ++e)
          mask |= pane_windows((long long)gkey_pane(it.Bv[ib + e].gkey, lb), K, it.wlo, it.whi);
      }
      // rows of this warp per window, then their offsets over the warps
      sm.wc[w][lane] = 0u;
      sm.wc[w][lane + 32] = 0u;
      const unsigned long long orm =
          ((unsigned long long)__reduce_or_sync(kFull, (unsigned)(mask >> 32)) << 32) |
          __reduce_or_sync(kFull, (unsigned)mask);
      __syncwarp();
      for (unsigned long long bits = orm; bits; bits &= bits - 1) {
        const int i = __ffsll((long long)bits) - 1;
        const unsigned bal = __ballot_sync(kFull, (mask >> i) & 1ull);
        if (lane == 0) sm.wc[w][i] = (unsigned)__popc(bal);
      }
      __syncthreads();
      for (int i = tid; i < nw; i += kEmT) {  // warp offsets inside window i
        unsigned acc = (unsigned)sm.run[i];
#pragma unroll
        for (int ww = 0; ww < kEmWarps; ++ww) {
          const unsigned t = sm.wc[ww][i];
          sm.wc[ww][i] = acc;
          acc += t;
        }
        sm.run[i] = acc;
      }
      __syncthreads();
      // the rows: per window of the key, combine its groups in the window
      const unsigned n_k = na_k + nb_k;
      unsigned lo = 0u, hi = 0u;
      for (unsigned long long bits = orm; bits; bits &= bits - 1) {
        const int i = __ffsll((long long)bits) - 1;
        const bool mine = (mask >> i) & 1ull;
        const unsigned bal = __ballot_sync(kFull, mine);
        if (!mine) continue;
        const long long W = it.wlo + i;
        auto entry = [&](unsigned e) -> const Grp* {
          return e < na_k ? it.A + ia + e : it.Bv + ib + (e - na_k);
        };
        while (lo < n_k && (long long)gkey_pane(entry(lo)->gkey, lb) < W) ++lo;
        if (hi < lo) hi = lo;
        while (hi < n_k && (long long)gkey_pane(entry(hi)->gkey, lb) <= W + K - 1) ++hi;
        if (lo >= hi) continue;  // cannot happen: the mask says a group lies in the window
        const Grp g0 = load_grp_v(entry(lo));
        long long cnt = g0.cnt;
        unsigned long long isum = g0.sum;
        double fsum = __longlong_as_double((long long)g0.sum);
        unsigned mn = g0.mn, mx = g0.mx;
        for (unsigned e = lo + 1; e < hi; ++e) {
          const Grp g = load_grp_v(entry(e));
          cnt += g.cnt;
          mn = min(mn, g.mn);
          mx = max(mx, g.mx);
          if (FLOAT) fsum += __longlong_as_double((long long)g.sum);
          else isum += g.sum;
        }
        const unsigned long long sb = FLOAT ? (unsigned long long)__double_as_longlong(fsum) : isum;
        const unsigned long long pos =
            sm.woff[i] + sm.wc[w][i] + (unsigned)__popc(bal & lt);
        const long long wstart = (W - kPaneBias) * (long long)q.slide + q.base;
        write_row<FLOAT>(q, out + pos, wstart, key, cnt, sb, mn, mx);
      }
      __syncthreads();
    }
  });
}

// Emits the closed windows.  CTAs take items in ticket order; for each item:
// its rows per window (count_item), its row offset by the look-back, then the
// rows (write_item).
template <bool FLOAT>
__global__ void __launch_bounds__(kEmT, 3)
    k_emit(const QueryDev q, const Scratch s, ResultRowDev* rows, unsigned long long rows_cap) {
  __shared__ EmSmem sm;
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long NI = c->n_items;
  const unsigned long long row_base = c->row_base;
  while (true) {
    if (threadIdx.x == 0) sm.ri = atomicAdd(&c->item_ticket, 1ull);
    __syncthreads();
    const unsigned long long ri = sm.ri;
    __syncthreads();
    if (ri >= NI) break;
    const Item it = load_item(q, s, c, ri);
    if (ri == 0 && (q.debug_flags & kDebugHoldFirstItem)) continue;  // never publishes
    count_item(q, it, sm);
    if (threadIdx.x == 0) {
      const unsigned long long n = sm.total;
      const unsigned long long off = item_lookback(s.item_stat, ri, n, c, q.lookback_ns);
      sm.off = off;
      if (off != ~0ull) {
        if (ri == NI - 1) c->rows_batch = off + n;
        if (row_base + off + n > rows_cap) atomicOr(&c->err, kErrRowsOverflow);
      }
    }
    __syncthreads();
    const unsigned long long off = sm.off;
    __syncthreads();
    if (off != ~0ull && row_base + off + sm.total <= rows_cap)
      write_item<FLOAT>(q, it, sm, rows + row_base + off);
    __syncthreads();
  }
}

// ---- carry the panes that stay open into the next batch's partial arrays --

// Advances the cursor past the closed windows and finds where the groups that
// may stay open start: the first block that holds panes >= the new cursor.
__global__ void k_trim_prep(const QueryDev q, const Scratch s) {
  if (threadIdx.x != 0) return;
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  c->row_base += c->rows_batch;
  if (c->w_hi >= c->cursor) c->cursor = c->w_hi + 1;
  const unsigned long long bstar = (unsigned long long)c->cursor >> q.lb;
  const unsigned long long P = c->n_blocks;
  unsigned long long lo = 0, hi = P;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if ((unsigned long long)s.blk_id[mid] < bstar) lo = mid + 1; else hi = mid;
  }
  c->trim_from = lo < P ? s.blk_begin[lo] : c->n_state;
  c->or_mask = 0ull;
  c->and_mask = ~0ull;
}

// Groups at or after trim_from whose pane is still open (pane >= cursor),
// counted per chunk; then written, in order, to the front of the partial
// arrays.
__device__ __forceinline__ bool keep_group(const QueryDev& q, const QCtl* c, unsigned long long g) {
  return (long long)gkey_pane(g, q.lb) >= c->cursor;
}

__global__ void __launch_bounds__(256) k_trim_count(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long from = c->trim_from, n = c->n_state - from;
  unsigned long long lo, hi;
  chunk_range(n, blockIdx.x, gridDim.x, &lo, &hi);
  unsigned long long cnt = 0;
  for (unsigned long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
    cnt += keep_group(q, c, q.state[from + i].gkey) ? 1ull : 0ull;
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  block_excl_scan(cnt, tmp, &tot);
  if (threadIdx.x == 0) s.chunk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_trim_scan(const QueryDev q, const Scratch s) {
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  __shared__ unsigned long long tmp[33];
  unsigned long long x[4], sum = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = 4 * (int)threadIdx.x + u;
    x[u] = i < kGrid ? s.chunk[i] : 0ull;
    sum += x[u];
  }
  unsigned long long tot;
  unsigned long long r = block_excl_scan(sum, tmp, &tot);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = 4 * (int)threadIdx.x + u;
    if (i < kGrid) s.chunk[i] = r;
    r += x[u];
  }
  if (threadIdx.x == 0) {
    c->carried = tot;
    c->n_parts = tot;
  }
}

__global__ void __launch_bounds__(256) k_trim_write(const QueryDev q, const Scratch s) {
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long from = c->trim_from, n = c->n_state - from;
  unsigned long long lo, hi;
  chunk_range(n, blockIdx.x, gridDim.x, &lo, &hi);
  __shared__ unsigned long long tmp[33];
  unsigned long long out = s.chunk[blockIdx.x];
  unsigned long long o_acc = 0ull, a_acc = ~0ull;
  for (unsigned long long i0 = lo; i0 < hi; i0 += blockDim.x) {
    const unsigned long long i = i0 + threadIdx.x;
    Grp g;
    bool keep = false;
    if (i < hi) {
      g = load_grp(q.state + from + i);
      keep = keep_group(q, c, g.gkey);
    }
    unsigned long long tot;
    const unsigned long long r = block_excl_scan(keep ? 1ull : 0ull, tmp, &tot);
    if (keep) {
      store_grp(q.parts + out + r, g.gkey, g.cnt, g.sum, g.mn, g.mx);
      q.pkeys[out + r] = g.gkey;
      o_acc |= g.gkey;
      a_acc &= g.gkey;
    }
    out += tot;
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

}  // namespace

void set_block_shape(QueryDev* d) {
  int lb = 0;
  while ((1 << lb) < d->k) ++lb;
  d->lb = lb;
  d->nw = (1 << lb) < kMaxItemWindows ? (1 << lb) : kMaxItemWindows;
}

cudaError_t set_smem_limit(const void* fn, int bytes, unsigned long long* done_mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(done_mask, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) __atomic_fetch_or(done_mask, bit, __ATOMIC_ACQ_REL);
  return e;
}

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

// ev4 (optional): events recorded before/after the item list and before/after
// the row kernel.
cudaError_t launch_emit(const QueryDev& q, const Scratch& s, ResultRowDev* rows,
                        unsigned long long rows_cap, int sms, cudaStream_t st, int* launches,
                        cudaEvent_t* ev4) {
  if (ev4) record_event(ev4[0], st);
  k_emit_begin<<<1, 32, 0, st>>>(q.ctl);
  k_item_count<<<kGrid, 256, 0, st>>>(q, s);
  k_item_scan<<<1, 1024, 0, st>>>(q, s);
  k_item_write<<<kGrid, 256, 0, st>>>(q, s);
  if (ev4) {
    record_event(ev4[1], st);
    record_event(ev4[2], st);
  }
  const int grid = 3 * sms;
  if (q.value_is_float) k_emit<true><<<grid, kEmT, 0, st>>>(q, s, rows, rows_cap);
  else k_emit<false><<<grid, kEmT, 0, st>>>(q, s, rows, rows_cap);
  if (ev4) record_event(ev4[3], st);
  if (launches) *launches += 5;
  return cudaGetLastError();
}

cudaError_t launch_trim(const QueryDev& q, const Scratch& s, int sms, cudaStream_t st,
                        int* launches) {
  (void)sms;
  k_trim_prep<<<1, 32, 0, st>>>(q, s);
  k_trim_count<<<kGrid, 256, 0, st>>>(q, s);
  k_trim_scan<<<1, 256, 0, st>>>(q, s);
  k_trim_write<<<kGrid, 256, 0, st>>>(q, s);
  if (launches) *launches += 4;
  return cudaGetLastError();
}

}  // namespace lms
