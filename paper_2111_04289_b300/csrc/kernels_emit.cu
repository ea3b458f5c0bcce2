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
// are key-major runs of the state; merged by key (merge path) they give every
// key's groups of the item in pane order.  An item's merged runs are cut at
// key boundaries into units of about 32K entries, and every unit is one CTA's
// work: it stages its merged entries chunk by chunk in shared memory, finds
// for each distinct key the windows of the item that hold it (a bit mask over
// the item's windows) and writes the key's row of each such window, combining
// the key's groups whose pane lies in the window.  Warp ballots over the masks
// give every row its rank among the window's keys, so the rows of one window
// and one warp land at consecutive positions.  Each group is read by the
// units of at most two items (instead of once per window that holds it).
//
// The output positions come first: k_emit_count finds every unit's rows per
// window (the same merge; each group is the key's first group in the windows
// between its previous pane + 1 and its own pane, added to a difference array
// over the item's windows), one exclusive scan over those counts laid out in
// (item, window, unit) order gives every (unit, window) its first output row,
// and k_emit_write writes the rows.  No CTA waits on another.
#include <climits>

#include "lms_device.cuh"

namespace lms {
namespace {

__device__ __forceinline__ long long floor_div_ll(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

__global__ void k_batch_begin(SCtl* sc, long long ts_floor, QCtl* c0, QCtl* c1, QCtl* c2,
                              QCtl* c3, QCtl* c4, QCtl* c5, QCtl* c6, QCtl* c7) {
  if (threadIdx.x != 0) return;
  sc->batch_max_ts = ts_floor;  // LLONG_MIN, or a watermark hint for the batch
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
  c->unit_ticket = 0ull;
  c->err &= ~kErrNeedRetry;
}

struct Item {
  const Grp* A;               // run A: block b, key-major (may be empty)
  unsigned long long na;
  const Grp* Bv;              // run B: block b + 1 (empty if the item's windows do not reach it)
  unsigned long long nb;
  long long wlo, whi;         // the item's closed windows (relative ids, inclusive)
  // the unit of the item (key-aligned range of its merged runs) one CTA takes
  unsigned long long a_lo, b_lo, a_hi, b_hi;  // A / B entries before the unit's start / end
  unsigned sub, nsub;         // the unit's index in the item, the item's units
};

// The runs of the item of window chunk cc anchored at block index ja.
__device__ __forceinline__ Item load_item(const QueryDev& q, const Scratch& s, const QCtl* c,
                                          long long cc, unsigned long long ja) {
  Item it;
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
  it.a_lo = it.b_lo = 0;
  it.a_hi = it.na;
  it.b_hi = it.nb;
  it.sub = 0;
  it.nsub = 1;
  return it;
}

// Merged entries per unit: an item's merged runs are cut into units of about
// this many entries (at key boundaries), so that a few closed windows over a
// large state still spread over the whole GPU.  A unit is one CTA's work on
// the general path and one warp's on the pane-word path (2B <= 32).
constexpr unsigned long long kUnitEntries = 32768;
constexpr unsigned long long kUnitEntriesPW = (unsigned long long)kPwChunkEntries * kPwUnitChunks;

__device__ __forceinline__ bool pane_word_path(const QueryDev& q) { return (2 << q.lb) <= 32; }

__device__ __forceinline__ unsigned long long unit_entries(const QueryDev& q) {
  return pane_word_path(q) ? kUnitEntriesPW : kUnitEntries;
}

__device__ __forceinline__ unsigned item_units(const QueryDev& q, const Item& it) {
  const unsigned long long L = it.na + it.nb, E = unit_entries(q);
  return L == 0 ? 1u : (unsigned)((L + E - 1) / E);
}

// Merge order of the two runs: by key; on equal keys run A first (its panes
// are the earlier ones).  Number of A entries among the first d merged
// entries (merge path, global memory).
__device__ unsigned long long merge_split_g(const Item& it, unsigned long long d, int lb) {
  unsigned long long lo = d > it.nb ? d - it.nb : 0ull, hi = d < it.na ? d : it.na;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if (gkey_key(it.A[mid].gkey, lb) <= gkey_key(it.Bv[d - 1 - mid].gkey, lb)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// First index of key k in g[lo, hi) (g is key-ordered there).
__device__ __forceinline__ unsigned long long key_lower_bound(const Grp* g, unsigned long long lo,
                                                              unsigned long long hi, unsigned k,
                                                              int lb) {
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if (gkey_key(g[mid].gkey, lb) < k) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Key-aligned merge split at merged position d: (A entries, B entries) before
// the first group of the key of merged entry d (d itself at 0 and L).  A key
// has at most B groups in each run, so the lower bounds search that far back.
__device__ __forceinline__ void aligned_split(const Item& it, unsigned long long d, int lb,
                                              unsigned long long* pa, unsigned long long* pb) {
  unsigned long long a = merge_split_g(it, d, lb), b = d - a;
  if (d > 0 && d < it.na + it.nb) {
    const unsigned ka = a < it.na ? gkey_key(it.A[a].gkey, lb) : 0xffffffffu;
    const unsigned kb = b < it.nb ? gkey_key(it.Bv[b].gkey, lb) : 0xffffffffu;
    const bool from_a = a < it.na && (b >= it.nb || ka <= kb);
    const unsigned k = from_a ? ka : kb;
    const unsigned long long span = 1ull << lb;
    a = key_lower_bound(it.A, a > span ? a - span : 0ull, a, k, lb);
    b = key_lower_bound(it.Bv, b > span ? b - span : 0ull, b, k, lb);
  }
  *pa = a;
  *pb = b;
}

// Unit u of the emission: its item's runs and its key-aligned range.
__device__ __forceinline__ Item load_unit(const QueryDev& q, const Scratch& s, const QCtl* c,
                                          unsigned long long u) {
  Item it = load_item(q, s, c, (long long)s.item_c[u], s.item_j[u]);
  const unsigned long long st = s.item_stat[u];
  it.sub = (unsigned)st;
  it.nsub = (unsigned)(st >> 32);
  const unsigned long long L = it.na + it.nb, E = unit_entries(q);
  if (it.nsub > 1) {
    const unsigned long long d0 = (unsigned long long)it.sub * E;
    const unsigned long long d1 = it.sub + 1 < it.nsub ? d0 + E : L;
    aligned_split(it, d0 < L ? d0 : L, q.lb, &it.a_lo, &it.b_lo);
    aligned_split(it, d1 < L ? d1 : L, q.lb, &it.a_hi, &it.b_hi);
  }
  return it;
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

// Units of the items anchored at block index j.
__device__ __forceinline__ unsigned long long block_units(const QueryDev& q, const Scratch& s,
                                                          const QCtl* c, unsigned long long j) {
  long long a, b;
  block_items(q, s, c, j, &a, &b);
  unsigned long long n = 0;
  for (long long cc = a; cc <= b; ++cc) n += item_units(q, load_item(q, s, c, cc, j));
  return n;
}

// The unit list (the "items" of the scratch): per item, item_units() units
// in order, each recorded as (window chunk, anchor block, sub | nsub << 32).
__global__ void __launch_bounds__(256) k_item_count(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  unsigned long long lo, hi;
  chunk_range(c->n_blocks, blockIdx.x, gridDim.x, &lo, &hi);
  unsigned long long cnt = 0;
  for (unsigned long long j = lo + threadIdx.x; j < hi; j += blockDim.x)
    cnt += block_units(q, s, c, j);
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
    const unsigned long long cnt = j < hi ? block_units(q, s, c, j) : 0ull;
    unsigned long long tot;
    unsigned long long o = out + block_excl_scan(cnt, tmp, &tot);
    for (long long cc = a; cc <= b; ++cc) {
      const unsigned nsub = item_units(q, load_item(q, s, c, cc, j));
      for (unsigned t = 0; t < nsub; ++t, ++o) {
        s.item_c[o] = (unsigned long long)cc;
        s.item_j[o] = (unsigned)j;
        s.item_stat[o] = (unsigned long long)t | ((unsigned long long)nsub << 32);
      }
    }
    out += tot;
  }
}

// Pane-word path: the chunk boundaries of every unit, one thread per boundary,
// so that the warps that count and write the units search nothing.  Boundary
// t of unit (item, sub) is the key-aligned split at merged entry (sub *
// kPwUnitChunks + t) * kPwChunkEntries, or the item's end.
__global__ void __launch_bounds__(256) k_unit_bounds(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  const unsigned long long NI = c->n_items;
  if (NI > s.item_cap) return;
  const unsigned long long n = NI * (kPwUnitChunks + 1);
  for (unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long u = x / (kPwUnitChunks + 1);
    const unsigned t = (unsigned)(x - u * (kPwUnitChunks + 1));
    const Item it = load_item(q, s, c, (long long)s.item_c[u], s.item_j[u]);
    const unsigned long long sub = (unsigned)s.item_stat[u];
    const unsigned long long d = (sub * kPwUnitChunks + t) * kPwChunkEntries;
    unsigned long long a = it.na, b = it.nb;
    if (d == 0) {
      a = 0;
      b = 0;
    } else if (d < it.na + it.nb) {
      aligned_split(it, d, q.lb, &a, &b);
    }
    s.unit_bnd[u * kUnitBnd + 2 * t] = (unsigned)a;
    s.unit_bnd[u * kUnitBnd + 2 * t + 1] = (unsigned)b;
  }
}

// ---- unit row counts -> output offsets ------------------------------------------
//
// Rows come out in (window, key) order: within an item, window i's rows are
// the rows of its units in unit order.  Unit u = (item, sub) writes its
// per-window counts to the item's slice of s.unit_off, at [u0 * nw + i * nsub
// + sub] (u0: the item's first unit, nw: the query's windows per item), so
// that one exclusive scan over the whole array, in index order, gives every
// (unit, window) its output row.

__global__ void __launch_bounds__(256) k_uoff_sum(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  unsigned long long lo, hi;
  chunk_range(c->n_items * (unsigned long long)q.nw, blockIdx.x, gridDim.x, &lo, &hi);
  unsigned long long acc = 0;
  for (unsigned long long i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += s.unit_off[i];
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  block_excl_scan(acc, tmp, &tot);
  if (threadIdx.x == 0) s.chunk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_uoff_scan(const QueryDev q, const Scratch s,
                                                    unsigned long long rows_cap) {
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  __shared__ unsigned long long tmp[33];
  const unsigned long long v = (int)threadIdx.x < kGrid ? s.chunk[threadIdx.x] : 0ull;
  unsigned long long tot;
  const unsigned long long r = block_excl_scan(v, tmp, &tot);
  if ((int)threadIdx.x < kGrid) s.chunk[threadIdx.x] = r;
  if (threadIdx.x == 0) {
    c->rows_batch = tot;
    if (c->row_base + tot > rows_cap) atomicOr(&c->err, kErrRowsOverflow);
  }
}

__global__ void __launch_bounds__(256) k_uoff_write(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  unsigned long long lo, hi;
  chunk_range(c->n_items * (unsigned long long)q.nw, blockIdx.x, gridDim.x, &lo, &hi);
  __shared__ unsigned long long tmp[33];
  unsigned long long run = s.chunk[blockIdx.x];
  for (unsigned long long i0 = lo; i0 < hi; i0 += blockDim.x) {
    const unsigned long long i = i0 + threadIdx.x;
    const unsigned long long v = i < hi ? s.unit_off[i] : 0ull;
    unsigned long long tot;
    const unsigned long long r = block_excl_scan(v, tmp, &tot);
    if (i < hi) s.unit_off[i] = run + r;
    run += tot;
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

// The last two 16-byte parts of a row (sum, avg | key, min, max, query id);
// the first is (window_start, count).
template <bool FLOAT>
__device__ __forceinline__ void row_parts(const QueryDev& q, unsigned key, long long cnt,
                                          unsigned long long sbits, unsigned mn, unsigned mx,
                                          uint4* p1, uint4* p2) {
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
  const unsigned long long ab = (unsigned long long)__double_as_longlong(avg);
  *p1 = make_uint4((unsigned)sbits, (unsigned)(sbits >> 32), (unsigned)ab, (unsigned)(ab >> 32));
  *p2 = make_uint4(key, mnv, mxv, (unsigned)q.qid);
}

// Rows are written once and read only by the host: streaming stores, so that
// they do not displace the state groups the next items read.
__device__ __forceinline__ void store_row(ResultRowDev* out, long long wstart, long long cnt,
                                          const uint4& p1, const uint4& p2) {
  uint4* o = reinterpret_cast<uint4*>(out);
  __stcs(o, make_uint4((unsigned)wstart, (unsigned)((unsigned long long)wstart >> 32),
                       (unsigned)cnt, (unsigned)((unsigned long long)cnt >> 32)));
  __stcs(o + 1, p1);
  __stcs(o + 2, p2);
}

template <bool FLOAT>
__device__ __forceinline__ void write_row(const QueryDev& q, ResultRowDev* out, long long wstart,
                                          unsigned key, long long cnt, unsigned long long sbits,
                                          unsigned mn, unsigned mx) {
  uint4 p1, p2;
  row_parts<FLOAT>(q, key, cnt, sbits, mn, mx, &p1, &p2);
  store_row(out, wstart, cnt, p1, p2);
}

// ---- assembly of an item's windows -------------------------------------------

constexpr int kEmT = 256;              // threads per CTA
constexpr int kEmE = 4;                // merged entries per thread and chunk
constexpr int kEmC = kEmT * kEmE;      // merged entries per chunk
constexpr int kEmWarps = kEmT / 32;
constexpr int kEmRows = 4096;          // row descriptors per round

// Per-CTA state of the emission kernel (static shared memory); the staged
// chunk and the round's row descriptors live in dynamic shared memory (EmDyn).
struct EmSmem {
  unsigned long long split[kEmT + 1];  // merge-path A counts at chunk starts
  unsigned long long split_b[kEmT + 1];// B counts at chunk starts (key-aligned chunks)
  long long cnt[kMaxItemWindows + 2];  // rows per window
  int wdiff[kEmWarps][kMaxItemWindows + 2];      // per-warp difference arrays of the count
  unsigned long long woff[kMaxItemWindows + 1];  // rows of the item before window i
  unsigned long long base[kMaxItemWindows];      // output row of descriptor 0 of window i
  unsigned run[kMaxItemWindows];       // rows of window i written by earlier rounds
  unsigned rb[kMaxItemWindows + 1];    // first descriptor of window i in the round
  unsigned wc[kEmWarps][kMaxItemWindows];        // per-warp rows, then the warps' offsets
  unsigned ball[kEmWarps][kMaxItemWindows];      // per-warp ballots of window i
  unsigned long long tmp[33];
  unsigned long long carry_g;          // the previous chunk's last merged gkey
  unsigned long long next_carry;
  unsigned long long open_ia, open_ib; // global runs of the chunk's last key, if it continues
  unsigned open_na;
  unsigned open_kh;                    // round index of the key read from global memory, or ~0
  int carry_valid;
  unsigned open_last;                  // the chunk's last key continues past the chunk
  unsigned long long ri, off, total;
};

// A chunk staged in shared memory as columns of its records (the A part, then
// the B part), the merged order (record slot of each merged position), the
// merged positions of the keys' first entries (heads), and the round's row
// descriptors in output order: (key of the round << 6 | window), the first of
// the key's groups in the window (a merged position, or for the key read from
// global memory an index into its groups) and their number.
struct EmDyn {
  unsigned long long* gk;    // [kEmC] gkeys
  long long* cnt;            // [kEmC]
  unsigned long long* sum;   // [kEmC]
  unsigned long long* mm;    // [kEmC] mn | mx << 32
  unsigned short* mo;        // [kEmC]
  unsigned short* hp;        // [kEmC + 1]
  unsigned* rln;             // [kEmRows] first group | number of groups << 16 (general path)
  unsigned short* rows;      // [kEmRows] (general path)
};
// Dynamic shared memory of the counting kernel (no row descriptors) and of the
// writer.
constexpr size_t kEmDynBytesCount = (size_t)kEmC * (4 * 8 + 2) + (kEmC + 1) * 2 + 6;
constexpr size_t kEmDynBytes = kEmDynBytesCount + (size_t)kEmRows * (4 + 2);

__device__ __forceinline__ EmDyn em_dyn() {
  extern __shared__ __align__(16) unsigned char em_smem[];
  EmDyn d;
  unsigned char* p = em_smem;
  d.gk = reinterpret_cast<unsigned long long*>(p); p += (size_t)kEmC * 8;
  d.cnt = reinterpret_cast<long long*>(p); p += (size_t)kEmC * 8;
  d.sum = reinterpret_cast<unsigned long long*>(p); p += (size_t)kEmC * 8;
  d.mm = reinterpret_cast<unsigned long long*>(p); p += (size_t)kEmC * 8;
  d.mo = reinterpret_cast<unsigned short*>(p); p += (size_t)kEmC * 2;
  d.hp = reinterpret_cast<unsigned short*>(p); p += (size_t)(kEmC + 1) * 2 + 6;
  d.rln = reinterpret_cast<unsigned*>(p); p += (size_t)kEmRows * 4;
  d.rows = reinterpret_cast<unsigned short*>(p);
  return d;
}

// The same within a staged chunk: A part gk[0 .. la), B part gk[la .. la + lbn).
__device__ __forceinline__ unsigned merge_split_s(const unsigned long long* gk, unsigned la,
                                                  unsigned lbn, unsigned d, int lb) {
  unsigned lo = d > lbn ? d - lbn : 0u, hi = d < la ? d : la;
  while (lo < hi) {
    const unsigned mid = (lo + hi) >> 1;
    if (gkey_key(gk[mid], lb) <= gkey_key(gk[la + d - 1 - mid], lb)) lo = mid + 1;
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

// Walks chunk by chunk over the merged runs of the item.  Each chunk is
// staged (records loaded with 16-byte vector loads; only the gkeys when
// full == false) and merged into d.mo; then f(len, la, a0, b0, last) runs
// with the chunk in shared memory (after a barrier) and must end with a
// barrier.  sm.carry_g holds the previous chunk's last merged gkey (if
// sm.carry_valid).
template <class F>
__device__ void for_merged_chunks(const QueryDev& q, const Item& it, EmSmem& sm, const EmDyn& d,
                                  bool full, F f) {
  const int tid = threadIdx.x;
  const int lb = q.lb;
  // the unit's merged range [D0, D1) (it starts and ends at key boundaries)
  const unsigned long long D0 = it.a_lo + it.b_lo, D1 = it.a_hi + it.b_hi;
  const unsigned long long L = D1 - D0;
  const unsigned long long C = (unsigned long long)kEmC;
  const unsigned long long nch = (L + C - 1) / C;
  if (tid == 0) sm.carry_valid = 0;
  for (unsigned long long k0 = 0; k0 < nch; k0 += kEmT) {
    const unsigned long long kn = nch - k0 < (unsigned long long)kEmT ? nch - k0 : kEmT;
    __syncthreads();  // the previous batch of chunks no longer reads sm.split
    for (unsigned long long t = tid; t <= kn; t += kEmT) {
      const unsigned long long off = (k0 + t) * C < L ? (k0 + t) * C : L;
      unsigned long long a, b;
      if (off == 0) {
        a = it.a_lo;
        b = it.b_lo;
      } else if (off == L) {
        a = it.a_hi;
        b = it.b_hi;
      } else {
        a = merge_split_g(it, D0 + off, lb);
        b = D0 + off - a;
      }
      sm.split[t] = a;
      sm.split_b[t] = b;
    }
    __syncthreads();
    for (unsigned long long kk = 0; kk < kn; ++kk) {
      const unsigned long long a0 = sm.split[kk], a1 = sm.split[kk + 1];
      const unsigned long long b0 = sm.split_b[kk], b1 = sm.split_b[kk + 1];
      const unsigned long long d1 = a1 + b1;
      const unsigned la = (unsigned)(a1 - a0), len = (unsigned)(a1 - a0 + b1 - b0);
      if (full) {  // two 16-byte halves per record
        for (unsigned h = tid; h < 2 * len; h += kEmT) {
          const unsigned r = h >> 1;
          const Grp* src = r < la ? it.A + a0 + r : it.Bv + b0 + (r - la);
          const uint4 v = reinterpret_cast<const uint4*>(src)[h & 1];
          const unsigned long long lo = ((unsigned long long)v.y << 32) | v.x;
          const unsigned long long hi = ((unsigned long long)v.w << 32) | v.z;
          if (h & 1) {
            d.sum[r] = lo;
            d.mm[r] = hi;
          } else {
            d.gk[r] = lo;
            d.cnt[r] = (long long)hi;
          }
        }
      } else {
        for (unsigned r = tid; r < len; r += kEmT)
          d.gk[r] = r < la ? it.A[a0 + r].gkey : it.Bv[b0 + (r - la)].gkey;
      }
      __syncthreads();
      const unsigned x0 = (unsigned)tid * kEmE;
      if (x0 < len) {
        unsigned i = merge_split_s(d.gk, la, len - la, x0, lb), j = x0 - i;
        const unsigned lbn = len - la;
#pragma unroll
        for (int e = 0; e < kEmE; ++e) {
          if (x0 + e < len) {
            const bool ta = j >= lbn || (i < la && gkey_key(d.gk[i], lb) <= gkey_key(d.gk[la + j], lb));
            d.mo[x0 + e] = (unsigned short)(ta ? i : la + j);
            if (ta) ++i; else ++j;
          }
        }
      }
      __syncthreads();
      if (tid == 0) sm.next_carry = d.gk[d.mo[len - 1]];
      f(len, la, a0, b0, d1 == D1);
      // f ended with a barrier: the chunk's last entry becomes the carry
      if (tid == 0) {
        sm.carry_g = sm.next_carry;
        sm.carry_valid = 1;
      }
    }
  }
  __syncthreads();
}

// gkey of the merged entry before position x of the staged chunk, if any.
__device__ __forceinline__ bool prev_gkey(const EmSmem& sm, const EmDyn& d, unsigned x,
                                          unsigned long long* g) {
  if (x > 0) {
    *g = d.gk[d.mo[x - 1]];
    return true;
  }
  *g = sm.carry_g;
  return sm.carry_valid != 0;
}

// Rows of each window of the item: a group is its key's first group in the
// windows from max(previous pane of the key + 1, pane - K + 1) to its pane.
__device__ void count_item(const QueryDev& q, const Item& it, EmSmem& sm, const EmDyn& d) {
  const int nw = (int)(it.whi - it.wlo + 1);
  const int lb = q.lb;
  for (int i = threadIdx.x; i <= nw; i += kEmT) sm.cnt[i] = 0;
  for (int i = threadIdx.x; i < kEmWarps * (kMaxItemWindows + 2); i += kEmT)
    (&sm.wdiff[0][0])[i] = 0;
  if (q.k == 1) {  // tumbling: one window, one pane, unique keys
    __syncthreads();
    if (threadIdx.x == 0) sm.cnt[0] = (long long)(it.a_hi - it.a_lo);
  } else {
    for_merged_chunks(q, it, sm, d, false, [&](unsigned len, unsigned, unsigned long long,
                                               unsigned long long, bool) {
      const unsigned x0 = threadIdx.x * kEmE;
#pragma unroll
      for (int e = 0; e < kEmE; ++e) {
        const unsigned x = x0 + e;
        if (x >= len) break;
        const unsigned long long g = d.gk[d.mo[x]];
        const long long p = (long long)gkey_pane(g, lb);
        long long lo = p - q.k + 1;
        unsigned long long pg;
        if (prev_gkey(sm, d, x, &pg) && gkey_key(pg, lb) == gkey_key(g, lb)) {
          const long long after = (long long)gkey_pane(pg, lb) + 1;
          lo = lo > after ? lo : after;
        }
        long long hi = p;
        lo = lo > it.wlo ? lo : it.wlo;
        hi = hi < it.whi ? hi : it.whi;
        if (lo <= hi) {
          int* wd = sm.wdiff[threadIdx.x >> 5];
          atomicAdd(&wd[lo - it.wlo], 1);
          atomicAdd(&wd[hi - it.wlo + 1], -1);
        }
      }
      __syncthreads();
    });
    if (threadIdx.x == 0) {
      long long acc = 0;
      for (int i = 0; i < nw; ++i) {
#pragma unroll
        for (int ww = 0; ww < kEmWarps; ++ww) acc += sm.wdiff[ww][i];
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

// gkey of group e (pane order) of a key whose first group is at merged
// position x0: staged, or in global memory for the chunk's last key when it
// continues past the chunk (A groups from open_ia, then B groups from open_ib).
__device__ __forceinline__ unsigned long long key_gkey(const EmSmem& sm, const EmDyn& d,
                                                       const Item& it, bool glob, unsigned x0,
                                                       unsigned e) {
  if (!glob) return d.gk[d.mo[x0 + e]];
  return e < sm.open_na ? it.A[sm.open_ia + e].gkey : it.Bv[sm.open_ib + (e - sm.open_na)].gkey;
}
// Writes the item's rows from out[0]: rows of window i from out[woff[i]], in
// key order.  Per chunk, rounds of up to kEmT keys (one per thread): each key's
// windows as a bit mask, the warps' ballots per window, then row descriptors
// laid out in output order, then one row per thread over the descriptors.
template <bool FLOAT>
__device__ void write_item(const QueryDev& q, const Item& it, EmSmem& sm, const EmDyn& d,
                           ResultRowDev* out) {
  const int tid = threadIdx.x, w = tid >> 5;
  const unsigned lane = lane_id(), lt = (1u << lane) - 1u;
  const int lb = q.lb, K = q.k;
  const int nw = (int)(it.whi - it.wlo + 1);
  if (K == 1) {  // tumbling: the unit's rows are its groups of the pane, in key order
    const long long wstart = (it.wlo - kPaneBias) * (long long)q.slide + q.base;
    for (unsigned long long i = it.a_lo + tid; i < it.a_hi; i += kEmT) {
      const Grp g = load_grp_v(it.A + i);
      write_row<FLOAT>(q, out + sm.woff[0] + (i - it.a_lo), wstart, gkey_key(g.gkey, lb), g.cnt,
                       g.sum, g.mn, g.mx);
    }
    __syncthreads();
    return;
  }
  // keys per round: one per thread, and at most kEmRows rows
  const unsigned kpr = kEmRows / nw < (unsigned)kEmT ? (unsigned)(kEmRows / nw) : (unsigned)kEmT;
  for (int i = tid; i < nw; i += kEmT) sm.run[i] = 0u;
  for_merged_chunks(q, it, sm, d, true, [&](unsigned len, unsigned la, unsigned long long a0,
                                            unsigned long long b0, bool last_chunk) {
    // heads: the merged positions that start a key
    unsigned nh_t = 0;
    bool head[kEmE];
    const unsigned x0 = (unsigned)tid * kEmE;
#pragma unroll
    for (int e = 0; e < kEmE; ++e) {
      head[e] = false;
      const unsigned x = x0 + e;
      if (x < len) {
        unsigned long long pg;
        head[e] = !(prev_gkey(sm, d, x, &pg) &&
                    gkey_key(pg, lb) == gkey_key(d.gk[d.mo[x]], lb));
        nh_t += head[e] ? 1u : 0u;
      }
    }
    unsigned long long htot;
    unsigned long long hpos = block_excl_scan((unsigned long long)nh_t, sm.tmp, &htot);
#pragma unroll
    for (int e = 0; e < kEmE; ++e)
      if (head[e]) d.hp[hpos++] = (unsigned short)(x0 + e);
    const unsigned nh = (unsigned)htot;
    if (tid == 0) {
      d.hp[nh] = (unsigned short)len;
      // does the chunk's last key continue in the next chunk?  Then its
      // groups are read from global memory: A from open_ia, then B from open_ib.
      unsigned open_n = 0u;
      if (!last_chunk && nh > 0) {
        const unsigned long long a1 = a0 + la, b1 = b0 + (len - la);
        const unsigned k = gkey_key(d.gk[d.mo[len - 1]], lb);
        if ((a1 < it.na && gkey_key(it.A[a1].gkey, lb) == k) ||
            (b1 < it.nb && gkey_key(it.Bv[b1].gkey, lb) == k)) {
          const unsigned hx = d.hp[nh - 1], slot = d.mo[hx];
          unsigned long long ia, ib;
          if (slot < la) {  // its first group is from A: hx - slot B groups precede it
            ia = a0 + slot;
            ib = b0 + (hx - slot);
          } else {
            ib = b0 + (slot - la);
            ia = a0 + (hx - (slot - la));
          }
          sm.open_ia = ia;
          sm.open_ib = ib;
          sm.open_na = (unsigned)(run_end(it.A, ia, it.na, k, lb) - ia);
          open_n = sm.open_na + (unsigned)(run_end(it.Bv, ib, it.nb, k, lb) - ib);
        }
      }
      sm.open_last = open_n;
    }
    __syncthreads();
    for (unsigned r0 = 0; r0 < nh; r0 += kpr) {
      // phase 1: this thread's key of the round and the item windows holding it
      const unsigned h = r0 + (unsigned)tid;
      const bool valid = (unsigned)tid < kpr && h < nh;
      const bool glob = valid && h + 1 == nh && sm.open_last != 0u;
      unsigned n = 0u, hx = 0u;
      unsigned long long mask = 0ull;
      long long pc0 = 0, pc1 = 0, pc2 = 0, pc3 = 0;  // the first four panes of the key
      if (valid) {
        hx = d.hp[h];
        n = glob ? sm.open_last : d.hp[h + 1] - hx;
        for (unsigned e = 0; e < n; ++e) {
          const long long p = (long long)gkey_pane(key_gkey(sm, d, it, glob, hx, e), lb);
          pc0 = e == 0 ? p : pc0;
          pc1 = e == 1 ? p : pc1;
          pc2 = e == 2 ? p : pc2;
          pc3 = e == 3 ? p : pc3;
          mask |= pane_windows(p, K, it.wlo, it.whi);
        }
      }
      if (tid == 0) sm.open_kh = sm.open_last != 0u && nh - 1 - r0 < kpr ? nh - 1 - r0 : ~0u;
      const unsigned long long orm =
          ((unsigned long long)__reduce_or_sync(kFull, (unsigned)(mask >> 32)) << 32) |
          __reduce_or_sync(kFull, (unsigned)mask);
      for (int i = lane; i < nw; i += 32) sm.wc[w][i] = 0u;
      __syncwarp();
      for (unsigned long long bits = orm; bits; bits &= bits - 1) {
        const int i = __ffsll((long long)bits) - 1;
        const unsigned bal = __ballot_sync(kFull, (mask >> i) & 1ull);
        if (lane == 0) {
          sm.ball[w][i] = bal;
          sm.wc[w][i] = (unsigned)__popc(bal);
        }
      }
      __syncthreads();
      // offsets: warps inside each window, windows inside the round
      if (tid < 32) {
        unsigned tot_i[2] = {0u, 0u};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int i = tid + 32 * u;
          if (i < nw) {
            unsigned acc = 0;
#pragma unroll
            for (int ww = 0; ww < kEmWarps; ++ww) {
              const unsigned t = sm.wc[ww][i];
              sm.wc[ww][i] = acc;
              acc += t;
            }
            tot_i[u] = acc;
          }
        }
        // exclusive scan of the per-window totals (windows tid and tid + 32)
        unsigned inc0 = tot_i[0], inc1 = tot_i[1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned y0 = __shfl_up_sync(kFull, inc0, o), y1 = __shfl_up_sync(kFull, inc1, o);
          if ((int)tid >= o) {
            inc0 += y0;
            inc1 += y1;
          }
        }
        const unsigned tot0 = __shfl_sync(kFull, inc0, 31);
        const unsigned e0 = inc0 - tot_i[0], e1 = tot0 + inc1 - tot_i[1];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int i = tid + 32 * u;
          if (i < nw) {
            const unsigned rb = u == 0 ? e0 : e1;
            sm.rb[i] = rb;
#pragma unroll
            for (int ww = 0; ww < kEmWarps; ++ww) sm.wc[ww][i] += rb;
            sm.base[i] = sm.woff[i] + sm.run[i] - rb;
            sm.run[i] += tot_i[u];
          }
        }
        const unsigned tot1 = __shfl_sync(kFull, inc1, 31);
        if (tid == 0) sm.rb[nw] = tot0 + tot1;
      }
      __syncthreads();
      // phase 2: each thread lays out its key's rows in output order: the
      // window, and the first of its groups in the window and their number
      {
        unsigned lo = 0u, hi = 0u;
        auto pane_at = [&](unsigned e) -> long long {
          if (e < 4) return e == 0 ? pc0 : e == 1 ? pc1 : e == 2 ? pc2 : pc3;
          return (long long)gkey_pane(key_gkey(sm, d, it, glob, hx, e), lb);
        };
        for (unsigned long long bits = mask; bits; bits &= bits - 1) {
          const int i = __ffsll((long long)bits) - 1;
          const long long W = it.wlo + i;
          while (lo < n && pane_at(lo) < W) ++lo;
          if (hi < lo) hi = lo;
          while (hi < n && pane_at(hi) <= W + K - 1) ++hi;
          const unsigned pos = sm.wc[w][i] + (unsigned)__popc(sm.ball[w][i] & lt);
          d.rows[pos] = (unsigned short)((tid << 6) | i);
          d.rln[pos] = (glob ? lo : hx + lo) | ((hi - lo) << 16);
        }
      }
      __syncthreads();
      // phase 3: one row per thread, two rows' inputs loaded before either is
      // combined and written
      const unsigned R = sm.rb[nw];
      const unsigned okh = sm.open_kh;
      auto group_at = [&](bool glob_key, unsigned x) -> Grp {
        if (glob_key)
          return load_grp_v(x < sm.open_na ? it.A + sm.open_ia + x
                                           : it.Bv + sm.open_ib + (x - sm.open_na));
        const unsigned slot = d.mo[x];
        Grp g;
        g.gkey = d.gk[slot];
        g.cnt = d.cnt[slot];
        g.sum = d.sum[slot];
        const unsigned long long m = d.mm[slot];
        g.mn = (unsigned)m;
        g.mx = (unsigned)(m >> 32);
        return g;
      };
      auto finish = [&](unsigned r, unsigned desc, unsigned x, unsigned nn, const Grp& g0) {
        const unsigned kh = desc >> 6, i = desc & 63u;
        const bool kg = kh == okh;
        long long cnt = g0.cnt;
        unsigned long long isum = g0.sum;
        double fsum = __longlong_as_double((long long)g0.sum);
        unsigned mn = g0.mn, mx = g0.mx;
        for (unsigned e = 1; e < nn; ++e) {
          const Grp g = group_at(kg, x + e);
          cnt += g.cnt;
          mn = min(mn, g.mn);
          mx = max(mx, g.mx);
          if (FLOAT) fsum += __longlong_as_double((long long)g.sum);
          else isum += g.sum;
        }
        const unsigned long long sb = FLOAT ? (unsigned long long)__double_as_longlong(fsum) : isum;
        const long long wstart = (it.wlo + (long long)i - kPaneBias) * (long long)q.slide + q.base;
        write_row<FLOAT>(q, out + sm.base[i] + r, wstart, gkey_key(g0.gkey, lb), cnt, sb, mn, mx);
      };
      for (unsigned r = tid; r < R; r += 2 * kEmT) {
        const unsigned r2 = r + kEmT;
        const bool two = r2 < R;
        const unsigned desc1 = d.rows[r], ln1 = d.rln[r];
        const unsigned desc2 = two ? d.rows[r2] : desc1, ln2 = two ? d.rln[r2] : ln1;
        const unsigned x1 = ln1 & 0xffffu, n1 = ln1 >> 16, x2 = ln2 & 0xffffu, n2 = ln2 >> 16;
        if (n1 == 0u || (two && n2 == 0u)) continue;  // cannot happen: a row has >= 1 group
        const Grp g1 = group_at((desc1 >> 6) == okh, x1);
        const Grp g2 = group_at((desc2 >> 6) == okh, x2);
        finish(r, desc1, x1, n1, g1);
        if (two) finish(r2, desc2, x2, n2, g2);
      }
      __syncthreads();
    }
  });
}

// ---- the pane-word path (2B <= 32): one warp per unit -------------------------
//
// An item of this path holds the windows starting in one block (nw = B <= 16,
// so lane i < 16 of a warp can speak for window i) and its units are small
// (kUnitEntriesPW merged entries).  One warp counts, and later writes, a unit
// alone, with no CTA barrier and no wait on another warp: the warp walks its
// unit in key-aligned chunks of at most kWC entries staged in its own slice of
// shared memory.  Per chunk every merged entry ORs the bit of its pane
// (relative to the item's block b) into its key's word; a key's windows are
// then the word dilated by K (a window whose first pane is r, relative to
// block b, holds the key iff a bit of [r, r + K) is set), and the groups of
// its row in that window are the set bits of [r, r + K): the first is the
// number of set bits below r (the key's groups are in pane order), their
// number the set bits in the range.  Per round of 32 keys (one per lane), the
// ballot of window i over the lanes counts the round's rows of the window;
// the writer then numbers the round's rows in output order (window, then key)
// and writes them 32 at a time, one per lane, so that consecutive lanes write
// consecutive rows.

constexpr int kWCn = kPwChunkEntries;  // nominal chunk
constexpr int kWC = kWCn + 32;         // staged entries: a key adds fewer than 2B <= 32
constexpr int kWE = kWC / 32;   // merged entries per lane
constexpr int kPwWarps = 8;
constexpr int kPwT = kPwWarps * 32;

// One warp's staged chunk: records as columns, the merged order, the keys'
// first merged positions and pane words, and the chunk starts of the unit.
struct PwWarp {
  unsigned long long gk[kWC];
  long long cnt[kWC];
  unsigned long long sum[kWC];
  unsigned long long mm[kWC];   // mn | mx << 32
  unsigned kw[kWC];             // per key of the chunk: its panes relative to block b, as bits
  unsigned sa[kPwUnitChunks + 1];  // the unit's chunk boundaries: A and B entries of the
  unsigned sb[kPwUnitChunks + 1];  // item before them
  unsigned char mo[kWC];        // record slot of each merged position
  unsigned char hp[kWC + 1];    // merged positions of the keys' first entries, then len
};

// Position of set bit number n (from 0, lowest first) of m, by a halving
// search on popcounts; some position below 32 if m has no more than n set bits.
__device__ __forceinline__ unsigned nth_set_bit(unsigned m, unsigned n) {
  unsigned pos = 0u;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const unsigned c = (unsigned)__popc(m & ((1u << w) - 1u));
    if (n >= c) {
      n -= c;
      m >>= w;
      pos += (unsigned)w;
    }
  }
  return pos & 31u;
}

// One warp over unit `it`, whose nch chunks are bounded by W.sa / W.sb.  Lane
// i < nw holds `off` for window i: on entry the output row of the unit's
// first row in the window (WRITE) or 0 (count); on return that plus the
// unit's rows in the window.  The key words start zeroed and are left zeroed.
template <bool WRITE, bool FLOAT>
__device__ void pw_unit(const QueryDev& q, const Item& it, unsigned nch, PwWarp& W,
                        unsigned long long& off, ResultRowDev* out) {
  const unsigned lane = lane_id();
  const int lb = q.lb, K = q.k;
  const int nw = (int)(it.whi - it.wlo + 1);
  if (K == 1) {  // tumbling: the unit's rows are its groups of the pane, in key order
    if (WRITE) {
      const unsigned long long o = __shfl_sync(kFull, off, 0);
      const long long wstart = (it.wlo - kPaneBias) * (long long)q.slide + q.base;
      for (unsigned long long i = it.a_lo + lane; i < it.a_hi; i += 32) {
        const Grp g = load_grp_v(it.A + i);
        write_row<FLOAT>(q, out + o + (i - it.a_lo), wstart, gkey_key(g.gkey, lb), g.cnt, g.sum,
                         g.mn, g.mx);
      }
    }
    if (lane == 0) off += it.a_hi - it.a_lo;
    return;
  }
  const unsigned long long blk = (unsigned long long)it.wlo >> lb;  // the item's block b
  const int wrel0 = (int)(it.wlo - (long long)(blk << lb));         // wlo relative to block b
  const unsigned wmask = (1u << nw) - 1u;
  const unsigned kmask = (1u << K) - 1u;
  const long long wstart0 = (it.wlo - kPaneBias) * (long long)q.slide + q.base;
  // the count stages only gkeys, the next chunk's while this one is processed
  unsigned long long pf[kWE];
  if (!WRITE && nch > 0) {
    const unsigned a0 = W.sa[0], b0 = W.sb[0], la = W.sa[1] - a0, len = la + W.sb[1] - b0;
#pragma unroll
    for (int e = 0; e < kWE; ++e) {
      const unsigned r = lane + 32u * e;
      pf[e] = r < len ? (r < la ? it.A[a0 + r].gkey : it.Bv[b0 + (r - la)].gkey) : 0ull;
    }
  }
  for (unsigned kk = 0; kk < nch; ++kk) {
    const unsigned a0 = W.sa[kk], b0 = W.sb[kk];
    const unsigned la = W.sa[kk + 1] - a0;
    const unsigned len = la + (W.sb[kk + 1] - b0);
    if (WRITE) {
      // the next chunk's records into L2 while this one is processed
      if (kk + 1 < nch) {
        const unsigned na = W.sa[kk + 2] - W.sa[kk + 1], nb = W.sb[kk + 2] - W.sb[kk + 1];
        const char* pa = reinterpret_cast<const char*>(it.A + W.sa[kk + 1]);
        const char* pb = reinterpret_cast<const char*>(it.Bv + W.sb[kk + 1]);
        if (lane * 128u < na * (unsigned)sizeof(Grp))
          asm volatile("prefetch.global.L2 [%0];" ::"l"(pa + lane * 128u));
        if (lane * 128u < nb * (unsigned)sizeof(Grp))
          asm volatile("prefetch.global.L2 [%0];" ::"l"(pb + lane * 128u));
      }
      // stage the chunk: two 16-byte halves per record
      for (unsigned h = lane; h < 2 * len; h += 32) {
        const unsigned r = h >> 1;
        const Grp* src = r < la ? it.A + a0 + r : it.Bv + b0 + (r - la);
        const uint4 v = reinterpret_cast<const uint4*>(src)[h & 1];
        const unsigned long long lo = ((unsigned long long)v.y << 32) | v.x;
        const unsigned long long hi = ((unsigned long long)v.w << 32) | v.z;
        if (h & 1) {
          W.sum[r] = lo;
          W.mm[r] = hi;
        } else {
          W.gk[r] = lo;
          W.cnt[r] = (long long)hi;
        }
      }
    } else {
#pragma unroll
      for (int e = 0; e < kWE; ++e) {
        const unsigned r = lane + 32u * e;
        if (r < len) W.gk[r] = pf[e];
      }
      if (kk + 1 < nch) {
        const unsigned c0 = W.sa[kk + 1], d0 = W.sb[kk + 1];
        const unsigned ca = W.sa[kk + 2] - c0, cl = ca + W.sb[kk + 2] - d0;
#pragma unroll
        for (int e = 0; e < kWE; ++e) {
          const unsigned r = lane + 32u * e;
          if (r < cl) pf[e] = r < ca ? it.A[c0 + r].gkey : it.Bv[d0 + (r - ca)].gkey;
        }
      }
    }
    __syncwarp();
    // merge (by key, A first on equal keys): lane takes kWE merged positions
    const unsigned x0 = lane * kWE;
    if (x0 < len) {
      const unsigned lbn = len - la;
      unsigned i = merge_split_s(W.gk, la, lbn, x0, lb), j = x0 - i;
#pragma unroll
      for (int e = 0; e < kWE; ++e) {
        if (x0 + e < len) {
          const bool ta =
              j >= lbn || (i < la && gkey_key(W.gk[i], lb) <= gkey_key(W.gk[la + j], lb));
          W.mo[x0 + e] = (unsigned char)(ta ? i : la + j);
          if (ta) ++i;
          else ++j;
        }
      }
    }
    __syncwarp();
    // heads and the keys' pane words
    bool head[kWE];
    unsigned nh_t = 0u;
    unsigned long long g[kWE];
#pragma unroll
    for (int e = 0; e < kWE; ++e) {
      const unsigned x = x0 + e;
      g[e] = x < len ? W.gk[W.mo[x]] : 0ull;
      head[e] = x < len && (x == 0 || gkey_key(W.gk[W.mo[x - 1]], lb) != gkey_key(g[e], lb));
      nh_t += head[e] ? 1u : 0u;
    }
    unsigned hinc = nh_t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(kFull, hinc, o);
      if ((int)lane >= o) hinc += v;
    }
    const unsigned nh = __shfl_sync(kFull, hinc, 31);
    unsigned ki = hinc - nh_t;  // key index + 1 of the current entry
    {
      unsigned hpos = ki;
#pragma unroll
      for (int e = 0; e < kWE; ++e)
        if (head[e]) W.hp[hpos++] = (unsigned char)(x0 + e);
    }
    if (lane == 0) W.hp[nh] = (unsigned char)len;
#pragma unroll
    for (int e = 0; e < kWE; ++e) {
      if (x0 + e < len) {
        ki += head[e] ? 1u : 0u;
        const unsigned rel = (unsigned)(g[e] & ((1ull << lb) - 1ull)) |
                             ((unsigned)(gkey_block(g[e], lb) - blk) << lb);
        atomicOr(&W.kw[ki - 1], 1u << rel);
      }
    }
    __syncwarp();
    for (unsigned r0 = 0; r0 < nh; r0 += 32) {
      const unsigned h = r0 + lane;
      unsigned hx = 0u, word = 0u, mask = 0u, key = 0u;
      if (h < nh) {
        hx = W.hp[h];
        word = W.kw[h];
        unsigned dl = word;  // dilation by K: bit r set iff a bit of [r, r + K) is
        int span = 1;
        while (2 * span <= K) {
          dl |= dl >> span;
          span <<= 1;
        }
        if (span < K) dl |= dl >> (K - span);
        mask = (dl >> wrel0) & wmask;
        if (WRITE) key = gkey_key(W.gk[W.mo[hx]], lb);
      }
      // lane i: the ballot of the round's keys that hold window i, its rows
      const unsigned orm = __reduce_or_sync(kFull, mask);
      unsigned bal = 0u;
      for (unsigned bits = orm; bits; bits &= bits - 1) {
        const int i = __ffs((int)bits) - 1;
        const unsigned b = __ballot_sync(kFull, (mask >> i) & 1u);
        if ((int)lane == i) bal = b;
      }
      const unsigned cw = (unsigned)__popc(bal);
      if (WRITE) {
        // the round's rows in output order (window by window, keys
        // ascending) are f = 0 .. total - 1; incl = rows of windows 0 .. lane
        unsigned incl = cw;
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
          const unsigned v = __shfl_up_sync(kFull, incl, o);
          if ((int)lane >= o) incl += v;
        }
        const unsigned total = __shfl_sync(kFull, incl, 15);
        const unsigned excl = incl - cw;
        // 32 rows at a time, row f on lane f mod 32: its window i is the
        // number of windows all of whose rows come before f, its rank in the
        // window picks the key (the rank-th set bit of the window's ballot)
        for (unsigned f0 = 0; f0 < total; f0 += 32) {
          const unsigned f = f0 + lane;
          unsigned i = 0u;  // at most 15
#pragma unroll
          for (unsigned st = 8; st >= 1; st >>= 1)
            if (__shfl_sync(kFull, incl, i + st - 1) <= f) i += st;
          const unsigned rk = f - __shfl_sync(kFull, excl, i);
          const unsigned bw = __shfl_sync(kFull, bal, i);
          const unsigned long long ow = __shfl_sync(kFull, off, i);
          const unsigned kl = nth_set_bit(bw, rk);
          const unsigned hk = __shfl_sync(kFull, hx, kl);
          const unsigned wk = __shfl_sync(kFull, word, kl);
          const unsigned yk = __shfl_sync(kFull, key, kl);
          if (f < total) {
            const int r = wrel0 + (int)i;  // the window's first pane, relative to block b
            const unsigned x = hk + (unsigned)__popc(wk & ((1u << r) - 1u));
            const unsigned nn = (unsigned)__popc((wk >> r) & kmask);
            unsigned slot = W.mo[x];
            long long cnt = W.cnt[slot];
            unsigned long long isum = W.sum[slot];
            double fsum = __longlong_as_double((long long)isum);
            unsigned long long m = W.mm[slot];
            unsigned mn = (unsigned)m, mx = (unsigned)(m >> 32);
            for (unsigned e = 1; e < nn; ++e) {
              slot = W.mo[x + e];
              cnt += W.cnt[slot];
              const unsigned long long sv = W.sum[slot];
              if (FLOAT) fsum += __longlong_as_double((long long)sv);
              else isum += sv;
              m = W.mm[slot];
              mn = min(mn, (unsigned)m);
              mx = max(mx, (unsigned)(m >> 32));
            }
            const unsigned long long sb =
                FLOAT ? (unsigned long long)__double_as_longlong(fsum) : isum;
            write_row<FLOAT>(q, out + (ow + rk), wstart0 + (long long)i * (long long)q.slide,
                             yk, cnt, sb, mn, mx);
          }
        }
      }
      off += cw;
    }
    for (unsigned k = lane; k < nh; k += 32) W.kw[k] = 0u;  // for the next chunk
    __syncwarp();
  }
}

// Emission, in two kernels over the units (units are taken by ticket, so the
// units of a large item spread over all SMs):
//   k_emit_count / k_emit_count_pw: each unit's rows per window, stored at the
//     unit's slots of s.unit_off;
//   (k_uoff_*: the exclusive scan of s.unit_off, in output order)
//   k_emit_write / k_emit_write_pw: each unit's rows, window i's from its
//     scanned slot.
// A unit is one CTA's on the general path, one warp's on the pane-word path;
// no CTA or warp waits on another.
__global__ void __launch_bounds__(kEmT, 4) k_emit_count(const QueryDev q, const Scratch s) {
  __shared__ EmSmem sm;
  const EmDyn d = em_dyn();
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long NI = c->n_items;
  while (true) {
    if (threadIdx.x == 0) sm.ri = atomicAdd(&c->item_ticket, 1ull);
    __syncthreads();
    const unsigned long long u = sm.ri;
    __syncthreads();
    if (u >= NI) break;
    const Item it = load_unit(q, s, c, u);
    count_item(q, it, sm, d);
    const int nw = (int)(it.whi - it.wlo + 1);
    unsigned long long* slot = s.unit_off + (u - it.sub) * (unsigned long long)q.nw + it.sub;
    for (int i = threadIdx.x; i < q.nw; i += kEmT)
      slot[(unsigned long long)i * it.nsub] = i < nw ? (unsigned long long)sm.cnt[i] : 0ull;
    __syncthreads();
  }
}

template <bool FLOAT>
__global__ void __launch_bounds__(kEmT, 3)
    k_emit_write(const QueryDev q, const Scratch s, ResultRowDev* rows) {
  __shared__ EmSmem sm;
  const EmDyn d = em_dyn();
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long NI = c->n_items;
  ResultRowDev* out = rows + c->row_base;
  while (true) {
    if (threadIdx.x == 0) sm.ri = atomicAdd(&c->unit_ticket, 1ull);
    __syncthreads();
    const unsigned long long u = sm.ri;
    __syncthreads();
    if (u >= NI) break;
    const Item it = load_unit(q, s, c, u);
    const int nw = (int)(it.whi - it.wlo + 1);
    const unsigned long long* slot = s.unit_off + (u - it.sub) * (unsigned long long)q.nw + it.sub;
    for (int i = threadIdx.x; i < nw; i += kEmT) sm.woff[i] = slot[(unsigned long long)i * it.nsub];
    __syncthreads();
    write_item<FLOAT>(q, it, sm, d, out);
    __syncthreads();
  }
}

// The pane-word path: each warp takes units by ticket and counts (WRITE =
// false) or writes them alone.
template <bool WRITE, bool FLOAT>
__global__ void __launch_bounds__(kPwT, 4)
    k_emit_pw(const QueryDev q, const Scratch s, ResultRowDev* rows) {
  __shared__ PwWarp ws[kPwWarps];
  PwWarp& W = ws[threadIdx.x >> 5];
  const unsigned lane = lane_id();
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long NI = c->n_items;
  ResultRowDev* out = WRITE ? rows + c->row_base : rows;
  unsigned long long* ticket = WRITE ? &c->unit_ticket : &c->item_ticket;
  for (unsigned k = lane; k < (unsigned)kWC; k += 32) W.kw[k] = 0u;
  while (true) {
    __syncwarp();  // the previous unit no longer reads W.sa / W.sb
    unsigned long long u = 0ull;
    if (lane == 0) u = atomicAdd(ticket, 1ull);
    u = __shfl_sync(kFull, u, 0);
    if (u >= NI) break;
    Item it = load_item(q, s, c, (long long)s.item_c[u], s.item_j[u]);
    const unsigned long long st = s.item_stat[u];
    it.sub = (unsigned)st;
    it.nsub = (unsigned)(st >> 32);
    // the unit's chunks (nominal) and their boundaries from the table
    const unsigned long long L = it.na + it.nb, d0 = (unsigned long long)it.sub * kUnitEntriesPW;
    const unsigned long long dn = d0 + kUnitEntriesPW < L ? d0 + kUnitEntriesPW : L;
    const unsigned nch = dn > d0 ? (unsigned)((dn - d0 + kWCn - 1) / kWCn) : 0u;
    if (lane <= nch) {
      W.sa[lane] = s.unit_bnd[u * kUnitBnd + 2 * lane];
      W.sb[lane] = s.unit_bnd[u * kUnitBnd + 2 * lane + 1];
    }
    __syncwarp();
    it.a_lo = W.sa[0];
    it.b_lo = W.sb[0];
    it.a_hi = W.sa[nch];
    it.b_hi = W.sb[nch];
    const int nw = (int)(it.whi - it.wlo + 1);
    unsigned long long* slot = s.unit_off + (u - it.sub) * (unsigned long long)q.nw + it.sub;
    unsigned long long off = 0ull;  // lane i < nw <= 16: window i
    if (WRITE && (int)lane < nw) off = slot[(unsigned long long)lane * it.nsub];
    pw_unit<WRITE, FLOAT>(q, it, nch, W, off, out);
    if (!WRITE && (int)lane < q.nw) slot[(unsigned long long)lane * it.nsub] = (int)lane < nw ? off : 0ull;
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
  // the first state group of a block >= the cursor's (a binary search over the
  // state: it is sorted by gkey, whose top bits are the block)
  const unsigned long long bstar = (unsigned long long)c->cursor >> q.lb;
  unsigned long long lo = 0, hi = c->n_state;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if (gkey_block(q.state[mid].gkey, q.lb) < bstar) lo = mid + 1; else hi = mid;
  }
  c->trim_from = lo;
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

cudaError_t launch_batch_begin(SCtl* sctl, QCtl* const* ctls, int nq, long long ts_floor,
                               cudaStream_t st) {
  QCtl* c[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int i = 0; i < nq && i < 8; ++i) c[i] = ctls[i];
  k_batch_begin<<<1, 32, 0, st>>>(sctl, ts_floor, c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7]);
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
  // devices whose smem limit is set, per kernel
  static unsigned long long done[3] = {0, 0, 0};
  const bool pw = (2 << q.lb) <= 32;
  const int g = kGrid;
  if (pw) {
    k_unit_bounds<<<kGrid, 256, 0, st>>>(q, s);
    // four CTAs of eight warps per SM (64 registers, 39 KB of shared memory)
    k_emit_pw<false, false><<<4 * sms, kPwT, 0, st>>>(q, s, rows);
  } else {
    cudaError_t e = set_smem_limit(reinterpret_cast<const void*>(k_emit_count),
                                   (int)kEmDynBytesCount, &done[2]);
    if (e != cudaSuccess) return e;
    k_emit_count<<<4 * sms, kEmT, kEmDynBytesCount, st>>>(q, s);
  }
  k_uoff_sum<<<g, 256, 0, st>>>(q, s);
  k_uoff_scan<<<1, 1024, 0, st>>>(q, s, rows_cap);
  k_uoff_write<<<g, 256, 0, st>>>(q, s);
  if (ev4) {
    record_event(ev4[1], st);
    record_event(ev4[2], st);
  }
  if (pw) {
    if (q.value_is_float) k_emit_pw<true, true><<<4 * sms, kPwT, 0, st>>>(q, s, rows);
    else k_emit_pw<true, false><<<4 * sms, kPwT, 0, st>>>(q, s, rows);
  } else {
    const void* fn = q.value_is_float ? reinterpret_cast<const void*>(k_emit_write<true>)
                                      : reinterpret_cast<const void*>(k_emit_write<false>);
    cudaError_t e = set_smem_limit(fn, (int)kEmDynBytes, &done[q.value_is_float ? 1 : 0]);
    if (e != cudaSuccess) return e;
    // three CTAs per SM (the row descriptors of the general path need the room)
    if (q.value_is_float) k_emit_write<true><<<3 * sms, kEmT, kEmDynBytes, st>>>(q, s, rows);
    else k_emit_write<false><<<3 * sms, kEmT, kEmDynBytes, st>>>(q, s, rows);
  }
  if (ev4) record_event(ev4[3], st);
  if (launches) *launches += pw ? 10 : 9;
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
