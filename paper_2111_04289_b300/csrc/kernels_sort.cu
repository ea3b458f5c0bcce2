// Partial groups -> sorted, unique window state.
//
// After the fused pass, a query's partial-group arrays hold the groups carried
// over from the previous batch (sorted and unique: the previous batch's state
// minus its closed panes) followed by this batch's per-tile groups, in no
// particular order.  This file turns them into the window state: an LSD radix
// sort of only the new groups' 64-bit keys (8-bit digits; digits that are
// equal in every key are skipped, which the OR/AND masks gathered by the
// producers reveal), a merge of the sorted new keys with the carried ones
// (merge path; on equal keys the carried group comes first), then a
// reduce-by-key that combines equal (pane, key) groups, then the index of
// distinct blocks.  So a batch costs a sort of its own groups plus a linear
// merge, however large the open state it carries.  All sizes are read on the
// device, so the whole sequence launches without a host round trip.
//
// Chunked kernels use a fixed grid of kGrid CTAs, each owning one contiguous
// chunk of the input; a per-chunk count, a single-CTA scan of the counts and a
// per-chunk write give stable, deterministic positions.
#include <climits>

#include "lms_device.cuh"

namespace lms {
namespace {

constexpr int kScatterTile = 2048;  // 8 warps x 8 rounds x 32 lanes

struct SortSrc {
  const unsigned long long* keys;
  const unsigned* vals;  // nullptr: identity
};

// Pass p reads the previous pass's output (or, for p == 0, the new partial
// keys, after the sort_base carried ones) and writes buffer (p & 1) of the
// scratch pair.  Values are indices into the partial arrays; nullptr means
// the identity (index = sort_base + position).
__device__ __forceinline__ SortSrc pass_src(const QueryDev& q, const Scratch& s, int p) {
  if (p == 0) return {q.pkeys + q.ctl->sort_base, nullptr};
  return ((p - 1) & 1) ? SortSrc{s.keysB, s.valsB} : SortSrc{s.keysA, s.valsA};
}
__device__ __forceinline__ SortSrc final_src(const QueryDev& q, const Scratch& s, int np) {
  if (np == 0) return {q.pkeys + q.ctl->sort_base, nullptr};
  return ((np - 1) & 1) ? SortSrc{s.keysB, s.valsB} : SortSrc{s.keysA, s.valsA};
}

// The key/value pair the final sort pass did not write (free after the sort).
__device__ __forceinline__ void free_pair(const Scratch& s, int np, unsigned long long** k,
                                          unsigned** v) {
  const bool final_b = np > 0 && ((np - 1) & 1);
  *k = final_b ? s.keysA : s.keysB;
  *v = final_b ? s.valsA : s.valsB;
}

// Input of the reduce: the merged keys (in the free pair) when groups were
// carried, else the sorted new keys; `other` gets the pair it does not use.
__device__ __forceinline__ SortSrc reduce_src(const QueryDev& q, const Scratch& s, int np,
                                              unsigned long long** ok, unsigned** ov) {
  unsigned long long* fk;
  unsigned* fv;
  free_pair(s, np, &fk, &fv);
  if (q.ctl->sort_base == 0) {
    *ok = fk;
    *ov = fv;
    return final_src(q, s, np);
  }
  const bool final_b = np > 0 && ((np - 1) & 1);  // the sort's own pair is free again
  *ok = final_b ? s.keysB : s.keysA;
  *ov = final_b ? s.valsB : s.valsA;
  return SortSrc{fk, fv};
}

// Number of items sorted: the partials after the carried ones.
__device__ __forceinline__ unsigned long long sort_count(const QCtl* c) {
  return c->n_parts - c->sort_base;
}

__global__ void k_sort_plan(QCtl* c) {
  if (threadIdx.x != 0) return;
  const unsigned long long n = c->n_parts;
  c->parts_at_sort = n;
  c->n_long = 0;
  const unsigned long long m = c->or_mask ^ c->and_mask;
  int nd = 0;  // digits that differ between keys
  for (int d = 0; d < 8; ++d)
    if ((m >> (8 * d)) & 0xffull) c->shifts[nd++] = 8 * d;
  // Merging costs one pass over all the partials; sorting the carried groups
  // along costs ~nd passes over them: when they are few, sort everything.
  const unsigned long long carried = c->carried < n ? c->carried : n;
  c->sort_base = carried * (unsigned long long)nd < n - carried ? 0ull : carried;
  c->npasses = n - c->sort_base > 1 ? nd : 0;
}

__global__ void __launch_bounds__(256) k_sort_hist(const QueryDev q, const Scratch s, int p) {
  const QCtl* c = q.ctl;
  if (p >= c->npasses) return;
  // one histogram per warp, plain shared atomics (lanes with equal digits are
  // serialised by the hardware; cheaper than grouping them first), summed at
  // the end
  __shared__ unsigned h[8][256];
  const int w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 8; ++j) h[j][threadIdx.x] = 0u;
  __syncthreads();
  const int shift = c->shifts[p];
  const SortSrc src = pass_src(q, s, p);
  unsigned long long lo, hi;
  chunk_range(sort_count(c), blockIdx.x, gridDim.x, &lo, &hi);
  constexpr int kU = 8;  // keys loaded per thread before any is counted
  for (unsigned long long i0 = lo; i0 < hi; i0 += kU * blockDim.x) {
    unsigned d[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const unsigned long long i = i0 + u * blockDim.x + threadIdx.x;
      d[u] = i < hi ? (unsigned)((src.keys[i] >> shift) & 0xffull) : 256u;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (d[u] < 256u) atomicAdd(&h[w][d[u]], 1u);
  }
  __syncthreads();
  unsigned t = 0u;
#pragma unroll
  for (int j = 0; j < 8; ++j) t += h[j][threadIdx.x];
  s.hist[threadIdx.x * gridDim.x + blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_sort_scan(const QueryDev q, const Scratch s, int p) {
  if (p >= q.ctl->npasses) return;
  __shared__ unsigned long long tmp[33];
  unsigned* h = s.hist + blockIdx.x * kGrid;
  const int a = 4 * threadIdx.x;
  unsigned x[4];
  unsigned sum = 0;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    x[u] = a + u < kGrid ? h[a + u] : 0u;
    sum += x[u];
  }
  unsigned long long tot;
  unsigned long long r = block_excl_scan((unsigned long long)sum, tmp, &tot);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (a + u < kGrid) h[a + u] = (unsigned)r;
    r += x[u];
  }
  if (threadIdx.x == 0) s.hist[256 * kGrid + blockIdx.x] = (unsigned)tot;
}

// One pass of the stable scatter.  Per tile of 2048 items: warp-aggregated
// ranks inside each warp's 256 items (match_any per round), the tile's
// per-digit counts and offsets, then the items are placed in shared memory in
// (digit, original order) and written out from there, so that consecutive
// threads write consecutive positions of each digit's run (coalesced).  The
// next tile's items are fetched into shared memory by asynchronous copies
// while the current tile is processed: each thread copies, and later reads,
// its own items only, so its own wait on the copies is all the ordering this
// needs.
constexpr size_t kScatterSmem = kScatterTile * (8 + 4)      // next tile's items (async copies)
                                + kScatterTile * (8 + 4)    // the tile in digit order
                                + 8 * 256 * 2;              // per-warp digit counts / offsets

__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc, int bytes, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gsrc),
                 "r"(valid ? 8 : 0) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gsrc),
                 "r"(valid ? 4 : 0) : "memory");
}

__global__ void __launch_bounds__(256, 4) k_sort_scatter(const QueryDev q, const Scratch s, int p) {
  const QCtl* c = q.ctl;
  if (p >= c->npasses) return;
  extern __shared__ __align__(16) unsigned char ssm[];
  unsigned long long* ikey = reinterpret_cast<unsigned long long*>(ssm);
  unsigned* ival = reinterpret_cast<unsigned*>(ikey + kScatterTile);
  unsigned long long* skey = reinterpret_cast<unsigned long long*>(ival + kScatterTile);
  unsigned* sval = reinterpret_cast<unsigned*>(skey + kScatterTile);
  unsigned short (*wcnt)[256] = reinterpret_cast<unsigned short (*)[256]>(sval + kScatterTile);
  __shared__ unsigned run[256];             // the CTA's next global position per digit
  __shared__ unsigned short lbase[257];     // the tile's first local position per digit
  __shared__ unsigned long long tmp[33];
  const int tid = threadIdx.x, w = tid >> 5;
  const unsigned lane = lane_id();
  const int shift = c->shifts[p];
  const SortSrc src = pass_src(q, s, p);
  unsigned long long* dk = (p & 1) ? s.keysB : s.keysA;
  unsigned* dv = (p & 1) ? s.valsB : s.valsA;
  unsigned long long lo, hi;
  chunk_range(sort_count(c), blockIdx.x, gridDim.x, &lo, &hi);
  const unsigned base = (unsigned)c->sort_base;
  {
    unsigned long long tot;
    const unsigned long long base =
        block_excl_scan((unsigned long long)s.hist[256 * kGrid + tid], tmp, &tot);
    run[tid] = (unsigned)base + s.hist[tid * gridDim.x + blockIdx.x];
  }
  const unsigned lt = (1u << lane) - 1u;
  const unsigned my = (unsigned)(w * 256) + lane;  // this thread's items: my + 32 r of each tile
  auto fetch = [&](unsigned long long tb) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const unsigned long long i = tb + my + 32 * r;
      const bool v = i < hi;
      const unsigned long long ic = v ? i : lo;  // a valid address even when nothing is read
      cp_async(ikey + my + 32 * r, src.keys + ic, 8, v);
      if (src.vals) cp_async(ival + my + 32 * r, src.vals + ic, 4, v);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (lo < hi) fetch(lo);
  for (unsigned long long tb = lo; tb < hi; tb += kScatterTile) {
#pragma unroll
    for (int j = 0; j < 8; ++j) wcnt[w][lane + 32 * j] = 0u;
    asm volatile("cp.async.wait_all;" ::: "memory");
    unsigned long long kk[8];
    unsigned vv[8], rr[4];  // ranks (< 256) packed two per word
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      kk[r] = ikey[my + 32 * r];
      vv[r] = src.vals ? ival[my + 32 * r] : base + (unsigned)(tb + my + 32 * r);
    }
    if (tb + kScatterTile < hi) fetch(tb + kScatterTile);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const bool v = tb + my + 32 * r < hi;
      const unsigned d = v ? (unsigned)((kk[r] >> shift) & 0xffull) : 256u;
      const unsigned peers = __match_any_sync(kFull, d);
      const unsigned rk = (v ? (unsigned)wcnt[w][d] : 0u) + __popc(peers & lt);
      if (r & 1) rr[r >> 1] |= rk << 16;
      else rr[r >> 1] = rk;
      __syncwarp();
      if (v && (int)lane == __ffs(peers) - 1)
        wcnt[w][d] = (unsigned short)(wcnt[w][d] + __popc(peers));
      __syncwarp();
    }
    __syncthreads();
    {  // thread tid = digit: offsets of the warps inside the tile's digit run
      unsigned acc = 0;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) {
        const unsigned cnt = wcnt[ww][tid];
        wcnt[ww][tid] = (unsigned short)acc;
        acc += cnt;
      }
      unsigned long long tot;
      lbase[tid] = (unsigned short)block_excl_scan((unsigned long long)acc, tmp, &tot);
      if (tid == 255) lbase[256] = (unsigned short)tot;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if (tb + my + 32 * r < hi) {
        const unsigned d = (unsigned)((kk[r] >> shift) & 0xffull);
        const unsigned rk = (rr[r >> 1] >> (16 * (r & 1))) & 0xffffu;
        const unsigned lp = (unsigned)lbase[d] + wcnt[w][d] + rk;
        skey[lp] = kk[r];
        sval[lp] = vv[r];
      }
    }
    __syncthreads();
    const unsigned nt = (unsigned)min((unsigned long long)kScatterTile, hi - tb);
    for (unsigned i = tid; i < nt; i += blockDim.x) {
      const unsigned long long k = skey[i];
      const unsigned d = (unsigned)((k >> shift) & 0xffull);
      const unsigned pos = run[d] + (i - lbase[d]);
      dk[pos] = k;
      dv[pos] = sval[i];
    }
    __syncthreads();
    run[tid] += (unsigned)lbase[tid + 1] - (unsigned)lbase[tid];
    __syncthreads();
  }
}

// ---- merge of the sorted new keys with the carried ones --------------------

// Number of carried keys among the first d keys of the merge of C[0, nc) and
// N[0, nn) (merge path; on equal keys C comes first).
__device__ __forceinline__ unsigned long long carry_split(const unsigned long long* C,
                                                          unsigned long long nc,
                                                          const unsigned long long* N,
                                                          unsigned long long nn,
                                                          unsigned long long d) {
  unsigned long long lo = d > nn ? d - nn : 0ull, hi = d < nc ? d : nc;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if (C[mid] <= N[d - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The merged (key, partial index) sequence of the carried groups (pkeys[0,
// sort_base), indices 0..) and the sorted new ones, written to the free pair.
// Each CTA owns a chunk of the output: tiles of kMergeTile outputs whose
// split points are found first (up to 256 at a time, in parallel), then each
// tile's two input runs are staged in shared memory and every thread merges
// kMergeItems consecutive outputs.
constexpr int kMergeItems = 8;
constexpr int kMergeTile = 256 * kMergeItems;

__global__ void __launch_bounds__(256) k_merge_carry(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  const unsigned long long nc = c->sort_base;
  if (nc == 0) return;
  const unsigned long long n = c->n_parts, nn = n - nc;
  const SortSrc N = final_src(q, s, c->npasses);
  const unsigned long long* C = q.pkeys;
  unsigned long long* mk;
  unsigned* mv;
  free_pair(s, c->npasses, &mk, &mv);
  __shared__ unsigned long long sp[257];
  __shared__ unsigned long long ck[kMergeTile], nk[kMergeTile];
  __shared__ unsigned nv[kMergeTile];
  const int tid = threadIdx.x;
  unsigned long long lo, hi;
  chunk_range(n, blockIdx.x, gridDim.x, &lo, &hi);
  for (unsigned long long t0 = lo; t0 < hi; t0 += 256ull * kMergeTile) {
    const unsigned long long span = hi - t0;
    const unsigned nt = (unsigned)min(256ull, (span + kMergeTile - 1) / kMergeTile);
    __syncthreads();  // the previous tiles no longer read sp
    for (unsigned j = tid; j <= nt; j += 256) {
      const unsigned long long d = min(t0 + (unsigned long long)j * kMergeTile, hi);
      sp[j] = carry_split(C, nc, N.keys, nn, d);
    }
    __syncthreads();
    for (unsigned j = 0; j < nt; ++j) {
      const unsigned long long d0 = t0 + (unsigned long long)j * kMergeTile;
      const unsigned long long d1 = min(d0 + kMergeTile, hi);
      const unsigned long long a0 = sp[j], a1 = sp[j + 1];
      const unsigned long long b0 = d0 - a0;
      const unsigned la = (unsigned)(a1 - a0), lb = (unsigned)(d1 - d0) - la;
      for (unsigned i = tid; i < la; i += 256) ck[i] = C[a0 + i];
      for (unsigned i = tid; i < lb; i += 256) {
        nk[i] = N.keys[b0 + i];
        nv[i] = N.vals ? N.vals[b0 + i] : (unsigned)(nc + b0 + i);
      }
      __syncthreads();
      // each thread merges kMergeItems consecutive outputs into registers; the
      // tile's outputs are then staged in ck / nv and written coalesced
      const unsigned x0 = (unsigned)tid * kMergeItems, len = la + lb;
      unsigned long long ok_[kMergeItems];
      unsigned ov_[kMergeItems];
      if (x0 < len) {
        unsigned ia = x0 > lb ? x0 - lb : 0u, ib = x0 < la ? x0 : la;  // merge path in the tile
        while (ia < ib) {
          const unsigned mid = (ia + ib) >> 1;
          if (ck[mid] <= nk[x0 - 1 - mid]) ia = mid + 1;
          else ib = mid;
        }
        unsigned i = ia, k = x0 - ia;
#pragma unroll
        for (int e = 0; e < kMergeItems; ++e) {
          const bool ta = k >= lb || (i < la && ck[i] <= nk[k]);
          ok_[e] = ta ? ck[i < la ? i : 0] : nk[k < lb ? k : 0];
          ov_[e] = ta ? (unsigned)(a0 + i) : nv[k < lb ? k : 0];
          if (ta) ++i; else ++k;
        }
      }
      __syncthreads();  // every thread is done reading ck / nk
#pragma unroll
      for (int e = 0; e < kMergeItems; ++e) {
        if (x0 + e < len) {
          ck[x0 + e] = ok_[e];
          nv[x0 + e] = ov_[e];
        }
      }
      __syncthreads();
      for (unsigned x = tid; x < len; x += 256) {
        mk[d0 + x] = ck[x];
        mv[d0 + x] = nv[x];
      }
      __syncthreads();
    }
  }
}

// ---- reduce-by-key: sorted partials -> unique groups (window state) -------

__global__ void __launch_bounds__(256) k_rbk_count(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  unsigned long long* ok;
  unsigned* ov;
  const SortSrc src = reduce_src(q, s, c->npasses, &ok, &ov);
  unsigned long long lo, hi;
  chunk_range(c->n_parts, blockIdx.x, gridDim.x, &lo, &hi);
  unsigned long long cnt = 0;
  for (unsigned long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
    cnt += (i == 0 || src.keys[i] != src.keys[i - 1]) ? 1ull : 0ull;
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  block_excl_scan(cnt, tmp, &tot);
  if (threadIdx.x == 0) s.chunk[blockIdx.x] = tot;
}

// Exclusive scan of g (<= 1024) per-chunk counts in place; total -> *total.
__global__ void __launch_bounds__(1024) k_scan_chunks(unsigned long long* a, int g,
                                                      unsigned long long* total) {
  __shared__ unsigned long long tmp[33];
  const unsigned long long v = (int)threadIdx.x < g ? a[threadIdx.x] : 0ull;
  unsigned long long tot;
  const unsigned long long r = block_excl_scan(v, tmp, &tot);
  if ((int)threadIdx.x < g) a[threadIdx.x] = r;
  if (threadIdx.x == 0) *total = tot;
}

// Reduce-by-key as a tiled segmented scan.  CTA c owns the runs of equal keys
// whose first element (head) lies in its chunk [lo, hi) of the sorted keys and
// processes [start, end): start = its first head, end = the end of the last run
// it owns — unless that run crosses hi and is longer than kLongRun, in which
// case it is listed for k_rbk_long (one CTA per run) and end stops at its
// head.  Tiles of 1024 elements (4 consecutive per thread): gather the groups,
// a segmented inclusive scan over the tile (thread-local, warp shuffles,
// warp totals in shared memory) carried across tiles, and the last element of
// each run writes the run's group at the run's rank among the CTA's heads.
constexpr unsigned long long kLongRun = 4096;
constexpr int kRbkItems = 4;
constexpr int kRbkTile = 256 * kRbkItems;

// first index in [a, b) whose key differs from k (keys sorted, keys[a-1..] >= k)
__device__ unsigned long long first_after(const unsigned long long* keys, unsigned long long a,
                                          unsigned long long b, unsigned long long k) {
  while (a < b) {
    const unsigned long long m = a + ((b - a) >> 1);
    if (keys[m] == k) a = m + 1;
    else b = m;
  }
  return a;
}

// first index in [a, b) whose key equals k (keys sorted, keys[b-1] == k)
__device__ unsigned long long first_equal(const unsigned long long* keys, unsigned long long a,
                                          unsigned long long b, unsigned long long k) {
  while (a < b) {
    const unsigned long long m = a + ((b - a) >> 1);
    if (keys[m] < k) a = m + 1;
    else b = m;
  }
  return a;
}

// Four CTAs per SM (64 registers, a few spilled): measured faster than two
// CTAs with every value in registers, the loads' latency being the bound.
template <bool FLOAT>
__global__ void __launch_bounds__(256, 4) k_rbk_write(const QueryDev q, const Scratch s) {
  QCtl* c = q.ctl;
  const unsigned long long n = c->n_parts;
  unsigned long long* lst;
  unsigned* lpos;
  const SortSrc src = reduce_src(q, s, c->npasses, &lst, &lpos);
  const unsigned long long* keys = src.keys;
  unsigned long long lo, hi;
  chunk_range(n, blockIdx.x, gridDim.x, &lo, &hi);
  __shared__ unsigned long long sh_start, sh_end;
  __shared__ unsigned long long tmp[33];
  __shared__ SegAgg wtot[8];
  __shared__ SegAgg carry;
  const unsigned long long out0 = s.chunk[blockIdx.x];
  if (threadIdx.x == 0) {
    unsigned long long st = lo, en = hi;
    if (lo < hi && lo > 0 && keys[lo] == keys[lo - 1]) st = first_after(keys, lo, hi, keys[lo - 1]);
    if (st < hi && hi < n && keys[hi] == keys[hi - 1]) {
      // the last run owned here crosses hi
      const unsigned long long k = keys[hi - 1];
      const unsigned long long h = first_equal(keys, st, hi - 1, k);
      unsigned long long b = hi, step = 256;  // gallop to its end
      while (b < n && keys[b] == k) {
        const unsigned long long t = b + step;
        if (t >= n || keys[t] != k) {
          b = first_after(keys, b + 1, t < n ? t : n, k);
          break;
        }
        b = t;
        step <<= 1;
      }
      if (b - h > kLongRun) {
        // rank of the run = number of heads owned before it
        const unsigned long long heads =
            (blockIdx.x + 1 < gridDim.x ? s.chunk[blockIdx.x + 1] : c->n_state) - out0;
        const unsigned long long slot = atomicAdd(&c->n_long, 1ull);
        lst[2 * slot] = h;
        lst[2 * slot + 1] = b;
        lpos[slot] = (unsigned)(out0 + heads - 1);
        en = h;
      } else {
        en = b;
      }
    }
    sh_start = st;
    sh_end = st < hi ? en : st;
    carry = seg_identity();
  }
  __syncthreads();
  const unsigned long long start = sh_start, end = sh_end;
  const unsigned lane = lane_id(), w = threadIdx.x >> 5;
  unsigned long long heads_before = 0;
  for (unsigned long long base = start; base < end; base += kRbkTile) {
    const unsigned long long i0 = base + (unsigned long long)threadIdx.x * kRbkItems;
    unsigned long long k[kRbkItems];
    bool head[kRbkItems], last[kRbkItems], valid[kRbkItems];
    SegAgg v[kRbkItems];
    unsigned nh = 0;
#pragma unroll
    for (int u = 0; u < kRbkItems; ++u) {
      const unsigned long long i = i0 + u;
      valid[u] = i < end;
      k[u] = valid[u] ? keys[i] : ~0ull;
    }
    // neighbours: previous key (for heads) and next key (for run ends)
    unsigned long long kprev = __shfl_up_sync(kFull, k[kRbkItems - 1], 1);
    unsigned long long knext = __shfl_down_sync(kFull, k[0], 1);
    if (lane == 0) kprev = (i0 > start && i0 < end) ? keys[i0 - 1] : ~0ull;
    if (lane == 31) knext = (i0 + kRbkItems < end) ? keys[i0 + kRbkItems] : ~0ull;
#pragma unroll
    for (int u = 0; u < kRbkItems; ++u) {
      const unsigned long long i = i0 + u;
      const unsigned long long kp = u == 0 ? kprev : k[u - 1];
      const unsigned long long kn = u + 1 < kRbkItems ? k[u + 1] : knext;
      head[u] = valid[u] && (i == start || k[u] != kp);
      last[u] = valid[u] && (i + 1 == end || k[u] != kn);
      nh += head[u] ? 1u : 0u;
      if (valid[u]) {
        const unsigned long long pi = src.vals ? src.vals[i] : i;
        const Grp g = load_grp_v(q.parts + pi);
        v[u].f = head[u] ? 1u : 0u;
        v[u].cnt = g.cnt;
        v[u].sum = g.sum;
        v[u].mn = g.mn;
        v[u].mx = g.mx;
      } else {
        v[u] = seg_identity();
      }
    }
    // output index of each element's run: the heads up to and including the
    // element, minus one (a run has no head after its own)
    unsigned long long htot;
    const unsigned long long hpre = block_excl_scan((unsigned long long)nh, tmp, &htot);
    int orank[kRbkItems];  // relative to out0 + heads_before (-1: a run headed in an earlier tile)
    {
      int hc = (int)hpre;
#pragma unroll
      for (int u = 0; u < kRbkItems; ++u) {
        if (head[u]) ++hc;
        orank[u] = hc - 1;
      }
    }
    // thread-local inclusive segmented scan
#pragma unroll
    for (int u = 1; u < kRbkItems; ++u) v[u] = seg_combine<FLOAT>(v[u - 1], v[u]);
    // warp inclusive scan of thread totals
    SegAgg t = v[kRbkItems - 1];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const SegAgg o = seg_shfl_up(t, d);
      if ((int)lane >= d) t = seg_combine<FLOAT>(o, t);
    }
    SegAgg ex = seg_shfl_up(t, 1);  // exclusive within the warp
    if (lane == 31) wtot[w] = t;
    __syncthreads();
    seg_scan_warp_totals<FLOAT>(wtot, 8, &carry);  // prefixes of the warps, from the carry
    __syncthreads();
    SegAgg pre = wtot[w];
    if (lane > 0) pre = seg_combine<FLOAT>(pre, ex);
#pragma unroll
    for (int u = 0; u < kRbkItems; ++u) {
      if (!last[u]) continue;
      const SegAgg r = seg_combine<FLOAT>(pre, v[u]);
      store_grp(q.state + (long long)(out0 + heads_before) + orank[u], k[u], r.cnt, r.sum, r.mn,
                r.mx);
    }
    heads_before += htot;
    __syncthreads();
  }
}

// One CTA per listed long run: strided gather of the run's groups, then a
// fixed-shape tree reduction (deterministic for a given run).
template <bool FLOAT>
__global__ void __launch_bounds__(256) k_rbk_long(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  const unsigned long long nl = c->n_long;
  unsigned long long* lst;
  unsigned* lpos;
  const SortSrc src = reduce_src(q, s, c->npasses, &lst, &lpos);
  __shared__ long long s_cnt[8];
  __shared__ unsigned long long s_sum[8];
  __shared__ unsigned s_mn[8], s_mx[8];
  const unsigned lane = lane_id(), w = threadIdx.x >> 5;
  for (unsigned long long m = blockIdx.x; m < nl; m += gridDim.x) {
    const unsigned long long a = lst[2 * m], b = lst[2 * m + 1];
    long long cnt = 0;
    unsigned long long isum = 0ull;
    double fsum = 0.0;
    unsigned mn = 0xffffffffu, mx = 0u;
    constexpr int kU = 4;  // gathers in flight per thread
    for (unsigned long long j0 = a + threadIdx.x; j0 < b; j0 += kU * blockDim.x) {
      Grp g[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const unsigned long long j = j0 + (unsigned long long)u * blockDim.x;
        const unsigned long long pi = j < b ? (src.vals ? src.vals[j] : j) : 0ull;
        if (j < b) g[u] = load_grp_v(q.parts + pi);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        if (j0 + (unsigned long long)u * blockDim.x >= b) break;
        cnt += g[u].cnt;
        if (FLOAT)
          fsum += __longlong_as_double((long long)g[u].sum);
        else
          isum += g[u].sum;
        mn = min(mn, g[u].mn);
        mx = max(mx, g[u].mx);
      }
    }
    unsigned long long sbits = FLOAT ? (unsigned long long)__double_as_longlong(fsum) : isum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_down_sync(kFull, cnt, o);
      const unsigned long long os = __shfl_down_sync(kFull, sbits, o);
      if (FLOAT)
        sbits = (unsigned long long)__double_as_longlong(
            __longlong_as_double((long long)sbits) + __longlong_as_double((long long)os));
      else
        sbits += os;
      mn = min(mn, __shfl_down_sync(kFull, mn, o));
      mx = max(mx, __shfl_down_sync(kFull, mx, o));
    }
    if (lane == 0) {
      s_cnt[w] = cnt;
      s_sum[w] = sbits;
      s_mn[w] = mn;
      s_mx[w] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long tc = s_cnt[0];
      unsigned long long ts = s_sum[0];
      unsigned tmn = s_mn[0], tmx = s_mx[0];
      for (int k = 1; k < 8; ++k) {
        tc += s_cnt[k];
        if (FLOAT)
          ts = (unsigned long long)__double_as_longlong(__longlong_as_double((long long)ts) +
                                                        __longlong_as_double((long long)s_sum[k]));
        else
          ts += s_sum[k];
        tmn = min(tmn, s_mn[k]);
        tmx = max(tmx, s_mx[k]);
      }
      store_grp(q.state + lpos[m], src.keys[a], tc, ts, tmn, tmx);
    }
    __syncthreads();
  }
}

// ---- distinct blocks of the window state -----------------------------------

// Block ids never decrease along the sorted state and blocks are runs of many
// groups, so each thread finds the block boundaries of its contiguous share of
// a chunk by galloping and binary search instead of reading every group.
__device__ __forceinline__ unsigned block_of(const QueryDev& q, unsigned long long i) {
  return (unsigned)gkey_block(q.state[i].gkey, q.lb);
}

// First index in (a, b) whose block differs from p (the block of a), else b.
__device__ unsigned long long next_block_change(const QueryDev& q, unsigned long long a,
                                                unsigned long long b, unsigned p) {
  unsigned long long lo = a, step = 1;  // block(lo) == p
  while (lo + step < b && block_of(q, lo + step) == p) {
    lo += step;
    step <<= 1;
  }
  unsigned long long hi = lo + step < b ? lo + step : b;  // block(hi) != p, or hi == b
  while (hi - lo > 1) {
    const unsigned long long mid = lo + ((hi - lo) >> 1);
    if (block_of(q, mid) == p) lo = mid;
    else hi = mid;
  }
  return hi;
}

// Calls f(i, block) for every first group of a block in [a, b), in order.
template <class F>
__device__ void for_block_heads(const QueryDev& q, unsigned long long a, unsigned long long b,
                                F f) {
  if (a >= b) return;
  unsigned p = block_of(q, a);
  if (a == 0 || block_of(q, a - 1) != p) f(a, p);
  for (unsigned long long i = next_block_change(q, a, b, p); i < b;
       i = next_block_change(q, i, b, p)) {
    p = block_of(q, i);
    f(i, p);
  }
}

// This thread's share [*a, *b) of the block's chunk of the state.
__device__ __forceinline__ void thread_share(unsigned long long n, unsigned long long* a,
                                             unsigned long long* b) {
  unsigned long long lo, hi;
  chunk_range(n, blockIdx.x, gridDim.x, &lo, &hi);
  const unsigned long long per = (hi - lo + blockDim.x - 1) / blockDim.x;
  *a = min(hi, lo + per * threadIdx.x);
  *b = min(hi, *a + per);
}

// Only emission reads the block index: when the batch closes no window (most
// batches of a stream whose slide spans many batches) it is left empty.
__device__ __forceinline__ bool closes_windows(const QCtl* c) { return c->w_hi >= c->cursor; }

__global__ void __launch_bounds__(256) k_blk_count(const QueryDev q, const Scratch s) {
  if (!closes_windows(q.ctl)) {
    if (threadIdx.x == 0) s.chunk[blockIdx.x] = 0ull;
    return;
  }
  unsigned long long a, b, cnt = 0;
  thread_share(q.ctl->n_state, &a, &b);
  for_block_heads(q, a, b, [&](unsigned long long, unsigned) { ++cnt; });
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  block_excl_scan(cnt, tmp, &tot);
  if (threadIdx.x == 0) s.chunk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_blk_write(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  if (!closes_windows(c)) return;
  const unsigned long long n = c->n_state;
  unsigned long long a, b, cnt = 0;
  thread_share(n, &a, &b);
  for_block_heads(q, a, b, [&](unsigned long long, unsigned) { ++cnt; });
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  unsigned long long out = s.chunk[blockIdx.x] + block_excl_scan(cnt, tmp, &tot);
  for_block_heads(q, a, b, [&](unsigned long long i, unsigned p) {
    s.blk_id[out] = p;
    s.blk_begin[out] = i;
    ++out;
  });
  if (a < b && b == n) s.blk_begin[c->n_blocks] = n;
  if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) s.blk_begin[0] = 0;
}

}  // namespace

cudaError_t launch_sort_reduce(const QueryDev& q, const Scratch& s, cudaStream_t st,
                               int* launches) {
  static unsigned long long done = 0;  // devices whose limit is set
  const cudaError_t attr =
      set_smem_limit(reinterpret_cast<const void*>(k_sort_scatter), (int)kScatterSmem, &done);
  if (attr != cudaSuccess) return attr;
  int nl = 0;
  k_sort_plan<<<1, 32, 0, st>>>(q.ctl);
  ++nl;
  for (int p = 0; p < 8; ++p) {
    k_sort_hist<<<kGrid, 256, 0, st>>>(q, s, p);
    k_sort_scan<<<256, 256, 0, st>>>(q, s, p);
    k_sort_scatter<<<kGrid, 256, kScatterSmem, st>>>(q, s, p);
    nl += 3;
  }
  k_merge_carry<<<kGrid, 256, 0, st>>>(q, s);
  k_rbk_count<<<kGrid, 256, 0, st>>>(q, s);
  k_scan_chunks<<<1, 1024, 0, st>>>(s.chunk, kGrid, &q.ctl->n_state);
  if (q.value_is_float) {
    k_rbk_write<true><<<kGrid, 256, 0, st>>>(q, s);
    k_rbk_long<true><<<kGrid, 256, 0, st>>>(q, s);
  } else {
    k_rbk_write<false><<<kGrid, 256, 0, st>>>(q, s);
    k_rbk_long<false><<<kGrid, 256, 0, st>>>(q, s);
  }
  nl += 5;
  if (launches) *launches += nl;
  return cudaGetLastError();
}

// Index of distinct blocks of q's window state (into the shared scratch; it
// must be rebuilt before every emission of q).
cudaError_t launch_block_index(const QueryDev& q, const Scratch& s, cudaStream_t st,
                               int* launches) {
  k_blk_count<<<kGrid, 256, 0, st>>>(q, s);
  k_scan_chunks<<<1, 1024, 0, st>>>(s.chunk, kGrid, &q.ctl->n_blocks);
  k_blk_write<<<kGrid, 256, 0, st>>>(q, s);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

}  // namespace lms
