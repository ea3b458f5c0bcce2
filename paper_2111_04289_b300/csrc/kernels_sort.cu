// Partial groups -> sorted, unique window state.
//
// After the fused pass, a query's partial-group arrays hold the groups carried
// over from the previous batch followed by this batch's per-tile groups, in no
// particular order.  This file turns them into the window state: an LSD radix
// sort of the 64-bit group keys (8-bit digits; digits that are equal in every
// key are skipped, which the OR/AND masks gathered by the producers reveal),
// then a reduce-by-key that combines equal (pane, key) groups, then the index
// of distinct panes.  All sizes are read on the device, so the whole sequence
// launches without a host round trip.
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

// Pass p reads the previous pass's output (or the partial keys for p == 0)
// and writes buffer (p & 1) of the scratch pair.
__device__ __forceinline__ SortSrc pass_src(const QueryDev& q, const Scratch& s, int p) {
  if (p == 0) return {q.pkeys, nullptr};
  return ((p - 1) & 1) ? SortSrc{s.keysB, s.valsB} : SortSrc{s.keysA, s.valsA};
}
__device__ __forceinline__ SortSrc final_src(const QueryDev& q, const Scratch& s, int np) {
  if (np == 0) return {q.pkeys, nullptr};
  return ((np - 1) & 1) ? SortSrc{s.keysB, s.valsB} : SortSrc{s.keysA, s.valsA};
}

// The key/value pair the final sort pass did not write (free after the sort).
__device__ __forceinline__ void free_pair(const Scratch& s, int np, unsigned long long** k,
                                          unsigned** v) {
  const bool final_b = np > 0 && ((np - 1) & 1);
  *k = final_b ? s.keysA : s.keysB;
  *v = final_b ? s.valsA : s.valsB;
}

__global__ void k_sort_plan(QCtl* c) {
  if (threadIdx.x != 0) return;
  const unsigned long long n = c->n_parts;
  c->parts_at_sort = n;
  c->n_long = 0;
  const unsigned long long m = c->or_mask ^ c->and_mask;
  int np = 0;
  if (n > 1)
    for (int d = 0; d < 8; ++d)
      if ((m >> (8 * d)) & 0xffull) c->shifts[np++] = 8 * d;
  c->npasses = np;
}

__global__ void __launch_bounds__(256) k_sort_hist(const QueryDev q, const Scratch s, int p) {
  const QCtl* c = q.ctl;
  if (p >= c->npasses) return;
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0u;
  __syncthreads();
  const int shift = c->shifts[p];
  const SortSrc src = pass_src(q, s, p);
  unsigned long long lo, hi;
  chunk_range(c->n_parts, blockIdx.x, gridDim.x, &lo, &hi);
  for (unsigned long long i0 = lo; i0 < hi; i0 += blockDim.x) {
    const unsigned long long i = i0 + threadIdx.x;
    const bool v = i < hi;
    const unsigned d = v ? (unsigned)((src.keys[i] >> shift) & 0xffull) : 256u;
    const unsigned peers = __match_any_sync(kFull, d);
    if (v && (int)lane_id() == __ffs(peers) - 1) atomicAdd(&h[d], (unsigned)__popc(peers));
  }
  __syncthreads();
  s.hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Per digit (one CTA each): exclusive scan over the chunks of hist[d][*] in
// place, digit total -> hist[256 * kGrid + d].
__global__ void __launch_bounds__(256) k_sort_scan(const QueryDev q, const Scratch s, int p) {
  if (p >= q.ctl->npasses) return;
  __shared__ unsigned long long tmp[33];
  unsigned* h = s.hist + blockIdx.x * kGrid;
  const int a = 2 * threadIdx.x;
  const unsigned x0 = a < kGrid ? h[a] : 0u;
  const unsigned x1 = a + 1 < kGrid ? h[a + 1] : 0u;
  unsigned long long tot;
  const unsigned long long r = block_excl_scan((unsigned long long)(x0 + x1), tmp, &tot);
  if (a < kGrid) h[a] = (unsigned)r;
  if (a + 1 < kGrid) h[a + 1] = (unsigned)(r + x0);
  if (threadIdx.x == 0) s.hist[256 * kGrid + blockIdx.x] = (unsigned)tot;
}

__global__ void __launch_bounds__(256) k_sort_scatter(const QueryDev q, const Scratch s, int p) {
  const QCtl* c = q.ctl;
  if (p >= c->npasses) return;
  __shared__ unsigned run[256];
  __shared__ unsigned wcnt[8][256];
  const int tid = threadIdx.x, w = tid >> 5;
  const unsigned lane = lane_id();
  const int shift = c->shifts[p];
  const SortSrc src = pass_src(q, s, p);
  unsigned long long* dk = (p & 1) ? s.keysB : s.keysA;
  unsigned* dv = (p & 1) ? s.valsB : s.valsA;
  unsigned long long lo, hi;
  chunk_range(c->n_parts, blockIdx.x, gridDim.x, &lo, &hi);
  {
    __shared__ unsigned long long tmp[33];
    unsigned long long tot;
    const unsigned long long base =
        block_excl_scan((unsigned long long)s.hist[256 * kGrid + tid], tmp, &tot);
    run[tid] = (unsigned)base + s.hist[tid * gridDim.x + blockIdx.x];
  }
  const unsigned lt = (1u << lane) - 1u;
  for (unsigned long long tb = lo; tb < hi; tb += kScatterTile) {
#pragma unroll
    for (int j = 0; j < 8; ++j) wcnt[w][lane + 32 * j] = 0u;
    __syncthreads();
    unsigned long long kk[8];
    unsigned vv[8], dd[8], rr[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const unsigned long long i = tb + (unsigned long long)(w * 256 + r * 32) + lane;
      const bool v = i < hi;
      kk[r] = v ? src.keys[i] : 0ull;
      vv[r] = v ? (src.vals ? src.vals[i] : (unsigned)i) : 0u;
      dd[r] = v ? (unsigned)((kk[r] >> shift) & 0xffull) : 256u;
      const unsigned peers = __match_any_sync(kFull, dd[r]);
      rr[r] = (v ? wcnt[w][dd[r]] : 0u) + __popc(peers & lt);
      __syncwarp();
      if (v && (int)lane == __ffs(peers) - 1) wcnt[w][dd[r]] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {
      unsigned acc = run[tid];
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) {
        const unsigned cnt = wcnt[ww][tid];
        wcnt[ww][tid] = acc;
        acc += cnt;
      }
      run[tid] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if (dd[r] < 256u) {
        const unsigned pos = wcnt[w][dd[r]] + rr[r];
        dk[pos] = kk[r];
        dv[pos] = vv[r];
      }
    }
    __syncthreads();
  }
}

// ---- reduce-by-key: sorted partials -> unique groups (window state) -------

__global__ void __launch_bounds__(256) k_rbk_count(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  const SortSrc src = final_src(q, s, c->npasses);
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

// Runs of equal keys up to this length are reduced by the thread at their head;
// longer runs (a hot key's groups from many tiles of one pane) are listed and
// reduced by whole CTAs in k_rbk_long.
constexpr unsigned long long kSerialRun = 32;

template <bool FLOAT>
__global__ void __launch_bounds__(256) k_rbk_write(const QueryDev q, const Scratch s) {
  QCtl* c = q.ctl;
  const unsigned long long n = c->n_parts;
  const SortSrc src = final_src(q, s, c->npasses);
  unsigned long long* lst;
  unsigned* lpos;
  free_pair(s, c->npasses, &lst, &lpos);
  unsigned long long lo, hi;
  chunk_range(n, blockIdx.x, gridDim.x, &lo, &hi);
  __shared__ unsigned long long tmp[33];
  unsigned long long out = s.chunk[blockIdx.x];
  for (unsigned long long i0 = lo; i0 < hi; i0 += blockDim.x) {
    const unsigned long long i = i0 + threadIdx.x;
    const bool v = i < hi;
    const unsigned long long k = v ? src.keys[i] : 0ull;
    const bool head = v && (i == 0 || k != src.keys[i - 1]);
    unsigned long long tot;
    const unsigned long long r = block_excl_scan(head ? 1ull : 0ull, tmp, &tot);
    if (head) {
      if (i + kSerialRun < n && src.keys[i + kSerialRun] == k) {
        // long run: find its end (gallop, then bisect) and hand it over
        unsigned long long a = i + kSerialRun, step = kSerialRun;
        unsigned long long b = n;
        while (true) {
          const unsigned long long t = a + step;
          if (t >= n || src.keys[t] != k) {
            b = t < n ? t : n;
            break;
          }
          a = t;
          step <<= 1;
        }
        while (b - a > 1) {  // keys[a] == k, keys[b] != k (or b == n)
          const unsigned long long m = a + ((b - a) >> 1);
          if (src.keys[m] == k) a = m;
          else b = m;
        }
        const unsigned long long slot = atomicAdd(&c->n_long, 1ull);
        lst[2 * slot] = i;
        lst[2 * slot + 1] = b;
        lpos[slot] = (unsigned)(out + r);
      } else {
        long long cnt = 0;
        unsigned long long isum = 0ull;
        double fsum = 0.0;
        unsigned mn = 0xffffffffu, mx = 0u;
        for (unsigned long long j = i; j < n && src.keys[j] == k; ++j) {
          const unsigned long long pi = src.vals ? src.vals[j] : j;
          const Grp g = load_grp(q.parts + pi);
          cnt += g.cnt;
          if (FLOAT)
            fsum += __longlong_as_double((long long)g.sum);
          else
            isum += g.sum;
          mn = min(mn, g.mn);
          mx = max(mx, g.mx);
        }
        store_grp(q.state + out + r, k, cnt,
                  FLOAT ? (unsigned long long)__double_as_longlong(fsum) : isum, mn, mx);
      }
    }
    out += tot;
  }
}

// One CTA per listed long run: strided gather of the run's groups, then a
// fixed-shape tree reduction (deterministic for a given run).
template <bool FLOAT>
__global__ void __launch_bounds__(256) k_rbk_long(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  const unsigned long long nl = c->n_long;
  const SortSrc src = final_src(q, s, c->npasses);
  unsigned long long* lst;
  unsigned* lpos;
  free_pair(s, c->npasses, &lst, &lpos);
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
    for (unsigned long long j = a + threadIdx.x; j < b; j += blockDim.x) {
      const unsigned long long pi = src.vals ? src.vals[j] : j;
      const Grp g = load_grp(q.parts + pi);
      cnt += g.cnt;
      if (FLOAT)
        fsum += __longlong_as_double((long long)g.sum);
      else
        isum += g.sum;
      mn = min(mn, g.mn);
      mx = max(mx, g.mx);
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

// ---- distinct panes of the window state ------------------------------------

__global__ void __launch_bounds__(256) k_pane_count(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  unsigned long long lo, hi;
  chunk_range(c->n_state, blockIdx.x, gridDim.x, &lo, &hi);
  unsigned long long cnt = 0;
  for (unsigned long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
    cnt += (i == 0 || (q.state[i].gkey >> 32) != (q.state[i - 1].gkey >> 32)) ? 1ull : 0ull;
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  block_excl_scan(cnt, tmp, &tot);
  if (threadIdx.x == 0) s.chunk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_pane_write(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  const unsigned long long n = c->n_state;
  unsigned long long lo, hi;
  chunk_range(n, blockIdx.x, gridDim.x, &lo, &hi);
  __shared__ unsigned long long tmp[33];
  unsigned long long out = s.chunk[blockIdx.x];
  for (unsigned long long i0 = lo; i0 < hi; i0 += blockDim.x) {
    const unsigned long long i = i0 + threadIdx.x;
    const bool v = i < hi;
    const unsigned p = v ? (unsigned)(q.state[i].gkey >> 32) : 0u;
    const bool head = v && (i == 0 || p != (unsigned)(q.state[i - 1].gkey >> 32));
    unsigned long long tot;
    const unsigned long long r = block_excl_scan(head ? 1ull : 0ull, tmp, &tot);
    if (head) {
      s.pane_id[out + r] = p;
      s.pane_begin[out + r] = i;
    }
    if (v && i == n - 1) s.pane_begin[c->n_panes] = n;
    out += tot;
  }
}

}  // namespace

cudaError_t launch_sort_reduce(const QueryDev& q, const Scratch& s, cudaStream_t st,
                               int* launches) {
  int nl = 0;
  k_sort_plan<<<1, 32, 0, st>>>(q.ctl);
  ++nl;
  for (int p = 0; p < 8; ++p) {
    k_sort_hist<<<kGrid, 256, 0, st>>>(q, s, p);
    k_sort_scan<<<256, 256, 0, st>>>(q, s, p);
    k_sort_scatter<<<kGrid, 256, 0, st>>>(q, s, p);
    nl += 3;
  }
  k_rbk_count<<<kGrid, 256, 0, st>>>(q, s);
  k_scan_chunks<<<1, 1024, 0, st>>>(s.chunk, kGrid, &q.ctl->n_state);
  if (q.value_is_float) {
    k_rbk_write<true><<<kGrid, 256, 0, st>>>(q, s);
    k_rbk_long<true><<<kGrid, 256, 0, st>>>(q, s);
  } else {
    k_rbk_write<false><<<kGrid, 256, 0, st>>>(q, s);
    k_rbk_long<false><<<kGrid, 256, 0, st>>>(q, s);
  }
  nl += 4;
  if (launches) *launches += nl;
  return cudaGetLastError();
}

// Index of distinct panes of q's window state (into the shared scratch; it
// must be rebuilt before every emission of q).
cudaError_t launch_pane_index(const QueryDev& q, const Scratch& s, cudaStream_t st,
                              int* launches) {
  k_pane_count<<<kGrid, 256, 0, st>>>(q, s);
  k_scan_chunks<<<1, 1024, 0, st>>>(s.chunk, kGrid, &q.ctl->n_panes);
  k_pane_write<<<kGrid, 256, 0, st>>>(q, s);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

}  // namespace lms
