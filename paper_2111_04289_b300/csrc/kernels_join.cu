// Windowed equi-join of two sides of a stream (Table III's LR1S / LR1T; Join
// of Table II), reported per (window, key) in factored form.
//
// Each side runs as a hidden windowed aggregation (its own query: filter =
// the side's predicate, the join's window), so after a batch both sides' rows
// of the windows it closed are sorted by (window_start, key).  A key of a
// window is in the join iff it has a row on both sides: every left row looks
// its (window_start, key) up in the right rows by binary search; the matches
// are counted per chunk, scanned, and written in left-row order (which is
// (window_start, key) order) with pairs = left count * right count and both
// sides' counts and sums.  Then the sides' row buffers are emptied.
#include "lms_device.cuh"

namespace lms {
namespace {

constexpr unsigned kJoinPending = kJoinPendingBit;    // the join of this batch has not completed
constexpr unsigned kJoinOverflow = kJoinOverflowBit;  // the join's row buffer is too small

__device__ __forceinline__ bool row_less(long long ws_a, unsigned k_a, long long ws_b,
                                         unsigned k_b) {
  return ws_a < ws_b || (ws_a == ws_b && k_a < k_b);
}

// Index of the right row with this (window_start, key), or -1.
__device__ __forceinline__ long long find_right(const ResultRowDev* r, unsigned long long n,
                                                long long ws, unsigned key) {
  unsigned long long lo = 0, hi = n;
  while (lo < hi) {
    const unsigned long long mid = (lo + hi) >> 1;
    if (row_less(r[mid].window_start, r[mid].key, ws, key)) lo = mid + 1;
    else hi = mid;
  }
  return (lo < n && r[lo].window_start == ws && r[lo].key == key) ? (long long)lo : -1ll;
}

__device__ __forceinline__ bool sides_ready(const JoinArgs& a) {
  return !((a.lc->err | a.rc->err) & kErrNeedRetry);
}

__global__ void k_join_begin(const JoinArgs a) {
  if (threadIdx.x != 0) return;
  a.jc->err = kJoinPending;
  a.jc->rows_batch = 0ull;
}

__global__ void __launch_bounds__(256) k_join_count(const JoinArgs a, const Scratch s) {
  if (!sides_ready(a) || !(a.jc->err & kJoinPending)) return;
  const unsigned long long nl = a.lc->rows_batch, nr = a.rc->rows_batch;
  const ResultRowDev* L = a.lrows + (a.lc->row_base - nl);
  const ResultRowDev* R = a.rrows + (a.rc->row_base - nr);
  unsigned long long lo, hi;
  chunk_range(nl, blockIdx.x, gridDim.x, &lo, &hi);
  unsigned long long cnt = 0;
  for (unsigned long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
    cnt += find_right(R, nr, L[i].window_start, L[i].key) >= 0 ? 1ull : 0ull;
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  block_excl_scan(cnt, tmp, &tot);
  if (threadIdx.x == 0) s.chunk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_join_scan(const JoinArgs a, const Scratch s) {
  if (!sides_ready(a) || !(a.jc->err & kJoinPending)) return;
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
    a.jc->rows_batch = tot;
    if (a.jc->row_base + tot > a.cap) a.jc->err |= kJoinOverflow;
    else a.jc->err &= ~kJoinOverflow;
  }
}

__global__ void __launch_bounds__(256) k_join_write(const JoinArgs a, const Scratch s) {
  if (!sides_ready(a) || !(a.jc->err & kJoinPending) || (a.jc->err & kJoinOverflow)) return;
  const unsigned long long nl = a.lc->rows_batch, nr = a.rc->rows_batch;
  const ResultRowDev* L = a.lrows + (a.lc->row_base - nl);
  const ResultRowDev* R = a.rrows + (a.rc->row_base - nr);
  JoinRowDev* out = a.out + a.jc->row_base;
  unsigned long long lo, hi;
  chunk_range(nl, blockIdx.x, gridDim.x, &lo, &hi);
  __shared__ unsigned long long tmp[33];
  unsigned long long o = s.chunk[blockIdx.x];
  for (unsigned long long i0 = lo; i0 < hi; i0 += blockDim.x) {
    const unsigned long long i = i0 + threadIdx.x;
    long long j = -1;
    if (i < hi) j = find_right(R, nr, L[i].window_start, L[i].key);
    unsigned long long tot;
    const unsigned long long p = block_excl_scan(j >= 0 ? 1ull : 0ull, tmp, &tot);
    if (j >= 0) {
      const ResultRowDev& l = L[i];
      const ResultRowDev& r = R[j];
      JoinRowDev* d = out + o + p;
      d->window_start = l.window_start;
      d->pairs = l.count * r.count;
      d->left_count = l.count;
      d->right_count = r.count;
      d->left_sum = l.sum;
      d->right_sum = r.sum;
      d->key = l.key;
      d->jid = (unsigned)a.jid;
    }
    o += tot;
  }
}

__global__ void k_join_done(const JoinArgs a) {
  if (threadIdx.x != 0) return;
  if (!sides_ready(a) || !(a.jc->err & kJoinPending) || (a.jc->err & kJoinOverflow)) return;
  a.jc->row_base += a.jc->rows_batch;
  a.lc->row_base = 0ull;  // the sides' rows are consumed
  a.rc->row_base = 0ull;
  a.jc->err &= ~kJoinPending;
}

}  // namespace

cudaError_t launch_join(const JoinArgs& a, const Scratch& s, bool begin, cudaStream_t st,
                        int* launches) {
  int nl = 0;
  if (begin) {
    k_join_begin<<<1, 32, 0, st>>>(a);
    ++nl;
  }
  k_join_count<<<kGrid, 256, 0, st>>>(a, s);
  k_join_scan<<<1, 256, 0, st>>>(a, s);
  k_join_write<<<kGrid, 256, 0, st>>>(a, s);
  k_join_done<<<1, 32, 0, st>>>(a);
  if (launches) *launches += nl + 4;
  return cudaGetLastError();
}

}  // namespace lms
