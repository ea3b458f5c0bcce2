// Post-aggregation over the rows one batch emitted (Table III: LR2S's HAVING
// avgSpeed < 40, CM1's ORDER BY SUM(cpu)), run after the emission and before
// the carry, on the batch's rows rows[row_base .. row_base + rows_batch):
//   * HAVING agg OP c: an order-preserving compaction keeps the rows whose
//     aggregate, as a double, passes the IEEE comparison (count / scan /
//     write into a scratch row buffer, then copied back);
//   * ORDER BY agg: each window's rows (contiguous, key-ordered) are sorted by
//     the aggregate, ascending or descending, equal values in key order: a
//     bitonic sort of (order-preserving code of the value, position) pairs in
//     shared memory, then the rows are gathered through the scratch buffer.
//     A window may hold at most kOrderMax rows (the flag kErrOrderBy otherwise).
#include <climits>

#include "lms_device.cuh"

namespace lms {
namespace {

constexpr int kOrderThreads = 512;
constexpr size_t kOrderSmem = (size_t)kOrderMax * (8 + 4);

// The value of aggregate `agg` (1 count, 2 sum, 3 min, 4 max, 5 avg) of a row.
template <bool FLOAT>
__device__ __forceinline__ double row_agg(const ResultRowDev& r, int agg) {
  switch (agg) {
    case 1: return (double)r.count;
    case 2: return FLOAT ? __longlong_as_double((long long)r.sum) : (double)(long long)r.sum;
    case 3: return FLOAT ? (double)__uint_as_float(r.mn) : (double)(int)r.mn;
    case 4: return FLOAT ? (double)__uint_as_float(r.mx) : (double)(int)r.mx;
    default: return r.avg;
  }
}

__device__ __forceinline__ ResultRowDev load_row(const ResultRowDev* p) {
  const uint4* s = reinterpret_cast<const uint4*>(p);
  const uint4 a = s[0], b = s[1], c = s[2];
  ResultRowDev r;
  r.window_start = (long long)(((unsigned long long)a.y << 32) | a.x);
  r.count = (long long)(((unsigned long long)a.w << 32) | a.z);
  r.sum = ((unsigned long long)b.y << 32) | b.x;
  r.avg = __longlong_as_double((long long)(((unsigned long long)b.w << 32) | b.z));
  r.key = c.x;
  r.mn = c.y;
  r.mx = c.z;
  r.qid = c.w;
  return r;
}

__device__ __forceinline__ void copy_row(ResultRowDev* dst, const ResultRowDev* src) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(dst);
  d[0] = s[0];
  d[1] = s[1];
  d[2] = s[2];
}

template <bool FLOAT>
__device__ __forceinline__ bool having_pass(const QueryDev& q, const ResultRowDev* p) {
  return filter_pass_f(q.having_op, row_agg<FLOAT>(load_row(p), q.having_agg), q.having_value);
}

template <bool FLOAT>
__global__ void __launch_bounds__(256) k_having_count(const QueryDev q, const Scratch s,
                                                      const ResultRowDev* rows) {
  const QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const ResultRowDev* r = rows + c->row_base;
  unsigned long long lo, hi;
  chunk_range(c->rows_batch, blockIdx.x, gridDim.x, &lo, &hi);
  unsigned long long cnt = 0;
  for (unsigned long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
    cnt += having_pass<FLOAT>(q, r + i) ? 1ull : 0ull;
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  block_excl_scan(cnt, tmp, &tot);
  if (threadIdx.x == 0) s.chunk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_having_scan(const QueryDev q, const Scratch s) {
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
  if (threadIdx.x == 0) c->rows_kept = tot;
}

template <bool FLOAT>
__global__ void __launch_bounds__(256) k_having_write(const QueryDev q, const Scratch s,
                                                      const ResultRowDev* rows, ResultRowDev* tmp_rows) {
  const QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const ResultRowDev* r = rows + c->row_base;
  unsigned long long lo, hi;
  chunk_range(c->rows_batch, blockIdx.x, gridDim.x, &lo, &hi);
  __shared__ unsigned long long tmp[33];
  unsigned long long out = s.chunk[blockIdx.x];
  for (unsigned long long i0 = lo; i0 < hi; i0 += blockDim.x) {
    const unsigned long long i = i0 + threadIdx.x;
    const bool keep = i < hi && having_pass<FLOAT>(q, r + i);
    unsigned long long tot;
    const unsigned long long p = block_excl_scan(keep ? 1ull : 0ull, tmp, &tot);
    if (keep) copy_row(tmp_rows + out + p, r + i);
    out += tot;
  }
}

__global__ void __launch_bounds__(256) k_having_copy(const QueryDev q, ResultRowDev* rows,
                                                     const ResultRowDev* tmp_rows) {
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long n = c->rows_kept;
  ResultRowDev* r = rows + c->row_base;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    copy_row(r + i, tmp_rows + i);
}

__global__ void k_having_done(const QueryDev q) {
  QCtl* c = q.ctl;
  if (threadIdx.x != 0 || (c->err & kErrNeedRetry)) return;
  c->rows_batch = c->rows_kept;
}

// Order-preserving code of a double (zeros of either sign equal).
__device__ __forceinline__ unsigned long long order_code(double x, bool desc) {
  if (x == 0.0) x = 0.0;
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long code = (u >> 63) ? ~u : (u | (1ull << 63));
  return desc ? ~code : code;
}

// One CTA per chunk of the batch's rows; it sorts the windows that start in
// its chunk (a window may run past the chunk).
template <bool FLOAT>
__global__ void __launch_bounds__(kOrderThreads, 1)
    k_order(const QueryDev q, ResultRowDev* rows, ResultRowDev* tmp_rows) {
  extern __shared__ __align__(16) unsigned char osm[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(osm);
  unsigned* pos = reinterpret_cast<unsigned*>(key + kOrderMax);
  __shared__ unsigned s_list[kOrderThreads];
  __shared__ unsigned long long s_tmp[33];
  __shared__ unsigned long long s_end;
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long n = c->rows_batch;
  ResultRowDev* r = rows + c->row_base;
  ResultRowDev* t = tmp_rows + c->row_base;
  const bool desc = q.order_desc != 0;
  unsigned long long lo, hi;
  chunk_range(n, blockIdx.x, gridDim.x, &lo, &hi);
  for (unsigned long long tb = lo; tb < hi; tb += kOrderThreads) {
    // the window starts in this tile, in order
    const unsigned long long i = tb + threadIdx.x;
    const bool st = i < hi && (i == 0 || r[i].window_start != r[i - 1].window_start);
    unsigned long long ns64;
    const unsigned long long sp = block_excl_scan(st ? 1ull : 0ull, s_tmp, &ns64);
    if (st) s_list[sp] = (unsigned)(i - tb);
    __syncthreads();
    const unsigned ns = (unsigned)ns64;
    for (unsigned w = 0; w < ns; ++w) {
      const unsigned long long a = tb + s_list[w];
      // its end: the first row after a with another window start
      const long long ws = r[a].window_start;
      unsigned long long e = n;
      for (unsigned long long j0 = a + 1; j0 < n; j0 += kOrderThreads) {
        const unsigned long long j = j0 + threadIdx.x;
        const bool diff = j < n && r[j].window_start != ws;
        const int any = __syncthreads_or(diff ? 1 : 0);
        if (any) {
          if (threadIdx.x == 0) s_end = n;
          __syncthreads();
          if (diff) atomicMin(&s_end, j);
          __syncthreads();
          e = s_end;
          break;
        }
      }
      __syncthreads();
      const unsigned long long len = e - a;
      if (len > (unsigned long long)kOrderMax) {
        if (threadIdx.x == 0) atomicOr(&c->err, kErrOrderBy);
        continue;
      }
      if (len < 2) continue;
      unsigned m = 2;
      while (m < len) m <<= 1;
      for (unsigned k = threadIdx.x; k < m; k += kOrderThreads) {
        if (k < len) {
          key[k] = order_code(row_agg<FLOAT>(load_row(r + a + k), q.order_agg), desc);
          pos[k] = k;
        } else {
          key[k] = ~0ull;
          pos[k] = 0xffffffffu;
        }
      }
      __syncthreads();
      // bitonic sort of (key, pos): equal values keep their key order
      for (unsigned kk = 2; kk <= m; kk <<= 1) {
        for (unsigned jj = kk >> 1; jj > 0; jj >>= 1) {
          for (unsigned x = threadIdx.x; x < m; x += kOrderThreads) {
            const unsigned y = x ^ jj;
            if (y > x) {
              const bool up = (x & kk) == 0;
              const unsigned long long kx = key[x], ky = key[y];
              const unsigned px = pos[x], py = pos[y];
              const bool gt = kx > ky || (kx == ky && px > py);
              if (gt == up) {
                key[x] = ky;
                key[y] = kx;
                pos[x] = py;
                pos[y] = px;
              }
            }
          }
          __syncthreads();
        }
      }
      for (unsigned k = threadIdx.x; k < len; k += kOrderThreads) copy_row(t + a + k, r + a + pos[k]);
      __syncthreads();
      for (unsigned k = threadIdx.x; k < len; k += kOrderThreads) copy_row(r + a + k, t + a + k);
      __syncthreads();
    }
  }
}

}  // namespace

cudaError_t launch_post(const QueryDev& q, const Scratch& s, ResultRowDev* rows,
                        ResultRowDev* tmp_rows, int sms, cudaStream_t st, int* launches) {
  int nl = 0;
  if (q.having_agg) {
    if (q.value_is_float) k_having_count<true><<<kGrid, 256, 0, st>>>(q, s, rows);
    else k_having_count<false><<<kGrid, 256, 0, st>>>(q, s, rows);
    k_having_scan<<<1, 256, 0, st>>>(q, s);
    if (q.value_is_float) k_having_write<true><<<kGrid, 256, 0, st>>>(q, s, rows, tmp_rows);
    else k_having_write<false><<<kGrid, 256, 0, st>>>(q, s, rows, tmp_rows);
    k_having_copy<<<2 * sms, 256, 0, st>>>(q, rows, tmp_rows);
    k_having_done<<<1, 32, 0, st>>>(q);
    nl += 5;
  }
  if (q.order_agg) {
    static unsigned long long done_f = 0, done_i = 0;
    cudaError_t e = q.value_is_float
                        ? set_smem_limit(reinterpret_cast<const void*>(k_order<true>), (int)kOrderSmem, &done_f)
                        : set_smem_limit(reinterpret_cast<const void*>(k_order<false>), (int)kOrderSmem, &done_i);
    if (e != cudaSuccess) return e;
    if (q.value_is_float) k_order<true><<<sms, kOrderThreads, kOrderSmem, st>>>(q, rows, tmp_rows);
    else k_order<false><<<sms, kOrderThreads, kOrderSmem, st>>>(q, rows, tmp_rows);
    ++nl;
  }
  if (launches) *launches += nl;
  return cudaGetLastError();
}

}  // namespace lms
