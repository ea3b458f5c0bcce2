// Watermark, window enumeration, window assembly from panes, row emission and
// the carry of still-open panes into the next micro-batch.
//
// After a micro-batch the watermark is max(previous, max ts of the batch -
// allowed lateness); every window whose end is <= the watermark closes (the
// paper's per-micro-batch output step, Section III-A; window semantics as in
// the public header).  A window of K panes is assembled from the sorted
// window state: its panes are K contiguous, key-sorted runs of the state, so
// the CTA that owns the window merges the runs (merge path, pairwise rounds)
// in shared memory — or, for windows larger than shared memory, in global
// scratch — and emits one row per distinct key, in key order.  Rows of all
// closed windows are written in (window_start, key) order at offsets from a
// device-wide scan of the per-window row counts.
#include <climits>

#include "lms_device.cuh"

namespace lms {
namespace {

constexpr int kEmitThreads = 512;
constexpr unsigned kEmitCap = 12288;  // entries per shared buffer (2 buffers, 192 KB)
constexpr size_t kEmitSmem = 2ull * kEmitCap * sizeof(unsigned long long);

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
  c->big_windows = 0ull;
  c->rows_batch = 0ull;
  c->n_windows = 0ull;
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
    }
    out += tot;
  }
}

// Pairwise merge rounds of `nr` sorted runs of A (boundaries bc[0..nr],
// bc[nr] = len), ping-ponging with B.  Values are distinct.  Returns the
// buffer holding the fully merged sequence.  All threads must call.
__device__ unsigned long long* merge_runs(unsigned long long* A, unsigned long long* B,
                                          unsigned* bc, unsigned* bn, int nr, unsigned len) {
  while (nr > 1) {
    const int np = (nr + 1) >> 1;
    for (unsigned ch = threadIdx.x; ch * 8u < len; ch += blockDim.x) {
      unsigned o = ch * 8u;
      const unsigned oe = min(len, o + 8u);
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
          if (A[s0 + mid] < A[s1 + diag - 1u - mid]) a = mid + 1u; else b = mid;
        }
        unsigned i = a, k = diag - a;
        const unsigned stop = min(oe, s2);
        while (o < stop) {
          if (k >= lb || (i < la && A[s0 + i] < A[s1 + k])) B[o++] = A[s0 + i++];
          else B[o++] = A[s1 + k++];
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

template <bool FLOAT>
__device__ __forceinline__ void write_row(const QueryDev& q, ResultRowDev* out, long long wstart,
                                          unsigned key, long long cnt, unsigned long long sbits,
                                          unsigned mn, unsigned mx) {
  double avg;
  if (FLOAT) avg = __longlong_as_double((long long)sbits) / (double)cnt;
  else avg = (double)(long long)sbits / (double)cnt;
  unsigned mnv = 0u, mxv = 0u;
  if (q.agg_mask & 4u) mnv = FLOAT ? dec_f32_bits(mn) : (unsigned)dec_i32(mn);
  if (q.agg_mask & 8u) mxv = FLOAT ? dec_f32_bits(mx) : (unsigned)dec_i32(mx);
  uint4* o = reinterpret_cast<uint4*>(out);
  o[0] = make_uint4((unsigned)wstart, (unsigned)((unsigned long long)wstart >> 32), (unsigned)cnt,
                    (unsigned)((unsigned long long)cnt >> 32));
  const unsigned long long ab = (unsigned long long)__double_as_longlong(avg);
  o[1] = make_uint4((unsigned)sbits, (unsigned)(sbits >> 32), (unsigned)ab, (unsigned)(ab >> 32));
  o[2] = make_uint4(key, mnv, mxv, (unsigned)q.qid);
}

// E1 (WRITE=false): rows per closed window.  E2 (WRITE=true): the rows.
template <bool FLOAT, bool WRITE>
__global__ void __launch_bounds__(kEmitThreads, 1)
    k_emit(const QueryDev q, const Scratch s, ResultRowDev* rows, unsigned cap) {
  extern __shared__ __align__(16) unsigned long long esm[];
  __shared__ unsigned bnd0[kMaxRuns + 1], bnd1[kMaxRuns + 1];
  __shared__ unsigned long long tmp[33];
  __shared__ unsigned long long s_off;
  QCtl* c = q.ctl;
  if (c->err & kErrNeedRetry) return;
  const unsigned long long W = c->n_windows;
  const int tid = threadIdx.x;
  const unsigned long long row_base = c->row_base;
  for (unsigned long long wi = blockIdx.x; wi < W; wi += gridDim.x) {
    const long long w = s.win_w[wi];
    const unsigned j0 = s.win_j0[wi], j1 = s.win_j1[wi];
    const unsigned long long b0 = s.pane_begin[j0], b1 = s.pane_begin[j1];
    const unsigned len = (unsigned)(b1 - b0);
    const int nr = (int)(j1 - j0);
    const long long wstart = (w - kPaneBias) * (long long)q.slide + q.base;
    if (nr == 1) {  // one pane: the state run is already key-sorted and unique
      if (!WRITE) {
        if (tid == 0) s.win_rows[wi] = len;
      } else {
        ResultRowDev* out = rows + row_base + s.win_rows[wi];
        for (unsigned i = tid; i < len; i += blockDim.x) {
          const unsigned long long g = b0 + i;
          write_row<FLOAT>(q, out + i, wstart, (unsigned)q.state.gkey[g], q.state.cnt[g],
                           q.state.sum[g], q.state.mn[g], q.state.mx[g]);
        }
      }
      continue;
    }
    const bool big = len > cap;
    unsigned long long* A;
    unsigned long long* B;
    unsigned long long* S;
    if (big) {
      if (!WRITE) {
        if (tid == 0) {
          unsigned long long off = atomicAdd(&c->pool_used, 2ull * len);
          if (off + 2ull * len > s.pool_cap) {
            atomicOr(&c->err, kErrPoolOverflow);
            off = ~0ull;
          } else {
            atomicAdd(&c->big_windows, 1ull);
          }
          s_off = off;
        }
        __syncthreads();
        const unsigned long long off = s_off;
        __syncthreads();
        if (off == ~0ull) {
          if (tid == 0) s.win_rows[wi] = 0ull;
          continue;
        }
        A = s.pool + off;
        B = A + len;
      } else {
        S = s.pool + s.win_scr[wi];
      }
    } else {
      A = esm;
      B = esm + cap;
    }
    if (!(WRITE && big)) {
      for (unsigned i = tid; i < len; i += blockDim.x)
        A[i] = ((q.state.gkey[b0 + i] & 0xffffffffull) << 32) | i;
      for (int r = tid; r <= nr; r += blockDim.x)
        bnd0[r] = (unsigned)(s.pane_begin[j0 + r] - b0);
      __syncthreads();
      S = merge_runs(A, B, bnd0, bnd1, nr, len);
      if (!WRITE && big && tid == 0) s.win_scr[wi] = (unsigned long long)(S - s.pool);
    }
    // distinct keys of the merged run
    unsigned long long run = 0;
    for (unsigned i0 = 0; i0 < len; i0 += blockDim.x) {
      const unsigned i = i0 + tid;
      const bool v = i < len;
      const unsigned long long x = v ? S[i] : 0ull;
      const bool head = v && (i == 0 || (x >> 32) != (S[i - 1] >> 32));
      unsigned long long tot;
      const unsigned long long r = block_excl_scan(head ? 1ull : 0ull, tmp, &tot);
      if (WRITE && head) {
        const unsigned key = (unsigned)(x >> 32);
        long long cnt = 0;
        unsigned long long isum = 0ull;
        double fsum = 0.0;
        unsigned mn = 0xffffffffu, mx = 0u;
        for (unsigned t = i; t < len && (unsigned)(S[t] >> 32) == key; ++t) {
          const unsigned long long g = b0 + (S[t] & 0xffffffffull);
          cnt += q.state.cnt[g];
          if (FLOAT) fsum += __longlong_as_double((long long)q.state.sum[g]);
          else isum += q.state.sum[g];
          mn = min(mn, q.state.mn[g]);
          mx = max(mx, q.state.mx[g]);
        }
        const unsigned long long sb =
            FLOAT ? (unsigned long long)__double_as_longlong(fsum) : isum;
        write_row<FLOAT>(q, rows + row_base + s.win_rows[wi] + run + r, wstart, key, cnt, sb, mn,
                         mx);
      }
      run += tot;
    }
    if (!WRITE && tid == 0) s.win_rows[wi] = run;
    __syncthreads();
  }
}

// Device-wide exclusive scan of win_rows[0..n_windows): per-chunk sums, chunk
// scan (total -> rows_batch, capacity check), per-chunk apply.
__global__ void __launch_bounds__(256) k_rows_sum(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  unsigned long long lo, hi;
  chunk_range(c->err & kErrNeedRetry ? 0ull : c->n_windows, blockIdx.x, gridDim.x, &lo, &hi);
  unsigned long long cnt = 0;
  for (unsigned long long i = lo + threadIdx.x; i < hi; i += blockDim.x) cnt += s.win_rows[i];
  __shared__ unsigned long long tmp[33];
  unsigned long long tot;
  block_excl_scan(cnt, tmp, &tot);
  if (threadIdx.x == 0) s.chunk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_rows_scan(const QueryDev q, const Scratch s,
                                                    unsigned long long rows_cap) {
  __shared__ unsigned long long tmp[33];
  const unsigned long long v = (int)threadIdx.x < kGrid ? s.chunk[threadIdx.x] : 0ull;
  unsigned long long tot;
  const unsigned long long r = block_excl_scan(v, tmp, &tot);
  if ((int)threadIdx.x < kGrid) s.chunk[threadIdx.x] = r;
  if (threadIdx.x == 0) {
    QCtl* c = q.ctl;
    c->rows_batch = tot;
    if (c->row_base + tot > rows_cap) atomicOr(&c->err, kErrRowsOverflow);
  }
}

__global__ void __launch_bounds__(256) k_rows_apply(const QueryDev q, const Scratch s) {
  const QCtl* c = q.ctl;
  unsigned long long lo, hi;
  chunk_range(c->err & kErrNeedRetry ? 0ull : c->n_windows, blockIdx.x, gridDim.x, &lo, &hi);
  __shared__ unsigned long long tmp[33];
  unsigned long long out = s.chunk[blockIdx.x];
  for (unsigned long long i0 = lo; i0 < hi; i0 += blockDim.x) {
    const unsigned long long i = i0 + threadIdx.x;
    const unsigned long long v = i < hi ? s.win_rows[i] : 0ull;
    unsigned long long tot;
    const unsigned long long r = block_excl_scan(v, tmp, &tot);
    if (i < hi) s.win_rows[i] = out + r;
    out += tot;
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
    const unsigned long long g = q.state.gkey[from + i];
    q.parts.gkey[i] = g;
    q.parts.cnt[i] = q.state.cnt[from + i];
    q.parts.sum[i] = q.state.sum[from + i];
    q.parts.mn[i] = q.state.mn[from + i];
    q.parts.mx[i] = q.state.mx[from + i];
    o_acc |= g;
    a_acc &= g;
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

template <bool FLOAT, bool WRITE>
cudaError_t launch_emit_t(const QueryDev& q, const Scratch& s, ResultRowDev* rows, int grid,
                          size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_emit<FLOAT, WRITE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kEmitSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_emit<FLOAT, WRITE><<<grid, kEmitThreads, smem, st>>>(q, s, rows, smem ? kEmitCap : 0u);
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
  const size_t smem = q.k > 1 ? kEmitSmem : 0;
  const int grid = q.k > 1 ? sms : 4 * sms;
  if (ev4) cudaEventRecord(ev4[0], st);
  cudaError_t e = q.value_is_float ? launch_emit_t<true, false>(q, s, rows, grid, smem, st)
                                   : launch_emit_t<false, false>(q, s, rows, grid, smem, st);
  if (ev4) cudaEventRecord(ev4[1], st);
  if (e != cudaSuccess) return e;
  k_rows_sum<<<kGrid, 256, 0, st>>>(q, s);
  k_rows_scan<<<1, 1024, 0, st>>>(q, s, rows_cap);
  k_rows_apply<<<kGrid, 256, 0, st>>>(q, s);
  if (ev4) cudaEventRecord(ev4[2], st);
  e = q.value_is_float ? launch_emit_t<true, true>(q, s, rows, grid, smem, st)
                       : launch_emit_t<false, true>(q, s, rows, grid, smem, st);
  if (ev4) cudaEventRecord(ev4[3], st);
  if (launches) *launches += 9;
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
