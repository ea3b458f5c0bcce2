// K1: the fused pass over one micro-batch, for every registered query.
//
// Per event (paper: Filtering, Projection, Expand and Aggregation operators of
// Table II, fused into one pass): evaluate the query's filter, map ts to its
// pane (window slice of length `slide`; a sliding window of size K*slide is K
// consecutive panes, so the Expand step costs nothing here), and add the
// event to the (pane, key) group.  Groups are pre-aggregated per CTA tile in a
// shared-memory open-addressing table (warp-aggregated with match_any first,
// so hot Zipf keys cost one shared atomic per warp), then the tile's groups
// are appended to the query's partial-group arrays in HBM.  The batch columns
// are read exactly once, with 16-byte vector loads, for all queries together.
#include <climits>

#include "lms_device.cuh"

namespace lms {
namespace {

constexpr int kK1Threads = 512;
constexpr int kK1Items = 4;                      // events per thread per tile
constexpr int kK1Tile = kK1Threads * kK1Items;   // 2048 events
constexpr int kK1HashBits = 12;                  // 4096 slots >= 2 * tile
constexpr int kK1Hash = 1 << kK1HashBits;
constexpr int kK1SlotsPerThread = kK1Hash / kK1Threads;
constexpr size_t kK1Smem = (size_t)kK1Hash * (8 + 8 + 4 + 4 + 4);

template <bool FLOAT>
__device__ __forceinline__ void smem_upsert(unsigned long long* hkey, unsigned* hcnt,
                                            unsigned long long* hsum, unsigned* hmn,
                                            unsigned* hmx, unsigned long long g, unsigned c,
                                            unsigned long long sbits, unsigned mn, unsigned mx,
                                            unsigned agg_mask, unsigned* s_err) {
  unsigned slot = hash_slot(g, kK1HashBits);
  int probes = 0;
  while (true) {
    unsigned long long cur = *((volatile unsigned long long*)&hkey[slot]);
    if (cur == g) break;
    if (cur == kEmpty) {
      unsigned long long prev = atomicCAS(&hkey[slot], kEmpty, g);
      if (prev == kEmpty || prev == g) break;
    }
    slot = (slot + 1) & (kK1Hash - 1);
    if (++probes >= kK1Hash) {  // cannot happen: a tile has <= kK1Hash/2 groups
      atomicOr(s_err, kErrProbe);
      return;
    }
  }
  atomicAdd(&hcnt[slot], c);
  if (FLOAT)
    atomicAdd(reinterpret_cast<double*>(&hsum[slot]), __longlong_as_double((long long)sbits));
  else
    atomicAdd(&hsum[slot], sbits);
  if (agg_mask & 4u) atomicMin(&hmn[slot], mn);
  if (agg_mask & 8u) atomicMax(&hmx[slot], mx);
}

template <bool FLOAT, bool WARP_AGG>
__global__ void __launch_bounds__(kK1Threads, 1) k1_fused(const __grid_constant__ K1Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* hkey = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* hsum = hkey + kK1Hash;
  unsigned* hcnt = reinterpret_cast<unsigned*>(hsum + kK1Hash);
  unsigned* hmn = hcnt + kK1Hash;
  unsigned* hmx = hmn + kK1Hash;

  __shared__ unsigned long long s_tmp[33];
  __shared__ unsigned long long s_or[kMaxQueries], s_and[kMaxQueries];
  __shared__ unsigned long long s_late[kMaxQueries], s_range[kMaxQueries];
  __shared__ long long s_cursor[kMaxQueries];
  __shared__ unsigned long long s_base;
  __shared__ long long s_maxts;
  __shared__ unsigned s_err[kMaxQueries];

  const int tid = threadIdx.x;
  const unsigned lane = lane_id();
  for (int s = tid; s < kK1Hash; s += kK1Threads) {
    hkey[s] = kEmpty;
    hsum[s] = 0ull;
    hcnt[s] = 0u;
    hmn[s] = 0xffffffffu;
    hmx[s] = 0u;
  }
  if (tid < a.nq) {
    s_or[tid] = 0ull;
    s_and[tid] = ~0ull;
    s_late[tid] = 0ull;
    s_range[tid] = 0ull;
    s_cursor[tid] = a.q[tid].ctl->cursor;
    s_err[tid] = 0u;
  }
  if (tid == 0) s_maxts = LLONG_MIN;
  __syncthreads();

  const long long n = a.n;
  const long long ntiles = (n + kK1Tile - 1) / kK1Tile;
  const bool vec_ok =
      ((reinterpret_cast<uintptr_t>(a.ts) | reinterpret_cast<uintptr_t>(a.key) |
        reinterpret_cast<uintptr_t>(a.value)) & 15u) == 0 &&
      (a.type == nullptr || (reinterpret_cast<uintptr_t>(a.type) & 3u) == 0);
  long long tmax = LLONG_MIN;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- load this thread's events (blocked: 4 consecutive events) ----
    const long long e0 = tile * kK1Tile + (long long)tid * kK1Items;
    long long ts[kK1Items];
    unsigned key[kK1Items], val[kK1Items], typ[kK1Items];
    bool valid[kK1Items];
    if (vec_ok && e0 + kK1Items <= n) {
      const longlong2 t01 = __ldcs(reinterpret_cast<const longlong2*>(a.ts + e0));
      const longlong2 t23 = __ldcs(reinterpret_cast<const longlong2*>(a.ts + e0) + 1);
      const uint4 k4 = __ldcs(reinterpret_cast<const uint4*>(a.key + e0));
      const uint4 v4 = __ldcs(reinterpret_cast<const uint4*>(static_cast<const unsigned*>(a.value) + e0));
      ts[0] = t01.x; ts[1] = t01.y; ts[2] = t23.x; ts[3] = t23.y;
      key[0] = k4.x; key[1] = k4.y; key[2] = k4.z; key[3] = k4.w;
      val[0] = v4.x; val[1] = v4.y; val[2] = v4.z; val[3] = v4.w;
      unsigned t4 = a.type ? __ldcs(reinterpret_cast<const unsigned*>(a.type + e0)) : 0u;
#pragma unroll
      for (int i = 0; i < kK1Items; ++i) {
        typ[i] = (t4 >> (8 * i)) & 0xffu;
        valid[i] = true;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kK1Items; ++i) {
        const long long e = e0 + i;
        valid[i] = e < n;
        ts[i] = valid[i] ? a.ts[e] : 0;
        key[i] = valid[i] ? a.key[e] : 0u;
        val[i] = valid[i] ? static_cast<const unsigned*>(a.value)[e] : 0u;
        typ[i] = (valid[i] && a.type) ? a.type[e] : 0u;
      }
    }
#pragma unroll
    for (int i = 0; i < kK1Items; ++i)
      if (valid[i] && ts[i] > tmax) tmax = ts[i];

    for (int qi = 0; qi < a.nq; ++qi) {
      const QueryDev& Q = a.q[qi];
      const int fcol = Q.filter_col, fop = Q.filter_op;
      const unsigned amask = Q.agg_mask;
      const long long cursor = s_cursor[qi];
      unsigned n_late = 0, n_range = 0;
#pragma unroll
      for (int i = 0; i < kK1Items; ++i) {
        // ---- filter ----
        bool ok = valid[i];
        if (ok && fop != 0) {
          if (fcol == 2 && FLOAT)
            ok = filter_pass_f32(fop, __uint_as_float(val[i]), Q.filter_lo, Q.filter_hi,
                                 Q.filter_exact);
          else {
            long long x = fcol == 0 ? ts[i]
                          : fcol == 1 ? (long long)key[i]
                          : fcol == 3 ? (long long)typ[i]
                                      : (long long)(int)val[i];
            ok = filter_pass_i(fop, x, Q.filter_i);
          }
        }
        // ---- pane (window slice) id ----
        unsigned long long g = 0ull;
        if (ok) {
          const unsigned long long u = (unsigned long long)ts[i] + Q.ts_off;
          if (u >= Q.u_limit) {
            ++n_range;
            ok = false;
          } else {
            const unsigned long long prel = udiv_inv(u, Q.magic, Q.sh1, Q.sh2);
            if ((long long)prel < cursor) {  // every window of this event was emitted
              ++n_late;
              ok = false;
            } else {
              g = (prel << 32) | key[i];
            }
          }
        }
        const unsigned enc = FLOAT ? enc_f32(__uint_as_float(val[i])) : enc_i32((int)val[i]);
        // ---- aggregate into the tile's shared table ----
        if (WARP_AGG) {
          const unsigned act = __ballot_sync(kFull, ok);
          if (ok) {
            const unsigned peers = __match_any_sync(act, g);
            const unsigned c = __popc(peers);
            const unsigned mn = __reduce_min_sync(peers, enc);
            const unsigned mx = __reduce_max_sync(peers, enc);
            unsigned long long sbits;
            if (FLOAT) {
              double s = 0.0;
              const double v = (double)__uint_as_float(val[i]);
              for (unsigned m = peers; m; m &= m - 1)
                s += __shfl_sync(peers, v, __ffs(m) - 1);
              sbits = (unsigned long long)__double_as_longlong(s);
            } else {
              const int v = (int)val[i];
              const unsigned lo = __reduce_add_sync(peers, (unsigned)(v & 0xffff));
              const int hi = __reduce_add_sync(peers, v >> 16);
              sbits = (unsigned long long)((long long)hi * 65536ll + (long long)lo);
            }
            if ((int)lane == __ffs(peers) - 1)
              smem_upsert<FLOAT>(hkey, hcnt, hsum, hmn, hmx, g, c, sbits, mn, mx, amask,
                                 &s_err[qi]);
          }
        } else if (ok) {
          const unsigned long long sbits =
              FLOAT ? (unsigned long long)__double_as_longlong((double)__uint_as_float(val[i]))
                    : (unsigned long long)(long long)(int)val[i];
          smem_upsert<FLOAT>(hkey, hcnt, hsum, hmn, hmx, g, 1u, sbits, enc, enc, amask,
                             &s_err[qi]);
        }
      }
      // per-warp drop counters
      n_late = __reduce_add_sync(kFull, n_late);
      n_range = __reduce_add_sync(kFull, n_range);
      if (lane == 0 && (n_late | n_range)) {
        atomicAdd(&s_late[qi], (unsigned long long)n_late);
        atomicAdd(&s_range[qi], (unsigned long long)n_range);
      }
      __syncthreads();

      // ---- flush the tile's groups to the partial arrays ----
      const int s0 = tid * kK1SlotsPerThread;
      unsigned occ = 0;
#pragma unroll
      for (int j = 0; j < kK1SlotsPerThread; ++j)
        if (hkey[s0 + j] != kEmpty) occ |= 1u << j;
      unsigned long long total;
      const unsigned long long off = block_excl_scan((unsigned long long)__popc(occ), s_tmp, &total);
      if (tid == 0) s_base = total ? atomicAdd(&Q.ctl->n_parts, total) : 0ull;
      __syncthreads();
      const unsigned long long base = s_base;
      const bool fits = base + total <= Q.parts_cap;
      if (tid == 0 && !fits) atomicOr(&s_err[qi], kErrPartsOverflow);
      unsigned long long o_acc = 0ull, a_acc = ~0ull;
      unsigned long long w = base + off;
#pragma unroll
      for (int j = 0; j < kK1SlotsPerThread; ++j) {
        const int s = s0 + j;
        if (occ & (1u << j)) {
          if (fits) {
            const unsigned long long g = hkey[s];
            store_grp(Q.parts + w, g, (long long)hcnt[s], hsum[s], hmn[s], hmx[s]);
            Q.pkeys[w] = g;
            o_acc |= g;
            a_acc &= g;
          }
          ++w;
          hkey[s] = kEmpty;
          hsum[s] = 0ull;
          hcnt[s] = 0u;
          hmn[s] = 0xffffffffu;
          hmx[s] = 0u;
        }
      }
      const unsigned olo = __reduce_or_sync(kFull, (unsigned)o_acc);
      const unsigned ohi = __reduce_or_sync(kFull, (unsigned)(o_acc >> 32));
      const unsigned alo = __reduce_and_sync(kFull, (unsigned)a_acc);
      const unsigned ahi = __reduce_and_sync(kFull, (unsigned)(a_acc >> 32));
      if (lane == 0) {
        atomicOr(&s_or[qi], ((unsigned long long)ohi << 32) | olo);
        atomicAnd(&s_and[qi], ((unsigned long long)ahi << 32) | alo);
      }
      __syncthreads();
    }
  }

  // ---- per-CTA results: batch max ts, masks, counters ----
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long other = __shfl_xor_sync(kFull, tmax, o);
    tmax = other > tmax ? other : tmax;
  }
  if (lane == 0 && tmax != LLONG_MIN) atomicMax(&s_maxts, tmax);
  __syncthreads();
  if (tid == 0 && s_maxts != LLONG_MIN) atomicMax(&a.sctl->batch_max_ts, s_maxts);
  if (tid < a.nq) {
    QCtl* c = a.q[tid].ctl;
    if (s_or[tid]) atomicOr(&c->or_mask, s_or[tid]);
    if (s_and[tid] != ~0ull) atomicAnd(&c->and_mask, s_and[tid]);
    if (s_late[tid]) atomicAdd(&c->late_rows, s_late[tid]);
    if (s_range[tid]) atomicAdd(&c->range_rows, s_range[tid]);
    if (s_err[tid]) atomicOr(&c->err, s_err[tid]);
  }
}

template <bool FLOAT, bool WARP_AGG>
cudaError_t launch_k1_t(const K1Args& a, int grid, cudaStream_t st) {
  static bool attr_set = false;  // per instantiation; set once per process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k1_fused<FLOAT, WARP_AGG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kK1Smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k1_fused<FLOAT, WARP_AGG><<<grid, kK1Threads, kK1Smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_k1(const K1Args& a, int variant, int grid, cudaStream_t st) {
  const bool wagg = variant == 2;  // measured slower on the Zipf workload; opt-in
  if (a.value_is_float)
    return wagg ? launch_k1_t<true, true>(a, grid, st) : launch_k1_t<true, false>(a, grid, st);
  return wagg ? launch_k1_t<false, true>(a, grid, st) : launch_k1_t<false, false>(a, grid, st);
}

int k1_tile_events() { return kK1Tile; }

int k1_max_grid(int device, int variant, int value_is_float) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  (void)variant;
  (void)value_is_float;
  return sms > 0 ? sms : 148;  // one resident CTA per SM (112 KB shared table)
}

}  // namespace lms
