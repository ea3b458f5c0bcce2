// K1: the fused pass over one micro-batch, for every registered query.
//
// Per event (paper: Filtering, Projection, Expand and Aggregation operators of
// Table II, fused into one pass): evaluate the query's filter, map ts to its
// pane (window slice of length `slide`; a sliding window of size K*slide is K
// consecutive panes, so the Expand step costs nothing here), and add the
// event to the (pane, key) group.  The batch columns are read exactly once,
// with vector loads, for all queries together.
//
// Per tile of 1024 events and per query, the groups are built in shared
// memory without any floating-point atomics:
//   A. every surviving event inserts its group key into an open-addressing
//      table (integer CAS on the key only); a new key is appended to the
//      tile's group list;
//   B. each event takes a rank inside its group (warp-aggregated atomic add
//      on the group's counter);
//   C. a scan of the group counters gives every group a contiguous range and
//      the events scatter their values into it;
//   D. each group is reduced (count, sum, min, max) — one thread per small
//      group, one warp per large one — and appended to the query's
//      partial-group array in HBM.  Float32 values are summed on the integer
//      pipe: every value is aligned to the group's largest exponent B as a
//      64-bit fixed-point number whose unit is 2^(B-178) (the largest value
//      occupies bits 28..51, so 2048 of them could not overflow), then the sum is
//      converted to double once.  The error is at most 2^-41 of the group's
//      largest |value| (FP64 is slow on this part; groups holding Inf or NaN
//      are summed in FP64 instead).
#include <climits>

#include "lms_device.cuh"

namespace lms {
namespace {

constexpr int kK1Threads = 512;                  // two CTAs per SM
constexpr int kK1Warps = kK1Threads / 32;
constexpr int kK1Items = 2;                      // events per thread per tile
constexpr int kK1Tile = kK1Threads * kK1Items;   // 1024 events
constexpr int kK1HashBits = 11;                  // 2048 slots >= 2 * tile
constexpr int kK1Hash = 1 << kK1HashBits;
constexpr unsigned kBigGroup = 32;               // groups above this are reduced by a warp
constexpr unsigned kNoSlot = 0xffffu;

// hkey u64[H] | hidx u16[H] | list u16[T] | lcnt u32[T] | loff u32[T+4] | vals u32[T]
constexpr size_t kK1Smem = (size_t)kK1Hash * 8 + kK1Hash * 2 + kK1Tile * 2 + kK1Tile * 4 +
                           (kK1Tile + 4) * 4 + kK1Tile * 4;

// Phase A: the slot of group key g (inserted if new).  Returns the slot, or
// kNoSlot if the probe bound is hit (cannot happen: a tile has <= H/2 groups).
__device__ __forceinline__ unsigned insert_key(unsigned long long* hkey, unsigned short* hidx,
                                               unsigned short* list, unsigned* nlist,
                                               unsigned long long g) {
  unsigned slot = hash_slot(g, kK1HashBits);
  for (int probes = 0; probes < kK1Hash; ++probes) {
    const unsigned long long cur = *((volatile unsigned long long*)&hkey[slot]);
    if (cur == g) return slot;
    if (cur == kEmpty) {
      const unsigned long long prev = atomicCAS(&hkey[slot], kEmpty, g);
      if (prev == kEmpty) {
        const unsigned li = atomicAdd(nlist, 1u);
        list[li] = (unsigned short)slot;
        hidx[slot] = (unsigned short)li;
        return slot;
      }
      if (prev == g) return slot;
    }
    slot = (slot + 1) & (kK1Hash - 1);
  }
  return kNoSlot;
}

// Biased exponent used for alignment (denormals count as exponent 1) and the
// 24-bit significand of a float32 given by its bits.
__device__ __forceinline__ unsigned f32_exp(unsigned x) {
  const unsigned be = (x >> 23) & 0xffu;
  return be ? be : 1u;
}
__device__ __forceinline__ long long f32_fixed(unsigned x, unsigned B) {
  const unsigned be = (x >> 23) & 0xffu;
  const long long m = be ? (long long)((x & 0x7fffffu) | 0x800000u) : (long long)(x & 0x7fffffu);
  const int sh = (int)(be ? be : 1u) - (int)B + 28;  // <= 28
  long long t;
  if (sh >= 0) t = m << sh;
  else if (sh > -40) t = (m + (1ll << (-sh - 1))) >> (-sh);  // round half up
  else t = 0;
  return (x & 0x80000000u) ? -t : t;
}
// double value of a fixed-point sum with unit 2^(B - 178)
__device__ __forceinline__ double fixed_to_double(long long t, unsigned B) {
  return (double)t * __longlong_as_double((long long)(1023 + (int)B - 178) << 52);
}

// Count of values, sum (int64, or double bits) and encoded min/max of
// v[b], v[b + step], ... below e.  With step = 32 every lane of a warp calls it
// and the caller combines the lanes with warp reductions.
template <bool FLOAT>
__device__ __forceinline__ void reduce_values(const unsigned* v, unsigned b, unsigned e,
                                              unsigned step, unsigned* bmax, long long* fixed,
                                              double* fsum, unsigned* mn, unsigned* mx) {
  unsigned lo = 0xffffffffu, hi = 0u, B = 1u;
  for (unsigned t = b; t < e; t += step) {
    const unsigned x = v[t];
    const unsigned enc = FLOAT ? enc_f32(__uint_as_float(x)) : enc_i32((int)x);
    lo = min(lo, enc);
    hi = max(hi, enc);
    if (FLOAT) B = max(B, f32_exp(x));
  }
  *mn = lo;
  *mx = hi;
  *bmax = B;
  *fsum = 0.0;
  long long acc = 0;
  if (!FLOAT) {
    for (unsigned t = b; t < e; t += step) acc += (long long)(int)v[t];
  }
  *fixed = acc;
}

template <bool FLOAT>
__device__ __forceinline__ long long fixed_sum(const unsigned* v, unsigned b, unsigned e,
                                               unsigned step, unsigned B, double* fsum) {
  long long acc = 0;
  if (B == 255u) {  // Inf or NaN present: plain FP64 sum
    double d = 0.0;
    for (unsigned t = b; t < e; t += step) d += (double)__uint_as_float(v[t]);
    *fsum = d;
    return 0;
  }
  for (unsigned t = b; t < e; t += step) acc += f32_fixed(v[t], B);
  return acc;
}

template <bool FLOAT>
__global__ void __launch_bounds__(kK1Threads, 2) k1_fused(const __grid_constant__ K1Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* hkey = reinterpret_cast<unsigned long long*>(smem);
  unsigned short* hidx = reinterpret_cast<unsigned short*>(hkey + kK1Hash);
  unsigned short* list = hidx + kK1Hash;
  unsigned* lcnt = reinterpret_cast<unsigned*>(list + kK1Tile);
  unsigned* loff = lcnt + kK1Tile;
  unsigned* vals = loff + kK1Tile + 4;

  __shared__ unsigned long long s_or[kMaxQueries], s_and[kMaxQueries];
  __shared__ unsigned long long s_late[kMaxQueries], s_range[kMaxQueries];
  __shared__ long long s_cursor[kMaxQueries];
  __shared__ unsigned long long s_base;
  __shared__ long long s_maxts;
  __shared__ unsigned s_err[kMaxQueries];
  __shared__ unsigned s_nlist, s_nbig;
  __shared__ unsigned s_wsum[kK1Warps + 1];
  __shared__ unsigned short s_big[kK1Tile];

  const int tid = threadIdx.x;
  const unsigned lane = lane_id();
  const int warp = tid >> 5;
  for (int s = tid; s < kK1Hash; s += kK1Threads) hkey[s] = kEmpty;
  for (int s = tid; s < kK1Tile; s += kK1Threads) lcnt[s] = 0u;
  if (tid < a.nq) {
    s_or[tid] = 0ull;
    s_and[tid] = ~0ull;
    s_late[tid] = 0ull;
    s_range[tid] = 0ull;
    s_cursor[tid] = a.q[tid].ctl->cursor;
    s_err[tid] = 0u;
  }
  if (tid == 0) {
    s_maxts = LLONG_MIN;
    s_nlist = 0u;
    s_nbig = 0u;
  }
  __syncthreads();

  const long long n = a.n;
  const long long ntiles = (n + kK1Tile - 1) / kK1Tile;
  const bool vec_ok =
      ((reinterpret_cast<uintptr_t>(a.ts) | reinterpret_cast<uintptr_t>(a.key) |
        reinterpret_cast<uintptr_t>(a.value)) & 15u) == 0 &&
      (a.type == nullptr || (reinterpret_cast<uintptr_t>(a.type) & 1u) == 0);
  long long tmax = LLONG_MIN;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // ---- load this thread's 2 consecutive events (16/8/8/2-byte loads) ----
    const long long e0 = tile * kK1Tile + (long long)tid * kK1Items;
    long long ts[kK1Items];
    unsigned key[kK1Items], val[kK1Items], typ[kK1Items];
    bool valid[kK1Items];
    if (vec_ok && e0 + kK1Items <= n) {
      const longlong2 t01 = __ldcs(reinterpret_cast<const longlong2*>(a.ts + e0));
      const uint2 k2 = __ldcs(reinterpret_cast<const uint2*>(a.key + e0));
      const uint2 v2 =
          __ldcs(reinterpret_cast<const uint2*>(static_cast<const unsigned*>(a.value) + e0));
      ts[0] = t01.x; ts[1] = t01.y;
      key[0] = k2.x; key[1] = k2.y;
      val[0] = v2.x; val[1] = v2.y;
      const unsigned t2 =
          a.type ? (unsigned)__ldcs(reinterpret_cast<const unsigned short*>(a.type + e0)) : 0u;
#pragma unroll
      for (int i = 0; i < kK1Items; ++i) {
        typ[i] = (t2 >> (8 * i)) & 0xffu;
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
      const long long cursor = s_cursor[qi];
      unsigned n_late = 0, n_range = 0;
      unsigned slot[kK1Items];
      // ---- A: filter, pane id, insert the group key ----
#pragma unroll
      for (int i = 0; i < kK1Items; ++i) {
        bool ok = valid[i];
        if (ok && fop != 0) {
          if (fcol == 2 && FLOAT) {
            ok = filter_pass_f32(fop, __uint_as_float(val[i]), Q.filter_lo, Q.filter_hi,
                                 Q.filter_exact);
          } else {
            const long long x = fcol == 0 ? ts[i]
                                : fcol == 1 ? (long long)key[i]
                                : fcol == 3 ? (long long)typ[i]
                                            : (long long)(int)val[i];
            ok = filter_pass_i(fop, x, Q.filter_i);
          }
        }
        slot[i] = kNoSlot;
        if (ok) {
          const unsigned long long u = (unsigned long long)ts[i] + Q.ts_off;
          if (u >= Q.u_limit) {
            ++n_range;
          } else {
            const unsigned long long prel = udiv_inv(u, Q.magic, Q.sh1, Q.sh2);
            if ((long long)prel < cursor) {  // every window of this event was emitted
              ++n_late;
            } else {
              slot[i] = insert_key(hkey, hidx, list, &s_nlist, (prel << 32) | key[i]);
              if (slot[i] == kNoSlot) atomicOr(&s_err[qi], kErrProbe);
            }
          }
        }
      }
      n_late = __reduce_add_sync(kFull, n_late);
      n_range = __reduce_add_sync(kFull, n_range);
      if (lane == 0 && (n_late | n_range)) {
        atomicAdd(&s_late[qi], (unsigned long long)n_late);
        atomicAdd(&s_range[qi], (unsigned long long)n_range);
      }
      __syncthreads();
      // ---- B: rank inside the group (one atomic per group and warp) ----
      unsigned rank[kK1Items], gi[kK1Items];
#pragma unroll
      for (int i = 0; i < kK1Items; ++i) {
        const bool has = slot[i] != kNoSlot;
        gi[i] = has ? (unsigned)hidx[slot[i]] : 0xffffffffu;
        const unsigned act = __ballot_sync(kFull, has);
        rank[i] = 0;
        if (has) {
          const unsigned peers = __match_any_sync(act, gi[i]);
          const int leader = __ffs(peers) - 1;
          unsigned base = 0;
          if ((int)lane == leader) base = atomicAdd(&lcnt[gi[i]], (unsigned)__popc(peers));
          base = __shfl_sync(peers, base, leader);
          rank[i] = base + __popc(peers & ((1u << lane) - 1u));
        }
      }
      __syncthreads();
      // ---- C: group ranges (scan of the counters in list order), scatter ----
      const unsigned nl = s_nlist;
      {
        const unsigned i0 = 2u * tid;
        const unsigned c0 = i0 < nl ? lcnt[i0] : 0u;
        const unsigned c1 = i0 + 1 < nl ? lcnt[i0 + 1] : 0u;
        const unsigned x = c0 + c1;
        unsigned inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned y = __shfl_up_sync(kFull, inc, o);
          if ((int)lane >= o) inc += y;
        }
        if (lane == 31) s_wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
          const unsigned w = lane < kK1Warps ? s_wsum[lane] : 0u;
          unsigned wi = w;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, wi, o);
            if ((int)lane >= o) wi += y;
          }
          if (lane < kK1Warps) s_wsum[lane] = wi - w;
          if (lane == kK1Warps - 1) s_wsum[kK1Warps] = wi;
        }
        __syncthreads();
        const unsigned ex = s_wsum[warp] + inc - x;
        if (i0 < nl) loff[i0] = ex;
        if (i0 + 1 < nl) loff[i0 + 1] = ex + c0;
        if (tid == 0) loff[nl] = s_wsum[kK1Warps];
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kK1Items; ++i)
        if (slot[i] != kNoSlot) vals[loff[gi[i]] + rank[i]] = val[i];
      if (tid == 0) s_base = nl ? atomicAdd(&Q.ctl->n_parts, (unsigned long long)nl) : 0ull;
      __syncthreads();
      // ---- D: reduce every group and append it to the partial arrays ----
      const unsigned long long base = s_base;
      const bool fits = base + nl <= Q.parts_cap;
      if (tid == 0 && !fits) atomicOr(&s_err[qi], kErrPartsOverflow);
      unsigned long long o_acc = 0ull, a_acc = ~0ull;
      for (unsigned i = tid; i < nl; i += kK1Threads) {
        const unsigned b = loff[i], e = loff[i + 1];
        if (e - b > kBigGroup) {
          s_big[atomicAdd(&s_nbig, 1u)] = (unsigned short)i;
          continue;
        }
        const unsigned long long g = hkey[list[i]];
        unsigned B, mn, mx;
        long long acc;
        double fs;
        reduce_values<FLOAT>(vals, b, e, 1u, &B, &acc, &fs, &mn, &mx);
        unsigned long long sb = (unsigned long long)acc;
        if (FLOAT) {
          acc = fixed_sum<FLOAT>(vals, b, e, 1u, B, &fs);
          sb = (unsigned long long)__double_as_longlong(B == 255u ? fs : fixed_to_double(acc, B));
        }
        if (fits) {
          store_grp(Q.parts + base + i, g, (long long)(e - b), sb, mn, mx);
          Q.pkeys[base + i] = g;
        }
        o_acc |= g;
        a_acc &= g;
      }
      __syncthreads();
      const unsigned nbig = s_nbig;
      for (unsigned bi = warp; bi < nbig; bi += kK1Warps) {
        const unsigned i = s_big[bi];
        const unsigned b = loff[i], e = loff[i + 1];
        unsigned B, mn, mx;
        long long acc;
        double fs;
        reduce_values<FLOAT>(vals, b + lane, e, 32u, &B, &acc, &fs, &mn, &mx);
        mn = __reduce_min_sync(kFull, mn);
        mx = __reduce_max_sync(kFull, mx);
        unsigned long long sb;
        if (FLOAT) {
          B = __reduce_max_sync(kFull, B);
          acc = fixed_sum<FLOAT>(vals, b + lane, e, 32u, B, &fs);
          if (B == 255u) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) fs += __shfl_xor_sync(kFull, fs, o);
            sb = (unsigned long long)__double_as_longlong(fs);
          } else {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
            sb = (unsigned long long)__double_as_longlong(fixed_to_double(acc, B));
          }
        } else {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
          sb = (unsigned long long)acc;
        }
        if (lane == 0) {
          const unsigned long long g = hkey[list[i]];
          if (fits) {
            store_grp(Q.parts + base + i, g, (long long)(e - b), sb, mn, mx);
            Q.pkeys[base + i] = g;
          }
          o_acc |= g;
          a_acc &= g;
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
      // ---- reset the table for the next tile / query ----
      for (unsigned i = tid; i < nl; i += kK1Threads) {
        hkey[list[i]] = kEmpty;
        lcnt[i] = 0u;
      }
      if (tid == 0) {
        s_nlist = 0u;
        s_nbig = 0u;
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

template <bool FLOAT>
cudaError_t launch_k1_t(const K1Args& a, int grid, cudaStream_t st) {
  // once per process and instantiation (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(
      k1_fused<FLOAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kK1Smem);
  if (attr != cudaSuccess) return attr;
  k1_fused<FLOAT><<<grid, kK1Threads, kK1Smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_k1(const K1Args& a, int variant, int grid, cudaStream_t st) {
  (void)variant;  // a single variant; the config field is kept for ABI stability
  return a.value_is_float ? launch_k1_t<true>(a, grid, st) : launch_k1_t<false>(a, grid, st);
}

int k1_tile_events() { return kK1Tile; }

int k1_max_grid(int device, int variant, int value_is_float) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  (void)variant;
  (void)value_is_float;
  return 2 * (sms > 0 ? sms : 148);  // two resident CTAs per SM
}

}  // namespace lms
