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
// memory with integer atomics only:
//   A. every surviving event inserts its group key into an open-addressing
//      table (CAS on the key; a new key is appended to the tile's group list)
//      and updates the group's min and max (order-preserving u32 codes) and
//      its count (for int32 values, count and sum share one 64-bit word);
//   B. (float32 values) every event adds its value to the group's sum as a
//      64-bit fixed-point number whose unit is 2^(B-178), B the largest
//      exponent in the group (that of its min or its max; the largest value
//      occupies bits 28..51, so 2^11 of them cannot overflow int64): integer adds,
//      so the sum is exact and independent of the order; it is converted to
//      double once.  The error is at most 2^-41 of the group's largest
//      |value| (FP64 is slow on this part; a group holding Inf or NaN is
//      summed in FP64 instead).  Int32 values are summed exactly in A;
//   C. each group of the list is appended to the query's partial-group array
//      in HBM and its slot is cleared for the next tile.
#include <climits>

#include "lms_device.cuh"

namespace lms {
namespace {

// Two tile shapes (the autotuner in the engine picks one per batch-size
// class): ITEMS events per thread, 512 threads, a table of 4 * ITEMS * 512
// slots (load factor <= 1/2).  ITEMS = 2: 1024-event tiles, two CTAs per SM;
// ITEMS = 4: 2048-event tiles (fewer partial groups), one CTA per SM.
constexpr int kK1Threads = 512;
constexpr unsigned kNoSlot = 0xffffffffu;
template <int ITEMS> struct K1Shape {
  static constexpr int kTile = kK1Threads * ITEMS;
  static constexpr int kHashBits = ITEMS == 2 ? 11 : 12;
  static constexpr int kHash = 1 << kHashBits;
  // hkey u64[H] | gsum u64[H] | gcnt u32[H] | gmn u32[H] | gmx u32[H] | list u16[T]
  static constexpr size_t kSmem = (size_t)kHash * (8 + 8 + 4 + 4 + 4) + kTile * 2;
  static constexpr int kCtasPerSm = ITEMS == 2 ? 2 : 1;
};

// Int32 values: count and sum share one 64-bit word: each event adds
// 2^43 + (value + 2^31), so count = word >> 43 and sum = low 43 bits - count * 2^31
// (at most 2048 events of at most 2^32 each: the low part stays below 2^43).
constexpr int kCntShift = 43;

// Phase A: the slot of group key g (inserted if new; *created tells whether
// this call inserted it).  Returns the slot, or kNoSlot if the probe bound is
// hit (cannot happen: a tile has <= H/2 groups).
template <int BITS>
__device__ __forceinline__ unsigned insert_key(unsigned long long* hkey, unsigned long long g,
                                               bool* created) {
  constexpr int H = 1 << BITS;
  unsigned slot = hash_slot(g, BITS);
  for (int probes = 0; probes < H; ++probes) {
    const unsigned long long cur = *((volatile unsigned long long*)&hkey[slot]);
    if (cur == g) return slot;
    if (cur == kEmpty) {
      const unsigned long long prev = atomicCAS(&hkey[slot], kEmpty, g);
      if (prev == kEmpty) {
        *created = true;
        return slot;
      }
      if (prev == g) return slot;
    }
    slot = (slot + 1) & (H - 1);
  }
  return kNoSlot;
}

// The tile's list of new groups: the lanes of a warp that inserted a key in
// this step reserve their entries with one atomic (instead of one each: every
// new group of a tile would otherwise meet on the same counter).  Called by
// every lane of the warp.
__device__ __forceinline__ void append_new(unsigned short* list, unsigned* nlist, bool created,
                                           unsigned slot, unsigned lane) {
  const unsigned cm = __ballot_sync(kFull, created);
  if (!cm) return;
  const int leader = __ffs(cm) - 1;
  unsigned base = 0u;
  if ((int)lane == leader) base = atomicAdd(nlist, (unsigned)__popc(cm));
  base = __shfl_sync(kFull, base, leader);
  if (created) list[base + __popc(cm & ((1u << lane) - 1u))] = (unsigned short)slot;
}

// Biased exponent used for alignment (denormals count as exponent 1).
__device__ __forceinline__ unsigned f32_exp(unsigned x) {
  const unsigned be = (x >> 23) & 0xffu;
  return be ? be : 1u;
}
// Largest exponent among a group's values, from its min and max codes: the
// value of largest magnitude is the group's min or its max.
__device__ __forceinline__ unsigned group_exp(unsigned mn_code, unsigned mx_code) {
  return max(f32_exp(dec_f32_bits(mn_code)), f32_exp(dec_f32_bits(mx_code)));
}
// x as a fixed-point number with unit 2^(B - 178) (B >= exponent of x).
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
// Bits of the double nearest (ties to even) to the fixed-point sum t with unit
// 2^(B - 178), built with integer operations (FP64 is slow on this part):
// normalise |t|, keep 52 fraction bits, round on the 11 dropped ones.  For
// 1 <= B <= 254 and |t| < 2^63 the result is always a normal double.
__device__ __forceinline__ unsigned long long fixed_to_double_bits(long long t, unsigned B) {
  if (t == 0) return 0ull;
  const unsigned long long sgn = t < 0 ? (1ull << 63) : 0ull;
  unsigned long long m = t < 0 ? (unsigned long long)(-t) : (unsigned long long)t;
  const int lz = __clzll((long long)m);
  m <<= lz;  // leading one at bit 63
  const unsigned long long e = (unsigned long long)(63 - lz + (int)B - 178 + 1023);
  const unsigned long long frac = (m >> 11) & ((1ull << 52) - 1ull);
  const unsigned long long rest = m & 0x7ffull;
  unsigned long long bits = (e << 52) | frac;
  if (rest > 0x400ull || (rest == 0x400ull && (frac & 1ull))) bits += 1ull;  // carries into e
  return sgn | bits;
}
// Adds a 64-bit two's-complement value to a shared 64-bit word with 32-bit
// atomics (faster than the 64-bit one here): the low word's old value tells
// whether the add carried into the high word.
__device__ __forceinline__ void shared_add_u64_split(unsigned long long* p, unsigned long long x) {
  unsigned* w = reinterpret_cast<unsigned*>(p);
  const unsigned lo = (unsigned)x;
  const unsigned old = atomicAdd(&w[0], lo);
  const unsigned hi = (unsigned)(x >> 32) + ((old + lo) < old ? 1u : 0u);
  if (hi) atomicAdd(&w[1], hi);
}
// FP64 add into a shared-memory word (groups holding Inf or NaN only)
__device__ __forceinline__ void shared_add_f64(unsigned long long* p, double v) {
  unsigned long long old = *p, assumed;
  do {
    assumed = old;
    old = atomicCAS(p, assumed,
                    (unsigned long long)__double_as_longlong(__longlong_as_double((long long)assumed) + v));
  } while (old != assumed);
}

template <bool FLOAT, int ITEMS, bool WAGG>
__global__ void __launch_bounds__(kK1Threads, K1Shape<ITEMS>::kCtasPerSm)
    k1_fused(const __grid_constant__ K1Args a) {
  constexpr int kK1Items = ITEMS;
  constexpr int kK1Tile = K1Shape<ITEMS>::kTile;
  constexpr int kK1HashBits = K1Shape<ITEMS>::kHashBits;
  constexpr int kK1Hash = K1Shape<ITEMS>::kHash;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* hkey = reinterpret_cast<unsigned long long*>(smem);
  unsigned long long* gsum = hkey + kK1Hash;
  unsigned* gcnt = reinterpret_cast<unsigned*>(gsum + kK1Hash);
  unsigned* gmn = gcnt + kK1Hash;
  unsigned* gmx = gmn + kK1Hash;
  unsigned short* list = reinterpret_cast<unsigned short*>(gmx + kK1Hash);

  __shared__ unsigned long long s_or[kMaxQueries], s_and[kMaxQueries];
  __shared__ unsigned long long s_late[kMaxQueries], s_range[kMaxQueries];
  __shared__ long long s_cursor[kMaxQueries];
  __shared__ unsigned long long s_base;
  __shared__ long long s_maxts;
  __shared__ unsigned s_err[kMaxQueries];
  __shared__ unsigned s_nlist;

  const int tid = threadIdx.x;
  const unsigned lane = lane_id();
  for (int s = tid; s < kK1Hash; s += kK1Threads) {
    hkey[s] = kEmpty;
    gsum[s] = 0ull;
    gcnt[s] = 0u;
    gmn[s] = 0xffffffffu;
    gmx[s] = 0u;
  }
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
  }
  __syncthreads();

  const long long n = a.n;
  const long long ntiles = (n + kK1Tile - 1) / kK1Tile;
  const bool vec_ok =
      ((reinterpret_cast<uintptr_t>(a.ts) | reinterpret_cast<uintptr_t>(a.key) |
        reinterpret_cast<uintptr_t>(a.value)) & 15u) == 0 &&
      (a.type == nullptr || (reinterpret_cast<uintptr_t>(a.type) & 1u) == 0);
  long long tmax = LLONG_MIN;

  // columns of this thread's kK1Items consecutive events of a tile (vector
  // loads when aligned); the next tile's are loaded while this one is processed
  auto load_tile = [&](long long tile, long long* ts, unsigned* key, unsigned* val, unsigned* typ,
                       bool* valid) {
    const long long e0 = tile * kK1Tile + (long long)tid * kK1Items;
    if (tile >= ntiles) {
#pragma unroll
      for (int i = 0; i < kK1Items; ++i) valid[i] = false;
      return;
    }
    if (vec_ok && e0 + kK1Items <= n) {
#pragma unroll
      for (int h = 0; h < kK1Items; h += 2) {
        const longlong2 t01 = __ldcs(reinterpret_cast<const longlong2*>(a.ts + e0 + h));
        ts[h] = t01.x;
        ts[h + 1] = t01.y;
      }
      unsigned t4 = 0u;
      if (kK1Items == 2) {
        const uint2 k2 = __ldcs(reinterpret_cast<const uint2*>(a.key + e0));
        const uint2 v2 =
            __ldcs(reinterpret_cast<const uint2*>(static_cast<const unsigned*>(a.value) + e0));
        key[0] = k2.x; key[1] = k2.y;
        val[0] = v2.x; val[1] = v2.y;
        if (a.type) t4 = (unsigned)__ldcs(reinterpret_cast<const unsigned short*>(a.type + e0));
      } else {
#pragma unroll
        for (int h = 0; h < kK1Items; h += 4) {
          const uint4 k4 = __ldcs(reinterpret_cast<const uint4*>(a.key + e0 + h));
          const uint4 v4 = __ldcs(
              reinterpret_cast<const uint4*>(static_cast<const unsigned*>(a.value) + e0 + h));
          key[h] = k4.x; key[h + 1] = k4.y; key[h + 2] = k4.z; key[h + 3] = k4.w;
          val[h] = v4.x; val[h + 1] = v4.y; val[h + 2] = v4.z; val[h + 3] = v4.w;
        }
        if (a.type) t4 = __ldcs(reinterpret_cast<const unsigned*>(a.type + e0));
      }
#pragma unroll
      for (int i = 0; i < kK1Items; ++i) {
        typ[i] = (t4 >> (8 * (i & 3))) & 0xffu;
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
  };
  long long nts[kK1Items];
  unsigned nkey[kK1Items], nval[kK1Items], ntyp[kK1Items];
  bool nvalid[kK1Items];
  load_tile(blockIdx.x, nts, nkey, nval, ntyp, nvalid);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    long long ts[kK1Items];
    unsigned key[kK1Items], val[kK1Items], typ[kK1Items];
    bool valid[kK1Items];
#pragma unroll
    for (int i = 0; i < kK1Items; ++i) {
      ts[i] = nts[i];
      key[i] = nkey[i];
      val[i] = nval[i];
      typ[i] = ntyp[i];
      valid[i] = nvalid[i];
    }
    load_tile(tile + gridDim.x, nts, nkey, nval, ntyp, nvalid);
#pragma unroll
    for (int i = 0; i < kK1Items; ++i)
      if (valid[i] && ts[i] > tmax) tmax = ts[i];

    for (int qi = 0; qi < a.nq; ++qi) {
      const QueryDev& Q = a.q[qi];
      const int fcol = Q.filter_col, fop = Q.filter_op;
      const long long cursor = s_cursor[qi];
      unsigned n_late = 0, n_range = 0;
      unsigned slot[kK1Items], peer[kK1Items];
      // ---- A: filter, pane id, insert the group key, count / min / max / exponent ----
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
        unsigned long long g = kEmpty;  // the event's group key, if it is aggregated
        if (ok) {
          const unsigned long long u = (unsigned long long)ts[i] + Q.ts_off;
          if (u >= Q.u_limit) {
            ++n_range;
          } else {
            const unsigned long long prel = udiv_inv(u, Q.magic, Q.sh1, Q.sh2);
            if ((long long)prel < cursor) ++n_late;  // every window of this event was emitted
            else g = make_gkey(prel, key[i] & Q.key_mask, Q.lb);
          }
        }
        const unsigned enc = FLOAT ? enc_f32(__uint_as_float(val[i])) : enc_i32((int)val[i]);
        if (WAGG) {
          // lanes of the warp with the same group key update it once, through
          // a leader: count, min, max (and the int sum) reduced over the peers
          const unsigned peers = __match_any_sync(kFull, g);
          peer[i] = peers;
          const int leader = __ffs(peers) - 1;
          const unsigned mn = __reduce_min_sync(peers, enc);
          const unsigned mx = __reduce_max_sync(peers, enc);
          unsigned long long add = 0ull;
          if (!FLOAT) {
            const unsigned lo = __reduce_add_sync(peers, enc & 0xffffu);
            const unsigned hi = __reduce_add_sync(peers, enc >> 16);
            add = ((unsigned long long)__popc(peers) << kCntShift) + lo + ((unsigned long long)hi << 16);
          }
          unsigned sl = kNoSlot;
          bool created = false;
          if (g != kEmpty && (int)lane == leader) {
            sl = insert_key<kK1HashBits>(hkey, g, &created);
            if (sl == kNoSlot) {
              atomicOr(&s_err[qi], kErrProbe);
            } else {
              atomicMin(&gmn[sl], mn);
              atomicMax(&gmx[sl], mx);
              if (FLOAT) atomicAdd(&gcnt[sl], (unsigned)__popc(peers));
              else atomicAdd(&gsum[sl], add);
            }
          }
          append_new(list, &s_nlist, created, sl, lane);
          sl = __shfl_sync(peers, sl, leader);
          slot[i] = g != kEmpty ? sl : kNoSlot;
        } else {
          bool created = false;
          const unsigned sl = g != kEmpty ? insert_key<kK1HashBits>(hkey, g, &created) : kNoSlot;
          append_new(list, &s_nlist, created, sl, lane);
          if (sl == kNoSlot) {
            if (g != kEmpty) atomicOr(&s_err[qi], kErrProbe);
          } else {
            slot[i] = sl;
            atomicMin(&gmn[sl], enc);
            atomicMax(&gmx[sl], enc);
            if (FLOAT)
              atomicAdd(&gcnt[sl], 1u);
            else  // count and sum in one word (enc = value + 2^31)
              atomicAdd(&gsum[sl], (1ull << kCntShift) + (unsigned long long)enc);
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
      // ---- B: float sums in fixed point at the group's exponent ----
      if (FLOAT) {
#pragma unroll
        for (int i = 0; i < kK1Items; ++i) {
          const bool has = slot[i] != kNoSlot;
          const unsigned B = has ? group_exp(gmn[slot[i]], gmx[slot[i]]) : 0u;
          if (WAGG) {
            // all peers share the slot (and B): one add of the peers' sum,
            // reduced in three 26-bit slices so that no partial sum overflows
            if (!has) continue;
            if (B == 255u) {
              shared_add_f64(&gsum[slot[i]], (double)__uint_as_float(val[i]));
              continue;
            }
            const unsigned long long x = (unsigned long long)f32_fixed(val[i], B);
            const unsigned s0 = __reduce_add_sync(peer[i], (unsigned)(x & 0x3ffffffull));
            const unsigned s1 = __reduce_add_sync(peer[i], (unsigned)((x >> 26) & 0x3ffffffull));
            const unsigned s2 = __reduce_add_sync(peer[i], (unsigned)(x >> 52));
            if ((int)lane == __ffs(peer[i]) - 1)
              shared_add_u64_split(&gsum[slot[i]], (unsigned long long)s0 +
                                                       ((unsigned long long)s1 << 26) +
                                                       ((unsigned long long)s2 << 52));
          } else {
            if (!has) continue;
            if (B == 255u)
              shared_add_f64(&gsum[slot[i]], (double)__uint_as_float(val[i]));
            else
              shared_add_u64_split(&gsum[slot[i]], (unsigned long long)f32_fixed(val[i], B));
          }
        }
      }
      const unsigned nl = s_nlist;
      if (tid == 0) s_base = nl ? atomicAdd(&Q.ctl->n_parts, (unsigned long long)nl) : 0ull;
      __syncthreads();
      // ---- C: append every group to the partial arrays, clear its slot ----
      const unsigned long long base = s_base;
      const bool fits = base + nl <= Q.parts_cap;
      if (tid == 0 && !fits) atomicOr(&s_err[qi], kErrPartsOverflow);
      unsigned long long o_acc = 0ull, a_acc = ~0ull;
      for (unsigned i = tid; i < nl; i += kK1Threads) {
        const unsigned sl = list[i];
        const unsigned long long g = hkey[sl];
        unsigned long long sb = gsum[sl];
        const unsigned mn = gmn[sl], mx = gmx[sl];
        long long cnt;
        if (FLOAT) {
          cnt = (long long)gcnt[sl];
          const unsigned B = group_exp(mn, mx);
          if (B != 255u)
            sb = fixed_to_double_bits((long long)sb, B);
        } else {
          cnt = (long long)(sb >> kCntShift);
          sb = (sb & ((1ull << kCntShift) - 1ull)) - ((unsigned long long)cnt << 31);
        }
        if (fits) {
          store_grp(Q.parts + base + i, g, cnt, sb, mn, mx);
          Q.pkeys[base + i] = g;
        }
        o_acc |= g;
        a_acc &= g;
        hkey[sl] = kEmpty;
        gsum[sl] = 0ull;
        gcnt[sl] = 0u;
        gmn[sl] = 0xffffffffu;
        gmx[sl] = 0u;
      }
      const unsigned olo = __reduce_or_sync(kFull, (unsigned)o_acc);
      const unsigned ohi = __reduce_or_sync(kFull, (unsigned)(o_acc >> 32));
      const unsigned alo = __reduce_and_sync(kFull, (unsigned)a_acc);
      const unsigned ahi = __reduce_and_sync(kFull, (unsigned)(a_acc >> 32));
      if (lane == 0 && nl) {
        atomicOr(&s_or[qi], ((unsigned long long)ohi << 32) | olo);
        atomicAnd(&s_and[qi], ((unsigned long long)ahi << 32) | alo);
      }
      if (tid == 0) s_nlist = 0u;
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

template <bool FLOAT, int ITEMS, bool WAGG>
cudaError_t launch_k1_t(const K1Args& a, int grid, cudaStream_t st) {
  static unsigned long long done = 0;  // devices whose limit is set
  const cudaError_t attr = set_smem_limit(reinterpret_cast<const void*>(k1_fused<FLOAT, ITEMS, WAGG>),
                                          (int)K1Shape<ITEMS>::kSmem, &done);
  if (attr != cudaSuccess) return attr;
  k1_fused<FLOAT, ITEMS, WAGG><<<grid, kK1Threads, K1Shape<ITEMS>::kSmem, st>>>(a);
  return cudaGetLastError();
}

template <bool FLOAT>
cudaError_t launch_k1_v(const K1Args& a, int variant, int grid, cudaStream_t st) {
  switch (variant) {
    case 2: return launch_k1_t<FLOAT, 4, false>(a, grid, st);
    case 3: return launch_k1_t<FLOAT, 2, true>(a, grid, st);
    case 4: return launch_k1_t<FLOAT, 4, true>(a, grid, st);
    default: return launch_k1_t<FLOAT, 2, false>(a, grid, st);
  }
}

}  // namespace

// Variants: 1 = 1024-event tiles, 2 = 2048-event tiles, 3 / 4 = the same with
// warp aggregation of equal group keys.
cudaError_t launch_k1(const K1Args& a, int variant, int grid, cudaStream_t st) {
  return a.value_is_float ? launch_k1_v<true>(a, variant, grid, st)
                          : launch_k1_v<false>(a, variant, grid, st);
}

int k1_tile_events(int variant) {
  return (variant == 2 || variant == 4) ? K1Shape<4>::kTile : K1Shape<2>::kTile;
}

int k1_max_grid(int device, int variant, int value_is_float) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  (void)value_is_float;
  const int per = (variant == 2 || variant == 4) ? K1Shape<4>::kCtasPerSm : K1Shape<2>::kCtasPerSm;
  return per * (sms > 0 ? sms : 148);  // resident CTAs
}

}  // namespace lms
