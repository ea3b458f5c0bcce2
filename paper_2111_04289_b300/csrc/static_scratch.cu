// lms_aggregate_batch_static: the one-shot windowed aggregation of a single
// device-resident batch, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not
// allowed — for example a plug-in loaded into a host process that owns the
// device memory budget and forbids its guests from allocating, or an engine
// that must not allocate on its serving path.  The stream API allocates (and
// grows) its buffers; this entry point instead carves every intermediate
// buffer of the hot path (partial groups, window state, sort buffers, block
// index, emission item list, control blocks) out of one
// fixed array in device memory that the library declares at file scope.  The
// caller passes the input columns and the output row buffer.
//
// The array (kStaticBytes, about 34 MiB) exists on every GPU that loads the
// library, for the life of the process.  Its device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the first
// call made on that device.  Every call reads the batch's first event time
// back to the host and waits for its stream, so no call may be made while a
// stream is being captured into a CUDA graph.
// Every call on a device shares the array and leaves its contents behind; each
// call re-initialises what must start from zero (the control blocks).  Calls
// are serialised by a process-wide lock and each one synchronises its stream
// before returning, so calls made through this function never overlap; work
// that someone else launches on the array's memory concurrently would race.
#include <climits>
#include <cstring>
#include <mutex>

#include "../../include/lmstream.h"
#include "lms_internal.h"

namespace lms {
namespace {

constexpr unsigned long long kStaticGroups = LMS_STATIC_MAX_ROWS;  // one group per row at most
constexpr unsigned long long kStaticItems = 1ull << 15;  // emission units (item pieces)

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t sctl, qctl;
  size_t parts, pkeys, state;
  size_t keysA, keysB, valsA, valsB, hist, chunk, blk_id, blk_begin;
  size_t item_c, item_j, item_stat, unit_off, unit_bnd, total;
};

constexpr Layout make_layout() {
  Layout L{};
  size_t o = 0;
  L.sctl = o; o += al(sizeof(SCtl));
  L.qctl = o; o += al(sizeof(QCtl));
  L.parts = o; o += al(sizeof(Grp) * kStaticGroups);
  L.pkeys = o; o += al(8 * kStaticGroups);
  L.state = o; o += al(sizeof(Grp) * kStaticGroups);
  L.keysA = o; o += al(8 * kStaticGroups);
  L.keysB = o; o += al(8 * kStaticGroups);
  L.valsA = o; o += al(4 * kStaticGroups);
  L.valsB = o; o += al(4 * kStaticGroups);
  L.hist = o; o += al(4ull * (256 * kGrid + 256));
  L.chunk = o; o += al(8ull * (kGrid + 1));
  L.blk_id = o; o += al(4 * (kStaticGroups + 1));
  L.blk_begin = o; o += al(8 * (kStaticGroups + 1));
  L.item_c = o; o += al(8 * kStaticItems);
  L.item_j = o; o += al(4 * kStaticItems);
  L.item_stat = o; o += al(8 * kStaticItems);
  L.unit_off = o; o += al(8 * kMaxItemWindows * kStaticItems);
  L.unit_bnd = o; o += al(4 * kUnitBnd * kStaticItems);
  L.total = o;
  return L;
}

constexpr Layout kL = make_layout();
constexpr size_t kStaticBytes = kL.total;
static_assert(kStaticBytes < (36ull << 20), "static scratch must stay modest");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Puts the control blocks in the array back to their initial state (names the
// array directly, so the device image always keeps it).
__global__ void k_static_reset() {
  if (blockIdx.x != 0) return;
  unsigned char* q = g_static_scratch + kL.qctl;
  for (size_t i = threadIdx.x; i < sizeof(QCtl); i += blockDim.x) q[i] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    reinterpret_cast<QCtl*>(q)->and_mask = ~0ull;
    SCtl* sc = reinterpret_cast<SCtl*>(g_static_scratch + kL.sctl);
    sc->batch_max_ts = LLONG_MIN;
    sc->wm = 0;
    sc->wm_valid = 0;
    sc->pad = 0;
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_base[kMaxDevices] = {};

// Device address of the scratch array on `dev` (must be the current device).
cudaError_t scratch_base(int dev, unsigned char** out) {
  if (!g_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_base[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_base[dev];
  return cudaSuccess;
}

long long floor_div_s(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

}  // namespace
}  // namespace lms

using namespace lms;

extern "C" lms_status lms_aggregate_batch_static(const lms_query_spec* q, int32_t value_type,
                                                 const int64_t* ts, const uint32_t* key,
                                                 const void* value, const uint8_t* type,
                                                 int64_t n_rows, void* cuda_stream,
                                                 lms_result_row* rows, size_t rows_cap,
                                                 size_t* n_out) {
  if (!q || !n_out || n_rows < 0) return LMS_EINVAL;
  if ((unsigned long long)n_rows > kStaticGroups) return LMS_EINVAL;  // above the fixed maximum
  if (n_rows > 0 && (!ts || !key || !value)) return LMS_EINVAL;
  if (rows_cap > 0 && !rows) return LMS_EINVAL;
  if (value_type != LMS_VALUE_INT32 && value_type != LMS_VALUE_FLOAT32) return LMS_EINVAL;
  const long long size = q->window_size_ms;
  const long long slide = q->window_slide_ms == 0 ? size : q->window_slide_ms;
  if (size <= 0 || slide <= 0 || size % slide != 0 || size / slide > kMaxRuns ||
      slide >= (1ll << 31))
    return LMS_EINVAL;
  if (q->filter_col < LMS_COL_TS || q->filter_col > LMS_COL_TYPE || q->filter_op < LMS_OP_NONE ||
      q->filter_op > LMS_OP_GE)
    return LMS_EINVAL;
  if (q->group_fields || q->having_agg || q->order_agg) return LMS_EINVAL;  // not offered here

  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LMS_ECUDA;
  unsigned char* base = nullptr;
  if (scratch_base(dev, &base) != cudaSuccess) return LMS_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  // ---- carve the buffers out of the fixed array ----
  SCtl* sctl = reinterpret_cast<SCtl*>(base + kL.sctl);
  QueryDev d{};
  d.ctl = reinterpret_cast<QCtl*>(base + kL.qctl);
  d.parts = reinterpret_cast<Grp*>(base + kL.parts);
  d.pkeys = reinterpret_cast<unsigned long long*>(base + kL.pkeys);
  d.state = reinterpret_cast<Grp*>(base + kL.state);
  d.parts_cap = kStaticGroups;
  Scratch s{};
  s.keysA = reinterpret_cast<unsigned long long*>(base + kL.keysA);
  s.keysB = reinterpret_cast<unsigned long long*>(base + kL.keysB);
  s.valsA = reinterpret_cast<unsigned*>(base + kL.valsA);
  s.valsB = reinterpret_cast<unsigned*>(base + kL.valsB);
  s.cap = kStaticGroups;
  s.hist = reinterpret_cast<unsigned*>(base + kL.hist);
  s.chunk = reinterpret_cast<unsigned long long*>(base + kL.chunk);
  s.blk_id = reinterpret_cast<unsigned*>(base + kL.blk_id);
  s.blk_begin = reinterpret_cast<unsigned long long*>(base + kL.blk_begin);
  s.blk_cap = kStaticGroups;
  s.item_c = reinterpret_cast<unsigned long long*>(base + kL.item_c);
  s.item_j = reinterpret_cast<unsigned*>(base + kL.item_j);
  s.item_stat = reinterpret_cast<unsigned long long*>(base + kL.item_stat);
  s.unit_off = reinterpret_cast<unsigned long long*>(base + kL.unit_off);
  s.unit_bnd = reinterpret_cast<unsigned*>(base + kL.unit_bnd);
  s.item_cap = kStaticItems;

  // ---- the query, with the batch's first row as event-time origin ----
  d.filter_col = q->filter_col;
  d.filter_op = q->filter_op;
  d.filter_i = q->filter_i;
  d.filter_f = q->filter_f;
  set_float_filter(&d);
  d.slide = (unsigned long long)slide;
  udiv_constants(d.slide, &d.magic, &d.sh1, &d.sh2);
  d.size = size;
  d.k = (int)(size / slide);
  set_block_shape(&d);
  d.key_mask = 0xffffffffu;
  d.agg_mask = q->agg_mask ? q->agg_mask : LMS_AGG_ALL;
  d.qid = 0;
  d.value_is_float = value_type == LMS_VALUE_FLOAT32;
  // the origin is read on the caller's stream, after whatever work of the
  // caller's on that stream produced the columns
  long long origin = 0;
  if (n_rows > 0 &&
      (cudaMemcpyAsync(&origin, ts, sizeof(origin), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    return LMS_ECUDA;
  d.origin_pane = floor_div_s(origin, slide);
  d.base = d.origin_pane * slide;
  d.ts_off = (unsigned long long)kPaneBias * (unsigned long long)slide - (unsigned long long)d.base;
  d.u_limit = 0xffffffffull * (unsigned long long)slide;

  // ---- reset the control blocks the previous call left behind ----
  k_static_reset<<<1, 128, 0, st>>>();
  if (cudaGetLastError() != cudaSuccess) return LMS_ECUDA;

  // ---- the hot path, end of stream: every window is emitted ----
  QCtl* ctls[1] = {d.ctl};
  if (launch_batch_begin(sctl, ctls, 1, LLONG_MIN, st) != cudaSuccess) return LMS_ECUDA;
  if (n_rows > 0) {
    K1Args a{};
    a.ts = reinterpret_cast<const long long*>(ts);
    a.key = key;
    a.value = value;
    a.type = type;
    a.n = n_rows;
    a.nq = 1;
    a.value_is_float = d.value_is_float;
    a.sctl = sctl;
    a.q[0] = d;
    const long long ntiles = (n_rows + k1_tile_events(1) - 1) / k1_tile_events(1);
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    if (launch_k1(a, 1, grid, st) != cudaSuccess) return LMS_ECUDA;
  }
  if (launch_watermark(sctl, &d, 1, 0, 1, st) != cudaSuccess) return LMS_ECUDA;
  if (launch_sort_reduce(d, s, st, nullptr) != cudaSuccess) return LMS_ECUDA;
  if (launch_block_index(d, s, st, nullptr) != cudaSuccess) return LMS_ECUDA;
  if (launch_emit(d, s, reinterpret_cast<ResultRowDev*>(rows), rows_cap, sms, st, nullptr,
                  nullptr) != cudaSuccess)
    return LMS_ECUDA;
  QCtl h{};
  if (cudaMemcpyAsync(&h, d.ctl, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LMS_ECUDA;
  if (h.err & (kErrPartsOverflow | kErrProbe)) return LMS_EDEVICE;
  if (h.err & kErrNeedRetry) return LMS_ENOMEM;  // item list or rows_cap too small
  *n_out = (size_t)h.rows_batch;
  return LMS_OK;
}
