// Internal declarations shared by the engine (host) and the CUDA kernels.
//
// Data model of one query's window state (all in device memory):
//   * a group is one (pane, key) pair; a pane is one slide-long slice of event
//     time (pane p covers [p*slide, (p+1)*slide)).  A window of size K*slide is
//     the union of K consecutive panes, so every event updates exactly one
//     group, whatever K is; windows are assembled from panes at emission.
//   * panes are numbered relative to the stream's origin, pane_rel = pane -
//     origin_pane + 2^31 (< 2^32), and grouped into blocks of B = 2^lb panes,
//     B the smallest power of two >= K.  The group key is
//       gkey = (block << (32 + lb)) | (key << lb) | (pane_rel mod B),
//     so sorting gkeys as uint64 orders groups by (block, key, pane): inside a
//     block the state is key-major.  The windows starting in one block touch
//     only that block and the next, so each of them is assembled from two
//     key-sorted runs.  Tumbling windows have B = 1 (the (pane, key) order).
//   * Groups are 32-byte records {gkey, cnt, sum, mn, mx} (Grp); min/max are
//     stored order-preserving encoded as uint32 (see lms_device.cuh).  The
//     partial groups' keys are also kept in a compact array for the sort.
// Per micro-batch, the fused pass appends per-tile partial groups after the
// carried state; a radix sort + reduce-by-key turns them into the sorted,
// unique window state; closed windows are assembled from their blocks and
// emitted.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lms {

constexpr int kMaxQueries = 8;
constexpr int kMaxRuns = 4096;           // max size/slide of a sliding window
constexpr long long kPaneBias = 1ll << 31;  // pane_rel = pane - origin_pane + kPaneBias

// Error bits raised by kernels (QCtl::err).
constexpr unsigned kErrPartsOverflow = 1u;   // partial-group buffer too small
constexpr unsigned kErrItemOverflow = 2u;    // emission item list too small
constexpr unsigned kErrRowsOverflow = 4u;    // result buffer too small
constexpr unsigned kErrProbe = 16u;          // shared hash probe bound hit (never expected)
constexpr unsigned kErrOrderBy = 64u;        // ORDER BY: a window holds more than kOrderMax rows
constexpr unsigned kErrNeedRetry = kErrItemOverflow | kErrRowsOverflow;

// Largest window ORDER BY sorts (in shared memory).
constexpr int kOrderMax = 16384;

// Windows per emission item (an item is a run of consecutive window ids that
// start in one block).
constexpr int kMaxItemWindows = 64;
// Pane-word emission (2B <= 32): a unit is kPwUnitChunks chunks of nominally
// kPwChunkEntries merged entries; its chunk boundaries take 2 * (chunks + 1)
// words of the unit boundary table.
constexpr int kPwChunkEntries = 96;
constexpr int kPwUnitChunks = 11;
constexpr int kUnitBnd = 2 * (kPwUnitChunks + 1);


// One (pane, key) group: a 32-byte record, so that a random gather of a group
// touches one DRAM sector.
struct __align__(32) Grp {
  unsigned long long gkey;
  long long cnt;
  unsigned long long sum;  // int64 sum, or the bits of a double sum
  unsigned mn;             // encoded min
  unsigned mx;             // encoded max
};

// Per-query device control block.
struct QCtl {
  unsigned long long n_parts;    // partial groups (carried + this batch)
  unsigned long long or_mask;    // OR of all partial gkeys
  unsigned long long and_mask;   // AND of all partial gkeys
  unsigned long long n_state;    // unique groups in the window state
  unsigned long long n_blocks;   // distinct blocks in the window state
  unsigned long long n_items;    // emission items of the windows closed by this batch
  long long cursor;              // first (relative) window id not yet closed
  long long w_hi;                // last (relative) window id closed by this batch
  unsigned long long late_rows;  // cumulative
  unsigned long long range_rows; // cumulative
  unsigned long long rows_batch; // rows emitted by this batch
  unsigned long long row_base;   // rows held in the device result buffer
  unsigned long long carried;    // groups carried into the next batch
  unsigned long long trim_from;  // first state index that may be carried into the next batch
  unsigned long long item_ticket;// next emission unit of the row count (CTAs take units by ticket)
  unsigned long long unit_ticket;// next emission unit of the row writes
  unsigned long long rows_kept;  // rows HAVING kept of this batch's
  unsigned long long parts_at_sort; // partial groups the sort of this batch consumed
  unsigned long long n_long;     // long runs of equal keys left to the cooperative reduce
  unsigned long long sort_base;  // carried groups at the front of the partials: only the rest
                                 // is sorted, then merged with them
  unsigned int err;
  int npasses;
  int shifts[8];
};

// Stream-level device control block.
struct SCtl {
  long long batch_max_ts;  // max ts of the current batch (LLONG_MIN if empty)
  long long wm;            // watermark
  int wm_valid;
  int pad;
};

// Everything a kernel needs to know about one query.
struct QueryDev {
  int filter_col, filter_op;
  long long filter_i;
  double filter_f;
  // Float32 image of `(double)v OP filter_f` for float32 values v: with
  // lo = largest float <= filter_f and hi = smallest float >= filter_f,
  // v > c <=> v > lo, v >= c <=> v >= hi, v < c <=> v < hi, v <= c <=> v <= lo,
  // v == c <=> (lo == hi) && v == lo.  Set by set_float_filter().
  float filter_lo, filter_hi;
  int filter_exact;
  int pad0;
  unsigned long long slide;
  unsigned long long magic;  // invariant-division constants for `slide`
  int sh1, sh2;
  unsigned long long ts_off;   // u = (u64)ts + ts_off  (= 2^31*slide - base)
  unsigned long long u_limit;  // event valid iff u < u_limit (= (2^32-1)*slide)
  long long size;
  long long base;              // origin_pane * slide
  long long origin_pane;
  int k;                       // size / slide
  int lb;                      // log2 of the block size B (smallest power of two >= k)
  int nw;                      // windows per emission item: min(B, kMaxItemWindows)
  unsigned key_mask;           // GROUP BY: the bits of the key's selected fields
  int having_agg, having_op;   // HAVING agg OP having_value (agg 0: none)
  double having_value;
  int order_agg, order_desc;   // ORDER BY agg (0: none), descending
  unsigned agg_mask;
  int qid;
  int value_is_float;
  Grp* parts;                  // partial groups (carried + this batch)
  unsigned long long* pkeys;   // their keys, compact (first radix pass reads these)
  Grp* state;                  // sorted, unique window state
  unsigned long long parts_cap;
  QCtl* ctl;
};

struct K1Args {
  const long long* ts;
  const unsigned* key;
  const void* value;
  const unsigned char* type;
  long long n;
  int nq;
  int value_is_float;
  SCtl* sctl;
  QueryDev q[kMaxQueries];
};

// Scratch shared by the per-query pipelines: each query's sort/reduce, block
// index, emission and carry run back to back before the next query's start.
struct Scratch {
  unsigned long long* keysA;
  unsigned* valsA;
  unsigned long long* keysB;
  unsigned* valsB;
  unsigned long long cap;        // entries of keysA/B, valsA/B
  unsigned* hist;                // 256 * kGrid per-chunk digit counts, then 256 digit totals
  unsigned long long* chunk;     // kGrid (+1) per-chunk counts / offsets
  unsigned* blk_id;              // distinct blocks of the state [blk_cap]
  unsigned long long* blk_begin; // their first state index [blk_cap + 1]
  unsigned long long blk_cap;
  unsigned long long* item_c;    // emission items: window chunk c (windows [c*nw, c*nw + nw))
  unsigned* item_j;              // index of the block that anchors the item
  unsigned long long* item_stat; // per unit: its index in the item | the item's units << 32
  unsigned long long* unit_off;  // kMaxItemWindows per unit: row counts, then output rows
                                 // (a query uses nw of them per unit)
  unsigned* unit_bnd;            // pane-word path, kUnitBnd per unit: its chunk boundaries,
                                 // each as the (A, B) entries of the item before it
  unsigned long long item_cap;   // units the unit arrays hold
};

struct ResultRowDev {  // device image of lms_result_row (48 bytes)
  long long window_start;
  long long count;
  unsigned long long sum;
  double avg;
  unsigned key;
  unsigned mn;
  unsigned mx;
  unsigned qid;
};

constexpr int kGrid = 592;         // CTAs of the chunked (count/scan/write) kernels: 4 per SM
constexpr int kChunkThreads = 256;

// Windowed equi-join: device image of lms_join_row (56 bytes), its control
// block, and what the join kernels read.
struct JoinRowDev {
  long long window_start;
  long long pairs;
  long long left_count;
  long long right_count;
  unsigned long long left_sum;   // int64 or the bits of a double
  unsigned long long right_sum;
  unsigned key;
  unsigned jid;
};
struct JCtl {
  unsigned long long rows_batch;  // join rows of this batch
  unsigned long long row_base;    // join rows held in the device buffer
  unsigned err;                   // pending / overflow bits
  unsigned pad;
};
struct JoinArgs {
  const ResultRowDev* lrows;  // the left side's (hidden query's) rows
  QCtl* lc;
  const ResultRowDev* rrows;
  QCtl* rc;
  JoinRowDev* out;
  unsigned long long cap;
  JCtl* jc;
  int jid;
  int pad;
};
constexpr unsigned kJoinPendingBit = 1u, kJoinOverflowBit = 2u;

// ---- launch wrappers (kernels_*.cu) -------------------------------------
// All enqueue on `st` and return the launch error.
// ts_floor: LLONG_MIN, or a lower bound of the batch's max event time (a
// watermark hint, lms_stream_set_batch_max_ts).
cudaError_t launch_batch_begin(SCtl* sctl, QCtl* const* ctls, int nq, long long ts_floor,
                               cudaStream_t st);
cudaError_t launch_k1(const K1Args& a, int variant, int grid, cudaStream_t st);
int k1_max_grid(int device, int variant, int value_is_float);
int k1_tile_events(int variant);
cudaError_t launch_watermark(SCtl* sctl, const QueryDev* qs, int nq, long long lateness, int eos,
                             cudaStream_t st);
cudaError_t launch_sort_reduce(const QueryDev& q, const Scratch& s, cudaStream_t st,
                               int* launches);
cudaError_t launch_block_index(const QueryDev& q, const Scratch& s, cudaStream_t st,
                               int* launches);
cudaError_t launch_emit(const QueryDev& q, const Scratch& s, ResultRowDev* rows,
                        unsigned long long rows_cap, int sms, cudaStream_t st, int* launches,
                        cudaEvent_t* ev4);
cudaError_t launch_trim(const QueryDev& q, const Scratch& s, int sms, cudaStream_t st,
                        int* launches);
// The join of this batch's rows of both sides (begin: mark it pending first).
cudaError_t launch_join(const JoinArgs& a, const Scratch& s, bool begin, cudaStream_t st,
                        int* launches);
// HAVING and ORDER BY over the rows the emission just wrote (tmp_rows: a
// scratch row buffer as large as rows).
cudaError_t launch_post(const QueryDev& q, const Scratch& s, ResultRowDev* rows,
                        ResultRowDev* tmp_rows, int sms, cudaStream_t st, int* launches);

// Synthetic load generator of the serving backend (kernels_gen.cu).
struct GenChunk {
  double t0_ms, width_ms;
  long long n_total, j_begin, first_event;
  long long offset;  // index of the chunk's first event in the batch
};
cudaError_t launch_gen_pool(unsigned long long seed, const double* cdf, unsigned n_keys,
                            long long pool, long long n, unsigned* key, float* value, int sms,
                            cudaStream_t st);
cudaError_t launch_gen_ts(const GenChunk* chunks, int n_chunks, long long n, long long* ts,
                          int sms, cudaStream_t st);

// Records a timing event on st; while st is being captured into a graph the
// record becomes an external event node, so that every replay records it.
inline cudaError_t record_event(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  return cudaEventRecord(e, st);
}

// Fills filter_lo / filter_hi / filter_exact from filter_f.
void set_float_filter(QueryDev* d);

// Fills lb and nw from k.
void set_block_shape(QueryDev* d);

// Sets a kernel's dynamic shared-memory limit once per device (the attribute
// belongs to the function's instance on the current device).
cudaError_t set_smem_limit(const void* fn, int bytes, unsigned long long* done_mask);

// Invariant division constants (Granlund & Montgomery 1994, unsigned, N=64).
void udiv_constants(unsigned long long d, unsigned long long* magic, int* sh1, int* sh2);

}  // namespace lms
