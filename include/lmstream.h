/*
 * lmstream.h — C ABI of the B300 micro-batch stream engine.
 *
 * The engine runs the data-parallel hot path of LMStream's micro-batch stream
 * queries on one GPU: every pushed micro-batch is filtered and projected, each
 * surviving event is given its tumbling or sliding window(s), the events are
 * group-by aggregated (count, int64 / double sum, min, max, avg) into window
 * state that stays in device memory, and every window that the watermark has
 * passed is emitted.  The paper states the problem as micro-batches of
 * datasets that are processed as one unit (Section III-B, Table I) by SQL
 * queries over windows (Table III); it leaves window semantics to Spark.  The
 * engine fixes them as follows (event time, ms):
 *
 *   - window k of an event: [s, s + size) with s = (floor(ts/slide) - k)*slide,
 *     k = 0 .. size/slide - 1 (tumbling: slide == size);
 *   - watermark after a batch: max(previous, max ts of ALL rows of the batch
 *     - allowed_lateness); a window is emitted once its end <= watermark;
 *     end-of-stream emits everything;
 *   - an event is not added to a window that was already emitted; an event all
 *     of whose windows were emitted is a "late row" and is counted;
 *   - rows come out ordered by (window_start, key); avg = (double)sum / count.
 *
 * Threading: one producer thread per stream calls push_microbatch; any thread
 * may call poll_results / lms_stream_stats (the stream serialises them).
 * Memory: the library allocates and owns all device and pinned memory of a
 * stream; callers own the buffers they pass in and may reuse them as soon as
 * a call returns.  CUDA errors are latched: the failing call and every later
 * call return LMS_ECUDA; lms_last_error() gives the message.
 * Out-parameters are written only when a call returns LMS_OK.
 */
#ifndef LMSTREAM_H
#define LMSTREAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lms_stream lms_stream; /* opaque; owned by the library */
typedef int32_t lms_status;

/* Status codes. */
#define LMS_OK 0
#define LMS_EINVAL (-1)    /* bad argument or specification */
#define LMS_ENOMEM (-2)    /* device/pinned allocation failed or state cap exceeded */
#define LMS_EAGAIN (-3)    /* no result rows available (poll) */
#define LMS_ETIMEDOUT (-4) /* a bounded device wait ran out */
#define LMS_ECUDA (-5)     /* a CUDA call failed (latched) */
#define LMS_ECLOSED (-6)   /* stream already at end-of-stream */
#define LMS_ERANGE (-7)    /* event time outside the supported span (see origin_ts) */
#define LMS_EDEVICE (-8)   /* a kernel raised an internal error flag */

/* Value column type. */
#define LMS_VALUE_INT32 0
#define LMS_VALUE_FLOAT32 1

/* Columns a filter can test. */
#define LMS_COL_TS 0    /* int64 event time, ms */
#define LMS_COL_KEY 1   /* uint32 group-by key */
#define LMS_COL_VALUE 2 /* int32 or float32 aggregated value */
#define LMS_COL_TYPE 3  /* uint8 event type (reads as 0 if the stream has none) */

/* Filter operators: `column OP constant`.  Integer columns compare as int64
 * against filter_i; a float32 value column compares as double against
 * filter_f (IEEE semantics: NaN passes only NE). */
#define LMS_OP_NONE 0
#define LMS_OP_EQ 1
#define LMS_OP_NE 2
#define LMS_OP_LT 3
#define LMS_OP_LE 4
#define LMS_OP_GT 5
#define LMS_OP_GE 6

/* Aggregates (bit mask).  All five are always computed; the mask says which
 * result fields a caller wants (the kernels skip min/max work when unset). */
#define LMS_AGG_COUNT 1u
#define LMS_AGG_SUM 2u
#define LMS_AGG_MIN 4u
#define LMS_AGG_MAX 8u
#define LMS_AGG_AVG 16u
#define LMS_AGG_ALL 31u

/* Where the columns of a pushed batch live. */
#define LMS_MEM_HOST 0   /* host memory (pinned or pageable); copied in by the call */
#define LMS_MEM_DEVICE 1 /* device memory of the stream's GPU; read in place */

/* Batch flags. */
#define LMS_BATCH_EOS 1u /* end of stream: emit every remaining window */
#define LMS_INGEST_STABLE 2u /* lms_ingest: the host columns are pinned and stay unchanged until
                                the lms_push_ingested that covers them returns, so the library
                                copies them to the device directly instead of through its own
                                pinned ring */

/* origin_ts value that means "the first row of the first pushed batch". */
#define LMS_ORIGIN_AUTO INT64_MIN

typedef struct lms_stream_config {
  int32_t device;              /* CUDA device ordinal */
  int32_t value_type;          /* LMS_VALUE_INT32 or LMS_VALUE_FLOAT32 */
  int32_t has_type;            /* 1 if batches carry the uint8 type column */
  int32_t enable_timing;       /* 1: record per-phase CUDA-event times (stats) */
  int64_t allowed_lateness_ms; /* watermark = max ts - allowed_lateness_ms (>= 0) */
  int64_t max_batch_rows;      /* sizing hint for the largest push (buffers grow on demand) */
  uint64_t state_cap_bytes;    /* cap on the stream's device memory, 0 = no cap */
  void *cuda_stream;           /* cudaStream_t to run on, or NULL: the library creates one */
  int64_t origin_ts;           /* event-time origin; LMS_ORIGIN_AUTO by default.  Window ids
                                  are kept relative to it: events must satisfy
                                  |floor(ts/slide) - floor(origin_ts/slide)| < 2^31 - 1,
                                  others are dropped and counted (stats.range_rows). */
  int32_t k1_variant;          /* fused pass: 0 = autotuned per batch-size class; 1 = 1024-event
                                  tiles (two CTAs per SM); 2 = 2048-event tiles (one CTA per SM);
                                  3 / 4 = 1 / 2 with warp aggregation of equal group keys */
  int32_t graph_mode;          /* LMS_GRAPH_*: replay the per-batch launch sequence from a CUDA graph */
  int32_t reserved0;           /* 0 */
  uint32_t reserved1;          /* 0 */
  uint32_t key_fields;         /* the key column as up to four packed fields: byte f holds the
                                  bit width of field f (field 0 in the lowest bits); 0 = one
                                  32-bit field.  Widths must sum to <= 32. */
  int32_t reserved[3];
} lms_stream_config;

/* graph_mode.  Everything a push launches after the fused pass reads its sizes
 * on the device, so the sequence is captured once into a CUDA graph and
 * replayed; a new capture follows every reallocation of a stream buffer. */
#define LMS_GRAPH_DEFAULT 0 /* = LMS_GRAPH_ON */
#define LMS_GRAPH_OFF 1     /* plain launches */
#define LMS_GRAPH_ON 2

typedef struct lms_query_spec {
  int32_t filter_col;     /* LMS_COL_* */
  int32_t filter_op;      /* LMS_OP_* */
  int64_t filter_i;       /* constant for integer columns */
  double filter_f;        /* constant for the float32 value column */
  int64_t window_size_ms; /* > 0 */
  int64_t window_slide_ms;/* 0 or == size: tumbling; else size % slide == 0 and
                             size/slide <= 4096 (sliding) */
  uint32_t agg_mask;      /* LMS_AGG_* bits; 0 means LMS_AGG_ALL */
  uint32_t group_fields;  /* GROUP BY the key fields whose bits are set (of the stream's
                             key_fields, bit f = field f); 0 = the whole key.  A row's key
                             holds the selected fields in place, the others zero. */
  int32_t having_agg;     /* HAVING: LMS_POST_* aggregate, 0 = none */
  int32_t having_op;      /* LMS_OP_*: a row is kept iff (double)agg OP having_value */
  double having_value;
  int32_t order_agg;      /* ORDER BY: LMS_POST_* aggregate, 0 = none (rows in key order) */
  int32_t order_desc;     /* 1: descending; equal values keep key order either way */
} lms_query_spec;

/* Aggregates HAVING and ORDER BY refer to (Table III: LR2S's HAVING
 * avgSpeed < 40.0, CM1's ORDER BY SUM(cpu)).  ORDER BY sorts each window's
 * rows in device shared memory: a window may then hold at most
 * LMS_ORDER_MAX_ROWS rows (push returns LMS_EINVAL otherwise). */
#define LMS_POST_COUNT 1
#define LMS_POST_SUM 2
#define LMS_POST_MIN 3
#define LMS_POST_MAX 4
#define LMS_POST_AVG 5
#define LMS_ORDER_MAX_ROWS 16384

typedef struct lms_batch {
  int64_t n_rows;       /* rows in the batch (>= 0) */
  const int64_t *ts;    /* [n_rows] event time, ms */
  const uint32_t *key;  /* [n_rows] group-by key */
  const void *value;    /* [n_rows] int32 or float32 per the stream's value_type */
  const uint8_t *type;  /* [n_rows] or NULL; required iff has_type */
  int32_t memory;       /* LMS_MEM_HOST or LMS_MEM_DEVICE */
  uint32_t flags;       /* LMS_BATCH_* */
  int64_t arrival_ns;   /* caller's arrival timestamp (latency accounting), 0 if unknown */
} lms_batch;

/* One emitted window-group, 48 bytes.  sum/min/max are integer for an
 * INT32 stream and floating for a FLOAT32 stream. */
typedef struct lms_result_row {
  int64_t window_start; /* ms; the window is [window_start, window_start + size) */
  int64_t count;
  union { int64_t i; double f; } sum;
  double avg;           /* (double)sum / count */
  uint32_t key;
  union { int32_t i; float f; } min;
  union { int32_t i; float f; } max;
  uint32_t query_id;
} lms_result_row;

typedef struct lms_stats {
  uint64_t batches;        /* micro-batches pushed */
  uint64_t events;         /* rows pushed */
  uint64_t late_rows;      /* surviving rows all of whose windows were already emitted (all queries) */
  uint64_t range_rows;     /* rows dropped for lying outside the supported event-time span */
  uint64_t rows_emitted;   /* result rows produced (all queries) */
  uint64_t rows_pending;   /* result rows not yet polled (all queries) */
  int64_t watermark;       /* current watermark (INT64_MIN before the first row) */
  uint64_t state_groups;   /* (window-pane, key) groups held in device state (all queries) */
  uint64_t device_bytes;   /* device memory held by the stream */
  double last_batch_ms;    /* wall time of the last push_microbatch */
  /* Per-phase device time, summed over batches (only if enable_timing): */
  double k1_ms;            /* fused filter/window/pre-aggregate pass */
  double sort_ms;          /* sort + reduce of partial groups into window state */
  double emit_ms;          /* window enumeration, merge and row emission */
  double h2d_ms;           /* host-to-device input copies */
  uint64_t k1_launches;    /* launches of the fused pass */
  uint64_t kernel_launches;/* all kernel launches of the hot path */
  double e1_ms;            /* window assembly: distinct-key count per closed window */
  double e2_ms;            /* window assembly + row write */
  uint64_t partials;       /* partial groups written by the fused pass (all batches, queries) */
  uint64_t groups_built;   /* window-state groups produced by the reduce (all batches, queries) */
  uint64_t graph_launches; /* pushes whose tail ran as one CUDA graph launch */
  uint64_t graph_captures; /* graph (re)captures */
  uint64_t k1_tile_events; /* tile of the last fused pass */
  uint64_t autotune_samples; /* fused passes timed by the autotuner */
} lms_stats;

/* Opens a stream on cfg->device.  Defined by the paper's problem statement
 * (Section III-B, Table I: a stream is cut into micro-batches that one query
 * plan processes).  cfg is copied.  Returns LMS_EINVAL for a bad config,
 * LMS_ECUDA if the device cannot be used.  *out is owned by the caller until
 * stream_close(). */
lms_status stream_open(const lms_stream_config *cfg, lms_stream **out);

/* Registers a windowed group-by query (Table III: WHERE filter, window
 * [range size slide s], GROUPBY key, SUM/AVG/...).  Must precede the first
 * push.  *query_id receives 0, 1, ... in registration order (at most 8
 * queries per stream; they run fused over each batch).  LMS_EINVAL if the
 * window or filter is invalid. */
lms_status query_register(lms_stream *s, const lms_query_spec *q, int32_t *query_id);

/* ---- windowed equi-join of two streams -------------------------------------
 *
 * Table III's LR1S / LR1T join a windowed stream with a stream on vehicle
 * (Join: Table II, base cost 0.9).  Here the two sides are the rows of the
 * stream that pass a left and a right predicate (a type column can tell two
 * streams apart; for a self-join both predicates may be LMS_OP_NONE).  For
 * every window (as for queries: [start, start + size), sliding by slide,
 * emitted once the watermark passes its end) the join's result is the
 * multiset of pairs (l, r) of the window's left and right rows with equal
 * keys.  It is reported in factored form, one lms_join_row per (window, key)
 * present on both sides, in (window_start, key) order: pairs = left_count *
 * right_count, with both sides' counts and value sums (every aggregate over
 * the pairs that separates per side follows, e.g. the sum of the left values
 * over all pairs is left_sum * right_count).  The pairs are not listed one by
 * one: with Zipf-distributed keys their number grows with the square of a hot
 * key's count.  Each side runs as an aggregation query of the stream, so a
 * join takes two of the stream's eight query slots (their ids are not
 * returned and cannot be polled); register joins before the first push. */
typedef struct lms_join_spec {
  int64_t window_size_ms;  /* > 0 */
  int64_t window_slide_ms; /* 0 or == size: tumbling; else as for queries */
  int32_t left_col, left_op;   /* left side predicate: LMS_COL_*, LMS_OP_* */
  int64_t left_i;
  double left_f;
  int32_t right_col, right_op; /* right side predicate */
  int64_t right_i;
  double right_f;
} lms_join_spec;

typedef struct lms_join_row { /* 56 bytes */
  int64_t window_start;
  int64_t pairs;        /* left_count * right_count */
  int64_t left_count;
  int64_t right_count;
  union { int64_t i; double f; } left_sum;  /* integer for an INT32 stream */
  union { int64_t i; double f; } right_sum;
  uint32_t key;
  uint32_t join_id;
} lms_join_row;

/* Registers a join; *join_id receives 0, 1, ... (at most 4 joins).  LMS_EINVAL
 * for a bad window or predicate, or when fewer than two query slots remain. */
lms_status lms_join_register(lms_stream *s, const lms_join_spec *j, int32_t *join_id);
/* Copies up to cap of the join's rows, oldest first, into out (host) and
 * removes them; LMS_EAGAIN if there are none. */
lms_status lms_join_poll(lms_stream *s, int32_t join_id, lms_join_row *out, size_t cap,
                         size_t *n_out);

/* Processes one micro-batch (the paper's processing phase, Section III-A)
 * through every registered query and emits the windows it closes.  Returns
 * when the results are ready to poll.  Columns are read from host or device
 * memory per b->memory; the caller keeps ownership.  After a batch with
 * LMS_BATCH_EOS, further pushes return LMS_ECLOSED.  An empty batch only
 * advances nothing unless it carries EOS. */
lms_status push_microbatch(lms_stream *s, const lms_batch *b);

/* Copies up to `cap` of query `query_id`'s emitted rows, oldest first, into
 * the caller's host buffer `out` and removes them from the stream.
 * *n_out receives the number copied.  LMS_EAGAIN if there are none (results
 * are complete when push_microbatch returns, so timeout_ms only bounds the
 * wait for a concurrent push and may be 0). */
lms_status poll_results(lms_stream *s, int32_t query_id, lms_result_row *out, size_t cap,
                        size_t *n_out, int32_t timeout_ms);

/* Waits for outstanding device work, frees every device and pinned buffer
 * and destroys the stream (and its CUDA stream if the library created it).
 * `s` is invalid afterwards.  NULL is accepted. */
lms_status stream_close(lms_stream *s);

/* ---- extras ---------------------------------------------------------- */

/* Counters and timings of the stream (see lms_stats). */
lms_status lms_stream_stats(lms_stream *s, lms_stats *out);

/* Message of the last error on this stream ("" if none); valid until the
 * next call on the stream. */
const char *lms_last_error(lms_stream *s);

/* Device-resident view of query_id's unpolled rows: *rows receives a device
 * pointer to *n rows in the same order poll_results would return them.  The
 * view stays valid until the next push, poll or discard on the stream. */
lms_status lms_results_device(lms_stream *s, int32_t query_id, const lms_result_row **rows,
                              size_t *n);

/* Grows the stream's buffers now so that a push of n_rows rows (from host
 * memory if host_input is 1; through the ingest ring if host_input is 2)
 * allocates nothing.  Queries must be registered.  LMS_ENOMEM if that exceeds
 * state_cap_bytes or the device. */
lms_status lms_stream_reserve(lms_stream *s, int64_t n_rows, int32_t host_input);

/* Device bytes a push of n_rows rows (from host memory if host_input is 1)
 * would newly allocate for its group, sort and input buffers (and the first
 * push's emission buffers; later growth of the result and window buffers
 * follows the rows a batch emits and is not included), and the device bytes
 * the stream holds now. */
lms_status lms_stream_push_bytes(lms_stream *s, int64_t n_rows, int32_t host_input,
                                 uint64_t *bytes);
lms_status lms_stream_device_bytes(lms_stream *s, uint64_t *bytes);

/* Admission by device memory (the serving loop's; the paper has none): the
 * largest n_rows the next push can take without the stream's device memory
 * exceeding cfg.state_cap_bytes, counting the growth of every buffer a push of
 * that size may need (group arrays for the carried groups plus one group per
 * row, sort scratch, the input copy when host_input is 1) and a reserve of
 * max(cap/16, 64 MiB) for result rows and window lists.  *n_out = -1 when the
 * stream has no cap; 0 when nothing fits. */
lms_status lms_stream_admissible_rows(lms_stream *s, int32_t host_input, int64_t *n_out);

/* Per-query split of the batch work (times need enable_timing; the fused
 * pass is shared by all queries and counted in lms_stats.k1_ms only):
 * sort + merge + reduce into the window state, emission row counts (unit list,
 * counts, offsets) and emission row writes, in ms summed over the pushes; the
 * rows the query emitted and the groups it carries into the next batch. */
typedef struct lms_query_stats_t {
  double sort_ms;
  double emit_count_ms;
  double emit_write_ms;
  uint64_t rows_emitted;
  uint64_t state_groups;
} lms_query_stats_t;
lms_status lms_query_stats(lms_stream *s, int32_t query_id, lms_query_stats_t *out);

/* Drops query_id's unpolled rows (e.g. after consuming them on the device). */
lms_status lms_results_discard(lms_stream *s, int32_t query_id);

/* ---- ingest ring: arriving data goes to the device while it is buffered ----
 *
 * The paper's micro-batches are built from datasets that arrive and wait in a
 * buffer until ConstructMicroBatch (Alg. 1, Section III-C) admits them; the
 * buffering phase takes 13-93 % of the time (Table IV).  lms_ingest takes one
 * arriving dataset (host columns, b->memory = LMS_MEM_HOST): it copies the
 * rows into a pinned host ring that the library owns (unless b->flags holds
 * LMS_INGEST_STABLE) and enqueues their host-to-device copy into a device
 * ring on a side stream, then returns; the caller may reuse its buffers at
 * once (with LMS_INGEST_STABLE: once the covering lms_push_ingested returns).
 * The copy runs while the data waits and while earlier micro-batches compute.
 * lms_push_ingested then processes the oldest n_rows ingested rows as one
 * micro-batch exactly as push_microbatch would (flags: LMS_BATCH_EOS): the
 * compute stream waits only for the copies still in flight.  Both rings grow
 * on demand (device memory counts against state_cap_bytes).  While ingested
 * rows are pending, push_microbatch returns LMS_EINVAL.  Errors: LMS_EINVAL
 * for bad arguments or n_rows above the rows pending; LMS_ENOMEM if a ring
 * cannot grow; LMS_ECLOSED after end of stream. */
lms_status lms_ingest(lms_stream *s, const lms_batch *b);
lms_status lms_push_ingested(lms_stream *s, int64_t n_rows, uint32_t flags);
/* Rows ingested and not yet pushed. */
lms_status lms_ingest_pending(lms_stream *s, int64_t *n_rows);

/* ---- key sharding across devices (one stream per device) ----
 *
 * A group (window, key) depends only on the rows of its key, so the key space
 * can be split over G streams, one per GPU, each owning the keys with
 * lms_shard_of(key, key_mask, G) == its index (the "Shuffling" operation of
 * Table II, done on the host before the copy to the device).  Every shard
 * stream must be opened with the same configuration and an explicit event-time
 * origin (lms_stream_config.origin_ts or lms_stream_set_origin), register the
 * same queries and joins in the same order, and be pushed once per global
 * micro-batch (an empty shard included) after lms_stream_set_batch_max_ts with
 * the global batch's max event time: then every shard advances the same
 * watermark (Section II-A's event-time windows close on the max event time
 * seen) and closes the same windows.  The union of the shards' rows of a
 * window is the single stream's; rows of one window are ordered by key (or by
 * the ORDER BY aggregate, equal values in key order) on each shard.
 *
 * key_mask selects the key bits every query of the stream groups by (the
 * fields common to all GROUP BYs; 0xffffffff without GROUP BY): rows whose
 * masked keys are equal land on one shard. */

/* Shard of a key: h = fmix32(key & key_mask) (MurmurHash3's 32-bit finaliser:
 * h ^= h >> 16; h *= 0x85ebca6b; h ^= h >> 13; h *= 0xc2b2ae35; h ^= h >> 16),
 * then (h * n_shards) >> 32 (multiply-shift range reduction).  n_shards >= 1. */
uint32_t lms_shard_of(uint32_t key, uint32_t key_mask, int32_t n_shards);

/* Splits the host batch `in` (n_rows rows, host columns) by lms_shard_of into
 * caller-owned host columns of in->n_rows rows each: shard g's rows, in their
 * input order, are rows [offsets[g], offsets[g+1]) of ts_out/key_out/value_out
 * (and type_out, which may be NULL when in->type is NULL); offsets has
 * n_shards + 1 entries.  *max_ts (may be NULL) receives the batch's max event
 * time (INT64_MIN if it is empty): the watermark hint for every shard.  Large
 * batches are split by up to 8 host threads.  Errors: LMS_EINVAL for NULL
 * pointers, n_shards < 1 or device columns. */
lms_status lms_shard_split(const lms_batch *in, uint32_t key_mask, int32_t n_shards,
                           int64_t *ts_out, uint32_t *key_out, uint32_t *value_out,
                           uint8_t *type_out, int64_t *offsets, int64_t *max_ts);

/* The next push (push_microbatch or lms_push_ingested) treats its batch's max
 * event time as at least ts (a watermark hint: the max over all shards of a
 * global micro-batch).  It applies to one push only, which then advances the
 * watermark even when it carries no rows. */
lms_status lms_stream_set_batch_max_ts(lms_stream *s, int64_t ts);

/* Fixes the event-time origin (what origin_ts of the configuration does)
 * before the first push; LMS_EINVAL once it is set. */
lms_status lms_stream_set_origin(lms_stream *s, int64_t origin_ts);

/* ---- snapshot / resume of a stream's device state ----
 *
 * Between pushes a stream's state is: its configuration and queries, the
 * event-time origin and watermark, every query's carried partial groups of
 * still-open panes (32 bytes each) and control block, and the rows not yet
 * polled (queries and joins).  lms_stream_snapshot writes all of it into a
 * host buffer (the state flushing / checkpoint step that follows each
 * micro-batch in Section III-E's processing cycle); lms_stream_restore opens a
 * new stream on `device` (-1: the snapshot's) in exactly that state, so that
 * pushing the rest of the input gives the rows the original stream would have.
 * The format is the library's own: a header with a magic and a version, then
 * per query and per join its spec, control block and arrays.  Not saved: the
 * cuda_stream of the configuration (the restored stream creates its own), a
 * variant chooser, the fused-pass autotuner's timings.  Snapshot: with buf
 * NULL only *size is set; LMS_EINVAL if cap < *size or ingested rows are
 * pending.  Restore: LMS_EINVAL for a buffer that is not a snapshot of this
 * library's format; LMS_ENOMEM / LMS_ECUDA as stream_open. */
lms_status lms_stream_snapshot(lms_stream *s, void *buf, size_t cap, size_t *size);
/* The stream's configuration (origin_ts as set, cuda_stream as in use). */
lms_status lms_stream_get_config(lms_stream *s, lms_stream_config *out);
lms_status lms_stream_restore(const void *buf, size_t size, int32_t device, lms_stream **out);

/* ---- control plane: dynamic micro-batching and per-operation planning ---- */

/* Alg. 1 policies.  PAPER: ConstructMicroBatch as printed (decides only when
 * new data arrived; admits when EstMaxLat >= target).  GUARDED: also
 * re-evaluates buffered data on every poll and admits when
 * EstMaxLat + poll period >= target. */
#define LMS_ADMIT_PAPER 0
#define LMS_ADMIT_GUARDED 1

/* Query operations of Table II, in this order (base costs 1.0 1.0 1.0 0.9 0.9
 * 0.9 0.8 0.8). */
#define LMS_QOP_AGGREGATION 0
#define LMS_QOP_FILTER 1
#define LMS_QOP_SHUFFLE 2
#define LMS_QOP_PROJECT 3
#define LMS_QOP_JOIN 4
#define LMS_QOP_EXPAND 5
#define LMS_QOP_SCAN 6
#define LMS_QOP_SORT 7

typedef struct lms_admission lms_admission; /* opaque, owned by the caller */

/* Predictor of a micro-batch's processing time (ms) from its bytes and
 * dataset count; replaces Eq. 5's bytes / AvgThPut term when installed. */
typedef double (*lms_proc_predictor)(void *ctx, double batch_bytes, int32_t n_datasets);

/* ConstructMicroBatch state (Section III-C, Alg. 1).  slide_ms > 0: sliding
 * window, target = SlideTime (Eq. 1); slide_ms == 0: tumbling, target = mean
 * of the past MaxLat (Eq. 2).  NULL for bad arguments. */
lms_admission *lms_admission_create(double slide_ms, int32_t policy, double poll_ms);
void lms_admission_destroy(lms_admission *a);
void lms_admission_set_predictor(lms_admission *a, lms_proc_predictor fn, void *ctx);

/* One poll of Alg. 1 at now_ms: n_new datasets (arrival time ms, bytes) arrived
 * since the previous poll.  Returns 1 if the buffered plus new datasets are
 * admitted as the next micro-batch (*n_admitted = their number), 0 if they
 * stay buffered, LMS_EINVAL for bad arguments.  *est_ms (optional) receives
 * EstMaxLat (Eq. 5) of the candidate batch. */
int32_t lms_admission_poll(lms_admission *a, double now_ms, const double *arrival_ms,
                           const double *bytes, int32_t n_new, double *est_ms,
                           int32_t *n_admitted);

/* The admitted micro-batch ran for proc_ms: records it in AvgThPut (Eq. 3) and
 * returns its MaxLat (Eq. 4); -1 if no batch was admitted. */
double lms_admission_complete(lms_admission *a, double proc_ms);
double lms_admission_avg_thput(const lms_admission *a);   /* Eq. 3, bytes/ms (0 before any) */
int32_t lms_admission_buffered(const lms_admission *a);   /* datasets still buffered */
double lms_admission_last_estimate(const lms_admission *a);

/* MapDevice (Alg. 2) over a chain of n_ops operations (ops[0] = leaf) with the
 * costs of Eqs. 6-8: partition = batch_bytes / num_cores.  device[o] receives
 * 0 (GPU) or 1 (CPU); cpu_cost / gpu_cost (optional) the costs after the
 * transition term was added.  This engine runs every operation on the GPU;
 * the plan is provided for callers that place operations themselves. */
lms_status lms_map_device(const int32_t *ops, int32_t n_ops, double batch_bytes,
                          int32_t num_cores, double infpt_bytes, double base_trans_cost,
                          int32_t *device, double *cpu_cost, double *gpu_cost);

/* Online regression of the inflection point (Section III-E, Eq. 9):
 * InfPT = b0 + b1 * Throughput + b2 * Latency by least squares over the last
 * history_len samples (0 = all).  fit() evaluates it at the targets and
 * returns LMS_EAGAIN (with b = (mean, 0, 0)) while fewer than 3 samples exist;
 * a singular system also gives b = (mean, 0, 0). */
typedef struct lms_regressor lms_regressor;
lms_regressor *lms_regressor_create(int32_t history_len);
void lms_regressor_destroy(lms_regressor *r);
void lms_regressor_add(lms_regressor *r, double thput, double lat, double infpt);
lms_status lms_regressor_fit(lms_regressor *r, double target_thput, double target_lat,
                             double *beta3, double *infpt);

/* ---- per-operation variant choice (Alg. 2 and Eq. 9 re-read) -------------
 *
 * The engine runs every operation on the GPU, so MapDevice's choice between a
 * CPU and a GPU implementation of an operation (Alg. 2, Eqs. 6-8) is re-read
 * as the choice between two implementations of the fused pass: variant 1
 * (1024-event tiles, two CTAs per SM; the paper's CPU side: its cost grows
 * with the partition) and variant 2 (2048-event tiles; the GPU side).  A
 * chooser is asked before every fused pass and, if it installs an observer,
 * told the pass's measured time afterwards. */
typedef int32_t (*lms_variant_chooser)(void *ctx, int64_t rows, int32_t n_queries);
typedef void (*lms_variant_observer)(void *ctx, int64_t rows, int32_t variant, double ms);
/* Installs (or with NULL removes) the chooser of s's fused-pass variant; it
 * takes precedence over cfg.k1_variant and the timing autotuner.  Results do
 * not depend on the variant. */
lms_status lms_stream_set_variant_chooser(lms_stream *s, lms_variant_chooser choose,
                                          lms_variant_observer observe, void *ctx);

/* The analytic chooser: Alg. 2 over the one-operation chain (Aggregation,
 * Table II base cost 1.0, transition base cost 0.1) with Part = batch bytes /
 * partitions (bytes_per_row each) and the current inflection point.  Each
 * variant is first tried `explore` times.  After each pass: the observed
 * inflection point is where the two variants' fitted costs (ms = c rows^b,
 * least squares on logs over each variant's latest 16 passes) cross, kept
 * within [1/2 smallest, 2 x largest] size seen; Eq. 9 is refitted on
 * (throughput = rows/ms, latency = ms, observed InfPT) over the last
 * history_len passes (0 = all) and evaluated at the targets (the largest
 * throughput seen, the mean latency) to give the next inflection point.
 * choose / observe have the chooser / observer signatures (ctx = the
 * chooser).  predict: a variant's fitted cost in ms at `rows` (< 0 if not
 * fitted yet).  state: the inflection point (bytes per partition) and the
 * picks of variants 1 and 2. */
typedef struct lms_variant_analytic lms_variant_analytic;
lms_variant_analytic *lms_variant_analytic_create(int32_t partitions, double bytes_per_row,
                                                  double infpt0_bytes, int32_t history_len,
                                                  int32_t explore);
void lms_variant_analytic_destroy(lms_variant_analytic *v);
int32_t lms_variant_analytic_choose(void *ctx, int64_t rows, int32_t n_queries);
void lms_variant_analytic_observe(void *ctx, int64_t rows, int32_t variant, double ms);
double lms_variant_analytic_predict(const lms_variant_analytic *v, int64_t rows, int32_t variant);
void lms_variant_analytic_state(const lms_variant_analytic *v, double *infpt_bytes,
                                int64_t *picks);

/* Keeps only the first n_keep datasets of the micro-batch Alg. 1 just admitted
 * (the caller re-offers the others as new datasets at its next poll); when
 * last_bytes > 0 it replaces the size of the last kept dataset (a dataset that
 * was split).  This is the serving loop's admission by memory, which the
 * paper does not have.  LMS_EINVAL if nothing is admitted or n_keep is out of
 * [1, admitted]. */
lms_status lms_admission_truncate(lms_admission *a, int32_t n_keep, double last_bytes);

/* ---- serving loop: dynamic micro-batching over an arrival process --------
 *
 * A virtual-clock loop (Section III-C's setting: datasets arrive every poll
 * period and ConstructMicroBatch decides when they form a micro-batch) whose
 * processing step is real: the backend runs each admitted micro-batch and
 * returns its measured processing time, which advances the clock.  Arrivals
 * are given as events per poll tick: tick t covers [t*poll_ms, (t+1)*poll_ms)
 * and becomes visible at its end; event j of a tick with n events arrives at
 * t*poll_ms + (j + 0.5) * poll_ms / n.  An event's latency is the completion
 * time of the micro-batch that processed it minus its arrival time (Eq. 4 per
 * event).  Decisions are taken at completions and on the poll grid. */
#define LMS_POLICY_FIXED_SIZE 0    /* admit exactly fixed_rows events once buffered */
#define LMS_POLICY_FIXED_TRIGGER 1 /* admit everything buffered every trigger_ms */
#define LMS_POLICY_ANALYTIC 2      /* Alg. 1 with Eq. 5 (target = latency bound) */
#define LMS_POLICY_LEARNED 3       /* Alg. 1 with the installed processing-time predictor */

/* One piece of a tick handed to the backend: events j_begin .. j_end-1 of a
 * tick starting at t0_ms with n_total events over width_ms; first_event is the
 * stream-wide index of the tick's event 0 (a counter for generators). */
typedef struct lms_serve_chunk {
  double t0_ms;
  double width_ms;
  int64_t n_total;
  int64_t j_begin;
  int64_t j_end;
  int64_t first_event;
} lms_serve_chunk;

/* Per micro-batch record of a serving run. */
typedef struct lms_serve_batch {
  double admit_ms;      /* virtual time the batch was admitted */
  double proc_ms;       /* processing time reported by the backend */
  double maxlat_ms;     /* completion - earliest arrival in the batch (Eq. 4) */
  double est_ms;        /* the policy's EstMaxLat at admission (0 for fixed policies) */
  double decide_ms;     /* wall time of the admission decision */
  int64_t n_events;
  int32_t n_chunks;
  int32_t forced;       /* 1: end-of-arrivals flush or memory cap forced the batch */
  /* filled by the backend, if it measures them: */
  double h2d_ms, k1_ms, sort_ms, emit_ms;
  uint64_t state_groups_before; /* window-state groups carried into the batch */
  uint64_t rows_out;            /* result rows the batch emitted */
} lms_serve_batch;

/* The processing side of a serving run.  process() runs one micro-batch made
 * of chunks[0 .. n_chunks) (n_events in all), fills what it measures in *rec,
 * and returns the processing time in ms (< 0: error, the run stops).
 * admissible_rows() (optional) returns the largest batch the backend can take
 * now (admission by memory), or < 0 for no limit. */
typedef struct lms_serve_backend {
  void *ctx;
  double (*process)(void *ctx, const lms_serve_chunk *chunks, int32_t n_chunks, int64_t n_events,
                    lms_serve_batch *rec);
  int64_t (*admissible_rows)(void *ctx);
  /* optional: called with each tick (j_begin = 0, j_end = n_total) when it
   * becomes visible, before any micro-batch that holds it is processed; an
   * ingest step that runs beside the loop (its wall time is reported as
   * arrive_ms and does not advance the clock).  Returns 0, or < 0 to stop the
   * run with LMS_EDEVICE. */
  int32_t (*arrive)(void *ctx, const lms_serve_chunk *tick);
} lms_serve_backend;

typedef struct lms_serve_config {
  int32_t policy;            /* LMS_POLICY_* */
  int32_t admit_rule;        /* LMS_ADMIT_PAPER or LMS_ADMIT_GUARDED (Alg. 1 policies) */
  int64_t fixed_rows;        /* FIXED_SIZE: events per micro-batch (> 0) */
  double trigger_ms;         /* FIXED_TRIGGER: period (> 0) */
  double latency_bound_ms;   /* p99 bound, and Alg. 1's target */
  double poll_ms;            /* tick length = Alg. 1's polling period (> 0) */
  double bytes_per_event;    /* dataset size = events * bytes_per_event (Alg. 1's Part) */
  int32_t add_decide_time;   /* 1: the decision's wall time also advances the clock */
  int32_t stop_when_missed;  /* 1: stop as soon as the p99 bound can no longer hold */
  double quantile_hi;        /* the tail quantile reported as p_hi (0.99) */
  int32_t reserved[8];
} lms_serve_config;

typedef struct lms_serve_result {
  int64_t offered_events;    /* sum of the tick counts */
  int64_t processed_events;
  int64_t batches;
  int32_t completed;         /* 1: every event was processed; 0: stopped early */
  int32_t met_bound;         /* completed and p_hi <= latency_bound_ms */
  double arrival_span_ms;    /* n_ticks * poll_ms */
  double end_ms;             /* virtual time of the last completion */
  double busy_ms;            /* sum of processing times */
  double p50_ms, p_hi_ms, mean_ms, max_ms;  /* per-event latency */
  double events_per_s;       /* processed_events / arrival span */
  int64_t max_backlog_events;
  double decide_ms;          /* wall time of all admission decisions */
  double observe_ms;         /* wall time the observer blocked the loop */
  double arrive_ms;          /* wall time of the backend's arrive() calls (not on the clock) */
} lms_serve_result;

/* Called after every micro-batch with its record (for example to train a
 * learned predictor online); returns the wall time in ms it blocked the loop,
 * which advances the clock when add_decide_time is set. */
typedef double (*lms_batch_observer)(void *ctx, const lms_serve_batch *rec);

/* Runs the loop over n_ticks ticks (tick_counts[t] events each) until every
 * event is processed (or, with stop_when_missed, until the bound is missed).
 * pred/pred_ctx: the predictor for LMS_POLICY_LEARNED (ignored otherwise);
 * observe (optional) is called with pred_ctx after each batch.
 * log (optional, log_cap entries) receives one record per micro-batch;
 * *n_log their number.  LMS_EINVAL for a bad config; the backend's error
 * stops the run with LMS_EDEVICE. */
lms_status lms_serve_run(const lms_serve_config *cfg, const int64_t *tick_counts, int64_t n_ticks,
                         const lms_serve_backend *backend, lms_proc_predictor pred,
                         void *pred_ctx, lms_batch_observer observe, lms_serve_result *out,
                         lms_serve_batch *log, size_t log_cap, size_t *n_log);

/* The engine as a serving backend (large float stream: value float32, no type
 * column).  It owns a stream opened with *cfg and the nq queries.  The load:
 * key Zipf(zipf_s) over n_keys keys and value lognormal(0, 1), drawn once for
 * a pool of 2^26 event counters (SplitMix64 under `seed`; event c of the stream
 * takes entry c mod 2^26), ts = floor(arrival ms) written per batch; all of it
 * outside the measured time.  Each micro-batch is processed as a client would:
 * push_microbatch, then poll_results of every row into pinned host memory; the
 * wall time of push + polls is the processing time.  Flags:
 * LMS_SERVE_DEVICE_INPUT keeps the columns in device memory (push reads them
 * in place); otherwise they are in pinned host memory and the host-to-device
 * copy is inside the measured time.  LMS_SERVE_KEEP_ROWS keeps every polled
 * row (lms_serve_gpu_kept_rows) for checks.  admissible_rows is
 * lms_stream_admissible_rows capped at max_batch_rows (<= 2^26).  Creation
 * warms the kernels up on a throwaway stream and reserves the stream's
 * buffers for the largest admissible batch. */
#define LMS_SERVE_KEEP_ROWS 1
#define LMS_SERVE_DEVICE_INPUT 2
#define LMS_SERVE_INGEST 4 /* host columns sent to the device as ticks arrive (lms_ingest), each
                              micro-batch pushed with lms_push_ingested (arrive() is set) */
typedef struct lms_serve_gpu lms_serve_gpu;
lms_status lms_serve_gpu_create(const lms_stream_config *cfg, const lms_query_spec *qs,
                                int32_t nq, uint64_t seed, uint32_t n_keys, double zipf_s,
                                int64_t max_batch_rows, int32_t flags, lms_serve_gpu **out);
lms_status lms_serve_gpu_backend(lms_serve_gpu *g, lms_serve_backend *out);
lms_stream *lms_serve_gpu_stream(lms_serve_gpu *g);
int32_t lms_serve_gpu_device_input(const lms_serve_gpu *g); /* 1 if created with LMS_SERVE_DEVICE_INPUT */
/* Brings the window state to steady state before a serving run: n_batches
 * micro-batches of events_per_batch events of the load, with event times
 * spread evenly over [t0_ms, t0_ms + span_ms), are pushed (as the backend's
 * input mode pushes) and their rows discarded; nothing is measured.  A run
 * whose arrivals start at t = 0 then finds the open panes of the last window
 * already full, as a stream that has been running for span_ms would.
 * events_per_batch <= the backend's max_batch_rows. */
lms_status lms_serve_gpu_prefill(lms_serve_gpu *g, double t0_ms, double span_ms,
                                 int32_t n_batches, int64_t events_per_batch);
/* Writes the events the backend would generate for these chunks into host
 * arrays (for checks against the oracle). */
lms_status lms_serve_gpu_generate(lms_serve_gpu *g, const lms_serve_chunk *chunks,
                                  int32_t n_chunks, int64_t n_events, int64_t *ts, uint32_t *key,
                                  float *value);
/* Copies up to cap kept rows of query_id (out == NULL: *n_out = how many). */
lms_status lms_serve_gpu_kept_rows(lms_serve_gpu *g, int32_t query_id, lms_result_row *out,
                                   size_t cap, size_t *n_out);
void lms_serve_gpu_destroy(lms_serve_gpu *g);

/* ---- learned cost model ------------------------------------------------
 *
 * A multilayer perceptron 8 -> 64 -> 64 -> 64 -> 1 (ReLU hidden layers,
 * linear output) that predicts ln(latency in microseconds) of one operator of
 * a micro-batch from the eight features of lms_cost_features.  The paper's
 * cost model is analytic (Eqs. 5-9); this one is trained on the engine's own
 * timings and, installed as Alg. 1's predictor, replaces Eq. 5's
 * bytes / AvgThPut term.  Master weights are FP32; forward and backward use
 * them rounded to bf16 (round to nearest even) with FP32 accumulation; the
 * loss is the mean squared error; training is Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8) on the GPU with the library's own kernels.
 *
 * Parameter vector (FP32, LMS_MLP_PARAMS entries, row-major W[out][in]):
 * W1[64][8], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4. */
#define LMS_MLP_INPUTS 8
#define LMS_MLP_HIDDEN 64
#define LMS_MLP_PARAMS 8961
#define LMS_MLP_MAX_BATCH 4096

typedef struct lms_mlp lms_mlp;
/* On `device` with the given initial parameters; NULL on failure. */
lms_mlp *lms_mlp_create(int32_t device, const float *params);
void lms_mlp_destroy(lms_mlp *m);
/* Replaces the master weights (and resets Adam's moments and step count). */
lms_status lms_mlp_set_params(lms_mlp *m, const float *params);
lms_status lms_mlp_get_params(lms_mlp *m, float *params);
/* y[i] = network(x[i*8 .. i*8+8)) for n host samples (GPU inference kernel). */
lms_status lms_mlp_forward(lms_mlp *m, const float *x, int32_t n, float *y);
/* `steps` Adam steps (learning rate lr) on the full batch of n <= 4096 host
 * samples (x [n][8], targets t [n]).  grad_out (optional, LMS_MLP_PARAMS) and
 * *loss_out (optional) receive the gradient and the loss of the last step's
 * forward pass, i.e. at the weights before its update; steps == 0 computes
 * them without updating. */
lms_status lms_mlp_train(lms_mlp *m, const float *x, const float *t, int32_t n, int32_t steps,
                         float lr, float *grad_out, float *loss_out);

/* Operators whose latency the model predicts, per micro-batch. */
#define LMS_OP_H2D 0   /* host-to-device copy of the batch */
#define LMS_OP_K1 1    /* fused filter / window / pre-aggregate pass */
#define LMS_OP_SORT 2  /* sort + reduce into window state */
#define LMS_OP_EMIT 3  /* window assembly, emission and carry */
#define LMS_OP_HOST 4  /* the rest of the processing time (launches, syncs, result copies) */
#define LMS_N_OPS 5
/* The fused pass run as variant v (1 or 2), for the learned variant chooser. */
#define LMS_OP_K1_VARIANT(v) (4 + (v))

/* The model's eight input features of operator `op` of a micro-batch:
 * log2(1+rows)/32, log2(1+carried state groups)/32, log2(key cardinality)/32,
 * filter selectivity, log2(panes per window)/12, queries/8,
 * log2(1 + event-time span in panes)/16, op/4. */
void lms_cost_features(double rows, double carried_groups, double key_card, double selectivity,
                       double panes_per_window, double n_queries, double span_panes, int32_t op,
                       float *out8);

/* Alg. 1 predictor backed by the network, with the paper's analytic estimate
 * (Eq. 5: bytes / AvgThPut of Eq. 3 over the batches it observed) as fallback
 * and judge.  A candidate batch has rows = bytes / bytes_per_event, an
 * event-time span of n_datasets * poll_ms, and the carried groups the serving
 * backend's stream holds now; the network's prediction is the sum over the
 * five operators of exp(output) us.  After each batch (lms_learned_observe, a
 * lms_batch_observer) both predictions of that batch are compared with its
 * measured time (moving average of |ln(predicted / measured)|); predict()
 * answers with Eq. 5 until the network has been fitted and whenever the
 * network's error is the larger.  Observed batches become training samples
 * (one per operator, ln of its time in us; "host" = the processing time not
 * covered by the four device phases) in a ring of the latest 4096 samples;
 * lms_learned_fit takes Adam steps on them, and with online refitting set,
 * observe() does so every refit_every batches (its wall time is returned to
 * the loop as blocking time).  set_backend() starts a serving run: it binds
 * the backend (whose stream's carried groups the features read, and whose
 * input mode decides whether the host-to-device copy is one of the operators)
 * and restarts Eq. 5's history and the judge's errors; the network and its
 * samples are kept.  A candidate larger than the backend's stream admits
 * (lms_stream_admissible_rows) is predicted as the capped batches it will
 * run as. */
typedef struct lms_learned lms_learned;
lms_learned *lms_learned_create(lms_mlp *m, lms_serve_gpu *g, double key_card,
                                double selectivity, double panes_per_window, double n_queries,
                                double slide_ms, double poll_ms, double bytes_per_event);
void lms_learned_destroy(lms_learned *l);
void lms_learned_set_backend(lms_learned *l, lms_serve_gpu *g);
void lms_learned_set_online(lms_learned *l, int32_t refit_every, int32_t refit_steps, float lr);
int32_t lms_learned_samples(const lms_learned *l);
lms_status lms_learned_fit(lms_learned *l, int32_t steps, float lr, float *loss);
double lms_learned_observe(void *learned, const lms_serve_batch *rec);
double lms_learned_predict(void *learned, double batch_bytes, int32_t n_datasets);
/* Judge's moving errors and how often each estimate answered. */
void lms_learned_stats(const lms_learned *l, double *err_net, double *err_eq5, int64_t *uses_net,
                       int64_t *uses_eq5);

/* Learned chooser of the fused pass's variant (see lms_variant_analytic): the
 * network m predicts ln(us) of the pass for each variant from the features of
 * lms_cost_features (rows, no carried groups, the stream's key cardinality,
 * selectivity, panes per window and queries, span 0, operator
 * LMS_OP_K1_VARIANT(v)); it picks the variant of the smaller prediction, and
 * every 16th pick the other one, so both stay measured.  The analytic chooser
 * `judge` (owned by the caller) answers while the network is untrained or
 * while its moving |ln(predicted / measured)| error is the larger of the two;
 * it also sees every measurement.  Measured passes become training samples
 * (a ring of LMS_MLP_MAX_BATCH); fit() trains on them, and with online
 * refitting on, observe() does so every refit_every passes.  choose / observe
 * have the chooser / observer signatures (ctx = the learned chooser). */
typedef struct lms_variant_learned lms_variant_learned;
lms_variant_learned *lms_variant_learned_create(lms_mlp *m, lms_variant_analytic *judge,
                                                double key_card, double selectivity,
                                                double panes_per_window, double n_queries);
void lms_variant_learned_destroy(lms_variant_learned *v);
void lms_variant_learned_set_online(lms_variant_learned *v, int32_t refit_every,
                                    int32_t refit_steps, float lr);
lms_status lms_variant_learned_fit(lms_variant_learned *v, int32_t steps, float lr, float *loss);
int32_t lms_variant_learned_choose(void *ctx, int64_t rows, int32_t n_queries);
void lms_variant_learned_observe(void *ctx, int64_t rows, int32_t variant, double ms);
void lms_variant_learned_stats(const lms_variant_learned *v, double *err_net, double *err_an,
                               int64_t *uses_net, int64_t *uses_an, int64_t *picks);

/* ---- continuous batching across streams --------------------------------
 *
 * A server with `slots` worker threads runs pushes of many streams at once on
 * one GPU: each worker takes the oldest queued request whose stream is not
 * already running and whose memory fits, and runs push_microbatch on that
 * stream's own CUDA stream, so micro-batches of different streams overlap on
 * the device while each stream's batches run one at a time in submission
 * order.  Admission by memory: a request starts only if the device bytes held
 * by every stream the server has seen, plus what the running requests and this
 * one may allocate (lms_stream_push_bytes), stay within memory_budget_bytes
 * (0 = no budget); otherwise it waits for a running request to finish, and
 * fails with LMS_ENOMEM if nothing is running.  Results are polled from each
 * stream as usual once its ticket has completed.  The paper has no
 * counterpart: it processes one query's micro-batches one after another.
 * Streams used with a server must have their own CUDA streams
 * (cfg.cuda_stream = NULL) and must not be pushed outside the server meanwhile;
 * the caller keeps every submitted batch's columns valid until its ticket
 * completes. */
typedef struct lms_server lms_server;
typedef struct lms_server_config {
  int32_t slots;                /* concurrent micro-batches (1..64) */
  int32_t reserved0;
  uint64_t memory_budget_bytes; /* device memory all streams may hold together, 0 = none */
  int32_t reserved[8];
} lms_server_config;
typedef struct lms_server_stats {
  int64_t submitted, completed, queued;
  int64_t max_concurrent;       /* most requests running at once */
  int64_t memory_waits;         /* times a worker found only requests that did not fit */
  uint64_t peak_bytes;          /* largest held + reserved device bytes at a completion */
  uint64_t held_bytes;          /* device bytes the known streams hold now */
  double busy_ms;               /* sum of request run times */
} lms_server_stats;
lms_status lms_server_create(const lms_server_config *cfg, lms_server **out);
/* The operations a server applies to streams; lms_server_create uses the
 * engine's (push_microbatch, lms_stream_push_bytes, lms_stream_device_bytes).
 * Other implementations serve to test the scheduling on the host. */
typedef struct lms_server_ops {
  void *ctx;
  lms_status (*push)(void *ctx, lms_stream *s, const lms_batch *b);
  lms_status (*push_bytes)(void *ctx, lms_stream *s, int64_t n_rows, int32_t host_input,
                           uint64_t *bytes);
  lms_status (*device_bytes)(void *ctx, lms_stream *s, uint64_t *bytes);
} lms_server_ops;
lms_status lms_server_create_ops(const lms_server_config *cfg, const lms_server_ops *ops,
                                 lms_server **out);
/* Queues a push of *b on s; *ticket identifies it.  Returns at once. */
lms_status lms_server_submit(lms_server *sv, lms_stream *s, const lms_batch *b, uint64_t *ticket);
/* Waits (timeout_ms < 0: without limit) for a ticket: *result = the push's
 * status; start_ms / end_ms (optional) = when it ran, ms since the server was
 * created.  LMS_ETIMEDOUT if it is not done in time (it can be waited again). */
lms_status lms_server_wait(lms_server *sv, uint64_t ticket, int32_t timeout_ms,
                           lms_status *result, double *start_ms, double *end_ms);
/* Stops counting a stream's memory (before closing it); LMS_EAGAIN while it
 * has queued or running requests. */
lms_status lms_server_forget(lms_server *sv, lms_stream *s);
lms_status lms_server_get_stats(lms_server *sv, lms_server_stats *out);
/* Runs every queued request, then stops the workers and frees the server. */
lms_status lms_server_destroy(lms_server *sv);

/* Largest n_rows lms_aggregate_batch_static accepts. */
#define LMS_STATIC_MAX_ROWS 131072

/* Allocation-free variant for callers that may not allocate device memory
 * (plug-ins hosted in a process that owns the device memory budget, serving
 * paths where allocation is forbidden).  The paper has no counterpart: it is
 * the stream API's hot path run once, as a whole stream, over one batch.
 *
 * Aggregates the n_rows events in device memory (ts, key, value, optional type)
 * for query q exactly as stream_open + query_register + one push_microbatch
 * with LMS_BATCH_EOS + poll_results would (same kernels, same rows, same
 * order), on the calling thread's current device and on cuda_stream (NULL:
 * the legacy default stream).  Rows go to the caller's DEVICE buffer
 * rows[0 .. rows_cap); *n_out receives their number.  The first row's ts is
 * the event-time origin.  Returns when the rows are written.
 *
 * Every intermediate buffer lives in one fixed array of about 34 MiB that the
 * library declares in device memory: it is present on every GPU that loads the
 * library until the process exits, and this function calls no cudaMalloc,
 * cudaFree or other allocating routine.  The first call on a device looks the
 * array up (cudaGetSymbolAddress).  Every call reads the first event time back
 * to the host and waits for cuda_stream, so no call may be made while any
 * stream is being captured into a CUDA graph.  All
 * calls share the array and leave their data in it; each call first resets the
 * parts that must start from zero.  Calls are serialised inside the library;
 * other work touching the array concurrently would race.
 *
 * The query's post-aggregation fields (group_fields, having_agg, order_agg)
 * must be 0.
 *
 * Errors: LMS_EINVAL for a bad argument or n_rows > LMS_STATIC_MAX_ROWS;
 * LMS_ENOMEM if the emission units (runs of up to 64 consecutive closed
 * windows, cut into pieces of about 32K state groups, or of about 1K when a
 * window spans at most 16 panes; at most 32768) or the
 * rows do not fit (rows_cap >= n_rows * size/slide always suffices);
 * LMS_ECUDA for a CUDA failure; LMS_EDEVICE for an internal kernel flag. */
lms_status lms_aggregate_batch_static(const lms_query_spec *q, int32_t value_type,
                                      const int64_t *ts, const uint32_t *key, const void *value,
                                      const uint8_t *type, int64_t n_rows, void *cuda_stream,
                                      lms_result_row *rows, size_t rows_cap, size_t *n_out);

/* The fused-pass variant the autotuner chose for batches of `rows` rows of a
 * stream with this value type and number of queries (process-wide; 1 below
 * 2^15 rows), or 0 while it is still timing the variants of that size class. */
int32_t lms_k1_tuned_variant(int32_t value_type, int32_t n_queries, int64_t rows);

#ifdef __cplusplus
}
#endif

#endif /* LMSTREAM_H */
