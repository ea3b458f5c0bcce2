"""Python binding of the C ABI in include/lmstream.h (argument marshalling only).

Every step of the hot path runs in the CUDA library `liblmstream.so` built
in-tree by `paper_2111_04289_b300.build`; this module only converts Python /
numpy / torch arguments into the C structs and pointers the ABI takes.  There
is no CPU fallback: if the library is missing, importing it raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

LMS_OK, LMS_EINVAL, LMS_ENOMEM, LMS_EAGAIN, LMS_ETIMEDOUT = 0, -1, -2, -3, -4
LMS_ECUDA, LMS_ECLOSED, LMS_ERANGE, LMS_EDEVICE = -5, -6, -7, -8
STATUS_NAMES = {0: "LMS_OK", -1: "LMS_EINVAL", -2: "LMS_ENOMEM", -3: "LMS_EAGAIN",
                -4: "LMS_ETIMEDOUT", -5: "LMS_ECUDA", -6: "LMS_ECLOSED", -7: "LMS_ERANGE",
                -8: "LMS_EDEVICE"}
VALUE_INT32, VALUE_FLOAT32 = 0, 1
COLS = {"ts": 0, "key": 1, "value": 2, "type": 3}
OPS = {"none": 0, "eq": 1, "ne": 2, "lt": 3, "le": 4, "gt": 5, "ge": 6}
AGG_COUNT, AGG_SUM, AGG_MIN, AGG_MAX, AGG_AVG, AGG_ALL = 1, 2, 4, 8, 16, 31
MEM_HOST, MEM_DEVICE = 0, 1
BATCH_EOS = 1
INGEST_STABLE = 2
GRAPH_DEFAULT, GRAPH_OFF, GRAPH_ON = 0, 1, 2
ORIGIN_AUTO = -(2 ** 63)

# numpy images of lms_result_row (48 bytes) for the two value types
ROW_DTYPE_INT = np.dtype([("window_start", "<i8"), ("count", "<i8"), ("sum", "<i8"),
                          ("avg", "<f8"), ("key", "<u4"), ("min", "<i4"), ("max", "<i4"),
                          ("query_id", "<u4")])
ROW_DTYPE_FLOAT = np.dtype([("window_start", "<i8"), ("count", "<i8"), ("sum", "<f8"),
                            ("avg", "<f8"), ("key", "<u4"), ("min", "<f4"), ("max", "<f4"),
                            ("query_id", "<u4")])


class StreamConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("value_type", ctypes.c_int32),
                ("has_type", ctypes.c_int32), ("enable_timing", ctypes.c_int32),
                ("allowed_lateness_ms", ctypes.c_int64), ("max_batch_rows", ctypes.c_int64),
                ("state_cap_bytes", ctypes.c_uint64), ("cuda_stream", ctypes.c_void_p),
                ("origin_ts", ctypes.c_int64), ("k1_variant", ctypes.c_int32),
                ("graph_mode", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("reserved1", ctypes.c_uint32), ("key_fields", ctypes.c_uint32),
                ("reserved", ctypes.c_int32 * 3)]




class QuerySpec(ctypes.Structure):
    _fields_ = [("filter_col", ctypes.c_int32), ("filter_op", ctypes.c_int32),
                ("filter_i", ctypes.c_int64), ("filter_f", ctypes.c_double),
                ("window_size_ms", ctypes.c_int64), ("window_slide_ms", ctypes.c_int64),
                ("agg_mask", ctypes.c_uint32), ("group_fields", ctypes.c_uint32),
                ("having_agg", ctypes.c_int32), ("having_op", ctypes.c_int32),
                ("having_value", ctypes.c_double), ("order_agg", ctypes.c_int32),
                ("order_desc", ctypes.c_int32)]


POST_AGGS = {"count": 1, "sum": 2, "min": 3, "max": 4, "avg": 5}
ORDER_MAX_ROWS = 16384


class JoinSpec(ctypes.Structure):
    _fields_ = [("window_size_ms", ctypes.c_int64), ("window_slide_ms", ctypes.c_int64),
                ("left_col", ctypes.c_int32), ("left_op", ctypes.c_int32),
                ("left_i", ctypes.c_int64), ("left_f", ctypes.c_double),
                ("right_col", ctypes.c_int32), ("right_op", ctypes.c_int32),
                ("right_i", ctypes.c_int64), ("right_f", ctypes.c_double)]


JOIN_ROW_DTYPE_INT = np.dtype([("window_start", "<i8"), ("pairs", "<i8"), ("left_count", "<i8"),
                               ("right_count", "<i8"), ("left_sum", "<i8"), ("right_sum", "<i8"),
                               ("key", "<u4"), ("join_id", "<u4")])
JOIN_ROW_DTYPE_FLOAT = np.dtype([("window_start", "<i8"), ("pairs", "<i8"),
                                 ("left_count", "<i8"), ("right_count", "<i8"),
                                 ("left_sum", "<f8"), ("right_sum", "<f8"), ("key", "<u4"),
                                 ("join_id", "<u4")])


class QueryStatsC(ctypes.Structure):
    _fields_ = [("sort_ms", ctypes.c_double), ("emit_count_ms", ctypes.c_double),
                ("emit_write_ms", ctypes.c_double), ("rows_emitted", ctypes.c_uint64),
                ("state_groups", ctypes.c_uint64)]


class BatchC(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("ts", ctypes.c_void_p), ("key", ctypes.c_void_p),
                ("value", ctypes.c_void_p), ("type", ctypes.c_void_p),
                ("memory", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("arrival_ns", ctypes.c_int64)]


class StatsC(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_uint64), ("events", ctypes.c_uint64),
                ("late_rows", ctypes.c_uint64), ("range_rows", ctypes.c_uint64),
                ("rows_emitted", ctypes.c_uint64), ("rows_pending", ctypes.c_uint64),
                ("watermark", ctypes.c_int64), ("state_groups", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("last_batch_ms", ctypes.c_double),
                ("k1_ms", ctypes.c_double), ("sort_ms", ctypes.c_double),
                ("emit_ms", ctypes.c_double), ("h2d_ms", ctypes.c_double),
                ("k1_launches", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("e1_ms", ctypes.c_double), ("e2_ms", ctypes.c_double),
                ("partials", ctypes.c_uint64), ("groups_built", ctypes.c_uint64),
                ("graph_launches", ctypes.c_uint64), ("graph_captures", ctypes.c_uint64),
                ("k1_tile_events", ctypes.c_uint64), ("autotune_samples", ctypes.c_uint64)]


EXPORTED_SYMBOLS = ("stream_open", "query_register", "push_microbatch", "poll_results",
                    "stream_close", "lms_stream_stats", "lms_last_error", "lms_results_device",
                    "lms_results_discard", "lms_udiv_invariant", "lms_aggregate_batch_static",
                    "lms_admission_create", "lms_admission_destroy", "lms_admission_set_predictor",
                    "lms_admission_poll", "lms_admission_complete", "lms_admission_avg_thput",
                    "lms_admission_buffered", "lms_admission_last_estimate", "lms_map_device",
                    "lms_regressor_create", "lms_regressor_destroy", "lms_regressor_add",
                    "lms_regressor_fit", "lms_admission_truncate", "lms_serve_run",
                    "lms_stream_admissible_rows", "lms_serve_gpu_create", "lms_serve_gpu_backend",
                    "lms_serve_gpu_stream", "lms_serve_gpu_generate", "lms_serve_gpu_kept_rows",
                    "lms_serve_gpu_destroy", "lms_stream_reserve", "lms_mlp_create",
                    "lms_mlp_destroy", "lms_mlp_set_params", "lms_mlp_get_params",
                    "lms_mlp_forward", "lms_mlp_train", "lms_cost_features",
                    "lms_learned_create", "lms_learned_destroy", "lms_learned_set_backend",
                    "lms_learned_set_online", "lms_learned_samples", "lms_learned_fit",
                    "lms_learned_observe", "lms_learned_predict", "lms_learned_stats",
                    "lms_serve_gpu_device_input", "lms_stream_push_bytes",
                    "lms_stream_device_bytes", "lms_server_create", "lms_server_submit",
                    "lms_server_wait", "lms_server_forget", "lms_server_get_stats",
                    "lms_server_destroy", "lms_server_create_ops", "lms_k1_tuned_variant",
                    "lms_ingest", "lms_push_ingested", "lms_ingest_pending",
                    "lms_stream_set_variant_chooser", "lms_variant_analytic_create",
                    "lms_variant_analytic_destroy", "lms_variant_analytic_choose",
                    "lms_variant_analytic_observe", "lms_variant_analytic_predict",
                    "lms_variant_analytic_state", "lms_variant_learned_create",
                    "lms_variant_learned_destroy", "lms_variant_learned_set_online",
                    "lms_variant_learned_fit", "lms_variant_learned_choose",
                    "lms_variant_learned_observe", "lms_variant_learned_stats",
                    "lms_join_register", "lms_join_poll", "lms_shard_of", "lms_shard_split",
                    "lms_stream_set_batch_max_ts", "lms_stream_set_origin",
                    "lms_stream_snapshot", "lms_stream_restore", "lms_stream_get_config",
                    "lms_serve_gpu_prefill", "lms_query_stats")
ADMIT_PAPER, ADMIT_GUARDED = 0, 1
QOPS = {"aggregation": 0, "filter": 1, "shuffle": 2, "project": 3, "join": 4, "expand": 5,
        "scan": 6, "sort": 7}
PROC_PREDICTOR = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_void_p, ctypes.c_double, ctypes.c_int32)
POLICY_FIXED_SIZE, POLICY_FIXED_TRIGGER, POLICY_ANALYTIC, POLICY_LEARNED = 0, 1, 2, 3


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("memory_budget_bytes", ctypes.c_uint64), ("reserved", ctypes.c_int32 * 8)]


SERVER_PUSH = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.POINTER(BatchC))
SERVER_PUSH_BYTES = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_uint64))
SERVER_DEVICE_BYTES = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_uint64))


class ServerOps(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("push", ctypes.c_void_p),
                ("push_bytes", ctypes.c_void_p), ("device_bytes", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("max_concurrent", ctypes.c_int64),
                ("memory_waits", ctypes.c_int64), ("peak_bytes", ctypes.c_uint64),
                ("held_bytes", ctypes.c_uint64), ("busy_ms", ctypes.c_double)]


class ServeChunk(ctypes.Structure):
    _fields_ = [("t0_ms", ctypes.c_double), ("width_ms", ctypes.c_double),
                ("n_total", ctypes.c_int64), ("j_begin", ctypes.c_int64),
                ("j_end", ctypes.c_int64), ("first_event", ctypes.c_int64)]


class ServeBatch(ctypes.Structure):
    _fields_ = [("admit_ms", ctypes.c_double), ("proc_ms", ctypes.c_double),
                ("maxlat_ms", ctypes.c_double), ("est_ms", ctypes.c_double),
                ("decide_ms", ctypes.c_double), ("n_events", ctypes.c_int64),
                ("n_chunks", ctypes.c_int32), ("forced", ctypes.c_int32),
                ("h2d_ms", ctypes.c_double), ("k1_ms", ctypes.c_double),
                ("sort_ms", ctypes.c_double), ("emit_ms", ctypes.c_double),
                ("state_groups_before", ctypes.c_uint64), ("rows_out", ctypes.c_uint64)]


SERVE_PROCESS = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ServeChunk),
                                 ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ServeBatch))
SERVE_ADMISSIBLE = ctypes.CFUNCTYPE(ctypes.c_int64, ctypes.c_void_p)


class ServeBackend(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("process", ctypes.c_void_p),
                ("admissible_rows", ctypes.c_void_p), ("arrive", ctypes.c_void_p)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("policy", ctypes.c_int32), ("admit_rule", ctypes.c_int32),
                ("fixed_rows", ctypes.c_int64), ("trigger_ms", ctypes.c_double),
                ("latency_bound_ms", ctypes.c_double), ("poll_ms", ctypes.c_double),
                ("bytes_per_event", ctypes.c_double), ("add_decide_time", ctypes.c_int32),
                ("stop_when_missed", ctypes.c_int32), ("quantile_hi", ctypes.c_double),
                ("reserved", ctypes.c_int32 * 8)]


class ServeResult(ctypes.Structure):
    _fields_ = [("offered_events", ctypes.c_int64), ("processed_events", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("completed", ctypes.c_int32),
                ("met_bound", ctypes.c_int32), ("arrival_span_ms", ctypes.c_double),
                ("end_ms", ctypes.c_double), ("busy_ms", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p_hi_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("events_per_s", ctypes.c_double), ("max_backlog_events", ctypes.c_int64),
                ("decide_ms", ctypes.c_double), ("observe_ms", ctypes.c_double),
                ("arrive_ms", ctypes.c_double)]
STATIC_MAX_ROWS = 131072

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads liblmstream.so (building it first if asked); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"CUDA engine library not built: {_build.LIB}")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    P = ctypes.c_void_p
    lib.stream_open.restype = ctypes.c_int32
    lib.stream_open.argtypes = [ctypes.POINTER(StreamConfig), ctypes.POINTER(P)]
    lib.query_register.restype = ctypes.c_int32
    lib.query_register.argtypes = [P, ctypes.POINTER(QuerySpec), ctypes.POINTER(ctypes.c_int32)]
    lib.push_microbatch.restype = ctypes.c_int32
    lib.push_microbatch.argtypes = [P, ctypes.POINTER(BatchC)]
    lib.poll_results.restype = ctypes.c_int32
    lib.poll_results.argtypes = [P, ctypes.c_int32, P, ctypes.c_size_t,
                                 ctypes.POINTER(ctypes.c_size_t), ctypes.c_int32]
    lib.stream_close.restype = ctypes.c_int32
    lib.stream_close.argtypes = [P]
    lib.lms_stream_stats.restype = ctypes.c_int32
    lib.lms_stream_stats.argtypes = [P, ctypes.POINTER(StatsC)]
    lib.lms_last_error.restype = ctypes.c_char_p
    lib.lms_last_error.argtypes = [P]
    lib.lms_results_device.restype = ctypes.c_int32
    lib.lms_results_device.argtypes = [P, ctypes.c_int32, ctypes.POINTER(P),
                                       ctypes.POINTER(ctypes.c_size_t)]
    lib.lms_results_discard.restype = ctypes.c_int32
    lib.lms_results_discard.argtypes = [P, ctypes.c_int32]
    lib.lms_udiv_invariant.restype = ctypes.c_uint64
    lib.lms_udiv_invariant.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.lms_ingest.restype = ctypes.c_int32
    lib.lms_ingest.argtypes = [P, P]
    lib.lms_push_ingested.restype = ctypes.c_int32
    lib.lms_push_ingested.argtypes = [P, ctypes.c_int64, ctypes.c_uint32]
    lib.lms_ingest_pending.restype = ctypes.c_int32
    lib.lms_ingest_pending.argtypes = [P, P]
    lib.lms_join_register.restype = ctypes.c_int32
    lib.lms_join_register.argtypes = [P, P, P]
    lib.lms_join_poll.restype = ctypes.c_int32
    lib.lms_join_poll.argtypes = [P, ctypes.c_int32, P, ctypes.c_size_t, P]
    lib.lms_stream_set_variant_chooser.restype = ctypes.c_int32
    lib.lms_stream_set_variant_chooser.argtypes = [P, P, P, P]
    lib.lms_shard_of.restype = ctypes.c_uint32
    lib.lms_shard_of.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32]
    lib.lms_shard_split.restype = ctypes.c_int32
    lib.lms_shard_split.argtypes = [P, ctypes.c_uint32, ctypes.c_int32, P, P, P, P, P, P]
    lib.lms_stream_set_batch_max_ts.restype = ctypes.c_int32
    lib.lms_stream_set_batch_max_ts.argtypes = [P, ctypes.c_int64]
    lib.lms_stream_set_origin.restype = ctypes.c_int32
    lib.lms_stream_set_origin.argtypes = [P, ctypes.c_int64]
    lib.lms_stream_snapshot.restype = ctypes.c_int32
    lib.lms_stream_snapshot.argtypes = [P, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    lib.lms_stream_restore.restype = ctypes.c_int32
    lib.lms_stream_restore.argtypes = [P, ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(P)]
    lib.lms_stream_get_config.restype = ctypes.c_int32
    lib.lms_stream_get_config.argtypes = [P, ctypes.POINTER(StreamConfig)]
    lib.lms_variant_analytic_create.restype = P
    lib.lms_variant_analytic_create.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_int32, ctypes.c_int32]
    lib.lms_variant_analytic_destroy.argtypes = [P]
    lib.lms_variant_analytic_choose.restype = ctypes.c_int32
    lib.lms_variant_analytic_choose.argtypes = [P, ctypes.c_int64, ctypes.c_int32]
    lib.lms_variant_analytic_observe.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_double]
    lib.lms_variant_analytic_predict.restype = ctypes.c_double
    lib.lms_variant_analytic_predict.argtypes = [P, ctypes.c_int64, ctypes.c_int32]
    lib.lms_variant_analytic_state.argtypes = [P, P, P]
    lib.lms_variant_learned_create.restype = P
    lib.lms_variant_learned_create.argtypes = [P, P, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double]
    lib.lms_variant_learned_destroy.argtypes = [P]
    lib.lms_variant_learned_set_online.argtypes = [P, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_float]
    lib.lms_variant_learned_fit.restype = ctypes.c_int32
    lib.lms_variant_learned_fit.argtypes = [P, ctypes.c_int32, ctypes.c_float, P]
    lib.lms_variant_learned_choose.restype = ctypes.c_int32
    lib.lms_variant_learned_choose.argtypes = [P, ctypes.c_int64, ctypes.c_int32]
    lib.lms_variant_learned_observe.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_double]
    lib.lms_variant_learned_stats.argtypes = [P, P, P, P, P, P]
    lib.lms_aggregate_batch_static.restype = ctypes.c_int32
    lib.lms_aggregate_batch_static.argtypes = [
        ctypes.POINTER(QuerySpec), ctypes.c_int32, P, P, P, P, ctypes.c_int64, P, P,
        ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    D, I = ctypes.c_double, ctypes.c_int32
    lib.lms_admission_create.restype = P
    lib.lms_admission_create.argtypes = [D, I, D]
    lib.lms_admission_destroy.argtypes = [P]
    lib.lms_admission_set_predictor.argtypes = [P, P, P]
    lib.lms_admission_poll.restype = I
    lib.lms_admission_poll.argtypes = [P, D, P, P, I, ctypes.POINTER(D), ctypes.POINTER(I)]
    lib.lms_admission_complete.restype = D
    lib.lms_admission_complete.argtypes = [P, D]
    lib.lms_admission_avg_thput.restype = D
    lib.lms_admission_avg_thput.argtypes = [P]
    lib.lms_admission_buffered.restype = I
    lib.lms_admission_buffered.argtypes = [P]
    lib.lms_admission_last_estimate.restype = D
    lib.lms_admission_last_estimate.argtypes = [P]
    lib.lms_map_device.restype = I
    lib.lms_map_device.argtypes = [P, I, D, I, D, D, P, P, P]
    lib.lms_regressor_create.restype = P
    lib.lms_regressor_create.argtypes = [I]
    lib.lms_regressor_destroy.argtypes = [P]
    lib.lms_regressor_add.argtypes = [P, D, D, D]
    lib.lms_regressor_fit.restype = I
    lib.lms_regressor_fit.argtypes = [P, D, D, P, ctypes.POINTER(D)]
    lib.lms_admission_truncate.restype = I
    lib.lms_admission_truncate.argtypes = [P, I, D]
    lib.lms_serve_run.restype = I
    lib.lms_serve_run.argtypes = [ctypes.POINTER(ServeConfig), P, ctypes.c_int64,
                                  ctypes.POINTER(ServeBackend), P, P, P,
                                  ctypes.POINTER(ServeResult), P, ctypes.c_size_t,
                                  ctypes.POINTER(ctypes.c_size_t)]
    F = ctypes.c_float
    lib.lms_mlp_create.restype = P
    lib.lms_mlp_create.argtypes = [I, P]
    lib.lms_mlp_destroy.argtypes = [P]
    lib.lms_mlp_set_params.restype = I
    lib.lms_mlp_set_params.argtypes = [P, P]
    lib.lms_mlp_get_params.restype = I
    lib.lms_mlp_get_params.argtypes = [P, P]
    lib.lms_mlp_forward.restype = I
    lib.lms_mlp_forward.argtypes = [P, P, I, P]
    lib.lms_mlp_train.restype = I
    lib.lms_mlp_train.argtypes = [P, P, P, I, I, F, P, ctypes.POINTER(F)]
    lib.lms_cost_features.restype = None
    lib.lms_cost_features.argtypes = [D, D, D, D, D, D, D, I, P]
    lib.lms_learned_create.restype = P
    lib.lms_learned_create.argtypes = [P, P, D, D, D, D, D, D, D]
    lib.lms_learned_destroy.argtypes = [P]
    lib.lms_learned_set_backend.argtypes = [P, P]
    lib.lms_learned_set_online.argtypes = [P, I, I, F]
    lib.lms_learned_samples.restype = I
    lib.lms_learned_samples.argtypes = [P]
    lib.lms_learned_fit.restype = I
    lib.lms_learned_fit.argtypes = [P, I, F, ctypes.POINTER(F)]
    lib.lms_learned_observe.restype = D
    lib.lms_learned_observe.argtypes = [P, P]
    lib.lms_learned_predict.restype = D
    lib.lms_learned_predict.argtypes = [P, D, I]
    lib.lms_learned_stats.restype = None
    lib.lms_learned_stats.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(D),
                                      ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64)]
    lib.lms_stream_reserve.restype = I
    lib.lms_stream_reserve.argtypes = [P, ctypes.c_int64, I]
    lib.lms_stream_admissible_rows.restype = I
    lib.lms_stream_admissible_rows.argtypes = [P, I, ctypes.POINTER(ctypes.c_int64)]
    lib.lms_serve_gpu_create.restype = I
    lib.lms_serve_gpu_create.argtypes = [ctypes.POINTER(StreamConfig), P, I, ctypes.c_uint64,
                                         ctypes.c_uint32, D, ctypes.c_int64, I, ctypes.POINTER(P)]
    lib.lms_serve_gpu_backend.restype = I
    lib.lms_serve_gpu_backend.argtypes = [P, ctypes.POINTER(ServeBackend)]
    lib.lms_stream_push_bytes.restype = I
    lib.lms_stream_push_bytes.argtypes = [P, ctypes.c_int64, I, ctypes.POINTER(ctypes.c_uint64)]
    lib.lms_stream_device_bytes.restype = I
    lib.lms_stream_device_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_uint64)]
    lib.lms_server_create.restype = I
    lib.lms_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(P)]
    lib.lms_k1_tuned_variant.restype = I
    lib.lms_k1_tuned_variant.argtypes = [I, I, ctypes.c_int64]
    lib.lms_server_create_ops.restype = I
    lib.lms_server_create_ops.argtypes = [ctypes.POINTER(ServerConfig),
                                          ctypes.POINTER(ServerOps), ctypes.POINTER(P)]
    lib.lms_server_submit.restype = I
    lib.lms_server_submit.argtypes = [P, P, ctypes.POINTER(BatchC),
                                      ctypes.POINTER(ctypes.c_uint64)]
    lib.lms_server_wait.restype = I
    lib.lms_server_wait.argtypes = [P, ctypes.c_uint64, I, ctypes.POINTER(I), ctypes.POINTER(D),
                                    ctypes.POINTER(D)]
    lib.lms_server_forget.restype = I
    lib.lms_server_forget.argtypes = [P, P]
    lib.lms_server_get_stats.restype = I
    lib.lms_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
    lib.lms_server_destroy.restype = I
    lib.lms_server_destroy.argtypes = [P]
    lib.lms_serve_gpu_device_input.restype = I
    lib.lms_serve_gpu_device_input.argtypes = [P]
    lib.lms_serve_gpu_stream.restype = P
    lib.lms_serve_gpu_stream.argtypes = [P]
    lib.lms_serve_gpu_prefill.restype = I
    lib.lms_serve_gpu_prefill.argtypes = [P, D, D, I, ctypes.c_int64]
    lib.lms_query_stats.restype = I
    lib.lms_query_stats.argtypes = [P, I, ctypes.POINTER(QueryStatsC)]
    lib.lms_serve_gpu_generate.restype = I
    lib.lms_serve_gpu_generate.argtypes = [P, P, I, ctypes.c_int64, P, P, P]
    lib.lms_serve_gpu_kept_rows.restype = I
    lib.lms_serve_gpu_kept_rows.argtypes = [P, I, P, ctypes.c_size_t,
                                            ctypes.POINTER(ctypes.c_size_t)]
    lib.lms_serve_gpu_destroy.argtypes = [P]
    _lib = lib
    return lib


class LmsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr_and_mem(x):
    """(address, memory kind, keepalive) of a numpy array or torch tensor column."""
    if x is None:
        return None, None, None
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x)
        return x.ctypes.data, MEM_HOST, x
    # torch tensor
    if not x.is_contiguous():
        x = x.contiguous()
    return x.data_ptr(), (MEM_DEVICE if x.is_cuda else MEM_HOST), x


class Stream:
    """One engine stream: register queries, push micro-batches, poll rows."""

    def __init__(self, value_type: str = "int32", has_type: bool = False, device: int = 0,
                 allowed_lateness_ms: int = 0, max_batch_rows: int = 0, state_cap_bytes: int = 0,
                 cuda_stream: Optional[int] = None, origin_ts: Optional[int] = None,
                 enable_timing: bool = False, k1_variant: int = 0, graph_mode: int = 0,
                 key_fields=None):
        self._lib = load()
        self.value_type = value_type
        self.is_float = value_type == "float32"
        cfg = StreamConfig()
        cfg.device = device
        cfg.value_type = VALUE_FLOAT32 if self.is_float else VALUE_INT32
        cfg.has_type = int(bool(has_type))
        cfg.enable_timing = int(bool(enable_timing))
        cfg.allowed_lateness_ms = int(allowed_lateness_ms)
        cfg.max_batch_rows = int(max_batch_rows)
        cfg.state_cap_bytes = int(state_cap_bytes)
        cfg.cuda_stream = cuda_stream
        cfg.origin_ts = ORIGIN_AUTO if origin_ts is None else int(origin_ts)
        cfg.k1_variant = int(k1_variant)
        cfg.graph_mode = int(graph_mode)
        # key_fields: bit widths of up to four packed key fields (field 0 lowest)
        cfg.key_fields = sum(int(w) << (8 * f) for f, w in enumerate(key_fields or ()))
        h = ctypes.c_void_p()
        st = self._lib.stream_open(ctypes.byref(cfg), ctypes.byref(h))
        if st != LMS_OK:
            raise LmsError(st, "stream_open failed")
        self._h = h
        self.has_type = bool(has_type)
        self.row_dtype = ROW_DTYPE_FLOAT if self.is_float else ROW_DTYPE_INT
        self.queries = []
        self._ingest_keep = []

    def _check(self, st: int, what: str):
        if st != LMS_OK:
            msg = self._lib.lms_last_error(self._h)
            raise LmsError(st, f"{what}: {msg.decode() if msg else ''}")

    def register_query(self, size_ms: int, slide_ms: int = 0, filter_col: str = "ts",
                       filter_op: str = "none", filter_value=0, agg_mask: int = AGG_ALL,
                       group_fields: int = 0, having=None, order_by=None) -> int:
        """having = (agg, op, value): keep rows with (double)agg OP value;
        order_by = (agg, descending): each window's rows sorted by agg (ties in
        key order); group_fields: bit mask of the stream's key fields."""
        q = QuerySpec()
        q.filter_col = COLS[filter_col]
        q.filter_op = OPS[filter_op]
        if filter_col == "value" and self.is_float:
            q.filter_f = float(filter_value)
        else:
            q.filter_i = int(filter_value)
        q.window_size_ms = int(size_ms)
        q.window_slide_ms = int(slide_ms)
        q.agg_mask = int(agg_mask)
        q.group_fields = int(group_fields)
        if having is not None:
            q.having_agg, q.having_op, q.having_value = (POST_AGGS[having[0]], OPS[having[1]],
                                                         float(having[2]))
        if order_by is not None:
            q.order_agg, q.order_desc = POST_AGGS[order_by[0]], int(bool(order_by[1]))
        qid = ctypes.c_int32()
        self._check(self._lib.query_register(self._h, ctypes.byref(q), ctypes.byref(qid)),
                    "query_register")
        self.queries.append((size_ms, slide_ms or size_ms))
        return qid.value

    def make_batch(self, ts, key, value, type_=None, eos: bool = False, arrival_ns: int = 0):
        """(lms_batch, keepalive objects) for the given columns."""
        pt, mem, k0 = _ptr_and_mem(ts)
        pk, mk, k1 = _ptr_and_mem(key)
        pv, mv, k2 = _ptr_and_mem(value)
        py, my, k3 = _ptr_and_mem(type_ if self.has_type else None)
        if len({m for m in (mem, mk, mv, my) if m is not None}) > 1:
            raise ValueError("all columns of a batch must live in the same memory")
        b = BatchC()
        b.n_rows = int(ts.shape[0])
        b.ts, b.key, b.value, b.type = pt, pk, pv, py
        b.memory = MEM_HOST if mem is None else mem
        b.flags = BATCH_EOS if eos else 0
        b.arrival_ns = int(arrival_ns)
        return b, (k0, k1, k2, k3)

    def push(self, ts, key, value, type_=None, eos: bool = False, arrival_ns: int = 0) -> int:
        """Pushes one micro-batch (numpy host arrays or torch host/device tensors)."""
        b, keep = self.make_batch(ts, key, value, type_, eos, arrival_ns)
        st = self._lib.push_microbatch(self._h, ctypes.byref(b))
        del keep
        self._check(st, "push_microbatch")
        return int(b.n_rows)

    def ingest(self, ts, key, value, type_=None, stable: bool = False) -> int:
        """lms_ingest of one arriving dataset (host numpy arrays or pinned torch
        tensors); with stable=True the columns must stay unchanged until the
        push_ingested that covers them returns."""
        b, keep = self.make_batch(ts, key, value, type_)
        if b.memory != MEM_HOST:
            raise ValueError("lms_ingest takes host columns")
        b.flags = INGEST_STABLE if stable else 0
        st = self._lib.lms_ingest(self._h, ctypes.byref(b))
        if stable:
            self._ingest_keep.append(keep)
        del keep
        self._check(st, "lms_ingest")
        return int(b.n_rows)

    def push_ingested(self, n_rows: int, eos: bool = False) -> int:
        """lms_push_ingested: the oldest n_rows ingested rows as one micro-batch."""
        st = self._lib.lms_push_ingested(self._h, int(n_rows), BATCH_EOS if eos else 0)
        self._check(st, "lms_push_ingested")
        if self.ingest_pending() == 0:
            self._ingest_keep = []
        return int(n_rows)

    def ingest_pending(self) -> int:
        n = ctypes.c_int64()
        self._check(self._lib.lms_ingest_pending(self._h, ctypes.byref(n)), "lms_ingest_pending")
        return n.value

    def register_join(self, size_ms: int, slide_ms: int = 0, left=("ts", "none", 0),
                      right=("ts", "none", 0)) -> int:
        """lms_join_register: left / right = (column, op, value) side predicates."""
        j = JoinSpec()
        j.window_size_ms, j.window_slide_ms = int(size_ms), int(slide_ms)
        for side, (col, op, v) in (("left", left), ("right", right)):
            setattr(j, side + "_col", COLS[col])
            setattr(j, side + "_op", OPS[op])
            if col == "value" and self.is_float:
                setattr(j, side + "_f", float(v))
            else:
                setattr(j, side + "_i", int(v))
        jid = ctypes.c_int32()
        self._check(self._lib.lms_join_register(self._h, ctypes.byref(j), ctypes.byref(jid)),
                    "lms_join_register")
        return jid.value

    def poll_join(self, join_id: int, chunk: int = 1 << 20) -> np.ndarray:
        """All pending rows of a join (lms_join_poll), oldest first."""
        dt = JOIN_ROW_DTYPE_FLOAT if self.is_float else JOIN_ROW_DTYPE_INT
        parts = []
        while True:
            out = np.zeros(chunk, dtype=dt)
            got = ctypes.c_size_t()
            st = self._lib.lms_join_poll(self._h, int(join_id), out.ctypes.data, chunk,
                                         ctypes.byref(got))
            if st == LMS_EAGAIN:
                break
            self._check(st, "lms_join_poll")
            parts.append(out[: got.value])
            if got.value < chunk:
                break
        return np.concatenate(parts) if parts else np.zeros(0, dtype=dt)

    def set_batch_max_ts(self, ts: int) -> None:
        """Watermark hint for the next push (lms_stream_set_batch_max_ts)."""
        self._check(self._lib.lms_stream_set_batch_max_ts(self._h, int(ts)),
                    "lms_stream_set_batch_max_ts")

    def set_origin(self, origin_ts: int) -> None:
        self._check(self._lib.lms_stream_set_origin(self._h, int(origin_ts)),
                    "lms_stream_set_origin")

    def snapshot(self) -> bytes:
        """lms_stream_snapshot: the stream's state as bytes."""
        n = ctypes.c_size_t()
        self._check(self._lib.lms_stream_snapshot(self._h, None, 0, ctypes.byref(n)),
                    "lms_stream_snapshot")
        buf = ctypes.create_string_buffer(max(1, n.value))
        self._check(self._lib.lms_stream_snapshot(self._h, buf, n.value, ctypes.byref(n)),
                    "lms_stream_snapshot")
        return buf.raw[: n.value]

    @classmethod
    def restore(cls, blob: bytes, device: int = -1) -> "Stream":
        """lms_stream_restore: a new stream in the state a snapshot holds."""
        lib = load()
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        st = lib.lms_stream_restore(buf, len(blob), int(device), ctypes.byref(h))
        if st != LMS_OK:
            raise LmsError(st, "lms_stream_restore failed")
        self = cls.__new__(cls)
        self._lib = lib
        self._h = h
        cfg = StreamConfig()
        self._check(lib.lms_stream_get_config(h, ctypes.byref(cfg)), "lms_stream_get_config")
        self.value_type = "float32" if cfg.value_type == VALUE_FLOAT32 else "int32"
        self.is_float = cfg.value_type == VALUE_FLOAT32
        self.has_type = bool(cfg.has_type)
        self.row_dtype = ROW_DTYPE_FLOAT if self.is_float else ROW_DTYPE_INT
        self.queries = []
        self._ingest_keep = []
        return self

    def set_variant_chooser(self, chooser) -> None:
        """Installs a VariantAnalytic / VariantLearned (or None) as the chooser of
        the fused pass's variant."""
        self._chooser = chooser
        hooks = (None, None, None) if chooser is None else chooser.hooks()
        self._check(self._lib.lms_stream_set_variant_chooser(self._h, *hooks),
                    "lms_stream_set_variant_chooser")

    def poll(self, qid: int, max_rows: Optional[int] = None) -> np.ndarray:
        """All (or up to max_rows) pending rows of query qid, oldest first."""
        avail = self.pending(qid)
        m = avail if max_rows is None else min(avail, max_rows)
        out = np.zeros(m, dtype=self.row_dtype)
        if m == 0:
            return out
        got = ctypes.c_size_t()
        st = self._lib.poll_results(self._h, qid, out.ctypes.data, m, ctypes.byref(got), 0)
        self._check(st, "poll_results")
        return out[: got.value]

    def poll_into(self, qid: int, out_ptr: int, cap: int) -> int:
        """poll_results into a caller buffer (e.g. pinned memory); returns rows copied."""
        got = ctypes.c_size_t()
        st = self._lib.poll_results(self._h, qid, out_ptr, cap, ctypes.byref(got), 0)
        if st == LMS_EAGAIN:
            return 0
        self._check(st, "poll_results")
        return got.value

    def pending(self, qid: int) -> int:
        p = ctypes.c_void_p()
        n = ctypes.c_size_t()
        self._check(self._lib.lms_results_device(self._h, qid, ctypes.byref(p), ctypes.byref(n)),
                    "lms_results_device")
        return n.value

    def results_device(self, qid: int):
        p = ctypes.c_void_p()
        n = ctypes.c_size_t()
        self._check(self._lib.lms_results_device(self._h, qid, ctypes.byref(p), ctypes.byref(n)),
                    "lms_results_device")
        return p.value, n.value

    def discard(self, qid: int):
        self._check(self._lib.lms_results_discard(self._h, qid), "lms_results_discard")

    def stats(self) -> dict:
        s = StatsC()
        self._check(self._lib.lms_stream_stats(self._h, ctypes.byref(s)), "lms_stream_stats")
        return {name: getattr(s, name) for name, _ in StatsC._fields_}

    def query_stats(self, qid: int) -> dict:
        """lms_query_stats: the query's share of the batch work."""
        s = QueryStatsC()
        self._check(self._lib.lms_query_stats(self._h, int(qid), ctypes.byref(s)),
                    "lms_query_stats")
        return {name: getattr(s, name) for name, _ in QueryStatsC._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stream_close(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def k1_tuned_variant(value_type: str, n_queries: int, rows: int) -> int:
    """The autotuner's fused-pass variant for this size class (0: still timing)."""
    return int(load().lms_k1_tuned_variant(VALUE_FLOAT32 if value_type == "float32" else VALUE_INT32,
                                           int(n_queries), int(rows)))


def udiv_invariant(n: int, d: int) -> int:
    return int(load().lms_udiv_invariant(n, d))


def aggregate_batch_static(ts, key, value, type_=None, *, value_type: str, size_ms: int,
                           slide_ms: int = 0, filter_col: str = "ts", filter_op: str = "none",
                           filter_value=0, agg_mask: int = AGG_ALL, rows_ptr: int, rows_cap: int,
                           cuda_stream: Optional[int] = None) -> int:
    """lms_aggregate_batch_static on device tensors; rows go to the device buffer
    at rows_ptr (rows_cap rows of 48 bytes).  Returns the number of rows."""
    lib = load()
    q = QuerySpec()
    q.filter_col = COLS[filter_col]
    q.filter_op = OPS[filter_op]
    if filter_col == "value" and value_type == "float32":
        q.filter_f = float(filter_value)
    else:
        q.filter_i = int(filter_value)
    q.window_size_ms = int(size_ms)
    q.window_slide_ms = int(slide_ms)
    q.agg_mask = int(agg_mask)
    cols = [_ptr_and_mem(c) for c in (ts, key, value, type_)]
    if any(m == MEM_HOST for _, m, _ in cols):
        raise ValueError("lms_aggregate_batch_static reads device memory only")
    n = ctypes.c_size_t()
    st = lib.lms_aggregate_batch_static(
        ctypes.byref(q), VALUE_FLOAT32 if value_type == "float32" else VALUE_INT32,
        cols[0][0], cols[1][0], cols[2][0], cols[3][0], int(ts.shape[0]), cuda_stream,
        rows_ptr, int(rows_cap), ctypes.byref(n))
    if st != LMS_OK:
        raise LmsError(st, "lms_aggregate_batch_static")
    return n.value


class VariantAnalytic:
    """lms_variant_analytic: Alg. 2 + Eq. 9 chooser of the fused pass's variant."""

    def __init__(self, partitions: int = 148, bytes_per_row: float = 16.0,
                 infpt0: float = 150 * 1024, history: int = 0, explore: int = 2):
        self._lib = load()
        self._h = self._lib.lms_variant_analytic_create(int(partitions), float(bytes_per_row),
                                                        float(infpt0), int(history), int(explore))
        if not self._h:
            raise LmsError(LMS_EINVAL, "lms_variant_analytic_create")

    def choose(self, rows: int, n_queries: int = 1) -> int:
        return int(self._lib.lms_variant_analytic_choose(self._h, int(rows), int(n_queries)))

    def observe(self, rows: int, variant: int, ms: float) -> None:
        self._lib.lms_variant_analytic_observe(self._h, int(rows), int(variant), float(ms))

    def predict(self, rows: int, variant: int) -> float:
        return float(self._lib.lms_variant_analytic_predict(self._h, int(rows), int(variant)))

    def state(self) -> dict:
        inf = ctypes.c_double()
        picks = (ctypes.c_int64 * 2)()
        self._lib.lms_variant_analytic_state(self._h, ctypes.byref(inf), picks)
        return {"infpt_bytes": inf.value, "picks": [picks[0], picks[1]]}

    def hooks(self):
        lib = self._lib
        return (ctypes.cast(lib.lms_variant_analytic_choose, ctypes.c_void_p).value,
                ctypes.cast(lib.lms_variant_analytic_observe, ctypes.c_void_p).value, self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lms_variant_analytic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VariantLearned:
    """lms_variant_learned: the network's chooser of the fused pass's variant,
    with a VariantAnalytic as fallback and judge."""

    def __init__(self, mlp, judge: VariantAnalytic, *, key_card, selectivity, panes, n_queries):
        self._lib = load()
        self.judge = judge
        self._h = self._lib.lms_variant_learned_create(mlp.handle, judge._h, float(key_card),
                                                       float(selectivity), float(panes),
                                                       float(n_queries))
        if not self._h:
            raise LmsError(LMS_EINVAL, "lms_variant_learned_create")

    def set_online(self, refit_every: int, refit_steps: int, lr: float = 1e-3):
        self._lib.lms_variant_learned_set_online(self._h, int(refit_every), int(refit_steps),
                                                 float(lr))

    def fit(self, steps: int, lr: float = 1e-3) -> float:
        loss = ctypes.c_float()
        st = self._lib.lms_variant_learned_fit(self._h, int(steps), float(lr), ctypes.byref(loss))
        if st not in (LMS_OK, LMS_EAGAIN):
            raise LmsError(st, "lms_variant_learned_fit")
        return float(loss.value)

    def stats(self) -> dict:
        en, ea = ctypes.c_double(), ctypes.c_double()
        un, ua = ctypes.c_int64(), ctypes.c_int64()
        picks = (ctypes.c_int64 * 2)()
        self._lib.lms_variant_learned_stats(self._h, ctypes.byref(en), ctypes.byref(ea),
                                            ctypes.byref(un), ctypes.byref(ua), picks)
        return {"err_net": en.value, "err_analytic": ea.value, "uses_net": un.value,
                "uses_analytic": ua.value, "picks": [picks[0], picks[1]]}

    def hooks(self):
        lib = self._lib
        return (ctypes.cast(lib.lms_variant_learned_choose, ctypes.c_void_p).value,
                ctypes.cast(lib.lms_variant_learned_observe, ctypes.c_void_p).value, self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lms_variant_learned_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Admission:
    """ConstructMicroBatch (Alg. 1) state held by the engine library."""

    def __init__(self, slide_ms: float, policy: int = ADMIT_PAPER, poll_ms: float = 10.0):
        self._lib = load()
        self._h = self._lib.lms_admission_create(float(slide_ms), int(policy), float(poll_ms))
        if not self._h:
            raise ValueError("bad admission arguments")
        self._pred = None

    def set_predictor(self, fn):
        self._pred = None if fn is None else PROC_PREDICTOR(lambda ctx, b, n: float(fn(b, n)))
        self._lib.lms_admission_set_predictor(self._h, self._pred, None)

    def poll(self, now_ms: float, arrivals=(), nbytes=()):
        a = np.ascontiguousarray(arrivals, dtype=np.float64)
        b = np.ascontiguousarray(nbytes, dtype=np.float64)
        est = ctypes.c_double()
        nadm = ctypes.c_int32()
        r = self._lib.lms_admission_poll(self._h, float(now_ms), a.ctypes.data, b.ctypes.data,
                                         int(a.shape[0]), ctypes.byref(est), ctypes.byref(nadm))
        if r < 0:
            raise LmsError(r, "lms_admission_poll")
        return bool(r), est.value, nadm.value

    def complete(self, proc_ms: float) -> float:
        return float(self._lib.lms_admission_complete(self._h, float(proc_ms)))

    def avg_thput(self) -> float:
        return float(self._lib.lms_admission_avg_thput(self._h))

    def buffered(self) -> int:
        return int(self._lib.lms_admission_buffered(self._h))

    def __del__(self):
        try:
            if self._h:
                self._lib.lms_admission_destroy(self._h)
        except Exception:
            pass


def map_device(ops, batch_bytes: float, num_cores: int, infpt: float, base_trans_cost=0.1):
    lib = load()
    o = np.ascontiguousarray([QOPS[x] for x in ops], dtype=np.int32)
    dev = np.zeros(len(ops), np.int32)
    cpu = np.zeros(len(ops))
    gpu = np.zeros(len(ops))
    st = lib.lms_map_device(o.ctypes.data, len(ops), float(batch_bytes), int(num_cores),
                            float(infpt), float(base_trans_cost), dev.ctypes.data,
                            cpu.ctypes.data, gpu.ctypes.data)
    if st != LMS_OK:
        raise LmsError(st, "lms_map_device")
    return [("CPU" if d else "GPU", c, g) for d, c, g in zip(dev, cpu, gpu)]


class Regressor:
    """Online least-squares model of the inflection point (Eq. 9)."""

    def __init__(self, history_len: int = 0):
        self._lib = load()
        self._h = self._lib.lms_regressor_create(int(history_len))

    def add(self, thput, lat, infpt):
        self._lib.lms_regressor_add(self._h, float(thput), float(lat), float(infpt))

    def fit(self, target_thput, target_lat):
        beta = np.zeros(3)
        out = ctypes.c_double()
        st = self._lib.lms_regressor_fit(self._h, float(target_thput), float(target_lat),
                                         beta.ctypes.data, ctypes.byref(out))
        return st, beta, out.value

    def __del__(self):
        try:
            if self._h:
                self._lib.lms_regressor_destroy(self._h)
        except Exception:
            pass


def _struct_dict(x) -> dict:
    return {f[0]: getattr(x, f[0]) for f in x._fields_ if f[0] != "reserved"}


def serve_run(tick_counts, *, poll_ms: float, policy: int, bound_ms: float, backend=None,
              process=None, admissible=None, predictor=None, observer=None, fixed_rows: int = 0,
              trigger_ms: float = 0.0, bytes_per_event: float = 16.0,
              admit_rule: int = ADMIT_GUARDED, add_decide_time: bool = False,
              stop_when_missed: bool = False, quantile_hi: float = 0.99, log_cap: int = 1 << 16):
    """Runs the serving loop (lms_serve_run).  Either `backend` (a ServeBackend
    from a native backend) or Python callables `process(chunks, n_events, rec)`
    -> ms and optional `admissible()` -> rows.  `predictor` is a Python callable
    (bytes, n_datasets) -> ms or a (PROC_PREDICTOR-compatible address, ctx) pair;
    `observer` an lms_batch_observer address called with that ctx (Learned.hooks()).
    Returns (result dict, per-batch records as a list of dicts)."""
    lib = load()
    counts = np.ascontiguousarray(tick_counts, dtype=np.int64)
    cfg = ServeConfig(policy=int(policy), admit_rule=int(admit_rule), fixed_rows=int(fixed_rows),
                      trigger_ms=float(trigger_ms), latency_bound_ms=float(bound_ms),
                      poll_ms=float(poll_ms), bytes_per_event=float(bytes_per_event),
                      add_decide_time=int(bool(add_decide_time)),
                      stop_when_missed=int(bool(stop_when_missed)), quantile_hi=float(quantile_hi))
    keep = []
    if backend is None:
        def _proc(ctx, chunks, n_chunks, n_events, rec):
            return float(process([chunks[i] for i in range(n_chunks)], int(n_events), rec[0]))
        cb = SERVE_PROCESS(_proc)
        keep.append(cb)
        adm = None
        if admissible is not None:
            adm = SERVE_ADMISSIBLE(lambda ctx: int(admissible()))
            keep.append(adm)
        backend = ServeBackend(None, ctypes.cast(cb, ctypes.c_void_p).value,
                               ctypes.cast(adm, ctypes.c_void_p).value if adm else None)
    pred_fn, pred_ctx = None, None
    if predictor is not None:
        if callable(predictor):
            f = PROC_PREDICTOR(lambda ctx, b, n: float(predictor(b, n)))
            keep.append(f)
            pred_fn = ctypes.cast(f, ctypes.c_void_p).value
        else:
            pred_fn, pred_ctx = predictor
    log = (ServeBatch * int(log_cap))()
    n_log = ctypes.c_size_t()
    res = ServeResult()
    st = lib.lms_serve_run(ctypes.byref(cfg), counts.ctypes.data, int(counts.shape[0]),
                           ctypes.byref(backend), pred_fn, pred_ctx, observer, ctypes.byref(res),
                           ctypes.cast(log, ctypes.c_void_p), int(log_cap), ctypes.byref(n_log))
    if st != LMS_OK:
        raise LmsError(st, "lms_serve_run")
    recs = [_struct_dict(log[i]) for i in range(min(n_log.value, log_cap))]
    return _struct_dict(res), recs


def _query_spec(q: dict) -> QuerySpec:
    fv = q.get("value", 0)
    return QuerySpec(filter_col=COLS[q.get("col", "ts")], filter_op=OPS[q.get("op", "none")],
                     filter_i=0 if isinstance(fv, float) else int(fv), filter_f=float(fv),
                     window_size_ms=int(q["size"]), window_slide_ms=int(q.get("slide", 0)),
                     agg_mask=AGG_ALL)


class ServeGpu:
    """The engine as a serving backend (lms_serve_gpu_*): a float32 stream with
    the given queries and a device load generator (Zipf keys, lognormal values,
    ts = floor(arrival ms))."""

    def __init__(self, queries, *, seed: int, n_keys: int = 1_000_000, zipf_s: float = 1.1,
                 max_batch_rows: int = 1 << 24, state_cap_bytes: int = 0,
                 enable_timing: bool = True, keep_rows: bool = False, device_input: bool = False,
                 ingest: bool = False, device: int = 0):
        self._lib = load()
        cfg = StreamConfig(device=device, value_type=VALUE_FLOAT32, has_type=0,
                           enable_timing=int(enable_timing), allowed_lateness_ms=0,
                           max_batch_rows=int(max_batch_rows),
                           state_cap_bytes=int(state_cap_bytes), cuda_stream=None,
                           origin_ts=ORIGIN_AUTO, k1_variant=0)
        specs = (QuerySpec * len(queries))(*[_query_spec(q) for q in queries])
        h = ctypes.c_void_p()
        st = self._lib.lms_serve_gpu_create(ctypes.byref(cfg), specs, len(queries), int(seed),
                                            int(n_keys), float(zipf_s), int(max_batch_rows),
                                            (1 if keep_rows else 0) | (2 if device_input else 0)
                                            | (4 if ingest else 0),
                                            ctypes.byref(h))
        if st != LMS_OK:
            raise LmsError(st, "lms_serve_gpu_create")
        self._h = h.value
        self.nq = len(queries)
        self.max_batch_rows = int(max_batch_rows)

    def backend(self) -> ServeBackend:
        b = ServeBackend()
        st = self._lib.lms_serve_gpu_backend(self._h, ctypes.byref(b))
        if st != LMS_OK:
            raise LmsError(st, "lms_serve_gpu_backend")
        return b

    def stats(self) -> dict:
        out = StatsC()
        self._lib.lms_stream_stats(self._lib.lms_serve_gpu_stream(self._h), ctypes.byref(out))
        return {f[0]: getattr(out, f[0]) for f in StatsC._fields_}

    def prefill(self, t0_ms: float, span_ms: float, n_batches: int, events_per_batch: int):
        """lms_serve_gpu_prefill: window state to steady state before a run."""
        st = self._lib.lms_serve_gpu_prefill(self._h, float(t0_ms), float(span_ms),
                                             int(n_batches), int(events_per_batch))
        if st != LMS_OK:
            raise LmsError(st, "lms_serve_gpu_prefill")

    def admissible_rows(self) -> int:
        n = ctypes.c_int64()
        st = self._lib.lms_stream_admissible_rows(self._lib.lms_serve_gpu_stream(self._h), 1,
                                                  ctypes.byref(n))
        if st != LMS_OK:
            raise LmsError(st, "lms_stream_admissible_rows")
        return n.value

    def generate(self, chunks):
        """chunks: list of (t0_ms, width_ms, n_total, j_begin, j_end, first_event)."""
        arr = (ServeChunk * len(chunks))(*[ServeChunk(*c) for c in chunks])
        n = int(sum(c[4] - c[3] for c in chunks))
        ts = np.empty(n, np.int64)
        key = np.empty(n, np.uint32)
        val = np.empty(n, np.float32)
        st = self._lib.lms_serve_gpu_generate(self._h, arr, len(chunks), n, ts.ctypes.data,
                                              key.ctypes.data, val.ctypes.data)
        if st != LMS_OK:
            raise LmsError(st, "lms_serve_gpu_generate")
        return ts, key, val

    def kept_rows(self, qid: int) -> np.ndarray:
        n = ctypes.c_size_t()
        self._lib.lms_serve_gpu_kept_rows(self._h, int(qid), None, 0, ctypes.byref(n))
        out = np.zeros(n.value, ROW_DTYPE_FLOAT)
        if n.value:
            self._lib.lms_serve_gpu_kept_rows(self._h, int(qid), out.ctypes.data, n.value,
                                              ctypes.byref(n))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lms_serve_gpu_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_INPUTS, MLP_PARAMS, MLP_MAX_BATCH = 8, 8961, 4096
_MLP_SHAPES = [(64, 8), (64,), (64, 64), (64,), (64, 64), (64,), (64,), (1,)]


def mlp_init_params(seed: int) -> np.ndarray:
    """Initial network weights: He-uniform (limit sqrt(6 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, shp in enumerate(_MLP_SHAPES):
        if i % 2 == 0:
            fan_in = shp[-1] if len(shp) == 2 else 64
            lim = np.sqrt(6.0 / fan_in)
            parts.append(rng.uniform(-lim, lim, shp).ravel())
        else:
            parts.append(np.zeros(int(np.prod(shp))))
    return np.concatenate(parts).astype(np.float32)
OP_H2D, OP_K1, OP_SORT, OP_EMIT, OP_HOST, N_OPS = 0, 1, 2, 3, 4, 5


class Mlp:
    """The learned cost model's network on the GPU (lms_mlp_*)."""

    def __init__(self, params, device: int = 0):
        self._lib = load()
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.shape == (MLP_PARAMS,)
        self._h = self._lib.lms_mlp_create(int(device), p.ctypes.data)
        if not self._h:
            raise LmsError(LMS_ECUDA, "lms_mlp_create")

    @property
    def handle(self):
        return self._h

    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        st = self._lib.lms_mlp_get_params(self._h, out.ctypes.data)
        if st != LMS_OK:
            raise LmsError(st, "lms_mlp_get_params")
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        st = self._lib.lms_mlp_set_params(self._h, p.ctypes.data)
        if st != LMS_OK:
            raise LmsError(st, "lms_mlp_set_params")

    def forward(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, MLP_INPUTS)
        y = np.empty(x.shape[0], np.float32)
        st = self._lib.lms_mlp_forward(self._h, x.ctypes.data, x.shape[0], y.ctypes.data)
        if st != LMS_OK:
            raise LmsError(st, "lms_mlp_forward")
        return y

    def train(self, x, t, steps: int, lr: float = 1e-3, want_grad: bool = False):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, MLP_INPUTS)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.empty(MLP_PARAMS, np.float32) if want_grad else None
        loss = ctypes.c_float()
        st = self._lib.lms_mlp_train(self._h, x.ctypes.data, t.ctypes.data, x.shape[0],
                                     int(steps), float(lr), None if g is None else g.ctypes.data,
                                     ctypes.byref(loss))
        if st != LMS_OK:
            raise LmsError(st, "lms_mlp_train")
        return (loss.value, g) if want_grad else loss.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lms_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cost_features(rows, carried, key_card, selectivity, panes, n_queries, span_panes, op):
    out = np.empty(MLP_INPUTS, np.float32)
    load().lms_cost_features(float(rows), float(carried), float(key_card), float(selectivity),
                             float(panes), float(n_queries), float(span_panes), int(op),
                             out.ctypes.data)
    return out


class Learned:
    """Alg. 1 predictor backed by an Mlp, with Eq. 5 as fallback and judge
    (lms_learned_*)."""

    def __init__(self, mlp: Mlp, serve_gpu=None, *, key_card, selectivity, panes, n_queries,
                 slide_ms, poll_ms, bytes_per_event=16.0):
        self._lib = load()
        self.mlp = mlp
        self._h = self._lib.lms_learned_create(
            mlp.handle, None if serve_gpu is None else serve_gpu._h, float(key_card),
            float(selectivity), float(panes), float(n_queries), float(slide_ms), float(poll_ms),
            float(bytes_per_event))
        if not self._h:
            raise LmsError(LMS_EINVAL, "lms_learned_create")

    def set_backend(self, serve_gpu):
        self._lib.lms_learned_set_backend(self._h, None if serve_gpu is None else serve_gpu._h)

    def set_online(self, refit_every: int, refit_steps: int, lr: float = 1e-3):
        self._lib.lms_learned_set_online(self._h, int(refit_every), int(refit_steps), float(lr))

    def observe(self, rec: dict) -> float:
        b = ServeBatch(**{k: rec[k] for k, _ in ServeBatch._fields_})
        return float(self._lib.lms_learned_observe(self._h, ctypes.byref(b)))

    def samples(self) -> int:
        return int(self._lib.lms_learned_samples(self._h))

    def fit(self, steps: int, lr: float = 1e-3) -> float:
        loss = ctypes.c_float()
        st = self._lib.lms_learned_fit(self._h, int(steps), float(lr), ctypes.byref(loss))
        if st != LMS_OK:
            raise LmsError(st, "lms_learned_fit")
        return loss.value

    def predict(self, batch_bytes: float, n_datasets: int) -> float:
        return float(self._lib.lms_learned_predict(self._h, float(batch_bytes), int(n_datasets)))

    def stats(self) -> dict:
        en, ee = ctypes.c_double(), ctypes.c_double()
        un, ue = ctypes.c_int64(), ctypes.c_int64()
        self._lib.lms_learned_stats(self._h, ctypes.byref(en), ctypes.byref(ee), ctypes.byref(un),
                                    ctypes.byref(ue))
        return {"err_net": en.value, "err_eq5": ee.value, "uses_net": un.value,
                "uses_eq5": ue.value}

    def hooks(self):
        """(predictor, observer) arguments for serve_run."""
        pred = ctypes.cast(self._lib.lms_learned_predict, ctypes.c_void_p).value
        obs = ctypes.cast(self._lib.lms_learned_observe, ctypes.c_void_p).value
        return (pred, self._h), obs

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lms_learned_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching across streams (lms_server_*): `slots` concurrent
    micro-batches, admission by a device memory budget."""

    def __init__(self, slots: int, memory_budget_bytes: int = 0, ops=None):
        """ops: None for the engine, or Python callables (push(stream, batch) ->
        status, push_bytes(stream, n_rows, host_input) -> bytes,
        device_bytes(stream) -> bytes) to exercise the scheduling alone."""
        self._lib = load()
        cfg = ServerConfig(slots=int(slots), memory_budget_bytes=int(memory_budget_bytes))
        h = ctypes.c_void_p()
        if ops is None:
            st = self._lib.lms_server_create(ctypes.byref(cfg), ctypes.byref(h))
        else:
            push, push_bytes, device_bytes = ops

            def _pb(ctx, s, n, host, out):
                out[0] = int(push_bytes(s, n, host))
                return LMS_OK

            def _db(ctx, s, out):
                out[0] = int(device_bytes(s))
                return LMS_OK
            self._cbs = (SERVER_PUSH(lambda ctx, s, b: int(push(s, b[0]))),
                         SERVER_PUSH_BYTES(_pb), SERVER_DEVICE_BYTES(_db))
            o = ServerOps(None, *[ctypes.cast(c, ctypes.c_void_p).value for c in self._cbs])
            st = self._lib.lms_server_create_ops(ctypes.byref(cfg), ctypes.byref(o),
                                                 ctypes.byref(h))
        if st != LMS_OK:
            raise LmsError(st, "lms_server_create")
        self._h = h.value
        self._keep = {}

    def submit(self, stream, ts=None, key=None, value=None, type_=None, eos: bool = False,
               batch=None) -> int:
        """Queues a push of the columns on `stream` (a Stream), or of a ready
        BatchC `batch` on a raw stream handle."""
        if batch is None:
            b, keep = stream.make_batch(ts, key, value, type_, eos)
            handle = stream._h
        else:
            b, keep, handle = batch, None, stream
        t = ctypes.c_uint64()
        st = self._lib.lms_server_submit(self._h, handle, ctypes.byref(b), ctypes.byref(t))
        if st != LMS_OK:
            raise LmsError(st, "lms_server_submit")
        self._keep[t.value] = keep  # columns must outlive the request
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(status of the push, start ms, end ms) of a ticket."""
        res = ctypes.c_int32()
        a, b = ctypes.c_double(), ctypes.c_double()
        st = self._lib.lms_server_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(res),
                                       ctypes.byref(a), ctypes.byref(b))
        if st != LMS_OK:
            raise LmsError(st, "lms_server_wait")
        self._keep.pop(int(ticket), None)
        return res.value, a.value, b.value

    def forget(self, stream):
        st = self._lib.lms_server_forget(self._h, getattr(stream, "_h", stream))
        if st != LMS_OK:
            raise LmsError(st, "lms_server_forget")

    def stats(self) -> dict:
        out = ServerStats()
        self._lib.lms_server_get_stats(self._h, ctypes.byref(out))
        return {f[0]: getattr(out, f[0]) for f in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lms_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
