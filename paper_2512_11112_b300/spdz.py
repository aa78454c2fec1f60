"""Thin ctypes binding of ``include/spdz.h`` (libspdz.so).

Every function here has the name of the C entry point it wraps and only
marshals arguments: device buffers are torch tensors (int64 storage holding
the uint64 words of each field element; int32 storage of the uint32 elements
of p = 2^32-5), host buffers are numpy arrays.  A
non-OK status raises :class:`SpdzError` carrying the code and the library's
message.  There is no fallback: if the CUDA library is missing the import
fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspdz.so")

SPDZ_OK, SPDZ_ERR_ARG, SPDZ_ERR_ALIGN, SPDZ_ERR_OOM, SPDZ_ERR_TRIPLES = 0, 1, 2, 3, 4
SPDZ_ERR_MAC, SPDZ_ERR_TIMEOUT, SPDZ_ERR_CUDA, SPDZ_ERR_STATE = 5, 6, 7, 8
SPDZ_F61, SPDZ_F127, SPDZ_F32 = 0, 1, 2
SPDZ_OP_ADD, SPDZ_OP_SUB, SPDZ_OP_CMUL, SPDZ_OP_CADD, SPDZ_OP_MUL = 0, 1, 2, 3, 4
SPDZ_KIND_ALPHA, SPDZ_KIND_TRIPLE_A, SPDZ_KIND_TRIPLE_B, SPDZ_KIND_TRIPLE_C = 1, 2, 3, 4
SPDZ_KIND_INPUT, SPDZ_KIND_CHECK = 5, 6
SPDZ_KIND_MTRIPLE_A, SPDZ_KIND_MTRIPLE_B, SPDZ_KIND_MTRIPLE_C = 7, 8, 9
SPDZ_KIND_INPUT_MASK = 10
SPDZ_MAX_PARTIES = 8
P61 = (1 << 61) - 1
P127 = (1 << 127) - 1
P32 = (1 << 32) - 5


class SpdzError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"spdz error {code}: {msg}")
        self.code = code


class spdz_buf(C.Structure):
    _fields_ = [("val", C.c_void_p), ("mac", C.c_void_p), ("stride", C.c_int64)]


SPDZ_SCHED_PER_LAYER, SPDZ_SCHED_FUSED, SPDZ_SCHED_TAGGED = 0, 1, 2
SPDZ_MAX_GROUPS = 256


class spdz_dag_desc(C.Structure):
    _fields_ = [("n_inputs", C.c_int64), ("n_gates", C.c_int64), ("depth", C.c_int32),
                ("layer_offsets", C.c_void_p), ("ops", C.c_void_p), ("in0", C.c_void_p),
                ("in1", C.c_void_p), ("kconst", C.c_void_p)]


class spdz_plan(C.Structure):
    _fields_ = [("mode", C.c_int32), ("block", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("use_graph", C.c_int32), ("n_groups", C.c_int32),
                ("group_end", C.c_int32 * SPDZ_MAX_GROUPS),
                ("group_flush", C.c_uint8 * SPDZ_MAX_GROUPS),
                ("group_ctas_per_sm", C.c_int32 * SPDZ_MAX_GROUPS),
                ("record_layer_times", C.c_int32), ("spin_limit_us", C.c_uint32),
                ("barrier_extra_arrivals", C.c_int32),
                ("group_cluster", C.c_int32 * SPDZ_MAX_GROUPS),
                ("group_block", C.c_int32 * SPDZ_MAX_GROUPS), ("poll_ns", C.c_uint32),
                ("barrier_slack", C.c_uint32), ("test_unwritten_tag", C.c_int32),
                ("group_tagged", C.c_int32 * SPDZ_MAX_GROUPS)]


class spdz_stats(C.Structure):
    _fields_ = [("device_ms", C.c_double), ("passed", C.c_int32), ("launches", C.c_int32),
                ("n_gates", C.c_int64), ("n_mul", C.c_int64)]


class spdz_sched_report(C.Structure):
    _fields_ = [("default_ms", C.c_double), ("autotuned_ms", C.c_double), ("learned_ms", C.c_double),
                ("predicted_ms", C.c_double), ("switch_us", C.c_double), ("chosen", C.c_int32),
                ("learned_groups", C.c_int32), ("samples", C.c_int32), ("train_loss", C.c_float),
                ("tagged_ms", C.c_double), ("learned_is_autotuned", C.c_int32)]


SPDZ_SERVE_SEQUENTIAL, SPDZ_SERVE_BATCHED, SPDZ_SERVE_HEURISTIC, SPDZ_SERVE_LEARNED = 0, 1, 2, 3
SPDZ_MATMUL_CUDA_CORE, SPDZ_MATMUL_TENSOR = 0, 1
TENSOR_PATH = True          # the library has the tensor-core matrix path


class spdz_serve_request(C.Structure):
    _fields_ = [("dag", C.POINTER(spdz_dag_desc)), ("circuit_id", C.c_int64), ("field", C.c_int32),
                ("seed", C.c_uint64), ("arrival_s", C.c_double), ("in_val_host", C.c_void_p),
                ("in_mac_host", C.c_void_p), ("out_val_host", C.c_void_p), ("out_mac_host", C.c_void_p)]


class spdz_serve_result(C.Structure):
    _fields_ = [("latency_s", C.c_double), ("online_s", C.c_double), ("passed", C.c_int32), ("mode", C.c_int32),
                ("status", C.c_int32), ("pad", C.c_int32), ("req_id", C.c_uint64)]


class spdz_serve_stats(C.Structure):
    _fields_ = [("wall_s", C.c_double), ("gates_per_s", C.c_double), ("p50_s", C.c_double), ("p99_s", C.c_double),
                ("mean_s", C.c_double), ("requests", C.c_int64), ("gates", C.c_int64), ("ticks", C.c_int64),
                ("cluster_requests", C.c_int64), ("dealer_s", C.c_double), ("peak_bytes", C.c_int64),
                ("max_active", C.c_int32), ("host_admit_s", C.c_double), ("host_tick_s", C.c_double),
                ("host_complete_s", C.c_double), ("host_idle_s", C.c_double), ("host_ring_wait_s", C.c_double),
                ("device_tick_s", C.c_double), ("device_ticks_timed", C.c_int64), ("grid_requests", C.c_int64)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libspdz.so is not built ({LIB_PATH}); run paper_2512_11112_b300/build.py")

lib = C.CDLL(LIB_PATH)
_vp, _i64, _u64, _int = C.c_void_p, C.c_int64, C.c_uint64, C.c_int
_bufp = C.POINTER(spdz_buf)

_SIGS = {
    "spdz_ctx_create": [C.POINTER(_vp), _int, _int, _vp],
    "spdz_ctx_destroy": [_vp],
    "spdz_ctx_set_stream": [_vp, _vp],
    "spdz_deal_alpha": [_vp, _u64, _vp],
    "spdz_deal_shared": [_vp, _u64, C.c_uint32, _u64, _u64, _i64, _vp, _vp, _bufp, _vp],
    "spdz_deal_triples": [_vp, _u64, _u64, _i64, _vp, _bufp, _bufp, _bufp],
    "spdz_load_preproc": [_vp, _vp, _bufp, _bufp, _bufp, _i64],
    "spdz_triples_left": [_vp, C.POINTER(_i64)],
    "spdz_linear": [_vp, _int, _bufp, _bufp, _vp, _bufp, _i64],
    "spdz_mul_batch": [_vp, _bufp, _bufp, _bufp, _i64, _vp],
    "spdz_open": [_vp, _bufp, _vp, _i64],
    "spdz_set_check_seed": [_vp, _u64],
    "spdz_mac_check": [_vp, C.POINTER(_int), _vp],
    "spdz_check_state": [_vp, C.POINTER(_i64), C.POINTER(_i64)],
    "spdz_innerprod_batch": [_vp, _bufp, _bufp, _bufp, _i64, _i64],
    "spdz_field_op": [_vp, _int, _vp, _vp, _vp, _i64],
    "spdz_dag_create": [_vp, C.POINTER(spdz_dag_desc), C.POINTER(_vp)],
    "spdz_dag_destroy": [_vp],
    "spdz_run_dag": [_vp, _vp, C.POINTER(spdz_plan), _bufp, C.POINTER(spdz_stats)],
    "spdz_check_result": [_vp, C.POINTER(_int), _vp],
    "spdz_dag_layer_times": [_vp, _vp],
    "spdz_dag_time_kernels": [_vp, C.c_int32],
    "spdz_dag_kernel_ms": [_vp, C.POINTER(C.c_float)],
    "spdz_dag_layer_counts": [_vp, _vp],
    "spdz_mul_check_noalloc": [_int, _int, _vp, _bufp, _bufp, _bufp, _bufp, _bufp, _vp, _bufp, _i64, _u64,
                               _u64, _vp],
    "spdz_mlp_create": [C.POINTER(_vp), C.c_int32, C.c_int32, C.c_int32, _u64, _vp],
    "spdz_mlp_destroy": [_vp],
    "spdz_mlp_num_params": [_vp, C.POINTER(_i64)],
    "spdz_mlp_get_params": [_vp, _vp],
    "spdz_mlp_set_params": [_vp, _vp],
    "spdz_mlp_forward": [_vp, _vp, _i64, _vp],
    "spdz_mlp_loss_grad": [_vp, _vp, _vp, _i64, _vp, _vp],
    "spdz_mlp_train": [_vp, _vp, _vp, _i64, C.c_int32, C.c_int32, C.c_float, _vp],
    "spdz_mlp_adam_step": [_vp, _vp, C.c_float],
    "spdz_run_dag_host": [_vp, _vp, C.POINTER(spdz_plan), _bufp, _vp, _vp, C.POINTER(_vp), _i64, _i64, _vp, _vp],
    "spdz_int_peak": [_int, _i64, _vp, _vp, C.POINTER(C.c_double)],
    "spdz_party_create": [C.POINTER(_vp), _int, _int, _int, _vp],
    "spdz_party_destroy": [_vp],
    "spdz_party_load_alpha": [_vp, _vp],
    "spdz_party_set_check_seed": [_vp, _u64],
    "spdz_party_mask": [_vp, _bufp, _bufp, _bufp, _bufp, _vp, _vp, _i64],
    "spdz_party_open_sum": [_vp, _vp, _i64, _vp],
    "spdz_party_combine": [_vp, _vp, _vp, _bufp, _bufp, _bufp, _bufp, _bufp, _bufp, _i64],
    "spdz_party_sigma": [_vp, _vp, C.POINTER(_i64)],
    "spdz_sched_num_configs": [C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "spdz_sched_config_plan": [_vp, C.c_int32, C.POINTER(spdz_plan)],
    "spdz_sched_record": [_vp, _vp, _bufp, C.c_int32],
    "spdz_sched_samples": [_vp, _vp, _vp, C.POINTER(_i64), C.POINTER(C.c_double)],
    "spdz_sched_train": [_vp, C.c_int32, C.c_float, _u64, C.POINTER(C.c_float)],
    "spdz_sched_add_samples": [_vp, _vp, _vp, _i64],
    "spdz_sched_predict": [_vp, _vp, C.c_int32, _vp],
    "spdz_sched_learned_plan": [_vp, _vp, C.POINTER(spdz_plan), C.POINTER(C.c_double)],
    "spdz_sched_autotune": [_vp, _vp, _bufp, C.c_int32, C.POINTER(spdz_plan), C.POINTER(C.c_double)],
    "spdz_sched_choose": [_vp, _vp, _bufp, C.c_int32, C.POINTER(spdz_plan), C.POINTER(spdz_sched_report)],
    "spdz_serve_create": [C.POINTER(_vp), _int, _u64, C.c_int32, C.c_int32, _vp, _u64, _i64],
    "spdz_serve_run": [_vp, C.POINTER(spdz_serve_request), _i64, C.POINTER(spdz_serve_result),
                       C.POINTER(spdz_serve_stats)],
    "spdz_serve_destroy": [_vp],
    "spdz_serve_register": [_vp, _vp, C.c_int32, C.POINTER(_i64)],
    "spdz_serve_unregister": [_vp, _i64],
    "spdz_serve_start": [_vp],
    "spdz_serve_submit": [_vp, C.POINTER(spdz_serve_request), C.POINTER(_u64)],
    "spdz_serve_poll": [_vp, _u64, C.POINTER(C.c_int32), C.POINTER(spdz_serve_result)],
    "spdz_serve_stop": [_vp, C.POINTER(spdz_serve_stats)],
    "spdz_deal_matrix_triple": [_vp, _u64, _u64, _i64, _i64, _i64, _vp, _bufp, _bufp, _bufp],
    "spdz_load_matrix_preproc": [_vp, _bufp, _bufp, _bufp, _i64, _i64, _i64],
    "spdz_matmul": [_vp, _bufp, _bufp, _bufp, _i64, _i64, _i64, _int, _vp, _vp],
    "spdz_serve_set_mode": [_vp, C.c_int32, _vp, _i64],
    "spdz_deal_input_masks": [_vp, _u64, C.c_int32, _u64, _i64, _vp, _bufp, _vp],
    "spdz_input": [_vp, _vp, _vp, _bufp, _bufp, _i64, _vp],
    "spdz_reveal": [_vp, _bufp, _vp, _i64, C.POINTER(_int), _vp],
    "spdz_deal_matvec_triples": [_vp, _u64, _u64, _i64, _i64, _i64, _vp, _bufp, _bufp, _bufp],
    "spdz_load_matvec_preproc": [_vp, _bufp, _bufp, _bufp, _i64, _i64, _i64],
    "spdz_linear_layer": [_vp, _bufp, _bufp, _bufp, _bufp, _i64, _i64, _i64, _vp, _vp],
}
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _int
lib.spdz_last_error.argtypes = [_vp]
lib.spdz_last_error.restype = C.c_char_p

HEADER_SYMBOLS = sorted(list(_SIGS) + ["spdz_last_error"])


def spdz_last_error(ctx) -> str:
    return lib.spdz_last_error(ctx).decode(errors="replace")


def _chk(ctx, rc: int) -> int:
    if rc != SPDZ_OK:
        raise SpdzError(rc, spdz_last_error(ctx) if ctx else "")
    return rc


def ptr(t) -> int | None:
    """Device (or host) address of a torch tensor / numpy array, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def buf(val, mac, stride: int | None = None, offset: int = 0, words: int = 1) -> spdz_buf:
    """spdz_buf over party-major tensors [n, stride(, 2)], starting at element offset
    (the element size is taken from the tensor: int32 words, int64 words, or
    pairs of int64 words)."""
    if stride is None:
        stride = val.shape[1]
    eb = val.element_size() * (val.shape[2] if val.dim() == 3 else 1)
    return spdz_buf(val.data_ptr() + offset * eb, mac.data_ptr() + offset * eb, stride)


def _b(b):
    return None if b is None else C.byref(b)


def spdz_ctx_create(n_parties: int, field: int, stream: int | None = None):
    h = _vp()
    rc = lib.spdz_ctx_create(C.byref(h), n_parties, field, stream)
    if rc != SPDZ_OK:
        raise SpdzError(rc, "context creation failed")
    return h


def spdz_ctx_destroy(ctx) -> None:
    lib.spdz_ctx_destroy(ctx)


def spdz_ctx_set_stream(ctx, stream: int | None) -> None:
    _chk(ctx, lib.spdz_ctx_set_stream(ctx, stream))


def spdz_deal_alpha(ctx, seed: int, alpha_shares) -> None:
    _chk(ctx, lib.spdz_deal_alpha(ctx, seed, ptr(alpha_shares)))


def spdz_deal_shared(ctx, seed, kind, sub, j0, count, alpha_shares, secret, out: spdz_buf,
                     secret_out=None) -> None:
    _chk(ctx, lib.spdz_deal_shared(ctx, seed, kind, sub, j0, count, ptr(alpha_shares), ptr(secret),
                                   C.byref(out), ptr(secret_out)))


def spdz_deal_triples(ctx, seed, j0, count, alpha_shares, a: spdz_buf, b: spdz_buf, c: spdz_buf) -> None:
    _chk(ctx, lib.spdz_deal_triples(ctx, seed, j0, count, ptr(alpha_shares), C.byref(a), C.byref(b),
                                    C.byref(c)))


def spdz_load_preproc(ctx, alpha_shares, a, b, c, n_triples: int) -> None:
    _chk(ctx, lib.spdz_load_preproc(ctx, ptr(alpha_shares), _b(a), _b(b), _b(c), n_triples))


def spdz_triples_left(ctx) -> int:
    v = _i64()
    _chk(ctx, lib.spdz_triples_left(ctx, C.byref(v)))
    return v.value


def spdz_linear(ctx, op: int, x: spdz_buf, y: spdz_buf | None, k_host, z: spdz_buf, N: int) -> None:
    _chk(ctx, lib.spdz_linear(ctx, op, C.byref(x), _b(y), ptr(k_host), C.byref(z), N))


def spdz_mul_batch(ctx, x: spdz_buf, y: spdz_buf, z: spdz_buf, N: int, opened=None) -> None:
    _chk(ctx, lib.spdz_mul_batch(ctx, C.byref(x), C.byref(y), C.byref(z), N, ptr(opened)))


def spdz_open(ctx, x: spdz_buf, out, N: int) -> None:
    _chk(ctx, lib.spdz_open(ctx, C.byref(x), ptr(out), N))


def spdz_set_check_seed(ctx, seed: int) -> None:
    _chk(ctx, lib.spdz_set_check_seed(ctx, seed))


def spdz_mac_check(ctx, sigma_host: np.ndarray | None = None) -> bool:
    """Runs the check; returns True/False (False is SPDZ_ERR_MAC: abort)."""
    ok = _int(0)
    rc = lib.spdz_mac_check(ctx, C.byref(ok), ptr(sigma_host))
    if rc not in (SPDZ_OK, SPDZ_ERR_MAC):
        _chk(ctx, rc)
    return bool(ok.value)


def spdz_check_state(ctx):
    o, e = _i64(), _i64()
    _chk(ctx, lib.spdz_check_state(ctx, C.byref(o), C.byref(e)))
    return o.value, e.value


def spdz_innerprod_batch(ctx, x: spdz_buf, y: spdz_buf, z: spdz_buf, count: int, length: int) -> None:
    _chk(ctx, lib.spdz_innerprod_batch(ctx, C.byref(x), C.byref(y), C.byref(z), count, length))


def spdz_field_op(ctx, op: int, a, b, out, N: int) -> None:
    _chk(ctx, lib.spdz_field_op(ctx, op, ptr(a), ptr(b), ptr(out), N))


def plan(mode: int = SPDZ_SCHED_FUSED, block: int = 256, ctas_per_sm: int = 0, use_graph: int = 1,
         groups=None, flush=None, group_ctas=None, record_layer_times: int = 0,
         spin_limit_us: int = 0, barrier_extra_arrivals: int = 0, group_cluster=None,
         group_block=None, poll_ns: int = 0, barrier_slack: int = 0, test_unwritten_tag: int = 0,
         group_tagged=None) -> spdz_plan:
    """Builds a spdz_plan; groups = list of exclusive end layers;
    group_cluster[g] > 0 runs group g inside one cluster of that many CTAs."""
    p = spdz_plan()
    p.mode, p.block, p.ctas_per_sm, p.use_graph = mode, block, ctas_per_sm, use_graph
    groups = list(groups or [])
    p.n_groups = len(groups)
    for g, e in enumerate(groups):
        p.group_end[g] = int(e)
        p.group_flush[g] = int(flush[g]) if flush else 0
        p.group_ctas_per_sm[g] = int(group_ctas[g]) if group_ctas else 0
        p.group_cluster[g] = int(group_cluster[g]) if group_cluster else 0
        p.group_block[g] = int(group_block[g]) if group_block else 0
        p.group_tagged[g] = int(group_tagged[g]) if group_tagged else 0
    p.record_layer_times, p.spin_limit_us = record_layer_times, spin_limit_us
    p.barrier_extra_arrivals = barrier_extra_arrivals
    p.poll_ns = poll_ns
    p.barrier_slack = barrier_slack
    p.test_unwritten_tag = test_unwritten_tag
    return p


def spdz_dag_create(ctx, n_inputs: int, layer_offsets, ops, in0, in1, kconst):
    """Uploads a layered circuit given as numpy arrays (int64 offsets, uint8
    ops, uint32 operand wires, uint64 constants [G] or [G, 2])."""
    off = np.ascontiguousarray(layer_offsets, dtype=np.int64)
    ops = np.ascontiguousarray(ops, dtype=np.uint8)
    in0 = np.ascontiguousarray(in0, dtype=np.uint32)
    in1 = np.ascontiguousarray(in1, dtype=np.uint32)
    k = np.ascontiguousarray(kconst, dtype=np.uint64)
    d = spdz_dag_desc(n_inputs, ops.size, off.size - 1, off.ctypes.data, ops.ctypes.data,
                      in0.ctypes.data, in1.ctypes.data, k.ctypes.data)
    h = _vp()
    _chk(ctx, lib.spdz_dag_create(ctx, C.byref(d), C.byref(h)))
    return h


def spdz_dag_destroy(dag) -> None:
    lib.spdz_dag_destroy(dag)


def spdz_run_dag(ctx, dag, plan_: spdz_plan | None, wires: spdz_buf, want_stats: bool = True):
    """Runs the circuit; returns spdz_stats (want_stats) or None (enqueued
    only).  A failed MAC check returns stats with passed == 0."""
    st = spdz_stats() if want_stats else None
    rc = lib.spdz_run_dag(ctx, dag, _b(plan_), C.byref(wires), _b(st))
    if rc not in (SPDZ_OK, SPDZ_ERR_MAC):
        _chk(ctx, rc)
    return st


def spdz_run_dag_host(ctx, dag, plan_: spdz_plan | None, wires: spdz_buf, in_val, in_mac, tri, out_first: int,
                      out_count: int, out_val, out_mac) -> None:
    """Host-buffer circuit run (asynchronous): in_val / in_mac, the six triple
    arrays `tri` and out_val / out_mac are host tensors or arrays (pinned for
    asynchronous copies) that must outlive the run."""
    arr = (_vp * 6)(*[ptr(t) for t in tri]) if tri is not None else None
    _chk(ctx, lib.spdz_run_dag_host(ctx, dag, C.byref(plan_) if plan_ is not None else None, C.byref(wires),
                                    ptr(in_val), ptr(in_mac), arr, out_first, out_count, ptr(out_val), ptr(out_mac)))


def spdz_check_result(ctx, sigma_host: np.ndarray | None = None) -> bool:
    ok = _int(0)
    rc = lib.spdz_check_result(ctx, C.byref(ok), ptr(sigma_host))
    if rc not in (SPDZ_OK, SPDZ_ERR_MAC):
        _chk(ctx, rc)
    return bool(ok.value)


def spdz_dag_layer_times(dag, depth: int) -> np.ndarray:
    out = np.zeros(depth, dtype=np.float32)
    rc = lib.spdz_dag_layer_times(dag, out.ctypes.data)
    if rc != SPDZ_OK:
        raise SpdzError(rc, "layer times")
    return out


def spdz_dag_time_kernels(dag, on: bool) -> None:
    rc = lib.spdz_dag_time_kernels(dag, 1 if on else 0)
    if rc != SPDZ_OK:
        raise SpdzError(rc, "dag kernel timing")


def spdz_dag_kernel_ms(dag) -> float:
    ms = C.c_float(0.0)
    rc = lib.spdz_dag_kernel_ms(dag, C.byref(ms))
    if rc != SPDZ_OK:
        raise SpdzError(rc, "dag kernel time")
    return float(ms.value)


def spdz_dag_layer_counts(dag, depth: int) -> np.ndarray:
    out = np.zeros((depth, 5), dtype=np.int32)
    rc = lib.spdz_dag_layer_counts(dag, out.ctypes.data)
    if rc != SPDZ_OK:
        raise SpdzError(rc, "layer counts")
    return out


def spdz_mul_check_noalloc(n_parties: int, field: int, stream, x: spdz_buf, y: spdz_buf, a: spdz_buf,
                           b: spdz_buf, c: spdz_buf, alpha_shares, z: spdz_buf, N: int, check_seed: int,
                           epoch: int, result) -> None:
    """Allocation-free Beaver batch plus MAC check (no context): result
    receives [n + 1] elements on the device, sigma_i then the pass flag."""
    rc = lib.spdz_mul_check_noalloc(n_parties, field, stream, C.byref(x), C.byref(y), C.byref(a),
                                    C.byref(b), C.byref(c), ptr(alpha_shares), C.byref(z), N,
                                    check_seed, epoch, ptr(result))
    if rc != SPDZ_OK:
        raise SpdzError(rc, "spdz_mul_check_noalloc failed")


# --------------------------------------------------------- cost model (MLP)

def spdz_mlp_create(n_in: int, hidden: int, hidden_layers: int, seed: int, stream=None):
    h = _vp()
    rc = lib.spdz_mlp_create(C.byref(h), n_in, hidden, hidden_layers, seed, stream)
    if rc != SPDZ_OK:
        raise SpdzError(rc, "mlp create")
    return h


def spdz_mlp_destroy(m) -> None:
    lib.spdz_mlp_destroy(m)


def spdz_mlp_num_params(m) -> int:
    c = _i64()
    _chk(None, lib.spdz_mlp_num_params(m, C.byref(c)))
    return c.value


def spdz_mlp_get_params(m) -> np.ndarray:
    out = np.zeros(spdz_mlp_num_params(m), dtype=np.float32)
    _chk(None, lib.spdz_mlp_get_params(m, out.ctypes.data))
    return out


def spdz_mlp_set_params(m, params: np.ndarray) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == spdz_mlp_num_params(m)
    _chk(None, lib.spdz_mlp_set_params(m, p.ctypes.data))


def spdz_mlp_forward(m, X, Y, B: int) -> None:
    _chk(None, lib.spdz_mlp_forward(m, ptr(X), B, ptr(Y)))


def spdz_mlp_loss_grad(m, X, T, B: int):
    loss = np.zeros(1, dtype=np.float32)
    grad = np.zeros(spdz_mlp_num_params(m), dtype=np.float32)
    _chk(None, lib.spdz_mlp_loss_grad(m, ptr(X), ptr(T), B, loss.ctypes.data, grad.ctypes.data))
    return float(loss[0]), grad


def spdz_mlp_train(m, X, T, B: int, epochs: int, batch: int, lr: float) -> float:
    loss = np.zeros(1, dtype=np.float32)
    _chk(None, lib.spdz_mlp_train(m, ptr(X), ptr(T), B, epochs, batch, lr, loss.ctypes.data))
    return float(loss[0])


def spdz_mlp_adam_step(m, grad, lr: float) -> None:
    _chk(None, lib.spdz_mlp_adam_step(m, ptr(grad), lr))


# ------------------------------------------------------------- scheduling

def spdz_sched_num_configs():
    c, f = C.c_int32(), C.c_int32()
    lib.spdz_sched_num_configs(C.byref(c), C.byref(f))
    return c.value, f.value


def spdz_sched_config_plan(dag, cfg: int) -> spdz_plan:
    p = spdz_plan()
    _chk(None, lib.spdz_sched_config_plan(dag, cfg, C.byref(p)))
    return p


def spdz_sched_record(ctx, dag, wires: spdz_buf, reps: int) -> None:
    _chk(ctx, lib.spdz_sched_record(ctx, dag, C.byref(wires), reps))


def spdz_sched_samples(ctx):
    n = _i64()
    sw = C.c_double()
    _chk(ctx, lib.spdz_sched_samples(ctx, None, None, C.byref(n), C.byref(sw)))
    _, nf = spdz_sched_num_configs()
    X = np.zeros((n.value, nf), dtype=np.float32)
    Y = np.zeros(n.value, dtype=np.float32)
    _chk(ctx, lib.spdz_sched_samples(ctx, X.ctypes.data, Y.ctypes.data, C.byref(n), C.byref(sw)))
    return X, Y, sw.value


def spdz_sched_add_samples(ctx, X: np.ndarray, Y: np.ndarray) -> None:
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float32)
    _chk(ctx, lib.spdz_sched_add_samples(ctx, X.ctypes.data, Y.ctypes.data, Y.size))


def spdz_sched_train(ctx, epochs: int, lr: float, seed: int = 1) -> float:
    loss = C.c_float()
    _chk(ctx, lib.spdz_sched_train(ctx, epochs, lr, seed, C.byref(loss)))
    return loss.value


def spdz_sched_predict(ctx, dag, cfg: int, depth: int) -> np.ndarray:
    out = np.zeros(depth, dtype=np.float32)
    _chk(ctx, lib.spdz_sched_predict(ctx, dag, cfg, out.ctypes.data))
    return out


def spdz_sched_learned_plan(ctx, dag):
    p, ms = spdz_plan(), C.c_double()
    _chk(ctx, lib.spdz_sched_learned_plan(ctx, dag, C.byref(p), C.byref(ms)))
    return p, ms.value


def spdz_sched_autotune(ctx, dag, wires: spdz_buf, reps: int):
    p, ms = spdz_plan(), C.c_double()
    _chk(ctx, lib.spdz_sched_autotune(ctx, dag, C.byref(wires), reps, C.byref(p), C.byref(ms)))
    return p, ms.value


def spdz_sched_choose(ctx, dag, wires: spdz_buf, reps: int):
    p, r = spdz_plan(), spdz_sched_report()
    _chk(ctx, lib.spdz_sched_choose(ctx, dag, C.byref(wires), reps, C.byref(p), C.byref(r)))
    return p, r


# ------------------------------------------------------------------ serving

def spdz_serve_create(n_parties: int, budget_bytes: int, max_active: int, mode: int, model_ctx=None,
                      check_seed: int = 0, cluster_width: int = 0):
    h = _vp()
    rc = lib.spdz_serve_create(C.byref(h), n_parties, budget_bytes, max_active, mode, model_ctx, check_seed,
                               cluster_width)
    if rc != SPDZ_OK:
        raise SpdzError(rc, "serve create")
    return h


def spdz_serve_destroy(server) -> None:
    lib.spdz_serve_destroy(server)


def dag_desc(dag):
    """spdz_dag_desc over a circuit's numpy arrays (kept alive on the result)."""
    arrs = (np.ascontiguousarray(dag.layer_offsets, dtype=np.int64), np.ascontiguousarray(dag.ops, dtype=np.uint8),
            np.ascontiguousarray(dag.in0, dtype=np.uint32), np.ascontiguousarray(dag.in1, dtype=np.uint32),
            np.ascontiguousarray(dag.kconst, dtype=np.uint64))
    d = spdz_dag_desc(dag.n_inputs, arrs[1].size, arrs[0].size - 1, *[a.ctypes.data for a in arrs])
    d._keep = arrs
    return d


def spdz_serve_register(server, dag, field: int) -> int:
    """Registers a circuit for any number of requests; returns its id."""
    d = dag_desc(dag)
    cid = C.c_int64()
    _chk(None, lib.spdz_serve_register(server, C.byref(d), field, C.byref(cid)))
    return cid.value


def spdz_serve_unregister(server, circuit_id: int) -> None:
    _chk(None, lib.spdz_serve_unregister(server, circuit_id))


def spdz_serve_set_mode(server, mode: int, model_ctx=None, cluster_width: int = 0) -> None:
    _chk(None, lib.spdz_serve_set_mode(server, mode, model_ctx, cluster_width))


def spdz_serve_start(server) -> None:
    _chk(None, lib.spdz_serve_start(server))


def _request(circuit, field: int, seed: int, arrival_s: float = 0.0, inputs=None, out=None):
    """A spdz_serve_request: circuit is a registered id (int) or a circuit
    object; inputs / out are (values, MACs) numpy arrays or None.  Returns the
    struct and the objects it points into."""
    r = spdz_serve_request()
    keep = []
    if isinstance(circuit, int):
        r.dag, r.circuit_id = None, circuit
    else:
        d = dag_desc(circuit)
        keep.append(d)
        r.dag, r.circuit_id = C.pointer(d), -1
    r.field, r.seed, r.arrival_s = field, seed, arrival_s
    if inputs is not None:
        iv, im = (np.ascontiguousarray(a) for a in inputs)
        keep += [iv, im]
        r.in_val_host, r.in_mac_host = iv.ctypes.data, im.ctypes.data
    if out is not None:
        assert out[0].flags.c_contiguous and out[1].flags.c_contiguous
        keep += list(out)
        r.out_val_host, r.out_mac_host = out[0].ctypes.data, out[1].ctypes.data
    return r, keep


_PENDING = {}


def spdz_serve_submit(server, circuit, field: int, seed: int, inputs=None, out=None, arrival_s: float = 0.0) -> int:
    """Submits one request; the buffers stay referenced until it is polled done."""
    r, keep = _request(circuit, field, seed, arrival_s, inputs, out)
    rid = C.c_uint64()
    _chk(None, lib.spdz_serve_submit(server, C.byref(r), C.byref(rid)))
    _PENDING[(server.value if hasattr(server, "value") else server, rid.value)] = (r, keep)
    return rid.value


def spdz_serve_poll(server, req_id: int):
    """(done, spdz_serve_result or None)."""
    done = C.c_int32()
    res = spdz_serve_result()
    _chk(None, lib.spdz_serve_poll(server, req_id, C.byref(done), C.byref(res)))
    if done.value:
        _PENDING.pop((server.value if hasattr(server, "value") else server, req_id), None)
        return True, res
    return False, None


def spdz_serve_stop(server) -> spdz_serve_stats:
    st = spdz_serve_stats()
    _chk(None, lib.spdz_serve_stop(server, C.byref(st)))
    return st


def spdz_serve_run(server, requests):
    """requests: list of (circuit or registered id, field, seed, arrival_s,
    out_val or None, out_mac or None).  Returns (results list, spdz_serve_stats)."""
    n = len(requests)
    arr = (spdz_serve_request * max(1, n))()
    keep = []
    for k, (circ, field, seed, t, ov, om) in enumerate(requests):
        r, kp = _request(circ, field, seed, t, None, None if ov is None else (ov, om))
        keep.append(kp)
        arr[k] = r
    res = (spdz_serve_result * max(1, n))()
    st = spdz_serve_stats()
    rc = lib.spdz_serve_run(server, arr, n, res, C.byref(st))
    if rc != SPDZ_OK:
        raise SpdzError(rc, "serve run")
    return [res[k] for k in range(n)], st


# --------------------------------------------------------- matrix products

def spdz_deal_matrix_triple(ctx, seed: int, sub: int, m: int, k: int, n: int, alpha_shares, A: spdz_buf,
                            B: spdz_buf, Cb: spdz_buf) -> None:
    _chk(ctx, lib.spdz_deal_matrix_triple(ctx, seed, sub, m, k, n, ptr(alpha_shares), C.byref(A), C.byref(B),
                                          C.byref(Cb)))


def spdz_load_matrix_preproc(ctx, A: spdz_buf, B: spdz_buf, Cb: spdz_buf, m: int, k: int, n: int) -> None:
    _chk(ctx, lib.spdz_load_matrix_preproc(ctx, C.byref(A), C.byref(B), C.byref(Cb), m, k, n))


def spdz_matmul(ctx, X: spdz_buf, Y: spdz_buf, Z: spdz_buf, m: int, k: int, n: int, path: int,
                E_out=None, F_out=None) -> None:
    _chk(ctx, lib.spdz_matmul(ctx, C.byref(X), C.byref(Y), C.byref(Z), m, k, n, path, ptr(E_out), ptr(F_out)))


# ------------------------------------------------------------ linear layer

def spdz_deal_matvec_triples(ctx, seed: int, sub: int, dout: int, din: int, tile_rows: int, alpha_shares,
                             A: spdz_buf, B: spdz_buf, Cb: spdz_buf) -> None:
    _chk(ctx, lib.spdz_deal_matvec_triples(ctx, seed, sub, dout, din, tile_rows, ptr(alpha_shares), C.byref(A),
                                           C.byref(B), C.byref(Cb)))


def spdz_load_matvec_preproc(ctx, A: spdz_buf, B: spdz_buf, Cb: spdz_buf, dout: int, din: int, tile_rows: int) -> None:
    _chk(ctx, lib.spdz_load_matvec_preproc(ctx, C.byref(A), C.byref(B), C.byref(Cb), dout, din, tile_rows))


def spdz_linear_layer(ctx, W: spdz_buf, x: spdz_buf, b: spdz_buf, y: spdz_buf, dout: int, din: int, tile_rows: int,
                      D_out=None, E_out=None) -> None:
    _chk(ctx, lib.spdz_linear_layer(ctx, C.byref(W), C.byref(x), C.byref(b), C.byref(y), dout, din, tile_rows,
                                    ptr(D_out), ptr(E_out)))


# --------------------------------------------------------- inputs, outputs

def spdz_deal_input_masks(ctx, seed: int, owner: int, j0: int, count: int, alpha_shares, masks: spdz_buf,
                          r_clear) -> None:
    _chk(ctx, lib.spdz_deal_input_masks(ctx, seed, owner, j0, count, ptr(alpha_shares), C.byref(masks),
                                        ptr(r_clear)))


def spdz_input(ctx, x, r_clear, masks: spdz_buf, out: spdz_buf, N: int, eps_out=None) -> None:
    _chk(ctx, lib.spdz_input(ctx, ptr(x), ptr(r_clear), C.byref(masks), C.byref(out), N, ptr(eps_out)))


def spdz_reveal(ctx, x: spdz_buf, out, N: int, sigma_host=None) -> bool:
    """Opens and checks; True when the check passed (the values are in out),
    False when it failed (out zeroed)."""
    ok = _int(0)
    rc = lib.spdz_reveal(ctx, C.byref(x), ptr(out), N, C.byref(ok), ptr(sigma_host))
    if rc not in (SPDZ_OK, SPDZ_ERR_MAC):
        _chk(ctx, rc)
    return bool(ok.value)


# ------------------------------------------------------------ measurement

def spdz_int_peak(kind: int, iters: int, stream, scratch) -> float:
    """Thread-level integer instructions per second of one kind (see spdz.h)."""
    r = C.c_double()
    _chk(None, lib.spdz_int_peak(kind, iters, stream, ptr(scratch), C.byref(r)))
    return r.value


# ------------------------------------------------------------ party per GPU

def spdz_party_create(party: int, n_parties: int, field: int, stream=None):
    h = _vp()
    _chk(None, lib.spdz_party_create(C.byref(h), party, n_parties, field, stream))
    return h


def spdz_party_destroy(p) -> None:
    lib.spdz_party_destroy(p)


def spdz_party_load_alpha(p, alpha_share) -> None:
    _chk(None, lib.spdz_party_load_alpha(p, ptr(alpha_share)))


def spdz_party_set_check_seed(p, seed: int) -> None:
    _chk(None, lib.spdz_party_set_check_seed(p, seed))


def spdz_party_mask(p, x: spdz_buf, y: spdz_buf, a: spdz_buf, b: spdz_buf, eps, dlt, N: int) -> None:
    _chk(None, lib.spdz_party_mask(p, C.byref(x), C.byref(y), C.byref(a), C.byref(b), ptr(eps), ptr(dlt), N))


def spdz_party_open_sum(p, rows, N: int, out) -> None:
    _chk(None, lib.spdz_party_open_sum(p, ptr(rows), N, ptr(out)))


def spdz_party_combine(p, eps, dlt, x: spdz_buf, y: spdz_buf, a: spdz_buf, b: spdz_buf, c: spdz_buf, z: spdz_buf,
                       N: int) -> None:
    _chk(None, lib.spdz_party_combine(p, ptr(eps), ptr(dlt), C.byref(x), C.byref(y), C.byref(a), C.byref(b),
                                      C.byref(c), C.byref(z), N))


def spdz_party_sigma(p, words: int):
    """(sigma_i as 64-bit words [words], values opened in the epoch)."""
    out = np.zeros(words, dtype=np.uint64)
    opened = _i64()
    _chk(None, lib.spdz_party_sigma(p, out.ctypes.data, C.byref(opened)))
    return out, opened.value
