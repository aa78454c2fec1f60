"""CPU oracle for the SPDZ online phase -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is a plain, slow simulation of all
parties share by share, written from the paper's definitions (arXiv
2512.11112, Sec. II-A and III-D) in C (``spdz_oracle.c``) with a generic
prime; this module only marshals numpy arrays to it.  It shares no code with
the CUDA path.

Array conventions: a field element is one uint64 (p < 2^64) or two uint64
words, little-endian (p < 2^127).  Share arrays are ``[n, count]`` or
``[n, count, 2]``.  Secrets and public values are ``[count]`` or
``[count, 2]``.

Parity status: see the header of ``spdz_oracle.c`` -- every function is pinned
by tests/test_oracle_pins.py except the individual share values of the
dealer, which only the PRG specification fixes.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

P61 = (1 << 61) - 1
P127 = (1 << 127) - 1
P32 = (1 << 32) - 5        # the prime of the paper's evaluation (Sec. IV-A)
OP_ADD, OP_SUB, OP_CMUL, OP_CADD, OP_MUL = 0, 1, 2, 3, 4
K_ALPHA, K_TRIPLE_A, K_TRIPLE_B, K_TRIPLE_C, K_INPUT, K_CHECK = 1, 2, 3, 4, 5, 6
K_MTRIPLE_A, K_MTRIPLE_B, K_MTRIPLE_C = 7, 8, 9
K_INPUT_MASK = 10          # masks of private inputs (sub = the owning party)
R_SECRET, R_VAL_SHARE, R_MAC_SHARE = 0, 1, 2

_lib = None
_u64p = C.POINTER(C.c_uint64)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _lib.orc_sm64.restype = C.c_uint64
        _lib.orc_sm64.argtypes = [C.c_uint64, C.c_uint64]
        _lib.orc_stream_id.restype = C.c_uint64
        _lib.orc_stream_id.argtypes = [C.c_uint64] * 4
        _lib.orc_stream_key.restype = C.c_uint64
        _lib.orc_stream_key.argtypes = [C.c_uint64, C.c_uint64]
        _lib.orc_check_finish.restype = C.c_int
        _lib.orc_get_threads.restype = C.c_int
    return _lib


def words(p: int) -> int:
    return 1 if p < (1 << 64) else 2


def _pp(p: int):
    return C.c_uint64(p & (2**64 - 1)), C.c_uint64(p >> 64)


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"], "uint64 C-contiguous arrays only"
    return a.ctypes.data_as(_u64p)


def _shape(p: int, *dims) -> tuple:
    return tuple(dims) + ((2,) if words(p) == 2 else ())


def zeros(p: int, *dims) -> np.ndarray:
    return np.zeros(_shape(p, *dims), dtype=np.uint64)


def to_array(p: int, values) -> np.ndarray:
    """Python ints -> element array."""
    vals = [int(v) % p for v in values]
    if words(p) == 1:
        return np.array(vals, dtype=np.uint64)
    return np.array([[v & (2**64 - 1), v >> 64] for v in vals], dtype=np.uint64).reshape(-1, 2)


def to_ints(p: int, arr: np.ndarray) -> list:
    """Element array -> flat list of Python ints."""
    a = np.ascontiguousarray(arr, dtype=np.uint64)
    if words(p) == 1:
        return [int(v) for v in a.reshape(-1)]
    a = a.reshape(-1, 2)
    return [int(lo) | (int(hi) << 64) for lo, hi in a]


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def get_threads() -> int:
    return int(lib().orc_get_threads())


# ------------------------------------------------------------------ scalars

def fop(p: int, name: str, a: int, b: int) -> int:
    x, y, out = to_array(p, [a]), to_array(p, [b]), zeros(p, 1)
    getattr(lib(), "orc_f" + name)(*_pp(p), _ptr(x), _ptr(y), _ptr(out))
    return to_ints(p, out)[0]


def sm64(key: int, i: int) -> int:
    return int(lib().orc_sm64(key, i))


def stream_id(kind: int, role: int, party: int, sub: int) -> int:
    return int(lib().orc_stream_id(kind, role, party, sub))


def draw(p: int, seed: int, stream: int, j0: int, count: int) -> np.ndarray:
    out = zeros(p, count)
    lib().orc_draw(*_pp(p), C.c_uint64(seed), C.c_uint64(stream), C.c_uint64(j0),
                   C.c_int64(count), _ptr(out))
    return out


# ------------------------------------------------------------------- dealer

def deal_alpha(p: int, n: int, seed: int):
    """Returns (alpha [w], alpha shares [n, w])."""
    a, sh = zeros(p, 1), zeros(p, n)
    lib().orc_deal_alpha(*_pp(p), C.c_int(n), C.c_uint64(seed), _ptr(a), _ptr(sh))
    return a[0], sh


def deal_shared(p: int, n: int, seed: int, kind: int, sub: int, j0: int, count: int,
                alpha, secret=None):
    """Returns (val [n, count], mac [n, count], secret [count])."""
    al = np.ascontiguousarray(np.asarray(alpha, dtype=np.uint64).reshape(-1))
    sec_in = None if secret is None else np.ascontiguousarray(secret, dtype=np.uint64)
    v, m, s = zeros(p, n, count), zeros(p, n, count), zeros(p, count)
    lib().orc_deal_shared(*_pp(p), C.c_int(n), C.c_uint64(seed), C.c_uint64(kind),
                          C.c_uint64(sub), C.c_uint64(j0), C.c_int64(count), _ptr(al),
                          _ptr(sec_in), _ptr(v), _ptr(m), _ptr(s))
    return v, m, (s if secret is None else sec_in)


@dataclass
class Triples:
    av: np.ndarray
    am: np.ndarray
    bv: np.ndarray
    bm: np.ndarray
    cv: np.ndarray
    cm: np.ndarray

    def slice(self, lo: int, hi: int) -> "Triples":
        return Triples(*[np.ascontiguousarray(x[:, lo:hi]) for x in
                         (self.av, self.am, self.bv, self.bm, self.cv, self.cm)])


def deal_triples(p: int, n: int, seed: int, j0: int, count: int, alpha) -> Triples:
    al = np.ascontiguousarray(np.asarray(alpha, dtype=np.uint64).reshape(-1))
    arrs = [zeros(p, n, count) for _ in range(6)]
    lib().orc_deal_triples(*_pp(p), C.c_int(n), C.c_uint64(seed), C.c_uint64(j0),
                           C.c_int64(count), _ptr(al), *[_ptr(a) for a in arrs])
    return Triples(*arrs)


def deal_matrix_triple(p: int, n: int, seed: int, sub: int, M: int, K: int, N: int, alpha):
    al = np.ascontiguousarray(np.asarray(alpha, dtype=np.uint64).reshape(-1))
    Av, Am = zeros(p, n, M * K), zeros(p, n, M * K)
    Bv, Bm = zeros(p, n, K * N), zeros(p, n, K * N)
    Cv, Cm = zeros(p, n, M * N), zeros(p, n, M * N)
    lib().orc_deal_matrix_triple(*_pp(p), C.c_int(n), C.c_uint64(seed), C.c_uint64(sub),
                                 C.c_int64(M), C.c_int64(K), C.c_int64(N), _ptr(al),
                                 _ptr(Av), _ptr(Am), _ptr(Bv), _ptr(Bm), _ptr(Cv), _ptr(Cm))
    return Triples(Av, Am, Bv, Bm, Cv, Cm)


def deal_matvec_triples(p: int, n: int, seed: int, sub: int, dout: int, din: int, R: int, alpha) -> Triples:
    """Per-tile matrix-vector triples of a row-tiled linear layer: A [n, dout*din],
    B [n, T*din], C [n, dout] (C_t = A_t B_t), T = ceil(dout / R)."""
    al = np.ascontiguousarray(np.asarray(alpha, dtype=np.uint64).reshape(-1))
    T = -(-dout // R)
    Av, Am = zeros(p, n, dout * din), zeros(p, n, dout * din)
    Bv, Bm = zeros(p, n, T * din), zeros(p, n, T * din)
    Cv, Cm = zeros(p, n, dout), zeros(p, n, dout)
    lib().orc_deal_matvec_triples(*_pp(p), C.c_int(n), C.c_uint64(seed), C.c_uint64(sub), C.c_int64(dout),
                                  C.c_int64(din), C.c_int64(R), _ptr(al), _ptr(Av), _ptr(Am), _ptr(Bv),
                                  _ptr(Bm), _ptr(Cv), _ptr(Cm))
    return Triples(Av, Am, Bv, Bm, Cv, Cm)


# ---------------------------------------------------------------- protocol

def linear(p: int, op: int, xv, xm, yv, ym, k, alpha_sh):
    n, count = xv.shape[0], xv.shape[1]
    zv, zm = zeros(p, n, count), zeros(p, n, count)
    kk = to_array(p, [0 if k is None else k])
    lib().orc_linear(*_pp(p), C.c_int(n), C.c_int(op), C.c_int64(count), _ptr(xv), _ptr(xm),
                     _ptr(yv), _ptr(ym), _ptr(kk), _ptr(alpha_sh), _ptr(zv), _ptr(zm))
    return zv, zm


def open_(p: int, xv) -> np.ndarray:
    n, count = xv.shape[0], xv.shape[1]
    out = zeros(p, count)
    lib().orc_open(*_pp(p), C.c_int(n), C.c_int64(count), _ptr(xv), _ptr(out))
    return out


@dataclass
class OpenLog:
    """Opened values (in opening order) and their MAC shares [n, m]."""
    vals: np.ndarray
    macs: np.ndarray


def mul(p: int, xv, xm, yv, ym, tri: Triples, alpha_sh):
    """Beaver batch.  Returns (zv, zm, eps, dlt, OpenLog) where the log holds
    eps_j at 2j and delta_j at 2j+1."""
    n, count = xv.shape[0], xv.shape[1]
    zv, zm = zeros(p, n, count), zeros(p, n, count)
    eps, dlt = zeros(p, count), zeros(p, count)
    em, dm = zeros(p, n, count), zeros(p, n, count)
    lib().orc_mul(*_pp(p), C.c_int(n), C.c_int64(count), _ptr(xv), _ptr(xm), _ptr(yv), _ptr(ym),
                  _ptr(tri.av), _ptr(tri.am), _ptr(tri.bv), _ptr(tri.bm), _ptr(tri.cv),
                  _ptr(tri.cm), _ptr(alpha_sh), _ptr(zv), _ptr(zm), _ptr(eps), _ptr(dlt),
                  _ptr(em), _ptr(dm))
    return zv, zm, eps, dlt, interleave_log(p, eps, dlt, em, dm)


def interleave_log(p, eps, dlt, em, dm) -> OpenLog:
    """Opening order of a Beaver batch: eps_0, delta_0, eps_1, delta_1, ..."""
    count = eps.shape[0]
    vals = np.stack([eps, dlt], axis=1).reshape(_shape(p, 2 * count))
    n = em.shape[0]
    macs = np.stack([em, dm], axis=2).reshape(_shape(p, n, 2 * count))
    return OpenLog(np.ascontiguousarray(vals), np.ascontiguousarray(macs))


def innerprod(p: int, P: int, L: int, xv, xm, yv, ym, tri: Triples, alpha_sh):
    n = xv.shape[0]
    T = P * L
    zv, zm = zeros(p, n, P), zeros(p, n, P)
    eps, dlt = zeros(p, T), zeros(p, T)
    em, dm = zeros(p, n, T), zeros(p, n, T)
    lib().orc_innerprod(*_pp(p), C.c_int(n), C.c_int64(P), C.c_int64(L), _ptr(xv), _ptr(xm),
                        _ptr(yv), _ptr(ym), _ptr(tri.av), _ptr(tri.am), _ptr(tri.bv),
                        _ptr(tri.bm), _ptr(tri.cv), _ptr(tri.cm), _ptr(alpha_sh), _ptr(zv),
                        _ptr(zm), _ptr(eps), _ptr(dlt), _ptr(em), _ptr(dm))
    return zv, zm, eps, dlt, interleave_log(p, eps, dlt, em, dm)


def check_coeffs(p: int, check_seed: int, epoch: int, j0: int, m: int) -> np.ndarray:
    r = zeros(p, m)
    lib().orc_check_coeffs(*_pp(p), C.c_uint64(check_seed), C.c_uint64(epoch),
                           C.c_uint64(j0), C.c_int64(m), _ptr(r))
    return r


def rlc(p: int, log: OpenLog, check_seed: int, epoch: int, j0: int = 0):
    """(A, S [n]) of one chunk of the opened log whose first entry has index j0."""
    n = log.macs.shape[0]
    m = log.vals.shape[0]
    A, S = zeros(p, 1), zeros(p, n)
    lib().orc_rlc(*_pp(p), C.c_int(n), C.c_int64(m), _ptr(log.vals), _ptr(log.macs),
                  C.c_uint64(check_seed), C.c_uint64(epoch), C.c_uint64(j0), _ptr(A), _ptr(S))
    return A[0], S


def check_finish(p: int, A, S, alpha_sh):
    n = S.shape[0]
    sigma = zeros(p, n)
    Aa = np.ascontiguousarray(np.asarray(A, dtype=np.uint64).reshape(-1))
    ok = lib().orc_check_finish(*_pp(p), C.c_int(n), _ptr(Aa), _ptr(np.ascontiguousarray(S)),
                                _ptr(alpha_sh), _ptr(sigma))
    return sigma, bool(ok)


def mac_check(p: int, logs, alpha_sh, check_seed: int, epoch: int):
    """Check over the concatenation of ``logs`` (opening order); returns
    (passed, sigma [n], A, S)."""
    vals = np.concatenate([l.vals for l in logs], axis=0)
    macs = np.concatenate([l.macs for l in logs], axis=1)
    A, S = rlc(p, OpenLog(np.ascontiguousarray(vals), np.ascontiguousarray(macs)),
               check_seed, epoch, 0)
    sigma, ok = check_finish(p, A, S, alpha_sh)
    return ok, sigma, A, S


def mat_open(p: int, M, K, N, X: Triples | tuple, Y, tri: Triples):
    """E = sum(X_i - A_i), F = sum(Y_i - B_i) and their MAC shares."""
    n = tri.av.shape[0]
    Xv, Xm = X
    Yv, Ym = Y
    E, F = zeros(p, M * K), zeros(p, K * N)
    Em, Fm = zeros(p, n, M * K), zeros(p, n, K * N)
    lib().orc_mat_open(*_pp(p), C.c_int(n), C.c_int64(M), C.c_int64(K), C.c_int64(N),
                       _ptr(Xv), _ptr(Xm), _ptr(Yv), _ptr(Ym), _ptr(tri.av), _ptr(tri.am),
                       _ptr(tri.bv), _ptr(tri.bm), _ptr(E), _ptr(F), _ptr(Em), _ptr(Fm))
    return E, F, Em, Fm


def mat_entries(p: int, M, K, N, E, F, tri: Triples, alpha_sh, rows, cols):
    n = tri.av.shape[0]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    Zv, Zm = zeros(p, n, rows.size), zeros(p, n, rows.size)
    lib().orc_mat_entries(*_pp(p), C.c_int(n), C.c_int64(M), C.c_int64(K), C.c_int64(N),
                          _ptr(E), _ptr(F), _ptr(tri.av), _ptr(tri.am), _ptr(tri.bv),
                          _ptr(tri.bm), _ptr(tri.cv), _ptr(tri.cm), _ptr(alpha_sh),
                          C.c_int64(rows.size), rows.ctypes.data_as(C.POINTER(C.c_int64)),
                          cols.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(Zv), _ptr(Zm))
    return Zv, Zm


def linear_layer(p: int, dout: int, din: int, R: int, W, x, b, tri: Triples, alpha_sh, rows=None):
    """y = W x + b with row tiles of R rows (one matvec triple per tile): the
    shares (yv, ym) [n, len(rows)] of the listed rows (all rows by default).
    W, x, b are (values, MACs) pairs of [n, .] arrays."""
    n = tri.av.shape[0]
    rows = np.arange(dout, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    yv, ym = zeros(p, n, rows.size), zeros(p, n, rows.size)
    lib().orc_linear_layer(*_pp(p), C.c_int(n), C.c_int64(dout), C.c_int64(din), C.c_int64(R),
                           _ptr(W[0]), _ptr(W[1]), _ptr(x[0]), _ptr(x[1]), _ptr(b[0]), _ptr(b[1]),
                           _ptr(tri.av), _ptr(tri.am), _ptr(tri.bv), _ptr(tri.bm), _ptr(tri.cv), _ptr(tri.cm),
                           _ptr(alpha_sh), C.c_int64(rows.size), rows.ctypes.data_as(C.POINTER(C.c_int64)),
                           _ptr(yv), _ptr(ym))
    return yv, ym


def linear_open(p: int, dout: int, din: int, R: int, W, x, tri: Triples) -> OpenLog:
    """The layer's opened values in log order (per tile: E_t, then D_t row by
    row) with their MAC shares."""
    n = tri.av.shape[0]
    T = -(-dout // R)
    m = T * din + dout * din
    vals, macs = zeros(p, m), zeros(p, n, m)
    lib().orc_linear_open(*_pp(p), C.c_int(n), C.c_int64(dout), C.c_int64(din), C.c_int64(R),
                          _ptr(W[0]), _ptr(W[1]), _ptr(x[0]), _ptr(x[1]), _ptr(tri.av), _ptr(tri.am),
                          _ptr(tri.bv), _ptr(tri.bm), _ptr(vals), _ptr(macs))
    return OpenLog(vals, macs)


def linear_rlc(p: int, dout: int, din: int, R: int, W, x, tri: Triples, check_seed: int, epoch: int,
               j0: int = 0):
    """(A, S [n]) of the layer's whole log, streamed (the log is not stored)."""
    n = tri.av.shape[0]
    A, S = zeros(p, 1), zeros(p, n)
    lib().orc_linear_rlc(*_pp(p), C.c_int(n), C.c_int64(dout), C.c_int64(din), C.c_int64(R),
                         _ptr(W[0]), _ptr(W[1]), _ptr(x[0]), _ptr(x[1]), _ptr(tri.av), _ptr(tri.am),
                         _ptr(tri.bv), _ptr(tri.bm), C.c_uint64(check_seed), C.c_uint64(epoch),
                         C.c_uint64(j0), _ptr(A), _ptr(S))
    return A[0], S


def deal_input_masks(p: int, n: int, seed: int, owner: int, j0: int, count: int, alpha):
    """Masks for inputs owned by party `owner`: (rv, rm) shares [n, count] and
    the clear masks r [count] the owner holds (kind INPUT_MASK, sub = owner)."""
    return deal_shared(p, n, seed, K_INPUT_MASK, owner, j0, count, alpha)


def input_share(p: int, x, r_clear, rv, rm, alpha_sh):
    """The owner publishes eps = x - r; [x] = [r] + eps.  Returns (xv, xm, eps)."""
    n, count = rv.shape[0], rv.shape[1]
    xv, xm, eps = zeros(p, n, count), zeros(p, n, count), zeros(p, count)
    lib().orc_input(*_pp(p), C.c_int(n), C.c_int64(count), _ptr(np.ascontiguousarray(x)),
                    _ptr(np.ascontiguousarray(r_clear)), _ptr(rv), _ptr(rm), _ptr(alpha_sh), _ptr(xv), _ptr(xm),
                    _ptr(eps))
    return xv, xm, eps


def dag_eval(p: int, dag, wv, wm, tri: Triples, alpha_sh):
    """Evaluates the circuit in gate order on the shared wires [n, W] (inputs
    filled in); returns (eps, dlt, OpenLog).  ``tri`` holds at least n_mul
    triples, the first consumed first."""
    n = wv.shape[0]
    T = tri.av.shape[1]
    nm = int(np.count_nonzero(dag.ops == OP_MUL))
    eps, dlt = zeros(p, nm), zeros(p, nm)
    em, dm = zeros(p, n, nm), zeros(p, n, nm)
    ops = np.ascontiguousarray(dag.ops, dtype=np.uint8)
    in0 = np.ascontiguousarray(dag.in0, dtype=np.uint32)
    in1 = np.ascontiguousarray(dag.in1, dtype=np.uint32)
    k = np.ascontiguousarray(dag.kconst, dtype=np.uint64)
    lib().orc_dag_eval(*_pp(p), C.c_int(n), C.c_int64(dag.n_inputs), C.c_int64(dag.n_gates),
                       ops.ctypes.data_as(C.POINTER(C.c_uint8)),
                       in0.ctypes.data_as(C.POINTER(C.c_uint32)),
                       in1.ctypes.data_as(C.POINTER(C.c_uint32)), _ptr(k), _ptr(alpha_sh),
                       _ptr(wv), _ptr(wm), C.c_int64(T), _ptr(tri.av), _ptr(tri.am),
                       _ptr(tri.bv), _ptr(tri.bm), _ptr(tri.cv), _ptr(tri.cm),
                       _ptr(eps), _ptr(dlt), _ptr(em), _ptr(dm))
    return eps, dlt, interleave_log(p, eps, dlt, em, dm)


def dag_eval_layers(p: int, dag, wv, wm, tri: Triples, alpha_sh):
    """The same evaluation as dag_eval, layer by layer with each layer's gates
    spread over the oracle's threads (set_threads); returns the same
    (eps, dlt, OpenLog)."""
    n = wv.shape[0]
    T = tri.av.shape[1]
    nm = int(np.count_nonzero(dag.ops == OP_MUL))
    eps, dlt = zeros(p, nm), zeros(p, nm)
    em, dm = zeros(p, n, nm), zeros(p, n, nm)
    ops = np.ascontiguousarray(dag.ops, dtype=np.uint8)
    in0 = np.ascontiguousarray(dag.in0, dtype=np.uint32)
    in1 = np.ascontiguousarray(dag.in1, dtype=np.uint32)
    k = np.ascontiguousarray(dag.kconst, dtype=np.uint64)
    off = np.ascontiguousarray(dag.layer_offsets, dtype=np.int64)
    rc = lib().orc_dag_eval_layers(*_pp(p), C.c_int(n), C.c_int64(dag.n_inputs), C.c_int64(dag.n_gates),
                                   C.c_int(off.size - 1), off.ctypes.data_as(C.POINTER(C.c_int64)),
                                   ops.ctypes.data_as(C.POINTER(C.c_uint8)),
                                   in0.ctypes.data_as(C.POINTER(C.c_uint32)),
                                   in1.ctypes.data_as(C.POINTER(C.c_uint32)), _ptr(k), _ptr(alpha_sh),
                                   _ptr(wv), _ptr(wm), C.c_int64(T), _ptr(tri.av), _ptr(tri.am),
                                   _ptr(tri.bv), _ptr(tri.bm), _ptr(tri.cv), _ptr(tri.cm),
                                   _ptr(eps), _ptr(dlt), _ptr(em), _ptr(dm))
    if rc != 0:
        raise ValueError("dag_eval_layers: an operand is not written before its layer")
    return eps, dlt, interleave_log(p, eps, dlt, em, dm)


def dag_clear(p: int, dag, inputs) -> np.ndarray:
    """Cleartext evaluation: wires [W] from the input secrets [n_inputs]."""
    wires = zeros(p, dag.n_wires)
    wires[:dag.n_inputs] = inputs
    ops = np.ascontiguousarray(dag.ops, dtype=np.uint8)
    in0 = np.ascontiguousarray(dag.in0, dtype=np.uint32)
    in1 = np.ascontiguousarray(dag.in1, dtype=np.uint32)
    k = np.ascontiguousarray(dag.kconst, dtype=np.uint64)
    lib().orc_dag_clear(*_pp(p), C.c_int64(dag.n_inputs), C.c_int64(dag.n_gates),
                        ops.ctypes.data_as(C.POINTER(C.c_uint8)),
                        in0.ctypes.data_as(C.POINTER(C.c_uint32)),
                        in1.ctypes.data_as(C.POINTER(C.c_uint32)), _ptr(k), _ptr(wires))
    return wires


def reconstruct(p: int, shares) -> list:
    """Sum of the shares over parties, as Python ints (uses orc_open)."""
    return to_ints(p, open_(p, np.ascontiguousarray(shares)))
