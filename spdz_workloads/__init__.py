"""Seeded synthetic workloads for the SPDZ online phase.

This module is the one input generator that both the CUDA path and the CPU
oracle may use.  It draws *structure* only (circuit shapes, gate kinds,
wiring, public constants, request sizes and arrival times) and holds none of
the protocol's arithmetic: no field operation, no sharing, no MAC.  The
secret-shared values themselves are produced by each side's own dealer from
the counter PRG specification.

Random numbers here come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014)
in counter form, ``sm64(key, i) = mix(key + (i + 1) * GAMMA)``, vectorised
with numpy; only this module uses this copy.

Workloads follow the paper's setting (arXiv 2512.11112): arithmetic circuits
whose independent gates are grouped into batches (Sec. III-B), evaluated
layer by layer.  Shapes follow the benchmark configurations:

* ``layered_dag(...)``: a layered circuit of ``total_gates`` gates in
  ``depth`` layers, widths log-uniform in ``[wmin, wmax]`` scaled to the total,
  gate kinds in exact counts shuffled over the circuit, ``in0`` drawn from the
  previous layer (which fixes the depth) and ``in1`` from every earlier wire.
* ``serving_requests(...)``: Poisson arrivals of circuits with log-uniform
  gate counts and uniform depths, each field p61 or p127 with probability 1/2.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

P61 = (1 << 61) - 1
P127 = (1 << 127) - 1
P32 = (1 << 32) - 5

# gate opcodes shared by the circuit format, the C ABI and the oracle
OP_ADD, OP_SUB, OP_CMUL, OP_CADD, OP_MUL = 0, 1, 2, 3, 4
OP_NAMES = {"add": OP_ADD, "sub": OP_SUB, "cmul": OP_CMUL, "cadd": OP_CADD, "mul": OP_MUL}

# The benchmark circuit's gate-kind counts: 60% Beaver mul, 30% add/sub read
# as 15% add + 15% sub, 10% public-constant mul, of 2^20 gates.
CONFIG2_MIX = {"mul": 629146, "add": 157286, "sub": 157286, "cmul": 104858}

# stream ids of this module's own draws (kept apart from the dealer's kinds)
_S_WIDTH, _S_OPS, _S_IN0, _S_IN1, _S_CONST, _S_REQ = 101, 102, 103, 104, 105, 106


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def sm64(key: int, idx) -> np.ndarray:
    """Outputs ``idx`` (array of counters) of SplitMix64 started at ``key``."""
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (i + np.uint64(1)) * GAMMA
    return _mix(z)


def stream_key(seed: int, stream: int) -> int:
    return int(sm64(seed & (2**64 - 1), np.array([stream], dtype=np.uint64))[0])


def draws(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    key = stream_key(seed, stream)
    return sm64(key, np.arange(start, start + count, dtype=np.uint64))


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each draw."""
    return (draws(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 2**53)


def uniform_int(seed: int, stream: int, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """One integer per entry, uniform in [lo, hi) (hi > lo), by reduction of
    a 64-bit draw (bias below 2^-40 for the ranges used here)."""
    lo = np.asarray(lo, dtype=np.uint64)
    hi = np.asarray(hi, dtype=np.uint64)
    d = draws(seed, stream, lo.size)
    return (lo + d % (hi - lo)).astype(np.uint64)


def layer_widths(seed: int, total: int, depth: int, wmin: float, wmax: float,
                 stream: int = _S_WIDTH) -> np.ndarray:
    """``depth`` integer widths, log-uniform in [wmin, wmax], summing to ``total``.

    Draw depth values uniformly in log space, then scale multiplicatively to the
    total and clamp to [wmin, wmax], repeating until stable; round down and give
    the remainder +1 at a time to the widest layers still below wmax.
    """
    if not (depth * wmin <= total <= depth * wmax):
        raise ValueError("total gates outside [depth*wmin, depth*wmax]")
    u = uniform01(seed, stream, depth)
    w = np.exp(math.log(wmin) + (math.log(wmax) - math.log(wmin)) * u)
    for _ in range(1000):
        w = np.clip(w * (total / w.sum()), wmin, wmax)
        if abs(w.sum() - total) < 0.5:
            break
    wi = np.floor(w).astype(np.int64)
    wi = np.clip(wi, int(math.ceil(wmin)), int(wmax))
    rem = int(total - wi.sum())
    order = np.argsort(-w, kind="stable")
    while rem != 0:
        moved = False
        for k in order:
            if rem > 0 and wi[k] < wmax:
                wi[k] += 1
                rem -= 1
                moved = True
            elif rem < 0 and wi[k] > wmin:
                wi[k] -= 1
                rem += 1
                moved = True
            if rem == 0:
                break
        if not moved:
            raise ValueError("cannot meet the total within the width bounds")
    return wi


def random_constants(seed: int, stream: int, count: int, p: int) -> np.ndarray:
    """Public constants uniform in [1, p): shape [count] (p61, p32) or [count, 2] (p127)."""
    if p in (P61, P32):
        d = draws(seed, stream, count)
        return (np.uint64(1) + d % np.uint64(p - 1)).astype(np.uint64)
    if p == P127:
        d = draws(seed, stream, 2 * count).reshape(count, 2)
        out = d.copy()
        out[:, 1] >>= np.uint64(1)                       # top 63 bits: value < 2^127
        zero = (out[:, 0] == 0) & (out[:, 1] == 0)
        full = (out[:, 0] == np.uint64(2**64 - 1)) & (out[:, 1] == np.uint64(2**63 - 1))
        out[zero | full] = np.array([1, 0], dtype=np.uint64)
        return out
    raise ValueError("unsupported prime")


@dataclass
class Dag:
    """A layered straight-line circuit.

    Gate ``g`` reads wires ``in0[g]`` and ``in1[g]`` and writes wire
    ``n_inputs + g``; gates ``layer_offsets[k] .. layer_offsets[k+1]-1`` form
    layer ``k`` and depend only on earlier layers.  ``kconst[g]`` is the public
    constant of a CMUL/CADD gate (zero elsewhere).  The t-th MUL gate in gate
    order consumes triple t of the run.
    """

    p: int
    n_inputs: int
    ops: np.ndarray            # uint8 [G]
    in0: np.ndarray            # uint32 [G]
    in1: np.ndarray            # uint32 [G]
    kconst: np.ndarray         # uint64 [G] or [G, 2]
    layer_offsets: np.ndarray  # int64 [depth + 1]
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_gates(self) -> int:
        return int(self.ops.size)

    @property
    def depth(self) -> int:
        return int(self.layer_offsets.size - 1)

    @property
    def n_wires(self) -> int:
        return self.n_inputs + self.n_gates

    @property
    def n_mul(self) -> int:
        return int(np.count_nonzero(self.ops == OP_MUL))

    @property
    def widths(self) -> np.ndarray:
        return np.diff(self.layer_offsets)

    @property
    def words(self) -> int:
        return 1 if self.p == P61 else 2


def _mix_counts(mix: dict, total: int) -> dict:
    """Exact integer counts for a proportional mix (largest remainder)."""
    s = sum(mix.values())
    raw = {k: v * total / s for k, v in mix.items()}
    cnt = {k: int(math.floor(r)) for k, r in raw.items()}
    rem = total - sum(cnt.values())
    for k in sorted(raw, key=lambda k: raw[k] - cnt[k], reverse=True)[:rem]:
        cnt[k] += 1
    return cnt


def dag_from_widths(seed: int, p: int, n_inputs: int, widths: np.ndarray, mix: dict) -> Dag:
    widths = np.asarray(widths, dtype=np.int64)
    total = int(widths.sum())
    counts = mix if sum(mix.values()) == total else _mix_counts(mix, total)
    ops = np.concatenate([np.full(c, OP_NAMES[k], dtype=np.uint8)
                          for k, c in sorted(counts.items()) if c > 0])
    perm = np.argsort(draws(seed, _S_OPS, total), kind="stable")
    ops = ops[perm]
    offs = np.zeros(widths.size + 1, dtype=np.int64)
    offs[1:] = np.cumsum(widths)
    # in0 from the previous layer (inputs for layer 0), in1 from all earlier wires
    layer_of = np.repeat(np.arange(widths.size), widths)
    start = n_inputs + offs[layer_of]                      # first wire of the gate's layer
    prev_lo = np.where(layer_of == 0, 0, n_inputs + offs[np.maximum(layer_of - 1, 0)])
    in0 = uniform_int(seed, _S_IN0, prev_lo, start).astype(np.uint32)
    in1 = uniform_int(seed, _S_IN1, np.zeros(total, np.uint64), start).astype(np.uint32)
    unary = (ops == OP_CMUL) | (ops == OP_CADD)
    in1[unary] = in0[unary]
    k = random_constants(seed, _S_CONST, total, p)
    k[~unary] = 0
    return Dag(p=p, n_inputs=n_inputs, ops=ops, in0=in0, in1=in1, kconst=k,
               layer_offsets=offs, seed=seed,
               meta={"widths": widths.tolist(), "mix": {kk: int(v) for kk, v in counts.items()}})


def layered_dag(seed: int = 2, p: int = P61, total_gates: int = 2**20, depth: int = 32,
                wmin: int = 1024, wmax: int = 65536, n_inputs: int = 65536,
                mix: dict | None = None) -> Dag:
    """The benchmark circuit: defaults give 2^20 gates in 32 layers, widths
    log-uniform in [1k, 64k], 65,536 secret input wires and the 60/15/15/10
    mul/add/sub/cmul mix."""
    if mix is None:
        mix = CONFIG2_MIX if total_gates == 2**20 else {"mul": 60, "add": 15, "sub": 15, "cmul": 10}
    w = layer_widths(seed, total_gates, depth, wmin, wmax)
    return dag_from_widths(seed, p, n_inputs, w, mix)


def small_dag(seed: int, p: int, n_inputs: int, widths, mix=None) -> Dag:
    """Circuit with the given widths (used for small parity cases)."""
    if mix is None:
        mix = {"mul": 50, "add": 15, "sub": 15, "cmul": 10, "cadd": 10}
    return dag_from_widths(seed, p, n_inputs, np.asarray(widths), mix)


@dataclass
class Request:
    rid: int
    arrival_s: float
    p: int
    gates: int
    depth: int
    seed: int


def serving_requests(seed: int = 5, count: int = 10000, rate_per_s: float = 100.0,
                     gmin: int = 2**10, gmax: int = 2**22, dmin: int = 4, dmax: int = 64):
    """Poisson arrivals (exponential gaps at ``rate_per_s``) of circuit
    requests: gate count log-uniform in [gmin, gmax], depth uniform in
    [dmin, dmax], field p61 or p127 with probability 1/2."""
    u = uniform01(seed, _S_REQ, 4 * count).reshape(count, 4)
    gaps = -np.log1p(-u[:, 0]) / rate_per_s
    t = np.cumsum(gaps)
    gates = np.exp(math.log(gmin) + (math.log(gmax) - math.log(gmin)) * u[:, 1])
    gates = np.maximum(gmin, np.round(gates)).astype(np.int64)
    depth = (dmin + np.floor(u[:, 2] * (dmax - dmin + 1))).astype(np.int64)
    field_is_127 = u[:, 3] >= 0.5
    return [Request(rid=i, arrival_s=float(t[i]), p=P127 if field_is_127[i] else P61,
                    gates=int(gates[i]), depth=int(min(depth[i], gates[i])),
                    seed=(seed << 32) + i + 1) for i in range(count)]


def request_dag(req: Request, n_inputs: int | None = None) -> Dag:
    """Circuit of one serving request: widths log-uniform in [1, 65536] scaled
    to the request's gate count (minimum 1, no upper clamp), the benchmark mix."""
    u = uniform01(req.seed, _S_WIDTH, req.depth)
    w = np.exp(math.log(65536.0) * u)
    w = w * (req.gates / w.sum())
    wi = np.maximum(1, np.floor(w)).astype(np.int64)
    rem = req.gates - int(wi.sum())
    order = np.argsort(-w, kind="stable")
    i = 0
    while rem != 0:
        k = order[i % req.depth]
        if rem > 0:
            wi[k] += 1
            rem -= 1
        elif wi[k] > 1:
            wi[k] -= 1
            rem += 1
        i += 1
    if n_inputs is None:
        n_inputs = int(max(1, min(65536, wi[0])))
    return dag_from_widths(req.seed, req.p, n_inputs, wi,
                           {"mul": 60, "add": 15, "sub": 15, "cmul": 10})


def calibration_dags(p: int, seed: int = 77, depth: int = 12):
    """Circuits whose per-layer timings train the scheduler's cost model:
    uniform widths from 1 to 32k, and mixed circuits with log-uniform widths,
    each with the benchmark's gate mix."""
    mix = {"mul": 60, "add": 15, "sub": 15, "cmul": 10}
    out = []
    for k, w in enumerate((1, 8, 64, 256, 1024, 4096, 16384, 32768)):
        out.append(dag_from_widths(seed + k, p, max(64, w), np.full(depth, w), mix))
    for k in range(3):
        w = layer_widths(seed + 100 + k, total=depth * 3000, depth=depth, wmin=16, wmax=16384)
        out.append(dag_from_widths(seed + 200 + k, p, 4096, w, mix))
    return out
