"""Pins of the CPU oracle against what the mathematics fixes.

Each test checks the oracle against something other than itself: Python's
own integer arithmetic, the published SplitMix64 outputs, closed forms of the
protocol (reconstruct(z) == x*y mod p, sum of MAC shares == alpha * value,
linearity, X*Y for matrices, cleartext circuit evaluation), brute force over
tiny primes, and the deterministic effect of a tampered share on the MAC
check.  A dropped term, a wrong sign, a swapped operand or a wrong party
index in any oracle function fails at least one of them.
"""
import itertools
import os
import random

import numpy as np
import pytest

import oracle as O
import spdz_workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PRIMES = [7, 11, 101, (1 << 31) - 1, O.P32, O.P61, O.P127]


def rec(p, shares):
    return O.reconstruct(p, shares)


def ints(p, arr):
    return O.to_ints(p, arr)


# --------------------------------------------------------------------- field

def _edge(p):
    vals = {0, 1, 2, p - 1, p - 2, p // 2, p // 2 + 1}
    for e in (32, 61, 63, 64, 126):
        for d in (-1, 0, 1):
            v = (1 << e) + d
            if 0 <= v < p:
                vals.add(v)
    if p > 2**64:
        vals |= {(2**64 - 1), (2**64 - 1) << 63 & (p - 1), p - 2**64}
    return sorted(v for v in vals if 0 <= v < p)


@pytest.mark.parametrize("p", PRIMES)
def test_field_ops_match_python_ints(p):
    rng = random.Random(p)
    vals = _edge(p) + [rng.randrange(p) for _ in range(40)]
    for a in vals:
        for b in vals[::3]:
            assert O.fop(p, "add", a, b) == (a + b) % p
            assert O.fop(p, "sub", a, b) == (a - b) % p
            assert O.fop(p, "mul", a, b) == (a * b) % p


# ----------------------------------------------------------------------- PRG

def test_splitmix64_published_outputs():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt"))
            if l.strip() and not l.startswith("#")]
    for idx, val in rows:
        assert O.sm64(0, int(idx)) == int(val, 16)
    # the workload module's numpy copy follows the same definition
    got = W.sm64(0, np.arange(4, dtype=np.uint64))
    assert [int(v) for v in got] == [int(v, 16) for _, v in rows]


@pytest.mark.parametrize("p", [O.P61, O.P127, O.P32, 7, 11])
def test_draw_elements_in_range_and_distinct_streams(p):
    a = ints(p, O.draw(p, 9, O.stream_id(2, 1, 0, 0), 0, 2000))
    b = ints(p, O.draw(p, 9, O.stream_id(2, 1, 1, 0), 0, 2000))
    assert all(0 <= v < p for v in a + b)
    if p > 2**32:
        assert len(set(a)) == 2000 and a != b
    # counter form: a window starting at j0 equals the tail of a longer draw
    c = ints(p, O.draw(p, 9, O.stream_id(2, 1, 0, 0), 700, 100))
    assert c == a[700:800]


def test_draw_p61_is_top_61_bits():
    key = O.lib().orc_stream_key(5, O.stream_id(5, 0, 0, 3))
    got = ints(O.P61, O.draw(O.P61, 5, O.stream_id(5, 0, 0, 3), 0, 50))
    for j, g in enumerate(got):
        v = O.sm64(key, j) >> 3
        assert g == (0 if v == O.P61 else v)


def test_draw_p32_is_top_32_bits_reduced_once():
    """p = 2^32-5: the top 32 bits of the draw, minus p when they are p or above
    (the five values 2^32-5 .. 2^32-1 map to 0 .. 4)."""
    key = O.lib().orc_stream_key(5, O.stream_id(5, 0, 0, 3))
    got = ints(O.P32, O.draw(O.P32, 5, O.stream_id(5, 0, 0, 3), 0, 200))
    for j, g in enumerate(got):
        v = O.sm64(key, j) >> 32
        assert g == (v - O.P32 if v >= O.P32 else v)


def test_draw_p127_two_words():
    key = O.lib().orc_stream_key(5, O.stream_id(5, 0, 0, 3))
    got = ints(O.P127, O.draw(O.P127, 5, O.stream_id(5, 0, 0, 3), 0, 50))
    for j, g in enumerate(got):
        v = ((O.sm64(key, 2 * j + 1) >> 1) << 64) | O.sm64(key, 2 * j)
        assert g == (0 if v == O.P127 else v)


# -------------------------------------------------------------------- dealer

@pytest.mark.parametrize("p,n", [(O.P61, 2), (O.P61, 3), (O.P127, 3), (101, 4), (O.P32, 3)])
def test_dealer_sharing_and_mac_relation(p, n):
    alpha, ash = O.deal_alpha(p, n, 17)
    al = ints(p, np.array([alpha]))[0]
    assert al != 0
    assert sum(ints(p, ash)) % p == al
    v, m, s = O.deal_shared(p, n, 17, O.K_INPUT, 0, 0, 300, alpha)
    sec = ints(p, s)
    assert rec(p, v) == sec
    assert rec(p, m) == [(al * x) % p for x in sec]
    # shares of different parties are independent draws, not copies
    assert ints(p, v[0]) != ints(p, v[1])
    # index-addressable: a window equals the same range of a larger call
    v2, m2, s2 = O.deal_shared(p, n, 17, O.K_INPUT, 0, 100, 50, alpha)
    assert np.array_equal(v2, v[:, 100:150]) and np.array_equal(m2, m[:, 100:150])


@pytest.mark.parametrize("p,n", [(O.P61, 2), (O.P127, 3), (11, 3), (O.P32, 2)])
def test_dealer_triples_are_products(p, n):
    alpha, ash = O.deal_alpha(p, n, 3)
    al = ints(p, np.array([alpha]))[0]
    t = O.deal_triples(p, n, 3, 0, 500, alpha)
    a, b, c = rec(p, t.av), rec(p, t.bv), rec(p, t.cv)
    assert c == [(x * y) % p for x, y in zip(a, b)]
    for val, mac in ((t.av, t.am), (t.bv, t.bm), (t.cv, t.cm)):
        assert rec(p, mac) == [(al * x) % p for x in rec(p, val)]


# ------------------------------------------------------------- linear gates

@pytest.mark.parametrize("p,n", [(O.P61, 3), (O.P127, 3), (101, 2), (O.P32, 3)])
def test_linear_gates_closed_form(p, n):
    alpha, ash = O.deal_alpha(p, n, 8)
    al = ints(p, np.array([alpha]))[0]
    xv, xm, xs = O.deal_shared(p, n, 8, O.K_INPUT, 0, 0, 200, alpha)
    yv, ym, ys = O.deal_shared(p, n, 8, O.K_INPUT, 1, 0, 200, alpha)
    x, y = ints(p, xs), ints(p, ys)
    k = (p - 12345) % p if p > 12345 else p - 3
    expect = {O.OP_ADD: [(a + b) % p for a, b in zip(x, y)],
              O.OP_SUB: [(a - b) % p for a, b in zip(x, y)],
              O.OP_CMUL: [(k * a) % p for a in x],
              O.OP_CADD: [(a + k) % p for a in x]}
    for op, exp in expect.items():
        zv, zm = O.linear(p, op, xv, xm, yv, ym, k, ash)
        assert rec(p, zv) == exp, op
        assert rec(p, zm) == [(al * e) % p for e in exp], op
    # CADD touches only party 0's value share
    zv, zm = O.linear(p, O.OP_CADD, xv, xm, yv, ym, k, ash)
    assert np.array_equal(zv[1:], xv[1:])


def test_open_sums_parties():
    p, n = O.P127, 3
    alpha, _ = O.deal_alpha(p, n, 1)
    xv, _, xs = O.deal_shared(p, n, 1, O.K_INPUT, 4, 0, 64, alpha)
    assert ints(p, O.open_(p, xv)) == ints(p, xs)


# -------------------------------------------------------------------- Beaver

def _share(rng, p, n, v):
    s = [rng.randrange(p) for _ in range(n - 1)]
    return s + [(v - sum(s)) % p]


def _arr(p, n, cols):
    """cols: list over elements of per-party share lists -> [n, count]."""
    out = O.zeros(p, n, len(cols))
    for i in range(n):
        out[i] = O.to_array(p, [c[i] for c in cols]).reshape(out[i].shape)
    return out


@pytest.mark.parametrize("p,n", [(7, 2), (7, 3), (11, 2)])
def test_beaver_brute_force_tiny_field(p, n):
    """Every (x, y, a, b) in a tiny field, with random share splits and a
    random alpha: reconstruct(z) == x*y, MAC relation on z, opened values."""
    rng = random.Random(p * 10 + n)
    alpha = rng.randrange(1, p)
    ash = _share(rng, p, n, alpha)
    combos = list(itertools.product(range(p), repeat=4))
    cols = {k: [] for k in ("xv", "xm", "yv", "ym", "av", "am", "bv", "bm", "cv", "cm")}
    for x, y, a, b in combos:
        c = a * b % p
        for name, v in (("x", x), ("y", y), ("a", a), ("b", b), ("c", c)):
            cols[name + "v"].append(_share(rng, p, n, v))
            cols[name + "m"].append(_share(rng, p, n, alpha * v % p))
    A = {k: _arr(p, n, v) for k, v in cols.items()}
    tri = O.Triples(A["av"], A["am"], A["bv"], A["bm"], A["cv"], A["cm"])
    ash_a = O.to_array(p, ash)
    zv, zm, eps, dlt, log = O.mul(p, A["xv"], A["xm"], A["yv"], A["ym"], tri, ash_a)
    z, gz = rec(p, zv), rec(p, zm)
    e, d = ints(p, eps), ints(p, dlt)
    for t, (x, y, a, b) in enumerate(combos):
        assert z[t] == x * y % p
        assert gz[t] == alpha * x * y % p
        assert e[t] == (x - a) % p and d[t] == (y - b) % p
    # opened values carry valid MACs: sum_i gamma_i(eps) == alpha * eps
    lv, lm = ints(p, log.vals), rec(p, log.macs)
    assert lm == [alpha * v % p for v in lv]


@pytest.mark.parametrize("p,n", [(O.P61, 2), (O.P61, 3), (O.P127, 3), (O.P32, 3)])
def test_beaver_large_field_closed_form(p, n):
    alpha, ash = O.deal_alpha(p, n, 11)
    al = ints(p, np.array([alpha]))[0]
    xv, xm, xs = O.deal_shared(p, n, 11, O.K_INPUT, 0, 0, 400, alpha)
    yv, ym, ys = O.deal_shared(p, n, 11, O.K_INPUT, 1, 0, 400, alpha)
    tri = O.deal_triples(p, n, 11, 0, 400, alpha)
    zv, zm, eps, dlt, log = O.mul(p, xv, xm, yv, ym, tri, ash)
    x, y = ints(p, xs), ints(p, ys)
    assert rec(p, zv) == [(a * b) % p for a, b in zip(x, y)]
    assert rec(p, zm) == [(al * a * b) % p for a, b in zip(x, y)]
    assert ints(p, eps) == [(a - b) % p for a, b in zip(x, rec(p, tri.av))]
    assert ints(p, dlt) == [(a - b) % p for a, b in zip(y, rec(p, tri.bv))]
    # only party 0 adds eps*delta: dropping it from party 0 or adding it at
    # another party would change the reconstruction, so the closed form above
    # already pins the party index; check the log ordering explicitly
    assert ints(p, log.vals)[0::2] == ints(p, eps) and ints(p, log.vals)[1::2] == ints(p, dlt)


# ----------------------------------------------------------------- MAC check

@pytest.mark.parametrize("p,n", [(O.P61, 2), (O.P61, 3), (O.P127, 3), (O.P32, 2)])
def test_mac_check_accepts_honest_and_rejects_tamper(p, n):
    alpha, ash = O.deal_alpha(p, n, 21)
    al = ints(p, np.array([alpha]))[0]
    xv, xm, _ = O.deal_shared(p, n, 21, O.K_INPUT, 0, 0, 256, alpha)
    yv, ym, _ = O.deal_shared(p, n, 21, O.K_INPUT, 1, 0, 256, alpha)
    tri = O.deal_triples(p, n, 21, 0, 256, alpha)
    *_, log = O.mul(p, xv, xm, yv, ym, tri, ash)
    ok, sigma, A, S = O.mac_check(p, [log], ash, check_seed=99, epoch=0)
    assert ok and sum(ints(p, sigma)) % p == 0
    r = ints(p, O.check_coeffs(p, 99, 0, 0, 512))
    assert all(v != 0 for v in r) and al != 0
    # A is the random linear combination of the opened values
    assert ints(p, np.array([A]))[0] == sum(ri * vi for ri, vi in zip(r, ints(p, log.vals))) % p
    # value tamper at opened index j by Delta: sum sigma changes by -alpha*r_j*Delta
    for j, delta, party in ((5, 1, 0), (300, 123456789, n - 1)):
        bad = O.OpenLog(log.vals.copy(), log.macs.copy())
        v = ints(p, bad.vals[j:j + 1])[0]
        bad.vals[j] = O.to_array(p, [(v + delta) % p])[0]
        ok2, sig2, *_ = O.mac_check(p, [bad], ash, 99, 0)
        assert not ok2
        assert sum(ints(p, sig2)) % p == (-al * r[j] * delta) % p
        # MAC tamper of one party's share: sum sigma changes by r_j*Delta
        bad = O.OpenLog(log.vals.copy(), log.macs.copy())
        m = ints(p, bad.macs[party, j:j + 1])[0]
        bad.macs[party, j] = O.to_array(p, [(m + delta) % p])[0]
        ok3, sig3, *_ = O.mac_check(p, [bad], ash, 99, 0)
        assert not ok3
        assert sum(ints(p, sig3)) % p == (r[j] * delta) % p


def test_mac_check_chunks_add_and_epochs_differ():
    p, n = O.P61, 3
    alpha, ash = O.deal_alpha(p, n, 2)
    xv, xm, _ = O.deal_shared(p, n, 2, O.K_INPUT, 0, 0, 128, alpha)
    log = O.OpenLog(O.open_(p, xv), xm)
    A, S = O.rlc(p, log, 7, 3, 0)
    A1, S1 = O.rlc(p, O.OpenLog(log.vals[:50].copy(), np.ascontiguousarray(log.macs[:, :50])), 7, 3, 0)
    A2, S2 = O.rlc(p, O.OpenLog(log.vals[50:].copy(), np.ascontiguousarray(log.macs[:, 50:])), 7, 3, 50)
    assert ints(p, np.array([A]))[0] == (ints(p, np.array([A1]))[0] + ints(p, np.array([A2]))[0]) % p
    assert ints(p, S) == [(a + b) % p for a, b in zip(ints(p, S1), ints(p, S2))]
    assert ints(p, O.check_coeffs(p, 7, 3, 0, 8)) != ints(p, O.check_coeffs(p, 7, 4, 0, 8))


# ------------------------------------------------------------ inner products

@pytest.mark.parametrize("p", [O.P61, O.P127, O.P32])
def test_innerprod_closed_form(p):
    n, P, L = 3, 7, 33
    alpha, ash = O.deal_alpha(p, n, 4)
    al = ints(p, np.array([alpha]))[0]
    xv, xm, xs = O.deal_shared(p, n, 4, O.K_INPUT, 0, 0, P * L, alpha)
    yv, ym, ys = O.deal_shared(p, n, 4, O.K_INPUT, 1, 0, P * L, alpha)
    tri = O.deal_triples(p, n, 4, 0, P * L, alpha)
    zv, zm, eps, dlt, log = O.innerprod(p, P, L, xv, xm, yv, ym, tri, ash)
    x, y = ints(p, xs), ints(p, ys)
    exp = [sum(x[t * L + k] * y[t * L + k] for k in range(L)) % p for t in range(P)]
    assert rec(p, zv) == exp
    assert rec(p, zm) == [(al * e) % p for e in exp]
    ok, *_ = O.mac_check(p, [log], ash, 5, 0)
    assert ok


# -------------------------------------------------------------------- matrix

@pytest.mark.parametrize("p,M,K,N", [(O.P61, 5, 7, 3), (O.P61, 16, 16, 16), (101, 4, 6, 5)])
def test_matrix_beaver_closed_form(p, M, K, N):
    n = 3
    alpha, ash = O.deal_alpha(p, n, 6)
    al = ints(p, np.array([alpha]))[0]
    Xv, Xm, Xs = O.deal_shared(p, n, 6, O.K_INPUT, 10, 0, M * K, alpha)
    Yv, Ym, Ys = O.deal_shared(p, n, 6, O.K_INPUT, 11, 0, K * N, alpha)
    tri = O.deal_matrix_triple(p, n, 6, 0, M, K, N, alpha)
    Aa, Bb, Cc = rec(p, tri.av), rec(p, tri.bv), rec(p, tri.cv)
    for r in range(M):
        for c in range(N):
            assert Cc[r * N + c] == sum(Aa[r * K + k] * Bb[k * N + c] for k in range(K)) % p
    E, F, Em, Fm = O.mat_open(p, M, K, N, (Xv, Xm), (Yv, Ym), tri)
    rows, cols = np.divmod(np.arange(M * N), N)
    Zv, Zm = O.mat_entries(p, M, K, N, E, F, tri, ash, rows, cols)
    X, Y = ints(p, Xs), ints(p, Ys)
    exp = [sum(X[r * K + k] * Y[k * N + c] for k in range(K)) % p for r, c in zip(rows, cols)]
    assert rec(p, Zv) == exp
    assert rec(p, Zm) == [(al * e) % p for e in exp]
    assert ints(p, E) == [(a - b) % p for a, b in zip(X, Aa)]
    log = O.OpenLog(np.concatenate([E, F]), np.ascontiguousarray(np.concatenate([Em, Fm], axis=1)))
    ok, *_ = O.mac_check(p, [log], ash, 1, 0)
    assert ok


# ----------------------------------------------------------------------- DAG

def _clear_python(p, dag, inputs):
    w = list(inputs) + [0] * dag.n_gates
    for g in range(dag.n_gates):
        a, b, k = w[int(dag.in0[g])], w[int(dag.in1[g])], O.to_ints(p, dag.kconst[g:g + 1])[0]
        op = int(dag.ops[g])
        w[dag.n_inputs + g] = {O.OP_ADD: a + b, O.OP_SUB: a - b, O.OP_CMUL: k * a,
                               O.OP_CADD: a + k, O.OP_MUL: a * b}[op] % p
    return w


@pytest.mark.parametrize("p", [O.P61, O.P127, O.P32])
def test_dag_shared_equals_cleartext(p):
    n = 3
    dag = W.small_dag(seed=12, p=p, n_inputs=40, widths=[30, 17, 1, 25, 9])
    alpha, ash = O.deal_alpha(p, n, 12)
    al = ints(p, np.array([alpha]))[0]
    iv, im, isec = O.deal_shared(p, n, 12, O.K_INPUT, 16, 0, dag.n_inputs, alpha)
    wv, wm = O.zeros(p, n, dag.n_wires), O.zeros(p, n, dag.n_wires)
    wv[:, :dag.n_inputs], wm[:, :dag.n_inputs] = iv, im
    tri = O.deal_triples(p, n, 12, 0, dag.n_mul, alpha)
    eps, dlt, log = O.dag_eval(p, dag, wv, wm, tri, ash)
    clear = _clear_python(p, dag, ints(p, isec))
    assert ints(p, O.dag_clear(p, dag, isec)) == clear
    assert rec(p, wv) == clear
    assert rec(p, wm) == [(al * v) % p for v in clear]
    ok, *_ = O.mac_check(p, [log], ash, 3, 0)
    assert ok


@pytest.mark.parametrize("p,widths", [(O.P61, [5000, 7, 1, 6000, 4097]), (O.P127, [4500, 300, 4100]),
                                      (O.P32, [9000, 1, 8192])])
def test_layer_parallel_eval_equals_gate_order(p, widths):
    """The layer-parallel evaluation on 4 threads (layers wide enough to be
    split) gives every wire share and every opened value and MAC share of the
    gate-order evaluation; a gate whose operand is written in its own layer
    is refused."""
    n = 3
    dag = W.small_dag(seed=21, p=p, n_inputs=512, widths=widths)
    alpha, ash = O.deal_alpha(p, n, 21)
    iv, im, _ = O.deal_shared(p, n, 21, O.K_INPUT, 16, 0, dag.n_inputs, alpha)
    tri = O.deal_triples(p, n, 21, 0, dag.n_mul, alpha)
    outs = []
    for fn, threads in ((O.dag_eval, 1), (O.dag_eval_layers, 4)):
        O.set_threads(threads)
        wv, wm = O.zeros(p, n, dag.n_wires), O.zeros(p, n, dag.n_wires)
        wv[:, :dag.n_inputs], wm[:, :dag.n_inputs] = iv, im
        eps, dlt, log = fn(p, dag, wv, wm, tri, ash)
        outs.append((wv, wm, eps, dlt, log.vals, log.macs))
    O.set_threads(1)
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    bad = W.small_dag(seed=21, p=p, n_inputs=512, widths=widths)
    g = int(bad.layer_offsets[1]) + 3
    bad.in0[g] = bad.n_inputs + g - 1                 # an output of the same layer
    wv, wm = O.zeros(p, n, dag.n_wires), O.zeros(p, n, dag.n_wires)
    with pytest.raises(ValueError):
        O.dag_eval_layers(p, bad, wv, wm, tri, ash)


# ---------------------------------------------------------- workload shapes

def test_benchmark_dag_shape():
    dag = W.layered_dag(seed=2)
    w = dag.widths
    assert dag.n_gates == 2**20 and dag.depth == 32
    assert w.min() >= 1024 and w.max() <= 65536 and int(w.sum()) == 2**20
    counts = {k: int(np.count_nonzero(dag.ops == v)) for k, v in W.OP_NAMES.items()}
    assert counts == {"mul": 629146, "add": 157286, "sub": 157286, "cmul": 104858, "cadd": 0}
    offs = dag.layer_offsets
    for k in (0, 1, 17, 31):
        lo, hi = offs[k], offs[k + 1]
        start = dag.n_inputs + lo
        prev_lo = 0 if k == 0 else dag.n_inputs + offs[k - 1]
        assert dag.in0[lo:hi].min() >= prev_lo and dag.in0[lo:hi].max() < start
        assert dag.in1[lo:hi].max() < start
    assert W.layered_dag(seed=2).in1[:100].tolist() == dag.in1[:100].tolist()


def test_serving_requests_shape():
    reqs = W.serving_requests(seed=5, count=2000)
    g = np.array([r.gates for r in reqs])
    d = np.array([r.depth for r in reqs])
    assert g.min() >= 2**10 and g.max() <= 2**22
    assert d.min() >= 4 and d.max() <= 64
    assert np.all(np.diff([r.arrival_s for r in reqs]) > 0)
    frac127 = np.mean([r.p == W.P127 for r in reqs])
    assert 0.45 < frac127 < 0.55
    dag = W.request_dag(reqs[3])
    assert dag.n_gates == reqs[3].gates and dag.depth == reqs[3].depth
