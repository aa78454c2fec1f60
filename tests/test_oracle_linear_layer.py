"""Pins of the oracle's LinearLayer (y = W x + b with row tiles and one
matrix-vector triple per tile, Sec. III-D.3): reconstruction against the
cleartext W x + b computed with Python ints, the MAC relation, the tile
triples against their products, the check over the opened values (and the
exact effect of a tampered share), and the streamed check sums against the
stored log."""
import numpy as np
import pytest

import oracle as O

SEED, SUB, CHK = 17, 3, 29
W_SUB, X_SUB, B_SUB = 20, 21, 22


def world(p, n, dout, din, R):
    alpha, ash = O.deal_alpha(p, n, SEED)
    Wv, Wm, Ws = O.deal_shared(p, n, SEED, O.K_INPUT, W_SUB, 0, dout * din, alpha)
    xv, xm, xs = O.deal_shared(p, n, SEED, O.K_INPUT, X_SUB, 0, din, alpha)
    bv, bm, bs = O.deal_shared(p, n, SEED, O.K_INPUT, B_SUB, 0, dout, alpha)
    tri = O.deal_matvec_triples(p, n, SEED, SUB, dout, din, R, alpha)
    return alpha, ash, (Wv, Wm, Ws), (xv, xm, xs), (bv, bm, bs), tri


def ints(p, a):
    return O.to_ints(p, a)


SHAPES = [(O.P32, 2, 7, 5, 3), (O.P61, 3, 8, 4, 8), (101, 2, 5, 6, 1), (O.P32, 3, 9, 16, 4), (O.P61, 2, 6, 3, 100)]


@pytest.mark.parametrize("p,n,dout,din,R", SHAPES)
def test_linear_layer_reconstructs_Wx_plus_b(p, n, dout, din, R):
    alpha, ash, W, x, b, tri = world(p, n, dout, din, R)
    yv, ym = O.linear_layer(p, dout, din, R, W[:2], x[:2], b[:2], tri, ash)
    Wc, xc, bc = ints(p, W[2]), ints(p, x[2]), ints(p, b[2])
    expect = [(sum(Wc[r * din + k] * xc[k] for k in range(din)) + bc[r]) % p for r in range(dout)]
    y = O.reconstruct(p, yv)
    assert y == expect
    a = ints(p, np.asarray([alpha]))[0]
    assert O.reconstruct(p, ym) == [(a * v) % p for v in y]


@pytest.mark.parametrize("p,n,dout,din,R", SHAPES[:3])
def test_matvec_triples_are_tile_products(p, n, dout, din, R):
    alpha, ash, W, x, b, tri = world(p, n, dout, din, R)
    T = -(-dout // R)
    A, B, Cc = O.reconstruct(p, tri.av), O.reconstruct(p, tri.bv), O.reconstruct(p, tri.cv)
    assert len(B) == T * din
    for r in range(dout):
        t = r // R
        assert Cc[r] == sum(A[r * din + k] * B[t * din + k] for k in range(din)) % p
    a = ints(p, np.asarray([alpha]))[0]
    for v, m in ((tri.av, tri.am), (tri.bv, tri.bm), (tri.cv, tri.cm)):
        assert O.reconstruct(p, m) == [(a * s) % p for s in O.reconstruct(p, v)]


@pytest.mark.parametrize("p,n,dout,din,R", [(O.P32, 2, 7, 5, 3), (O.P61, 3, 9, 4, 2)])
def test_opened_values_check_and_tamper_is_exact(p, n, dout, din, R):
    alpha, ash, W, x, b, tri = world(p, n, dout, din, R)
    log = O.linear_open(p, dout, din, R, W[:2], x[:2], tri)
    T = -(-dout // R)
    assert log.vals.shape[0] == T * din + dout * din
    # the log holds E_t = x - B_t then D_t = W_t - A_t, tile by tile
    xc, Bc = O.reconstruct(p, x[0]), O.reconstruct(p, tri.bv)
    Wc, Ac = O.reconstruct(p, W[0]), O.reconstruct(p, tri.av)
    vals = ints(p, log.vals)
    pos = 0
    for t in range(T):
        assert vals[pos:pos + din] == [(xc[k] - Bc[t * din + k]) % p for k in range(din)]
        pos += din
        for r in range(t * R, min((t + 1) * R, dout)):
            assert vals[pos:pos + din] == [(Wc[r * din + k] - Ac[r * din + k]) % p for k in range(din)]
            pos += din
    ok, sigma, A, S = O.mac_check(p, [log], ash, CHK, 0)
    assert ok
    # the streamed sums equal the stored log's
    A2, S2 = O.linear_rlc(p, dout, din, R, W[:2], x[:2], tri, CHK, 0)
    assert ints(p, np.asarray([A2])) == ints(p, np.asarray([A])) and ints(p, S2) == ints(p, S)
    # party 1 adds delta to its share of W[r, k]: D[r, k] moves by delta and
    # sum(sigma) by -alpha * r_j * delta (j: the position of D[r, k] in the log)
    r, k, delta = dout - 1, din - 2, 12345
    Wt = W[0].copy()
    Wt_int = ints(p, Wt[1])
    Wt[1] = O.to_array(p, [(v + delta) % p if q == r * din + k else v for q, v in enumerate(Wt_int)])
    A3, S3 = O.linear_rlc(p, dout, din, R, (Wt, W[1]), x[:2], tri, CHK, 0)
    sig3, ok3 = O.check_finish(p, A3, S3, ash)
    assert not ok3
    t = r // R
    j = t * (din + R * din) + din + (r - t * R) * din + k
    rj = ints(p, O.check_coeffs(p, CHK, 0, j, 1))[0]
    a = ints(p, np.asarray([alpha]))[0]
    assert sum(ints(p, sig3)) % p == (-a * rj * delta) % p


def test_rows_subset_equals_full():
    p, n, dout, din, R = O.P32, 2, 11, 7, 4
    alpha, ash, W, x, b, tri = world(p, n, dout, din, R)
    yv, ym = O.linear_layer(p, dout, din, R, W[:2], x[:2], b[:2], tri, ash)
    rows = np.array([10, 0, 4, 7], dtype=np.int64)
    sv, sm = O.linear_layer(p, dout, din, R, W[:2], x[:2], b[:2], tri, ash, rows=rows)
    assert np.array_equal(sv, yv[:, rows]) and np.array_equal(sm, ym[:, rows])
