"""The LinearLayer operator on the GPU against the CPU oracle: the device
dealer's matrix-vector triples, the opened E and D, every share of y and
gamma(y), and the check's sigma, bit-exact, on ragged shapes of both fields;
at 4096 x 4096 and at the paper's 8192 x 8192 (2 parties, 32-row tiles) on
sampled rows the oracle computes one by one, with sigma from the oracle's
streamed check sums."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

from gpu_helpers import assert_equal, ctx_for  # noqa: E402

SEED, SUB, CHK = 17, 3, 29
W_SUB, X_SUB, B_SUB = 20, 21, 22


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    global S, SH
    from paper_2512_11112_b300 import shares as SH  # noqa: F401
    from paper_2512_11112_b300 import spdz as S  # noqa: F401
    yield
    torch.cuda.synchronize()


def device_layer(p, n, dout, din, R, want_opened=True):
    ctx = ctx_for(n, p)
    f = SH.field_of(p)
    T = -(-dout // R)
    try:
        ash = SH.zeros(f, n)
        S.spdz_deal_alpha(ctx, SEED, ash)
        W, x, b = SH.alloc(f, n, dout * din), SH.alloc(f, n, din), SH.alloc(f, n, dout)
        S.spdz_deal_shared(ctx, SEED, S.SPDZ_KIND_INPUT, W_SUB, 0, dout * din, ash, None, W.buf())
        S.spdz_deal_shared(ctx, SEED, S.SPDZ_KIND_INPUT, X_SUB, 0, din, ash, None, x.buf())
        S.spdz_deal_shared(ctx, SEED, S.SPDZ_KIND_INPUT, B_SUB, 0, dout, ash, None, b.buf())
        A, B, Cm = SH.alloc(f, n, dout * din), SH.alloc(f, n, T * din), SH.alloc(f, n, dout)
        S.spdz_deal_matvec_triples(ctx, SEED, SUB, dout, din, R, ash, A.buf(), B.buf(), Cm.buf())
        S.spdz_load_preproc(ctx, ash, None, None, None, 0)
        S.spdz_set_check_seed(ctx, CHK)
        S.spdz_load_matvec_preproc(ctx, A.buf(), B.buf(), Cm.buf(), dout, din, R)
        y = SH.alloc(f, n, dout)
        D = SH.zeros(f, dout * din) if want_opened else None
        E = SH.zeros(f, T * din) if want_opened else None
        S.spdz_linear_layer(ctx, W.buf(), x.buf(), b.buf(), y.buf(), dout, din, R, D, E)
        sig = O.zeros(p, n)
        passed = S.spdz_mac_check(ctx, sig)
        out = dict(y=y.host(), sig=sig, passed=passed, B=B.host(), C=Cm.host())
        if want_opened:
            out.update(A=A.host(), D=SH.to_host(D), E=SH.to_host(E))
        else:
            out.update(A0=SH.to_host(A.val[:, :din]))
        # the triples are consumed by one layer
        with pytest.raises(S.SpdzError) as e:
            S.spdz_linear_layer(ctx, W.buf(), x.buf(), b.buf(), y.buf(), dout, din, R)
        assert e.value.code == S.SPDZ_ERR_TRIPLES
        return out
    finally:
        S.spdz_ctx_destroy(ctx)


def oracle_world(p, n, dout, din, R):
    alpha, ash = O.deal_alpha(p, n, SEED)
    W = O.deal_shared(p, n, SEED, O.K_INPUT, W_SUB, 0, dout * din, alpha)
    x = O.deal_shared(p, n, SEED, O.K_INPUT, X_SUB, 0, din, alpha)
    b = O.deal_shared(p, n, SEED, O.K_INPUT, B_SUB, 0, dout, alpha)
    tri = O.deal_matvec_triples(p, n, SEED, SUB, dout, din, R, alpha)
    return ash, W, x, b, tri


@pytest.mark.parametrize("p,n,dout,din,R", [
    (O.P32, 2, 7, 5, 3), (O.P32, 3, 130, 67, 16), (O.P32, 2, 1, 1, 1), (O.P32, 2, 96, 1000, 32),
    # the staged two-party row kernel: several rounds of rows per CTA (each
    # thread's next-step copies cross into its next row), a ragged wide half
    (O.P32, 2, 5000, 64, 7), (O.P32, 2, 300, 2052, 32),
    (O.P61, 2, 33, 100, 8), (O.P61, 3, 64, 64, 64), (O.P61, 4, 50, 257, 7), (O.P61, 2, 9, 300, 1000),
])
def test_linear_layer_matches_oracle(p, n, dout, din, R):
    d = device_layer(p, n, dout, din, R)
    ash, W, x, b, tri = oracle_world(p, n, dout, din, R)
    for name, (v, m) in (("A", (tri.av, tri.am)), ("B", (tri.bv, tri.bm)), ("C", (tri.cv, tri.cm))):
        assert_equal(d[name][0], v, f"triple {name} values")
        assert_equal(d[name][1], m, f"triple {name} MACs")
    log = O.linear_open(p, dout, din, R, W[:2], x[:2], tri)
    T = -(-dout // R)
    Re = min(R, dout)
    vals = log.vals
    pos, E, D = 0, [], []
    for t in range(T):
        E.append(vals[pos:pos + din])
        rows = min((t + 1) * Re, dout) - t * Re
        pos += din
        D.append(vals[pos:pos + rows * din])
        pos += rows * din
    assert_equal(d["E"], np.concatenate(E), "E")
    assert_equal(d["D"], np.concatenate(D), "D")
    yv, ym = O.linear_layer(p, dout, din, R, W[:2], x[:2], b[:2], tri, ash)
    assert_equal(d["y"][0], yv, "y values")
    assert_equal(d["y"][1], ym, "y MACs")
    ok, osig, _, _ = O.mac_check(p, [log], ash, CHK, 0)
    assert d["passed"] and ok
    assert_equal(d["sig"], osig, "sigma")


@pytest.mark.parametrize("p,size", [(O.P32, 4096), (O.P61, 4096), (O.P32, 8192)])
def test_linear_layer_large_sampled_rows(p, size):
    """size x size, 2 parties, 32-row tiles: sampled rows (first, last, tile
    edges, random) of every share of y against the oracle, the device
    triples' first row, and sigma against the oracle's streamed check sums
    over all opened values (16.9M at 4096, 67.1M at 8192).  8192 x 8192 at
    p = 2^32-5 is the paper's workload (Sec. IV-B); there the row kernel
    gives each row to two warps and deals rows out in rounds over every
    resident warp, so rows at the round boundaries of 148 SMs x 16 warps
    (multiples of 2368 / 2 rows) are sampled as well."""
    n, dout, din, R = 2, size, size, 32
    d = device_layer(p, n, dout, din, R, want_opened=False)
    assert d["passed"]
    O.set_threads(8)
    ash, W, x, b, tri = oracle_world(p, n, dout, din, R)
    assert_equal(d["A0"], tri.av[:, :din], "A row 0")
    assert_equal(d["B"][0], tri.bv, "B values")
    assert_equal(d["C"][1], tri.cm, "C MACs")
    rng = np.random.default_rng(4)
    edges = [0, dout - 1, R - 1, R, 31 * R, 31 * R + 1]
    if dout > 4096:
        edges += [1183, 1184, 2367, 2368, 3551, 3552, 4735, 4736, 7103, 7104, 8160, 8191 - 31]
    rows = np.unique(np.concatenate([edges, rng.integers(0, dout, 34)])).astype(np.int64)
    yv, ym = O.linear_layer(p, dout, din, R, W[:2], x[:2], b[:2], tri, ash, rows=rows)
    assert_equal(d["y"][0][:, rows], yv, "sampled y values")
    assert_equal(d["y"][1][:, rows], ym, "sampled y MACs")
    A, Sx = O.linear_rlc(p, dout, din, R, W[:2], x[:2], tri, CHK, 0)
    osig, ok = O.check_finish(p, A, Sx, ash)
    assert ok
    assert_equal(d["sig"], osig, "sigma")


def test_linear_layer_rejects_p127_and_shape_mismatch():
    ctx = ctx_for(2, O.P127)
    try:
        f = S.SPDZ_F127
        z = SH.alloc(f, 2, 16)
        with pytest.raises(S.SpdzError) as e:
            S.spdz_linear_layer(ctx, z.buf(), z.buf(), z.buf(), z.buf(), 4, 4, 2)
        assert e.value.code in (S.SPDZ_ERR_ARG, S.SPDZ_ERR_STATE)
    finally:
        S.spdz_ctx_destroy(ctx)
