"""Parity of the CUDA online-phase kernels with the CPU oracle, element by
element, bit-exact (integer arithmetic mod p), through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

from gpu_helpers import DeviceWorld, OracleWorld, assert_equal, ctx_for, host  # noqa: E402


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    global S, SH
    from paper_2512_11112_b300 import shares as SH  # noqa: F401
    from paper_2512_11112_b300 import spdz as S  # noqa: F401
    yield
    torch.cuda.synchronize()


def _edges(p):
    vals = [0, 1, 2, 3, p - 1, p - 2, p // 2, p // 2 + 1, (1 << 32) - 1, 1 << 32, (1 << 32) + 1,
            (1 << 60), (1 << 61) - 2]
    if p > 2**64:
        vals += [(1 << 64) - 1, 1 << 64, (1 << 64) + 1, (1 << 126), p - (1 << 64), (1 << 127) - 2,
                 ((1 << 64) - 1) << 63 & (p - 1), 0xFFFFFFFFFFFFFFFF0000000000000000 % p]
    rng = np.random.default_rng(7)
    vals += [int(x) for x in rng.integers(0, 2**62, 40, dtype=np.uint64)]
    if p > 2**64:
        vals += [(int(a) << 64 | int(b)) % p for a, b in rng.integers(0, 2**63, (40, 2), dtype=np.uint64)]
    return [v % p for v in vals]


@pytest.mark.parametrize("p", [O.P61, O.P127, O.P32])
def test_field_ops_match_python_ints(p):
    ctx = ctx_for(2, p)
    try:
        ev = _edges(p)
        a = [x for x in ev for _ in ev]
        b = [y for _ in ev for y in ev]
        f = SH.field_of(p)
        A, B = SH.from_host(O.to_array(p, a), field=f), SH.from_host(O.to_array(p, b), field=f)
        out = torch.zeros_like(A)
        for op, fn in ((S.SPDZ_OP_ADD, lambda x, y: (x + y) % p), (S.SPDZ_OP_SUB, lambda x, y: (x - y) % p),
                       (S.SPDZ_OP_CMUL, lambda x, y: (x * y) % p)):
            S.spdz_field_op(ctx, op, A, B, out, len(a))
            got = O.to_ints(p, SH.to_host(out))
            exp = [fn(x, y) for x, y in zip(a, b)]
            assert got == exp, op
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p,n", [(O.P61, 2), (O.P61, 3), (O.P127, 3), (O.P61, 5), (O.P32, 3)])
def test_device_dealer_matches_oracle_dealer(p, n):
    N, T, seed = 1000, 777, 31
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, seed, N, T)
        ow = OracleWorld(p, n, seed, N, T)
        assert_equal(host(dw.alpha_sh), ow.alpha_sh, "alpha shares")
        for k in range(2):
            dv, dm = dw.inputs[k].host()
            assert_equal(dv, ow.inputs[k][0], f"input {k} val")
            assert_equal(dm, ow.inputs[k][1], f"input {k} mac")
        for t, (ev, em) in zip(dw.tri, ((ow.tri.av, ow.tri.am), (ow.tri.bv, ow.tri.bm), (ow.tri.cv, ow.tri.cm))):
            dv, dm = t.host()
            assert_equal(dv, ev, "triple val")
            assert_equal(dm, em, "triple mac")
    finally:
        S.spdz_ctx_destroy(ctx)


MUL_CASES = [
    # p, n, N, view offset (an odd offset breaks 16-byte alignment -> scalar path)
    (O.P61, 2, 2**16, 0),      # the plain 2-party batch of 2^16 products
    (O.P61, 3, 1001, 0),
    (O.P61, 3, 777, 1),
    (O.P61, 2, 1, 0),
    (O.P61, 4, 5003, 0),
    (O.P127, 3, 4099, 0),
    (O.P127, 2, 3, 0),
    (O.P127, 2, 70001, 0),    # more products than the staged p127 grid has threads
    (O.P127, 4, 1000, 0),     # more parties than the staged p127 kernel's slots hold
    (O.P32, 3, 4097, 0),      # p = 2^32-5, the prime of the paper's evaluation
    (O.P32, 2, 777, 1),
]


@pytest.mark.parametrize("p,n,N,off", MUL_CASES)
def test_mul_batch_and_check_match_oracle(p, n, N, off):
    seed, chk = 1 + N, 4242
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, seed, N + off, N)
        S.spdz_set_check_seed(ctx, chk)
        field = dw.field
        z = SH.alloc(field, n, N + off)
        opened = SH.zeros(field, 2 * N)
        x, y = dw.inputs
        S.spdz_mul_batch(ctx, x.buf(off), y.buf(off), z.buf(off), N, opened)
        sigma = O.zeros(p, n)
        passed = S.spdz_mac_check(ctx, sigma)
        # oracle
        ow = OracleWorld(p, n, seed, N + off, N)
        (xv, xm, _), (yv, ym, _) = ow.inputs
        sl = lambda a: np.ascontiguousarray(a[:, off:off + N])
        zv, zm, eps, dlt, log = O.mul(p, sl(xv), sl(xm), sl(yv), sl(ym), ow.tri, ow.alpha_sh)
        ok, osig, _, _ = O.mac_check(p, [log], ow.alpha_sh, chk, 0)
        gv, gm = z.host()
        assert_equal(gv[:, off:off + N], zv, "z val")
        assert_equal(gm[:, off:off + N], zm, "z mac")
        assert_equal(host(opened), log.vals, "opened eps/delta")
        assert passed and ok
        assert_equal(sigma, osig, "sigma")
        assert S.spdz_triples_left(ctx) == 0
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p", [O.P61, O.P127])
def test_mul_batch_full_size_sampled(p):
    """The batch the benchmark times: 2^24 products, 3 parties, in one call on
    the full buffers.  Sampled products (the ends, the middle, 16-byte vector
    edges and random indices) against the oracle, which deals each sampled
    index's inputs and triple from the same counters; the check over all
    2^25 opened values passes and its sigma sums to zero."""
    n, N, seed, chk = 3, 2**24, 91, 17
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, seed, N, N)
        S.spdz_set_check_seed(ctx, chk)
        z = SH.alloc(dw.field, n, N)
        opened = SH.zeros(dw.field, 2 * N)
        x, y = dw.inputs
        S.spdz_mul_batch(ctx, x.buf(), y.buf(), z.buf(), N, opened)
        sigma = O.zeros(p, n)
        assert S.spdz_mac_check(ctx, sigma)
        assert sum(O.to_ints(p, sigma)) % p == 0
        rng = np.random.default_rng(3)
        idx = np.unique(np.concatenate([[0, 1, 2, 3, N // 2 - 1, N // 2, N - 2, N - 1],
                                        rng.integers(0, N, 24)])).astype(np.int64)
        ti = torch.from_numpy(idx).to(z.val.device)
        gv, gm = SH.to_host(z.val[:, ti]), SH.to_host(z.mac[:, ti])
        go = SH.to_host(opened[torch.from_numpy(np.stack([2 * idx, 2 * idx + 1], 1).reshape(-1)).to(opened.device)])
        alpha, ash = O.deal_alpha(p, n, seed)
        for s_, j in enumerate(idx.tolist()):
            xv, xm, _ = O.deal_shared(p, n, seed, O.K_INPUT, 0, j, 1, alpha)
            yv, ym, _ = O.deal_shared(p, n, seed, O.K_INPUT, 1, j, 1, alpha)
            tri = O.deal_triples(p, n, seed, j, 1, alpha)
            zv, zm, _, _, log = O.mul(p, xv, xm, yv, ym, tri, ash)
            assert_equal(gv[:, s_], zv[:, 0], f"z val at {j}")
            assert_equal(gm[:, s_], zm[:, 0], f"z mac at {j}")
            assert_equal(go[2 * s_:2 * s_ + 2], log.vals, f"eps/delta at {j}")
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p", [O.P61, O.P127, O.P32])
def test_two_batches_one_epoch_then_next_epoch(p):
    n, N, seed, chk = 3, 3000, 77, 9
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, seed, N, 2 * N)
        S.spdz_set_check_seed(ctx, chk)
        x, y = dw.inputs
        z1, z2 = SH.alloc(dw.field, n, N), SH.alloc(dw.field, n, N)
        h = N // 3
        S.spdz_mul_batch(ctx, x.buf(), y.buf(), z1.buf(), h)
        S.spdz_mul_batch(ctx, x.buf(h), y.buf(h), z1.buf(h), N - h)
        assert S.spdz_check_state(ctx) == (2 * N, 0)
        sig1 = O.zeros(p, n)
        assert S.spdz_mac_check(ctx, sig1)
        S.spdz_mul_batch(ctx, y.buf(), x.buf(), z2.buf(), N)
        sig2 = O.zeros(p, n)
        assert S.spdz_mac_check(ctx, sig2)
        assert S.spdz_check_state(ctx) == (0, 2)

        ow = OracleWorld(p, n, seed, N, 2 * N)
        (xv, xm, _), (yv, ym, _) = ow.inputs
        zv, zm, _, _, log1 = O.mul(p, xv, xm, yv, ym, ow.tri.slice(0, N), ow.alpha_sh)
        _, osig1, _, _ = O.mac_check(p, [log1], ow.alpha_sh, chk, 0)
        zv2, zm2, _, _, log2 = O.mul(p, yv, ym, xv, xm, ow.tri.slice(N, 2 * N), ow.alpha_sh)
        _, osig2, _, _ = O.mac_check(p, [log2], ow.alpha_sh, chk, 1)
        assert_equal(z1.host()[0], zv, "z1")
        assert_equal(z2.host()[1], zm2, "z2 mac")
        assert_equal(sig1, osig1, "sigma epoch 0")
        assert_equal(sig2, osig2, "sigma epoch 1")
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p,n,N,off", [(O.P61, 3, 4097, 0), (O.P61, 2, 999, 1), (O.P127, 3, 513, 0), (O.P32, 3, 1025, 1)])
def test_linear_gates_match_oracle(p, n, N, off):
    seed = 5
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, seed, N + off, 0)
        ow = OracleWorld(p, n, seed, N + off, 0)
        (xv, xm, _), (yv, ym, _) = ow.inputs
        sl = lambda a: np.ascontiguousarray(a[:, off:off + N])
        x, y = dw.inputs
        k = (p - 987654321) % p
        for op in (S.SPDZ_OP_ADD, S.SPDZ_OP_SUB, S.SPDZ_OP_CMUL, S.SPDZ_OP_CADD):
            z = SH.alloc(dw.field, n, N + off)
            kh = O.to_array(p, [k])
            S.spdz_linear(ctx, op, x.buf(off), y.buf(off) if op <= 1 else None, kh, z.buf(off), N)
            ev, em = O.linear(p, op, sl(xv), sl(xm), sl(yv), sl(ym), k, ow.alpha_sh)
            gv, gm = z.host()
            assert_equal(gv[:, off:off + N], ev, f"op {op} val")
            assert_equal(gm[:, off:off + N], em, f"op {op} mac")
        # in place: z aliases x
        S.spdz_linear(ctx, S.SPDZ_OP_ADD, x.buf(off), y.buf(off), None, x.buf(off), N)
        ev, em = O.linear(p, O.OP_ADD, sl(xv), sl(xm), sl(yv), sl(ym), 0, ow.alpha_sh)
        assert_equal(x.host()[0][:, off:off + N], ev, "in-place add")
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p,n,off", [(O.P61, 3, 0), (O.P127, 2, 0), (O.P32, 3, 0), (O.P61, 2, 1), (O.P32, 4, 3)])
def test_open_and_check_match_oracle(p, n, off):
    # off = 0 takes the 16-byte vector path with a ragged tail; an odd
    # offset misaligns the rows and takes the one-element path
    N, seed, chk = 2049, 12, 3
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, seed, N + off, 0)
        S.spdz_set_check_seed(ctx, chk)
        out = SH.zeros(dw.field, N)
        S.spdz_open(ctx, dw.inputs[0].buf(off), out, N)
        sig = O.zeros(p, n)
        assert S.spdz_mac_check(ctx, sig)
        ow = OracleWorld(p, n, seed, N + off, 0)
        xv, xm, xs = ow.inputs[0]
        xv, xm, xs = (np.ascontiguousarray(a) for a in (xv[:, off:], xm[:, off:], xs[off:]))
        assert_equal(host(out), xs, "opened values")
        _, osig, _, _ = O.mac_check(p, [O.OpenLog(O.open_(p, xv), xm)], ow.alpha_sh, chk, 0)
        assert_equal(sig, osig, "sigma")
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p,P,L", [(O.P127, 37, 100), (O.P61, 64, 1024), (O.P61, 5, 7), (O.P61, 9, 70), (O.P32, 19, 300)])
def test_innerprod_matches_oracle(p, P, L):
    n, seed, chk = 3, 8, 5
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, seed, P * L, P * L)
        S.spdz_set_check_seed(ctx, chk)
        z = SH.alloc(dw.field, n, P)
        S.spdz_innerprod_batch(ctx, dw.inputs[0].buf(), dw.inputs[1].buf(), z.buf(), P, L)
        sig = O.zeros(p, n)
        assert S.spdz_mac_check(ctx, sig)
        ow = OracleWorld(p, n, seed, P * L, P * L)
        (xv, xm, _), (yv, ym, _) = ow.inputs
        zv, zm, _, _, log = O.innerprod(p, P, L, xv, xm, yv, ym, ow.tri, ow.alpha_sh)
        _, osig, _, _ = O.mac_check(p, [log], ow.alpha_sh, chk, 0)
        gv, gm = z.host()
        assert_equal(gv, zv, "ip val")
        assert_equal(gm, zm, "ip mac")
        assert_equal(sig, osig, "sigma")
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p,n,P,L", [(O.P61, 2, 300, 65), (O.P61, 5, 41, 97), (O.P61, 8, 23, 40),
                                     (O.P32, 4, 77, 129), (O.P61, 3, 5000, 33), (O.P32, 2, 4100, 31),
                                     (O.P61, 3, 3000, 1), (O.P127, 3, 50, 1), (O.P127, 2, 300, 65),
                                     (O.P127, 3, 2000, 33), (O.P127, 4, 23, 40)])
def test_innerprod_party_counts_and_wrapping(p, n, P, L):
    """Inner products for other party counts (the staged kernel's buffer
    grows with n: at n = 8 one CTA per SM) and with more products than the
    grid has warps, so each warp's next-term copies cross into its next
    product; lengths that leave lanes idle in the last step.  For p127 the
    staged kernel takes n = 2 and 3 (2000 products wrap its 1776 warps) and
    the register kernel n = 4."""
    seed, chk = 12, 3
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, seed, P * L, P * L)
        S.spdz_set_check_seed(ctx, chk)
        z = SH.alloc(dw.field, n, P)
        S.spdz_innerprod_batch(ctx, dw.inputs[0].buf(), dw.inputs[1].buf(), z.buf(), P, L)
        sig = O.zeros(p, n)
        assert S.spdz_mac_check(ctx, sig)
        ow = OracleWorld(p, n, seed, P * L, P * L)
        (xv, xm, _), (yv, ym, _) = ow.inputs
        zv, zm, _, _, log = O.innerprod(p, P, L, xv, xm, yv, ym, ow.tri, ow.alpha_sh)
        _, osig, _, _ = O.mac_check(p, [log], ow.alpha_sh, chk, 0)
        gv, gm = z.host()
        assert_equal(gv, zv, "ip val")
        assert_equal(gm, zm, "ip mac")
        assert_equal(sig, osig, "sigma")
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p", [O.P127, O.P61])
def test_innerprod_full_size_sampled(p):
    """The inner-product workload at its full size (16,384 products of
    length 1024, 3 parties, p = 2^127-1 and 2^61-1) in one call: sampled
    products (the first, the last and random ones) against the oracle over
    each product's own 1024 dealt terms; the check over all 2^24 products'
    opened values passes and its sigma sums to zero."""
    n, P, L, seed, chk = 3, 16384, 1024, 23, 6
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, seed, P * L, P * L)
        S.spdz_set_check_seed(ctx, chk)
        z = SH.alloc(dw.field, n, P)
        S.spdz_innerprod_batch(ctx, dw.inputs[0].buf(), dw.inputs[1].buf(), z.buf(), P, L)
        sig = O.zeros(p, n)
        assert S.spdz_mac_check(ctx, sig)
        assert sum(O.to_ints(p, sig)) % p == 0
        gv, gm = z.host()
        alpha, ash = O.deal_alpha(p, n, seed)
        rng = np.random.default_rng(5)
        for q in sorted({0, 1, P // 2, P - 1, *rng.integers(0, P, 8).tolist()}):
            j0 = q * L
            xv, xm, _ = O.deal_shared(p, n, seed, O.K_INPUT, 0, j0, L, alpha)
            yv, ym, _ = O.deal_shared(p, n, seed, O.K_INPUT, 1, j0, L, alpha)
            tri = O.deal_triples(p, n, seed, j0, L, alpha)
            zv, zm, _, _, _ = O.innerprod(p, 1, L, xv, xm, yv, ym, tri, ash)
            assert_equal(gv[:, q], zv[:, 0], f"ip val {q}")
            assert_equal(gm[:, q], zm[:, 0], f"ip mac {q}")
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p", [O.P61, O.P127, O.P32])
def test_tampered_share_fails_check_like_oracle(p):
    """A cheating party shifts its share of a by Delta before the multiply:
    the opened eps no longer matches its MACs and the check must fail, with
    the same sigma the oracle computes for the same tamper."""
    n, N, seed, chk, j, party, delta = 3, 512, 40, 41, 100, 1, 123456789
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, seed, N, N)
        ow = OracleWorld(p, n, seed, N, N)
        av = ow.tri.av.copy()
        old = O.to_ints(p, av[party, j:j + 1])[0]
        av[party, j] = O.to_array(p, [(old + delta) % p])[0]
        dw.tri[0].val[party, j] = SH.from_host(av[party, j:j + 1], field=dw.field)[0]
        S.spdz_set_check_seed(ctx, chk)
        z = SH.alloc(dw.field, n, N)
        S.spdz_mul_batch(ctx, dw.inputs[0].buf(), dw.inputs[1].buf(), z.buf(), N)
        sig = O.zeros(p, n)
        assert not S.spdz_mac_check(ctx, sig)
        tri = O.Triples(av, ow.tri.am, ow.tri.bv, ow.tri.bm, ow.tri.cv, ow.tri.cm)
        (xv, xm, _), (yv, ym, _) = ow.inputs
        *_, log = O.mul(p, xv, xm, yv, ym, tri, ow.alpha_sh)
        ok, osig, _, _ = O.mac_check(p, [log], ow.alpha_sh, chk, 0)
        assert not ok
        assert_equal(sig, osig, "sigma under tamper")
        r = O.to_ints(p, O.check_coeffs(p, chk, 0, 2 * j, 1))[0]
        al = O.to_ints(p, np.array([ow.alpha]))[0]
        assert sum(O.to_ints(p, sig)) % p == (al * r * delta) % p   # eps_j shifted by -Delta
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p", [O.P61, O.P127, O.P32])
def test_degenerate_sizes(p):
    """Empty calls: a batch, an open and a linear gate of 0 elements do
    nothing and consume no triples; inner products of length 0 are empty
    sums, every share and MAC share 0; the check afterwards passes."""
    n = 3
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, 2, 64, 64)
        x, y = dw.inputs
        z = SH.alloc(dw.field, n, 8)
        left = S.spdz_triples_left(ctx)
        S.spdz_mul_batch(ctx, x.buf(), y.buf(), z.buf(), 0)
        S.spdz_innerprod_batch(ctx, x.buf(), y.buf(), z.buf(), 0, 16)
        S.spdz_linear(ctx, S.SPDZ_OP_ADD, x.buf(), y.buf(), None, z.buf(), 0)
        out = torch.zeros(16, dtype=torch.int64, device="cuda")
        S.spdz_open(ctx, x.buf(), out, 0)
        assert S.spdz_triples_left(ctx) == left
        # 8 inner products of length 0: fill the outputs with nonzero words first
        z.val.fill_(1)
        z.mac.fill_(1)
        S.spdz_innerprod_batch(ctx, x.buf(), y.buf(), z.buf(), 8, 0)
        gv, gm = z.host()
        assert not np.any(O.to_ints(p, gv)) and not np.any(O.to_ints(p, gm))
        assert S.spdz_triples_left(ctx) == left
        assert S.spdz_mac_check(ctx)
    finally:
        S.spdz_ctx_destroy(ctx)


def test_errors_are_status_codes():
    p, n = O.P61, 2
    ctx = ctx_for(n, p)
    try:
        dw = DeviceWorld(ctx, p, n, 1, 64, 10)
        z = SH.alloc(dw.field, n, 64)
        x, y = dw.inputs
        with pytest.raises(S.SpdzError) as e:
            S.spdz_mul_batch(ctx, x.buf(), y.buf(), z.buf(), 64)
        assert e.value.code == S.SPDZ_ERR_TRIPLES
        assert S.spdz_triples_left(ctx) == 10
        bad = S.spdz_buf(x.val.data_ptr() + 4, x.mac.data_ptr(), x.stride)
        with pytest.raises(S.SpdzError) as e:
            S.spdz_linear(ctx, S.SPDZ_OP_ADD, bad, y.buf(), None, z.buf(), 8)
        assert e.value.code == S.SPDZ_ERR_ALIGN
        short = S.spdz_buf(x.val.data_ptr(), x.mac.data_ptr(), 8)
        with pytest.raises(S.SpdzError) as e:
            S.spdz_linear(ctx, S.SPDZ_OP_ADD, short, y.buf(), None, z.buf(), 64)
        assert e.value.code == S.SPDZ_ERR_ARG
        S.spdz_mul_batch(ctx, x.buf(), y.buf(), z.buf(), 5)
        with pytest.raises(S.SpdzError) as e:
            S.spdz_set_check_seed(ctx, 3)
        assert e.value.code == S.SPDZ_ERR_STATE
        assert S.spdz_mac_check(ctx)
        S.spdz_set_check_seed(ctx, 3)
        with pytest.raises(S.SpdzError) as e:
            S.spdz_ctx_create(9, S.SPDZ_F61)
        assert e.value.code == S.SPDZ_ERR_ARG
    finally:
        S.spdz_ctx_destroy(ctx)
