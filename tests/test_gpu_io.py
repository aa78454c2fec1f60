"""Input sharing and the checked reveal on the GPU: the device's input masks
and input shares equal the oracle's, a reveal releases the values only when
the MAC check passes, and a whole run -- clear inputs of two owners shared,
a circuit evaluated, its outputs revealed -- gives the cleartext circuit's
outputs."""
import numpy as np
import pytest
import torch

import oracle as O
import spdz_workloads as W

pytestmark = pytest.mark.gpu

from gpu_helpers import assert_equal, ctx_for  # noqa: E402


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    global S, SH
    from paper_2512_11112_b300 import shares as SH  # noqa: F401
    from paper_2512_11112_b300 import spdz as S  # noqa: F401
    yield
    torch.cuda.synchronize()


def clear_values(p, count, seed):
    rng = np.random.default_rng(seed)
    xs = [int(v) % p for v in rng.integers(0, 2**62, count)]
    if count >= 3:
        xs[:3] = [0, 1, p - 1]
    return xs


@pytest.mark.parametrize("p,n,count,off", [(O.P61, 2, 1000, 0), (O.P127, 3, 333, 0), (O.P32, 4, 4097, 0),
                                           (O.P61, 3, 1001, 1), (O.P32, 2, 999, 3)])
def test_input_sharing_matches_oracle(p, n, count, off):
    # off = 0: 16-byte vector accesses (with a ragged tail for odd counts);
    # an output offset that breaks the rows' 16-byte alignment takes the
    # one-element path
    seed, owner = 9, n - 1
    ctx = ctx_for(n, p)
    f = SH.field_of(p)
    try:
        ash = SH.zeros(f, n)
        S.spdz_deal_alpha(ctx, seed, ash)
        S.spdz_load_preproc(ctx, ash, None, None, None, 0)
        S.spdz_set_check_seed(ctx, 5)
        masks, r = SH.alloc(f, n, count), SH.zeros(f, count)
        S.spdz_deal_input_masks(ctx, seed, owner, 0, count, ash, masks.buf(), r)
        xs = clear_values(p, count, p % 997)
        x = SH.from_host(O.to_array(p, xs), field=f)
        out, eps = SH.alloc(f, n, count + off), SH.zeros(f, count)
        S.spdz_input(ctx, x, r, masks.buf(), out.buf(off), count, eps)
        alpha, oash = O.deal_alpha(p, n, seed)
        rv, rm, rc = O.deal_input_masks(p, n, seed, owner, 0, count, alpha)
        assert_equal(masks.host()[0], rv, "mask values")
        assert_equal(masks.host()[1], rm, "mask MACs")
        assert_equal(SH.to_host(r), rc, "clear masks")
        xv, xm, oeps = O.input_share(p, O.to_array(p, xs), rc, rv, rm, oash)
        assert_equal(SH.to_host(eps), oeps, "eps")
        assert_equal(out.host()[0][:, off:], xv, "input value shares")
        assert_equal(out.host()[1][:, off:], xm, "input MAC shares")
        # the reveal releases exactly the inputs
        got = SH.zeros(f, count)
        sig = O.zeros(p, n)
        assert S.spdz_reveal(ctx, out.buf(off), got, count, sig)
        assert_equal(SH.to_host(got), O.to_array(p, xs), "revealed")
        ok, osig, _, _ = O.mac_check(p, [O.OpenLog(O.to_array(p, xs), xm)], oash, 5, 0)
        assert ok
        assert_equal(sig, osig, "sigma of the reveal")
        assert sum(O.to_ints(p, sig)) % p == 0
        # a tampered share: the check fails and nothing is released
        out.val[1, off + 7] = out.val[1, off + 8]
        got2 = SH.zeros(f, count)
        assert not S.spdz_reveal(ctx, out.buf(off), got2, count)
        assert not np.any(SH.to_host(got2))
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p,n", [(O.P61, 3), (O.P32, 2), (O.P127, 2)])
def test_inputs_circuit_reveal_equals_cleartext(p, n):
    """Inputs 0..h-1 belong to party 0 and h.. to party 1; both are shared
    with their masks, the circuit runs (fused plan), the last layer's outputs
    are revealed; they equal the cleartext evaluation of the circuit."""
    dag = W.small_dag(seed=5, p=p, n_inputs=80, widths=[60, 1, 45, 33])
    seed = 12
    ctx = ctx_for(n, p)
    f = SH.field_of(p)
    try:
        ash = SH.zeros(f, n)
        S.spdz_deal_alpha(ctx, seed, ash)
        T = max(1, dag.n_mul)
        tri = [SH.alloc(f, n, T) for _ in range(3)]
        S.spdz_deal_triples(ctx, seed, 0, T, ash, *[t.buf() for t in tri])
        S.spdz_load_preproc(ctx, ash, *[t.buf() for t in tri], T)
        S.spdz_set_check_seed(ctx, 3)
        wires = SH.alloc(f, n, dag.n_wires)
        xs = clear_values(p, dag.n_inputs, 77)
        h = dag.n_inputs // 2
        for owner, lo, hi in ((0, 0, h), (1, h, dag.n_inputs)):
            masks, r = SH.alloc(f, n, hi - lo), SH.zeros(f, hi - lo)
            S.spdz_deal_input_masks(ctx, seed, owner, 0, hi - lo, ash, masks.buf(), r)
            x = SH.from_host(O.to_array(p, xs[lo:hi]), field=f)
            S.spdz_input(ctx, x, r, masks.buf(), wires.buf(lo), hi - lo)
        h_dag = S.spdz_dag_create(ctx, dag.n_inputs, dag.layer_offsets, dag.ops, dag.in0, dag.in1, dag.kconst)
        try:
            S.spdz_run_dag(ctx, h_dag, S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=0), wires.buf())
        finally:
            S.spdz_dag_destroy(h_dag)
        first = dag.n_inputs + int(dag.layer_offsets[-2])
        count = dag.n_wires - first
        got = SH.zeros(f, count)
        assert S.spdz_reveal(ctx, wires.buf(first), got, count)
        clear = O.dag_clear(p, dag, O.to_array(p, xs))
        assert_equal(SH.to_host(got), clear[first:], "revealed outputs")
    finally:
        S.spdz_ctx_destroy(ctx)


@pytest.mark.parametrize("p", [O.P61, O.P32])
def test_open_input_reveal_full_size_sampled(p):
    """The sizes the batch benchmark times: 2^24 elements, 3 parties, one
    call each on the full buffers (16-byte vector kernels).  The open of
    dealt shares, the input sharing of the opened values and their reveal;
    sampled elements (the ends, the middle, vector edges, random indices)
    against the oracle dealing each sampled index from the same counters;
    both checks pass and the first one's sigma sums to zero."""
    n, N, seed, chk, owner = 3, 2**24, 57, 23, 1
    f = SH.field_of(p)
    ctx = ctx_for(n, p)
    try:
        ash = SH.zeros(f, n)
        S.spdz_deal_alpha(ctx, seed, ash)
        S.spdz_load_preproc(ctx, ash, None, None, None, 0)
        S.spdz_set_check_seed(ctx, chk)
        x = SH.alloc(f, n, N)
        S.spdz_deal_shared(ctx, seed, S.SPDZ_KIND_INPUT, 0, 0, N, ash, None, x.buf())
        pub = SH.zeros(f, N)
        S.spdz_open(ctx, x.buf(), pub, N)
        sigma = O.zeros(p, n)
        assert S.spdz_mac_check(ctx, sigma)
        assert sum(O.to_ints(p, sigma)) % p == 0
        masks, r = SH.alloc(f, n, N), SH.zeros(f, N)
        S.spdz_deal_input_masks(ctx, seed, owner, 0, N, ash, masks.buf(), r)
        out, eps = SH.alloc(f, n, N), SH.zeros(f, N)
        S.spdz_input(ctx, pub, r, masks.buf(), out.buf(), N, eps)
        got = SH.zeros(f, N)
        assert S.spdz_reveal(ctx, out.buf(), got, N)
        rng = np.random.default_rng(5)
        idx = np.unique(np.concatenate([[0, 1, 2, 3, 4, N // 2 - 1, N // 2, N - 5, N - 2, N - 1],
                                        rng.integers(0, N, 20)])).astype(np.int64)
        ti = torch.from_numpy(idx).to(pub.device)
        g_pub, g_eps, g_rev = SH.to_host(pub[ti]), SH.to_host(eps[ti]), SH.to_host(got[ti])
        g_ov, g_om = SH.to_host(out.val[:, ti]), SH.to_host(out.mac[:, ti])
        alpha, oash = O.deal_alpha(p, n, seed)
        for s_, j in enumerate(idx.tolist()):
            xv, xm, xs = O.deal_shared(p, n, seed, O.K_INPUT, 0, j, 1, alpha)
            assert_equal(g_pub[s_:s_ + 1], O.open_(p, xv), f"opened value at {j}")
            assert_equal(g_pub[s_:s_ + 1], xs, f"opened value = dealt secret at {j}")
            rv, rm, rc = O.deal_input_masks(p, n, seed, owner, j, 1, alpha)
            iv, im, ieps = O.input_share(p, xs, rc, rv, rm, oash)
            assert_equal(g_eps[s_:s_ + 1], ieps, f"eps at {j}")
            assert_equal(g_ov[:, s_:s_ + 1], iv, f"input value shares at {j}")
            assert_equal(g_om[:, s_:s_ + 1], im, f"input MAC shares at {j}")
            assert_equal(g_rev[s_:s_ + 1], xs, f"revealed at {j}")
    finally:
        S.spdz_ctx_destroy(ctx)
