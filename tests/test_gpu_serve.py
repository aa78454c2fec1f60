"""The serving loop: requests of both fields arrive over time, are admitted by
a device-memory budget and served by continuous batching (and by cluster
launches for narrow requests).  Every request's shares must equal the CPU
oracle's evaluation of that request alone -- the same alone and in the mix,
in every mode."""
import numpy as np
import pytest
import torch

import oracle as O
import spdz_workloads as W

pytestmark = pytest.mark.gpu

from gpu_helpers import assert_equal  # noqa: E402

N = 3


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    global S, SH
    from paper_2512_11112_b300 import shares as SH  # noqa: F401
    from paper_2512_11112_b300 import spdz as S  # noqa: F401
    yield


def small_trace(count=10, seed=31, rate=2000.0):
    reqs = W.serving_requests(seed=seed, count=count, rate_per_s=rate, gmin=64, gmax=3000, dmin=2, dmax=9)
    return [(r, W.request_dag(r)) for r in reqs]


def oracle_wires(req, dag):
    p = req.p
    alpha, ash = O.deal_alpha(p, N, req.seed)
    iv, im, _ = O.deal_shared(p, N, req.seed, O.K_INPUT, 16, 0, dag.n_inputs, alpha)
    wv, wm = O.zeros(p, N, dag.n_wires), O.zeros(p, N, dag.n_wires)
    wv[:, :dag.n_inputs], wm[:, :dag.n_inputs] = iv, im
    tri = O.deal_triples(p, N, req.seed, 0, dag.n_mul, alpha)
    O.dag_eval(p, dag, wv, wm, tri, ash)
    return wv, wm


def serve(trace, mode, budget=1 << 30, max_active=64, arrivals=True, model_ctx=None, cluster_width=0):
    server = S.spdz_serve_create(N, budget, max_active, mode, model_ctx, 0, cluster_width)
    try:
        outs, items = [], []
        for r, dag in trace:
            ov, om = O.zeros(r.p, N, dag.n_wires), O.zeros(r.p, N, dag.n_wires)
            outs.append((ov, om))
            field = S.SPDZ_F61 if r.p == O.P61 else S.SPDZ_F127
            items.append((dag, field, r.seed, r.arrival_s if arrivals else 0.0, ov, om))
        res, st = S.spdz_serve_run(server, items)
        return outs, res, st
    finally:
        S.spdz_serve_destroy(server)


def test_served_results_equal_oracle_alone_and_in_the_mix():
    trace = small_trace()
    expect = [oracle_wires(r, d) for r, d in trace]
    for mode, kw in ((S.SPDZ_SERVE_BATCHED, {}), (S.SPDZ_SERVE_HEURISTIC, {"cluster_width": 1024}),
                     (S.SPDZ_SERVE_SEQUENTIAL, {})):
        outs, res, st = serve(trace, mode, **kw)
        assert st.requests == len(trace) and st.gates == sum(d.n_gates for _, d in trace)
        for k, ((ov, om), (ev, em)) in enumerate(zip(outs, expect)):
            assert res[k].passed == 1, (mode, k)
            assert_equal(ov, ev, f"mode {mode} request {k} values")
            assert_equal(om, em, f"mode {mode} request {k} MACs")
        if mode == S.SPDZ_SERVE_HEURISTIC:
            assert st.cluster_requests > 0
        if mode == S.SPDZ_SERVE_SEQUENTIAL:
            assert st.max_active == 1
    # each request alone gives the same shares as in the mix
    for k in (0, 3):
        outs, res, st = serve([trace[k]], S.SPDZ_SERVE_BATCHED, arrivals=False)
        assert_equal(outs[0][0], expect[k][0], f"request {k} alone")


def test_wide_layers_equal_oracle():
    """Layers of 70k-440k gates (up to 1,720 tiles of one request in a tick,
    each tile finding its request on the device): two wide requests (p61 and
    p127) in the mix with small ones, every wire equals the oracle's and
    every check passes."""
    wide = [W.Request(rid=0, arrival_s=0.0, p=O.P61, gates=600000, depth=3, seed=41),
            W.Request(rid=1, arrival_s=0.0, p=O.P127, gates=300000, depth=2, seed=42)]
    trace = [(r, W.request_dag(r)) for r in wide] + small_trace(count=4, seed=43)
    assert max(int(np.max(np.diff(d.layer_offsets))) for _, d in trace[:2]) > 65536
    expect = [oracle_wires(r, d) for r, d in trace]
    for mode, kw in ((S.SPDZ_SERVE_BATCHED, {}), (S.SPDZ_SERVE_HEURISTIC, {"cluster_width": 1024})):
        outs, res, st = serve(trace, mode, **kw)
        assert st.requests == len(trace)
        for k, ((ov, om), (ev, em)) in enumerate(zip(outs, expect)):
            assert res[k].passed == 1, (mode, k)
            assert_equal(ov, ev, f"mode {mode} request {k} values")
            assert_equal(om, em, f"mode {mode} request {k} MACs")


def test_grid_launch_requests_equal_oracle():
    """Requests of at least 2^20 gates (p61 and p127) run in the heuristic
    mode as one fused launch each (a cooperative launch with device barriers
    between layers, on a side stream), beside small requests in ticks and
    cluster launches: every wire equals the oracle's and every check
    passes."""
    big = [W.Request(rid=0, arrival_s=0.0, p=O.P61, gates=1200000, depth=4, seed=51),
           W.Request(rid=1, arrival_s=0.0, p=O.P127, gates=1100000, depth=3, seed=52)]
    trace = [(r, W.request_dag(r)) for r in big] + small_trace(count=4, seed=53)
    assert all(d.n_gates >= 2**20 for _, d in trace[:2])
    O.set_threads(8)
    expect = [oracle_wires(r, d) for r, d in trace]
    outs, res, st = serve(trace, S.SPDZ_SERVE_HEURISTIC, budget=2 << 30, cluster_width=1024)
    assert st.requests == len(trace) and st.grid_requests == 2
    assert [res[k].mode for k in range(2)] == [2, 2]
    for k, ((ov, om), (ev, em)) in enumerate(zip(outs, expect)):
        assert res[k].passed == 1, k
        assert_equal(ov, ev, f"grid-launch trace, request {k} values")
        assert_equal(om, em, f"grid-launch trace, request {k} MACs")


def test_admission_respects_the_memory_budget():
    trace = small_trace(count=12, seed=8, rate=1e6)     # all arrive at once
    per = []
    for r, d in trace:
        eb = 8 if r.p == O.P61 else 16
        per.append(2 * N * d.n_wires * eb + 6 * N * max(1, d.n_mul) * eb + (16 + eb) * d.n_gates)
    budget = int(max(per) * 2.5) + (1 << 20)
    outs, res, st = serve(trace, S.SPDZ_SERVE_BATCHED, budget=budget)
    assert st.peak_bytes <= budget
    assert st.max_active < len(trace)                   # the budget held requests back
    assert all(r.passed == 1 for r in res)
    expect = oracle_wires(*trace[-1])
    assert_equal(outs[-1][0], expect[0], "last request values")
    # a request that can never fit is refused
    r = W.Request(rid=0, arrival_s=0.0, p=O.P127, gates=200000, depth=4, seed=5)
    big = [(r, W.request_dag(r))]
    with pytest.raises(S.SpdzError) as e:
        serve(big, S.SPDZ_SERVE_BATCHED, budget=1 << 20)
    assert e.value.code == S.SPDZ_ERR_OOM


def test_two_hundred_request_trace_every_result_equals_oracle():
    """200 requests of both fields (gate counts 2^6..2^12, depths 2..16),
    arriving over time, served with continuous batching and cluster launches
    for narrow requests: every request's wires equal the oracle's."""
    reqs = W.serving_requests(seed=77, count=200, rate_per_s=20000.0, gmin=64, gmax=4096, dmin=2, dmax=16)
    trace = [(r, W.request_dag(r)) for r in reqs]
    outs, res, st = serve(trace, S.SPDZ_SERVE_HEURISTIC, max_active=32, cluster_width=512)
    assert st.requests == 200 and st.cluster_requests > 0 and st.max_active > 1
    O.set_threads(8)
    for k, (r, d) in enumerate(trace):
        ev, em = oracle_wires(r, d)
        assert res[k].passed == 1, k
        assert_equal(outs[k][0], ev, f"request {k} values")
        assert_equal(outs[k][1], em, f"request {k} MACs")


@pytest.fixture(scope="module")
def model_ctx():
    """A p61 context whose cost model is trained (the library's own training
    kernels) on per-layer timings it records of the calibration circuits."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2512_11112_b300 import shares as SH_
    from paper_2512_11112_b300 import spdz as S_
    p = O.P61
    f = SH_.field_of(p)
    ctx = S_.spdz_ctx_create(N, f, torch.cuda.current_stream().cuda_stream)
    ash = SH_.zeros(f, N)
    S_.spdz_deal_alpha(ctx, 3, ash)
    dags = W.calibration_dags(p)
    ncfg, _ = S_.spdz_sched_num_configs()
    T = sum(d.n_mul for d in dags) * (ncfg + 2) * 2
    tri = [SH_.alloc(f, N, T) for _ in range(3)]
    S_.spdz_deal_triples(ctx, 3, 0, T, ash, *[t.buf() for t in tri])
    S_.spdz_load_preproc(ctx, ash, *[t.buf() for t in tri], T)
    for d in dags:
        w = SH_.alloc(f, N, d.n_wires)
        S_.spdz_deal_shared(ctx, 3, S_.SPDZ_KIND_INPUT, 16, 0, d.n_inputs, ash, None, w.buf())
        h = S_.spdz_dag_create(ctx, d.n_inputs, d.layer_offsets, d.ops, d.in0, d.in1, d.kconst)
        S_.spdz_sched_record(ctx, h, w.buf(), 1)
        S_.spdz_dag_destroy(h)
    loss = S_.spdz_sched_train(ctx, epochs=300, lr=2e-3, seed=1)
    assert loss < 0.1, loss
    yield ctx
    S_.spdz_ctx_destroy(ctx)


def test_learned_mode_every_result_equals_oracle(model_ctx):
    """The learned serving mode (the cost model decides, per request, between
    ticks, one cluster launch and one grid launch): every request of a mixed-field trace
    equals the oracle's evaluation of that request alone, with its check
    passed; the same requests alone give the same shares.  The p99 latency of
    the learned, heuristic and batched modes on the same 200-request trace
    is printed beside the result."""
    trace = small_trace()
    expect = [oracle_wires(r, d) for r, d in trace]
    outs, res, st = serve(trace, S.SPDZ_SERVE_LEARNED, model_ctx=model_ctx)
    assert st.requests == len(trace)
    for k, ((ov, om), (ev, em)) in enumerate(zip(outs, expect)):
        assert res[k].passed == 1 and res[k].mode in (0, 1, 2), k
        assert_equal(ov, ev, f"learned mode request {k} values")
        assert_equal(om, em, f"learned mode request {k} MACs")
    for k in (1, 4):
        o1, r1, _ = serve([trace[k]], S.SPDZ_SERVE_LEARNED, arrivals=False, model_ctx=model_ctx)
        assert r1[0].passed == 1
        assert_equal(o1[0][0], expect[k][0], f"learned mode request {k} alone, values")
        assert_equal(o1[0][1], expect[k][1], f"learned mode request {k} alone, MACs")

    reqs = W.serving_requests(seed=77, count=200, rate_per_s=20000.0, gmin=64, gmax=4096, dmin=2, dmax=16)
    big = [(r, W.request_dag(r)) for r in reqs]
    outs, res, st = serve(big, S.SPDZ_SERVE_LEARNED, max_active=32, model_ctx=model_ctx)
    assert st.requests == 200 and st.max_active > 1
    O.set_threads(8)
    for k, (r, d) in enumerate(big):
        ev, em = oracle_wires(r, d)
        assert res[k].passed == 1, k
        assert_equal(outs[k][0], ev, f"learned mode, 200-request trace, request {k} values")
        assert_equal(outs[k][1], em, f"learned mode, 200-request trace, request {k} MACs")
    p99 = {"learned": st.p99_s * 1e3, "learned_cluster_requests": int(st.cluster_requests)}
    for name, mode in (("heuristic", S.SPDZ_SERVE_HEURISTIC), ("batched", S.SPDZ_SERVE_BATCHED)):
        _, r2, s2 = serve(big, mode, max_active=32, cluster_width=512)
        assert all(x.passed == 1 for x in r2)
        p99[name] = s2.p99_s * 1e3
    print("p99 ms on the 200-request trace:", p99)


def test_submit_while_others_run_poll_and_stop():
    """The server's own calls: requests are submitted from the host while
    earlier ones are still on the GPU (a poll just before each later
    submission finds an earlier request not yet done), some by registered
    circuit id and some as one-off circuits, some with the caller's own input
    shares (the oracle's dealt shares, the same values the device dealer
    would produce); every result, collected by polling, equals the oracle's
    evaluation of that request alone."""
    import time
    reqs = W.serving_requests(seed=41, count=24, rate_per_s=1e6, gmin=2000, gmax=60000, dmin=6, dmax=24)
    trace = [(r, W.request_dag(r)) for r in reqs]
    server = S.spdz_serve_create(N, 2 << 30, 8, S.SPDZ_SERVE_HEURISTIC, None, 0, 2048)
    try:
        reg = {}
        for k in range(0, len(trace), 3):
            r, d = trace[k]
            reg[k] = S.spdz_serve_register(server, d, S.SPDZ_F61 if r.p == O.P61 else S.SPDZ_F127)
        S.spdz_serve_start(server)
        ids, outs, overlapped = [], [], 0
        for k, (r, d) in enumerate(trace):
            field = S.SPDZ_F61 if r.p == O.P61 else S.SPDZ_F127
            out = (O.zeros(r.p, N, d.n_wires), O.zeros(r.p, N, d.n_wires))
            inputs = None
            if k % 2 == 1:
                alpha, _ = O.deal_alpha(r.p, N, r.seed)
                iv, im, _ = O.deal_shared(r.p, N, r.seed, O.K_INPUT, 16, 0, d.n_inputs, alpha)
                inputs = (iv, im)
            if ids:
                done, _ = S.spdz_serve_poll(server, ids[-1])
                if not done:
                    overlapped += 1
                else:
                    ids[-1] = -ids[-1]          # collected already (result checked below)
            rid = S.spdz_serve_submit(server, reg.get(k, d), field, r.seed, inputs=inputs, out=out)
            ids.append(rid)
            outs.append(out)
        assert overlapped > 0
        results = {}
        t0 = time.time()
        while len(results) < sum(1 for i in ids if i > 0) and time.time() - t0 < 120:
            for i in ids:
                if i > 0 and i not in results:
                    done, res = S.spdz_serve_poll(server, i)
                    if done:
                        results[i] = res
            time.sleep(0.002)
        st = S.spdz_serve_stop(server)
        assert st.requests == len(trace) and st.max_active > 1
        with pytest.raises(S.SpdzError) as e:                 # not running
            S.spdz_serve_submit(server, trace[0][1], S.SPDZ_F61 if trace[0][0].p == O.P61 else S.SPDZ_F127, 1)
        assert e.value.code == S.SPDZ_ERR_STATE
        for i in results:
            with pytest.raises(S.SpdzError):                  # handed out once
                S.spdz_serve_poll(server, i)
        O.set_threads(8)
        for k, ((r, d), i, (ov, om)) in enumerate(zip(trace, ids, outs)):
            if i > 0:
                assert results[i].passed == 1 and results[i].status == S.SPDZ_OK, k
            ev, em = oracle_wires(r, d)
            assert_equal(ov, ev, f"submitted request {k} values")
            assert_equal(om, em, f"submitted request {k} MACs")
    finally:
        S.spdz_serve_destroy(server)


def test_registered_circuits_count_against_the_budget():
    """A registered circuit's gate records live in the arena: registering more
    than the budget holds is refused (SPDZ_ERR_OOM), unregistering gives the
    room back, and registration is refused while the server runs."""
    r = W.Request(rid=0, arrival_s=0.0, p=O.P61, gates=40000, depth=8, seed=3)
    d = W.request_dag(r)
    server = S.spdz_serve_create(N, 1 << 20, 4, S.SPDZ_SERVE_BATCHED, None, 0, 0)
    try:
        with pytest.raises(S.SpdzError) as e:
            for _ in range(4):                                # 40k gates x 24 B: about 1 MB each
                S.spdz_serve_register(server, d, S.SPDZ_F61)
        assert e.value.code == S.SPDZ_ERR_OOM
    finally:
        S.spdz_serve_destroy(server)
    server = S.spdz_serve_create(N, 64 << 20, 4, S.SPDZ_SERVE_BATCHED, None, 0, 0)
    try:
        cid = S.spdz_serve_register(server, d, S.SPDZ_F61)
        S.spdz_serve_unregister(server, cid)
        cid = S.spdz_serve_register(server, d, S.SPDZ_F61)
        S.spdz_serve_start(server)
        with pytest.raises(S.SpdzError) as e:
            S.spdz_serve_register(server, d, S.SPDZ_F61)
        assert e.value.code == S.SPDZ_ERR_STATE
        out = (O.zeros(r.p, N, d.n_wires), O.zeros(r.p, N, d.n_wires))
        rid = S.spdz_serve_submit(server, cid, S.SPDZ_F61, r.seed, out=out)
        st = S.spdz_serve_stop(server)
        done, res = S.spdz_serve_poll(server, rid)
        assert done and res.passed == 1 and st.requests == 1
        assert st.peak_bytes <= 64 << 20
        ev, em = oracle_wires(r, d)
        assert_equal(out[0], ev, "registered circuit values")
        assert_equal(out[1], em, "registered circuit MACs")
    finally:
        S.spdz_serve_destroy(server)
