"""Layered-circuit runs on the GPU against the CPU oracle: every wire share
and MAC share, the opened values' check sigma and the verdict, bit-exact, for
every execution form (per-layer launches, fused persistent kernels with one or
several groups and partial checks, CUDA-graph replay)."""
import numpy as np
import pytest
import torch

import oracle as O
import spdz_workloads as W

pytestmark = pytest.mark.gpu

from gpu_helpers import assert_equal, ctx_for  # noqa: E402

INPUT_SUB = 16


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    global S, SH
    from paper_2512_11112_b300 import shares as SH  # noqa: F401
    from paper_2512_11112_b300 import spdz as S  # noqa: F401
    yield
    torch.cuda.synchronize()


class DeviceCircuit:
    def __init__(self, dag, n, seed, runs=1, check_seed=7):
        self.dag, self.n, self.seed = dag, n, seed
        self.field = SH.field_of(dag.p)
        self.ctx = ctx_for(n, dag.p)
        self.alpha_sh = SH.zeros(self.field, n)
        S.spdz_deal_alpha(self.ctx, seed, self.alpha_sh)
        self.wires = SH.alloc(self.field, n, dag.n_wires)
        self.deal_inputs()
        T = runs * dag.n_mul
        self.tri = [SH.alloc(self.field, n, max(T, 1)) for _ in range(3)]
        if T:
            S.spdz_deal_triples(self.ctx, seed, 0, T, self.alpha_sh, *[t.buf() for t in self.tri])
        S.spdz_load_preproc(self.ctx, self.alpha_sh, *[t.buf() for t in self.tri], T)
        S.spdz_set_check_seed(self.ctx, check_seed)
        self.h = S.spdz_dag_create(self.ctx, dag.n_inputs, dag.layer_offsets, dag.ops, dag.in0,
                                   dag.in1, dag.kconst)

    def deal_inputs(self):
        S.spdz_deal_shared(self.ctx, self.seed, S.SPDZ_KIND_INPUT, INPUT_SUB, 0, self.dag.n_inputs,
                           self.alpha_sh, None, self.wires.buf())

    def run(self, plan):
        st = S.spdz_run_dag(self.ctx, self.h, plan, self.wires.buf())
        sig = O.zeros(self.dag.p, self.n)
        passed = S.spdz_check_result(self.ctx, sig)
        return st, passed, sig

    def close(self):
        S.spdz_dag_destroy(self.h)
        S.spdz_ctx_destroy(self.ctx)


def oracle_run(dag, n, seed, run_index=0, check_seed=7):
    p = dag.p
    alpha, ash = O.deal_alpha(p, n, seed)
    iv, im, _ = O.deal_shared(p, n, seed, O.K_INPUT, INPUT_SUB, 0, dag.n_inputs, alpha)
    wv, wm = O.zeros(p, n, dag.n_wires), O.zeros(p, n, dag.n_wires)
    wv[:, :dag.n_inputs], wm[:, :dag.n_inputs] = iv, im
    tri = O.deal_triples(p, n, seed, run_index * dag.n_mul, dag.n_mul, alpha)
    _, _, log = O.dag_eval(p, dag, wv, wm, tri, ash)
    ok, sigma, _, _ = O.mac_check(p, [log], ash, check_seed, run_index)
    return wv, wm, ok, sigma


def plans(depth, p=None):
    mid = max(1, depth // 2)
    out = {
        "per_layer": S.plan(mode=S.SPDZ_SCHED_PER_LAYER, use_graph=0),
        "per_layer_graph": S.plan(mode=S.SPDZ_SCHED_PER_LAYER, use_graph=1),
        "fused": S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=0),
        "fused_graph": S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1),
        "fused_1cta": S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=0, ctas_per_sm=1, block=64),
    }
    if depth > 1:
        out["groups_flush"] = S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1, groups=[mid, depth],
                                     flush=[1, 0], group_ctas=[1, 0])
    if depth > 2:
        out["every_layer_group"] = S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=0,
                                          groups=list(range(1, depth + 1)), flush=[1] * depth)
    out["one_cluster16"] = S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1, groups=[depth], group_cluster=[16])
    if depth > 1:
        out["cluster_then_grid"] = S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1, groups=[mid, depth],
                                          group_cluster=[8, 0], flush=[1, 0])
        out["grid_then_cluster_small_block"] = S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=0, block=64,
                                                      groups=[mid, depth], group_cluster=[0, 3])
    if p == O.P61:
        out["tagged"] = S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=0)
        out["tagged_graph"] = S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=1)
        out["tagged_1cta_small_block"] = S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=0, ctas_per_sm=1, block=32)
        out["tagged_slack"] = S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=1, barrier_slack=3)
        # slack above the grid size: no CTA ever waits at a layer barrier
        out["tagged_no_wait"] = S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=0, barrier_slack=10**6, poll_ns=32)
        # tagged groups inside fused plans: a whole-circuit tagged group; a
        # grid group, then a tagged group (its first layer reads the grid
        # group's outputs from the party-major wires); tagged, cluster,
        # tagged (the last group's last CTA runs the check) with a flush
        out["tagged_group"] = S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1, groups=[depth], group_tagged=[1],
                                     barrier_slack=2)
        if depth > 1:
            out["grid_then_tagged"] = S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=0, groups=[mid, depth],
                                             group_tagged=[0, 1], flush=[1, 0])
        if depth > 2:
            out["tagged_cluster_tagged"] = S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1, groups=[1, mid + 1, depth],
                                                  group_tagged=[1, 0, 1], group_cluster=[0, 8, 0], flush=[1, 0, 0],
                                                  barrier_slack=1)
    return out


SMALL = [
    (O.P61, 3, [30, 17, 1, 25, 9, 300, 2]),
    (O.P127, 2, [64, 3, 129, 40]),
    (O.P61, 2, [1]),
    (O.P127, 3, [5, 1000, 77]),
    (O.P32, 3, [40, 1, 300, 77]),       # p = 2^32-5
]


@pytest.mark.parametrize("p,n,widths", SMALL)
def test_small_circuits_every_plan_matches_oracle(p, n, widths):
    dag = W.small_dag(seed=len(widths) * 7 + n, p=p, n_inputs=50, widths=widths)
    n_plans = len(plans(dag.depth, p))
    dc = DeviceCircuit(dag, n, seed=3, runs=n_plans)
    try:
        for r, (name, plan) in enumerate(plans(dag.depth, p).items()):
            st, passed, sig = dc.run(plan)
            ev, em, ok, osig = oracle_run(dag, n, seed=3, run_index=r)
            gv, gm = dc.wires.host()
            assert_equal(gv, ev, f"{name}: wire values")
            assert_equal(gm, em, f"{name}: wire MACs")
            assert passed and ok and st.passed == 1, name
            assert_equal(sig, osig, f"{name}: sigma")
            assert st.n_mul == dag.n_mul
    finally:
        dc.close()


def test_benchmark_sized_circuit_matches_oracle():
    """The 2^20-gate, 32-layer, 3-party p61 circuit: the fused graph run, the
    per-layer run and the tagged graph run all equal the oracle on every
    wire."""
    dag = W.layered_dag(seed=2)
    n = 3
    dc = DeviceCircuit(dag, n, seed=2, runs=4)
    try:
        O.set_threads(8)
        ev, em, ok, osig = oracle_run(dag, n, seed=2, run_index=0)
        st, passed, sig = dc.run(S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1))
        gv, gm = dc.wires.host()
        assert_equal(gv, ev, "fused values")
        assert_equal(gm, em, "fused MACs")
        assert passed and ok
        assert_equal(sig, osig, "fused sigma")
        ev1, em1, ok1, osig1 = oracle_run(dag, n, seed=2, run_index=1)
        st, passed, sig = dc.run(S.plan(mode=S.SPDZ_SCHED_PER_LAYER, use_graph=0))
        gv, gm = dc.wires.host()
        assert_equal(gv, ev1, "per-layer values")
        assert_equal(gm, em1, "per-layer MACs")
        assert passed and ok1
        assert_equal(sig, osig1, "per-layer sigma")
        ev2, em2, ok2, osig2 = oracle_run(dag, n, seed=2, run_index=2)
        st, passed, sig = dc.run(S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=1, barrier_slack=24))
        gv, gm = dc.wires.host()
        assert_equal(gv, ev2, "tagged values")
        assert_equal(gm, em2, "tagged MACs")
        assert passed and ok2
        assert_equal(sig, osig2, "tagged sigma")
        # two tagged groups inside a fused plan (the second group's first
        # layer reads the first group's outputs from the party-major wires)
        ev3, em3, ok3, osig3 = oracle_run(dag, n, seed=2, run_index=3)
        st, passed, sig = dc.run(S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1, groups=[16, 32], group_tagged=[1, 1],
                                        barrier_slack=24))
        gv, gm = dc.wires.host()
        assert_equal(gv, ev3, "tagged groups values")
        assert_equal(gm, em3, "tagged groups MACs")
        assert passed and ok3
        assert_equal(sig, osig3, "tagged groups sigma")
    finally:
        dc.close()


@pytest.mark.parametrize("widths", [[80000, 2000, 300], [70000, 500, 40], [4000, 3000, 7]])
def test_tagged_first_layer_input_paths(widths):
    """The tagged kernel's first layer reads its input operands from the
    caller's wires while the inputs are copied into the tagged copy for the
    later layers: by the threads without a first-layer gate (4000 gates), or
    by every thread after its gate when the first layer is wider than the
    grid (80000) or leaves fewer than a quarter of the threads idle (70000).
    70,000 inputs, 2 parties, p61; every wire and sigma against the oracle."""
    p, n = O.P61, 2
    dag = W.small_dag(seed=sum(widths) % 97, p=p, n_inputs=70000, widths=widths)
    dc = DeviceCircuit(dag, n, seed=4, runs=1)
    try:
        st, passed, sig = dc.run(S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=0, barrier_slack=24))
        ev, em, ok, osig = oracle_run(dag, n, seed=4, run_index=0)
        gv, gm = dc.wires.host()
        assert_equal(gv, ev, "wire values")
        assert_equal(gm, em, "wire MACs")
        assert passed and ok and st.passed == 1
        assert_equal(sig, osig, "sigma")
    finally:
        dc.close()


def test_tagged_runs_cycle_over_many_replays():
    """Sixteen graph replays of the tagged plan (more than two cycles of the
    seven run tags, so the tagged wire copy is zeroed twice in between): every
    run equals the oracle, so no operand of an earlier run is ever taken for
    the current one."""
    dag = W.layered_dag(seed=13, total_gates=2**13, depth=10, wmin=32, wmax=2048, n_inputs=512)
    n = 3
    R = 16
    dc = DeviceCircuit(dag, n, seed=6, runs=R)
    try:
        plan = S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=1, barrier_slack=4)
        for r in range(R):
            # fresh inputs every run: a stale operand would show in the outputs
            S.spdz_deal_shared(dc.ctx, dc.seed + r, S.SPDZ_KIND_INPUT, INPUT_SUB, 0, dag.n_inputs,
                               dc.alpha_sh, None, dc.wires.buf())
            st, passed, sig = dc.run(plan)
            p = dag.p
            alpha, ash = O.deal_alpha(p, n, dc.seed)
            iv, im, _ = O.deal_shared(p, n, dc.seed + r, O.K_INPUT, INPUT_SUB, 0, dag.n_inputs, alpha)
            wv, wm = O.zeros(p, n, dag.n_wires), O.zeros(p, n, dag.n_wires)
            wv[:, :dag.n_inputs], wm[:, :dag.n_inputs] = iv, im
            tri = O.deal_triples(p, n, dc.seed, r * dag.n_mul, dag.n_mul, alpha)
            _, _, log = O.dag_eval(p, dag, wv, wm, tri, ash)
            ok, osig, _, _ = O.mac_check(p, [log], ash, 7, r)
            gv, gm = dc.wires.host()
            assert_equal(gv, wv, f"replay {r} values")
            assert_equal(gm, wm, f"replay {r} MACs")
            assert passed and ok
            assert_equal(sig, osig, f"replay {r} sigma")
    finally:
        dc.close()


def test_tagged_plan_rules():
    """The tagged mode is p61-only, has no layer groups and bounds its poll interval."""
    dag = W.small_dag(seed=2, p=O.P127, n_inputs=20, widths=[10, 10])
    dc = DeviceCircuit(dag, 2, seed=2, runs=1)
    try:
        with pytest.raises(S.SpdzError) as e:
            S.spdz_run_dag(dc.ctx, dc.h, S.plan(mode=S.SPDZ_SCHED_TAGGED), dc.wires.buf())
        assert e.value.code == S.SPDZ_ERR_ARG
    finally:
        dc.close()
    dag = W.small_dag(seed=2, p=O.P61, n_inputs=20, widths=[10, 10])
    dc = DeviceCircuit(dag, 2, seed=2, runs=1)
    try:
        for kw in ({"groups": [1, 2]}, {"poll_ns": 10**6}):
            with pytest.raises(S.SpdzError) as e:
                S.spdz_run_dag(dc.ctx, dc.h, S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=0, **kw), dc.wires.buf())
            assert e.value.code == S.SPDZ_ERR_ARG
    finally:
        dc.close()


def test_graph_replays_consume_fresh_triples():
    dag = W.layered_dag(seed=11, total_gates=2**14, depth=12, wmin=64, wmax=4096, n_inputs=1024)
    n = 3
    dc = DeviceCircuit(dag, n, seed=5, runs=3)
    try:
        plan = S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1)
        for r in range(3):
            st, passed, sig = dc.run(plan)
            ev, em, ok, osig = oracle_run(dag, n, seed=5, run_index=r)
            gv, gm = dc.wires.host()
            assert_equal(gv, ev, f"replay {r}")
            assert_equal(gm, em, f"replay {r} macs")
            assert_equal(sig, osig, f"replay {r} sigma")
        assert S.spdz_triples_left(dc.ctx) == 0
        with pytest.raises(S.SpdzError) as e:
            dc.run(plan)
        assert e.value.code == S.SPDZ_ERR_TRIPLES
    finally:
        dc.close()


def test_layer_times_recorded():
    dag = W.layered_dag(seed=4, total_gates=2**15, depth=16, wmin=256, wmax=8192, n_inputs=2048)
    dc = DeviceCircuit(dag, 3, seed=4, runs=3)
    try:
        for mode in (S.SPDZ_SCHED_PER_LAYER, S.SPDZ_SCHED_FUSED, S.SPDZ_SCHED_TAGGED):
            st, passed, _ = dc.run(S.plan(mode=mode, use_graph=0, record_layer_times=1))
            t = S.spdz_dag_layer_times(dc.h, dag.depth)
            assert passed and np.all(t > 0) and np.all(t < 1e5)
        counts = S.spdz_dag_layer_counts(dc.h, dag.depth)
        assert counts.sum() == dag.n_gates and counts[:, 0].sum() == dag.n_mul
    finally:
        dc.close()


def test_kernel_times_recorded():
    """spdz_dag_time_kernels: events around a run's circuit kernels, in a
    captured graph and without one, for the tagged and the fused plan; the
    kernel time lies inside the run's device time, and timing changes no
    result (a run after it, captured again without the events, equals the
    oracle)."""
    dag = W.layered_dag(seed=4, total_gates=2**15, depth=16, wmin=256, wmax=8192, n_inputs=2048)
    n = 3
    dc = DeviceCircuit(dag, n, seed=4, runs=5)
    try:
        with pytest.raises(S.SpdzError) as e:
            S.spdz_dag_kernel_ms(dc.h)
        assert e.value.code == S.SPDZ_ERR_STATE
        S.spdz_dag_time_kernels(dc.h, True)
        for plan in (S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=1), S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=0),
                     S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1), S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=0)):
            st, passed, _ = dc.run(plan)
            k = S.spdz_dag_kernel_ms(dc.h)
            assert passed and 0 < k <= st.device_ms, (k, st.device_ms)
        S.spdz_dag_time_kernels(dc.h, False)
        st, passed, sig = dc.run(S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=1))
        ev, em, ok, osig = oracle_run(dag, n, seed=4, run_index=4)
        gv, gm = dc.wires.host()
        assert passed and ok
        assert_equal(gv, ev, "run after kernel timing")
        assert_equal(gm, em, "run after kernel timing, macs")
        assert_equal(sig, osig, "run after kernel timing, sigma")
    finally:
        dc.close()


def test_barrier_timeout_is_a_status_not_a_hang():
    """Every barrier waits for one arrival that never comes; the bounded wait
    runs out, the run reports SPDZ_ERR_TIMEOUT, and the context stays usable."""
    dag = W.small_dag(seed=9, p=O.P61, n_inputs=64, widths=[200, 100, 50])
    dc = DeviceCircuit(dag, 3, seed=9, runs=2)
    try:
        plan = S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=0, spin_limit_us=2000, barrier_extra_arrivals=1)
        with pytest.raises(S.SpdzError) as e:
            S.spdz_run_dag(dc.ctx, dc.h, plan, dc.wires.buf())
        assert e.value.code == S.SPDZ_ERR_TIMEOUT
        dc.deal_inputs()
        st, passed, sig = dc.run(S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=0))
        ev, em, ok, osig = oracle_run(dag, 3, seed=9, run_index=1)
        assert passed and ok
        assert_equal(dc.wires.host()[0], ev, "after timeout")
    finally:
        dc.close()


def test_tagged_operand_wait_timeout_is_a_status_not_a_hang():
    """Gates after the first layer wait for a tag that is never written; the
    bounded operand wait runs out, the run reports SPDZ_ERR_TIMEOUT and does
    not pass, and the next tagged run on the context is exact."""
    dag = W.small_dag(seed=10, p=O.P61, n_inputs=64, widths=[200, 100, 50])
    dc = DeviceCircuit(dag, 3, seed=10, runs=2)
    try:
        plan = S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=0, spin_limit_us=2000, test_unwritten_tag=1)
        with pytest.raises(S.SpdzError) as e:
            S.spdz_run_dag(dc.ctx, dc.h, plan, dc.wires.buf())
        assert e.value.code == S.SPDZ_ERR_TIMEOUT
        # the barrier's extra-arrival hook means nothing in tagged mode: refused
        with pytest.raises(S.SpdzError) as e:
            S.spdz_run_dag(dc.ctx, dc.h, S.plan(mode=S.SPDZ_SCHED_TAGGED, barrier_extra_arrivals=1), dc.wires.buf())
        assert e.value.code == S.SPDZ_ERR_ARG
        dc.deal_inputs()
        st, passed, sig = dc.run(S.plan(mode=S.SPDZ_SCHED_TAGGED, use_graph=0))
        ev, em, ok, osig = oracle_run(dag, 3, seed=10, run_index=1)
        assert passed and ok
        assert_equal(dc.wires.host()[0], ev, "after timeout")
        assert_equal(dc.wires.host()[1], em, "after timeout (MACs)")
    finally:
        dc.close()


def test_tampered_input_share_fails_circuit_check():
    dag = W.small_dag(seed=1, p=O.P61, n_inputs=40, widths=[50, 50, 50])
    dc = DeviceCircuit(dag, 3, seed=1, runs=1)
    try:
        # party 1 shifts its share of the first operand of the first MUL gate
        g = int(np.flatnonzero(dag.ops == O.OP_MUL)[0])
        w = int(dag.in0[g])
        v = O.to_ints(dag.p, SH.to_host(dc.wires.val[1, w:w + 1]))[0]
        dc.wires.val[1, w] = int(np.array([(v + 1) % dag.p], dtype=np.uint64).view(np.int64)[0])
        st, passed, sig = dc.run(S.plan(mode=S.SPDZ_SCHED_FUSED))
        assert not passed and st.passed == 0
    finally:
        dc.close()


def test_invalid_circuit_rejected():
    ctx = ctx_for(2, O.P61)
    try:
        off = np.array([0, 2], dtype=np.int64)
        ops = np.array([O.OP_ADD, O.OP_MUL], dtype=np.uint8)
        in0 = np.array([0, 3], dtype=np.uint32)     # gate 1 reads gate 0's output, same layer
        in1 = np.array([1, 1], dtype=np.uint32)
        with pytest.raises(S.SpdzError) as e:
            S.spdz_dag_create(ctx, 3, off, ops, in0, in1, np.zeros(2, np.uint64))
        assert e.value.code == S.SPDZ_ERR_ARG
    finally:
        S.spdz_ctx_destroy(ctx)


def test_tagged_groups_refused_outside_p61_and_with_clusters():
    dag = W.small_dag(seed=4, p=O.P127, n_inputs=20, widths=[10, 10])
    dc = DeviceCircuit(dag, 2, seed=4, runs=1)
    try:
        with pytest.raises(S.SpdzError) as e:
            S.spdz_run_dag(dc.ctx, dc.h, S.plan(mode=S.SPDZ_SCHED_FUSED, groups=[2], group_tagged=[1]), dc.wires.buf())
        assert e.value.code == S.SPDZ_ERR_ARG
    finally:
        dc.close()
    dag = W.small_dag(seed=4, p=O.P61, n_inputs=20, widths=[10, 10])
    dc = DeviceCircuit(dag, 2, seed=4, runs=1)
    try:
        with pytest.raises(S.SpdzError) as e:
            S.spdz_run_dag(dc.ctx, dc.h, S.plan(mode=S.SPDZ_SCHED_FUSED, groups=[2], group_tagged=[1],
                                                group_cluster=[8]), dc.wires.buf())
        assert e.value.code == S.SPDZ_ERR_ARG
    finally:
        dc.close()


@pytest.mark.parametrize("p", [O.P61, O.P127])
def test_host_buffer_runs_match_oracle(p):
    """spdz_run_dag_host: three runs in a row whose input shares and triples
    come from page-locked host memory (the oracle's own dealt shares; the
    device pool is registered but never dealt, so only the host copies can
    fill it) and whose last-layer output shares are copied back: every copied
    share equals the oracle's run, and every run's check passes.  The calls
    are enqueued back to back, so a run's triple copy overlaps the run
    before it."""
    n, seed, runs = 3, 8, 3
    dag = W.small_dag(seed=8, p=p, n_inputs=300, widths=[500, 64, 1, 900, 33])
    field = SH.field_of(p)
    ctx = ctx_for(n, p)
    try:
        ash = SH.zeros(field, n)
        S.spdz_deal_alpha(ctx, seed, ash)
        wires = SH.alloc(field, n, dag.n_wires)
        pool = [SH.alloc(field, n, runs * dag.n_mul) for _ in range(3)]
        S.spdz_load_preproc(ctx, ash, *[t.buf() for t in pool], runs * dag.n_mul)
        S.spdz_set_check_seed(ctx, 7)
        h = S.spdz_dag_create(ctx, dag.n_inputs, dag.layer_offsets, dag.ops, dag.in0, dag.in1, dag.kconst)
        alpha, _ = O.deal_alpha(p, n, seed)
        iv, im, _ = O.deal_shared(p, n, seed, O.K_INPUT, INPUT_SUB, 0, dag.n_inputs, alpha)
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).pin_memory()  # noqa: E731
        h_in = [pin(iv), pin(im)]
        out_lo = dag.n_inputs + int(dag.layer_offsets[-2])
        cnt = dag.n_wires - out_lo
        keep, outs = [], []
        for r in range(runs):
            t = O.deal_triples(p, n, seed, r * dag.n_mul, dag.n_mul, alpha)
            h_tri = [pin(a) for a in (t.av, t.am, t.bv, t.bm, t.cv, t.cm)]
            ov, om = pin(O.zeros(p, n, cnt)), pin(O.zeros(p, n, cnt))
            keep.append(h_tri)
            outs.append((ov, om))
            S.spdz_run_dag_host(ctx, h, S.plan(mode=S.SPDZ_SCHED_FUSED, use_graph=1), wires.buf(), h_in[0], h_in[1],
                                h_tri, out_lo, cnt, ov, om)
        assert S.spdz_check_result(ctx)
        for r in range(runs):
            ev, em, ok, _ = oracle_run(dag, n, seed, run_index=r)
            assert ok
            gv = outs[r][0].numpy().view(np.uint64).reshape(ev[:, out_lo:].shape)
            gm = outs[r][1].numpy().view(np.uint64).reshape(em[:, out_lo:].shape)
            assert_equal(gv, ev[:, out_lo:], f"host run {r} output values")
            assert_equal(gm, em[:, out_lo:], f"host run {r} output MACs")
        assert S.spdz_triples_left(ctx) == 0
        S.spdz_dag_destroy(h)
    finally:
        S.spdz_ctx_destroy(ctx)
