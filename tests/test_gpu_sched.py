"""The scheduler on the GPU: per-layer timings recorded by the pipeline train
the cost model with the library's own kernels; the learned plan (dynamic
programming over predicted layer times) is judged against the autotuned and
default plans by measurement; every plan gives the oracle's shares."""
import numpy as np
import pytest
import torch

import oracle as O
import spdz_workloads as W

pytestmark = pytest.mark.gpu

from gpu_helpers import assert_equal, ctx_for  # noqa: E402
from test_gpu_dag import INPUT_SUB, oracle_run  # noqa: E402


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    global S, SH
    from paper_2512_11112_b300 import shares as SH  # noqa: F401
    from paper_2512_11112_b300 import spdz as S  # noqa: F401
    yield


class World:
    """One context with a triple pool shared by several circuits."""

    def __init__(self, p, n, seed, dags, runs_each):
        self.p, self.n, self.seed = p, n, seed
        self.field = SH.field_of(p)
        self.ctx = ctx_for(n, p)
        self.ash = SH.zeros(self.field, n)
        S.spdz_deal_alpha(self.ctx, seed, self.ash)
        T = sum(d.n_mul for d in dags) * runs_each
        self.tri = [SH.alloc(self.field, n, T) for _ in range(3)]
        S.spdz_deal_triples(self.ctx, seed, 0, T, self.ash, *[t.buf() for t in self.tri])
        S.spdz_load_preproc(self.ctx, self.ash, *[t.buf() for t in self.tri], T)
        S.spdz_set_check_seed(self.ctx, 7)
        self.items = []
        for d in dags:
            w = SH.alloc(self.field, n, d.n_wires)
            S.spdz_deal_shared(self.ctx, seed, S.SPDZ_KIND_INPUT, INPUT_SUB, 0, d.n_inputs, self.ash, None, w.buf())
            h = S.spdz_dag_create(self.ctx, d.n_inputs, d.layer_offsets, d.ops, d.in0, d.in1, d.kconst)
            self.items.append((d, h, w))

    def close(self):
        for _, h, _ in self.items:
            S.spdz_dag_destroy(h)
        S.spdz_ctx_destroy(self.ctx)


def test_learned_scheduler_matches_or_beats_autotuned_and_stays_exact():
    p, n = O.P61, 3
    cal = W.calibration_dags(p)
    narrow = W.small_dag(seed=5, p=p, n_inputs=256, widths=[64] * 24,
                         mix={"mul": 60, "add": 15, "sub": 15, "cmul": 10})
    held = W.layered_dag(seed=9, total_gates=2**16, depth=16, wmin=32, wmax=16384, n_inputs=2048)
    ncfg, _ = S.spdz_sched_num_configs()
    runs_record = ncfg * 3 + 8
    w = World(p, n, 4, cal + [narrow, held], runs_record + 40)
    try:
        for d, h, wires in w.items[:len(cal)]:
            S.spdz_sched_record(w.ctx, h, wires.buf(), 2)
        X, Y, switch_us = S.spdz_sched_samples(w.ctx)
        assert len(Y) == ncfg * sum(d.depth for d in cal)
        assert 0 <= switch_us < 50
        loss = S.spdz_sched_train(w.ctx, epochs=400, lr=2e-3, seed=3)
        assert loss < 0.05, loss        # mean squared error of ln(us): about 22% typical error

        # held-out circuit: predicted layer times against measured ones
        dh, hh, wh = w.items[-1]
        S.spdz_sched_record(w.ctx, hh, wh.buf(), 2)
        Xh, Yh, _ = S.spdz_sched_samples(w.ctx)
        meas = np.exp(Yh[-ncfg * dh.depth:]).reshape(ncfg, dh.depth)
        errs = []
        for c in range(ncfg):
            pred = S.spdz_sched_predict(w.ctx, hh, c, dh.depth)
            errs.append(np.median(np.abs(pred - meas[c]) / meas[c]))
        assert np.median(errs) < 0.35, errs

        # the held-out circuit (mixed widths, p61): the learned planner picks,
        # without running it, the plan that the autotuner finds by measuring
        # every configuration (the tagged form), so that plan is the learned one
        _, rep_h = S.spdz_sched_choose(w.ctx, hh, wh.buf(), 3)
        assert rep_h.learned_ms > 0 and rep_h.learned_ms <= 1.1 * rep_h.autotuned_ms, (rep_h.learned_ms,
                                                                                    rep_h.autotuned_ms)
        if rep_h.learned_is_autotuned:
            assert rep_h.chosen == 2
        # narrow circuit: the learned plan (cluster groups) against the
        # autotuned fallback and the default plan
        dn, hn, wn = w.items[len(cal)]
        plan, rep = S.spdz_sched_choose(w.ctx, hn, wn.buf(), 5)
        # (the measured gain over the default plan is 5-10 % from box to box,
        # about as wide as the run-to-run noise of these medians, so the check
        # is only that the learned plan is not slower than the default beyond
        # that noise; the gain itself is reported by the bench, not asserted)
        assert rep.learned_ms > 0 and rep.learned_ms <= 1.05 * rep.default_ms, (rep.learned_ms, rep.default_ms)
        # (the model's error is about 11 %, ln-space loss near 0.012: the
        # learned plan is held to 20 % of the autotuned plan)
        assert rep.learned_ms <= 1.2 * rep.autotuned_ms, (rep.learned_ms, rep.autotuned_ms)
        assert rep.chosen in (1, 2)
        assert abs(rep.predicted_ms - rep.learned_ms) < 0.5 * rep.learned_ms

        # a run with no explicit plan uses the chosen plan and equals the oracle
        for r in range(2):
            S.spdz_deal_shared(w.ctx, w.seed, S.SPDZ_KIND_INPUT, INPUT_SUB, 0, dn.n_inputs, w.ash, None, wn.buf())
            used_before = (w.tri[0].count - S.spdz_triples_left(w.ctx))
            st = S.spdz_run_dag(w.ctx, hn, None, wn.buf())
            assert st.passed == 1
        # oracle of the last run: the triples it consumed start at used_before
        alpha, oash = O.deal_alpha(p, n, w.seed)
        iv, im, _ = O.deal_shared(p, n, w.seed, O.K_INPUT, INPUT_SUB, 0, dn.n_inputs, alpha)
        wv, wm = O.zeros(p, n, dn.n_wires), O.zeros(p, n, dn.n_wires)
        wv[:, :dn.n_inputs], wm[:, :dn.n_inputs] = iv, im
        tri = O.deal_triples(p, n, w.seed, used_before, dn.n_mul, alpha)
        O.dag_eval(p, dn, wv, wm, tri, oash)
        gv, gm = wn.host()
        assert_equal(gv, wv, "learned-plan run values")
        assert_equal(gm, wm, "learned-plan run MACs")
    finally:
        w.close()
