// check.cuh -- the batched MAC check step on one context's (or request's)
// device state.
#pragma once
#include "common.cuh"

namespace spdz {

// Batched MAC check over the accumulated random linear combination:
// sigma_i = S_i - alpha_i * A; a check passes iff sum_i sigma_i == 0.  A
// partial check (final == 0) adds its sigma to the epoch's running sigma and
// records a failure; the final check publishes the epoch's result and moves
// to the next epoch's coefficient key.  Runs on one thread.
template <class F, int NP>
__device__ void check_epoch(DevState *ds, int final_check) {
    using T = typename F::T;
    T A = acc_reduce<F>(ds->acc[0]);
    T tot = F::zero();
    for (int i = 0; i < NP; ++i) {
        T S = acc_reduce<F>(ds->acc[1 + i]);
        T sig = F::sub(S, F::mul(load_alpha<F>(ds, i), A));
        tot = F::add(tot, sig);
        T run;
        if constexpr (F::WORDS == 1) {
            run = F::add(ds->sig_run[i][0], sig);
            ds->sig_run[i][0] = run;
            ds->res_S[i][0] = S;
            ds->res_S[i][1] = 0;
        } else {
            run = F::add(T{ds->sig_run[i][0], ds->sig_run[i][1]}, sig);
            ds->sig_run[i][0] = run.lo;
            ds->sig_run[i][1] = run.hi;
            ds->res_S[i][0] = S.lo;
            ds->res_S[i][1] = S.hi;
        }
    }
    if constexpr (F::WORDS == 1) {
        ds->res_A[0] = A;
        ds->res_A[1] = 0;
    } else {
        ds->res_A[0] = A.lo;
        ds->res_A[1] = A.hi;
    }
    if (!F::is_zero(tot)) ds->partial_fail = 1;
    for (int k = 0; k < NP + 1; ++k)
        for (int w = 0; w < 4; ++w) ds->acc[k][w] = 0;
    if (final_check) {
        for (int i = 0; i < NP; ++i) {
            ds->res_sigma[i][0] = ds->sig_run[i][0];
            ds->res_sigma[i][1] = ds->sig_run[i][1];
            ds->sig_run[i][0] = ds->sig_run[i][1] = 0;
        }
        // a run whose device wait timed out is incomplete: it never passes
        ds->res_passed = (ds->partial_fail || (ds->err_flags & ERR_TIMEOUT)) ? 0u : 1u;
        ds->res_epoch = (uint32_t)ds->epoch;
        ds->partial_fail = 0;
        ds->epoch += 1;
        ds->key = stream_key(ds->check_seed, stream_id(SPDZ_KIND_CHECK, 0, 0, ds->epoch));
    }
}

}  // namespace spdz
