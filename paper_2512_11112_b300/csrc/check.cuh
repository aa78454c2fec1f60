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
    // every input is loaded before anything is stored (stores through ds
    // would otherwise order each load behind the previous iteration's stores)
    unsigned long long w[NP + 1][3];
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc_words(ds->acc[k], w[k]);
    T alpha[NP], run[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        alpha[i] = load_alpha<F>(ds, i);
        if constexpr (F::WORDS == 1)
            run[i] = (T)ds->sig_run[i][0];
        else
            run[i] = T{ds->sig_run[i][0], ds->sig_run[i][1]};
    }
    const uint32_t pfail = ds->partial_fail, errs = ds->err_flags;
    const uint64_t epoch = ds->epoch, seed = ds->check_seed;
    const T A = acc_reduce_w<F>(w[0]);
    T tot = F::zero(), S[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        S[i] = acc_reduce_w<F>(w[1 + i]);
        const T sig = F::sub(S[i], F::mul(alpha[i], A));
        tot = F::add(tot, sig);
        run[i] = F::add(run[i], sig);
    }
    // stores
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        if constexpr (F::WORDS == 1) {
            ds->res_S[i][0] = S[i];
            ds->res_S[i][1] = 0;
        } else {
            ds->res_S[i][0] = S[i].lo;
            ds->res_S[i][1] = S[i].hi;
        }
    }
    if constexpr (F::WORDS == 1) {
        ds->res_A[0] = A;
        ds->res_A[1] = 0;
    } else {
        ds->res_A[0] = A.lo;
        ds->res_A[1] = A.hi;
    }
    const bool failed = pfail || !F::is_zero(tot);
    for (int k = 0; k < NP + 1; ++k)
        for (int q = 0; q < 4; ++q) ds->acc[k][q] = 0;
    if (final_check) {
        for (int i = 0; i < NP; ++i) {
            if constexpr (F::WORDS == 1) {
                ds->res_sigma[i][0] = run[i];
                ds->res_sigma[i][1] = 0;
            } else {
                ds->res_sigma[i][0] = run[i].lo;
                ds->res_sigma[i][1] = run[i].hi;
            }
            ds->sig_run[i][0] = ds->sig_run[i][1] = 0;
        }
        // a run whose device wait timed out is incomplete: it never passes
        ds->res_passed = (failed || (errs & ERR_TIMEOUT)) ? 0u : 1u;
        ds->res_epoch = (uint32_t)epoch;
        ds->partial_fail = 0;
        ds->epoch = epoch + 1;
        ds->key = stream_key(seed, stream_id(SPDZ_KIND_CHECK, 0, 0, epoch + 1));
    } else {
        for (int i = 0; i < NP; ++i) {
            if constexpr (F::WORDS == 1) {
                ds->sig_run[i][0] = run[i];
                ds->sig_run[i][1] = 0;
            } else {
                ds->sig_run[i][0] = run[i].lo;
                ds->sig_run[i][1] = run[i].hi;
            }
        }
        if (failed) ds->partial_fail = 1;
    }
}

}  // namespace spdz
