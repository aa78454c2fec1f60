// dealer.cuh -- device dealer ("fake preprocessing"): alpha shares, shared
// arrays and Beaver triples generated from the counter PRG specification.
#pragma once
#include "common.cuh"

namespace spdz {

// ---------------------------------------------------------------- dealer

template <class F>
__global__ void k_deal_alpha(uint64_t seed, int n, typename F::T *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    using T = typename F::T;
    T alpha = Draw<F>::at(stream_key(seed, stream_id(SPDZ_KIND_ALPHA, ROLE_SECRET, 0, 0)), 0);
    T sum = F::zero();
    for (int i = 0; i < n - 1; ++i) {
        T s = Draw<F>::at(stream_key(seed, stream_id(SPDZ_KIND_ALPHA, ROLE_VAL_SHARE, i, 0)), 0);
        F::st(out + i, s);
        sum = F::add(sum, s);
    }
    F::st(out + n - 1, F::sub(alpha, sum));
}

template <int NP> struct ShareKeys {
    uint64_t secret;
    uint64_t v[NP];
    uint64_t m[NP];
};

template <int NP>
inline ShareKeys<NP> make_keys(uint64_t seed, uint64_t kind, uint64_t sub) {
    ShareKeys<NP> k{};
    k.secret = stream_key(seed, stream_id(kind, ROLE_SECRET, 0, sub));
    for (int i = 0; i < NP - 1; ++i) {
        k.v[i] = stream_key(seed, stream_id(kind, ROLE_VAL_SHARE, i, sub));
        k.m[i] = stream_key(seed, stream_id(kind, ROLE_MAC_SHARE, i, sub));
    }
    return k;
}

template <class F, int NP>
__device__ __forceinline__ void share_store(const ShareKeys<NP> &k, typename F::T alpha, uint64_t gj,
                                            typename F::T v, typename F::T *val, typename F::T *mac,
                                            int64_t stride, int64_t j) {
    using T = typename F::T;
    T m = F::mul(alpha, v);
    T sv = F::zero(), sm = F::zero();
#pragma unroll
    for (int i = 0; i < NP - 1; ++i) {
        T vi = Draw<F>::at(k.v[i], gj), mi = Draw<F>::at(k.m[i], gj);
        F::st(val + i * stride + j, vi);
        F::st(mac + i * stride + j, mi);
        sv = F::add(sv, vi);
        sm = F::add(sm, mi);
    }
    F::st(val + (NP - 1) * stride + j, F::sub(v, sv));
    F::st(mac + (NP - 1) * stride + j, F::sub(m, sm));
}

template <class F, int NP>
__device__ __forceinline__ typename F::T sum_alpha(const typename F::T *alpha_sh) {
    typename F::T a = F::zero();
#pragma unroll
    for (int i = 0; i < NP; ++i) a = F::add(a, F::ld(alpha_sh + i));
    return a;
}

template <class F, int NP>
__global__ void k_deal_shared(ShareKeys<NP> keys, uint64_t j0, int64_t count,
                              const typename F::T *alpha_sh, const typename F::T *secret_in,
                              typename F::T *val, typename F::T *mac, int64_t stride,
                              typename F::T *secret_out) {
    using T = typename F::T;
    T alpha = sum_alpha<F, NP>(alpha_sh);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        uint64_t gj = j0 + (uint64_t)j;
        T v = secret_in ? F::ld(secret_in + j) : Draw<F>::at(keys.secret, gj);
        if (secret_out) F::st(secret_out + j, v);
        share_store<F, NP>(keys, alpha, gj, v, val, mac, stride, j);
    }
}

template <class F, int NP>
__global__ void k_deal_triples(ShareKeys<NP> ka, ShareKeys<NP> kb, ShareKeys<NP> kc, uint64_t j0,
                               int64_t count, const typename F::T *alpha_sh,
                               typename F::T *av, typename F::T *am, int64_t as,
                               typename F::T *bv, typename F::T *bm, int64_t bs,
                               typename F::T *cv, typename F::T *cm, int64_t cs) {
    using T = typename F::T;
    T alpha = sum_alpha<F, NP>(alpha_sh);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        uint64_t gj = j0 + (uint64_t)j;
        T a = Draw<F>::at(ka.secret, gj), b = Draw<F>::at(kb.secret, gj);
        share_store<F, NP>(ka, alpha, gj, a, av, am, as, j);
        share_store<F, NP>(kb, alpha, gj, b, bv, bm, bs, j);
        share_store<F, NP>(kc, alpha, gj, F::mul(a, b), cv, cm, cs, j);
    }
}


}  // namespace spdz
