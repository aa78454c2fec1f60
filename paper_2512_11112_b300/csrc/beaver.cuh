// beaver.cuh -- the arithmetic of one Beaver product and of the linear gates,
// on shares already in registers (Sec. II-A.3 of the paper).
#pragma once
#include <type_traits>
#include "common.cuh"

namespace spdz {

// Inputs per party i: x_i, gamma(x)_i, y_i, gamma(y)_i and the triple shares
// (a, b, c) with their MAC shares (read through an accessor, so they can stay
// in shared memory until used).  Opens eps = sum(x_i - a_i) and
// delta = sum(y_i - b_i) and combines
//   z_i = c_i + eps*b_i + delta*a_i + [i == 0] eps*delta
//   gamma(z)_i = gamma(c)_i + eps*gamma(b)_i + delta*gamma(a)_i + alpha_i*eps*delta.
// The opened eps (index j) and delta (index j+1) of the check's log add
// r_j*eps + r_{j+1}*delta to acc[0] and r_j*(gamma(x)_i - gamma(a)_i) +
// r_{j+1}*(gamma(y)_i - gamma(b)_i) to acc[1+i].
// p61 form with the check coefficients given (re for eps, rd for delta):
// every output is one exact sum of at most three 122-bit products and one or
// two canonical terms (below 2^124), reduced once.
template <int NP, class TRI>
__device__ __forceinline__ void beaver_math61(const uint64_t (&x)[NP], const uint64_t (&gx)[NP], const uint64_t (&y)[NP],
                                              const uint64_t (&gy)[NP], const TRI &tri, const uint64_t (&alpha)[NP],
                                              uint64_t re, uint64_t rd, uint64_t (&acc)[NP + 1], uint64_t (&z)[NP],
                                              uint64_t (&gz)[NP]) {
    using F = F61;
    uint64_t eps = 0, dlt = 0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        eps = F::add(eps, F::sub(x[i], tri(0, i)));
        dlt = F::add(dlt, F::sub(y[i], tri(2, i)));
    }
    const uint64_t de = F::mul(eps, dlt);
    W61 a0;
    a0.add(acc[0]);
    a0.mac(re, eps);
    a0.mac(rd, dlt);
    acc[0] = a0.reduce();
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        W61 v, m, c;
        v.add(tri(4, i));
        if (i == 0) v.add(de);
        v.mac(eps, tri(2, i));
        v.mac(dlt, tri(0, i));
        z[i] = v.reduce();
        m.add(tri(5, i));
        m.mac(eps, tri(3, i));
        m.mac(dlt, tri(1, i));
        m.mac(alpha[i], de);
        gz[i] = m.reduce();
        c.add(acc[1 + i]);
        c.mac(re, F::sub(gx[i], tri(1, i)));
        c.mac(rd, F::sub(gy[i], tri(3, i)));
        acc[1 + i] = c.reduce();
    }
}

template <class F, int NP, class TRI>
__device__ __forceinline__ void beaver_math_src(
    const typename F::T (&x)[NP], const typename F::T (&gx)[NP], const typename F::T (&y)[NP],
    const typename F::T (&gy)[NP], const TRI &tri, const typename F::T (&alpha)[NP], uint64_t key, uint64_t j,
    typename F::T (&acc)[NP + 1], typename F::T (&z)[NP], typename F::T (&gz)[NP]) {
    // tri(k, i): triple share k of party i, k = 0..5 for a, gamma(a), b,
    // gamma(b), c, gamma(c)
    using T = typename F::T;
    if constexpr (std::is_same_v<F, F61>) {
        beaver_math61<NP>(x, gx, y, gy, tri, alpha, Draw<F>::at(key, j), Draw<F>::at(key, j + 1), acc, z, gz);
        return;
    }
    T eps = F::zero(), dlt = F::zero();
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        eps = F::add(eps, F::sub(x[i], tri(0, i)));
        dlt = F::add(dlt, F::sub(y[i], tri(2, i)));
    }
    const T de = F::mul(eps, dlt);
    const T re = Draw<F>::at(key, j), rd = Draw<F>::at(key, j + 1);
    // each output one sum of products, reduced once where the field allows
    acc[0] = Fma<F>::f2(acc[0], re, eps, rd, dlt);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        z[i] = Fma<F>::f2(i == 0 ? F::add(tri(4, i), de) : tri(4, i), eps, tri(2, i), dlt, tri(0, i));
        gz[i] = Fma<F>::f3(tri(5, i), eps, tri(3, i), dlt, tri(1, i), alpha[i], de);
        acc[1 + i] = Fma<F>::f2(acc[1 + i], re, F::sub(gx[i], tri(1, i)), rd, F::sub(gy[i], tri(3, i)));
    }
}

template <class F, int NP>
__device__ __forceinline__ void beaver_math(
    const typename F::T (&x)[NP], const typename F::T (&gx)[NP], const typename F::T (&y)[NP],
    const typename F::T (&gy)[NP], const typename F::T (&a)[NP], const typename F::T (&ga)[NP],
    const typename F::T (&b)[NP], const typename F::T (&gb)[NP], const typename F::T (&c)[NP],
    const typename F::T (&gc)[NP], const typename F::T (&alpha)[NP], uint64_t key, uint64_t j,
    typename F::T (&acc)[NP + 1], typename F::T (&z)[NP], typename F::T (&gz)[NP]) {
    auto tri = [&](int k, int i) -> typename F::T {
        return k == 0 ? a[i] : k == 1 ? ga[i] : k == 2 ? b[i] : k == 3 ? gb[i] : k == 4 ? c[i] : gc[i];
    };
    beaver_math_src<F, NP>(x, gx, y, gy, tri, alpha, key, j, acc, z, gz);
}

// Linear gate on one party's shares.  kal = alpha_i * k (used by CADD only).
template <class F>
__device__ __forceinline__ void linear_math(int op, int party, typename F::T x, typename F::T gx,
                                            typename F::T y, typename F::T gy, typename F::T k,
                                            typename F::T kal, typename F::T &z, typename F::T &gz) {
    switch (op) {
        case SPDZ_OP_ADD: z = F::add(x, y); gz = F::add(gx, gy); break;
        case SPDZ_OP_SUB: z = F::sub(x, y); gz = F::sub(gx, gy); break;
        case SPDZ_OP_CMUL: z = F::mul(k, x); gz = F::mul(k, gx); break;
        default: z = party == 0 ? F::add(x, k) : x; gz = F::add(gx, kal); break;
    }
}

}  // namespace spdz
