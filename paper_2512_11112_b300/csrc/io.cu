// io.cu -- the steps on either side of the online core: secret-sharing a
// party's private input with a dealer mask, and the MAC-checked reveal of
// outputs (Sec. I: parties share their inputs and combine shares of f only
// to reveal the output; Sec. II-A.2: a revealed value is accepted after the
// MAC check; Sec. IV: all inputs are secret-shared before the computation).
//
// Input: the owner of x holds a dealer mask r in the clear and the parties
// hold [r] with MACs.  The owner publishes eps = x - r, and [x] = [r] + eps is
// the public-constant addition: party 0 adds eps to its value share, every
// party adds alpha_i * eps to its MAC share.  Reveal: the shares are opened
// (logged for the check), the check runs over the epoch, and the values are
// released only if it passes.
#include <type_traits>

#include "dealer.cuh"
#include "vec.cuh"

namespace spdz {

int launch_check(spdz_ctx *ctx, int final_check);

template <class F> struct InArgs {
    using T = typename F::T;
    const T *x, *r, *mv, *mm;
    int64_t ms;
    T *ov, *om;
    int64_t os;
    int64_t N;
    T *eps;       // optional: eps = x - r, published by the owner
};

// V consecutive elements: eps = x - r; party 0's value share gains eps,
// every party's MAC share gains alpha_i * eps.
template <class F, int NP, int V>
__device__ __forceinline__ void input_elems(const InArgs<F> &a, int64_t j, const typename F::T (&alpha)[NP]) {
    using T = typename F::T;
    T x[V], r[V], e[V];
    vld<F, V, true>(a.x + j, x);
    vld<F, V, true>(a.r + j, r);
#pragma unroll
    for (int q = 0; q < V; ++q) e[q] = F::sub(x[q], r[q]);
    if (a.eps) vst<F, V>(a.eps + j, e);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        T v[V], g[V];
        vld<F, V, true>(a.mv + i * a.ms + j, v);
        vld<F, V, true>(a.mm + i * a.ms + j, g);
#pragma unroll
        for (int q = 0; q < V; ++q) {
            if (i == 0) v[q] = F::add(v[q], e[q]);
            g[q] = F::add(g[q], F::mul(alpha[i], e[q]));
        }
        vst<F, V>(a.ov + i * a.os + j, v);
        vst<F, V>(a.om + i * a.os + j, g);
    }
}

// V elements per thread (16-byte accesses when every row and vector is
// 16-byte aligned), the N % V tail one element per thread.
template <class F, int NP, int V>
__global__ void __launch_bounds__(256) k_input(InArgs<F> a, const DevState *ds) {
    using T = typename F::T;
    T alpha[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(ds, i);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t ng = a.N / V;
    for (int64_t g = tid; g < ng; g += stride) input_elems<F, NP, V>(a, g * V, alpha);
    for (int64_t j = ng * V + tid; j < a.N; j += stride) input_elems<F, NP, 1>(a, j, alpha);
}

template <class F, int NP>
static void launch_input(spdz_ctx *ctx, const void *x, const void *r, const spdz_buf *m, const spdz_buf *o, int64_t N,
                         void *eps) {
    using T = typename F::T;
    InArgs<F> a{(const T *)x, (const T *)r, (const T *)m->val, (const T *)m->mac, m->stride,
                (T *)o->val, (T *)o->mac, o->stride, N, (T *)eps};
    const size_t eb = sizeof(T);
    auto al = [](const void *q) { return ((uintptr_t)q & 15) == 0; };
    constexpr int VV = std::is_same_v<F, F61> ? 2 : std::is_same_v<F, F32> ? 4 : 1;
    const bool vec = VV > 1 && buf_vec_ok(m, eb) && buf_vec_ok(o, eb) && al(x) && al(r) && (!eps || al(eps));
    if (vec) {
        auto kern = k_input<F, NP, VV>;
        kern<<<grid_for(ctx, (const void *)kern, 256, 0, (N + VV - 1) / VV), 256, 0, ctx->stream>>>(a, ctx->ds);
    } else {
        auto kern = k_input<F, NP, 1>;
        kern<<<grid_for(ctx, (const void *)kern, 256, 0, N), 256, 0, ctx->stream>>>(a, ctx->ds);
    }
}

}  // namespace spdz

using namespace spdz;

extern "C" {

int spdz_deal_input_masks(spdz_ctx *ctx, uint64_t seed, int32_t owner, uint64_t j0, int64_t count,
                          const void *alpha_shares_dev, const spdz_buf *masks, void *r_clear_dev) {
    if (!ctx) return SPDZ_ERR_ARG;
    if (!alpha_shares_dev || !r_clear_dev || count < 0 || owner < 0 || owner >= ctx->n)
        return set_err(ctx, SPDZ_ERR_ARG, "deal_input_masks: bad argument");
    if (count == 0) return SPDZ_OK;
    int rc;
    if ((rc = validate_buf(ctx, masks, count, "deal_input_masks.masks"))) return rc;
    const size_t eb = elem_bytes(ctx->field);
    if ((uintptr_t)r_clear_dev % eb || (uintptr_t)alpha_shares_dev % eb)
        return set_err(ctx, SPDZ_ERR_ALIGN, "deal_input_masks: misaligned pointer");
    SPDZ_FIELD_SWITCH(ctx->field, SPDZ_NP_SWITCH(ctx->n, {
        using T = typename F::T;
        auto keys = make_keys<NP>(seed, SPDZ_KIND_INPUT_MASK, (uint64_t)owner);
        auto kern = k_deal_shared<F, NP>;
        kern<<<grid_for(ctx, (const void *)kern, 256, 0, count), 256, 0, ctx->stream>>>(
            keys, j0, count, (const T *)alpha_shares_dev, nullptr, (T *)masks->val, (T *)masks->mac, masks->stride,
            (T *)r_clear_dev);
    }));
    return check_launch(ctx, "deal_input_masks");
}

int spdz_input(spdz_ctx *ctx, const void *x_dev, const void *r_clear_dev, const spdz_buf *masks, const spdz_buf *out,
               int64_t N, void *eps_out_dev) {
    if (!ctx) return SPDZ_ERR_ARG;
    if (!x_dev || !r_clear_dev || N < 0) return set_err(ctx, SPDZ_ERR_ARG, "input: bad argument");
    if (!ctx->alpha_loaded) return set_err(ctx, SPDZ_ERR_STATE, "input: preprocessing not loaded");
    if (N == 0) return SPDZ_OK;
    int rc;
    if ((rc = validate_buf(ctx, masks, N, "input.masks")) || (rc = validate_buf(ctx, out, N, "input.out"))) return rc;
    const size_t eb = elem_bytes(ctx->field);
    if ((uintptr_t)x_dev % eb || (uintptr_t)r_clear_dev % eb || (eps_out_dev && (uintptr_t)eps_out_dev % eb))
        return set_err(ctx, SPDZ_ERR_ALIGN, "input: misaligned pointer");
    SPDZ_FIELD_SWITCH(ctx->field, SPDZ_NP_SWITCH(ctx->n, (launch_input<F, NP>(ctx, x_dev, r_clear_dev, masks, out, N, eps_out_dev))));
    return check_launch(ctx, "input");
}

int spdz_reveal(spdz_ctx *ctx, const spdz_buf *x, void *out_dev, int64_t N, int *passed, void *sigma_host) {
    if (!ctx) return SPDZ_ERR_ARG;
    if (!passed) return set_err(ctx, SPDZ_ERR_ARG, "reveal: null verdict");
    *passed = 0;
    int rc = spdz_open(ctx, x, out_dev, N);
    if (rc) return rc;
    rc = spdz_mac_check(ctx, passed, sigma_host);
    if (rc == SPDZ_ERR_MAC || !*passed) {
        // a failed check releases nothing
        if (N > 0) cudaMemsetAsync(out_dev, 0, (size_t)N * elem_bytes(ctx->field), ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        return set_err(ctx, SPDZ_ERR_MAC, "reveal: MAC check failed, outputs withheld");
    }
    return rc;
}

}  // extern "C"
