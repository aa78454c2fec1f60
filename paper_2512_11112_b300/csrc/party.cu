// party.cu -- the online phase for one party whose shares live on its own
// GPU (a deployment with one process and one GPU per party; the paper runs
// its parties as separate processes, Sec. IV-A, and names one GPU per party
// as future work, Sec. V-B).  A Beaver product then splits at the open:
//   mask:    eps_i = x_i - a_i, delta_i = y_i - b_i          (local)
//   open:    every party's eps_i, delta_i rows are exchanged (an all-gather,
//            outside this file) and summed: eps = sum_i eps_i      (local)
//   combine: z_i = c_i + eps b_i + delta a_i + [i == 0] eps delta,
//            gamma(z)_i = gamma(c)_i + eps gamma(b)_i + delta gamma(a)_i
//                         + alpha_i eps delta                        (local)
// and the batched MAC check splits the same way: every party accumulates
// A = sum_j r_j v_j over the public opened values and its own
// S_i = sum_j r_j gamma_i(v_j), publishes sigma_i = S_i - alpha_i A, and the
// check passes iff the published sigmas sum to zero.
#include <algorithm>

#include "common.cuh"
#include "prg.cuh"

struct PartyState {
    unsigned long long acc[2][4];   // A, S_i: exact 192-bit sums
    uint64_t alpha[2];
    uint64_t sigma[2];              // last sigma_i
};

struct spdz_party {
    int party = 0, n = 0, field = 0;
    cudaStream_t stream = nullptr;
    PartyState *d = nullptr;
    PartyState *h = nullptr;        // pinned
    bool alpha_loaded = false;
    uint64_t seed = 0, epoch = 0, key = 0;
    int64_t opened = 0;
    int sm_count = 0;
};

namespace spdz {

template <class F> __device__ __forceinline__ typename F::T party_alpha(const PartyState *s) {
    if constexpr (F::WORDS == 1) return (typename F::T)s->alpha[0];
    else return typename F::T{s->alpha[0], s->alpha[1]};
}

template <class F>
__global__ void k_party_alpha(PartyState *s, const typename F::T *alpha) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const typename F::T a = F::ld(alpha);
    if constexpr (F::WORDS == 1) {
        s->alpha[0] = a;
        s->alpha[1] = 0;
    } else {
        s->alpha[0] = a.lo;
        s->alpha[1] = a.hi;
    }
    for (int k = 0; k < 2; ++k)
        for (int w = 0; w < 4; ++w) s->acc[k][w] = 0;
}

template <class F>
__global__ void __launch_bounds__(256) k_party_mask(const typename F::T *x, const typename F::T *y,
                                                    const typename F::T *a, const typename F::T *b,
                                                    typename F::T *eps, typename F::T *dlt, int64_t N) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        F::st(eps + j, F::sub(F::ld(x + j), F::ld(a + j)));
        F::st(dlt + j, F::sub(F::ld(y + j), F::ld(b + j)));
    }
}

// out[j] = sum over the n gathered rows (row k at rows + k * N).
template <class F>
__global__ void __launch_bounds__(256) k_party_open(const typename F::T *rows, int n, int64_t N, typename F::T *out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        typename F::T s = F::zero();
        for (int k = 0; k < n; ++k) s = F::add(s, F::ld(rows + (int64_t)k * N + j));
        F::st(out + j, s);
    }
}

template <class F> struct PartyArgs {
    using T = typename F::T;
    const T *eps, *dlt;                  // public opened values
    const T *xm, *ym;                    // this party's MAC shares of x, y
    const T *av, *am, *bv, *bm, *cv, *cm;
    T *zv, *zm;
    int64_t N;
    uint64_t key, base;                  // check coefficients: r at base + 2j (eps), base + 2j + 1 (delta)
    int first;                           // party 0 adds eps delta to its value share
    PartyState *s;
};

template <class F>
__global__ void __launch_bounds__(256) k_party_combine(PartyArgs<F> a) {
    using T = typename F::T;
    const T alpha = party_alpha<F>(a.s);
    T acc[2] = {F::zero(), F::zero()};
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.N; j += (int64_t)gridDim.x * blockDim.x) {
        const T eps = F::ld(a.eps + j), dlt = F::ld(a.dlt + j);
        const T de = F::mul(eps, dlt);
        const T av = F::ld(a.av + j), bv = F::ld(a.bv + j), am = F::ld(a.am + j), bm = F::ld(a.bm + j);
        const T c = F::ld(a.cv + j);
        F::st(a.zv + j, Fma<F>::f2(a.first ? F::add(c, de) : c, eps, bv, dlt, av));
        F::st(a.zm + j, Fma<F>::f3(F::ld(a.cm + j), eps, bm, dlt, am, alpha, de));
        const T re = Draw<F>::at(a.key, a.base + 2 * (uint64_t)j), rd = Draw<F>::at(a.key, a.base + 2 * (uint64_t)j + 1);
        acc[0] = Fma<F>::f2(acc[0], re, eps, rd, dlt);
        acc[1] = Fma<F>::f2(acc[1], re, F::sub(F::ld(a.xm + j), am), rd, F::sub(F::ld(a.ym + j), bm));
    }
    block_accumulate<F, 2>(acc, a.s->acc);
}

// sigma_i = S_i - alpha_i A; the sums restart for the next epoch.
template <class F>
__global__ void k_party_sigma(PartyState *s) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    using T = typename F::T;
    const T A = acc_reduce<F>(s->acc[0]), S = acc_reduce<F>(s->acc[1]);
    const T sig = F::sub(S, F::mul(party_alpha<F>(s), A));
    if constexpr (F::WORDS == 1) {
        s->sigma[0] = sig;
        s->sigma[1] = 0;
    } else {
        s->sigma[0] = sig.lo;
        s->sigma[1] = sig.hi;
    }
    for (int k = 0; k < 2; ++k)
        for (int w = 0; w < 4; ++w) s->acc[k][w] = 0;
}

static int party_grid(const spdz_party *p, int64_t N) {
    const int64_t need = (N + 255) / 256, cap = (int64_t)8 * p->sm_count;
    return (int)std::max<int64_t>(1, std::min(need, cap));
}

static bool aligned(const void *q, size_t eb) { return q && (uintptr_t)q % eb == 0; }

}  // namespace spdz

using namespace spdz;

extern "C" {

int spdz_party_create(spdz_party **out, int party, int n_parties, int field, void *stream) {
    if (!out || n_parties < 2 || n_parties > SPDZ_MAX_PARTIES || party < 0 || party >= n_parties ||
        (field != SPDZ_F61 && field != SPDZ_F127 && field != SPDZ_F32))
        return SPDZ_ERR_ARG;
    spdz_party *p = new spdz_party();
    p->party = party;
    p->n = n_parties;
    p->field = field;
    p->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (cudaMalloc(&p->d, sizeof(PartyState)) != cudaSuccess || cudaMallocHost(&p->h, sizeof(PartyState)) != cudaSuccess) {
        spdz_party_destroy(p);
        return SPDZ_ERR_OOM;
    }
    if (cudaMemsetAsync(p->d, 0, sizeof(PartyState), p->stream) != cudaSuccess) {
        spdz_party_destroy(p);
        return SPDZ_ERR_CUDA;
    }
    *out = p;
    return SPDZ_OK;
}

int spdz_party_destroy(spdz_party *p) {
    if (!p) return SPDZ_OK;
    if (p->stream) cudaStreamSynchronize(p->stream);
    else cudaDeviceSynchronize();
    if (p->d) cudaFree(p->d);
    if (p->h) cudaFreeHost(p->h);
    delete p;
    return SPDZ_OK;
}

int spdz_party_load_alpha(spdz_party *p, const void *alpha_share_dev) {
    if (!p || !alpha_share_dev) return SPDZ_ERR_ARG;
    if (!aligned(alpha_share_dev, elem_bytes(p->field))) return SPDZ_ERR_ALIGN;
    SPDZ_FIELD_SWITCH(p->field, (k_party_alpha<F><<<1, 32, 0, p->stream>>>(p->d, (const typename F::T *)alpha_share_dev)));
    if (cudaGetLastError() != cudaSuccess) return SPDZ_ERR_CUDA;
    p->alpha_loaded = true;
    p->opened = 0;
    return SPDZ_OK;
}

int spdz_party_set_check_seed(spdz_party *p, uint64_t seed) {
    if (!p) return SPDZ_ERR_ARG;
    if (p->opened != 0) return SPDZ_ERR_STATE;
    p->seed = seed;
    p->epoch = 0;
    p->key = stream_key(seed, stream_id(SPDZ_KIND_CHECK, 0, 0, 0));
    return SPDZ_OK;
}

int spdz_party_mask(spdz_party *p, const spdz_buf *x, const spdz_buf *y, const spdz_buf *a, const spdz_buf *b,
                    void *eps_dev, void *dlt_dev, int64_t N) {
    if (!p || N < 0 || !x || !y || !a || !b) return SPDZ_ERR_ARG;
    if (N == 0) return SPDZ_OK;
    const size_t eb = elem_bytes(p->field);
    if (!aligned(x->val, eb) || !aligned(y->val, eb) || !aligned(a->val, eb) || !aligned(b->val, eb) ||
        !aligned(eps_dev, eb) || !aligned(dlt_dev, eb))
        return SPDZ_ERR_ALIGN;
    SPDZ_FIELD_SWITCH(p->field, {
        using T = typename F::T;
        k_party_mask<F><<<party_grid(p, N), 256, 0, p->stream>>>((const T *)x->val, (const T *)y->val, (const T *)a->val,
                                                                 (const T *)b->val, (T *)eps_dev, (T *)dlt_dev, N);
    });
    return cudaGetLastError() == cudaSuccess ? SPDZ_OK : SPDZ_ERR_CUDA;
}

int spdz_party_open_sum(spdz_party *p, const void *rows_dev, int64_t N, void *out_dev) {
    if (!p || N < 0) return SPDZ_ERR_ARG;
    if (N == 0) return SPDZ_OK;
    const size_t eb = elem_bytes(p->field);
    if (!aligned(rows_dev, eb) || !aligned(out_dev, eb)) return SPDZ_ERR_ALIGN;
    SPDZ_FIELD_SWITCH(p->field, {
        using T = typename F::T;
        k_party_open<F><<<party_grid(p, N), 256, 0, p->stream>>>((const T *)rows_dev, p->n, N, (T *)out_dev);
    });
    return cudaGetLastError() == cudaSuccess ? SPDZ_OK : SPDZ_ERR_CUDA;
}

int spdz_party_combine(spdz_party *p, const void *eps_dev, const void *dlt_dev, const spdz_buf *x, const spdz_buf *y,
                       const spdz_buf *a, const spdz_buf *b, const spdz_buf *c, const spdz_buf *z, int64_t N) {
    if (!p || N < 0 || !x || !y || !a || !b || !c || !z) return SPDZ_ERR_ARG;
    if (!p->alpha_loaded) return SPDZ_ERR_STATE;
    if (N == 0) return SPDZ_OK;
    const size_t eb = elem_bytes(p->field);
    const spdz_buf *bufs[6] = {x, y, a, b, c, z};
    for (const spdz_buf *q : bufs)
        if (!aligned(q->val, eb) || !aligned(q->mac, eb)) return SPDZ_ERR_ALIGN;
    if (!aligned(eps_dev, eb) || !aligned(dlt_dev, eb)) return SPDZ_ERR_ALIGN;
    SPDZ_FIELD_SWITCH(p->field, {
        using T = typename F::T;
        PartyArgs<F> g{};
        g.eps = (const T *)eps_dev;
        g.dlt = (const T *)dlt_dev;
        g.xm = (const T *)x->mac;
        g.ym = (const T *)y->mac;
        g.av = (const T *)a->val; g.am = (const T *)a->mac;
        g.bv = (const T *)b->val; g.bm = (const T *)b->mac;
        g.cv = (const T *)c->val; g.cm = (const T *)c->mac;
        g.zv = (T *)z->val; g.zm = (T *)z->mac;
        g.N = N;
        g.key = p->key;
        g.base = (uint64_t)p->opened;
        g.first = p->party == 0;
        g.s = p->d;
        k_party_combine<F><<<party_grid(p, N), 256, 0, p->stream>>>(g);
    });
    if (cudaGetLastError() != cudaSuccess) return SPDZ_ERR_CUDA;
    p->opened += 2 * N;
    return SPDZ_OK;
}

int spdz_party_sigma(spdz_party *p, void *sigma_host, int64_t *opened_out) {
    if (!p || !sigma_host) return SPDZ_ERR_ARG;
    if (!p->alpha_loaded) return SPDZ_ERR_STATE;
    SPDZ_FIELD_SWITCH(p->field, (k_party_sigma<F><<<1, 32, 0, p->stream>>>(p->d)));
    if (cudaGetLastError() != cudaSuccess) return SPDZ_ERR_CUDA;
    if (cudaMemcpyAsync(p->h, p->d, sizeof(PartyState), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
        return SPDZ_ERR_CUDA;
    uint64_t *s = (uint64_t *)sigma_host;
    s[0] = p->h->sigma[0];
    if (p->field == SPDZ_F127) s[1] = p->h->sigma[1];
    if (opened_out) *opened_out = p->opened;
    p->opened = 0;
    p->epoch += 1;
    p->key = stream_key(p->seed, stream_id(SPDZ_KIND_CHECK, 0, 0, p->epoch));
    return SPDZ_OK;
}

}  // extern "C"
