// ctx.cu -- context lifetime, error reporting, preprocessing registration,
// the device dealer and the batched MAC check.
#include <cstdarg>
#include <cstring>
#include <unordered_map>
#include <mutex>

#include "check.cuh"
#include "dealer.cuh"

namespace spdz {

int set_err(spdz_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

int check_cuda(spdz_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SPDZ_OK;
    return set_err(ctx, SPDZ_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int check_launch(spdz_ctx *ctx, const char *what) {
    return check_cuda(ctx, cudaGetLastError(), what);
}

int validate_buf(spdz_ctx *ctx, const spdz_buf *b, int64_t N, const char *name) {
    if (!b || !b->val || !b->mac) return set_err(ctx, SPDZ_ERR_ARG, "%s: null buffer", name);
    if (ctx->n > 1 && b->stride < N)
        return set_err(ctx, SPDZ_ERR_ARG, "%s: stride %lld < length %lld", name,
                       (long long)b->stride, (long long)N);
    size_t al = elem_bytes(ctx->field);
    if ((uintptr_t)b->val % al || (uintptr_t)b->mac % al)
        return set_err(ctx, SPDZ_ERR_ALIGN, "%s: pointers must be %zu-byte aligned", name, al);
    return SPDZ_OK;
}

bool buf_vec_ok(const spdz_buf *b, size_t eb) {
    return ((uintptr_t)b->val % 16 == 0) && ((uintptr_t)b->mac % 16 == 0) && ((b->stride * (int64_t)eb) % 16 == 0);
}

bool buf_vec2_ok(const spdz_buf *b) {
    return ((uintptr_t)b->val % 16 == 0) && ((uintptr_t)b->mac % 16 == 0) && (b->stride % 2 == 0);
}

// Grid of at most (resident CTAs per SM x SM count) CTAs, enough for
// `work_items` threads; kernels loop grid-stride over the rest.
int grid_for(spdz_ctx *ctx, const void *kernel, int block, size_t smem, int64_t work_items) {
    static std::mutex mu;
    static std::unordered_map<const void *, int> occ_cache;
    int occ = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = occ_cache.find(kernel);
        if (it != occ_cache.end()) {
            occ = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, smem) != cudaSuccess)
                occ = 1;
            if (occ < 1) occ = 1;
            occ_cache[kernel] = occ;
        }
    }
    int64_t need = (work_items + block - 1) / block;
    int64_t cap = (int64_t)occ * ctx->sm_count;
    int64_t g = need < cap ? need : cap;
    return (int)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------ small kernels

__global__ void k_set_seed(DevState *ds, uint64_t seed) {
    ds->check_seed = seed;
    ds->epoch = 0;
    ds->key = stream_key(seed, stream_id(SPDZ_KIND_CHECK, 0, 0, 0));
    for (int k = 0; k < MAXP + 1; ++k)
        for (int w = 0; w < 4; ++w) ds->acc[k][w] = 0;
    for (int i = 0; i < MAXP; ++i) ds->sig_run[i][0] = ds->sig_run[i][1] = 0;
    ds->partial_fail = 0;
}

template <class F>
__global__ void k_load_alpha(DevState *ds, const typename F::T *alpha, int n) {
    int i = threadIdx.x;
    if (i < n) {
        typename F::T a = F::ld(alpha + i);
        if constexpr (F::WORDS == 1) {
            ds->alpha[i][0] = a;
            ds->alpha[i][1] = 0;
        } else {
            ds->alpha[i][0] = a.lo;
            ds->alpha[i][1] = a.hi;
        }
    }
}

template <class F, int NP>
__global__ void k_check(DevState *ds, int final_check) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    check_epoch<F, NP>(ds, final_check);
}

// Launches the check kernel on the context's stream (used by spdz_mac_check
// and by circuit runs at their flush points).
int launch_check(spdz_ctx *ctx, int final_check) {
    SPDZ_FIELD_SWITCH(ctx->field, SPDZ_NP_SWITCH(ctx->n, (k_check<F, NP><<<1, 32, 0, ctx->stream>>>(ctx->ds, final_check))));
    return check_launch(ctx, "check kernel");
}

}  // namespace spdz

using namespace spdz;

// =================================================================== C ABI

extern "C" {

int spdz_ctx_create(spdz_ctx **out, int n_parties, int field, void *stream) {
    if (!out) return SPDZ_ERR_ARG;
    *out = nullptr;
    if (n_parties < 2 || n_parties > SPDZ_MAX_PARTIES) return SPDZ_ERR_ARG;
    if (field != SPDZ_F61 && field != SPDZ_F127 && field != SPDZ_F32) return SPDZ_ERR_ARG;
    spdz_ctx *ctx = new spdz_ctx();
    ctx->n = n_parties;
    ctx->field = field;
    ctx->stream = (cudaStream_t)stream;
    int rc;
    if ((rc = check_cuda(ctx, cudaGetDevice(&ctx->device), "cudaGetDevice"))) { delete ctx; return rc; }
    if ((rc = check_cuda(ctx, cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount,
                                                     ctx->device), "sm count"))) { delete ctx; return rc; }
    if (cudaMalloc(&ctx->ds, sizeof(DevState)) != cudaSuccess) { delete ctx; return SPDZ_ERR_OOM; }
    if (cudaMallocHost(&ctx->hres, sizeof(DevState)) != cudaSuccess) {
        cudaFree(ctx->ds);
        delete ctx;
        return SPDZ_ERR_OOM;
    }
    memset(ctx->hres, 0, sizeof(DevState));
    if ((rc = check_cuda(ctx, cudaMemsetAsync(ctx->ds, 0, sizeof(DevState), ctx->stream), "memset")) ||
        (k_set_seed<<<1, 1, 0, ctx->stream>>>(ctx->ds, 0), (rc = check_launch(ctx, "set seed")))) {
        spdz_ctx_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return SPDZ_OK;
}

int spdz_ctx_destroy(spdz_ctx *ctx) {
    if (!ctx) return SPDZ_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    if (ctx->ds) cudaFree(ctx->ds);
    if (ctx->hres) cudaFreeHost(ctx->hres);
    sched_destroy(ctx);
    mat_destroy(ctx);
    ll_destroy(ctx);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    if (ctx->pool_ev) cudaEventDestroy(ctx->pool_ev);
    for (auto e : ctx->copy_ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
    return SPDZ_OK;
}

const char *spdz_last_error(const spdz_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int spdz_ctx_set_stream(spdz_ctx *ctx, void *stream) {
    if (!ctx) return SPDZ_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return SPDZ_OK;
}

int spdz_deal_alpha(spdz_ctx *ctx, uint64_t seed, void *alpha_shares_dev) {
    if (!ctx || !alpha_shares_dev) return set_err(ctx, SPDZ_ERR_ARG, "deal_alpha: null argument");
    if ((uintptr_t)alpha_shares_dev % elem_bytes(ctx->field))
        return set_err(ctx, SPDZ_ERR_ALIGN, "deal_alpha: misaligned output");
    SPDZ_FIELD_SWITCH(ctx->field,
                      (k_deal_alpha<F><<<1, 32, 0, ctx->stream>>>(seed, ctx->n, (typename F::T *)alpha_shares_dev)));
    return check_launch(ctx, "deal_alpha");
}

int spdz_deal_shared(spdz_ctx *ctx, uint64_t seed, uint32_t kind, uint64_t sub, uint64_t j0,
                     int64_t count, const void *alpha_shares_dev, const void *secret_dev,
                     const spdz_buf *out, void *secret_out_dev) {
    if (!ctx || !alpha_shares_dev || count < 0) return set_err(ctx, SPDZ_ERR_ARG, "deal_shared: bad argument");
    if (count == 0) return SPDZ_OK;
    int rc = validate_buf(ctx, out, count, "deal_shared.out");
    if (rc) return rc;
    SPDZ_FIELD_SWITCH(ctx->field, SPDZ_NP_SWITCH(ctx->n, {
        using T = typename F::T;
        auto keys = make_keys<NP>(seed, kind, sub);
        auto kern = k_deal_shared<F, NP>;
        int grid = grid_for(ctx, (const void *)kern, 256, 0, count);
        kern<<<grid, 256, 0, ctx->stream>>>(keys, j0, count, (const T *)alpha_shares_dev,
                                            (const T *)secret_dev, (T *)out->val, (T *)out->mac,
                                            out->stride, (T *)secret_out_dev);
    }));
    return check_launch(ctx, "deal_shared");
}

int spdz_deal_triples(spdz_ctx *ctx, uint64_t seed, uint64_t j0, int64_t count,
                      const void *alpha_shares_dev, const spdz_buf *a, const spdz_buf *b,
                      const spdz_buf *c) {
    if (!ctx || !alpha_shares_dev || count < 0) return set_err(ctx, SPDZ_ERR_ARG, "deal_triples: bad argument");
    if (count == 0) return SPDZ_OK;
    int rc;
    if ((rc = validate_buf(ctx, a, count, "deal_triples.a")) || (rc = validate_buf(ctx, b, count, "deal_triples.b")) ||
        (rc = validate_buf(ctx, c, count, "deal_triples.c")))
        return rc;
    SPDZ_FIELD_SWITCH(ctx->field, SPDZ_NP_SWITCH(ctx->n, {
        using T = typename F::T;
        auto ka = make_keys<NP>(seed, SPDZ_KIND_TRIPLE_A, 0);
        auto kb = make_keys<NP>(seed, SPDZ_KIND_TRIPLE_B, 0);
        auto kc = make_keys<NP>(seed, SPDZ_KIND_TRIPLE_C, 0);
        auto kern = k_deal_triples<F, NP>;
        int grid = grid_for(ctx, (const void *)kern, 256, 0, count);
        kern<<<grid, 256, 0, ctx->stream>>>(ka, kb, kc, j0, count, (const T *)alpha_shares_dev,
                                            (T *)a->val, (T *)a->mac, a->stride, (T *)b->val,
                                            (T *)b->mac, b->stride, (T *)c->val, (T *)c->mac, c->stride);
    }));
    return check_launch(ctx, "deal_triples");
}

int spdz_load_preproc(spdz_ctx *ctx, const void *alpha_shares_dev, const spdz_buf *a,
                      const spdz_buf *b, const spdz_buf *c, int64_t n_triples) {
    if (!ctx || !alpha_shares_dev || n_triples < 0) return set_err(ctx, SPDZ_ERR_ARG, "load_preproc: bad argument");
    if ((uintptr_t)alpha_shares_dev % elem_bytes(ctx->field))
        return set_err(ctx, SPDZ_ERR_ALIGN, "load_preproc: misaligned alpha shares");
    int rc;
    if (n_triples > 0) {
        if ((rc = validate_buf(ctx, a, n_triples, "load_preproc.a")) ||
            (rc = validate_buf(ctx, b, n_triples, "load_preproc.b")) ||
            (rc = validate_buf(ctx, c, n_triples, "load_preproc.c")))
            return rc;
        ctx->ta = *a;
        ctx->tb = *b;
        ctx->tc = *c;
    }
    ctx->tri_total = n_triples;
    ctx->tri_cursor = 0;
    SPDZ_FIELD_SWITCH(ctx->field,
                      (k_load_alpha<F><<<1, 32, 0, ctx->stream>>>(ctx->ds, (const typename F::T *)alpha_shares_dev, ctx->n)));
    if ((rc = check_launch(ctx, "load alpha"))) return rc;
    // host-buffer runs copy triples into this pool on their own stream, after
    // everything enqueued before the registration (which may still use the
    // same memory)
    if (!ctx->pool_ev && (rc = check_cuda(ctx, cudaEventCreateWithFlags(&ctx->pool_ev, cudaEventDisableTiming), "pool event")))
        return rc;
    if ((rc = check_cuda(ctx, cudaEventRecord(ctx->pool_ev, ctx->stream), "pool event"))) return rc;
    ctx->alpha_loaded = true;
    return SPDZ_OK;
}

int spdz_triples_left(const spdz_ctx *ctx, int64_t *left) {
    if (!ctx || !left) return SPDZ_ERR_ARG;
    *left = ctx->tri_total - ctx->tri_cursor;
    return SPDZ_OK;
}

int spdz_set_check_seed(spdz_ctx *ctx, uint64_t seed) {
    if (!ctx) return SPDZ_ERR_ARG;
    if (ctx->opened != 0)
        return set_err(ctx, SPDZ_ERR_STATE, "set_check_seed: %lld values opened since the last check",
                       (long long)ctx->opened);
    k_set_seed<<<1, 1, 0, ctx->stream>>>(ctx->ds, seed);
    int rc = check_launch(ctx, "set seed");
    if (rc) return rc;
    ctx->check_seed = seed;
    ctx->epoch = 0;
    return SPDZ_OK;
}

int spdz_check_state(const spdz_ctx *ctx, int64_t *opened, int64_t *epoch) {
    if (!ctx) return SPDZ_ERR_ARG;
    if (opened) *opened = ctx->opened;
    if (epoch) *epoch = ctx->epoch;
    return SPDZ_OK;
}

int spdz_mac_check(spdz_ctx *ctx, int *passed, void *sigma_host) {
    if (!ctx || !passed) return set_err(ctx, SPDZ_ERR_ARG, "mac_check: null argument");
    if (!ctx->alpha_loaded) return set_err(ctx, SPDZ_ERR_STATE, "mac_check: no alpha shares loaded");
    int rc = launch_check(ctx, 1);
    if (rc) return rc;
    if ((rc = check_cuda(ctx, cudaMemcpyAsync(ctx->hres, ctx->ds, sizeof(DevState), cudaMemcpyDeviceToHost,
                                              ctx->stream), "check readback")) ||
        (rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "check sync")))
        return rc;
    ctx->opened = 0;
    ctx->epoch += 1;
    *passed = (int)ctx->hres->res_passed;
    if (sigma_host) {
        uint64_t *s = (uint64_t *)sigma_host;
        for (int i = 0; i < ctx->n; ++i) {
            if (ctx->field != SPDZ_F127) {
                s[i] = ctx->hres->res_sigma[i][0];
            } else {
                s[2 * i] = ctx->hres->res_sigma[i][0];
                s[2 * i + 1] = ctx->hres->res_sigma[i][1];
            }
        }
    }
    if (ctx->hres->err_flags & ERR_TIMEOUT)
        return set_err(ctx, SPDZ_ERR_TIMEOUT, "a device wait timed out; results are invalid");
    if (!*passed) return set_err(ctx, SPDZ_ERR_MAC, "MAC check failed in epoch %u", ctx->hres->res_epoch);
    return SPDZ_OK;
}

}  // extern "C"
