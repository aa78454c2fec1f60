// matmul.cu -- secret-shared matrix products with Beaver matrix triples
// (Sec. III-D.3 of the paper: one triple (A, B, C = A*B) per product).
//
// For X (m x k) and Y (k x n) shared among the parties, with a matrix triple:
//   E = sum_i (X_i - A_i),  F = sum_i (Y_i - B_i)        (opened; their MAC
//   shares gamma(X)_i - gamma(A)_i and gamma(Y)_i - gamma(B)_i join the
//   MAC-check epoch, E first, row-major, then F)
//   Z_i        = C_i        + E * (B_i + [i == 0] F)         + A_i * F
//   gamma(Z)_i = gamma(C)_i + E * (gamma(B)_i + alpha_i F)   + gamma(A)_i * F
// The E*F term of the Beaver identity is folded into the right operand, so
// every output block is one modular GEMM of inner length 2k:
//   [E | A_i] (m x 2k) times [B'_i ; F] (2k x n).
// Two product paths: 64-bit integer arithmetic on the CUDA cores (this
// file) and exact small-digit products on the tensor cores (matmul_tc.cu).
#include <algorithm>
#include <cstring>

#include "dealer.cuh"

namespace spdz {

// ------------------------------------------------ 64-bit modular GEMM (p61)
// Sum of products of 61-bit values in a 128-bit accumulator: 32 products
// (each < 2^122) plus a reduced remainder (< 2^61) stay below 2^128, so the
// accumulator is folded mod p every 32 steps.
__device__ __forceinline__ void mac128(uint64_t &lo, uint64_t &hi, uint64_t a, uint64_t b) {
    const uint64_t pl = a * b, ph = __umul64hi(a, b);
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(pl), "l"(ph));
}

// (hi:lo) < 2^128 reduced mod 2^61 - 1, using 2^61 == 1 and 2^64 == 2^3.
__device__ __forceinline__ uint64_t fold128_p61(uint64_t lo, uint64_t hi) {
    uint64_t t = (lo & F61::P) + (lo >> 61) + ((hi << 3) & F61::P) + (hi >> 58);
    t = (t & F61::P) + (t >> 61);
    return t >= F61::P ? t - F61::P : t;
}

constexpr int MT = 64;    // output tile edge
constexpr int KT = 16;    // inner-dimension step

struct MatSeg {            // one inner segment of the product: left rows x right columns
    const uint64_t *L;     // left matrix, row-major, leading dimension ldl
    int64_t ldl;
    const uint64_t *R;     // right matrix, row-major, leading dimension ldr
    int64_t ldr;
    int64_t k;             // inner length of the segment
};

struct MatJob {            // out = add + seg0 + seg1 (mod p), m x n, row-major
    MatSeg seg[2];
    const uint64_t *add;   // m x n (leading dimension ldo), may be null
    uint64_t *out;
    int64_t ldo;
};

// One CTA computes a 64 x 64 tile of one job (blockIdx.z selects the job);
// each of 256 threads owns a 4 x 4 block of outputs.
__global__ void __launch_bounds__(256) k_gemm_p61(const MatJob *jobs, int64_t m, int64_t n) {
    __shared__ uint64_t sL[KT][MT + 1];
    __shared__ uint64_t sR[KT][MT + 1];
    const MatJob &J = jobs[blockIdx.z];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t r0 = (int64_t)blockIdx.y * MT, c0 = (int64_t)blockIdx.x * MT;
    uint64_t lo[4][4], hi[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) lo[a][b] = hi[a][b] = 0;
    int steps = 0;
    for (int sgi = 0; sgi < 2; ++sgi) {
        const MatSeg S = J.seg[sgi];
        for (int64_t kk = 0; kk < S.k; kk += KT) {
            // stage a 64 x 16 slab of the left rows and a 16 x 64 slab of the right columns
            for (int e = threadIdx.x; e < MT * KT; e += blockDim.x) {
                const int rr = e / KT, q = e % KT;
                const int64_t gr = r0 + rr, gk = kk + q;
                sL[q][rr] = (gr < m && gk < S.k) ? S.L[gr * S.ldl + gk] : 0;
                const int q2 = e / MT, cc = e % MT;
                const int64_t gk2 = kk + q2, gc = c0 + cc;
                sR[q2][cc] = (gk2 < S.k && gc < n) ? S.R[gk2 * S.ldr + gc] : 0;
            }
            __syncthreads();
#pragma unroll 4
            for (int q = 0; q < KT; ++q) {
                uint64_t la[4], rb[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) la[a] = sL[q][ty * 4 + a];
#pragma unroll
                for (int b = 0; b < 4; ++b) rb[b] = sR[q][tx * 4 + b];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) mac128(lo[a][b], hi[a][b], la[a], rb[b]);
                if (++steps == 31) {
                    steps = 0;
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            lo[a][b] = fold128_p61(lo[a][b], hi[a][b]);
                            hi[a][b] = 0;
                        }
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t gr = r0 + ty * 4 + a;
        if (gr >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t gc = c0 + tx * 4 + b;
            if (gc >= n) continue;
            uint64_t v = fold128_p61(lo[a][b], hi[a][b]);
            if (J.add) v = F61::add(v, J.add[gr * J.ldo + gc]);
            J.out[gr * J.ldo + gc] = v;
        }
    }
}

// -------------------------------------------------------------- opening
// v_j = sum_i (x_i[j] - a_i[j]) for j < count, with MAC shares
// gamma(x)_i[j] - gamma(a)_i[j]; the check terms of v_j use coefficient index
// base + j.
template <class F, int NP>
__global__ void __launch_bounds__(256) k_open_diff(const typename F::T *xv, const typename F::T *xm, int64_t xs,
                                                   const typename F::T *av, const typename F::T *am, int64_t as,
                                                   int64_t count, uint64_t base, typename F::T *out, DevState *ds) {
    using T = typename F::T;
    const uint64_t key = ds->key;
    T acc[NP + 1];
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count; j += (int64_t)gridDim.x * blockDim.x) {
        T v = F::zero(), g[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            v = F::add(v, F::sub(F::ld(xv + i * xs + j), F::ld(av + i * as + j)));
            g[i] = F::sub(F::ld(xm + i * xs + j), F::ld(am + i * as + j));
        }
        F::st(out + j, v);
        const T r = Draw<F>::at(key, base + (uint64_t)j);
        acc[0] = F::add(acc[0], F::mul(r, v));
#pragma unroll
        for (int i = 0; i < NP; ++i) acc[1 + i] = F::add(acc[1 + i], F::mul(r, g[i]));
    }
    block_accumulate<F, NP + 1>(acc, ds->acc);
}

// Right operands with E*F folded in: Bp_i = B_i + [i == 0] F and
// Gp_i = gamma(B)_i + alpha_i F (k x n each, stored [2n][k*n]).
template <class F, int NP>
__global__ void k_fold_right(const typename F::T *bv, const typename F::T *bm, int64_t bs, const typename F::T *Fm,
                             int64_t kn, typename F::T *out, const DevState *ds) {
    using T = typename F::T;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < kn; j += (int64_t)gridDim.x * blockDim.x) {
        const T f = F::ld(Fm + j);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const T b = F::ld(bv + i * bs + j);
            F::st(out + (int64_t)i * kn + j, i == 0 ? F::add(b, f) : b);
            F::st(out + (int64_t)(NP + i) * kn + j, F::add(F::ld(bm + i * bs + j), F::mul(load_alpha<F>(ds, i), f)));
        }
    }
}

}  // namespace spdz

using namespace spdz;

namespace spdz {

struct MatState {
    spdz_buf A{}, B{}, C{};
    int64_t m = 0, k = 0, n = 0;
    bool loaded = false;
    void *ws = nullptr;
    size_t ws_bytes = 0;
};

static MatState *mat_of(spdz_ctx *ctx) {
    if (!ctx->mat) ctx->mat = new MatState();
    return (MatState *)ctx->mat;
}

void mat_destroy(spdz_ctx *ctx) {
    MatState *s = (MatState *)ctx->mat;
    if (!s) return;
    if (s->ws) cudaFree(s->ws);
    delete s;
    ctx->mat = nullptr;
}

static int mat_ws(spdz_ctx *ctx, MatState *s, size_t bytes) {
    if (bytes <= s->ws_bytes) return SPDZ_OK;
    if (s->ws) cudaFree(s->ws);
    s->ws = nullptr;
    s->ws_bytes = 0;
    if (cudaMalloc(&s->ws, bytes) != cudaSuccess) return set_err(ctx, SPDZ_ERR_OOM, "matmul: workspace of %zu bytes", bytes);
    s->ws_bytes = bytes;
    return SPDZ_OK;
}

// Modular GEMM jobs on the CUDA cores (p61): jobs[z] over an m x n output.
int gemm_p61_launch(spdz_ctx *ctx, const MatJob *h_jobs, int njobs, int64_t m, int64_t n, MatJob *d_jobs) {
    cudaMemcpyAsync(d_jobs, h_jobs, sizeof(MatJob) * (size_t)njobs, cudaMemcpyHostToDevice, ctx->stream);
    dim3 grid((unsigned)((n + MT - 1) / MT), (unsigned)((m + MT - 1) / MT), (unsigned)njobs);
    k_gemm_p61<<<grid, 256, 0, ctx->stream>>>(d_jobs, m, n);
    return check_launch(ctx, "gemm");
}

int matmul_tensor(spdz_ctx *ctx, const uint64_t *E, const uint64_t *Fm, const uint64_t *Rfold, const spdz_buf *A,
                  const spdz_buf *C, const spdz_buf *Z, int64_t m, int64_t k, int64_t n);

}  // namespace spdz

extern "C" {

int spdz_deal_matrix_triple(spdz_ctx *ctx, uint64_t seed, uint64_t sub, int64_t m, int64_t k, int64_t n,
                            const void *alpha_shares_dev, const spdz_buf *A, const spdz_buf *B, const spdz_buf *C) {
    if (!ctx || !alpha_shares_dev || m <= 0 || k <= 0 || n <= 0) return set_err(ctx, SPDZ_ERR_ARG, "deal_matrix_triple: bad argument");
    if (ctx->field != SPDZ_F61) return set_err(ctx, SPDZ_ERR_ARG, "deal_matrix_triple: p61 only");
    int rc;
    if ((rc = validate_buf(ctx, A, m * k, "A")) || (rc = validate_buf(ctx, B, k * n, "B")) || (rc = validate_buf(ctx, C, m * n, "C")))
        return rc;
    MatState *s = mat_of(ctx);
    const size_t need = sizeof(uint64_t) * (size_t)(m * k + k * n + m * n) + sizeof(MatJob) * 4;
    if ((rc = mat_ws(ctx, s, need))) return rc;
    uint64_t *sa = (uint64_t *)s->ws, *sb = sa + m * k, *sc = sb + k * n;
    MatJob *dj = (MatJob *)(sc + m * n);
    SPDZ_NP_SWITCH(ctx->n, {
        using F = F61;
        auto ka = make_keys<NP>(seed, SPDZ_KIND_MTRIPLE_A, sub);
        auto kb = make_keys<NP>(seed, SPDZ_KIND_MTRIPLE_B, sub);
        auto kc = make_keys<NP>(seed, SPDZ_KIND_MTRIPLE_C, sub);
        const uint64_t *al = (const uint64_t *)alpha_shares_dev;
        auto kern = k_deal_shared<F, NP>;
        k_deal_shared<F, NP><<<grid_for(ctx, (const void *)kern, 256, 0, m * k), 256, 0, ctx->stream>>>(
            ka, 0, m * k, al, nullptr, (uint64_t *)A->val, (uint64_t *)A->mac, A->stride, sa);
        k_deal_shared<F, NP><<<grid_for(ctx, (const void *)kern, 256, 0, k * n), 256, 0, ctx->stream>>>(
            kb, 0, k * n, al, nullptr, (uint64_t *)B->val, (uint64_t *)B->mac, B->stride, sb);
        MatJob j{};
        j.seg[0] = MatSeg{sa, k, sb, n, k};
        j.seg[1] = MatSeg{sa, k, sb, n, 0};
        j.add = nullptr;
        j.out = sc;
        j.ldo = n;
        if ((rc = gemm_p61_launch(ctx, &j, 1, m, n, dj))) return rc;
        k_deal_shared<F, NP><<<grid_for(ctx, (const void *)kern, 256, 0, m * n), 256, 0, ctx->stream>>>(
            kc, 0, m * n, al, sc, (uint64_t *)C->val, (uint64_t *)C->mac, C->stride, nullptr);
    });
    return check_launch(ctx, "deal_matrix_triple");
}

int spdz_load_matrix_preproc(spdz_ctx *ctx, const spdz_buf *A, const spdz_buf *B, const spdz_buf *C, int64_t m,
                             int64_t k, int64_t n) {
    if (!ctx || m <= 0 || k <= 0 || n <= 0) return set_err(ctx, SPDZ_ERR_ARG, "load_matrix_preproc: bad sizes");
    int rc;
    if ((rc = validate_buf(ctx, A, m * k, "A")) || (rc = validate_buf(ctx, B, k * n, "B")) || (rc = validate_buf(ctx, C, m * n, "C")))
        return rc;
    MatState *s = mat_of(ctx);
    s->A = *A;
    s->B = *B;
    s->C = *C;
    s->m = m;
    s->k = k;
    s->n = n;
    s->loaded = true;
    return SPDZ_OK;
}

int spdz_matmul(spdz_ctx *ctx, const spdz_buf *X, const spdz_buf *Y, const spdz_buf *Z, int64_t m, int64_t k,
                int64_t n, int path, void *E_out_dev, void *F_out_dev) {
    if (!ctx || m <= 0 || k <= 0 || n <= 0) return set_err(ctx, SPDZ_ERR_ARG, "matmul: bad sizes");
    if (ctx->field != SPDZ_F61) return set_err(ctx, SPDZ_ERR_ARG, "matmul: p61 only");
    if (path != SPDZ_MATMUL_CUDA_CORE && path != SPDZ_MATMUL_TENSOR) return set_err(ctx, SPDZ_ERR_ARG, "matmul: bad path");
    if (!ctx->alpha_loaded) return set_err(ctx, SPDZ_ERR_STATE, "matmul: preprocessing not loaded");
    MatState *s = mat_of(ctx);
    if (!s->loaded || s->m != m || s->k != k || s->n != n)
        return set_err(ctx, SPDZ_ERR_TRIPLES, "matmul: no unused %lld x %lld x %lld matrix triple", (long long)m, (long long)k, (long long)n);
    int rc;
    if ((rc = validate_buf(ctx, X, m * k, "X")) || (rc = validate_buf(ctx, Y, k * n, "Y")) || (rc = validate_buf(ctx, Z, m * n, "Z")))
        return rc;
    const int NPn = ctx->n;
    const size_t need = sizeof(uint64_t) * (size_t)(m * k + k * n + 2 * NPn * k * n) + sizeof(MatJob) * 2 * SPDZ_MAX_PARTIES;
    if ((rc = mat_ws(ctx, s, need))) return rc;
    uint64_t *E = E_out_dev ? (uint64_t *)E_out_dev : (uint64_t *)s->ws;
    uint64_t *Fm = F_out_dev ? (uint64_t *)F_out_dev : (uint64_t *)s->ws + m * k;
    uint64_t *Rf = (uint64_t *)s->ws + m * k + k * n;
    MatJob *dj = (MatJob *)(Rf + 2 * NPn * k * n);
    s->loaded = false;   // the triple is consumed
    const uint64_t base = (uint64_t)ctx->opened;
    SPDZ_NP_SWITCH(ctx->n, {
        using F = F61;
        auto ko = k_open_diff<F, NP>;
        ko<<<grid_for(ctx, (const void *)ko, 256, 0, m * k), 256, 0, ctx->stream>>>(
            (const uint64_t *)X->val, (const uint64_t *)X->mac, X->stride, (const uint64_t *)s->A.val,
            (const uint64_t *)s->A.mac, s->A.stride, m * k, base, E, ctx->ds);
        ko<<<grid_for(ctx, (const void *)ko, 256, 0, k * n), 256, 0, ctx->stream>>>(
            (const uint64_t *)Y->val, (const uint64_t *)Y->mac, Y->stride, (const uint64_t *)s->B.val,
            (const uint64_t *)s->B.mac, s->B.stride, k * n, base + (uint64_t)(m * k), Fm, ctx->ds);
        auto kf = k_fold_right<F, NP>;
        kf<<<grid_for(ctx, (const void *)kf, 256, 0, k * n), 256, 0, ctx->stream>>>(
            (const uint64_t *)s->B.val, (const uint64_t *)s->B.mac, s->B.stride, Fm, k * n, Rf, ctx->ds);
    });
    if ((rc = check_launch(ctx, "matmul open"))) return rc;
    ctx->opened += m * k + k * n;
    if (path == SPDZ_MATMUL_TENSOR) return matmul_tensor(ctx, E, Fm, Rf, &s->A, &s->C, Z, m, k, n);
    // CUDA cores: Z_i = C_i + [E | A_i] [Bp_i ; F], gamma(Z)_i likewise
    MatJob jobs[2 * SPDZ_MAX_PARTIES];
    for (int i = 0; i < NPn; ++i)
        for (int w = 0; w < 2; ++w) {
            MatJob &j = jobs[w * NPn + i];
            const uint64_t *Ai = (const uint64_t *)(w == 0 ? s->A.val : s->A.mac) + (int64_t)i * s->A.stride;
            j.seg[0] = MatSeg{E, k, Rf + (int64_t)(w * NPn + i) * k * n, n, k};
            j.seg[1] = MatSeg{Ai, k, Fm, n, k};
            j.add = (const uint64_t *)(w == 0 ? s->C.val : s->C.mac) + (int64_t)i * s->C.stride;
            j.out = (uint64_t *)(w == 0 ? Z->val : Z->mac) + (int64_t)i * Z->stride;
            j.ldo = n;
        }
    // (the job table is copied from pageable memory: staged before the call returns)
    return gemm_p61_launch(ctx, jobs, 2 * NPn, m, n, dj);
}

}  // extern "C"
