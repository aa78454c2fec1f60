// linear_layer.cu -- the LinearLayer operator y = W x + b on a secret-shared
// dout x din matrix W, din vector x and dout vector b (Sec. III-D.3 "Data
// slicing" and "MPC-specific optimization"; the workload of Sec. IV).
//
// W is cut into tiles of R consecutive rows; tile t has its own
// matrix-vector triple (A_t: its rows of a dout x din matrix A, B_t: din
// values, C_t = A_t B_t).  The tile opens E_t = x - B_t and D_t = W_t - A_t,
// and every party computes
//   z_i = C_i + D_t B_{t,i} + A_{t,i} E_t + [i = 0] D_t E_t,
//   gamma(z)_i = gamma(C)_i + D_t gamma(B)_{t,i} + gamma(A)_{t,i} E_t + alpha_i D_t E_t,
// then y_i = z_i + b_i.  On one GPU every party's shares are resident, so the
// opening of D is fused with the products that use it: one pass reads each
// share of W and A once (the bytes that bound the operator), forms the
// opened D element in registers, adds its check terms and feeds the four
// matrix-vector sums of each party and D E.  E_t (din values per tile) is
// opened first by a small pass.  Opening order of the check log, from the
// epoch's current position: per tile, E_t, then D_t row by row.
#include <algorithm>
#include <type_traits>

#include "dealer.cuh"

namespace spdz {

struct LLState {
    spdz_buf A{}, B{}, C{};
    int64_t dout = 0, din = 0, R = 0;
    bool loaded = false;
    void *ws = nullptr;
    size_t ws_bytes = 0;
};

static LLState *ll_of(spdz_ctx *ctx) {
    if (!ctx->ll) ctx->ll = new LLState();
    return (LLState *)ctx->ll;
}

void ll_destroy(spdz_ctx *ctx) {
    LLState *s = (LLState *)ctx->ll;
    if (!s) return;
    if (s->ws) cudaFree(s->ws);
    delete s;
    ctx->ll = nullptr;
}

static int ll_ws(spdz_ctx *ctx, LLState *s, size_t need) {
    if (need <= s->ws_bytes) return SPDZ_OK;
    cudaStreamSynchronize(ctx->stream);
    if (s->ws) cudaFree(s->ws);
    s->ws = nullptr;
    s->ws_bytes = 0;
    if (cudaMalloc(&s->ws, need) != cudaSuccess) return set_err(ctx, SPDZ_ERR_OOM, "linear layer: workspace of %zu bytes", need);
    s->ws_bytes = need;
    return SPDZ_OK;
}

// Streaming (read once) and read-only cached loads of 4- and 8-byte words.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) { return __ldcs(reinterpret_cast<const unsigned int *>(p)); }
__device__ __forceinline__ uint64_t ld_stream(const uint64_t *p) {
    return __ldcs(reinterpret_cast<const unsigned long long *>(p));
}
__device__ __forceinline__ uint32_t ld_ro(const uint32_t *p) { return __ldg(reinterpret_cast<const unsigned int *>(p)); }
__device__ __forceinline__ uint64_t ld_ro(const uint64_t *p) { return __ldg(reinterpret_cast<const unsigned long long *>(p)); }

// ------------------------------------------------- deferred accumulation
// Sums of products kept unreduced and reduced once.  p = 2^32-5: a 64-bit
// product folds to 5 hi + lo < 2^35, so 2^29 terms fit a 64-bit sum.  p61:
// an exact 128-bit sum, folded back to its residue by flush() at most every
// three products (a residue and three 122-bit products stay below 2^124).
template <class F> struct LAcc;
template <> struct LAcc<F32> {
    uint64_t s = 0;
    __device__ __forceinline__ void mac(uint32_t a, uint32_t b) {
        const uint64_t x = (uint64_t)a * b;
        s += 5ull * (x >> 32) + (x & 0xffffffffull);
    }
    __device__ __forceinline__ void flush() {}
    __device__ __forceinline__ uint32_t get() const { return F32::reduce64(s); }
};
template <> struct LAcc<F61> {
    W61 w;    // after flush(): the residue so far, below 2^61
    __device__ __forceinline__ void mac(uint64_t a, uint64_t b) { w.mac(a, b); }
    __device__ __forceinline__ void flush() {
        w.lo = w.reduce();
        w.hi = 0;
    }
    __device__ __forceinline__ uint64_t get() const { return w.reduce(); }
};
template <class F> struct LUnroll { static constexpr int U = 3; };
template <> struct LUnroll<F32> { static constexpr int U = 4; };

// ------------------------------------------------------------- dealer
// c[r] = A_t[r] . B_t over the secrets (t = r / R), one warp per row.
template <class F>
__global__ void k_tile_matvec(const typename F::T *a, const typename F::T *b, typename F::T *c, int64_t dout,
                              int64_t din, int64_t R) {
    using T = typename F::T;
    constexpr int U = LUnroll<F>::U;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < dout; r += nwarps) {
        const T *ar = a + r * din, *bt = b + (r / R) * din;
        LAcc<F> s;
        for (int64_t k0 = lane; k0 < din; k0 += 32 * U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = k0 + 32 * u;
                if (k < din) s.mac(ar[k], ld_ro(bt + k));
            }
            s.flush();
        }
        const T v = warp_sum<F>(s.get());
        if (lane == 0) F::st(c + r, v);
    }
}

// ---------------------------------------------------------- the layer
// E_j = sum_i (x_i[k] - B_i[j]) for j = t*din + k, with its check terms.
template <class F, int NP>
__global__ void __launch_bounds__(256) k_ll_open_e(const typename F::T *xv, const typename F::T *xm, int64_t xs,
                                                   const typename F::T *bv, const typename F::T *bm, int64_t bs,
                                                   int64_t T, int64_t din, int64_t R, uint64_t base,
                                                   typename F::T *E, DevState *ds) {
    using Tt = typename F::T;
    const uint64_t key = ds->key;
    Tt acc[NP + 1];
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < T * din; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = j / din, k = j - t * din;
        Tt e = F::zero(), g[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            e = F::add(e, F::sub(F::ld(xv + i * xs + k), F::ld(bv + i * bs + j)));
            g[i] = F::sub(F::ld(xm + i * xs + k), F::ld(bm + i * bs + j));
        }
        F::st(E + j, e);
        const Tt r = Draw<F>::at(key, base + (uint64_t)(t * (din + R * din) + k));
        acc[0] = F::add(acc[0], F::mul(r, e));
#pragma unroll
        for (int i = 0; i < NP; ++i) acc[1 + i] = F::add(acc[1 + i], F::mul(r, g[i]));
    }
    block_accumulate<F, NP + 1>(acc, ds->acc);
}

// The same for p = 2^32-5 with 16-byte rows (din a multiple of 4): a
// thread takes four consecutive columns k .. k+3 of the tiles blockIdx.y,
// blockIdx.y + gridDim.y, ... (column index from the grid, no division), with
// 16-byte loads and stores, and keeps its check terms as exact 128-bit sums
// of the 64-bit products r * e, reduced once at the end (2^64 == 25 mod p).
struct Sum128 {
    uint64_t lo = 0, hi = 0;
    __device__ __forceinline__ void add(uint64_t v) {
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(lo), "+l"(hi) : "l"(v));
    }
    __device__ __forceinline__ uint32_t get() const { return F32::add(F32::reduce64(lo), F32::reduce64(25 * hi)); }
};

template <int NP>
__global__ void __launch_bounds__(256) k_ll_open_e4(const uint32_t *xv, const uint32_t *xm, int64_t xs,
                                                    const uint32_t *bv, const uint32_t *bm, int64_t bs, int64_t T,
                                                    int64_t din, int64_t R, uint64_t base, uint32_t *E,
                                                    DevState *ds) {
    using F = F32;
    const uint64_t key = ds->key;
    Sum128 sum[NP + 1];
    const int64_t k = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
    if (k < din) {
        uint32_t x[NP][4], gx[NP][4];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const uint4 v = *reinterpret_cast<const uint4 *>(xv + i * xs + k);
            const uint4 m = *reinterpret_cast<const uint4 *>(xm + i * xs + k);
            x[i][0] = v.x; x[i][1] = v.y; x[i][2] = v.z; x[i][3] = v.w;
            gx[i][0] = m.x; gx[i][1] = m.y; gx[i][2] = m.z; gx[i][3] = m.w;
        }
        for (int64_t t = blockIdx.y; t < T; t += gridDim.y) {
            const int64_t j = t * din + k;
            uint32_t e[4] = {0, 0, 0, 0}, g[NP][4];
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const uint4 b = __ldcs(reinterpret_cast<const uint4 *>(bv + i * bs + j));
                const uint4 gb = __ldcs(reinterpret_cast<const uint4 *>(bm + i * bs + j));
                const uint32_t bb[4] = {b.x, b.y, b.z, b.w}, gg[4] = {gb.x, gb.y, gb.z, gb.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    e[u] = F::add(e[u], F::sub(x[i][u], bb[u]));
                    g[i][u] = F::sub(gx[i][u], gg[u]);
                }
            }
            *reinterpret_cast<uint4 *>(E + j) = make_uint4(e[0], e[1], e[2], e[3]);
            const uint64_t j0 = base + (uint64_t)(t * (din + R * din) + k);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t r = Draw<F>::at(key, j0 + u);
                sum[0].add(r * e[u]);
#pragma unroll
                for (int i = 0; i < NP; ++i) sum[1 + i].add(r * g[i][u]);
            }
        }
    }
    uint32_t acc[NP + 1];
#pragma unroll
    for (int q = 0; q < NP + 1; ++q) acc[q] = sum[q].get();
    block_accumulate<F, NP + 1>(acc, ds->acc);
}

template <class F> struct LLArgs {
    using T = typename F::T;
    const T *wv, *wm;  int64_t ws;        // W   [n][dout*din]
    const T *av, *am;  int64_t as;        // A   [n][dout*din]
    const T *bv, *bm;  int64_t bs;        // B   [n][T*din]
    const T *cv, *cm;  int64_t cs;        // C   [n][dout]
    const T *pv, *pm;  int64_t ps;        // b (the bias) [n][dout]
    T *yv, *ym;        int64_t ys;        // y   [n][dout]
    const T *E;                           // [T*din] opened
    T *D;                                 // [dout*din] opened (optional)
    int64_t dout, din, R;
    uint64_t base;                        // check-log index of the layer's first opened value
    DevState *ds;
};

// One warp per row: the row's D elements (opened in registers), their check
// terms, and the row's sums D.B_i, D.gamma(B)_i, A_i.E, gamma(A)_i.E, D.E
// (element loads; used when the rows are not 16-byte aligned).
template <class F, int NP>
__global__ void __launch_bounds__(256) k_ll_rows(LLArgs<F> a) {
    using T = typename F::T;
    constexpr int U = LUnroll<F>::U;
    const int lane = threadIdx.x & 31;
    const uint64_t key = a.ds->key;
    T alpha[NP], chk[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) chk[k] = F::zero();
    const int64_t din = a.din, nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < a.dout; r += nwarps) {
        const int64_t t = r / a.R;
        const uint64_t pos0 = a.base + (uint64_t)(t * (din + a.R * din) + din + (r - t * a.R) * din);
        const int64_t row = r * din;
        const T *Et = a.E + t * din;
        LAcc<F> db[NP], dgb[NP], ae[NP], gae[NP], de, c0, ci[NP];
        for (int64_t k0 = lane; k0 < din; k0 += 32 * U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t k = k0 + 32 * u;
                if (k < din) {
                    T d = F::zero(), av[NP], gav[NP];
#pragma unroll
                    for (int i = 0; i < NP; ++i) {
                        const T w = ld_stream(a.wv + i * a.ws + row + k);
                        av[i] = ld_stream(a.av + i * a.as + row + k);
                        d = F::add(d, F::sub(w, av[i]));
                    }
                    const T e = ld_ro(Et + k);
                    const T rr = Draw<F>::at(key, pos0 + (uint64_t)k);
                    c0.mac(rr, d);
                    de.mac(d, e);
#pragma unroll
                    for (int i = 0; i < NP; ++i) {
                        gav[i] = ld_stream(a.am + i * a.as + row + k);
                        const T gw = ld_stream(a.wm + i * a.ws + row + k);
                        ci[i].mac(rr, F::sub(gw, gav[i]));
                        const int64_t q = i * a.bs + t * din + k;
                        db[i].mac(d, ld_ro(a.bv + q));
                        dgb[i].mac(d, ld_ro(a.bm + q));
                        ae[i].mac(av[i], e);
                        gae[i].mac(gav[i], e);
                    }
                    if (a.D) F::st(a.D + row + k, d);
                }
            }
            c0.flush();
            de.flush();
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                db[i].flush();
                dgb[i].flush();
                ae[i].flush();
                gae[i].flush();
                ci[i].flush();
            }
        }
        chk[0] = F::add(chk[0], c0.get());
#pragma unroll
        for (int i = 0; i < NP; ++i) chk[1 + i] = F::add(chk[1 + i], ci[i].get());
        const T sde = warp_sum<F>(de.get());
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const T z = warp_sum<F>(F::add(db[i].get(), ae[i].get()));
            const T gz = warp_sum<F>(F::add(dgb[i].get(), gae[i].get()));
            if (lane == 0) {
                T y = F::add(F::add(F::ld(a.cv + i * a.cs + r), z), F::ld(a.pv + i * a.ps + r));
                if (i == 0) y = F::add(y, sde);
                T gy = F::add(F::add(F::ld(a.cm + i * a.cs + r), gz), F::ld(a.pm + i * a.ps + r));
                gy = F::add(gy, F::mul(alpha[i], sde));
                F::st(a.yv + i * a.ys + r, y);
                F::st(a.ym + i * a.ys + r, gy);
            }
        }
    }
    block_accumulate<F, NP + 1>(chk, a.ds->acc);
}

// 16-byte vector of V elements (p = 2^32-5: 4, p61: 2).
template <class F> struct Vec16;
template <> struct Vec16<F32> {
    static constexpr int V = 4;
    __device__ __forceinline__ static void ld(const uint32_t *p, uint32_t (&o)[4], bool stream) {
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
        const uint4 t = stream ? __ldcs(q) : __ldg(q);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    }
};
template <> struct Vec16<F61> {
    static constexpr int V = 2;
    __device__ __forceinline__ static void ld(const uint64_t *p, uint64_t (&o)[2], bool stream) {
        const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(p);
        const ulonglong2 t = stream ? __ldcs(q) : __ldg(q);
        o[0] = t.x; o[1] = t.y;
    }
};

// The row kernel with 16-byte loads (din a multiple of V, every row and
// party row 16-byte aligned): each lane takes V consecutive columns per
// step.  Per step, a first pass over the parties reads W_i, A_i and their
// MACs and does everything that does not need the opened D (A_i E,
// gamma(A)_i E, the check terms r (gamma(W)_i - gamma(A)_i), and the sum
// forming D); a second pass reads B_i and gamma(B)_i for D B_i and
// D gamma(B)_i.
template <class F, int NP>
__device__ __forceinline__ void ll_rows_vec_body(const LLArgs<F> &a) {
    using T = typename F::T;
    constexpr int V = Vec16<F>::V;
    const int lane = threadIdx.x & 31;
    const uint64_t key = a.ds->key;
    T alpha[NP], chk[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) chk[k] = F::zero();
    const int64_t din = a.din, nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < a.dout; r += nwarps) {
        const int64_t t = r / a.R;
        const uint64_t pos0 = a.base + (uint64_t)(t * (din + a.R * din) + din + (r - t * a.R) * din);
        const int64_t row = r * din;
        const T *Et = a.E + t * din;
        LAcc<F> db[NP], dgb[NP], ae[NP], gae[NP], de, c0, ci[NP];
        for (int64_t k = (int64_t)lane * V; k < din; k += 32 * V) {
            T e[V], d[V], rr[V];
            Vec16<F>::ld(Et + k, e, false);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                d[j] = F::zero();
                rr[j] = Draw<F>::at(key, pos0 + (uint64_t)(k + j));
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                T w[V], av[V], gw[V], ga[V];
                Vec16<F>::ld(a.wv + i * a.ws + row + k, w, true);
                Vec16<F>::ld(a.av + i * a.as + row + k, av, true);
                Vec16<F>::ld(a.wm + i * a.ws + row + k, gw, true);
                Vec16<F>::ld(a.am + i * a.as + row + k, ga, true);
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    d[j] = F::add(d[j], F::sub(w[j], av[j]));
                    ae[i].mac(av[j], e[j]);
                    gae[i].mac(ga[j], e[j]);
                    ci[i].mac(rr[j], F::sub(gw[j], ga[j]));
                    if (j == 2) {          // at most three products between folds
                        ae[i].flush();
                        gae[i].flush();
                        ci[i].flush();
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < V; ++j) {
                c0.mac(rr[j], d[j]);
                de.mac(d[j], e[j]);
                if (j == 2) {
                    c0.flush();
                    de.flush();
                }
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                T bv[V], gb[V];
                const int64_t q = i * a.bs + t * din + k;
                Vec16<F>::ld(a.bv + q, bv, false);
                Vec16<F>::ld(a.bm + q, gb, false);
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    db[i].mac(d[j], bv[j]);
                    dgb[i].mac(d[j], gb[j]);
                    if (j == 2) {
                        db[i].flush();
                        dgb[i].flush();
                    }
                }
                ae[i].flush();
                gae[i].flush();
                ci[i].flush();
                db[i].flush();
                dgb[i].flush();
            }
            c0.flush();
            de.flush();
            if (a.D) {
#pragma unroll
                for (int j = 0; j < V; ++j) F::st(a.D + row + k + j, d[j]);
            }
        }
        chk[0] = F::add(chk[0], c0.get());
#pragma unroll
        for (int i = 0; i < NP; ++i) chk[1 + i] = F::add(chk[1 + i], ci[i].get());
        const T sde = warp_sum<F>(de.get());
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const T z = warp_sum<F>(F::add(db[i].get(), ae[i].get()));
            const T gz = warp_sum<F>(F::add(dgb[i].get(), gae[i].get()));
            if (lane == 0) {
                T y = F::add(F::add(F::ld(a.cv + i * a.cs + r), z), F::ld(a.pv + i * a.ps + r));
                if (i == 0) y = F::add(y, sde);
                T gy = F::add(F::add(F::ld(a.cm + i * a.cs + r), gz), F::ld(a.pm + i * a.ps + r));
                gy = F::add(gy, F::mul(alpha[i], sde));
                F::st(a.yv + i * a.ys + r, y);
                F::st(a.ym + i * a.ys + r, gy);
            }
        }
    }
    block_accumulate<F, NP + 1>(chk, a.ds->acc);
}

// The same row kernel with each row split between two warps (half of the
// columns each), a CTA taking blockDim/64 rows per round: with 8192 rows the
// rounds divide evenly over the CTAs, where one warp per row left the last
// of four rounds half empty.  Used for 2 parties at p = 2^32-5 (14 % faster
// at 8192 x 8192); with more parties or p61 the extra live sums cost more
// registers than the even rounds gain.
template <class F, int NP>
__device__ __forceinline__ void ll_rows_split_body(const LLArgs<F> &a) {
    using T = typename F::T;
    constexpr int V = Vec16<F>::V;
    const int lane = threadIdx.x & 31;
    const uint64_t key = a.ds->key;
    T alpha[NP], chk[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) chk[k] = F::zero();
    // Two warps share a row (each one half of the columns); a CTA takes
    // blockDim/64 rows per round, so the rounds divide the rows evenly over
    // the CTAs; the halves' row sums meet in shared memory (two buffers by
    // round parity, one CTA barrier per round).
    constexpr int RMAX = 16;
    __shared__ T part[2][RMAX][2 * NP + 1];
    const int warp = threadIdx.x >> 5, rpc = (int)(blockDim.x >> 6), h = warp & 1;
    const int64_t din = a.din, half = (din + 64 * V - 1) / (64 * V) * (32 * V);
    const int64_t klo = h * half, khi = min(din, (int64_t)(h + 1) * half);
    int par = 0;
    for (int64_t base = (int64_t)blockIdx.x * rpc; base < a.dout; base += (int64_t)gridDim.x * rpc, par ^= 1) {
        const int64_t r = base + (warp >> 1);
        const bool live = r < a.dout;
        const int64_t rr_ = live ? r : 0;
        const int64_t t = rr_ / a.R;
        const uint64_t pos0 = a.base + (uint64_t)(t * (din + a.R * din) + din + (rr_ - t * a.R) * din);
        const int64_t row = rr_ * din;
        const T *Et = a.E + t * din;
        LAcc<F> db[NP], dgb[NP], ae[NP], gae[NP], de, c0, ci[NP];
        for (int64_t k = klo + (int64_t)lane * V; live && k < khi; k += 32 * V) {
            T e[V], d[V], rr[V];
            Vec16<F>::ld(Et + k, e, false);
#pragma unroll
            for (int j = 0; j < V; ++j) {
                d[j] = F::zero();
                rr[j] = Draw<F>::at(key, pos0 + (uint64_t)(k + j));
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                T w[V], av[V], gw[V], ga[V];
                Vec16<F>::ld(a.wv + i * a.ws + row + k, w, true);
                Vec16<F>::ld(a.av + i * a.as + row + k, av, true);
                Vec16<F>::ld(a.wm + i * a.ws + row + k, gw, true);
                Vec16<F>::ld(a.am + i * a.as + row + k, ga, true);
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    d[j] = F::add(d[j], F::sub(w[j], av[j]));
                    ae[i].mac(av[j], e[j]);
                    gae[i].mac(ga[j], e[j]);
                    ci[i].mac(rr[j], F::sub(gw[j], ga[j]));
                    if (j == 2) {          // at most three products between folds
                        ae[i].flush();
                        gae[i].flush();
                        ci[i].flush();
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < V; ++j) {
                c0.mac(rr[j], d[j]);
                de.mac(d[j], e[j]);
                if (j == 2) {
                    c0.flush();
                    de.flush();
                }
            }
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                T bv[V], gb[V];
                const int64_t q = i * a.bs + t * din + k;
                Vec16<F>::ld(a.bv + q, bv, false);
                Vec16<F>::ld(a.bm + q, gb, false);
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    db[i].mac(d[j], bv[j]);
                    dgb[i].mac(d[j], gb[j]);
                    if (j == 2) {
                        db[i].flush();
                        dgb[i].flush();
                    }
                }
                ae[i].flush();
                gae[i].flush();
                ci[i].flush();
                db[i].flush();
                dgb[i].flush();
            }
            c0.flush();
            de.flush();
            if (a.D) {
#pragma unroll
                for (int j = 0; j < V; ++j) F::st(a.D + row + k + j, d[j]);
            }
        }
        chk[0] = F::add(chk[0], c0.get());
#pragma unroll
        for (int i = 0; i < NP; ++i) chk[1 + i] = F::add(chk[1 + i], ci[i].get());
        // this half's row sums: z_i, gamma(z)_i (D B_i + A_i E and MACs), D.E
        T zs[NP], gs[NP];
        const T sde = warp_sum<F>(de.get());
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            zs[i] = warp_sum<F>(F::add(db[i].get(), ae[i].get()));
            gs[i] = warp_sum<F>(F::add(dgb[i].get(), gae[i].get()));
        }
        if (h == 1 && lane == 0) {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                part[par][warp >> 1][i] = zs[i];
                part[par][warp >> 1][NP + i] = gs[i];
            }
            part[par][warp >> 1][2 * NP] = sde;
        }
        __syncthreads();
        if (h == 0 && lane == 0 && live) {
            const T sd = F::add(sde, part[par][warp >> 1][2 * NP]);
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                const T z = F::add(zs[i], part[par][warp >> 1][i]), gz = F::add(gs[i], part[par][warp >> 1][NP + i]);
                T y = F::add(F::add(F::ld(a.cv + i * a.cs + r), z), F::ld(a.pv + i * a.ps + r));
                if (i == 0) y = F::add(y, sd);
                T gy = F::add(F::add(F::ld(a.cm + i * a.cs + r), gz), F::ld(a.pm + i * a.ps + r));
                gy = F::add(gy, F::mul(alpha[i], sd));
                F::st(a.yv + i * a.ys + r, y);
                F::st(a.ym + i * a.ys + r, gy);
            }
        }
    }
    block_accumulate<F, NP + 1>(chk, a.ds->acc);
}

// The row kernel; the 2-party p61 layer runs three CTAs per SM (80
// registers, a little spilling: measured 10 % faster), every other instance
// the compiler's own register budget (three per SM made p = 2^32-5 no
// faster and 3 parties slower).
template <class F, int NP>
__global__ void __launch_bounds__(256) k_ll_rows_vec(LLArgs<F> a) {
    ll_rows_vec_body<F, NP>(a);
}
template <class F, int NP>
__global__ void __launch_bounds__(256, 3) k_ll_rows_vec3(LLArgs<F> a) {
    ll_rows_vec_body<F, NP>(a);
}
template <class F, int NP>
__global__ void __launch_bounds__(256) k_ll_rows_split(LLArgs<F> a) {
    ll_rows_split_body<F, NP>(a);
}

template <class F> static bool ll_vec_ok(const LLArgs<F> &a) {
    constexpr int V = Vec16<F>::V;
    auto al = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    auto st = [](int64_t s) { return (s * (int64_t)sizeof(typename F::T)) % 16 == 0; };
    return a.din % V == 0 && al(a.wv) && al(a.wm) && al(a.av) && al(a.am) && al(a.bv) && al(a.bm) && al(a.E) &&
           st(a.ws) && st(a.as) && st(a.bs);
}

template <class F, int NP>
static void deal_matvec(spdz_ctx *ctx, LLState *s, uint64_t seed, uint64_t sub, int64_t dout, int64_t din, int64_t R,
                        const void *alpha_shares_dev, const spdz_buf *A, const spdz_buf *B, const spdz_buf *C) {
    if constexpr (!std::is_same_v<F, F127>) {
        using Tt = typename F::T;
        const int64_t T = (dout + R - 1) / R;
        Tt *sa = (Tt *)s->ws, *sb = sa + dout * din, *sc = sb + T * din;
        const Tt *al = (const Tt *)alpha_shares_dev;
        auto kern = k_deal_shared<F, NP>;
        auto ka = make_keys<NP>(seed, SPDZ_KIND_MTRIPLE_A, sub);
        auto kb = make_keys<NP>(seed, SPDZ_KIND_MTRIPLE_B, sub);
        auto kc = make_keys<NP>(seed, SPDZ_KIND_MTRIPLE_C, sub);
        kern<<<grid_for(ctx, (const void *)kern, 256, 0, dout * din), 256, 0, ctx->stream>>>(
            ka, 0, dout * din, al, nullptr, (Tt *)A->val, (Tt *)A->mac, A->stride, sa);
        kern<<<grid_for(ctx, (const void *)kern, 256, 0, T * din), 256, 0, ctx->stream>>>(
            kb, 0, T * din, al, nullptr, (Tt *)B->val, (Tt *)B->mac, B->stride, sb);
        auto km = k_tile_matvec<F>;
        km<<<grid_for(ctx, (const void *)km, 256, 0, dout * 32), 256, 0, ctx->stream>>>(sa, sb, sc, dout, din, R);
        kern<<<grid_for(ctx, (const void *)kern, 256, 0, dout), 256, 0, ctx->stream>>>(
            kc, 0, dout, al, sc, (Tt *)C->val, (Tt *)C->mac, C->stride, nullptr);
    }
}

template <class F, int NP>
static void launch_ll(spdz_ctx *ctx, LLState *s, const spdz_buf *W, const spdz_buf *x, const spdz_buf *b,
                      const spdz_buf *y, int64_t dout, int64_t din, int64_t R, int64_t T, uint64_t base,
                      void *D_out_dev, void *E_out_dev) {
    if constexpr (!std::is_same_v<F, F127>) {
        using Tt = typename F::T;
        Tt *E = E_out_dev ? (Tt *)E_out_dev : (Tt *)s->ws;
        auto al16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
        const bool e4 = std::is_same_v<F, F32> && din % 4 == 0 && al16(x->val) && al16(x->mac) && al16(s->B.val) &&
                        al16(s->B.mac) && al16(E) && (x->stride * 4) % 16 == 0 && (s->B.stride * 4) % 16 == 0;
        if constexpr (std::is_same_v<F, F32>) {
            if (e4) {
                const dim3 g((unsigned)((din / 4 + 255) / 256), (unsigned)std::min<int64_t>(T, 65535));
                k_ll_open_e4<NP><<<g, 256, 0, ctx->stream>>>((const uint32_t *)x->val, (const uint32_t *)x->mac,
                                                             x->stride, (const uint32_t *)s->B.val,
                                                             (const uint32_t *)s->B.mac, s->B.stride, T, din, R, base,
                                                             E, ctx->ds);
            }
        }
        if (!e4) {
            auto ke = k_ll_open_e<F, NP>;
            ke<<<grid_for(ctx, (const void *)ke, 256, 0, T * din), 256, 0, ctx->stream>>>(
                (const Tt *)x->val, (const Tt *)x->mac, x->stride, (const Tt *)s->B.val, (const Tt *)s->B.mac,
                s->B.stride, T, din, R, base, E, ctx->ds);
        }
        LLArgs<F> a{};
        a.wv = (const Tt *)W->val; a.wm = (const Tt *)W->mac; a.ws = W->stride;
        a.av = (const Tt *)s->A.val; a.am = (const Tt *)s->A.mac; a.as = s->A.stride;
        a.bv = (const Tt *)s->B.val; a.bm = (const Tt *)s->B.mac; a.bs = s->B.stride;
        a.cv = (const Tt *)s->C.val; a.cm = (const Tt *)s->C.mac; a.cs = s->C.stride;
        a.pv = (const Tt *)b->val; a.pm = (const Tt *)b->mac; a.ps = b->stride;
        a.yv = (Tt *)y->val; a.ym = (Tt *)y->mac; a.ys = y->stride;
        a.E = E;
        a.D = (Tt *)D_out_dev;
        a.dout = dout; a.din = din; a.R = R;
        a.base = base;
        a.ds = ctx->ds;
        void (*kr)(LLArgs<F>) = k_ll_rows<F, NP>;
        if (ll_vec_ok(a)) {
            if constexpr (std::is_same_v<F, F61> && NP == 2) kr = k_ll_rows_vec3<F, NP>;
            else if constexpr (std::is_same_v<F, F32> && NP == 2) kr = k_ll_rows_split<F, NP>;
            else kr = k_ll_rows_vec<F, NP>;
        }
        kr<<<grid_for(ctx, (const void *)kr, 256, 0, dout * 32), 256, 0, ctx->stream>>>(a);
    }
}

}  // namespace spdz

using namespace spdz;

extern "C" {

int spdz_deal_matvec_triples(spdz_ctx *ctx, uint64_t seed, uint64_t sub, int64_t dout, int64_t din, int64_t tile_rows,
                             const void *alpha_shares_dev, const spdz_buf *A, const spdz_buf *B, const spdz_buf *C) {
    if (!ctx || !alpha_shares_dev || dout <= 0 || din <= 0 || tile_rows <= 0)
        return set_err(ctx, SPDZ_ERR_ARG, "deal_matvec_triples: bad argument");
    if (ctx->field == SPDZ_F127) return set_err(ctx, SPDZ_ERR_ARG, "deal_matvec_triples: p = 2^61-1 or 2^32-5 only");
    const int64_t R = std::min(tile_rows, dout), T = (dout + R - 1) / R;
    int rc;
    if ((rc = validate_buf(ctx, A, dout * din, "A")) || (rc = validate_buf(ctx, B, T * din, "B")) ||
        (rc = validate_buf(ctx, C, dout, "C")))
        return rc;
    LLState *s = ll_of(ctx);
    const size_t eb = elem_bytes(ctx->field);
    if ((rc = ll_ws(ctx, s, eb * (size_t)(dout * din + T * din + dout)))) return rc;
    SPDZ_FIELD_SWITCH(ctx->field, SPDZ_NP_SWITCH(ctx->n, (deal_matvec<F, NP>(ctx, s, seed, sub, dout, din, R, alpha_shares_dev, A, B, C))));
    return check_launch(ctx, "deal_matvec_triples");
}

int spdz_load_matvec_preproc(spdz_ctx *ctx, const spdz_buf *A, const spdz_buf *B, const spdz_buf *C, int64_t dout,
                             int64_t din, int64_t tile_rows) {
    if (!ctx || dout <= 0 || din <= 0 || tile_rows <= 0) return set_err(ctx, SPDZ_ERR_ARG, "load_matvec_preproc: bad sizes");
    const int64_t R = std::min(tile_rows, dout), T = (dout + R - 1) / R;
    int rc;
    if ((rc = validate_buf(ctx, A, dout * din, "A")) || (rc = validate_buf(ctx, B, T * din, "B")) ||
        (rc = validate_buf(ctx, C, dout, "C")))
        return rc;
    LLState *s = ll_of(ctx);
    s->A = *A;
    s->B = *B;
    s->C = *C;
    s->dout = dout;
    s->din = din;
    s->R = R;
    s->loaded = true;
    return SPDZ_OK;
}

int spdz_linear_layer(spdz_ctx *ctx, const spdz_buf *W, const spdz_buf *x, const spdz_buf *b, const spdz_buf *y,
                      int64_t dout, int64_t din, int64_t tile_rows, void *D_out_dev, void *E_out_dev) {
    if (!ctx || dout <= 0 || din <= 0 || tile_rows <= 0) return set_err(ctx, SPDZ_ERR_ARG, "linear_layer: bad sizes");
    if (ctx->field == SPDZ_F127) return set_err(ctx, SPDZ_ERR_ARG, "linear_layer: p = 2^61-1 or 2^32-5 only");
    if (!ctx->alpha_loaded) return set_err(ctx, SPDZ_ERR_STATE, "linear_layer: preprocessing not loaded");
    const int64_t R = std::min(tile_rows, dout), T = (dout + R - 1) / R;
    LLState *s = ll_of(ctx);
    if (!s->loaded || s->dout != dout || s->din != din || s->R != R)
        return set_err(ctx, SPDZ_ERR_TRIPLES, "linear_layer: no unused %lld x %lld matrix-vector triples with %lld-row tiles",
                       (long long)dout, (long long)din, (long long)R);
    int rc;
    if ((rc = validate_buf(ctx, W, dout * din, "W")) || (rc = validate_buf(ctx, x, din, "x")) ||
        (rc = validate_buf(ctx, b, dout, "b")) || (rc = validate_buf(ctx, y, dout, "y")))
        return rc;
    const size_t eb = elem_bytes(ctx->field);
    if ((D_out_dev && (uintptr_t)D_out_dev % eb) || (E_out_dev && (uintptr_t)E_out_dev % eb))
        return set_err(ctx, SPDZ_ERR_ALIGN, "linear_layer: misaligned D or E output");
    if (!E_out_dev && (rc = ll_ws(ctx, s, eb * (size_t)(T * din)))) return rc;
    s->loaded = false;   // the triples are consumed
    const uint64_t base = (uint64_t)ctx->opened;
    SPDZ_FIELD_SWITCH(ctx->field, SPDZ_NP_SWITCH(ctx->n, (launch_ll<F, NP>(ctx, s, W, x, b, y, dout, din, R, T, base, D_out_dev, E_out_dev))));
    if ((rc = check_launch(ctx, "linear_layer"))) return rc;
    ctx->opened += T * din + dout * din;
    return SPDZ_OK;
}

}  // extern "C"
