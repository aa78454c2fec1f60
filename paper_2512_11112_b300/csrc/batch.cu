// batch.cu -- elementwise online-phase kernels: local linear gates, Beaver
// multiplication (mask, open and combine fused in one pass, with the
// MAC-check random linear combination accumulated in the same pass), opens,
// inner products and public field arithmetic.
//
// Layout: party-major rows (party i's shares at ptr + i*stride); for p61 a
// thread moves two consecutive elements with one 128-bit access when every
// row is 16-byte aligned, for p127 one element per 128-bit access.
#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "vec.cuh"

namespace spdz {

int launch_check(spdz_ctx *ctx, int final_check);

// --------------------------------------------------------------- linear
template <class F> struct LinArgs {
    using T = typename F::T;
    const T *xv, *xm, *yv, *ym;
    int64_t xs, ys;
    T *zv, *zm;
    int64_t zs;
    int64_t N;
    int op;
    T k;
    const DevState *ds;
};

template <class F, int NP, int V>
__device__ __forceinline__ void linear_elems(const LinArgs<F> &a, int64_t e, const typename F::T (&kal)[NP]) {
    using T = typename F::T;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        T x[V], gx[V], z[V], gz[V];
        vld<F, V, false>(a.xv + i * a.xs + e, x);
        vld<F, V, false>(a.xm + i * a.xs + e, gx);
        if (a.op == SPDZ_OP_ADD || a.op == SPDZ_OP_SUB) {
            T y[V], gy[V];
            vld<F, V, false>(a.yv + i * a.ys + e, y);
            vld<F, V, false>(a.ym + i * a.ys + e, gy);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                z[v] = a.op == SPDZ_OP_ADD ? F::add(x[v], y[v]) : F::sub(x[v], y[v]);
                gz[v] = a.op == SPDZ_OP_ADD ? F::add(gx[v], gy[v]) : F::sub(gx[v], gy[v]);
            }
        } else if (a.op == SPDZ_OP_CMUL) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                z[v] = F::mul(a.k, x[v]);
                gz[v] = F::mul(a.k, gx[v]);
            }
        } else {  // CADD: party 0 adds k, every MAC share adds alpha_i * k
#pragma unroll
            for (int v = 0; v < V; ++v) {
                z[v] = i == 0 ? F::add(x[v], a.k) : x[v];
                gz[v] = F::add(gx[v], kal[i]);
            }
        }
        vst<F, V>(a.zv + i * a.zs + e, z);
        vst<F, V>(a.zm + i * a.zs + e, gz);
    }
}

template <class F, int NP, int V>
__global__ void __launch_bounds__(256) k_linear(LinArgs<F> a) {
    using T = typename F::T;
    T kal[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) kal[i] = a.op == SPDZ_OP_CADD ? F::mul(load_alpha<F>(a.ds, i), a.k) : F::zero();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t ng = a.N / V;
    for (int64_t g = tid; g < ng; g += stride) linear_elems<F, NP, V>(a, g * V, kal);
    for (int64_t e = ng * V + tid; e < a.N; e += stride) linear_elems<F, NP, 1>(a, e, kal);
}

// --------------------------------------------------------------- Beaver
template <class F> struct MulArgs {
    using T = typename F::T;
    const T *xv, *xm, *yv, *ym;
    int64_t xs, ys;
    const T *av, *am, *bv, *bm, *cv, *cm;   // triple rows at the consumed cursor
    int64_t as, bs, cs;
    T *zv, *zm;
    int64_t zs;
    T *opened;        // [2N] public values or null
    int64_t N;
    int64_t len;      // inner-product length (innerprod kernel only)
    uint64_t base;    // epoch index of the first opened value
    DevState *ds;
};

// One Beaver product per vector lane v at element e: masks, opens (sum over
// the party rows), combines, and adds the opened values' random-linear-
// combination terms to acc (acc[0] = A, acc[1+i] = S_i).
template <class F, int NP, int V>
__device__ __forceinline__ void beaver_core(const MulArgs<F> &a, int64_t e, int64_t opened_idx,
                                            uint64_t key, const typename F::T (&alpha)[NP],
                                            typename F::T (&acc)[NP + 1], typename F::T (&z)[NP][V],
                                            typename F::T (&gz)[NP][V], typename F::T (&eps)[V],
                                            typename F::T (&dlt)[V]) {
    using T = typename F::T;
    T av[NP][V], bv[NP][V];
#pragma unroll
    for (int v = 0; v < V; ++v) eps[v] = dlt[v] = F::zero();
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        T x[V], y[V];
        vld<F, V, false>(a.xv + i * a.xs + e, x);
        vld<F, V, false>(a.yv + i * a.ys + e, y);
        vld<F, V, true>(a.av + i * a.as + e, av[i]);
        vld<F, V, true>(a.bv + i * a.bs + e, bv[i]);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            eps[v] = F::add(eps[v], F::sub(x[v], av[i][v]));
            dlt[v] = F::add(dlt[v], F::sub(y[v], bv[i][v]));
        }
    }
    T de[V], re[V], rd[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        de[v] = F::mul(eps[v], dlt[v]);
        const uint64_t j = a.base + 2 * (uint64_t)(opened_idx + v);
        re[v] = Draw<F>::at(key, j);
        rd[v] = Draw<F>::at(key, j + 1);
        acc[0] = Fma<F>::f2(acc[0], re[v], eps[v], rd[v], dlt[v]);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        T c[V], gx[V], gy[V], ga[V], gb[V], gc[V];
        vld<F, V, true>(a.cv + i * a.cs + e, c);
        vld<F, V, false>(a.xm + i * a.xs + e, gx);
        vld<F, V, false>(a.ym + i * a.ys + e, gy);
        vld<F, V, true>(a.am + i * a.as + e, ga);
        vld<F, V, true>(a.bm + i * a.bs + e, gb);
        vld<F, V, true>(a.cm + i * a.cs + e, gc);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // each output one sum of products, reduced once where the field allows
            z[i][v] = Fma<F>::f2(i == 0 ? F::add(c[v], de[v]) : c[v], eps[v], bv[i][v], dlt[v], av[i][v]);
            gz[i][v] = Fma<F>::f3(gc[v], eps[v], gb[v], dlt[v], ga[v], alpha[i], de[v]);
            acc[1 + i] = Fma<F>::f2(acc[1 + i], re[v], F::sub(gx[v], ga[v]), rd[v], F::sub(gy[v], gb[v]));
        }
    }
}

// The operands of one p127 Beaver product at element e, read from the
// party-major rows (triple rows with the evict-first hint: read once).
// The hooks (before the value shares are read, after they are, before and
// after party i's other shares are read) do nothing here.
struct Src127Rows {
    const MulArgs<F127> &a;
    int64_t e;
    template <bool S> __device__ __forceinline__ static u128v g(const u128v *p) {
        u128v t[1];
        vld<F127, 1, S>(p, t);
        return t[0];
    }
    __device__ __forceinline__ u128v x(int i) const { return g<false>(a.xv + i * a.xs + e); }
    __device__ __forceinline__ u128v y(int i) const { return g<false>(a.yv + i * a.ys + e); }
    __device__ __forceinline__ u128v av(int i) const { return g<true>(a.av + i * a.as + e); }
    __device__ __forceinline__ u128v bv(int i) const { return g<true>(a.bv + i * a.bs + e); }
    __device__ __forceinline__ u128v c(int i) const { return g<true>(a.cv + i * a.cs + e); }
    __device__ __forceinline__ u128v gx(int i) const { return g<false>(a.xm + i * a.xs + e); }
    __device__ __forceinline__ u128v gy(int i) const { return g<false>(a.ym + i * a.ys + e); }
    __device__ __forceinline__ u128v ga(int i) const { return g<true>(a.am + i * a.as + e); }
    __device__ __forceinline__ u128v gb(int i) const { return g<true>(a.bm + i * a.bs + e); }
    __device__ __forceinline__ u128v gc(int i) const { return g<true>(a.cm + i * a.cs + e); }
    __device__ __forceinline__ void begin() const {}
    __device__ __forceinline__ void opened() const {}
    __device__ __forceinline__ void ready(int) const {}
    __device__ __forceinline__ void consumed(int) const {}
};

// p127 form of one Beaver product at element e, its operands from src.  The
// opened values' check terms go into exact three-word sums that stay
// unreduced across every element a thread handles (acc[0] = A, acc[1+i] =
// S_i); z and gamma(z) are one exact sum each, reduced once.  With sums !=
// nullptr the outputs are not reduced either: they are added to sums[i] /
// sums[NP + i] (inner products), without the eps delta terms (party 0's
// value, alpha_i eps delta in every MAC share), whose sum goes to *sde for
// one product per party at the end.
template <int NP, class SRC>
__device__ __forceinline__ void beaver_core127(const SRC &src, uint64_t j, uint64_t key, const u128v (&alpha)[NP],
                                               W127 (&acc)[NP + 1], u128v (&z)[NP], u128v (&gz)[NP], u128v &eps,
                                               u128v &dlt, W127 *sums, W127 *sde = nullptr) {
    using F = F127;
    u128v av[NP], bv[NP];
    eps = dlt = F::zero();
    src.begin();
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const u128v x = src.x(i), y = src.y(i);
        av[i] = src.av(i);
        bv[i] = src.bv(i);
        eps = F::add(eps, F::sub(x, av[i]));
        dlt = F::add(dlt, F::sub(y, bv[i]));
    }
    src.opened();
    const u128v de = W127::prod(eps, dlt).reduce();
    const u128v re = Draw<F>::at(key, j), rd = Draw<F>::at(key, j + 1);
    {
        // each product formed on its own; one three-word add into a sum
        W127 q = W127::prod(re, eps);
        q.add(W127::prod(rd, dlt));
        acc[0].add(q);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        src.ready(i);
        const u128v c = src.c(i), gx = src.gx(i), gy = src.gy(i), ga = src.ga(i), gb = src.gb(i), gc = src.gc(i);
        src.consumed(i);
        W127 v = W127::prod(eps, bv[i]), m = W127::prod(eps, gb);
        v.add(W127::prod(dlt, av[i]));
        v.add(c);
        if (!sums && i == 0) v.add(de);
        m.add(W127::prod(dlt, ga));
        if (sums) {
            m.add(gc);
        } else {
            W127 m2 = W127::prod(alpha[i], de);
            m2.add(gc);
            m.add(m2);
        }
        W127 q = W127::prod(re, F::sub(gx, ga));
        q.add(W127::prod(rd, F::sub(gy, gb)));
        acc[1 + i].add(q);
        if (sums) {
            sums[i].add(v);
            sums[NP + i].add(m);
        } else {
            z[i] = v.reduce();
            gz[i] = m.reduce();
        }
    }
    if (sums) sde->add(de);
}

template <int NP>
__device__ __forceinline__ void mul_elem127(const MulArgs<F127> &a, int64_t e, uint64_t key, const u128v (&alpha)[NP],
                                            W127 (&acc)[NP + 1]) {
    using F = F127;
    u128v z[NP], gz[NP], eps, dlt;
    beaver_core127<NP>(Src127Rows{a, e}, a.base + 2 * (uint64_t)e, key, alpha, acc, z, gz, eps, dlt, nullptr);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        F::st(a.zv + i * a.zs + e, z[i]);
        F::st(a.zm + i * a.zs + e, gz[i]);
    }
    if (a.opened) {
        F::st(a.opened + 2 * e, eps);
        F::st(a.opened + 2 * e + 1, dlt);
    }
}

template <class F, int NP, int V>
__device__ __forceinline__ void mul_elems(const MulArgs<F> &a, int64_t e, uint64_t key,
                                          const typename F::T (&alpha)[NP], typename F::T (&acc)[NP + 1]) {
    using T = typename F::T;
    T z[NP][V], gz[NP][V], eps[V], dlt[V];
    beaver_core<F, NP, V>(a, e, e, key, alpha, acc, z, gz, eps, dlt);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        vst<F, V>(a.zv + i * a.zs + e, z[i]);
        vst<F, V>(a.zm + i * a.zs + e, gz[i]);
    }
    if (a.opened) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            F::st(a.opened + 2 * (e + v), eps[v]);
            F::st(a.opened + 2 * (e + v) + 1, dlt[v]);
        }
    }
}

// Two CTAs of 256 threads per SM (at most 128 registers) while a thread's
// NP x V products fit them; larger instances keep one.
// p127 keeps its unreduced three-word check sums live across elements: one.
template <class F, int NP, int V> constexpr int mul_min_blocks() {
    return std::is_same_v<F, F127> ? 1 : NP * V <= 12 ? 2 : 1;
}

template <class F, int NP, int V>
__global__ void __launch_bounds__(256, (mul_min_blocks<F, NP, V>())) k_mul(MulArgs<F> a) {
    using T = typename F::T;
    const uint64_t key = a.ds->key;
    if constexpr (std::is_same_v<F, F127>) {
        u128v alpha[NP], acc[NP + 1];
        W127 wacc[NP + 1];
#pragma unroll
        for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.N; e += stride)
            mul_elem127<NP>(a, e, key, alpha, wacc);
#pragma unroll
        for (int k = 0; k < NP + 1; ++k) acc[k] = wacc[k].reduce();
        block_accumulate<F, NP + 1>(acc, a.ds->acc);
    } else {
        T alpha[NP], acc[NP + 1];
#pragma unroll
        for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
#pragma unroll
        for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const int64_t ng = a.N / V;
        for (int64_t g = tid; g < ng; g += stride) mul_elems<F, NP, V>(a, g * V, key, alpha, acc);
        for (int64_t e = ng * V + tid; e < a.N; e += stride) mul_elems<F, NP, 1>(a, e, key, alpha, acc);
        block_accumulate<F, NP + 1>(acc, a.ds->acc);
    }
}

__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_groups() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ------------------------------------------------ p127 Beaver batch, staged
// A p127 product is long integer arithmetic (about 2,400 instructions at
// n = 3).  Read straight from the rows, all of a product's loads are held in
// registers (233 of them: one CTA of 8 warps per SM) and each warp waits for
// them before it computes.  Here each thread streams its products' operands
// through private shared-memory slots with cp.async, one product ahead: the
// x, y, a, b value shares of every party are read from their slots when the
// party sums are formed, and the copies of the next product's value shares
// are issued at once; party i's c share and five MAC shares are read from
// their slots just before party i's combine, and the copies of the next
// product's are issued at once.  Every copy is in flight for about one
// product's arithmetic, and besides every party's a and b value shares only
// one party's other shares are read into registers at a time, so a thread
// needs 168 registers and 12 warps fit an SM.  Slot k of thread t is at
// k * B127S + t:
// a warp's 16-byte accesses of one slot cover 512 consecutive bytes.  Each
// thread reads only its own slots, after its own cp.async waits: no block
// barrier.  Per product 1 + NP copy groups are committed, in order: the
// value shares, then party 0's .. party NP-1's other shares; a read waits
// until at most NP groups (the ones committed after the one it needs) are
// pending.
constexpr int B127S = 384;
template <int NP, int BLK> constexpr size_t p127s_smem() { return (size_t)10 * NP * sizeof(u128v) * BLK; }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait_pending() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies of product e's value shares (slots 4i .. 4i+3: x, y, a, b of party i).
template <int NP, int BLK>
__device__ __forceinline__ void p127s_issue_values(const MulArgs<F127> &a, u128v *sm, int64_t e) {
    u128v *p = sm + threadIdx.x;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        cp_async16(p + (4 * i + 0) * BLK, a.xv + i * a.xs + e);
        cp_async16(p + (4 * i + 1) * BLK, a.yv + i * a.ys + e);
        cp_async16(p + (4 * i + 2) * BLK, a.av + i * a.as + e);
        cp_async16(p + (4 * i + 3) * BLK, a.bv + i * a.bs + e);
    }
}
// Copies of party i's c share and MAC shares of product e (slots 4 NP + 6i ..
// 4 NP + 6i + 5: c, gamma(x), gamma(y), gamma(a), gamma(b), gamma(c)).
template <int NP, int BLK>
__device__ __forceinline__ void p127s_issue_party(const MulArgs<F127> &a, u128v *sm, int64_t e, int i) {
    u128v *p = sm + (size_t)(4 * NP + 6 * i) * BLK + threadIdx.x;
    cp_async16(p + 0 * BLK, a.cv + i * a.cs + e);
    cp_async16(p + 1 * BLK, a.xm + i * a.xs + e);
    cp_async16(p + 2 * BLK, a.ym + i * a.ys + e);
    cp_async16(p + 3 * BLK, a.am + i * a.as + e);
    cp_async16(p + 4 * BLK, a.bm + i * a.bs + e);
    cp_async16(p + 5 * BLK, a.cm + i * a.cs + e);
}

// Operands of the current product from this thread's slots; the hooks wait
// for a set of slots before it is read and refill it (with element en, if
// en is valid) once it has been read.
template <int NP, int BLK> struct Src127Staged {
    const MulArgs<F127> &a;
    u128v *sm;
    int64_t en;
    bool more;          // en is an element to copy
    __device__ __forceinline__ u128v s(int k) const {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(sm + (size_t)k * BLK + threadIdx.x);
        return {v.x, v.y};
    }
    __device__ __forceinline__ u128v x(int i) const { return s(4 * i + 0); }
    __device__ __forceinline__ u128v y(int i) const { return s(4 * i + 1); }
    __device__ __forceinline__ u128v av(int i) const { return s(4 * i + 2); }
    __device__ __forceinline__ u128v bv(int i) const { return s(4 * i + 3); }
    __device__ __forceinline__ u128v c(int i) const { return s(4 * NP + 6 * i + 0); }
    __device__ __forceinline__ u128v gx(int i) const { return s(4 * NP + 6 * i + 1); }
    __device__ __forceinline__ u128v gy(int i) const { return s(4 * NP + 6 * i + 2); }
    __device__ __forceinline__ u128v ga(int i) const { return s(4 * NP + 6 * i + 3); }
    __device__ __forceinline__ u128v gb(int i) const { return s(4 * NP + 6 * i + 4); }
    __device__ __forceinline__ u128v gc(int i) const { return s(4 * NP + 6 * i + 5); }
    __device__ __forceinline__ void begin() const { cp_async_wait_pending<NP>(); }
    __device__ __forceinline__ void opened() const {
        if (more) p127s_issue_values<NP, BLK>(a, sm, en);
        cp_async_commit_group();
    }
    __device__ __forceinline__ void ready(int) const { cp_async_wait_pending<NP>(); }
    __device__ __forceinline__ void consumed(int i) const {
        if (more) p127s_issue_party<NP, BLK>(a, sm, en, i);
        cp_async_commit_group();
    }
};

// The first element's copies of a thread (if it has one), in the groups' order.
template <int NP, int BLK>
__device__ __forceinline__ void p127s_prologue(const MulArgs<F127> &a, u128v *sm, int64_t e, bool valid) {
    if (valid) p127s_issue_values<NP, BLK>(a, sm, e);
    cp_async_commit_group();
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        if (valid) p127s_issue_party<NP, BLK>(a, sm, e, i);
        cp_async_commit_group();
    }
}

template <int NP>
__global__ void __launch_bounds__(B127S, 1) k_mul127_staged(MulArgs<F127> a) {
    using F = F127;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u128v *sm = reinterpret_cast<u128v *>(smem_raw);
    const uint64_t key = a.ds->key;
    u128v alpha[NP], acc[NP + 1];
    W127 wacc[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
    const int64_t stride = (int64_t)gridDim.x * B127S;
    int64_t e = blockIdx.x * (int64_t)B127S + threadIdx.x;
    p127s_prologue<NP, B127S>(a, sm, e, e < a.N);
    for (; e < a.N; e += stride) {
        u128v z[NP], gz[NP], eps, dlt;
        beaver_core127<NP>(Src127Staged<NP, B127S>{a, sm, e + stride, e + stride < a.N}, a.base + 2 * (uint64_t)e,
                           key, alpha, wacc, z, gz, eps, dlt, nullptr);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            F::st(a.zv + i * a.zs + e, z[i]);
            F::st(a.zm + i * a.zs + e, gz[i]);
        }
        if (a.opened) {
            F::st(a.opened + 2 * e, eps);
            F::st(a.opened + 2 * e + 1, dlt);
        }
    }
    cp_async_wait_all_groups();
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = wacc[k].reduce();
    block_accumulate<F, NP + 1>(acc, a.ds->acc);
}

// Inner products: one warp per product t; lane l takes terms l, l+32, ...;
// the per-party sums of the term products (value and MAC) are reduced
// across the warp and stored by lane 0.  N = number of products.
template <class F, int NP>
__global__ void __launch_bounds__(256) k_innerprod(MulArgs<F> a) {
    using T = typename F::T;
    const uint64_t key = a.ds->key;
    T alpha[NP], acc[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
    const int lane = threadIdx.x & 31;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < a.N; t += wstride) {
        T sz[NP], sg[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) sz[i] = sg[i] = F::zero();
        for (int64_t k = lane; k < a.len; k += 32) {
            const int64_t e = t * a.len + k;
            T z[NP][1], gz[NP][1], eps[1], dlt[1];
            beaver_core<F, NP, 1>(a, e, e, key, alpha, acc, z, gz, eps, dlt);
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                sz[i] = F::add(sz[i], z[i][0]);
                sg[i] = F::add(sg[i], gz[i][0]);
            }
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            sz[i] = warp_sum<F>(sz[i]);
            sg[i] = warp_sum<F>(sg[i]);
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                F::st(a.zv + i * a.zs + t, sz[i]);
                F::st(a.zm + i * a.zs + t, sg[i]);
            }
        }
    }
    block_accumulate<F, NP + 1>(acc, a.ds->acc);
}

// Inner products, p61 and p = 2^32-5: the term's 10 NP words (value and MAC
// rows of x, y, a, b, c of every party) are copied with cp.async into a
// thread-private slot of a two-stage shared-memory buffer, the next term's
// copies issued before the current term's arithmetic, so each thread keeps a
// term of loads in flight while it computes (the register form issues a
// term's loads only after the last term's arithmetic: the 128-register
// budget has no room for two terms; deeper rings measured no faster).  Slots
// are [stage][word][thread]: a warp's accesses to one word are consecutive,
// conflict-free.  The MAC shares' alpha_i (eps delta) terms are summed as
// alpha_i (sum of eps delta) once per product, as the field allows: three
// fewer products per term at n = 3, the same sums; every sum is kept exact
// and reduced once (IpSum).
constexpr int IP_BLOCK = 128;

template <class F, int NP> constexpr size_t ip_stage_bytes() {
    return (size_t)2 * 10 * NP * sizeof(typename F::T) * IP_BLOCK;
}

__device__ __forceinline__ void cp_async_word(void *smem, const void *gmem, int bytes) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}

template <class F, int NP>
__device__ __forceinline__ void ip_issue(const MulArgs<F> &a, typename F::T *slot, int64_t e) {
    using T = typename F::T;
    const T *rows[10] = {a.xv, a.xm, a.yv, a.ym, a.av, a.am, a.bv, a.bm, a.cv, a.cm};
    const int64_t strides[10] = {a.xs, a.xs, a.ys, a.ys, a.as, a.as, a.bs, a.bs, a.cs, a.cs};
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int w = 0; w < 10; ++w)
            cp_async_word(slot + (i * 10 + w) * IP_BLOCK, rows[w] + i * strides[w] + e, (int)sizeof(T));
}

// Exact sums of the inner products' term products, reduced once per product
// (the term sums) or once per thread (the check sums): p61 in three words
// (S61); p = 2^32-5 as 128-bit sums of 64-bit products, with 2^64 == 25.
// lsub(a, b) is a value congruent to a - b that mac accepts.
template <class F> struct IpSum;
template <> struct IpSum<F61> {
    S61 s;
    __device__ __forceinline__ void add(uint64_t c) { s.add(c); }
    __device__ __forceinline__ void mac(uint64_t a, uint64_t b) { s.mac(a, b); }
    __device__ __forceinline__ uint64_t get() const { return s.reduce(); }
    __device__ __forceinline__ static uint64_t lsub(uint64_t a, uint64_t b) { return a + F61::P - b; }
};
template <> struct IpSum<F32> {
    uint64_t lo = 0, hi = 0;   // hi counts 2^64 carries: below 2^59 for any input that fits memory
    __device__ __forceinline__ void add64(uint64_t v) {
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(lo), "+l"(hi) : "l"(v));
    }
    __device__ __forceinline__ void add(uint32_t c) { add64(c); }
    __device__ __forceinline__ void mac(uint32_t a, uint32_t b) { add64((uint64_t)a * b); }
    __device__ __forceinline__ uint32_t get() const { return F32::add(F32::reduce64(lo), F32::reduce64(25 * hi)); }
    __device__ __forceinline__ static uint32_t lsub(uint32_t a, uint32_t b) { return F32::sub(a, b); }
};

template <class F, int NP>
__global__ void __launch_bounds__(IP_BLOCK) k_innerprod_staged(MulArgs<F> a) {
    using T = typename F::T;
    using Sum = IpSum<F>;
    static_assert(ip_stage_bytes<F, NP>() <= 227 * 1024, "buffer exceeds shared memory");
    extern __shared__ __align__(16) unsigned char ip_smem[];
    T *const stage0 = reinterpret_cast<T *>(ip_smem) + threadIdx.x;
    constexpr int W = 10 * NP * IP_BLOCK;   // elements of one stage
    const uint64_t key = a.ds->key;
    T alpha[NP];
    Sum acc[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
    const int lane = threadIdx.x & 31;
    const int64_t wstride = ((int64_t)gridDim.x * IP_BLOCK) >> 5;
    const int64_t nit = (a.len + 31) >> 5;
    int64_t t = (blockIdx.x * (int64_t)IP_BLOCK + threadIdx.x) >> 5;
    if (t < a.N && lane < a.len) ip_issue<F, NP>(a, stage0, t * a.len + lane);
    asm volatile("cp.async.commit_group;" ::: "memory");
    int s = 0;
    for (; t < a.N; t += wstride) {
        Sum sz[NP], sg[NP], sde;
        for (int64_t it = 0; it < nit; ++it) {
            const int64_t k = it * 32 + lane;
            // this thread's next term: later in the product, else the first
            // of the warp's next product
            const int64_t tn = it + 1 < nit ? t : t + wstride, kn = it + 1 < nit ? k + 32 : lane;
            if (tn < a.N && kn < a.len) ip_issue<F, NP>(a, stage0 + (s ^ 1) * W, tn * a.len + kn);
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            if (k < a.len) {
                const T *q = stage0 + s * W;
                auto word = [&](int i, int w) { return q[(i * 10 + w) * IP_BLOCK]; };
                T eps = F::zero(), dlt = F::zero();
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    eps = F::add(eps, F::sub(word(i, 0), word(i, 4)));
                    dlt = F::add(dlt, F::sub(word(i, 2), word(i, 6)));
                }
                sde.mac(eps, dlt);
                const uint64_t j = a.base + 2 * (uint64_t)(t * a.len + k);
                const T re = Draw<F>::at(key, j), rd = Draw<F>::at(key, j + 1);
                acc[0].mac(re, eps);
                acc[0].mac(rd, dlt);
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    const T am = word(i, 5), bm = word(i, 7);
                    sz[i].add(word(i, 8));
                    sz[i].mac(eps, word(i, 6));
                    sz[i].mac(dlt, word(i, 4));
                    sg[i].add(word(i, 9));
                    sg[i].mac(eps, bm);
                    sg[i].mac(dlt, am);
                    acc[1 + i].mac(re, Sum::lsub(word(i, 1), am));
                    acc[1 + i].mac(rd, Sum::lsub(word(i, 3), bm));
                }
            }
            s ^= 1;
        }
        // party 0's value share takes the sum of eps delta, every MAC share
        // alpha_i times it
        const T de = sde.get();
        T vz[NP], vg[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            vz[i] = sz[i].get();
            vg[i] = F::add(sg[i].get(), F::mul(alpha[i], de));
        }
        vz[0] = F::add(vz[0], de);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            vz[i] = warp_sum<F>(vz[i]);
            vg[i] = warp_sum<F>(vg[i]);
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                F::st(a.zv + i * a.zs + t, vz[i]);
                F::st(a.zm + i * a.zs + t, vg[i]);
            }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    T vacc[NP + 1];
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) vacc[k] = acc[k].get();
    block_accumulate<F, NP + 1>(vacc, a.ds->acc);
}

// p127 inner products: the term products' shares are summed unreduced
// across a lane's terms and reduced once per product before the warp sum.
// Two CTAs per SM: latency of the lanes' term loads is hidden by more
// resident warps (the sums then live in 128 registers with a few spilled,
// faster than one CTA and no spill).
// p127 inner products with their terms streamed through shared memory as in
// k_mul127_staged.  Each product goes to a pair of warps of one CTA: lane l
// of the pair's warp h takes terms 32 h + l, 32 h + l + 64, ...; a lane's
// next term (in this product, else the first of the pair's next product) is
// copied while it computes the current one.  At the end of a product the
// second warp hands its sums to the first through shared memory (a named
// barrier per pair).  With whole products per warp, 16,384 products over
// the 1776 resident warps take 10 rounds for 9.2 rounds of work; with pairs,
// 19 half-length rounds for 18.5.
constexpr int B127IP = 384;
constexpr int IP_PAIRS = B127IP / 64;

__device__ __forceinline__ void pair_sync(int pair) {
    asm volatile("bar.sync %0, 64;" ::"r"(1 + pair) : "memory");
}

template <int NP>
__global__ void __launch_bounds__(B127IP, 1) k_innerprod127_staged(MulArgs<F127> a) {
    using F = F127;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ u128v xch[IP_PAIRS][2 * NP];
    u128v *sm = reinterpret_cast<u128v *>(smem_raw);
    const uint64_t key = a.ds->key;
    u128v alpha[NP], acc[NP + 1];
    W127 wacc[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
    const int lane = threadIdx.x & 31, half = (threadIdx.x >> 5) & 1, pair = threadIdx.x >> 6;
    const int64_t pstride = (int64_t)gridDim.x * IP_PAIRS;
    const int64_t t0 = (int64_t)blockIdx.x * IP_PAIRS + pair;
    const int64_t k0 = 32 * half + lane;
    p127s_prologue<NP, B127IP>(a, sm, t0 * a.len + k0, t0 < a.N && k0 < a.len);
    for (int64_t t = t0; t < a.N; t += pstride) {
        W127 sums[2 * NP], sde;
        for (int64_t k = k0; k < a.len; k += 64) {
            // the lane's next term
            const bool same = k + 64 < a.len;
            const int64_t tn = same ? t : t + pstride, kn = same ? k + 64 : k0;
            const bool more = tn < a.N && kn < a.len;
            u128v z[NP], gz[NP], eps, dlt;
            const int64_t e = t * a.len + k;
            beaver_core127<NP>(Src127Staged<NP, B127IP>{a, sm, tn * a.len + kn, more}, a.base + 2 * (uint64_t)e, key,
                               alpha, wacc, z, gz, eps, dlt, sums, &sde);
        }
        const u128v de = sde.reduce();
        sums[0].add(de);
#pragma unroll
        for (int i = 0; i < NP; ++i) sums[NP + i].add(W127::prod(alpha[i], de));
        u128v sz[NP], sg[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            sz[i] = warp_sum<F>(sums[i].reduce());
            sg[i] = warp_sum<F>(sums[NP + i].reduce());
        }
        if (half && lane == 0) {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                xch[pair][i] = sz[i];
                xch[pair][NP + i] = sg[i];
            }
        }
        pair_sync(pair);
        if (!half && lane == 0) {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                F::st(a.zv + i * a.zs + t, F::add(sz[i], xch[pair][i]));
                F::st(a.zm + i * a.zs + t, F::add(sg[i], xch[pair][NP + i]));
            }
        }
        pair_sync(pair);   // the pair's slot is free for its next product
    }
    cp_async_wait_all_groups();
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = wacc[k].reduce();
    block_accumulate<F, NP + 1>(acc, a.ds->acc);
}

template <int NP>
__global__ void __launch_bounds__(256, 2) k_innerprod127(MulArgs<F127> a) {
    using F = F127;
    const uint64_t key = a.ds->key;
    u128v alpha[NP], acc[NP + 1];
    W127 wacc[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
    const int lane = threadIdx.x & 31;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < a.N; t += wstride) {
        W127 sums[2 * NP], sde;
        for (int64_t k = lane; k < a.len; k += 32) {
            u128v z[NP], gz[NP], eps, dlt;
            const int64_t e = t * a.len + k;
            beaver_core127<NP>(Src127Rows{a, e}, a.base + 2 * (uint64_t)e, key, alpha, wacc, z, gz, eps, dlt, sums,
                               &sde);
        }
        const u128v de = sde.reduce();
        sums[0].add(de);
#pragma unroll
        for (int i = 0; i < NP; ++i) sums[NP + i].add(W127::prod(alpha[i], de));
        u128v sz[NP], sg[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            sz[i] = warp_sum<F>(sums[i].reduce());
            sg[i] = warp_sum<F>(sums[NP + i].reduce());
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                F::st(a.zv + i * a.zs + t, sz[i]);
                F::st(a.zm + i * a.zs + t, sg[i]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = wacc[k].reduce();
    block_accumulate<F, NP + 1>(acc, a.ds->acc);
}

// ----------------------------------------------------------------- open
// Open V consecutive elements: sum the value shares, store the public value,
// and add the check terms r v and r gamma_i (one reduction per two products
// where the field allows it).
template <class F, int NP, int V>
__device__ __forceinline__ void open_elems(const MulArgs<F> &a, int64_t j, uint64_t key, typename F::T (&acc)[NP + 1]) {
    using T = typename F::T;
    T v[V], g[NP][V], r[V];
#pragma unroll
    for (int q = 0; q < V; ++q) v[q] = F::zero();
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        T x[V];
        vld<F, V, false>(a.xv + i * a.xs + j, x);
        vld<F, V, false>(a.xm + i * a.xs + j, g[i]);
#pragma unroll
        for (int q = 0; q < V; ++q) v[q] = F::add(v[q], x[q]);
    }
    vst<F, V>(a.opened + j, v);
#pragma unroll
    for (int q = 0; q < V; ++q) r[q] = Draw<F>::at(key, a.base + (uint64_t)(j + q));
    if constexpr (V % 2 == 0) {
#pragma unroll
        for (int q = 0; q < V; q += 2) {
            acc[0] = Fma<F>::f2(acc[0], r[q], v[q], r[q + 1], v[q + 1]);
#pragma unroll
            for (int i = 0; i < NP; ++i) acc[1 + i] = Fma<F>::f2(acc[1 + i], r[q], g[i][q], r[q + 1], g[i][q + 1]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < V; ++q) {
            acc[0] = F::add(acc[0], F::mul(r[q], v[q]));
#pragma unroll
            for (int i = 0; i < NP; ++i) acc[1 + i] = F::add(acc[1 + i], F::mul(r[q], g[i][q]));
        }
    }
}

// Stand-alone open: V elements per thread (16-byte loads when every row is
// 16-byte aligned), the N % V tail one element per thread.
template <class F, int NP, int V>
__global__ void __launch_bounds__(256) k_open(MulArgs<F> a) {
    using T = typename F::T;
    const uint64_t key = a.ds->key;
    T acc[NP + 1];
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t ng = a.N / V;
    for (int64_t g = tid; g < ng; g += stride) open_elems<F, NP, V>(a, g * V, key, acc);
    for (int64_t j = ng * V + tid; j < a.N; j += stride) open_elems<F, NP, 1>(a, j, key, acc);
    block_accumulate<F, NP + 1>(acc, a.ds->acc);
}

// ------------------------------------------------------ public field op
template <class F>
__global__ void k_field_op(int op, const typename F::T *x, const typename F::T *y, typename F::T *out, int64_t N) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        typename F::T a = F::ld(x + j), b = F::ld(y + j);
        F::st(out + j, op == SPDZ_OP_ADD ? F::add(a, b) : op == SPDZ_OP_SUB ? F::sub(a, b) : F::mul(a, b));
    }
}

template <class F> static typename F::T host_elem(const void *k) {
    if constexpr (std::is_same_v<F, F32>) {
        return (uint32_t)*(const uint64_t *)k;
    } else if constexpr (F::WORDS == 1) {
        return *(const uint64_t *)k;
    } else {
        const uint64_t *w = (const uint64_t *)k;
        return typename F::T{w[0], w[1]};
    }
}

template <class F> static bool host_canonical(const void *k) {
    if constexpr (std::is_same_v<F, F32>) {
        return *(const uint64_t *)k < F32::P;
    } else if constexpr (F::WORDS == 1) {
        return *(const uint64_t *)k < F61::P;
    } else {
        const uint64_t *w = (const uint64_t *)k;
        return w[1] < F127::PHI || (w[1] == F127::PHI && w[0] < F127::PLO);
    }
}


// The staged kernel's ring is above the default 48 KB of dynamic shared
// memory: raise the kernel's limit once per device.
template <class F, int NP> static void ip_smem_attr(spdz_ctx *ctx, const void *kern, size_t smem) {
    static std::atomic<uint64_t> done{0};
    const uint64_t bit = 1ull << (ctx->device & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    done.fetch_or(bit, std::memory_order_acq_rel);
}

// The staged p127 kernels' slots are above the default 48 KB of dynamic
// shared memory: raise a kernel's limit once per device (KIND: 0 the batch,
// 1 the inner products).
template <int NP, int KIND> static void p127s_smem_attr(spdz_ctx *ctx, const void *kern, size_t smem) {
    static std::atomic<uint64_t> done{0};
    const uint64_t bit = 1ull << (ctx->device & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    done.fetch_or(bit, std::memory_order_acq_rel);
}

template <class F, int NP>
static void launch_innerprod(spdz_ctx *ctx, const MulArgs<F> &a, int64_t count) {
    if constexpr (std::is_same_v<F, F127> && NP <= 3) {
        // terms staged through shared memory (up to 180 KB per CTA)
        auto kern = k_innerprod127_staged<NP>;
        constexpr size_t smem = p127s_smem<NP, B127IP>();
        p127s_smem_attr<NP, 1>(ctx, (const void *)kern, smem);
        kern<<<grid_for(ctx, (const void *)kern, B127IP, smem, count * 64), B127IP, smem, ctx->stream>>>(a);
    } else if constexpr (std::is_same_v<F, F127>) {
        auto kern = k_innerprod127<NP>;
        kern<<<grid_for(ctx, (const void *)kern, 256, 0, count * 32), 256, 0, ctx->stream>>>(a);
    } else {
        auto kern = k_innerprod_staged<F, NP>;
        constexpr size_t smem = ip_stage_bytes<F, NP>();
        ip_smem_attr<F, NP>(ctx, (const void *)kern, smem);
        kern<<<grid_for(ctx, (const void *)kern, IP_BLOCK, smem, count * 32), IP_BLOCK, smem, ctx->stream>>>(a);
    }
}

template <class F, int NP>
static void launch_linear(spdz_ctx *ctx, const LinArgs<F> &a, bool v2) {
    if constexpr (std::is_same_v<F, F61>) {
        if (v2) {
            auto kern = k_linear<F, NP, 2>;
            kern<<<grid_for(ctx, (const void *)kern, 256, 0, (a.N + 1) / 2), 256, 0, ctx->stream>>>(a);
            return;
        }
    } else if constexpr (std::is_same_v<F, F32>) {
        if (v2) {
            auto kern = k_linear<F, NP, 4>;
            kern<<<grid_for(ctx, (const void *)kern, 256, 0, (a.N + 3) / 4), 256, 0, ctx->stream>>>(a);
            return;
        }
    }
    auto kern = k_linear<F, NP, 1>;
    kern<<<grid_for(ctx, (const void *)kern, 256, 0, a.N), 256, 0, ctx->stream>>>(a);
}

template <class F, int NP>
static void launch_mul(spdz_ctx *ctx, const MulArgs<F> &a, bool v2) {
    if constexpr (std::is_same_v<F, F61>) {
        if (v2) {
            auto kern = k_mul<F, NP, 2>;
            kern<<<grid_for(ctx, (const void *)kern, 256, 0, (a.N + 1) / 2), 256, 0, ctx->stream>>>(a);
            return;
        }
    } else if constexpr (std::is_same_v<F, F32>) {
        if (v2) {
            auto kern = k_mul<F, NP, 4>;
            kern<<<grid_for(ctx, (const void *)kern, 256, 0, (a.N + 3) / 4), 256, 0, ctx->stream>>>(a);
            return;
        }
    }
    if constexpr (std::is_same_v<F, F127> && NP <= 3) {
        // operands staged through shared memory (up to 192 KB per CTA)
        auto kern = k_mul127_staged<NP>;
        constexpr size_t smem = p127s_smem<NP, B127S>();
        p127s_smem_attr<NP, 0>(ctx, (const void *)kern, smem);
        kern<<<grid_for(ctx, (const void *)kern, B127S, smem, a.N), B127S, smem, ctx->stream>>>(a);
        return;
    }
    auto kern = k_mul<F, NP, 1>;
    kern<<<grid_for(ctx, (const void *)kern, 256, 0, a.N), 256, 0, ctx->stream>>>(a);
}

}  // namespace spdz

using namespace spdz;

static int take_triples(spdz_ctx *ctx, int64_t count, int64_t *t0) {
    if (ctx->tri_total - ctx->tri_cursor < count)
        return set_err(ctx, SPDZ_ERR_TRIPLES, "need %lld triples, %lld left", (long long)count,
                       (long long)(ctx->tri_total - ctx->tri_cursor));
    *t0 = ctx->tri_cursor;
    ctx->tri_cursor += count;
    return SPDZ_OK;
}

template <class F>
static void fill_mul_args(spdz_ctx *ctx, MulArgs<F> &a, const spdz_buf *x, const spdz_buf *y, const spdz_buf *z,
                          int64_t t0) {
    using T = typename F::T;
    a.xv = (const T *)x->val; a.xm = (const T *)x->mac; a.xs = x->stride;
    a.yv = (const T *)y->val; a.ym = (const T *)y->mac; a.ys = y->stride;
    a.av = (const T *)ctx->ta.val + t0; a.am = (const T *)ctx->ta.mac + t0; a.as = ctx->ta.stride;
    a.bv = (const T *)ctx->tb.val + t0; a.bm = (const T *)ctx->tb.mac + t0; a.bs = ctx->tb.stride;
    a.cv = (const T *)ctx->tc.val + t0; a.cm = (const T *)ctx->tc.mac + t0; a.cs = ctx->tc.stride;
    a.zv = (T *)z->val; a.zm = (T *)z->mac; a.zs = z->stride;
    a.ds = ctx->ds;
    a.base = (uint64_t)ctx->opened;
}

extern "C" {

int spdz_linear(spdz_ctx *ctx, int op, const spdz_buf *x, const spdz_buf *y, const void *k_host,
                const spdz_buf *z, int64_t N) {
    if (!ctx) return SPDZ_ERR_ARG;
    if (N < 0 || op < SPDZ_OP_ADD || op > SPDZ_OP_CADD) return set_err(ctx, SPDZ_ERR_ARG, "linear: bad op or size");
    if (N == 0) return SPDZ_OK;
    int rc;
    const bool binary = op == SPDZ_OP_ADD || op == SPDZ_OP_SUB;
    if ((rc = validate_buf(ctx, x, N, "linear.x")) || (binary && (rc = validate_buf(ctx, y, N, "linear.y"))) ||
        (rc = validate_buf(ctx, z, N, "linear.z")))
        return rc;
    if (!binary && !k_host) return set_err(ctx, SPDZ_ERR_ARG, "linear: constant required");
    if (op == SPDZ_OP_CADD && !ctx->alpha_loaded) return set_err(ctx, SPDZ_ERR_STATE, "linear: CADD needs alpha shares");
    const size_t eb = elem_bytes(ctx->field);
    const bool v2 = ctx->field != SPDZ_F127 && buf_vec_ok(x, eb) && buf_vec_ok(z, eb) && (!binary || buf_vec_ok(y, eb));
    SPDZ_FIELD_SWITCH(ctx->field, {
        if (!binary && !host_canonical<F>(k_host)) return set_err(ctx, SPDZ_ERR_ARG, "linear: constant not in [0, p)");
        using T = typename F::T;
        LinArgs<F> a{};
        a.xv = (const T *)x->val; a.xm = (const T *)x->mac; a.xs = x->stride;
        if (binary) { a.yv = (const T *)y->val; a.ym = (const T *)y->mac; a.ys = y->stride; }
        a.zv = (T *)z->val; a.zm = (T *)z->mac; a.zs = z->stride;
        a.N = N; a.op = op; a.k = binary ? F::zero() : host_elem<F>(k_host); a.ds = ctx->ds;
        SPDZ_NP_SWITCH(ctx->n, launch_linear<F, NP>(ctx, a, v2));
    });
    return check_launch(ctx, "linear");
}

int spdz_mul_batch(spdz_ctx *ctx, const spdz_buf *x, const spdz_buf *y, const spdz_buf *z, int64_t N,
                   void *opened_dev) {
    if (!ctx) return SPDZ_ERR_ARG;
    if (N < 0) return set_err(ctx, SPDZ_ERR_ARG, "mul_batch: negative size");
    if (N == 0) return SPDZ_OK;
    if (!ctx->alpha_loaded) return set_err(ctx, SPDZ_ERR_STATE, "mul_batch: preprocessing not loaded");
    int rc;
    if ((rc = validate_buf(ctx, x, N, "mul_batch.x")) || (rc = validate_buf(ctx, y, N, "mul_batch.y")) ||
        (rc = validate_buf(ctx, z, N, "mul_batch.z")))
        return rc;
    if (opened_dev && (uintptr_t)opened_dev % elem_bytes(ctx->field))
        return set_err(ctx, SPDZ_ERR_ALIGN, "mul_batch: misaligned opened buffer");
    int64_t t0;
    if ((rc = take_triples(ctx, N, &t0))) return rc;
    SPDZ_FIELD_SWITCH(ctx->field, {
        MulArgs<F> a{};
        fill_mul_args<F>(ctx, a, x, y, z, t0);
        a.opened = (typename F::T *)opened_dev;
        a.N = N;
        // the vector path needs every row 16-byte aligned (2 p61 or 4 p32 elements)
        const size_t eb = sizeof(typename F::T);
        spdz_buf ta = ctx->ta, tb = ctx->tb, tc = ctx->tc;
        ta.val = (char *)ta.val + eb * t0; ta.mac = (char *)ta.mac + eb * t0;
        tb.val = (char *)tb.val + eb * t0; tb.mac = (char *)tb.mac + eb * t0;
        tc.val = (char *)tc.val + eb * t0; tc.mac = (char *)tc.mac + eb * t0;
        const bool v2 = F::WORDS == 1 && buf_vec_ok(x, eb) && buf_vec_ok(y, eb) && buf_vec_ok(z, eb) &&
                        buf_vec_ok(&ta, eb) && buf_vec_ok(&tb, eb) && buf_vec_ok(&tc, eb) &&
                        ((uintptr_t)opened_dev % 16 == 0);
        SPDZ_NP_SWITCH(ctx->n, launch_mul<F, NP>(ctx, a, v2));
    });
    if ((rc = check_launch(ctx, "mul_batch"))) return rc;
    ctx->opened += 2 * N;
    return SPDZ_OK;
}

int spdz_innerprod_batch(spdz_ctx *ctx, const spdz_buf *x, const spdz_buf *y, const spdz_buf *z, int64_t count,
                         int64_t len) {
    if (!ctx) return SPDZ_ERR_ARG;
    if (count < 0 || len < 0) return set_err(ctx, SPDZ_ERR_ARG, "innerprod: negative size");
    if (count == 0) return SPDZ_OK;
    if (!ctx->alpha_loaded) return set_err(ctx, SPDZ_ERR_STATE, "innerprod: preprocessing not loaded");
    const int64_t T = count * len;
    int rc;
    if ((rc = validate_buf(ctx, x, T, "innerprod.x")) || (rc = validate_buf(ctx, y, T, "innerprod.y")) ||
        (rc = validate_buf(ctx, z, count, "innerprod.z")))
        return rc;
    int64_t t0;
    if ((rc = take_triples(ctx, T, &t0))) return rc;
    SPDZ_FIELD_SWITCH(ctx->field, {
        MulArgs<F> a{};
        fill_mul_args<F>(ctx, a, x, y, z, t0);
        a.N = count;
        a.len = len;
        SPDZ_NP_SWITCH(ctx->n, launch_innerprod<F, NP>(ctx, a, count));
    });
    if ((rc = check_launch(ctx, "innerprod"))) return rc;
    ctx->opened += 2 * T;
    return SPDZ_OK;
}

int spdz_open(spdz_ctx *ctx, const spdz_buf *x, void *out_dev, int64_t N) {
    if (!ctx) return SPDZ_ERR_ARG;
    if (N < 0 || !out_dev) return set_err(ctx, SPDZ_ERR_ARG, "open: bad argument");
    if (N == 0) return SPDZ_OK;
    int rc;
    if ((rc = validate_buf(ctx, x, N, "open.x"))) return rc;
    if ((uintptr_t)out_dev % elem_bytes(ctx->field)) return set_err(ctx, SPDZ_ERR_ALIGN, "open: misaligned output");
    SPDZ_FIELD_SWITCH(ctx->field, {
        using T = typename F::T;
        MulArgs<F> a{};
        a.xv = (const T *)x->val; a.xm = (const T *)x->mac; a.xs = x->stride;
        a.opened = (T *)out_dev; a.N = N; a.ds = ctx->ds; a.base = (uint64_t)ctx->opened;
        // 16-byte vectors (2 p61 or 4 p32 elements) when every row is aligned
        const size_t eb = sizeof(T);
        constexpr int VV = std::is_same_v<F, F61> ? 2 : std::is_same_v<F, F32> ? 4 : 1;
        const bool vec = VV > 1 && buf_vec_ok(x, eb) && ((uintptr_t)out_dev % 16 == 0);
        SPDZ_NP_SWITCH(ctx->n, {
            if (vec) {
                auto kern = k_open<F, NP, VV>;
                kern<<<grid_for(ctx, (const void *)kern, 256, 0, (N + VV - 1) / VV), 256, 0, ctx->stream>>>(a);
            } else {
                auto kern = k_open<F, NP, 1>;
                kern<<<grid_for(ctx, (const void *)kern, 256, 0, N), 256, 0, ctx->stream>>>(a);
            }
        });
    });
    if ((rc = check_launch(ctx, "open"))) return rc;
    ctx->opened += N;
    return SPDZ_OK;
}

int spdz_field_op(spdz_ctx *ctx, int op, const void *a_dev, const void *b_dev, void *out_dev, int64_t N) {
    if (!ctx) return SPDZ_ERR_ARG;
    if (N < 0 || !a_dev || !b_dev || !out_dev || (op != SPDZ_OP_ADD && op != SPDZ_OP_SUB && op != SPDZ_OP_CMUL))
        return set_err(ctx, SPDZ_ERR_ARG, "field_op: bad argument");
    if (N == 0) return SPDZ_OK;
    SPDZ_FIELD_SWITCH(ctx->field, {
        using T = typename F::T;
        auto kern = k_field_op<F>;
        kern<<<grid_for(ctx, (const void *)kern, 256, 0, N), 256, 0, ctx->stream>>>(op, (const T *)a_dev,
                                                                                    (const T *)b_dev, (T *)out_dev, N);
    });
    return check_launch(ctx, "field_op");
}

}  // extern "C"
