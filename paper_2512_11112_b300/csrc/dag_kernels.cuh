// dag_kernels.cuh -- device code of layered-circuit execution, shared by the
// circuit executor (dag.cu) and the serving engine (serve.cu): gate records,
// the per-gate mask/open/combine or linear step, cp.async staging of a
// gate's layer-independent operands, the bounded device-wide barrier and
// the per-layer, fused and cluster kernels.
#pragma once
#include "beaver.cuh"
#include "dag.cuh"

namespace spdz {

template <class F> __device__ __forceinline__ typename F::T ld_cg(const typename F::T *p);
template <> __device__ __forceinline__ F61::T ld_cg<F61>(const F61::T *p) {
    return __ldcg(reinterpret_cast<const unsigned long long *>(p));
}
template <> __device__ __forceinline__ F127::T ld_cg<F127>(const F127::T *p) {
    ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(p));
    return {v.x, v.y};
}
template <class F> __device__ __forceinline__ typename F::T ld_cs(const typename F::T *p);
template <> __device__ __forceinline__ F61::T ld_cs<F61>(const F61::T *p) {
    return __ldcs(reinterpret_cast<const unsigned long long *>(p));
}
template <> __device__ __forceinline__ F127::T ld_cs<F127>(const F127::T *p) {
    ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2 *>(p));
    return {v.x, v.y};
}

enum : int { C_MUL = 0, C_ADD = 1, C_SUB = 2, C_CMUL = 3, C_CADD = 4 };

__device__ __forceinline__ int class_of(const LayerRow &L, int32_t r) {
    return r < L.s[1] ? C_MUL : r < L.s[2] ? C_ADD : r < L.s[3] ? C_SUB : r < L.s[4] ? C_CMUL : C_CADD;
}

__device__ __forceinline__ LayerRow load_row(const LayerRow *lay, int l) {
    const int4 *p = reinterpret_cast<const int4 *>(lay + l);
    int4 a = __ldg(p), b = __ldg(p + 1);
    LayerRow L;
    L.s[0] = a.x; L.s[1] = a.y; L.s[2] = a.z; L.s[3] = a.w;
    L.s[4] = b.x; L.s[5] = b.y; L.mulbase = b.z; L.pad = b.w;
    return L;
}

template <class F> struct DagArgs {
    using T = typename F::T;
    const uint4 *rec;                       // {in0, in1, out, 0} in execution order
    const T *kc;                            // constants in record order (CMUL/CADD records)
    const LayerRow *lay;                    // [depth]
    T *wv, *wm;
    int64_t ws;
    const T *tp[6];                         // triple rows: a, gamma(a), b, gamma(b), c, gamma(c)
    int64_t ts[6];                          // their party strides
    DevState *ds;
    int32_t l0, l1;                         // layers [l0, l1)
    int32_t r0, r1;                         // per-layer kernels: records [r0, r1) of layer l0
    uint32_t bar_base;                      // fused: barrier arrivals before this launch
    uint64_t spin_ns;
    int32_t record_ts;
    uint32_t extra_arrivals;                // testing: arrivals that never come
};

// Operands of one gate that do not depend on earlier layers: its record,
// its triple shares (MUL) or its constant (CMUL/CADD).
template <class F, int NP> struct GateIn {
    using T = typename F::T;
    uint4 rec;
    T tri[6][NP];
    T k;
};

template <class F, int NP>
__device__ __forceinline__ void gate_load_direct(const DagArgs<F> &a, const LayerRow &L, int32_t r, int cls,
                                                 uint64_t tri_base, GateIn<F, NP> &g) {
    g.rec = __ldg(&a.rec[r]);
    if (cls == C_MUL) {
        const int64_t t = (int64_t)tri_base + L.mulbase + (r - L.s[0]);
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int i = 0; i < NP; ++i) g.tri[k][i] = ld_cs<F>(a.tp[k] + i * a.ts[k] + t);
    } else if (cls >= C_CMUL) {
        g.k = F::ld(a.kc + r);
    }
}

// Masks, opens, combines (MUL) or applies the linear gate, reading the wire
// operands (written by earlier layers: L2, never L1) and storing the output.
template <class F, int NP, class TRI>
__device__ __forceinline__ void gate_exec(const DagArgs<F> &a, const LayerRow &L, int32_t r, int cls, uint4 rec,
                                          typename F::T kconst, const TRI &tri, uint64_t key,
                                          const typename F::T (&alpha)[NP], typename F::T (&acc)[NP + 1]) {
    using T = typename F::T;
    const uint32_t in0 = rec.x, in1 = rec.y, out = rec.z;
    if (cls == C_MUL) {
        T x[NP], gx[NP], y[NP], gy[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            x[i] = ld_cg<F>(a.wv + i * a.ws + in0);
            y[i] = ld_cg<F>(a.wv + i * a.ws + in1);
            gx[i] = ld_cg<F>(a.wm + i * a.ws + in0);
            gy[i] = ld_cg<F>(a.wm + i * a.ws + in1);
        }
        T z[NP], gz[NP];
        const uint64_t rank = (uint64_t)(L.mulbase + (r - L.s[0]));
        beaver_math_src<F, NP>(x, gx, y, gy, tri, alpha, key, 2 * rank, acc, z, gz);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            F::st(a.wv + i * a.ws + out, z[i]);
            F::st(a.wm + i * a.ws + out, gz[i]);
        }
    } else {
        const int op = cls == C_ADD ? SPDZ_OP_ADD : cls == C_SUB ? SPDZ_OP_SUB : cls == C_CMUL ? SPDZ_OP_CMUL : SPDZ_OP_CADD;
        const bool binary = cls <= C_SUB;
        const T k = binary ? F::zero() : kconst;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const T x = ld_cg<F>(a.wv + i * a.ws + in0), gx = ld_cg<F>(a.wm + i * a.ws + in0);
            T y = F::zero(), gy = F::zero();
            if (binary) {
                y = ld_cg<F>(a.wv + i * a.ws + in1);
                gy = ld_cg<F>(a.wm + i * a.ws + in1);
            }
            const T kal = cls == C_CADD ? F::mul(alpha[i], k) : F::zero();
            T z, gz;
            linear_math<F>(op, i, x, gx, y, gy, k, kal, z, gz);
            F::st(a.wv + i * a.ws + out, z);
            F::st(a.wm + i * a.ws + out, gz);
        }
    }
}

// ----------------------------------------------- asynchronous prefetch
// Each thread stages the layer-independent operands of its next gate in its
// own shared-memory slots (structure of arrays across the block, so the
// accesses are conflict-free) with cp.async; nothing is shared between
// threads, so only the thread's own wait is needed before use.
__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    if (bytes == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class F, int NP> struct Stage {
    using T = typename F::T;
    uint4 *rec;      // [B]
    T *tri;          // [6*NP][B]
    T *k;            // [B]
    int B;
    __device__ __forceinline__ void init(unsigned char *base, int block) {
        B = block;
        rec = reinterpret_cast<uint4 *>(base);
        tri = reinterpret_cast<T *>(base + sizeof(uint4) * block);
        k = tri + 6 * NP * block;
    }
    static constexpr size_t bytes_per_thread() { return sizeof(uint4) + (6 * NP + 1) * sizeof(T); }
};

template <class F, int NP>
__device__ __forceinline__ void stage_issue(const DagArgs<F> &a, const LayerRow &L, int32_t r, int cls,
                                            uint64_t tri_base, const Stage<F, NP> &st) {
    using T = typename F::T;
    const int t = threadIdx.x;
    cp_async(&st.rec[t], &a.rec[r], 16);
    if (cls == C_MUL) {
        const int64_t ti = (int64_t)tri_base + L.mulbase + (r - L.s[0]);
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
            for (int i = 0; i < NP; ++i) cp_async(&st.tri[(k * NP + i) * st.B + t], a.tp[k] + i * a.ts[k] + ti, (int)sizeof(T));
    } else if (cls >= C_CMUL) {
        cp_async(&st.k[t], a.kc + r, (int)sizeof(T));
    }
    cp_async_commit();
}

// Direct and staged sources of a gate's triple shares.
template <class F, int NP> struct TriRegs {
    const GateIn<F, NP> &g;
    __device__ __forceinline__ typename F::T operator()(int k, int i) const { return g.tri[k][i]; }
};
template <class F, int NP> struct TriSmem {
    const typename F::T *base;   // st.tri + threadIdx.x
    int B;
    __device__ __forceinline__ typename F::T operator()(int k, int i) const { return base[(k * NP + i) * B]; }
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Device-wide barrier over the CTAs of one launch.  Arrivals are counted on
// a run-wide counter with a release reduction (no returned value to wait
// for); thread 0 polls with acquire loads.  The wait is bounded by spin_ns,
// after which the CTA records a timeout, raises the abort flag and returns
// false (every later barrier of the run then returns false at once).
__device__ __forceinline__ bool grid_barrier(DevState *ds, unsigned int target, uint64_t spin_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ds->bar_count) : "memory");
        const unsigned long long t0 = gtimer();
        while (true) {
            unsigned int v, ab;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&ds->bar_count) : "memory");
            if ((int)(v - target) >= 0) break;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(ab) : "l"(&ds->bar_abort) : "memory");
            if (ab) { ok = 0; break; }
            if (gtimer() - t0 > spin_ns) {
                atomicOr(&ds->err_flags, ERR_TIMEOUT);
                atomicExch(&ds->bar_abort, 1u);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Start of a run: the triple cursor the run consumes from, fresh barrier
// counters and error flags.  Its argument is updated before every replay of
// a captured run.
static __global__ void k_run_begin(DevState *ds, uint64_t tri_base) {
    ds->tri_cursor = tri_base;
    ds->bar_count = 0;
    ds->bar_abort = 0;
    ds->err_flags = 0;
}

// Per-layer form: records [r0, r1) of layer l0 (one gate class range).
template <class F, int NP>
__global__ void __launch_bounds__(256) k_dag_segment(DagArgs<F> a) {
    using T = typename F::T;
    const uint64_t key = a.ds->key, tri_base = a.ds->tri_cursor;
    T alpha[NP], acc[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
    const LayerRow L = load_row(a.lay, a.l0);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = a.r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < a.r1; r += stride) {
        const int cls = class_of(L, (int32_t)r);
        GateIn<F, NP> g;
        gate_load_direct<F, NP>(a, L, (int32_t)r, cls, tri_base, g);
        gate_exec<F, NP>(a, L, (int32_t)r, cls, g.rec, g.k, TriRegs<F, NP>{g}, key, alpha, acc);
    }
    block_accumulate<F, NP + 1>(acc, a.ds->acc);
}

// Fused form: layers [l0, l1) in one persistent launch.  Each thread owns
// gates tid, tid + nthreads, ... of every layer (tid: see below); the
// operands of its first gate of layer l+1 are staged in shared memory while
// the CTA waits at the barrier that ends layer l.
// Cluster-scope barrier between layers of a group run by one thread-block
// cluster: a hardware barrier (every CTA of a cluster is co-resident, so it
// cannot wait forever); release/acquire order the wire writes at cluster
// scope, which covers global memory read through L2.
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned int cluster_rank() {
    unsigned int r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

template <class F, int NP, bool CLUSTER>
__device__ __forceinline__ void dag_fused_body(const DagArgs<F> &a) {
    using T = typename F::T;
    extern __shared__ __align__(16) unsigned char smem[];
    Stage<F, NP> st;
    st.init(smem, blockDim.x);
    const uint64_t key = a.ds->key, tri_base = a.ds->tri_cursor;
    T alpha[NP], acc[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
    // 32-gate tiles are dealt round-robin over the CTAs (tile t -> CTA
    // t mod G, then warp), so even a narrow layer spreads over every SM while
    // each warp still reads 32 consecutive records and triples
    const int32_t cta = CLUSTER ? (int32_t)cluster_rank() : (int32_t)blockIdx.x;
    const int32_t tid = 32 * (cta + gridDim.x * (threadIdx.x >> 5)) + (threadIdx.x & 31);
    const int32_t nthreads = gridDim.x * blockDim.x;
    const bool stamp = a.record_ts && cta == 0 && threadIdx.x == 0;
    if (stamp) a.ds->layer_ts[a.l0] = gtimer();
    LayerRow L = load_row(a.lay, a.l0);
    int32_t r = L.s[0] + tid;
    bool staged = r < L.s[5];
    if (staged) stage_issue<F, NP>(a, L, r, class_of(L, r), tri_base, st);
    bool ok = true;
    unsigned int nb = 0;
    for (int32_t l = a.l0; l < a.l1; ++l) {
        if (ok) {
            if (staged) {
                const int cls = class_of(L, r);
                cp_async_wait_all();
                const uint4 rec = st.rec[threadIdx.x];
                const T kk = cls >= C_CMUL ? st.k[threadIdx.x] : F::zero();
                gate_exec<F, NP>(a, L, r, cls, rec, kk, TriSmem<F, NP>{st.tri + threadIdx.x, st.B}, key, alpha, acc);
            }
            for (int32_t q = r + nthreads; q < L.s[5]; q += nthreads) {
                const int cls = class_of(L, q);
                GateIn<F, NP> g;
                gate_load_direct<F, NP>(a, L, q, cls, tri_base, g);
                gate_exec<F, NP>(a, L, q, cls, g.rec, g.k, TriRegs<F, NP>{g}, key, alpha, acc);
            }
        }
        staged = false;
        if (l + 1 < a.l1) {
            L = load_row(a.lay, l + 1);
            r = L.s[0] + tid;
            staged = ok && r < L.s[5];
            if (staged) stage_issue<F, NP>(a, L, r, class_of(L, r), tri_base, st);
        }
        if (l + 1 < a.l1 || a.record_ts) {
            if constexpr (CLUSTER) {
                cluster_barrier();
            } else {
                ++nb;
                ok = grid_barrier(a.ds, a.bar_base + nb * gridDim.x + a.extra_arrivals, a.spin_ns) && ok;
            }
            if (stamp) a.ds->layer_ts[l + 1] = gtimer();
        }
    }
    cp_async_wait_all();
    block_accumulate<F, NP + 1>(acc, a.ds->acc);
}

// Two CTAs of 256 threads per SM for p61 (128 registers); p127 operands are
// twice as wide, so its kernel is bounded for one CTA per SM instead.
template <class F, int NP>
__global__ void __launch_bounds__(256, 2) k_dag_fused(DagArgs<F> a) {
    dag_fused_body<F, NP, false>(a);
}
template <class F, int NP>
__global__ void __launch_bounds__(256, 1) k_dag_fused_wide(DagArgs<F> a) {
    dag_fused_body<F, NP, false>(a);
}
// One cluster of CTAs for a group of narrow layers (grid = the cluster).
template <class F, int NP>
__global__ void __launch_bounds__(256, 1) k_dag_cluster(DagArgs<F> a) {
    dag_fused_body<F, NP, true>(a);
}

template <class F, int NP> constexpr size_t fused_smem(int block) {
    return Stage<F, NP>::bytes_per_thread() * (size_t)block;
}

}  // namespace spdz
