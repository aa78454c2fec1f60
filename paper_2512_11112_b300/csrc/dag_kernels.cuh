// dag_kernels.cuh -- device code of layered-circuit execution, shared by the
// circuit executor (dag.cu) and the serving engine (serve.cu): gate records,
// the per-gate mask/open/combine or linear step, cp.async staging of a
// gate's layer-independent operands, the bounded device-wide barrier and
// the per-layer, fused and cluster kernels.
#pragma once
#include <cstddef>
#include "beaver.cuh"
#include "check.cuh"
#include "dag.cuh"

namespace spdz {

template <class F> __device__ __forceinline__ typename F::T ld_cg(const typename F::T *p);
template <> __device__ __forceinline__ F61::T ld_cg<F61>(const F61::T *p) {
    return __ldcg(reinterpret_cast<const unsigned long long *>(p));
}
template <> __device__ __forceinline__ F32::T ld_cg<F32>(const F32::T *p) { return __ldcg(p); }
template <> __device__ __forceinline__ F127::T ld_cg<F127>(const F127::T *p) {
    ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(p));
    return {v.x, v.y};
}
template <class F> __device__ __forceinline__ typename F::T ld_cs(const typename F::T *p);
template <> __device__ __forceinline__ F61::T ld_cs<F61>(const F61::T *p) {
    return __ldcs(reinterpret_cast<const unsigned long long *>(p));
}
template <> __device__ __forceinline__ F32::T ld_cs<F32>(const F32::T *p) { return __ldcs(p); }
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
    uint64_t *mir;                          // tagged: wire-major copy [wires][2*NP]
    int64_t n_in;                           // tagged: input wires copied into it
    uint32_t poll_ns;                       // tagged: first sleep between operand polls
    uint32_t slack;                         // tagged: arrivals a layer barrier does not wait for
    int32_t test_unwritten_tag;             // testing (tagged): operands wait for a tag never written
    uint64_t wbase;                         // tagged group starting after layer 0: wires below this
                                            // were finished by earlier groups (read party-major)
    int32_t final_check;                    // tagged: the last CTA runs the run's MAC check
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
// L2 eviction priorities: data read once (triples, records, constants, the
// party-major output rows) goes first; the tagged copy, whose wires later
// layers gather from anywhere in the run, goes last.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    const uint64_t pol = l2_evict_first();
    if (bytes == 16)
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "l"(pol) : "memory");
    else if (bytes == 8)
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;" ::"r"(s), "l"(gmem), "l"(pol) : "memory");
    else
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "l"(pol) : "memory");
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
// RELAXED: arrival and polls carry no ordering (no fence waits for the CTA's
// stores); for data that validates itself (tagged operands).
template <bool RELAXED = false>
__device__ __forceinline__ bool grid_barrier(DevState *ds, unsigned int target, uint64_t spin_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if constexpr (RELAXED)
            asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(&ds->bar_count) : "memory");
        else
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ds->bar_count) : "memory");
        const unsigned long long t0 = gtimer();
        while (true) {
            unsigned int v, ab;
            if constexpr (RELAXED)
                asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&ds->bar_count) : "memory");
            else
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

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// The relaxed barrier in two halves, so that a CTA can work between its
// arrival and its wait.  Arrival: every thread of the CTA has finished the
// layer; thread 0 counts the CTA (no ordering, as grid_barrier<true>).
__device__ __forceinline__ void grid_arrive_relaxed(DevState *ds) {
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(&ds->bar_count) : "memory");
}
// Wait: thread 0 polls until `target` arrivals (bounded by spin_ns, as in
// grid_barrier), then the CTA goes on together.  The arrival count and the
// abort flag are adjacent words, read by one 8-byte load per poll (one L2
// round trip, not two in a row); the time bound is read every 16th poll.
// (Four polls in flight at once, 30 ns apart, were slower: 139 -> 144 us
// per run of the benchmark circuit.)
__device__ __forceinline__ bool grid_wait_relaxed(DevState *ds, unsigned int target, uint64_t spin_ns) {
    static_assert(offsetof(DevState, bar_abort) == offsetof(DevState, bar_count) + 4, "count, abort adjacent");
    static_assert(offsetof(DevState, bar_count) % 8 == 0, "count 8-byte aligned");
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long t0 = gtimer();
        for (unsigned int it = 1;; ++it) {
            unsigned int v, ab;
            asm volatile("ld.relaxed.gpu.global.v2.u32 {%0, %1}, [%2];" : "=r"(v), "=r"(ab) : "l"(&ds->bar_count) : "memory");
            if ((int)(v - target) >= 0) break;
            if (ab) { ok = 0; break; }
            if ((it & 15) == 0 && gtimer() - t0 > spin_ns) {
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
static __global__ void k_run_begin(DevState *ds, uint64_t tri_base, uint32_t df_tag) {
    // a tagged kernel launched after this one may start its CTAs now: it
    // waits for this grid's writes (griddepcontrol.wait) before reading them
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    ds->tri_cursor = tri_base;
    ds->bar_count = 0;
    ds->bar_abort = 0;
    ds->err_flags = 0;
    ds->df_tag = df_tag;
    ds->run_done = 0;
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

// ---------------------------------------------- tagged execution (p61 only)
// A stored p61 share is below 2^61, so the top three bits of its 64-bit word
// are free.  In tagged mode every gate also stores its output shares -- the
// NP values, then the NP MACs -- into a wire-major copy of the wires with the
// run's tag (1..7) in those bits.  An aligned 8-byte store is observed whole
// or not at all, so a reader that finds the tag in all 2*NP words of an
// operand holds that operand's value of this run, whatever order the stores
// became visible in: no fence is needed between a gate's stores and their
// readers.  Tag 0 never matches; the host zeroes the copy before every 7th
// run of a circuit, so within the 7 runs that follow each word holds either
// nothing or this cycle's tags, all different.
constexpr int DF_TAG_SHIFT = 61;

__device__ __forceinline__ void df_st2(uint64_t *p, uint64_t a, uint64_t b) {
    asm volatile("st.relaxed.gpu.global.L2::cache_hint.v2.u64 [%0], {%1, %2}, %3;" ::"l"(p), "l"(a), "l"(b),
                 "l"(l2_evict_last()) : "memory");
}
__device__ __forceinline__ void df_ld2(const uint64_t *p, uint64_t &a, uint64_t &b) {
    asm volatile("ld.relaxed.gpu.global.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;" : "=l"(a), "=l"(b) : "l"(p),
                 "l"(l2_evict_last()) : "memory");
}
// A party-major output share, read by nobody during a tagged run.
__device__ __forceinline__ void st_first(uint64_t *p, uint64_t v) {
    asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(l2_evict_first()) : "memory");
}

// Issues the loads of the operand record of wire w (its first use waits).
template <int NP>
__device__ __forceinline__ void df_issue(const uint64_t *mir, uint32_t w, uint64_t (&v)[2 * NP]) {
    const uint64_t *p = mir + (size_t)w * (2 * NP);
#pragma unroll
    for (int k = 0; k < NP; ++k) df_ld2(p + 2 * k, v[2 * k], v[2 * k + 1]);
}
// True when every word of a loaded record carries `tag`.
template <int NP>
__device__ __forceinline__ bool df_tagged(const uint64_t (&v)[2 * NP], uint64_t tag) {
    uint64_t bad = 0;
#pragma unroll
    for (int k = 0; k < 2 * NP; ++k) bad |= (v[k] >> DF_TAG_SHIFT) ^ tag;
    return bad == 0;
}
// Reads the operand record of wire w; true when every word carries `tag`.
template <int NP>
__device__ __forceinline__ bool df_fetch(const uint64_t *mir, uint32_t w, uint64_t tag, uint64_t (&v)[2 * NP]) {
    df_issue<NP>(mir, w, v);
    return df_tagged<NP>(v, tag);
}

// Slow path of an operand wait: one sleep (doubling from poll_ns up to 16x),
// and every 8th call a look at the abort flag and at the bound of the wait
// (on timeout the run is marked failed and aborted).  False when the wait
// must give up.
__device__ __forceinline__ bool df_backoff(DevState *ds, uint64_t spin_ns, unsigned long long t0, unsigned int it,
                                           uint32_t poll_ns) {
    __nanosleep(poll_ns << min(it - 1u, 4u));
    if ((it & 7) != 0) return true;
    if (ld_relaxed_u32(&ds->bar_abort)) return false;
    if (gtimer() - t0 > spin_ns) {
        atomicOr(&ds->err_flags, ERR_TIMEOUT);
        atomicExch(&ds->bar_abort, 1u);
        return false;
    }
    return true;
}

__device__ __forceinline__ uint64_t df_ld1(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// The operand record of wire w once it carries `tag`, after a first read
// that did not (bounded wait).  While waiting, only the record's first word
// is polled (one sector); the whole record is read again once that word
// carries the tag.
template <int NP>
__device__ __forceinline__ bool df_wait(const DagArgs<F61> &a, uint32_t w, uint64_t tag, uint64_t (&v)[2 * NP]) {
    const uint64_t *p = a.mir + (size_t)w * (2 * NP);
    const unsigned long long t0 = gtimer();
    unsigned int it = 0;
    while (true) {
        if (!df_backoff(a.ds, a.spin_ns, t0, ++it, a.poll_ns)) return false;
        if ((df_ld1(p) >> DF_TAG_SHIFT) == tag && df_fetch<NP>(a.mir, w, tag, v)) return true;
    }
}

template <int NP>
__device__ __forceinline__ void df_store(uint64_t *mir, uint32_t w, uint64_t tag, const uint64_t (&z)[NP],
                                         const uint64_t (&gz)[NP]) {
    uint64_t t[2 * NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        t[i] = z[i] | (tag << DF_TAG_SHIFT);
        t[NP + i] = gz[i] | (tag << DF_TAG_SHIFT);
    }
    uint64_t *p = mir + (size_t)w * (2 * NP);
#pragma unroll
    for (int k = 0; k < NP; ++k) df_st2(p + 2 * k, t[2 * k], t[2 * k + 1]);
}

// An input wire's shares from the caller's party-major wires (written
// before the run, read-only during it), as a tagged-copy record.
template <int NP>
__device__ __forceinline__ void df_input(const DagArgs<F61> &a, uint32_t w, uint64_t (&v)[2 * NP]) {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        v[i] = __ldg(reinterpret_cast<const unsigned long long *>(a.wv + i * a.ws + w));
        v[NP + i] = __ldg(reinterpret_cast<const unsigned long long *>(a.wm + i * a.ws + w));
    }
}

// One gate in tagged mode: fetch (and if needed wait for) the operands,
// compute, store the output shares (caller's party-major wires, and the
// tagged copy).  inputs: every operand is an input wire (the first layer),
// read from the caller's wires with no tag to wait for.
template <int NP, class TRI>
__device__ __forceinline__ bool df_gate(const DagArgs<F61> &a, const LayerRow &L, int32_t r, int cls, uint4 rec,
                                        uint64_t kconst, const TRI &tri, uint64_t key, uint64_t tag, uint64_t wtag,
                                        const uint64_t (&alpha)[NP], uint64_t (&acc)[NP + 1], bool inputs) {
    using F = F61;
    const bool binary = cls <= C_SUB;
    uint64_t u[2 * NP], v[2 * NP];
    if (inputs) {
        df_input<NP>(a, rec.x, u);
        if (binary) df_input<NP>(a, rec.y, v);
    } else {
        // both operands' loads in flight at once; a wait only for a record
        // whose first read missed its tag.  Wires finished before the group
        // (below wbase) are read from the party-major wires, untagged.
        const bool xo = rec.x < a.wbase, yo = rec.y < a.wbase;
        if (xo) df_input<NP>(a, rec.x, u);
        else df_issue<NP>(a.mir, rec.x, u);
        if (binary) {
            if (yo) df_input<NP>(a, rec.y, v);
            else df_issue<NP>(a.mir, rec.y, v);
        }
        if (!xo && !df_tagged<NP>(u, wtag) && !df_wait<NP>(a, rec.x, wtag, u)) return false;
        if (binary && !yo && !df_tagged<NP>(v, tag) && !df_wait<NP>(a, rec.y, tag, v)) return false;
    }
    uint64_t z[NP], gz[NP];
    if (cls == C_MUL) {
        uint64_t x[NP], gx[NP], y[NP], gy[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            x[i] = u[i] & F::P;
            gx[i] = u[NP + i] & F::P;
            y[i] = v[i] & F::P;
            gy[i] = v[NP + i] & F::P;
        }
        const uint64_t rank = (uint64_t)(L.mulbase + (r - L.s[0]));
        beaver_math_src<F, NP>(x, gx, y, gy, tri, alpha, key, 2 * rank, acc, z, gz);
    } else {
        const int op = cls == C_ADD ? SPDZ_OP_ADD : cls == C_SUB ? SPDZ_OP_SUB : cls == C_CMUL ? SPDZ_OP_CMUL : SPDZ_OP_CADD;
        const uint64_t k = binary ? 0 : kconst;
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const uint64_t y = binary ? v[i] & F::P : 0, gy = binary ? v[NP + i] & F::P : 0;
            const uint64_t kal = cls == C_CADD ? F::mul(alpha[i], k) : 0;
            linear_math<F>(op, i, u[i] & F::P, u[NP + i] & F::P, y, gy, k, kal, z[i], gz[i]);
        }
    }
    const uint32_t out = rec.z;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        st_first(a.wv + i * a.ws + out, z[i]);
        st_first(a.wm + i * a.ws + out, gz[i]);
    }
    df_store<NP>(a.mir, out, tag, z, gz);
    return true;
}

// A thread's gates of one layer: its staged first gate, then the rest with
// direct loads.  False when an operand wait gave up.
template <int NP>
__device__ __forceinline__ bool df_layer(const DagArgs<F61> &a, const LayerRow &L, int32_t r, bool staged,
                                         int32_t nthreads, const Stage<F61, NP> &st, uint64_t tri_base, uint64_t key,
                                         uint64_t tag, uint64_t wtag, const uint64_t (&alpha)[NP],
                                         uint64_t (&acc)[NP + 1], bool inputs) {
    using F = F61;
    bool ok = true;
    if (staged) {
        const int cls = class_of(L, r);
        cp_async_wait_all();
        const uint4 rec = st.rec[threadIdx.x];
        const uint64_t kk = cls >= C_CMUL ? st.k[threadIdx.x] : 0;
        ok = df_gate<NP>(a, L, r, cls, rec, kk, TriSmem<F, NP>{st.tri + threadIdx.x, st.B}, key, tag, wtag, alpha,
                         acc, inputs);
    }
    for (int32_t q = r + nthreads; ok && q < L.s[5]; q += nthreads) {
        const int cls = class_of(L, q);
        GateIn<F, NP> g;
        gate_load_direct<F, NP>(a, L, q, cls, tri_base, g);
        ok = df_gate<NP>(a, L, q, cls, g.rec, g.k, TriRegs<F, NP>{g}, key, tag, wtag, alpha, acc, inputs);
    }
    return ok;
}

// The tagged form of the fused kernel (p61), over layers [l0, l1) (the whole
// circuit, or one group of a plan): gates read their operands from
// the tagged copy (one wire's shares of every party in 2*NP consecutive
// words, a third of the sectors of the party-major gathers) and validate
// them by tag, so the barrier between layers needs no fence: it only keeps
// the CTAs in step (few operands are still in flight when a layer starts,
// and their readers re-poll one word); with a slack it also lets a CTA start
// a layer before the last few CTAs have finished the one before, whose
// operands the tags then cover.  A thread's first gate of the next layer is
// staged between the CTA's arrival at the barrier and its wait, off the
// layer's critical path.
template <int NP>
__global__ void __launch_bounds__(256, 2) k_dag_tagged(DagArgs<F61> a) {
    using F = F61;
    // launched as a programmatic dependent of the kernel before it: wait for
    // that grid's writes (the run's state) before anything reads them
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem[];
    Stage<F, NP> st;
    st.init(smem, blockDim.x);
    const uint64_t key = a.ds->key, tri_base = a.ds->tri_cursor;
    const uint64_t tag = a.ds->df_tag;
    uint64_t alpha[NP], acc[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = 0;
    const int32_t nthreads = gridDim.x * blockDim.x;
    const int32_t tid = 32 * ((int32_t)blockIdx.x + gridDim.x * (threadIdx.x >> 5)) + (threadIdx.x & 31);
    const bool stamp = a.record_ts && blockIdx.x == 0 && threadIdx.x == 0;
    if (stamp) a.ds->layer_ts[a.l0] = gtimer();
    LayerRow L = load_row(a.lay, a.l0);
    int32_t r = L.s[0] + tid;
    bool staged = r < L.s[5];
    if (staged) stage_issue<F, NP>(a, L, r, class_of(L, r), tri_base, st);
    // The inputs into the tagged copy, for the layers after the first (whose
    // gates read them from the caller's wires): when at least a quarter of
    // the threads have no gate in the first layer, those copy them at once;
    // otherwise every thread copies after its first-layer gates.  Either way
    // before the first barrier.
    const int64_t w0 = (int64_t)L.s[5] - L.s[0];
    const bool idle_copy = nthreads - w0 >= nthreads / 4;
    const bool copy_first = idle_copy && tid >= w0;
    const int64_t cstart = idle_copy ? tid - w0 : tid, cstride = idle_copy ? nthreads - w0 : nthreads;
    auto copy_inputs = [&]() {
        for (int64_t w = cstart; w < a.n_in; w += cstride) {
            uint64_t z[NP], gz[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                // (canonical shares are below 2^61; the mask keeps a malformed
                // input from reaching the tag bits)
                z[i] = ld_cs<F>(a.wv + i * a.ws + w) & F::P;
                gz[i] = ld_cs<F>(a.wm + i * a.ws + w) & F::P;
            }
            df_store<NP>(a.mir, (uint32_t)w, tag, z, gz);
        }
    };
    if (copy_first) copy_inputs();
    bool ok = tag != 0;
    if (!ok && threadIdx.x == 0 && blockIdx.x == 0) atomicOr(&a.ds->err_flags, ERR_TIMEOUT);
    unsigned int nb = 0;
    for (int32_t l = a.l0; l < a.l1; ++l) {
        // testing: first operands after the first layer wait for a tag nobody
        // writes (tags are 1..7; the three tag bits cannot hold 8)
        const uint64_t wtag = (a.test_unwritten_tag && l > a.l0) ? 8u : tag;
        if (ok) ok = df_layer<NP>(a, L, r, staged, nthreads, st, tri_base, key, tag, wtag, alpha, acc, l == a.l0);
        if (l == a.l0 && !idle_copy) copy_inputs();
        staged = false;
        const bool more = l + 1 < a.l1;
        if (more || a.record_ts) {
            ++nb;
            grid_arrive_relaxed(a.ds);
            if (more) {
                L = load_row(a.lay, l + 1);
                r = L.s[0] + tid;
                staged = ok && r < L.s[5];
                if (staged) stage_issue<F, NP>(a, L, r, class_of(L, r), tri_base, st);
            }
            ok = grid_wait_relaxed(a.ds, a.bar_base + nb * gridDim.x - a.slack, a.spin_ns) && ok;
            if (stamp) a.ds->layer_ts[l + 1] = gtimer();
        }
    }
    cp_async_wait_all();
    block_accumulate<F, NP + 1>(acc, a.ds->acc);
    if (!a.final_check) return;
    // the last CTA to finish runs the run's MAC check (its accumulator
    // atomics, like every CTA's, are ordered before its count by the fence)
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&a.ds->run_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        check_epoch<F, NP>(a.ds, 1);
    }
}

template <int NP> constexpr size_t tagged_smem(int block) {
    return Stage<F61, NP>::bytes_per_thread() * (size_t)block;
}

}  // namespace spdz
