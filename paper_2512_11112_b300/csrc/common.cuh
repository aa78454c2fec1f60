// common.cuh -- context state, dispatch and reduction helpers shared by the
// kernels of the SPDZ library.
#pragma once
#include <cstring>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "spdz.h"
#include "field.cuh"
#include "prg.cuh"

namespace spdz {

constexpr int MAXP = SPDZ_MAX_PARTIES;

// Device-resident state of one context.  Everything a kernel needs across
// launches lives here, so that captured CUDA graphs can be replayed: the
// MAC-check key of the current epoch, the random-linear-combination
// accumulators, the triple cursor of circuit runs and the barrier counters of
// the fused circuit kernel.
struct DevState {
    uint64_t check_seed;
    uint64_t epoch;
    uint64_t key;                      // coefficient key of the current epoch
    uint64_t tri_cursor;               // triple cursor used by circuit runs
    // RLC accumulators: acc[0] = A = sum r_j v_j, acc[1+i] = S_i; each an
    // exact 192-bit integer (three words; the fourth is padding)
    unsigned long long acc[MAXP + 1][4];
    uint64_t sig_run[MAXP][2];         // sigma summed over partial checks of the epoch
    uint32_t partial_fail;             // a partial check of this epoch failed
    uint32_t err_flags;                // bit 0: a device wait timed out
    uint64_t alpha[MAXP][2];           // alpha shares
    // result of the last completed check (read back by the host)
    uint64_t res_sigma[MAXP][2];
    uint32_t res_passed;
    uint32_t res_epoch;
    uint64_t res_A[2];
    uint64_t res_S[MAXP][2];
    // grid barrier of the fused circuit kernel: arrivals counted over a run
    unsigned int bar_count;
    unsigned int bar_abort;            // set when a barrier wait timed out
    unsigned int df_tag;               // tag of the current tagged-mode run (1..7; 0: none)
    unsigned int run_done;             // CTAs of a tagged run that have finished
    unsigned int bar_pad[60];
    // per-layer timestamps written by the fused circuit kernel (globaltimer ns)
    unsigned long long layer_ts[1024];
};

enum : uint32_t { ERR_TIMEOUT = 1u };

template <class F> __device__ __forceinline__ typename F::T load_alpha(const DevState *ds, int i);
template <> __device__ __forceinline__ F61::T load_alpha<F61>(const DevState *ds, int i) {
    return ds->alpha[i][0];
}
template <> __device__ __forceinline__ F32::T load_alpha<F32>(const DevState *ds, int i) {
    return (F32::T)ds->alpha[i][0];
}
template <> __device__ __forceinline__ F127::T load_alpha<F127>(const DevState *ds, int i) {
    return {ds->alpha[i][0], ds->alpha[i][1]};
}

// ----------------------------------------------------------- accumulators
// Exact multi-word integer accumulation with 64-bit atomics: each add's
// carry is detected from the returned old value, so the sum is exact in any
// order.
__device__ __forceinline__ void acc_add(unsigned long long *acc, F61::T v) {
    unsigned long long old = atomicAdd(&acc[0], (unsigned long long)v);
    if (old + v < old) atomicAdd(&acc[1], 1ull);
}
__device__ __forceinline__ void acc_add(unsigned long long *acc, F32::T v) {
    acc_add(acc, (F61::T)v);
}
__device__ __forceinline__ void acc_add(unsigned long long *acc, F127::T v) {
    unsigned long long old0 = atomicAdd(&acc[0], (unsigned long long)v.lo);
    unsigned long long add1 = v.hi + (unsigned long long)(old0 + v.lo < old0);  // <= 2^63
    unsigned long long old1 = atomicAdd(&acc[1], add1);
    if (old1 + add1 < old1) atomicAdd(&acc[2], 1ull);
}

// 192-bit accumulator -> field element.  The words are read from L2 (they
// are written by other CTAs' atomics, and may share a cache line with
// state this SM read earlier).
__device__ __forceinline__ void acc_words(const unsigned long long *a, unsigned long long (&w)[3]) {
    w[0] = __ldcg(a);
    w[1] = __ldcg(a + 1);
    w[2] = __ldcg(a + 2);
}
__device__ __forceinline__ F61::T acc_reduce_f61(const unsigned long long (&a)[3]) {
    auto red = [](uint64_t w) -> uint64_t {          // one word mod p
        uint64_t s = (w & F61::P) + (w >> 61);
        return s >= F61::P ? s - F61::P : s;
    };
    // 2^64 == 2^3 and 2^128 == 2^6 (mod 2^61 - 1)
    return F61::add(red(a[0]), F61::add(F61::mul(red(a[1]), 8), F61::mul(red(a[2]), 64)));
}
__device__ __forceinline__ F127::T acc_reduce_f127(const unsigned long long (&a)[3]) {
    // (a1:a0) < 2^128 reduced by a fold, then + 2*a2 since 2^128 == 2
    uint64_t lo = a[0], hi = a[1];
    uint64_t top = hi >> 63;
    hi &= F127::PHI;
    uint64_t nlo = lo + top;
    hi += (nlo < lo);
    lo = nlo;                                          // <= 2^127
    F127::T v;
    if (hi >> 63) v = {1, 0};                          // 2^127 == 1
    else if (lo == F127::PLO && hi == F127::PHI) v = {0, 0};
    else v = {lo, hi};
    F127::T t = {a[2], 0};                             // a2 < 2^64 < p
    return F127::add(v, F127::add(t, t));
}
// 2^64 == 25 and 2^128 == 625 (mod 2^32 - 5)
__device__ __forceinline__ F32::T acc_reduce_f32(const unsigned long long (&a)[3]) {
    return F32::add(F32::reduce64(a[0]),
                    F32::add(F32::mul(F32::reduce64(a[1]), 25u), F32::mul(F32::reduce64(a[2]), 625u)));
}
// from words already loaded
template <class F> __device__ __forceinline__ typename F::T acc_reduce_w(const unsigned long long (&w)[3]);
template <> __device__ __forceinline__ F32::T acc_reduce_w<F32>(const unsigned long long (&w)[3]) {
    return acc_reduce_f32(w);
}
template <> __device__ __forceinline__ F61::T acc_reduce_w<F61>(const unsigned long long (&w)[3]) {
    return acc_reduce_f61(w);
}
template <> __device__ __forceinline__ F127::T acc_reduce_w<F127>(const unsigned long long (&w)[3]) {
    return acc_reduce_f127(w);
}
// from the accumulator in memory
template <class F> __device__ __forceinline__ typename F::T acc_reduce(const unsigned long long *a) {
    unsigned long long w[3];
    acc_words(a, w);
    return acc_reduce_w<F>(w);
}

// ------------------------------------------------------------- reductions
__device__ __forceinline__ F61::T shfl_xor(F61::T v, int m) {
    return __shfl_xor_sync(0xffffffffu, (unsigned long long)v, m);
}
__device__ __forceinline__ F32::T shfl_xor(F32::T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ F127::T shfl_xor(F127::T v, int m) {
    return {__shfl_xor_sync(0xffffffffu, (unsigned long long)v.lo, m),
            __shfl_xor_sync(0xffffffffu, (unsigned long long)v.hi, m)};
}

template <class F>
__device__ __forceinline__ typename F::T warp_sum(typename F::T v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = F::add(v, shfl_xor(v, m));
    return v;
}

// Reduces K field values per thread over the block and adds the block's sums
// to the device accumulators acc[0..K-1] (one atomic group per block).
// Must be called by every thread of the block.
template <class F, int K>
__device__ __forceinline__ void block_accumulate(typename F::T (&v)[K], unsigned long long (*acc)[4]) {
    using T = typename F::T;
    __shared__ T red[32][K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum<F>(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) red[warp][k] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
        // lane k adds sum k: the K atomic round trips overlap instead of
        // following each other in one lane
        T mine = F::zero();
#pragma unroll
        for (int k = 0; k < K; ++k) {
            T s = lane < nwarps ? red[lane][k] : F::zero();
            s = warp_sum<F>(s);
            if (lane == k) mine = s;
        }
        if (lane < K && !F::is_zero(mine)) acc_add(acc[lane], mine);
    }
    __syncthreads();
}

// ---------------------------------------------------------------- dispatch
#define SPDZ_CASE_NP(N, ...) \
    case N: {                \
        constexpr int NP = N; \
        __VA_ARGS__;         \
    } break;
#define SPDZ_NP_SWITCH(n, ...)                                                     \
    switch (n) {                                                                   \
        SPDZ_CASE_NP(2, __VA_ARGS__) SPDZ_CASE_NP(3, __VA_ARGS__)                 \
        SPDZ_CASE_NP(4, __VA_ARGS__) SPDZ_CASE_NP(5, __VA_ARGS__)                 \
        SPDZ_CASE_NP(6, __VA_ARGS__) SPDZ_CASE_NP(7, __VA_ARGS__)                 \
        SPDZ_CASE_NP(8, __VA_ARGS__)                                               \
        default: break;                                                            \
    }
#define SPDZ_FIELD_SWITCH(f, ...)          \
    if ((f) == SPDZ_F61) {                 \
        using F = spdz::F61;               \
        __VA_ARGS__;                       \
    } else if ((f) == SPDZ_F32) {          \
        using F = spdz::F32;               \
        __VA_ARGS__;                       \
    } else {                               \
        using F = spdz::F127;              \
        __VA_ARGS__;                       \
    }

}  // namespace spdz

// ------------------------------------------------------------ host context
struct spdz_ctx {
    int n = 0;
    int field = 0;
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    spdz::DevState *ds = nullptr;        // device
    spdz::DevState *hres = nullptr;      // pinned host copy of results
    bool alpha_loaded = false;
    spdz_buf ta{}, tb{}, tc{};
    int64_t tri_total = 0, tri_cursor = 0;
    int64_t opened = 0;                  // values opened in the current epoch
    int64_t epoch = 0;
    uint64_t check_seed = 0;
    std::string err;
    void *sched = nullptr;               // scheduler state (sched.cu)
    void *mat = nullptr;                 // matrix-product state (matmul.cu)
    void *ll = nullptr;                  // linear-layer state (linear_layer.cu)
    // host-buffer circuit runs: a copy stream for the triples, the event of
    // the last pool registration (copies into the pool wait for it) and a
    // ring of copy-done events
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t pool_ev = nullptr;
    cudaEvent_t copy_ev[4] = {};
    int copy_k = 0;
};

namespace spdz {

inline size_t elem_bytes(int field) { return field == SPDZ_F61 ? 8 : field == SPDZ_F32 ? 4 : 16; }
// Host arrays and constants hold 64-bit words: one per element (p61, p32),
// two for p127.
inline size_t host_elem_bytes(int field) { return field == SPDZ_F127 ? 16 : 8; }
// Copies a host element (64-bit words) into the field's device format.
inline void host_to_dev_elem(int field, const void *host, void *dev) {
    if (field == SPDZ_F32) {
        const uint32_t v = (uint32_t)*(const uint64_t *)host;
        memcpy(dev, &v, 4);
    } else {
        memcpy(dev, host, elem_bytes(field));
    }
}

int set_err(spdz_ctx *ctx, int code, const char *fmt, ...);
int check_cuda(spdz_ctx *ctx, cudaError_t e, const char *what);
int check_launch(spdz_ctx *ctx, const char *what);
int validate_buf(spdz_ctx *ctx, const spdz_buf *b, int64_t N, const char *name);
bool buf_vec2_ok(const spdz_buf *b);    // 16-byte aligned rows (p61 vector path)
bool buf_vec_ok(const spdz_buf *b, size_t elem_bytes);   // 16-byte aligned rows, any element size
int grid_for(spdz_ctx *ctx, const void *kernel, int block, size_t smem, int64_t work_items);
void sched_destroy(spdz_ctx *ctx);
void mat_destroy(spdz_ctx *ctx);
void ll_destroy(spdz_ctx *ctx);
void sched_forget(spdz_ctx *ctx, const spdz_dag *dag);

}  // namespace spdz
