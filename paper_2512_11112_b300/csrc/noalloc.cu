// noalloc.cu -- a Beaver batch with its MAC check that allocates nothing.
//
// Some callers cannot allocate device memory: a host program whose memory
// manager has already reserved the whole device for its own pool, a plugin
// that is handed buffers but no allocation rights, or a latency-sensitive
// loop that must not pay for cudaMalloc's implicit device-wide
// synchronisation.  Such callers cannot create a context (a context owns a
// small device workspace), so this entry point runs a Beaver batch and its
// MAC check with no context: the only memory it needs besides the caller's
// inputs and outputs is a small fixed scratch area compiled into the library
// (the file-scope array below), which every GPU that loads the library keeps
// until the process exits.
#include <mutex>

#include "beaver.cuh"

namespace spdz {

// Scratch of the no-allocation entry point: the random-linear-combination
// accumulators, the coefficient key and the alpha shares of the current
// call.  Shared by every call on a device.
constexpr size_t NOALLOC_SCRATCH_BYTES = 4096;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

struct NoallocState {
    unsigned long long acc[MAXP + 1][4];   // acc[0] = A, acc[1+i] = S_i (exact 192-bit sums)
    uint64_t key;                          // coefficient key of the call's epoch
    uint64_t alpha[MAXP][2];               // alpha shares
};
static_assert(sizeof(NoallocState) <= NOALLOC_SCRATCH_BYTES, "no-alloc scratch too small");

template <class F>
__device__ __forceinline__ typename F::T na_alpha(const NoallocState *s, int i) {
    if constexpr (F::WORDS == 1) return s->alpha[i][0];
    else return typename F::T{s->alpha[i][0], s->alpha[i][1]};
}

// Clears the accumulators (the scratch keeps the previous call's contents)
// and loads the call's key and alpha shares.
template <class F>
__global__ void k_na_init(NoallocState *s, const typename F::T *alpha_sh, int n, uint64_t key) {
    const int t = threadIdx.x;
    if (t < (MAXP + 1) * 4) s->acc[t / 4][t % 4] = 0;
    if (t < n) {
        const typename F::T a = F::ld(alpha_sh + t);
        if constexpr (F::WORDS == 1) {
            s->alpha[t][0] = a;
            s->alpha[t][1] = 0;
        } else {
            s->alpha[t][0] = a.lo;
            s->alpha[t][1] = a.hi;
        }
    }
    if (t == 0) s->key = key;
}

template <class F> struct NaArgs {
    using T = typename F::T;
    const T *xv, *xm, *yv, *ym;
    int64_t xs, ys;
    const T *tp[6];       // a, gamma(a), b, gamma(b), c, gamma(c) at the first triple used
    int64_t ts[6];
    T *zv, *zm;
    int64_t zs;
    int64_t N;
    NoallocState *s;
};

// Beaver products j = 0..N-1 (opened eps_j, delta_j at check indices 2j, 2j+1).
template <class F, int NP>
__global__ void __launch_bounds__(256) k_na_mul(NaArgs<F> a) {
    using T = typename F::T;
    const uint64_t key = a.s->key;
    T alpha[NP], acc[NP + 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) alpha[i] = na_alpha<F>(a.s, i);
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.N; j += (int64_t)gridDim.x * blockDim.x) {
        T x[NP], gx[NP], y[NP], gy[NP], tri[6][NP], z[NP], gz[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            x[i] = F::ld(a.xv + i * a.xs + j);
            gx[i] = F::ld(a.xm + i * a.xs + j);
            y[i] = F::ld(a.yv + i * a.ys + j);
            gy[i] = F::ld(a.ym + i * a.ys + j);
#pragma unroll
            for (int k = 0; k < 6; ++k) tri[k][i] = F::ld(a.tp[k] + i * a.ts[k] + j);
        }
        auto src = [&](int k, int i) -> T { return tri[k][i]; };
        beaver_math_src<F, NP>(x, gx, y, gy, src, alpha, key, 2 * (uint64_t)j, acc, z, gz);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            F::st(a.zv + i * a.zs + j, z[i]);
            F::st(a.zm + i * a.zs + j, gz[i]);
        }
    }
    block_accumulate<F, NP + 1>(acc, a.s->acc);
}

// sigma_i = S_i - alpha_i * A into result[0..n-1]; result[n] = 1 if the check
// passed (sum sigma_i == 0), else 0.
template <class F, int NP>
__global__ void k_na_finish(const NoallocState *s, typename F::T *result) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    using T = typename F::T;
    const T A = acc_reduce<F>(s->acc[0]);
    T tot = F::zero();
    for (int i = 0; i < NP; ++i) {
        const T sig = F::sub(acc_reduce<F>(s->acc[1 + i]), F::mul(na_alpha<F>(s, i), A));
        F::st(result + i, sig);
        tot = F::add(tot, sig);
    }
    T flag = F::zero();
    if (F::is_zero(tot)) {
        if constexpr (F::WORDS == 1) flag = 1;
        else flag = T{1, 0};
    }
    F::st(result + NP, flag);
}

// Device address of the scratch array, looked up once per device (host
// code must not use the array's name as a device pointer).  The address is
// kept for the life of the process: after cudaDeviceReset (or any teardown
// of the device's primary context) it is stale, so a process that resets a
// device must not call spdz_mul_check_noalloc on it again.
static std::mutex g_na_mu;
constexpr int NA_MAX_DEVICES = 64;
static void *g_na_ptr[NA_MAX_DEVICES];

static int na_scratch(NoallocState **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return SPDZ_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SPDZ_ERR_CUDA;
        g_na_ptr[dev] = p;
    }
    *out = (NoallocState *)g_na_ptr[dev];
    return SPDZ_OK;
}

static int na_check_buf(const spdz_buf *b, int64_t N, int n, size_t eb) {
    if (!b || !b->val || !b->mac) return SPDZ_ERR_ARG;
    if (n > 1 && b->stride < N) return SPDZ_ERR_ARG;
    if ((uintptr_t)b->val % eb || (uintptr_t)b->mac % eb) return SPDZ_ERR_ALIGN;
    return SPDZ_OK;
}

template <class F, int NP>
static int na_run(cudaStream_t st, const spdz_buf *x, const spdz_buf *y, const spdz_buf *a, const spdz_buf *b,
                  const spdz_buf *c, const void *alpha_sh, const spdz_buf *z, int64_t N, uint64_t key,
                  void *result, NoallocState *s) {
    using T = typename F::T;
    // each launch's status is read right after it, so an error reported here
    // belongs to this call's launches
    k_na_init<F><<<1, 64, 0, st>>>(s, (const T *)alpha_sh, NP, key);
    if (cudaGetLastError() != cudaSuccess) return SPDZ_ERR_CUDA;
    if (N > 0) {
        NaArgs<F> g{};
        g.xv = (const T *)x->val; g.xm = (const T *)x->mac; g.xs = x->stride;
        g.yv = (const T *)y->val; g.ym = (const T *)y->mac; g.ys = y->stride;
        const spdz_buf *tb[3] = {a, b, c};
        for (int k = 0; k < 3; ++k) {
            g.tp[2 * k] = (const T *)tb[k]->val;
            g.tp[2 * k + 1] = (const T *)tb[k]->mac;
            g.ts[2 * k] = g.ts[2 * k + 1] = tb[k]->stride;
        }
        g.zv = (T *)z->val; g.zm = (T *)z->mac; g.zs = z->stride;
        g.N = N;
        g.s = s;
        int dev = 0, sms = 1, occ = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_na_mul<F, NP>, 256, 0);
        const int64_t need = (N + 255) / 256, cap = (int64_t)(occ < 1 ? 1 : occ) * sms;
        k_na_mul<F, NP><<<(int)(need < cap ? need : cap), 256, 0, st>>>(g);
        if (cudaGetLastError() != cudaSuccess) return SPDZ_ERR_CUDA;
    }
    k_na_finish<F, NP><<<1, 32, 0, st>>>(s, (T *)result);
    return cudaGetLastError() == cudaSuccess ? SPDZ_OK : SPDZ_ERR_CUDA;
}

}  // namespace spdz

using namespace spdz;

extern "C" int spdz_mul_check_noalloc(int n_parties, int field, void *stream, const spdz_buf *x,
                                      const spdz_buf *y, const spdz_buf *a, const spdz_buf *b,
                                      const spdz_buf *c, const void *alpha_shares_dev, const spdz_buf *z,
                                      int64_t N, uint64_t check_seed, uint64_t epoch, void *result_dev) {
    if (field != SPDZ_F61 && field != SPDZ_F127 && field != SPDZ_F32) return SPDZ_ERR_ARG;
    // the scratch holds accumulators for at most SPDZ_MAX_PARTIES parties
    if (n_parties < 2 || n_parties > SPDZ_MAX_PARTIES) return SPDZ_ERR_ARG;
    if (N < 0 || !alpha_shares_dev || !result_dev) return SPDZ_ERR_ARG;
    const size_t eb = elem_bytes(field);
    if ((uintptr_t)alpha_shares_dev % eb || (uintptr_t)result_dev % eb) return SPDZ_ERR_ALIGN;
    if (N > 0) {
        const spdz_buf *bufs[6] = {x, y, a, b, c, z};
        for (const spdz_buf *q : bufs)
            if (int rc = na_check_buf(q, N, n_parties, eb)) return rc;
    }
    NoallocState *s = nullptr;
    if (int rc = na_scratch(&s)) return rc;
    const uint64_t key = stream_key(check_seed, stream_id(SPDZ_KIND_CHECK, 0, 0, epoch));
    int rc = SPDZ_ERR_ARG;
    SPDZ_FIELD_SWITCH(field, SPDZ_NP_SWITCH(n_parties, rc = (na_run<F, NP>((cudaStream_t)stream, x, y, a, b, c,
                                                                            alpha_shares_dev, z, N, key, result_dev, s))));
    return rc;
}
