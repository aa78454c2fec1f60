// serve.cu -- a serving loop for circuit requests: admission by a device
// memory budget, device-resident shares, and continuous batching of the
// layers of every active request (the paper's non-blocking scheduling of
// independent batched regions, Sec. III-C, applied across requests).
//
// Requests arrive over time.  An arriving request waits in a FIFO until the
// arena (one device allocation of `budget` bytes) can hold its wires,
// triples and circuit; its preprocessing is then dealt on an offline stream.
// Runnable requests are executed by ticks: one launch per field per tick
// evaluates the next layer of every active request, cut into tiles of at
// most 256 gates that each belong to one request, so every tile reduces its
// MAC-check terms into its own request's accumulators.  A request that has
// finished its last layer is checked (its own epoch) in the same tick.  A
// request that the scheduler judges narrow enough instead runs all of its
// layers in one cluster launch on a side stream, concurrently with the ticks
// (cluster barriers only, so the two kinds of launch cannot wait on each
// other).  Modes: sequential (one request at a time, one launch per layer),
// batched (ticks only), heuristic (cluster launch for requests whose widest
// layer is below a threshold) and learned (cluster launch when the cost model
// predicts it faster).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "check.cuh"
#include "dag_kernels.cuh"
#include "dealer.cuh"

namespace spdz {

int sched_predict_config(spdz_ctx *ctx, const spdz_dag *dag, int cfg, std::vector<double> &us);
int sched_cluster_config();
int sched_cluster_width();
int sched_grid_config();
double sched_switch_us(spdz_ctx *ctx);

// Device-side descriptor of one admitted request (pointers into the arena).
struct ReqDev {
    const uint4 *rec;
    const void *kc;
    const LayerRow *lay;
    void *wv, *wm;
    int64_t ws;
    const void *tp[6];
    int64_t ts[6];
    DevState *ds;
};

struct Tile {
    int32_t slot, layer, r0, r1;
};

template <class F>
__device__ __forceinline__ DagArgs<F> req_args(const ReqDev &R) {
    using T = typename F::T;
    DagArgs<F> a{};
    a.rec = R.rec;
    a.kc = (const T *)R.kc;
    a.lay = R.lay;
    a.wv = (T *)R.wv;
    a.wm = (T *)R.wm;
    a.ws = R.ws;
    for (int k = 0; k < 6; ++k) {
        a.tp[k] = (const T *)R.tp[k];
        a.ts[k] = R.ts[k];
    }
    a.ds = R.ds;
    return a;
}

// One tick: every tile is <= blockDim.x gates of one layer of one request.
template <class F, int NP>
__global__ void __launch_bounds__(256) k_serve_tick(const ReqDev *reqs, const Tile *tiles, int ntiles) {
    using T = typename F::T;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const Tile tl = tiles[t];
        const DagArgs<F> a = req_args<F>(reqs[tl.slot]);
        const LayerRow L = load_row(a.lay, tl.layer);
        const uint64_t key = a.ds->key;
        T alpha[NP], acc[NP + 1];
#pragma unroll
        for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
#pragma unroll
        for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
        const int32_t r = tl.r0 + (int32_t)threadIdx.x;
        if (r < tl.r1) {
            const int cls = class_of(L, r);
            GateIn<F, NP> g;
            gate_load_direct<F, NP>(a, L, r, cls, 0, g);
            gate_exec<F, NP>(a, L, r, cls, g.rec, g.k, TriRegs<F, NP>{g}, key, alpha, acc);
        }
        block_accumulate<F, NP + 1>(acc, a.ds->acc);
    }
}

// Final MAC check of one request (after its cluster launch).
template <class F, int NP>
__global__ void k_serve_check_one(DevState *ds) {
    if (threadIdx.x == 0 && blockIdx.x == 0) check_epoch<F, NP>(ds, 1);
}

// Final MAC check of the listed requests (one thread each).
template <class F, int NP>
__global__ void k_serve_check(const ReqDev *reqs, const int32_t *slots, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) check_epoch<F, NP>(reqs[slots[k]].ds, 1);
}

// Fresh device state of an admitted request: its alpha shares, the key of
// check epoch 0 under check_seed, zero accumulators, triple cursor 0.
template <class F>
__global__ void k_serve_init(DevState *ds, const typename F::T *alpha, int n, uint64_t check_seed) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ds->check_seed = check_seed;
    ds->epoch = 0;
    ds->key = stream_key(check_seed, stream_id(SPDZ_KIND_CHECK, 0, 0, 0));
    ds->tri_cursor = 0;
    for (int k = 0; k < MAXP + 1; ++k)
        for (int w = 0; w < 4; ++w) ds->acc[k][w] = 0;
    for (int i = 0; i < MAXP; ++i) ds->sig_run[i][0] = ds->sig_run[i][1] = 0;
    ds->partial_fail = 0;
    ds->err_flags = 0;
    ds->res_passed = 0;
    for (int i = 0; i < n; ++i) {
        const typename F::T a = F::ld(alpha + i);
        if constexpr (F::WORDS == 1) {
            ds->alpha[i][0] = a;
            ds->alpha[i][1] = 0;
        } else {
            ds->alpha[i][0] = a.lo;
            ds->alpha[i][1] = a.hi;
        }
    }
}

// ------------------------------------------------------------------ arena
// First-fit allocator over one device allocation; free blocks are merged
// with their neighbours.  Offsets are 256-byte aligned.
class Arena {
  public:
    bool init(size_t bytes) {
        size_ = bytes;
        if (cudaMalloc(&base_, bytes) != cudaSuccess) return false;
        free_[0] = bytes;
        return true;
    }
    ~Arena() {
        if (base_) cudaFree(base_);
    }
    long long alloc(size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return (long long)off;
            }
        }
        return -1;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char *ptr(size_t off) const { return (char *)base_ + off; }
    size_t peak() const { return peak_; }
    size_t size() const { return size_; }

  private:
    void *base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

}  // namespace spdz

using namespace spdz;

// A circuit uploaded once and shared read-only by every request that uses
// the same spdz_dag_desc (gate records, layer rows, constants).
struct ServeCircuit {
    uint4 *rec = nullptr;
    void *kc = nullptr;
    LayerRow *lay = nullptr;
    std::vector<LayerRow> h_lay;
    std::vector<int32_t> counts;
    int64_t n_mul = 0, wmax = 0, W = 0, gates = 0;
    int depth = 0;
    int field = 0;
    // cost-model predictions (learned mode), computed once per circuit
    bool predicted = false;
    double pred_cluster_us = 0;            // the whole circuit in one cluster launch
    std::vector<double> pred_grid_us;      // each layer on the grid
};

struct spdz_server {
    int n = 0;
    int mode = 0;
    int max_active = 0;
    uint64_t check_seed = 0;
    int64_t cluster_width = 4096;   // heuristic threshold (widest layer)
    spdz_ctx *model_ctx = nullptr;  // holds the trained cost model (learned mode)
    Arena arena;
    int sm_count = 0;
    double hbm_bytes_per_us = 0;    // theoretical DRAM bandwidth (memory clock x bus width)
    cudaStream_t tick_stream = nullptr, deal_stream = nullptr;
    std::vector<cudaStream_t> side;
    DevState *ds_slots = nullptr;   // [max_active]
    ReqDev *d_reqs = nullptr;       // [max_active]
    ReqDev *h_reqs = nullptr;       // pinned mirror
    // tick buffers (ring of pinned host + device tile lists)
    static constexpr int RING = 4;
    Tile *h_tiles[RING] = {}, *d_tiles[RING] = {};
    int32_t *h_slots[RING] = {}, *d_slots[RING] = {};
    cudaEvent_t ring_ev[RING] = {};       // end of the tick that used the slot
    cudaEvent_t ring_start[RING] = {};    // start of its kernels
    int64_t tile_cap = 0;
    std::map<const spdz_dag_desc *, ServeCircuit> circuits;
    double tick_us_ema = 0;                // measured duration of one tick (moving average)
    double tick_us_min = 0;                // shortest tick measured: the fixed cost of a tick
};

namespace {

struct Live {
    int64_t idx = -1;           // request index in the trace
    int slot = -1;
    int field = 0;
    long long off = -1;
    size_t bytes = 0;
    int depth = 0, next = 0;
    int64_t W = 0, n_mul = 0, gates = 0, wmax = 0;
    const ServeCircuit *circ = nullptr;
    bool cluster = false;
    cudaEvent_t deal0 = nullptr, dealt = nullptr, done = nullptr;
    bool dealt_ok = false, launched_cluster = false, finished = false;
    double t_runnable = 0;
    void *wv = nullptr, *wm = nullptr;
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Host build of a request's gate records, layer rows and constants (the
// same layout as spdz_dag_create).
int build_circuit(const spdz_dag_desc *d, size_t eb, std::vector<uint4> &rec, std::vector<unsigned char> &kc,
                  std::vector<LayerRow> &lay, std::vector<int32_t> &counts, int64_t &n_mul, int64_t &wmax) {
    if (!d || d->n_gates < 0 || d->depth < 1 || d->depth > 1020 || !d->layer_offsets) return SPDZ_ERR_ARG;
    const int64_t *off = d->layer_offsets;
    if (off[0] != 0 || off[d->depth] != d->n_gates) return SPDZ_ERR_ARG;
    rec.resize((size_t)d->n_gates);
    kc.assign((size_t)d->n_gates * eb, 0);
    lay.assign(d->depth, LayerRow{});
    counts.assign((size_t)d->depth * 5, 0);
    static const int cls_op[5] = {SPDZ_OP_MUL, SPDZ_OP_ADD, SPDZ_OP_SUB, SPDZ_OP_CMUL, SPDZ_OP_CADD};
    size_t pos = 0;
    n_mul = 0;
    wmax = 0;
    for (int l = 0; l < d->depth; ++l) {
        if (off[l + 1] < off[l]) return SPDZ_ERR_ARG;
        wmax = std::max<int64_t>(wmax, off[l + 1] - off[l]);
        const uint64_t limit = (uint64_t)d->n_inputs + (uint64_t)off[l];
        LayerRow &L = lay[l];
        L.mulbase = (int32_t)n_mul;
        for (int c = 0; c < 5; ++c) {
            L.s[c] = (int32_t)pos;
            for (int64_t i = off[l]; i < off[l + 1]; ++i) {
                const uint8_t op = d->ops[i];
                if (op > SPDZ_OP_MUL) return SPDZ_ERR_ARG;
                if (op != cls_op[c]) continue;
                const bool binary = op == SPDZ_OP_ADD || op == SPDZ_OP_SUB || op == SPDZ_OP_MUL;
                if (d->in0[i] >= limit || (binary && d->in1[i] >= limit)) return SPDZ_ERR_ARG;
                rec[pos] = make_uint4(d->in0[i], binary ? d->in1[i] : d->in0[i], (uint32_t)(d->n_inputs + i), 0u);
                if (op == SPDZ_OP_CMUL || op == SPDZ_OP_CADD)
                    memcpy(&kc[pos * eb], (const unsigned char *)d->kconst + (size_t)i * eb, eb);
                ++pos;
                counts[(size_t)l * 5 + c]++;
            }
        }
        L.s[5] = (int32_t)pos;
        n_mul += L.s[1] - L.s[0];
    }
    return SPDZ_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Builds and uploads a circuit once; later requests with the same
// descriptor share it.
int prepare_circuit(spdz_server *s, const spdz_dag_desc *d, int field, const ServeCircuit **out) {
    // the serving loop runs requests of the two Mersenne fields
    if (field != SPDZ_F61 && field != SPDZ_F127) return SPDZ_ERR_ARG;
    auto cit = s->circuits.find(d);
    if (cit == s->circuits.end()) {
        const size_t eb = field == SPDZ_F61 ? 8 : 16;
        ServeCircuit C;
        std::vector<uint4> rec;
        std::vector<unsigned char> kc;
        if (int rc = build_circuit(d, eb, rec, kc, C.h_lay, C.counts, C.n_mul, C.wmax)) return rc;
        C.depth = d->depth;
        C.W = d->n_inputs + d->n_gates;
        C.gates = d->n_gates;
        C.field = field;
        if (cudaMalloc(&C.rec, rec.size() * 16 + 16) != cudaSuccess || cudaMalloc(&C.kc, kc.size() + 16) != cudaSuccess ||
            cudaMalloc(&C.lay, C.h_lay.size() * sizeof(LayerRow)) != cudaSuccess)
            return SPDZ_ERR_OOM;
        cudaMemcpy(C.rec, rec.data(), rec.size() * 16, cudaMemcpyHostToDevice);
        cudaMemcpy(C.kc, kc.data(), kc.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(C.lay, C.h_lay.data(), C.h_lay.size() * sizeof(LayerRow), cudaMemcpyHostToDevice);
        cit = s->circuits.emplace(d, std::move(C)).first;
    }
    if (cit->second.field != field) return SPDZ_ERR_ARG;
    *out = &cit->second;
    return SPDZ_OK;
}

}  // namespace

extern "C" {

int spdz_serve_create(spdz_server **out, int n_parties, uint64_t budget_bytes, int32_t max_active, int32_t mode,
                      spdz_ctx *model_ctx, uint64_t check_seed, int64_t cluster_width) {
    if (!out || n_parties < 2 || n_parties > SPDZ_MAX_PARTIES || max_active < 1 || max_active > 4096 || mode < 0 ||
        mode > SPDZ_SERVE_LEARNED || budget_bytes < (1u << 20))
        return SPDZ_ERR_ARG;
    if (mode == SPDZ_SERVE_LEARNED && !model_ctx) return SPDZ_ERR_ARG;
    spdz_server *s = new spdz_server();
    s->n = n_parties;
    s->mode = mode;
    s->max_active = max_active;
    s->check_seed = check_seed;
    s->model_ctx = model_ctx;
    if (cluster_width > 0) s->cluster_width = cluster_width;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev);
    {
        int khz = 0, bits = 0;
        cudaDeviceGetAttribute(&khz, cudaDevAttrMemoryClockRate, dev);
        cudaDeviceGetAttribute(&bits, cudaDevAttrGlobalMemoryBusWidth, dev);
        // double data rate: 2 transfers per clock
        s->hbm_bytes_per_us = khz > 0 && bits > 0 ? 2.0 * khz * 1e3 * (bits / 8.0) * 1e-6 : 8e6;
    }
    if (!s->arena.init((size_t)budget_bytes) ||
        cudaMalloc(&s->ds_slots, sizeof(DevState) * (size_t)s->max_active) != cudaSuccess ||
        cudaMalloc(&s->d_reqs, sizeof(ReqDev) * (size_t)s->max_active) != cudaSuccess ||
        cudaMallocHost(&s->h_reqs, sizeof(ReqDev) * (size_t)s->max_active) != cudaSuccess) {
        spdz_serve_destroy(s);
        return SPDZ_ERR_OOM;
    }
    cudaStreamCreateWithFlags(&s->tick_stream, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&s->deal_stream, cudaStreamNonBlocking);
    s->side.resize(16);
    for (auto &st : s->side) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (int k = 0; k < spdz_server::RING; ++k) {
        cudaEventCreate(&s->ring_ev[k]);
        cudaEventCreate(&s->ring_start[k]);
    }
    *out = s;
    return SPDZ_OK;
}

int spdz_serve_prepare(spdz_server *s, const spdz_dag_desc *const *dags, const int32_t *fields, int64_t count) {
    if (!s || count < 0 || (count > 0 && (!dags || !fields))) return SPDZ_ERR_ARG;
    for (int64_t k = 0; k < count; ++k) {
        const ServeCircuit *c = nullptr;
        if (int rc = prepare_circuit(s, dags[k], fields[k], &c)) return rc;
    }
    return SPDZ_OK;
}

int spdz_serve_set_mode(spdz_server *s, int32_t mode, spdz_ctx *model_ctx, int64_t cluster_width) {
    if (!s || mode < 0 || mode > SPDZ_SERVE_LEARNED || (mode == SPDZ_SERVE_LEARNED && !model_ctx)) return SPDZ_ERR_ARG;
    if (mode == SPDZ_SERVE_SEQUENTIAL && s->max_active < 1) return SPDZ_ERR_ARG;
    s->mode = mode;
    s->model_ctx = model_ctx;
    if (cluster_width > 0) s->cluster_width = cluster_width;
    return SPDZ_OK;
}

int spdz_serve_destroy(spdz_server *s) {
    if (!s) return SPDZ_OK;
    cudaDeviceSynchronize();
    if (s->ds_slots) cudaFree(s->ds_slots);
    if (s->d_reqs) cudaFree(s->d_reqs);
    if (s->h_reqs) cudaFreeHost(s->h_reqs);
    for (int k = 0; k < spdz_server::RING; ++k) {
        if (s->h_tiles[k]) cudaFreeHost(s->h_tiles[k]);
        if (s->d_tiles[k]) cudaFree(s->d_tiles[k]);
        if (s->h_slots[k]) cudaFreeHost(s->h_slots[k]);
        if (s->d_slots[k]) cudaFree(s->d_slots[k]);
        if (s->ring_ev[k]) cudaEventDestroy(s->ring_ev[k]);
        if (s->ring_start[k]) cudaEventDestroy(s->ring_start[k]);
    }
    for (auto &kv : s->circuits) {
        cudaFree(kv.second.rec);
        cudaFree(kv.second.kc);
        cudaFree(kv.second.lay);
    }
    if (s->tick_stream) cudaStreamDestroy(s->tick_stream);
    if (s->deal_stream) cudaStreamDestroy(s->deal_stream);
    for (auto st : s->side) cudaStreamDestroy(st);
    delete s;
    return SPDZ_OK;
}

int spdz_serve_run(spdz_server *s, const spdz_serve_request *reqs, int64_t count, spdz_serve_result *results,
                   spdz_serve_stats *stats) {
    if (!s || (count > 0 && !reqs) || count < 0) return SPDZ_ERR_ARG;
    const int n = s->n;
    const auto t0 = std::chrono::steady_clock::now();
    std::deque<int64_t> queue;
    std::vector<Live *> admitted;                 // dealing, ticking or in a cluster launch
    std::vector<int> free_slots;
    const int active_cap = s->mode == SPDZ_SERVE_SEQUENTIAL ? 1 : s->max_active;
    for (int k = active_cap - 1; k >= 0; --k) free_slots.push_back(k);
    std::vector<double> lat;
    int64_t next_arrival = 0, done_count = 0, total_gates = 0, ticks = 0, cluster_reqs = 0;
    double dealer_s = 0;
    int ring = 0, max_active_seen = 0;
    std::vector<int> ring_busy(spdz_server::RING, 0);
    double h_admit = 0, h_tick = 0, h_done = 0, h_idle = 0, h_ringwait = 0;

    auto fail = [&](int rc) {
        cudaDeviceSynchronize();
        for (Live *L : admitted) {
            if (L->deal0) cudaEventDestroy(L->deal0);
            if (L->dealt) cudaEventDestroy(L->dealt);
            if (L->done) cudaEventDestroy(L->done);
            delete L;
        }
        return rc;
    };

    while (done_count < count) {
        const double now = now_s(t0);
        // arrivals
        while (next_arrival < count && reqs[next_arrival].arrival_s <= now) queue.push_back(next_arrival++);
        // admission, first come first served
        const double ta = now_s(t0);
        while (!queue.empty() && !free_slots.empty()) {
            const spdz_serve_request &R = reqs[queue.front()];
            const int field = R.field;
            const size_t eb = field == SPDZ_F61 ? 8 : 16;
            const ServeCircuit *Cp = nullptr;
            if (int rc = prepare_circuit(s, R.dag, field, &Cp)) return fail(rc);
            const ServeCircuit &C = *Cp;
            auto *L = new Live();
            L->circ = &C;
            L->idx = queue.front();
            L->field = field;
            L->depth = C.depth;
            L->W = C.W;
            L->gates = C.gates;
            L->n_mul = C.n_mul;
            L->wmax = C.wmax;
            const int64_t W = L->W, T = std::max<int64_t>(1, L->n_mul);
            const size_t b_w = align256((size_t)n * W * eb), b_t = align256((size_t)n * T * eb);
            const size_t b_al = align256((size_t)n * eb);
            L->bytes = 2 * b_w + 6 * b_t + b_al;
            if (L->bytes > s->arena.size()) {
                delete L;
                return fail(SPDZ_ERR_OOM);       // can never fit the budget
            }
            const long long off = s->arena.alloc(L->bytes);
            if (off < 0) {
                delete L;
                break;                           // wait for memory to free up
            }
            queue.pop_front();
            L->off = off;
            L->slot = free_slots.back();
            free_slots.pop_back();
            char *p = s->arena.ptr((size_t)off);
            L->wv = p;
            L->wm = p + b_w;
            char *tri = p + 2 * b_w;
            char *pal = tri + 6 * b_t;
            ReqDev &H = s->h_reqs[L->slot];
            H.rec = C.rec;
            H.kc = C.kc;
            H.lay = C.lay;
            H.wv = L->wv;
            H.wm = L->wm;
            H.ws = W;
            for (int k = 0; k < 6; ++k) {
                H.tp[k] = tri + (size_t)k * b_t;
                H.ts[k] = T;
            }
            H.ds = s->ds_slots + L->slot;
            cudaEventCreate(&L->deal0);
            cudaEventRecord(L->deal0, s->deal_stream);
            SPDZ_FIELD_SWITCH(field, SPDZ_NP_SWITCH(n, {
                using TT = typename F::T;
                k_deal_alpha<F><<<1, 32, 0, s->deal_stream>>>(R.seed, n, (TT *)pal);
                auto ki = make_keys<NP>(R.seed, SPDZ_KIND_INPUT, 16);
                const int64_t nin = R.dag->n_inputs;
                if (nin > 0)
                    k_deal_shared<F, NP><<<(int)std::min<int64_t>((nin + 255) / 256, 4 * s->sm_count), 256, 0, s->deal_stream>>>(
                        ki, 0, nin, (const TT *)pal, nullptr, (TT *)L->wv, (TT *)L->wm, W, nullptr);
                if (L->n_mul > 0) {
                    auto ka = make_keys<NP>(R.seed, SPDZ_KIND_TRIPLE_A, 0);
                    auto kb = make_keys<NP>(R.seed, SPDZ_KIND_TRIPLE_B, 0);
                    auto kcc = make_keys<NP>(R.seed, SPDZ_KIND_TRIPLE_C, 0);
                    k_deal_triples<F, NP><<<(int)std::min<int64_t>((L->n_mul + 255) / 256, 4 * s->sm_count), 256, 0, s->deal_stream>>>(
                        ka, kb, kcc, 0, L->n_mul, (const TT *)pal, (TT *)H.tp[0], (TT *)H.tp[1], T, (TT *)H.tp[2],
                        (TT *)H.tp[3], T, (TT *)H.tp[4], (TT *)H.tp[5], T);
                }
                k_serve_init<F><<<1, 1, 0, s->deal_stream>>>(H.ds, (const TT *)pal, n, s->check_seed);
            }));
            cudaMemcpyAsync(s->d_reqs + L->slot, &H, sizeof(ReqDev), cudaMemcpyHostToDevice, s->deal_stream);
            cudaEventCreate(&L->dealt);
            cudaEventRecord(L->dealt, s->deal_stream);
            if (cudaGetLastError() != cudaSuccess) return fail(SPDZ_ERR_CUDA);
            // execution mode of the request
            if (s->mode == SPDZ_SERVE_HEURISTIC) {
                L->cluster = L->wmax <= s->cluster_width;
            } else if (s->mode == SPDZ_SERVE_LEARNED) {
                // cluster launch when the whole circuit in one cluster is
                // predicted to finish before its layers would by ticks, each
                // tick lasting at least the shortest measured tick
                ServeCircuit &Cm = const_cast<ServeCircuit &>(C);
                if (!Cm.predicted) {
                    spdz_dag tmp;
                    tmp.field = field;
                    tmp.n = n;
                    tmp.depth = L->depth;
                    tmp.counts = C.counts;
                    std::vector<double> pc;
                    if (sched_predict_config(s->model_ctx, &tmp, sched_cluster_config(), pc) == SPDZ_OK &&
                        sched_predict_config(s->model_ctx, &tmp, sched_grid_config(), Cm.pred_grid_us) == SPDZ_OK) {
                        // a layer in one cluster of k CTAs (one per SM) cannot
                        // move its bytes faster than k SMs' share of DRAM
                        // bandwidth: the prediction is clamped to that floor,
                        // which also bounds the model outside the widths it
                        // was trained on
                        const int k = sched_cluster_width();
                        const double share = s->hbm_bytes_per_us * k / std::max(1, s->sm_count);
                        const double w = field == SPDZ_F61 ? 8.0 : 16.0;
                        for (int l = 0; l < L->depth; ++l) {
                            const int32_t *c = &C.counts[(size_t)l * 5];
                            const double bytes = n * w * (12.0 * c[0] + 6.0 * (c[1] + c[2]) + 4.0 * (c[3] + c[4]));
                            Cm.pred_cluster_us += std::max(pc[(size_t)l], bytes / share);
                        }
                        Cm.predicted = true;
                    }
                }
                if (Cm.predicted) {
                    double tick_mode = 0;
                    // each layer costs at least one tick's fixed cost (a long
                    // tick is long because of other requests' wide layers)
                    const double floor_us = s->tick_us_min > 0 ? s->tick_us_min : s->tick_us_ema;
                    for (double g : Cm.pred_grid_us) tick_mode += std::max(g, floor_us);
                    L->cluster = Cm.pred_cluster_us < tick_mode;
                }
            }
            admitted.push_back(L);
        }
        max_active_seen = std::max<int>(max_active_seen, (int)admitted.size());
        h_admit += now_s(t0) - ta;
        // dealt requests become runnable; cluster requests launch now
        for (Live *L : admitted) {
            if (L->dealt_ok) continue;
            if (cudaEventQuery(L->dealt) != cudaSuccess) continue;
            L->dealt_ok = true;
            L->t_runnable = now_s(t0);
            if (L->cluster) {
                cudaStream_t st = s->side[(size_t)(L->slot % (int)s->side.size())];
                cudaStreamWaitEvent(st, L->dealt, 0);
                const ReqDev &H = s->h_reqs[L->slot];
                SPDZ_FIELD_SWITCH(L->field, SPDZ_NP_SWITCH(n, {
                    DagArgs<F> a{};
                    using TT = typename F::T;
                    a.rec = H.rec; a.kc = (const TT *)H.kc; a.lay = H.lay;
                    a.wv = (TT *)H.wv; a.wm = (TT *)H.wm; a.ws = H.ws;
                    for (int k = 0; k < 6; ++k) { a.tp[k] = (const TT *)H.tp[k]; a.ts[k] = H.ts[k]; }
                    a.ds = H.ds; a.l0 = 0; a.l1 = L->depth;
                    const int blk = 256;
                    const size_t smem = fused_smem<F, NP>(blk);
                    auto ck = k_dag_cluster<F, NP>;
                    cudaFuncSetAttribute((const void *)ck, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
                    if (smem > 48 * 1024) cudaFuncSetAttribute((const void *)ck, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    cudaLaunchConfig_t cfg{};
                    cfg.gridDim = dim3(16);
                    cfg.blockDim = dim3(blk);
                    cfg.dynamicSmemBytes = smem;
                    cfg.stream = st;
                    cudaLaunchAttribute at[1];
                    at[0].id = cudaLaunchAttributeClusterDimension;
                    at[0].val.clusterDim.x = 16; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
                    cfg.attrs = at;
                    cfg.numAttrs = 1;
                    cudaLaunchKernelEx(&cfg, ck, a);
                    k_serve_check_one<F, NP><<<1, 32, 0, st>>>(H.ds);
                }));
                cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
                cudaEventRecord(L->done, st);
                L->launched_cluster = true;
                L->next = L->depth;
                ++cluster_reqs;
                if (cudaGetLastError() != cudaSuccess) return fail(SPDZ_ERR_CUDA);
            }
        }
        // one tick: next layer of every runnable ticking request
        std::vector<Live *> ticking;
        for (Live *L : admitted)
            if (L->dealt_ok && !L->cluster && L->next < L->depth) ticking.push_back(L);
        const double tt = now_s(t0);
        if (!ticking.empty()) {
            // wait for the ring slot to be free again
            if (ring_busy[ring]) {
                const double tw = now_s(t0);
                cudaEventSynchronize(s->ring_ev[ring]);
                h_ringwait += now_s(t0) - tw;
                // device duration of the tick that used this slot
                float ms = 0;
                if (cudaEventElapsedTime(&ms, s->ring_start[ring], s->ring_ev[ring]) == cudaSuccess && ms > 0) {
                    s->tick_us_ema = s->tick_us_ema == 0 ? ms * 1e3 : 0.9 * s->tick_us_ema + 0.1 * ms * 1e3;
                    s->tick_us_min = s->tick_us_min == 0 ? ms * 1e3 : std::min(s->tick_us_min, (double)ms * 1e3);
                }
            }
            int64_t need = 0;
            for (Live *L : ticking) {
                const LayerRow &R = L->circ->h_lay[L->next];
                need += (R.s[5] - R.s[0] + 255) / 256;
            }
            if (need > s->tile_cap) {
                for (int k = 0; k < spdz_server::RING; ++k) {
                    if (ring_busy[k]) cudaEventSynchronize(s->ring_ev[k]);
                    if (s->h_tiles[k]) cudaFreeHost(s->h_tiles[k]);
                    if (s->d_tiles[k]) cudaFree(s->d_tiles[k]);
                    if (s->h_slots[k]) cudaFreeHost(s->h_slots[k]);
                    if (s->d_slots[k]) cudaFree(s->d_slots[k]);
                    const int64_t cap = std::max<int64_t>(need * 2, 4096);
                    if (cudaMallocHost(&s->h_tiles[k], cap * sizeof(Tile)) != cudaSuccess ||
                        cudaMalloc(&s->d_tiles[k], cap * sizeof(Tile)) != cudaSuccess ||
                        cudaMallocHost(&s->h_slots[k], (size_t)s->max_active * sizeof(int32_t) * 2) != cudaSuccess ||
                        cudaMalloc(&s->d_slots[k], (size_t)s->max_active * sizeof(int32_t) * 2) != cudaSuccess)
                        return fail(SPDZ_ERR_OOM);
                    s->tile_cap = cap;
                    ring_busy[k] = 0;
                }
            }
            Tile *ht = s->h_tiles[ring];
            int32_t *hs = s->h_slots[ring];
            int nt[2] = {0, 0}, nf[2] = {0, 0};
            // tiles of each field grouped: p61 first, then p127
            for (int fld = 0; fld < 2; ++fld) {
                const int base = fld == 0 ? 0 : nt[0];
                int cnt = 0;
                for (Live *L : ticking) {
                    if (L->field != fld) continue;
                    const LayerRow &R = L->circ->h_lay[L->next];
                    for (int32_t r = R.s[0]; r < R.s[5]; r += 256) ht[base + cnt++] = Tile{L->slot, L->next, r, std::min(R.s[5], r + 256)};
                }
                nt[fld] = cnt;
            }
            // requests finishing with this tick (their last layer)
            for (int fld = 0; fld < 2; ++fld)
                for (Live *L : ticking)
                    if (L->field == fld && L->next + 1 == L->depth) hs[(fld == 0 ? 0 : s->max_active) + nf[fld]++] = L->slot;
            const int ntot = nt[0] + nt[1];
            cudaMemcpyAsync(s->d_tiles[ring], ht, (size_t)ntot * sizeof(Tile), cudaMemcpyHostToDevice, s->tick_stream);
            cudaMemcpyAsync(s->d_slots[ring], hs, (size_t)s->max_active * 2 * sizeof(int32_t), cudaMemcpyHostToDevice, s->tick_stream);
            // the tick must see every request's descriptor and dealt state
            for (Live *L : ticking)
                if (L->next == 0) cudaStreamWaitEvent(s->tick_stream, L->dealt, 0);
            cudaEventRecord(s->ring_start[ring], s->tick_stream);
            for (int fld = 0; fld < 2; ++fld) {
                if (nt[fld] == 0) continue;
                const Tile *dt = s->d_tiles[ring] + (fld == 0 ? 0 : nt[0]);
                const int grid = (int)std::min<int64_t>(nt[fld], (int64_t)8 * s->sm_count);
                SPDZ_FIELD_SWITCH(fld, SPDZ_NP_SWITCH(n, k_serve_tick<F, NP><<<grid, 256, 0, s->tick_stream>>>(s->d_reqs, dt, nt[fld])));
                if (nf[fld] > 0)
                    SPDZ_FIELD_SWITCH(fld, SPDZ_NP_SWITCH(n, k_serve_check<F, NP><<<(nf[fld] + 63) / 64, 64, 0, s->tick_stream>>>(
                                                               s->d_reqs, s->d_slots[ring] + (fld == 0 ? 0 : s->max_active), nf[fld])));
            }
            cudaEventRecord(s->ring_ev[ring], s->tick_stream);
            ring_busy[ring] = 1;
            for (Live *L : ticking) {
                L->next += 1;
                if (L->next == L->depth) {
                    cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
                    cudaEventRecord(L->done, s->tick_stream);
                }
            }
            ring = (ring + 1) % spdz_server::RING;
            ++ticks;
            if (cudaGetLastError() != cudaSuccess) return fail(SPDZ_ERR_CUDA);
        }
        h_tick += now_s(t0) - tt;
        // completions
        const double tc = now_s(t0);
        bool progressed = !ticking.empty();
        for (size_t k = 0; k < admitted.size();) {
            Live *L = admitted[k];
            if (L->done && cudaEventQuery(L->done) == cudaSuccess) {
                const spdz_serve_request &R = reqs[L->idx];
                DevState *ds = s->h_reqs[L->slot].ds;
                uint32_t passed = 0;
                cudaMemcpy(&passed, &ds->res_passed, sizeof(passed), cudaMemcpyDeviceToHost);
                const size_t eb = L->field == SPDZ_F61 ? 8 : 16;
                if (R.out_val_host)
                    cudaMemcpy(R.out_val_host, L->wv, (size_t)n * L->W * eb, cudaMemcpyDeviceToHost);
                if (R.out_mac_host)
                    cudaMemcpy(R.out_mac_host, L->wm, (size_t)n * L->W * eb, cudaMemcpyDeviceToHost);
                const double t = now_s(t0);
                if (results) {
                    results[L->idx].latency_s = t - R.arrival_s;
                    results[L->idx].online_s = t - L->t_runnable;
                    results[L->idx].passed = (int32_t)passed;
                    results[L->idx].mode = L->cluster ? 1 : 0;
                }
                lat.push_back(t - R.arrival_s);
                total_gates += L->gates;
                float dms = 0;
                if (cudaEventElapsedTime(&dms, L->deal0, L->dealt) == cudaSuccess) dealer_s += dms * 1e-3;
                s->arena.release((size_t)L->off, L->bytes);
                free_slots.push_back(L->slot);
                cudaEventDestroy(L->deal0);
                cudaEventDestroy(L->dealt);
                cudaEventDestroy(L->done);
                delete L;
                admitted.erase(admitted.begin() + (long)k);
                ++done_count;
                progressed = true;
            } else {
                ++k;
            }
        }
        h_done += now_s(t0) - tc;
        if (!progressed && ticking.empty()) {
            // nothing to launch: wait a little for arrivals or completions
            const double ti = now_s(t0);
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            h_idle += now_s(t0) - ti;
        }
    }
    cudaDeviceSynchronize();
    if (stats) {
        const double wall = now_s(t0);
        std::vector<double> v = lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)std::floor(q * (double)(v.size() - 1) + 0.5))]; };
        stats->wall_s = wall;
        stats->requests = count;
        stats->gates = total_gates;
        stats->gates_per_s = wall > 0 ? (double)total_gates / wall : 0;
        stats->p50_s = pct(0.50);
        stats->p99_s = pct(0.99);
        double m = 0;
        for (double x : v) m += x;
        stats->mean_s = v.empty() ? 0 : m / (double)v.size();
        stats->ticks = ticks;
        stats->cluster_requests = cluster_reqs;
        stats->dealer_s = dealer_s;
        stats->peak_bytes = (int64_t)s->arena.peak();
        stats->max_active = max_active_seen;
        stats->host_admit_s = h_admit;
        stats->host_tick_s = h_tick;
        stats->host_complete_s = h_done;
        stats->host_idle_s = h_idle;
        stats->host_ring_wait_s = h_ringwait;
    }
    return SPDZ_OK;
}

}  // extern "C"
