// serve.cu -- a serving loop for circuit requests: admission by a device
// memory budget, device-resident shares, and continuous batching of the
// layers of every active request (the paper's non-blocking scheduling of
// independent batched regions, Sec. III-C, applied across requests).
//
// A server runs on a host thread of its own between spdz_serve_start and
// spdz_serve_stop; callers submit requests at any time (spdz_serve_submit)
// and collect each result when it is ready (spdz_serve_poll).  A submitted
// request waits in a FIFO until the arena (one device allocation of
// `budget` bytes, which also holds every registered circuit) can hold its
// wires, triples and, for a one-off circuit, its gate records; its
// preprocessing is then dealt on an offline stream.  Runnable requests are
// executed by ticks: one launch per field per tick evaluates the next layer
// of every active request, cut into tiles of at most 256 gates that each
// belong to one request, so every tile reduces its MAC-check terms into its
// own request's accumulators.  A request that has finished its last layer is
// checked (its own epoch) in the same tick.  A request that the scheduler
// judges narrow enough instead runs all of its layers in one cluster launch
// on a side stream, concurrently with the ticks (cluster barriers only, so
// the two kinds of launch cannot wait on each other).  Modes: sequential (one
// request at a time, one launch per layer), batched (ticks only), heuristic
// (cluster launch for requests whose widest layer is below a threshold) and
// learned (cluster launch when the cost model predicts it faster).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <unordered_map>
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

// CTAs of a request's grid launch: half of what the GPU holds of the kernel
// (p61: two CTAs per SM, so one per SM; p127: one per SM, so one per two),
// so that two such launches (or one and the ticks) share the GPU.
static int serve_grid_ctas(int sm_count, int field) {
    return std::max(1, field == SPDZ_F61 ? sm_count : sm_count / 2);
}

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

// One request's part of a tick: its layer's records [r0, r1) are tiles
// tile0, tile0 + 1, ... of the tick, 256 records each (the last one short).
struct TickReq {
    int32_t slot, layer, r0, r1, tile0, pad;
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

// One tick: every tile is <= blockDim.x (256) gates of one layer of one
// request.  The tick's requests (sorted by tile0) are copied into shared
// memory when they fit (staged != 0), and a tile finds its request by a
// binary search over tile0.
template <class F, int NP>
__global__ void __launch_bounds__(256) k_serve_tick(const ReqDev *reqs, const TickReq *treq, int nreq, int ntiles,
                                                    int staged) {
    using T = typename F::T;
    extern __shared__ TickReq tq_smem[];
    const TickReq *tq = treq;
    if (staged) {
        for (int j = threadIdx.x; j < nreq; j += blockDim.x) tq_smem[j] = treq[j];
        __syncthreads();
        tq = tq_smem;
    }
    // A CTA's tiles (gridDim apart) mostly belong to one request: its check
    // sums are kept in registers and added to the request's accumulators
    // when the CTA moves to another request and at the end, not once per
    // tile.  The request of a tile is the same for every thread of the CTA.
    int cur = -1;
    DevState *cur_ds = nullptr;
    T acc[NP + 1];
#pragma unroll
    for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        int lo = 0, hi = nreq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tq[mid].tile0 <= t) lo = mid;
            else hi = mid - 1;
        }
        const TickReq q = tq[lo];
        const DagArgs<F> a = req_args<F>(reqs[q.slot]);
        if (lo != cur) {
            if (cur >= 0) {
                block_accumulate<F, NP + 1>(acc, cur_ds->acc);
#pragma unroll
                for (int k = 0; k < NP + 1; ++k) acc[k] = F::zero();
            }
            cur = lo;
            cur_ds = a.ds;
        }
        const int32_t r0 = q.r0 + 256 * (t - q.tile0), r1 = min(q.r1, r0 + 256);
        const LayerRow L = load_row(a.lay, q.layer);
        const uint64_t key = a.ds->key;
        T alpha[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) alpha[i] = load_alpha<F>(a.ds, i);
        const int32_t r = r0 + (int32_t)threadIdx.x;
        if (r < r1) {
            const int cls = class_of(L, r);
            GateIn<F, NP> g;
            gate_load_direct<F, NP>(a, L, r, cls, 0, g);
            gate_exec<F, NP>(a, L, r, cls, g.rec, g.k, TriRegs<F, NP>{g}, key, alpha, acc);
        }
    }
    if (cur >= 0) block_accumulate<F, NP + 1>(acc, cur_ds->acc);
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
    ds->bar_count = 0;     // (a grid launch's layer barriers)
    ds->bar_abort = 0;
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
    void reset_peak() { peak_ = used_; }
    size_t size() const { return size_; }

  private:
    void *base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

}  // namespace spdz

using namespace spdz;

namespace {

// A circuit's host build: gate records, constants and layer rows in the
// layout of spdz_dag_create, plus the shape figures the loop needs.
struct HostCircuit {
    std::vector<uint4> rec;
    std::vector<unsigned char> kc;
    std::vector<LayerRow> lay;
    std::vector<int32_t> counts;
    int64_t n_mul = 0, wmax = 0, n_inputs = 0, gates = 0;
    int depth = 0, field = 0;
    size_t dev_bytes() const {
        auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
        return a(rec.size() * 16 + 16) + a(kc.size() + 16) + a(lay.size() * sizeof(LayerRow));
    }
};

// Builds a circuit's records (same layout as spdz_dag_create); rejects a
// descriptor whose operands are not written before their layer.
int build_circuit(const spdz_dag_desc *d, int field, HostCircuit &h) {
    if (field != SPDZ_F61 && field != SPDZ_F127) return SPDZ_ERR_ARG;
    if (!d || d->n_gates < 0 || d->n_inputs < 0 || d->depth < 1 || d->depth > 1020 || !d->layer_offsets)
        return SPDZ_ERR_ARG;
    if (d->n_gates > 0 && (!d->ops || !d->in0 || !d->in1 || !d->kconst)) return SPDZ_ERR_ARG;
    if (d->n_gates >= (int64_t)INT32_MAX || d->n_inputs + d->n_gates > (int64_t)UINT32_MAX) return SPDZ_ERR_ARG;
    const int64_t *off = d->layer_offsets;
    if (off[0] != 0 || off[d->depth] != d->n_gates) return SPDZ_ERR_ARG;
    const size_t eb = field == SPDZ_F61 ? 8 : 16;
    h.field = field;
    h.depth = d->depth;
    h.n_inputs = d->n_inputs;
    h.gates = d->n_gates;
    h.rec.resize((size_t)d->n_gates);
    h.kc.assign((size_t)d->n_gates * eb, 0);
    h.lay.assign(d->depth, LayerRow{});
    h.counts.assign((size_t)d->depth * 5, 0);
    static const int cls_op[5] = {SPDZ_OP_MUL, SPDZ_OP_ADD, SPDZ_OP_SUB, SPDZ_OP_CMUL, SPDZ_OP_CADD};
    size_t pos = 0;
    h.n_mul = 0;
    h.wmax = 0;
    for (int l = 0; l < d->depth; ++l) {
        if (off[l + 1] < off[l]) return SPDZ_ERR_ARG;
        h.wmax = std::max<int64_t>(h.wmax, off[l + 1] - off[l]);
        const uint64_t limit = (uint64_t)d->n_inputs + (uint64_t)off[l];
        LayerRow &L = h.lay[l];
        L.mulbase = (int32_t)h.n_mul;
        for (int c = 0; c < 5; ++c) {
            L.s[c] = (int32_t)pos;
            for (int64_t i = off[l]; i < off[l + 1]; ++i) {
                const uint8_t op = d->ops[i];
                if (op > SPDZ_OP_MUL) return SPDZ_ERR_ARG;
                if (op != cls_op[c]) continue;
                const bool binary = op == SPDZ_OP_ADD || op == SPDZ_OP_SUB || op == SPDZ_OP_MUL;
                if (d->in0[i] >= limit || (binary && d->in1[i] >= limit)) return SPDZ_ERR_ARG;
                h.rec[pos] = make_uint4(d->in0[i], binary ? d->in1[i] : d->in0[i], (uint32_t)(d->n_inputs + i), 0u);
                if (op == SPDZ_OP_CMUL || op == SPDZ_OP_CADD)
                    memcpy(&h.kc[pos * eb], (const unsigned char *)d->kconst + (size_t)i * eb, eb);
                ++pos;
                h.counts[(size_t)l * 5 + c]++;
            }
        }
        L.s[5] = (int32_t)pos;
        h.n_mul += L.s[1] - L.s[0];
    }
    return SPDZ_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

double secs(std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
    return std::chrono::duration<double>(b - a).count();
}

}  // namespace

// A circuit on the device: its records inside the arena (registered
// circuits: a block of their own, kept until unregistered; one-off
// circuits: inside their request's block), its layer table on the host and
// the cost model's predictions for it.
struct ServeCircuit {
    uint4 *rec = nullptr;
    void *kc = nullptr;
    LayerRow *lay = nullptr;
    std::vector<LayerRow> h_lay;
    std::vector<int32_t> counts;
    int64_t n_mul = 0, wmax = 0, W = 0, gates = 0, n_inputs = 0;
    int depth = 0;
    int field = 0;
    long long off = -1;                    // registered: the arena block
    size_t bytes = 0;
    int users = 0;                         // admitted requests using it
    bool predicted = false;                // learned mode: predictions made
    double pred_cluster_us = 0;            // the whole circuit in one cluster launch
    std::vector<double> pred_grid_us;      // each layer on the grid
};

namespace {

// Places a host-built circuit at dev (a block of at least h.dev_bytes()) and
// enqueues its upload on st (the host vectors must live until it is done).
void place_circuit(const HostCircuit &h, char *dev, ServeCircuit &C, cudaStream_t st) {
    C.rec = (uint4 *)dev;
    C.kc = dev + align256(h.rec.size() * 16 + 16);
    C.lay = (LayerRow *)((char *)C.kc + align256(h.kc.size() + 16));
    C.h_lay = h.lay;
    C.counts = h.counts;
    C.n_mul = h.n_mul;
    C.wmax = h.wmax;
    C.W = h.n_inputs + h.gates;
    C.gates = h.gates;
    C.n_inputs = h.n_inputs;
    C.depth = h.depth;
    C.field = h.field;
    if (!h.rec.empty()) cudaMemcpyAsync(C.rec, h.rec.data(), h.rec.size() * 16, cudaMemcpyHostToDevice, st);
    if (!h.kc.empty()) cudaMemcpyAsync(C.kc, h.kc.data(), h.kc.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(C.lay, h.lay.data(), h.lay.size() * sizeof(LayerRow), cudaMemcpyHostToDevice, st);
}

// A submitted request waiting for admission.
struct Pending {
    uint64_t id = 0;
    spdz_serve_request r{};
    double arrival = 0;
    std::shared_ptr<HostCircuit> host;     // one-off circuit, built at submission
    ServeCircuit *reg = nullptr;           // registered circuit
};

// An admitted request.
struct Live {
    Pending p;
    int slot = -1;
    int field = 0;
    long long off = -1;
    size_t bytes = 0;
    int depth = 0, next = 0;
    int64_t W = 0, n_mul = 0, gates = 0, wmax = 0;
    ServeCircuit *circ = nullptr;
    std::unique_ptr<ServeCircuit> own;     // one-off circuit (inside the request's block)
    bool cluster = false;
    bool grid = false;                     // all its layers in one fused launch on part of the grid
    double backlog_us = 0;                 // learned: predicted cluster time it added to the backlog
    double grid_backlog_us = 0;            // learned: predicted grid-launch time it added
    cudaEvent_t deal0 = nullptr, dealt = nullptr, done = nullptr, up = nullptr;
    bool dealt_ok = false, launched_cluster = false;
    double t_runnable = 0;
    void *wv = nullptr, *wm = nullptr;
};

}  // namespace

struct spdz_server {
    int n = 0;
    int mode = 0;
    int max_active = 0;
    uint64_t check_seed = 0;
    int64_t cluster_width = 4096;   // heuristic threshold (widest layer)
    spdz_ctx *model_ctx = nullptr;  // holds the trained cost model (learned mode)
    Arena arena;
    size_t reserved = 0;            // arena bytes of registered circuits
    int device = 0;
    int sm_count = 0;
    double hbm_bytes_per_us = 0;    // theoretical DRAM bandwidth (memory clock x bus width)
    cudaStream_t tick_stream = nullptr, deal_stream = nullptr;
    // host-to-device copies of circuits and caller inputs (pageable sources):
    // a copy from pageable memory first waits for its stream's earlier work,
    // so they get a stream with no kernels on it
    cudaStream_t up_stream = nullptr;
    std::vector<cudaStream_t> side;
    DevState *ds_slots = nullptr;   // [max_active]
    ReqDev *d_reqs = nullptr;       // [max_active]
    ReqDev *h_reqs = nullptr;       // pinned mirror
    // tick buffers (ring of pinned host + device tile lists)
    static constexpr int RING = 4;
    // a tick's requests and finishing slots, pinned host and device, at most
    // max_active requests of each field
    void *h_tickbuf[RING] = {}, *d_tickbuf[RING] = {};
    cudaEvent_t ring_ev[RING] = {};       // end of the tick that used the slot
    cudaEvent_t ring_start[RING] = {};    // start of its kernels
    std::map<int64_t, std::unique_ptr<ServeCircuit>> circuits;   // registered, by id
    int64_t next_circuit = 0;
    double tick_us_ema = 0;                // measured duration of one tick (moving average)
    double tick_us_min = 0;                // shortest tick measured: the fixed cost of a tick
    double tick_us_per_gate = 0;           // ticks' device time per gate beyond the fixed cost (moving average)
    int64_t ring_gates[RING] = {};         // gates of the tick that used the slot
    double cluster_backlog_us = 0;         // learned: predicted time of cluster launches not yet done
    double grid_backlog_us = 0;            // learned: predicted time of grid launches not yet done
    int64_t grid_gates = (int64_t)1 << 20; // heuristic: requests of at least this many gates take a grid launch
    int64_t st_grid = 0;
    // the serving thread and what it shares with the callers
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Pending> inbox;             // submitted, not yet seen by the thread
    std::set<uint64_t> inflight;           // submitted, not yet completed
    std::unordered_map<uint64_t, spdz_serve_result> results;   // completed, not yet collected
    uint64_t next_id = 1;
    bool running = false, stopping = false;
    int worker_rc = SPDZ_OK;               // sticky: the first failure of the thread
    std::chrono::steady_clock::time_point t0;
    // statistics of the current session (start .. stop)
    std::vector<double> lat;
    int64_t st_requests = 0, st_gates = 0, st_ticks = 0, st_cluster = 0;
    double st_dealer_s = 0, st_last_done = 0;
    double st_tick_dev_s = 0;              // device time of the ticks measured so far
    int64_t st_tick_timed = 0;
    int st_max_active = 0;
    double h_admit = 0, h_tick = 0, h_done = 0, h_idle = 0, h_ringwait = 0;

    double now() const { return secs(t0, std::chrono::steady_clock::now()); }
    void loop();
    void finish(uint64_t id, const spdz_serve_result &res);
};

void spdz_server::finish(uint64_t id, const spdz_serve_result &res) {
    std::lock_guard<std::mutex> g(mu);
    inflight.erase(id);
    results[id] = res;
    cv.notify_all();
}

// The serving thread: takes submitted requests, admits them first come first
// served while memory and slots allow, deals their preprocessing, runs ticks
// and cluster launches, and publishes each result when its check is done.
void spdz_server::loop() {
    spdz_server *s = this;
    cudaSetDevice(device);
    const int n_ = n;
    std::deque<Pending> queue;
    std::vector<Live *> admitted;
    std::vector<int> free_slots;
    const int active_cap = mode == SPDZ_SERVE_SEQUENTIAL ? 1 : max_active;
    for (int k = active_cap - 1; k >= 0; --k) free_slots.push_back(k);
    int ring = 0;
    std::vector<int> ring_busy(RING, 0);
    int rc_fail = SPDZ_OK;

    auto release_live = [&](Live *L) {
        if (L->off >= 0) s->arena.release((size_t)L->off, L->bytes);
        s->cluster_backlog_us = std::max(0.0, s->cluster_backlog_us - L->backlog_us);
        s->grid_backlog_us = std::max(0.0, s->grid_backlog_us - L->grid_backlog_us);
        if (L->circ && !L->own) L->circ->users -= 1;
        if (L->deal0) cudaEventDestroy(L->deal0);
        if (L->dealt) cudaEventDestroy(L->dealt);
        if (L->done) cudaEventDestroy(L->done);
        if (L->up) cudaEventDestroy(L->up);
        delete L;
    };

    while (true) {
        // arrivals
        {
            std::unique_lock<std::mutex> g(mu);
            while (!inbox.empty()) {
                queue.push_back(std::move(inbox.front()));
                inbox.pop_front();
            }
            if (stopping && queue.empty() && admitted.empty()) break;
        }
        const double ta = now();
        // admission, first come first served
        while (!queue.empty() && !free_slots.empty()) {
            Pending &P = queue.front();
            // a copy: P leaves the queue (and is destroyed) once admitted
            const spdz_serve_request R = P.r;
            const int field = R.field;
            const size_t eb = field == SPDZ_F61 ? 8 : 16;
            const int64_t W = P.reg ? P.reg->W : P.host->n_inputs + P.host->gates;
            const int64_t nmul = P.reg ? P.reg->n_mul : P.host->n_mul;
            const int64_t T = std::max<int64_t>(1, nmul);
            const size_t b_w = align256((size_t)n_ * W * eb), b_t = align256((size_t)n_ * T * eb);
            const size_t b_al = align256((size_t)n_ * eb);
            const size_t b_c = P.reg ? 0 : align256(P.host->dev_bytes());
            const size_t bytes = 2 * b_w + 6 * b_t + b_al + b_c;
            if (bytes > arena.size() - reserved) {
                // can never fit the budget: refused
                spdz_serve_result res{};
                res.status = SPDZ_ERR_OOM;
                res.req_id = P.id;
                res.latency_s = now() - P.arrival;
                finish(P.id, res);
                queue.pop_front();
                continue;
            }
            const long long off = arena.alloc(bytes);
            if (off < 0) break;                      // wait for memory to free up
            auto *L = new Live();
            L->p = std::move(P);
            queue.pop_front();
            L->off = off;
            L->bytes = bytes;
            L->field = field;
            char *p = arena.ptr((size_t)off);
            if (L->p.reg) {
                L->circ = L->p.reg;
                L->circ->users += 1;
            } else {
                L->own.reset(new ServeCircuit());
                place_circuit(*L->p.host, p + 2 * b_w + 6 * b_t + b_al, *L->own, up_stream);
                L->circ = L->own.get();
            }
            const ServeCircuit &C = *L->circ;
            L->depth = C.depth;
            L->W = C.W;
            L->gates = C.gates;
            L->n_mul = C.n_mul;
            L->wmax = C.wmax;
            L->slot = free_slots.back();
            free_slots.pop_back();
            L->wv = p;
            L->wm = p + b_w;
            char *tri = p + 2 * b_w;
            char *pal = tri + 6 * b_t;
            ReqDev &H = h_reqs[L->slot];
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
            H.ds = ds_slots + L->slot;
            cudaEventCreate(&L->deal0);
            cudaEventRecord(L->deal0, deal_stream);
            const int64_t nin = C.n_inputs;
            if (R.in_val_host && nin > 0) {
                // the caller's input shares: party rows of n_inputs elements
                cudaMemcpy2DAsync(L->wv, (size_t)W * eb, R.in_val_host, (size_t)nin * eb, (size_t)nin * eb, (size_t)n_,
                                  cudaMemcpyHostToDevice, up_stream);
                cudaMemcpy2DAsync(L->wm, (size_t)W * eb, R.in_mac_host, (size_t)nin * eb, (size_t)nin * eb, (size_t)n_,
                                  cudaMemcpyHostToDevice, up_stream);
            }
            const bool uploads = !L->p.reg || (R.in_val_host && nin > 0);
            if (uploads) {
                cudaEventCreateWithFlags(&L->up, cudaEventDisableTiming);
                cudaEventRecord(L->up, up_stream);
            }
            SPDZ_FIELD_SWITCH(field, SPDZ_NP_SWITCH(n_, {
                using TT = typename F::T;
                k_deal_alpha<F><<<1, 32, 0, deal_stream>>>(R.seed, n_, (TT *)pal);
                if (!R.in_val_host && nin > 0) {
                    auto ki = make_keys<NP>(R.seed, SPDZ_KIND_INPUT, 16);
                    k_deal_shared<F, NP><<<(int)std::min<int64_t>((nin + 255) / 256, 4 * sm_count), 256, 0, deal_stream>>>(
                        ki, 0, nin, (const TT *)pal, nullptr, (TT *)L->wv, (TT *)L->wm, W, nullptr);
                }
                if (L->n_mul > 0) {
                    auto ka = make_keys<NP>(R.seed, SPDZ_KIND_TRIPLE_A, 0);
                    auto kb = make_keys<NP>(R.seed, SPDZ_KIND_TRIPLE_B, 0);
                    auto kcc = make_keys<NP>(R.seed, SPDZ_KIND_TRIPLE_C, 0);
                    k_deal_triples<F, NP><<<(int)std::min<int64_t>((L->n_mul + 255) / 256, 4 * sm_count), 256, 0, deal_stream>>>(
                        ka, kb, kcc, 0, L->n_mul, (const TT *)pal, (TT *)H.tp[0], (TT *)H.tp[1], T, (TT *)H.tp[2],
                        (TT *)H.tp[3], T, (TT *)H.tp[4], (TT *)H.tp[5], T);
                }
                k_serve_init<F><<<1, 1, 0, deal_stream>>>(H.ds, (const TT *)pal, n_, check_seed);
            }));
            // the request is dealt once its circuit and inputs are on the device
            if (uploads) cudaStreamWaitEvent(deal_stream, L->up, 0);
            cudaMemcpyAsync(d_reqs + L->slot, &H, sizeof(ReqDev), cudaMemcpyHostToDevice, deal_stream);
            cudaEventCreate(&L->dealt);
            cudaEventRecord(L->dealt, deal_stream);
            if (cudaGetLastError() != cudaSuccess) {
                rc_fail = SPDZ_ERR_CUDA;
                admitted.push_back(L);
                break;
            }
            // execution mode of the request
            if (mode == SPDZ_SERVE_HEURISTIC) {
                L->cluster = L->wmax <= cluster_width;
                L->grid = !L->cluster && L->gates >= grid_gates;
            } else if (mode == SPDZ_SERVE_LEARNED) {
                // the cheapest of ticks, one cluster launch and one grid
                // launch, each priced from the cost model's per-layer
                // predictions (below)
                ServeCircuit &Cm = *L->circ;
                if (!Cm.predicted) {
                    spdz_dag tmp;
                    tmp.field = field;
                    tmp.n = n_;
                    tmp.depth = L->depth;
                    tmp.counts = C.counts;
                    std::vector<double> pc;
                    Cm.pred_cluster_us = 0;
                    if (sched_predict_config(model_ctx, &tmp, sched_cluster_config(), pc) == SPDZ_OK &&
                        sched_predict_config(model_ctx, &tmp, sched_grid_config(), Cm.pred_grid_us) == SPDZ_OK) {
                        // a layer in one cluster of k CTAs (one per SM) cannot
                        // move its bytes faster than k SMs' share of DRAM
                        // bandwidth: the prediction is clamped to that floor,
                        // which also bounds the model outside the widths it
                        // was trained on
                        const int k = sched_cluster_width();
                        const double share = hbm_bytes_per_us * k / std::max(1, sm_count);
                        const double w = field == SPDZ_F61 ? 8.0 : 16.0;
                        for (int l = 0; l < L->depth; ++l) {
                            const int32_t *c = &C.counts[(size_t)l * 5];
                            const double bb = n_ * w * (12.0 * c[0] + 6.0 * (c[1] + c[2]) + 4.0 * (c[3] + c[4]));
                            Cm.pred_cluster_us += std::max(pc[(size_t)l], bb / share);
                        }
                        Cm.predicted = true;
                    }
                }
                if (Cm.predicted) {
                    double tick_mode = 0;
                    // a ticked layer costs at least the tick's fixed cost plus
                    // its gates at the ticks' measured time per gate, and at
                    // least its predicted time on the whole grid
                    const double floor_us = tick_us_min > 0 ? tick_us_min : tick_us_ema;
                    for (int l = 0; l < L->depth; ++l) {
                        const int32_t *c = &C.counts[(size_t)l * 5];
                        const double gl = (double)c[0] + c[1] + c[2] + c[3] + c[4];
                        tick_mode += std::max(Cm.pred_grid_us[(size_t)l], floor_us + gl * tick_us_per_gate);
                    }
                    // a cluster launch first waits for the cluster launches
                    // already queued: their predicted time spread over the
                    // clusters the SMs hold at once
                    const double conc = std::max(1, sm_count / std::max(1, sched_cluster_width()));
                    const double t_cluster = cluster_backlog_us / conc + Cm.pred_cluster_us;
                    // a grid launch: each layer at least its predicted time on
                    // the whole grid and its bytes at the launch's share of
                    // DRAM bandwidth (its CTAs over what the GPU holds), after
                    // the grid launches already waiting (two run at once)
                    const double share = hbm_bytes_per_us * serve_grid_ctas(sm_count, field) / std::max(1, (field == SPDZ_F61 ? 2 : 1) * sm_count);
                    const double w = field == SPDZ_F61 ? 8.0 : 16.0;
                    double pred_grid = 0;
                    for (int l = 0; l < L->depth; ++l) {
                        const int32_t *c = &C.counts[(size_t)l * 5];
                        const double bb = n_ * w * (12.0 * c[0] + 6.0 * (c[1] + c[2]) + 4.0 * (c[3] + c[4]));
                        pred_grid += std::max(Cm.pred_grid_us[(size_t)l], bb / std::max(1.0, share));
                    }
                    const double t_grid = grid_backlog_us / 2 + pred_grid;
                    L->cluster = t_cluster < tick_mode && t_cluster <= t_grid;
                    L->grid = !L->cluster && t_grid < tick_mode;
                    if (L->cluster) {
                        L->backlog_us = Cm.pred_cluster_us;
                        cluster_backlog_us += L->backlog_us;
                    }
                    if (L->grid) {
                        L->grid_backlog_us = pred_grid;
                        grid_backlog_us += pred_grid;
                    }
                }
            }
            admitted.push_back(L);
        }
        st_max_active = std::max<int>(st_max_active, (int)admitted.size());
        h_admit += now() - ta;
        if (rc_fail) break;
        // dealt requests become runnable; cluster requests launch now
        for (Live *L : admitted) {
            if (L->dealt_ok) continue;
            if (cudaEventQuery(L->dealt) != cudaSuccess) continue;
            L->dealt_ok = true;
            L->t_runnable = now();
            if (L->cluster) {
                cudaStream_t st = side[(size_t)(L->slot % (int)side.size())];
                cudaStreamWaitEvent(st, L->dealt, 0);
                const ReqDev &H = h_reqs[L->slot];
                SPDZ_FIELD_SWITCH(L->field, SPDZ_NP_SWITCH(n_, {
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
                ++st_cluster;
                if (cudaGetLastError() != cudaSuccess) rc_fail = SPDZ_ERR_CUDA;
            } else if (L->grid) {
                // all its layers in one fused launch with device barriers
                // between layers, on a side stream; a cooperative launch, so
                // that every CTA is resident at once
                cudaStream_t st = side[(size_t)(L->slot % (int)side.size())];
                cudaStreamWaitEvent(st, L->dealt, 0);
                const ReqDev &H = h_reqs[L->slot];
                SPDZ_FIELD_SWITCH(L->field, SPDZ_NP_SWITCH(n_, {
                    DagArgs<F> a{};
                    using TT = typename F::T;
                    a.rec = H.rec; a.kc = (const TT *)H.kc; a.lay = H.lay;
                    a.wv = (TT *)H.wv; a.wm = (TT *)H.wm; a.ws = H.ws;
                    for (int k = 0; k < 6; ++k) { a.tp[k] = (const TT *)H.tp[k]; a.ts[k] = H.ts[k]; }
                    a.ds = H.ds; a.l0 = 0; a.l1 = L->depth;
                    a.bar_base = 0;
                    a.spin_ns = 500000000ull;   // bound of one layer barrier wait
                    const int blk = 256;
                    const size_t smem = fused_smem<F, NP>(blk);
                    auto gk = F::WORDS == 1 ? k_dag_fused<F, NP> : k_dag_fused_wide<F, NP>;
                    if (smem > 48 * 1024) cudaFuncSetAttribute((const void *)gk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    void *args[1] = {&a};
                    cudaLaunchCooperativeKernel((const void *)gk, dim3(serve_grid_ctas(sm_count, L->field)), dim3(blk), args, smem, st);
                    k_serve_check_one<F, NP><<<1, 32, 0, st>>>(H.ds);
                }));
                cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
                cudaEventRecord(L->done, st);
                L->launched_cluster = true;
                L->next = L->depth;
                ++st_grid;
                if (cudaGetLastError() != cudaSuccess) rc_fail = SPDZ_ERR_CUDA;
            }
        }
        if (rc_fail) break;
        // one tick: next layer of every runnable ticking request
        std::vector<Live *> ticking;
        for (Live *L : admitted)
            if (L->dealt_ok && !L->cluster && !L->grid && L->next < L->depth) ticking.push_back(L);
        const double tt = now();
        if (!ticking.empty()) {
            // wait for the ring slot to be free again
            if (ring_busy[ring]) {
                const double tw = now();
                cudaEventSynchronize(ring_ev[ring]);
                h_ringwait += now() - tw;
                // device duration of the tick that used this slot
                float ms = 0;
                if (cudaEventElapsedTime(&ms, ring_start[ring], ring_ev[ring]) == cudaSuccess && ms > 0) {
                    tick_us_ema = tick_us_ema == 0 ? ms * 1e3 : 0.9 * tick_us_ema + 0.1 * ms * 1e3;
                    tick_us_min = tick_us_min == 0 ? ms * 1e3 : std::min(tick_us_min, (double)ms * 1e3);
                    if (ring_gates[ring] > 0) {
                        const double per = std::max(0.0, ms * 1e3 - tick_us_min) / (double)ring_gates[ring];
                        tick_us_per_gate = tick_us_per_gate == 0 ? per : 0.9 * tick_us_per_gate + 0.1 * per;
                    }
                    st_tick_dev_s += ms * 1e-3;
                    ++st_tick_timed;
                }
                ring_busy[ring] = 0;
            }
            // the tick's requests by field (p61 first, then p127), each with
            // its first tile index, then the slots of the requests finishing
            // with this tick: one copy
            TickReq *ht = reinterpret_cast<TickReq *>(h_tickbuf[ring]);
            int nq[2] = {0, 0}, nt[2] = {0, 0}, nf[2] = {0, 0};
            for (int fld = 0; fld < 2; ++fld)
                for (Live *L : ticking) {
                    if (L->field != fld) continue;
                    const LayerRow &R = L->circ->h_lay[L->next];
                    ht[nq[0] * fld + nq[fld]++] = TickReq{L->slot, L->next, R.s[0], R.s[5], nt[fld], 0};
                    nt[fld] += (R.s[5] - R.s[0] + 255) / 256;
                }
            const int nreq = nq[0] + nq[1];
            int32_t *hs = reinterpret_cast<int32_t *>(ht + nreq);
            for (int fld = 0; fld < 2; ++fld)
                for (Live *L : ticking)
                    if (L->field == fld && L->next + 1 == L->depth) hs[nf[0] * fld + nf[fld]++] = L->slot;
            const size_t tick_bytes = (size_t)nreq * sizeof(TickReq) + (size_t)(nf[0] + nf[1]) * sizeof(int32_t);
            cudaMemcpyAsync(d_tickbuf[ring], ht, tick_bytes, cudaMemcpyHostToDevice, tick_stream);
            const TickReq *dq = reinterpret_cast<const TickReq *>(d_tickbuf[ring]);
            const int32_t *dslots = reinterpret_cast<const int32_t *>(dq + nreq);
            // the tick must see every request's descriptor and dealt state
            for (Live *L : ticking)
                if (L->next == 0) cudaStreamWaitEvent(tick_stream, L->dealt, 0);
            cudaEventRecord(ring_start[ring], tick_stream);
            for (int fld = 0; fld < 2; ++fld) {
                if (nt[fld] == 0) continue;
                const TickReq *dqf = dq + (fld == 0 ? 0 : nq[0]);
                const int grid = (int)std::min<int64_t>(nt[fld], (int64_t)8 * sm_count);
                const size_t qb = (size_t)nq[fld] * sizeof(TickReq);
                const int staged = qb <= 48 * 1024;
                const size_t smem = staged ? qb : 0;
                SPDZ_FIELD_SWITCH(fld, SPDZ_NP_SWITCH(n_, k_serve_tick<F, NP><<<grid, 256, smem, tick_stream>>>(
                                                           d_reqs, dqf, nq[fld], nt[fld], staged)));
                if (nf[fld] > 0)
                    SPDZ_FIELD_SWITCH(fld, SPDZ_NP_SWITCH(n_, k_serve_check<F, NP><<<(nf[fld] + 63) / 64, 64, 0, tick_stream>>>(
                                                               d_reqs, dslots + (fld == 0 ? 0 : nf[0]), nf[fld])));
            }
            cudaEventRecord(ring_ev[ring], tick_stream);
            ring_busy[ring] = 1;
            ring_gates[ring] = 0;
            for (Live *L : ticking) {
                const LayerRow &R = L->circ->h_lay[L->next];
                ring_gates[ring] += R.s[5] - R.s[0];
            }
            for (Live *L : ticking) {
                L->next += 1;
                if (L->next == L->depth) {
                    cudaEventCreateWithFlags(&L->done, cudaEventDisableTiming);
                    cudaEventRecord(L->done, tick_stream);
                }
            }
            ring = (ring + 1) % RING;
            ++st_ticks;
            if (cudaGetLastError() != cudaSuccess) rc_fail = SPDZ_ERR_CUDA;
        }
        h_tick += now() - tt;
        if (rc_fail) break;
        // completions
        const double tc = now();
        bool progressed = !ticking.empty();
        for (size_t k = 0; k < admitted.size();) {
            Live *L = admitted[k];
            if (L->done && cudaEventQuery(L->done) == cudaSuccess) {
                const spdz_serve_request &R = L->p.r;
                DevState *ds = h_reqs[L->slot].ds;
                uint32_t passed = 0;
                cudaMemcpy(&passed, &ds->res_passed, sizeof(passed), cudaMemcpyDeviceToHost);
                const size_t eb = L->field == SPDZ_F61 ? 8 : 16;
                if (R.out_val_host) cudaMemcpy(R.out_val_host, L->wv, (size_t)n_ * L->W * eb, cudaMemcpyDeviceToHost);
                if (R.out_mac_host) cudaMemcpy(R.out_mac_host, L->wm, (size_t)n_ * L->W * eb, cudaMemcpyDeviceToHost);
                const double t = now();
                spdz_serve_result res{};
                res.latency_s = t - L->p.arrival;
                res.online_s = t - L->t_runnable;
                res.passed = (int32_t)passed;
                res.mode = L->cluster ? 1 : L->grid ? 2 : 0;
                res.status = passed ? SPDZ_OK : SPDZ_ERR_MAC;
                res.req_id = L->p.id;
                lat.push_back(res.latency_s);
                st_gates += L->gates;
                st_requests += 1;
                st_last_done = t;
                float dms = 0;
                if (cudaEventElapsedTime(&dms, L->deal0, L->dealt) == cudaSuccess) st_dealer_s += dms * 1e-3;
                free_slots.push_back(L->slot);
                const uint64_t id = L->p.id;
                release_live(L);
                admitted.erase(admitted.begin() + (long)k);
                finish(id, res);
                progressed = true;
            } else {
                ++k;
            }
        }
        h_done += now() - tc;
        if (!progressed && ticking.empty()) {
            const double ti = now();
            std::unique_lock<std::mutex> g(mu);
            if (admitted.empty() && queue.empty()) {
                // nothing on the device: sleep until a submission or stop
                cv.wait(g, [&] { return !inbox.empty() || stopping; });
            } else {
                // waiting for the device or for memory: look again shortly
                cv.wait_for(g, std::chrono::microseconds(20), [&] { return !inbox.empty(); });
            }
            h_idle += now() - ti;
        }
    }
    if (rc_fail) {
        // a CUDA failure ends the session: every request not completed is
        // reported with the failure
        cudaDeviceSynchronize();
        std::vector<uint64_t> ids;
        for (Live *L : admitted) {
            ids.push_back(L->p.id);
            release_live(L);
        }
        for (auto &P : queue) ids.push_back(P.id);
        {
            std::lock_guard<std::mutex> g(mu);
            for (auto &P : inbox) ids.push_back(P.id);
            inbox.clear();
            worker_rc = rc_fail;
        }
        for (uint64_t id : ids) {
            spdz_serve_result res{};
            res.status = rc_fail;
            res.req_id = id;
            finish(id, res);
        }
    }
    cudaStreamSynchronize(tick_stream);
    cudaStreamSynchronize(deal_stream);
    cudaStreamSynchronize(up_stream);
    for (auto st : side) cudaStreamSynchronize(st);
    // the ticks still in the ring
    for (int k = 0; k < RING; ++k) {
        float ms = 0;
        if (ring_busy[k] && cudaEventElapsedTime(&ms, ring_start[k], ring_ev[k]) == cudaSuccess && ms > 0) {
            st_tick_dev_s += ms * 1e-3;
            ++st_tick_timed;
        }
    }
}

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
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
    {
        int khz = 0, bits = 0;
        cudaDeviceGetAttribute(&khz, cudaDevAttrMemoryClockRate, s->device);
        cudaDeviceGetAttribute(&bits, cudaDevAttrGlobalMemoryBusWidth, s->device);
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
    cudaStreamCreateWithFlags(&s->up_stream, cudaStreamNonBlocking);
    s->side.resize(16);
    for (auto &st : s->side) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    const size_t tick_cap = (size_t)2 * s->max_active * (sizeof(TickReq) + sizeof(int32_t));
    for (int k = 0; k < spdz_server::RING; ++k) {
        cudaEventCreate(&s->ring_ev[k]);
        cudaEventCreate(&s->ring_start[k]);
        if (cudaMallocHost(&s->h_tickbuf[k], tick_cap) != cudaSuccess || cudaMalloc(&s->d_tickbuf[k], tick_cap) != cudaSuccess) {
            spdz_serve_destroy(s);
            return SPDZ_ERR_OOM;
        }
    }
    *out = s;
    return SPDZ_OK;
}

int spdz_serve_register(spdz_server *s, const spdz_dag_desc *dag, int32_t field, int64_t *circuit_id) {
    if (!s || !dag || !circuit_id) return SPDZ_ERR_ARG;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->running) return SPDZ_ERR_STATE;
    }
    HostCircuit h;
    if (int rc = build_circuit(dag, field, h)) return rc;
    const size_t bytes = align256(h.dev_bytes());
    const long long off = s->arena.alloc(bytes);
    if (off < 0) return SPDZ_ERR_OOM;
    std::unique_ptr<ServeCircuit> C(new ServeCircuit());
    place_circuit(h, s->arena.ptr((size_t)off), *C, s->deal_stream);
    C->off = off;
    C->bytes = bytes;
    if (cudaStreamSynchronize(s->deal_stream) != cudaSuccess) {
        s->arena.release((size_t)off, bytes);
        return SPDZ_ERR_CUDA;
    }
    s->reserved += bytes;
    const int64_t id = s->next_circuit++;
    s->circuits[id] = std::move(C);
    *circuit_id = id;
    return SPDZ_OK;
}

int spdz_serve_unregister(spdz_server *s, int64_t circuit_id) {
    if (!s) return SPDZ_ERR_ARG;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->running) return SPDZ_ERR_STATE;
    }
    auto it = s->circuits.find(circuit_id);
    if (it == s->circuits.end()) return SPDZ_ERR_ARG;
    s->arena.release((size_t)it->second->off, it->second->bytes);
    s->reserved -= it->second->bytes;
    s->circuits.erase(it);
    return SPDZ_OK;
}

int spdz_serve_set_mode(spdz_server *s, int32_t mode, spdz_ctx *model_ctx, int64_t cluster_width) {
    if (!s || mode < 0 || mode > SPDZ_SERVE_LEARNED || (mode == SPDZ_SERVE_LEARNED && !model_ctx)) return SPDZ_ERR_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->running) return SPDZ_ERR_STATE;
    s->mode = mode;
    s->model_ctx = model_ctx;
    if (cluster_width > 0) s->cluster_width = cluster_width;
    return SPDZ_OK;
}

int spdz_serve_start(spdz_server *s) {
    if (!s) return SPDZ_ERR_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->running) return SPDZ_ERR_STATE;
    if (s->worker_rc != SPDZ_OK) return s->worker_rc;
    s->running = true;
    s->stopping = false;
    s->t0 = std::chrono::steady_clock::now();
    s->lat.clear();
    s->st_requests = s->st_gates = s->st_ticks = s->st_cluster = s->st_grid = 0;
    s->st_dealer_s = s->st_last_done = 0;
    s->st_max_active = 0;
    s->h_admit = s->h_tick = s->h_done = s->h_idle = s->h_ringwait = 0;
    s->st_tick_dev_s = 0;
    s->st_tick_timed = 0;
    s->cluster_backlog_us = 0;
    s->grid_backlog_us = 0;
    s->arena.reset_peak();
    for (auto &kv : s->circuits) kv.second->users = 0;
    s->worker = std::thread([s] { s->loop(); });
    return SPDZ_OK;
}

int spdz_serve_submit(spdz_server *s, const spdz_serve_request *r, uint64_t *req_id) {
    if (!s || !r || !req_id) return SPDZ_ERR_ARG;
    Pending P;
    P.r = *r;
    if (r->circuit_id >= 0) {
        if (r->dag) return SPDZ_ERR_ARG;
        auto it = s->circuits.find(r->circuit_id);   // the table only changes while stopped
        if (it == s->circuits.end() || it->second->field != r->field) return SPDZ_ERR_ARG;
        P.reg = it->second.get();
        if (r->in_val_host && P.reg->n_inputs > 0 && !r->in_mac_host) return SPDZ_ERR_ARG;
    } else {
        // a one-off circuit: built here, on the caller's thread
        P.host = std::make_shared<HostCircuit>();
        if (int rc = build_circuit(r->dag, r->field, *P.host)) return rc;
        if (r->in_val_host && P.host->n_inputs > 0 && !r->in_mac_host) return SPDZ_ERR_ARG;
    }
    std::lock_guard<std::mutex> g(s->mu);
    if (!s->running || s->stopping) return SPDZ_ERR_STATE;
    if (s->worker_rc != SPDZ_OK) return s->worker_rc;
    const double now = s->now();
    P.arrival = r->arrival_s > 0 && r->arrival_s <= now ? r->arrival_s : now;
    P.id = s->next_id++;
    *req_id = P.id;
    s->inflight.insert(P.id);
    s->inbox.push_back(std::move(P));
    s->cv.notify_all();
    return SPDZ_OK;
}

int spdz_serve_poll(spdz_server *s, uint64_t req_id, int32_t *done, spdz_serve_result *result) {
    if (!s || !done) return SPDZ_ERR_ARG;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->results.find(req_id);
    if (it != s->results.end()) {
        *done = 1;
        if (result) *result = it->second;
        s->results.erase(it);
        return SPDZ_OK;
    }
    if (s->inflight.count(req_id)) {
        *done = 0;
        return SPDZ_OK;
    }
    return SPDZ_ERR_ARG;
}

int spdz_serve_stop(spdz_server *s, spdz_serve_stats *stats) {
    if (!s) return SPDZ_ERR_ARG;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (!s->running) return SPDZ_ERR_STATE;
        s->stopping = true;
        s->cv.notify_all();
    }
    s->worker.join();
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->running = false;
        s->stopping = false;
    }
    if (stats) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)std::floor(q * (double)(v.size() - 1) + 0.5))];
        };
        memset(stats, 0, sizeof *stats);
        const double wall = s->st_last_done;
        stats->wall_s = wall;
        stats->requests = s->st_requests;
        stats->gates = s->st_gates;
        stats->gates_per_s = wall > 0 ? (double)s->st_gates / wall : 0;
        stats->p50_s = pct(0.50);
        stats->p99_s = pct(0.99);
        double m = 0;
        for (double x : v) m += x;
        stats->mean_s = v.empty() ? 0 : m / (double)v.size();
        stats->ticks = s->st_ticks;
        stats->cluster_requests = s->st_cluster;
        stats->grid_requests = s->st_grid;
        stats->dealer_s = s->st_dealer_s;
        stats->peak_bytes = (int64_t)s->arena.peak();
        stats->max_active = s->st_max_active;
        stats->host_admit_s = s->h_admit;
        stats->host_tick_s = s->h_tick;
        stats->host_complete_s = s->h_done;
        stats->host_idle_s = s->h_idle;
        stats->host_ring_wait_s = s->h_ringwait;
        stats->device_tick_s = s->st_tick_dev_s;
        stats->device_ticks_timed = s->st_tick_timed;
    }
    return s->worker_rc;
}

int spdz_serve_destroy(spdz_server *s) {
    if (!s) return SPDZ_OK;
    bool run;
    {
        std::lock_guard<std::mutex> g(s->mu);
        run = s->running;
    }
    if (run) spdz_serve_stop(s, nullptr);
    cudaDeviceSynchronize();
    s->circuits.clear();
    if (s->ds_slots) cudaFree(s->ds_slots);
    if (s->d_reqs) cudaFree(s->d_reqs);
    if (s->h_reqs) cudaFreeHost(s->h_reqs);
    for (int k = 0; k < spdz_server::RING; ++k) {
        if (s->h_tickbuf[k]) cudaFreeHost(s->h_tickbuf[k]);
        if (s->d_tickbuf[k]) cudaFree(s->d_tickbuf[k]);
        if (s->ring_ev[k]) cudaEventDestroy(s->ring_ev[k]);
        if (s->ring_start[k]) cudaEventDestroy(s->ring_start[k]);
    }
    if (s->tick_stream) cudaStreamDestroy(s->tick_stream);
    if (s->deal_stream) cudaStreamDestroy(s->deal_stream);
    if (s->up_stream) cudaStreamDestroy(s->up_stream);
    for (auto st : s->side) cudaStreamDestroy(st);
    delete s;
    return SPDZ_OK;
}

// The trace driver: submits each request at its arrival time (seconds after
// the start) from the calling thread while the serving thread runs, then
// stops and collects every result.
int spdz_serve_run(spdz_server *s, const spdz_serve_request *reqs, int64_t count, spdz_serve_result *results,
                   spdz_serve_stats *stats) {
    if (!s || (count > 0 && !reqs) || count < 0) return SPDZ_ERR_ARG;
    if (int rc = spdz_serve_start(s)) return rc;
    std::vector<uint64_t> ids((size_t)count, 0);
    int rc = SPDZ_OK;
    for (int64_t k = 0; k < count && rc == SPDZ_OK; ++k) {
        const double t = reqs[k].arrival_s;
        if (t > 0) std::this_thread::sleep_until(s->t0 + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                                             std::chrono::duration<double>(t)));
        rc = spdz_serve_submit(s, &reqs[k], &ids[(size_t)k]);
    }
    const int rs = spdz_serve_stop(s, stats);
    if (rc == SPDZ_OK) rc = rs;
    for (int64_t k = 0; k < count; ++k) {
        if (!ids[(size_t)k]) continue;
        int32_t done = 0;
        spdz_serve_result res{};
        spdz_serve_poll(s, ids[(size_t)k], &done, &res);
        if (results) results[k] = res;
        if (rc == SPDZ_OK && res.status != SPDZ_OK) rc = res.status;
    }
    return rc;
}

}  // extern "C"
