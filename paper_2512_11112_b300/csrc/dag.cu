// dag.cu -- evaluation of layered arithmetic circuits (the batched regions of
// Sec. III-B/III-C of the paper, with the independent gates of a layer already
// grouped).
//
// Two executions of the same circuit, bit-identical by construction:
//   * per-layer: one kernel launch per layer and gate class (MUL, linear),
//     stream-ordered -- the plain baseline;
//   * fused: one persistent kernel per group of consecutive layers; CTAs
//     meet at a device-wide barrier between layers (bounded wait, timeout
//     status instead of a hang), the run is captured once as a CUDA graph and
//     replayed;
//   * tagged (p61): the fused form over a tagged wire-major copy of the wires;
//     operands validate themselves by tag, so the layer barrier needs no fence.
// In both, a MUL gate masks, opens (sum over the party rows in registers) and
// combines in one pass, and the MAC-check terms of its opened values are
// accumulated in registers and reduced once per kernel.
//
// Device layout of a circuit: 16-byte gate records {in0 wire, in1 wire, out
// wire, 0} sorted per layer by class (MUL, ADD, SUB, CMUL, CADD; gate order
// within a class), so a gate's class, triple index (MUL rank) and constant
// follow from its record index and a per-layer row of class boundaries;
// constants are stored in record order.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <type_traits>
#include <vector>

#include "dag_kernels.cuh"

namespace spdz {

int launch_check(spdz_ctx *ctx, int final_check);



}  // namespace spdz

using namespace spdz;


namespace spdz {

static void default_plan(spdz_plan &p) {
    memset(&p, 0, sizeof p);
    p.mode = SPDZ_SCHED_FUSED;
    p.block = 256;
    p.use_graph = 1;
}

// Plan choice when the caller passes none (defined by the scheduler).
int scheduler_plan(spdz_ctx *ctx, spdz_dag *dag, spdz_plan *out);

template <class F>
static DagArgs<F> base_args(spdz_ctx *ctx, spdz_dag *dag, const spdz_buf *w) {
    using T = typename F::T;
    DagArgs<F> a{};
    a.rec = dag->d_rec;
    a.kc = (const T *)dag->d_kc;
    a.lay = dag->d_lay;
    a.wv = (T *)w->val; a.wm = (T *)w->mac; a.ws = w->stride;
    const spdz_buf *tb[3] = {&ctx->ta, &ctx->tb, &ctx->tc};
    for (int k = 0; k < 3; ++k) {
        a.tp[2 * k] = (const T *)tb[k]->val;
        a.tp[2 * k + 1] = (const T *)tb[k]->mac;
        a.ts[2 * k] = a.ts[2 * k + 1] = tb[k]->stride;
    }
    a.ds = ctx->ds;
    return a;
}

static int occupancy(const void *kern, int block, size_t smem = 0) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, smem) != cudaSuccess) occ = 1;
    return occ < 1 ? 1 : occ;
}

// Launches the tagged kernel over layers [l0, l1) (p61 only); *grid_out is
// its grid, for the barrier count.  Returns 0 or a status.
template <class F, int NP>
static int launch_tagged(spdz_ctx *ctx, spdz_dag *dag, const spdz_plan &plan, DagArgs<F> a, int block, int l0, int l1,
                         uint32_t bar_base, bool final_check, int ctas_per_sm, cudaStream_t s, int *grid_out) {
    if constexpr (std::is_same_v<F, F61>) {
        auto kern = k_dag_tagged<NP>;
        const size_t smem = tagged_smem<NP>(block);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess)
                return set_err(ctx, SPDZ_ERR_CUDA, "tagged kernel shared memory (%zu bytes): %s", smem, cudaGetErrorString(e));
        }
        // every CTA must be resident (gates wait on gates of other CTAs)
        const int occ = occupancy((const void *)kern, block, smem);
        int cpsm = ctas_per_sm;
        if (cpsm <= 0 || cpsm > occ) cpsm = occ;
        int64_t wmax = 1;
        for (int l = l0; l < l1; ++l) wmax = std::max<int64_t>(wmax, dag->lay[l].s[5] - dag->lay[l].s[0]);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)cpsm * ctx->sm_count, (wmax + 31) / 32));
        a.mir = dag->d_mir;
        // the first group copies the inputs into the tagged copy; a later group
        // reads whatever earlier groups finished from the party-major wires
        a.n_in = l0 == 0 ? dag->n_inputs : 0;
        a.wbase = l0 == 0 ? 0 : (uint64_t)(dag->n_inputs + dag->lay[l0].s[0]);
        a.poll_ns = plan.poll_ns ? plan.poll_ns : 128u;
        a.slack = std::min<uint32_t>(plan.barrier_slack, (uint32_t)grid);
        a.bar_base = bar_base;
        a.final_check = final_check ? 1 : 0;
        a.l0 = l0;
        a.l1 = l1;
        // a programmatic dependent launch: its CTAs are scheduled while the
        // kernel before it (the run's begin kernel) finishes, and wait for it
        // in the kernel
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)block);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a); e != cudaSuccess)
            return set_err(ctx, SPDZ_ERR_CUDA, "tagged circuit launch: %s", cudaGetErrorString(e));
        *grid_out = grid;
        return SPDZ_OK;
    } else {
        return set_err(ctx, SPDZ_ERR_ARG, "tagged execution needs p = 2^61-1");
    }
}

// Records a timing event on s: while s is being captured, as an external
// record (an event node of the graph, recorded at every replay); otherwise
// as a plain record.
static void record_timing_event(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    else cudaEventRecord(ev, s);
}

// Enqueues every kernel of one run on stream s (begin, layers, checks).
// Returns the number of launches, or -status.
template <class F, int NP>
static int enqueue_run(spdz_ctx *ctx, spdz_dag *dag, const spdz_plan &plan, const spdz_buf *w, cudaStream_t s,
                       uint64_t tri_base, bool layer_events, uint32_t df_tag) {
    int launches = 0;
    k_run_begin<<<1, 1, 0, s>>>(ctx->ds, tri_base, df_tag);
    ++launches;
    if (dag->time_kernels) record_timing_event(dag->kev0, s);
    const int block = plan.block > 0 ? plan.block : 256;
    DagArgs<F> a = base_args<F>(ctx, dag, w);
    a.spin_ns = (uint64_t)(plan.spin_limit_us ? plan.spin_limit_us : 200000u) * 1000ull;
    a.extra_arrivals = plan.barrier_extra_arrivals > 0 ? (uint32_t)plan.barrier_extra_arrivals : 0u;
    a.test_unwritten_tag = plan.test_unwritten_tag != 0;
    cudaStream_t saved = ctx->stream;
    ctx->stream = s;
    bool checked = false;       // a tagged last group ran the final check
    if (plan.mode == SPDZ_SCHED_PER_LAYER) {
        auto kern = k_dag_segment<F, NP>;
        const int cap = occupancy((const void *)kern, block) * ctx->sm_count;
        for (int l = 0; l < dag->depth; ++l) {
            if (layer_events) cudaEventRecord(dag->lev[l], s);
            // one launch for the MUL gates, one for the linear gates
            const int32_t segs[3] = {dag->lay[l].s[0], dag->lay[l].s[1], dag->lay[l].s[5]};
            a.l0 = l;
            for (int c = 0; c < 2; ++c) {
                a.r0 = segs[c];
                a.r1 = segs[c + 1];
                if (a.r1 <= a.r0) continue;
                int grid = (int)std::min<int64_t>((a.r1 - a.r0 + block - 1) / block, cap);
                kern<<<grid, block, 0, s>>>(a);
                ++launches;
                if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) {
                    ctx->stream = saved;
                    return -set_err(ctx, SPDZ_ERR_CUDA, "per-layer launch: %s", cudaGetErrorString(e));
                }
            }
        }
        if (layer_events) cudaEventRecord(dag->lev[dag->depth], s);
    } else if (plan.mode == SPDZ_SCHED_TAGGED) {
        a.record_ts = layer_events ? 1 : 0;
        int grid = 0;
        if (int rc = launch_tagged<F, NP>(ctx, dag, plan, a, block, 0, dag->depth, 0, true, plan.ctas_per_sm, s, &grid)) {
            ctx->stream = saved;
            return -rc;
        }
        ++launches;
    } else {
        auto kern = F::WORDS == 1 ? k_dag_fused<F, NP> : k_dag_fused_wide<F, NP>;
        const int ng = plan.n_groups > 0 ? plan.n_groups : 1;
        uint32_t bar_base = 0;
        int l0 = 0;
        a.record_ts = layer_events ? 1 : 0;
        for (int g = 0; g < ng; ++g) {
            const int l1 = plan.n_groups > 0 ? plan.group_end[g] : dag->depth;
            const int ncl = plan.n_groups > 0 ? plan.group_cluster[g] : 0;
            const int gblock = plan.n_groups > 0 && plan.group_block[g] > 0 ? plan.group_block[g] : block;
            const size_t smem = fused_smem<F, NP>(gblock);
            if (plan.n_groups > 0 && plan.group_tagged[g]) {
                // a tagged group: fence-free barriers over the tagged copy
                int grid = 0;
                const int cpsm = plan.group_ctas_per_sm[g] > 0 ? plan.group_ctas_per_sm[g] : plan.ctas_per_sm;
                // the last group's last CTA runs the run's MAC check itself
                const bool last = g + 1 == ng;
                checked = checked || last;
                if (int rc = launch_tagged<F, NP>(ctx, dag, plan, a, gblock, l0, l1, bar_base, last, cpsm, s, &grid)) {
                    ctx->stream = saved;
                    return -rc;
                }
                ++launches;
                const int nbar = (l1 - l0 - 1) + (layer_events ? 1 : 0);
                bar_base += (uint32_t)grid * (uint32_t)nbar;
                if (g + 1 < ng && plan.group_flush[g]) {
                    if (int rc = launch_check(ctx, 0)) {
                        ctx->stream = saved;
                        return -rc;
                    }
                    ++launches;
                }
                l0 = l1;
                continue;
            }
            if (ncl > 0) {
                // the whole group inside one cluster of ncl CTAs
                auto ck = k_dag_cluster<F, NP>;
                static bool cattr = false;   // one flag per <F, NP> instantiation
                if (!cattr) {
                    cudaFuncSetAttribute((const void *)ck, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
                    cattr = true;
                }
                if (smem > 48 * 1024)
                    cudaFuncSetAttribute((const void *)ck, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                a.l0 = l0;
                a.l1 = l1;
                cudaLaunchConfig_t cfg{};
                cfg.gridDim = dim3((unsigned)ncl);
                cfg.blockDim = dim3((unsigned)gblock);
                cfg.dynamicSmemBytes = smem;
                cfg.stream = s;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = (unsigned)ncl;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                cudaError_t e = cudaLaunchKernelEx(&cfg, ck, a);
                ++launches;
                if (e != cudaSuccess) {
                    ctx->stream = saved;
                    return -set_err(ctx, SPDZ_ERR_CUDA, "cluster circuit launch (%d CTAs): %s", ncl, cudaGetErrorString(e));
                }
                if (g + 1 < ng && plan.group_flush[g]) {
                    if (int rc = launch_check(ctx, 0)) {
                        ctx->stream = saved;
                        return -rc;
                    }
                    ++launches;
                }
                l0 = l1;
                continue;
            }
            if (smem > 48 * 1024) {
                cudaError_t e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) {
                    ctx->stream = saved;
                    return -set_err(ctx, SPDZ_ERR_CUDA, "fused kernel shared memory (%zu bytes): %s", smem, cudaGetErrorString(e));
                }
            }
            const int occ = occupancy((const void *)kern, gblock, smem);
            int cpsm = plan.group_ctas_per_sm[g] > 0 ? plan.group_ctas_per_sm[g] : plan.ctas_per_sm;
            if (cpsm <= 0 || cpsm > occ) cpsm = occ;
            // no more CTAs than the widest layer of the group has 32-gate tiles
            int64_t wmax = 1;
            for (int l = l0; l < l1; ++l) wmax = std::max<int64_t>(wmax, dag->lay[l].s[5] - dag->lay[l].s[0]);
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)cpsm * ctx->sm_count,
                                                                         (wmax + 31) / 32));
            a.l0 = l0;
            a.l1 = l1;
            a.bar_base = bar_base;
            kern<<<grid, gblock, smem, s>>>(a);
            ++launches;
            if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) {
                ctx->stream = saved;
                return -set_err(ctx, SPDZ_ERR_CUDA, "fused circuit launch: %s", cudaGetErrorString(e));
            }
            const int nbar = (l1 - l0 - 1) + (layer_events ? 1 : 0);
            bar_base += (uint32_t)grid * (uint32_t)nbar;
            if (g + 1 < ng && plan.group_flush[g]) {
                if (int rc = launch_check(ctx, 0)) {
                    ctx->stream = saved;
                    return -rc;
                }
                ++launches;
            }
            l0 = l1;
        }
    }
    // the tagged kernel finishes with the run's check itself
    if (plan.mode != SPDZ_SCHED_TAGGED && !checked) {
        int rc = launch_check(ctx, 1);
        ++launches;
        if (rc) {
            ctx->stream = saved;
            return -rc;
        }
    }
    if (dag->time_kernels) record_timing_event(dag->kev1, s);
    ctx->stream = saved;
    return launches;
}

static int enqueue_dispatch(spdz_ctx *ctx, spdz_dag *dag, const spdz_plan &plan, const spdz_buf *w, cudaStream_t s,
                            uint64_t tri_base, bool layer_events, uint32_t df_tag) {
    int r = -SPDZ_ERR_ARG;
    SPDZ_FIELD_SWITCH(ctx->field, SPDZ_NP_SWITCH(ctx->n, r = (enqueue_run<F, NP>(ctx, dag, plan, w, s, tri_base, layer_events, df_tag))));
    return r;
}

static bool same_plan(const spdz_plan &a, const spdz_plan &b) { return memcmp(&a, &b, sizeof a) == 0; }

static int validate_plan(spdz_ctx *ctx, spdz_dag *dag, const spdz_plan &p) {
    if (p.mode != SPDZ_SCHED_PER_LAYER && p.mode != SPDZ_SCHED_FUSED && p.mode != SPDZ_SCHED_TAGGED)
        return set_err(ctx, SPDZ_ERR_ARG, "plan: bad mode");
    if (p.mode == SPDZ_SCHED_TAGGED) {
        if (dag->field != SPDZ_F61) return set_err(ctx, SPDZ_ERR_ARG, "plan: tagged mode needs p = 2^61-1");
        if (p.n_groups != 0) return set_err(ctx, SPDZ_ERR_ARG, "plan: tagged mode has no layer groups");
        if (p.poll_ns > 50000) return set_err(ctx, SPDZ_ERR_ARG, "plan: poll_ns above 50 us");
        if (p.barrier_extra_arrivals != 0) return set_err(ctx, SPDZ_ERR_ARG, "plan: tagged mode has no extra arrivals");
    }
    if (p.poll_ns > 50000) return set_err(ctx, SPDZ_ERR_ARG, "plan: poll_ns above 50 us");
    if (p.test_unwritten_tag != 0 && (p.mode != SPDZ_SCHED_TAGGED || p.test_unwritten_tag != 1))
        return set_err(ctx, SPDZ_ERR_ARG, "plan: test_unwritten_tag is 0 or 1, tagged mode only");
    if (p.block != 0 && (p.block < 32 || p.block > 256 || p.block % 32)) return set_err(ctx, SPDZ_ERR_ARG, "plan: block must be 32..256, a multiple of 32");
    if (p.n_groups < 0 || p.n_groups > SPDZ_MAX_GROUPS) return set_err(ctx, SPDZ_ERR_ARG, "plan: bad group count");
    if (p.barrier_extra_arrivals < 0 || p.barrier_extra_arrivals > 1024) return set_err(ctx, SPDZ_ERR_ARG, "plan: bad extra arrivals");
    for (int g = 0; g < p.n_groups; ++g) {
        if (p.group_cluster[g] < 0 || p.group_cluster[g] > 16 || (p.group_cluster[g] > 0 && p.mode != SPDZ_SCHED_FUSED))
            return set_err(ctx, SPDZ_ERR_ARG, "plan: cluster size must be 0..16 (fused mode)");
        if (p.group_tagged[g] != 0 && (p.group_tagged[g] != 1 || p.mode != SPDZ_SCHED_FUSED || p.group_cluster[g] != 0 ||
                                       dag->field != SPDZ_F61))
            return set_err(ctx, SPDZ_ERR_ARG, "plan: a tagged group is 1, fused mode, no cluster, p = 2^61-1");
        const int b = p.group_block[g];
        if (b != 0 && (b < 32 || b > 256 || b % 32)) return set_err(ctx, SPDZ_ERR_ARG, "plan: group block must be 32..256, a multiple of 32");
    }
    int prev = 0;
    for (int g = 0; g < p.n_groups; ++g) {
        if (p.group_end[g] <= prev || p.group_end[g] > dag->depth) return set_err(ctx, SPDZ_ERR_ARG, "plan: group ends must increase");
        prev = p.group_end[g];
    }
    if (p.n_groups > 0 && prev != dag->depth) return set_err(ctx, SPDZ_ERR_ARG, "plan: last group must end at depth");
    return SPDZ_OK;
}

}  // namespace spdz

extern "C" {

int spdz_dag_create(spdz_ctx *ctx, const spdz_dag_desc *d, spdz_dag **out) {
    if (!ctx || !d || !out) return set_err(ctx, SPDZ_ERR_ARG, "dag_create: null argument");
    *out = nullptr;
    if (d->n_inputs < 0 || d->n_gates < 0 || d->depth < 0 || !d->layer_offsets ||
        (d->n_gates > 0 && (!d->ops || !d->in0 || !d->in1 || !d->kconst)))
        return set_err(ctx, SPDZ_ERR_ARG, "dag_create: bad descriptor");
    if (d->n_gates >= (int64_t)INT32_MAX || d->n_inputs + d->n_gates > (int64_t)UINT32_MAX || d->depth > 1020)
        return set_err(ctx, SPDZ_ERR_ARG, "dag_create: circuit too large");
    const int64_t *off = d->layer_offsets;
    if (off[0] != 0 || off[d->depth] != d->n_gates)
        return set_err(ctx, SPDZ_ERR_ARG, "dag_create: layer offsets must span the gates");
    for (int l = 0; l < d->depth; ++l)
        if (off[l + 1] < off[l]) return set_err(ctx, SPDZ_ERR_ARG, "dag_create: layer offsets decrease");
    const size_t eb = elem_bytes(ctx->field);
    spdz_dag *g = new spdz_dag();
    g->ctx = ctx;
    g->field = ctx->field;
    g->n = ctx->n;
    g->n_inputs = d->n_inputs;
    g->n_gates = d->n_gates;
    g->depth = d->depth;
    std::vector<uint4> rec((size_t)d->n_gates);
    std::vector<unsigned char> kc((size_t)d->n_gates * eb, 0);
    g->lay.assign(d->depth, LayerRow{});
    g->counts.assign((size_t)d->depth * 5, 0);
    // records per layer in class order MUL, ADD, SUB, CMUL, CADD (gate order
    // within a class); MUL ranks follow gate order, so a layer's MUL ranks are
    // consecutive and start at the number of MUL gates in earlier layers
    static const int cls_op[5] = {SPDZ_OP_MUL, SPDZ_OP_ADD, SPDZ_OP_SUB, SPDZ_OP_CMUL, SPDZ_OP_CADD};
    size_t pos = 0;
    int64_t mul_before = 0;
    for (int l = 0; l < d->depth; ++l) {
        const uint64_t limit = (uint64_t)d->n_inputs + (uint64_t)off[l];   // wires written before layer l
        LayerRow &L = g->lay[l];
        L.mulbase = (int32_t)mul_before;
        for (int c = 0; c < 5; ++c) {
            L.s[c] = (int32_t)pos;
            for (int64_t i = off[l]; i < off[l + 1]; ++i) {
                const uint8_t op = d->ops[i];
                if (op > SPDZ_OP_MUL) {
                    spdz_dag_destroy(g);
                    return set_err(ctx, SPDZ_ERR_ARG, "dag_create: gate %lld has bad op", (long long)i);
                }
                if (op != cls_op[c]) continue;
                const bool binary = op == SPDZ_OP_ADD || op == SPDZ_OP_SUB || op == SPDZ_OP_MUL;
                if (d->in0[i] >= limit || (binary && d->in1[i] >= limit)) {
                    spdz_dag_destroy(g);
                    return set_err(ctx, SPDZ_ERR_ARG, "dag_create: gate %lld reads a wire not written before its layer",
                                   (long long)i);
                }
                rec[pos] = make_uint4(d->in0[i], binary ? d->in1[i] : d->in0[i], (uint32_t)(d->n_inputs + i), 0u);
                if (op == SPDZ_OP_CMUL || op == SPDZ_OP_CADD)
                    host_to_dev_elem(ctx->field, (const unsigned char *)d->kconst + (size_t)i * host_elem_bytes(ctx->field),
                                     &kc[pos * eb]);
                ++pos;
                g->counts[(size_t)l * 5 + c]++;
            }
        }
        L.s[5] = (int32_t)pos;
        mul_before += L.s[1] - L.s[0];
    }
    g->n_mul = mul_before;
    int rc = SPDZ_OK;
    if (cudaMalloc(&g->d_rec, std::max<size_t>(16, rec.size() * 16)) != cudaSuccess ||
        cudaMalloc(&g->d_lay, std::max<size_t>(32, (size_t)d->depth * sizeof(LayerRow))) != cudaSuccess ||
        cudaMalloc(&g->d_kc, std::max<size_t>(16, kc.size())) != cudaSuccess) {
        spdz_dag_destroy(g);
        return set_err(ctx, SPDZ_ERR_OOM, "dag_create: device allocation failed");
    }
    if ((rc = check_cuda(ctx, cudaMemcpy(g->d_rec, rec.data(), rec.size() * 16, cudaMemcpyHostToDevice), "dag upload")) ||
        (rc = check_cuda(ctx, cudaMemcpy(g->d_lay, g->lay.data(), (size_t)d->depth * sizeof(LayerRow), cudaMemcpyHostToDevice), "dag upload")) ||
        (rc = check_cuda(ctx, cudaMemcpy(g->d_kc, kc.data(), kc.size(), cudaMemcpyHostToDevice), "dag upload"))) {
        spdz_dag_destroy(g);
        return rc;
    }
    cudaEventCreate(&g->ev0);
    cudaEventCreate(&g->ev1);
    g->lev.resize(d->depth + 1);
    for (auto &e : g->lev) cudaEventCreate(&e);
    g->layer_us.assign(d->depth, 0.f);
    *out = g;
    return SPDZ_OK;
}

int spdz_dag_destroy(spdz_dag *g) {
    if (!g) return SPDZ_OK;
    cudaDeviceSynchronize();
    sched_forget(g->ctx, g);
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->kev0) cudaEventDestroy(g->kev0);
    if (g->kev1) cudaEventDestroy(g->kev1);
    if (g->d_rec) cudaFree(g->d_rec);
    if (g->d_lay) cudaFree(g->d_lay);
    if (g->d_kc) cudaFree(g->d_kc);
    if (g->d_mir) cudaFree(g->d_mir);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    for (auto &e : g->lev) cudaEventDestroy(e);
    delete g;
    return SPDZ_OK;
}

int spdz_dag_time_kernels(spdz_dag *dag, int32_t on) {
    if (!dag) return SPDZ_ERR_ARG;
    if (on && !dag->kev0) {
        if (cudaEventCreate(&dag->kev0) != cudaSuccess || cudaEventCreate(&dag->kev1) != cudaSuccess)
            return set_err(dag->ctx, SPDZ_ERR_CUDA, "dag_time_kernels: event creation failed");
    }
    dag->time_kernels = on != 0;
    return SPDZ_OK;
}

int spdz_dag_kernel_ms(spdz_dag *dag, float *ms) {
    if (!dag || !ms) return SPDZ_ERR_ARG;
    if (!dag->kev0) return set_err(dag->ctx, SPDZ_ERR_STATE, "dag_kernel_ms: kernel timing was never enabled");
    if (cudaEventSynchronize(dag->kev1) != cudaSuccess || cudaEventElapsedTime(ms, dag->kev0, dag->kev1) != cudaSuccess)
        return set_err(dag->ctx, SPDZ_ERR_CUDA, "dag_kernel_ms: no timed run has completed");
    return SPDZ_OK;
}

int spdz_run_dag(spdz_ctx *ctx, spdz_dag *dag, const spdz_plan *plan_in, const spdz_buf *wires, spdz_stats *stats) {
    if (!ctx || !dag || !wires) return set_err(ctx, SPDZ_ERR_ARG, "run_dag: null argument");
    if (dag->ctx != ctx && (dag->field != ctx->field || dag->n != ctx->n))
        return set_err(ctx, SPDZ_ERR_ARG, "run_dag: circuit built for another field or party count");
    if (!ctx->alpha_loaded) return set_err(ctx, SPDZ_ERR_STATE, "run_dag: preprocessing not loaded");
    if (ctx->opened != 0) return set_err(ctx, SPDZ_ERR_STATE, "run_dag: values opened since the last check");
    int rc = validate_buf(ctx, wires, dag->n_inputs + dag->n_gates, "run_dag.wires");
    if (rc) return rc;
    if (ctx->tri_total - ctx->tri_cursor < dag->n_mul)
        return set_err(ctx, SPDZ_ERR_TRIPLES, "run_dag: need %lld triples, %lld left", (long long)dag->n_mul,
                       (long long)(ctx->tri_total - ctx->tri_cursor));
    spdz_plan plan;
    if (plan_in) {
        plan = *plan_in;
    } else if (scheduler_plan(ctx, dag, &plan) != SPDZ_OK) {
        default_plan(plan);
    }
    if ((rc = validate_plan(ctx, dag, plan))) return rc;
    const uint64_t tri_base = (uint64_t)ctx->tri_cursor;
    const bool layer_events = plan.record_layer_times != 0;
    if (stats) cudaEventRecord(dag->ev0, ctx->stream);
    // tagged: the tagged copy (allocated on first use), the run's tag, and
    // the copy zeroed before the first run of every cycle of 7 tags
    uint32_t df_tag = 0;
    bool tags = plan.mode == SPDZ_SCHED_TAGGED;
    for (int g = 0; g < plan.n_groups; ++g) tags = tags || plan.group_tagged[g] != 0;
    if (tags) {
        const size_t need = (size_t)(dag->n_inputs + dag->n_gates) * 2 * (size_t)dag->n * sizeof(uint64_t);
        if (!dag->d_mir) {
            if (cudaMalloc(&dag->d_mir, std::max<size_t>(need, 16)) != cudaSuccess) {
                dag->d_mir = nullptr;
                return set_err(ctx, SPDZ_ERR_OOM, "run_dag: tagged wire copy (%zu bytes)", need);
            }
            dag->mir_bytes = need;
            dag->df_runs = 0;
        }
        df_tag = (uint32_t)(dag->df_runs % 7) + 1;
        ++dag->df_runs;
        if (df_tag == 1 && (rc = check_cuda(ctx, cudaMemsetAsync(dag->d_mir, 0, dag->mir_bytes, ctx->stream), "zero wire copy")))
            return rc;
    }
    int launches = 0;
    if (plan.use_graph && !layer_events) {
        const bool reuse = dag->gexec && same_plan(dag->gplan, plan) && dag->gwires.val == wires->val &&
                           dag->gwires.mac == wires->mac && dag->gwires.stride == wires->stride &&
                           dag->gtimed == dag->time_kernels;
        if (!reuse) {
            if (dag->gexec) { cudaGraphExecDestroy(dag->gexec); dag->gexec = nullptr; }
            if (dag->graph) { cudaGraphDestroy(dag->graph); dag->graph = nullptr; }
            if (!dag->cap_stream && (rc = check_cuda(ctx, cudaStreamCreateWithFlags(&dag->cap_stream, cudaStreamNonBlocking), "stream")))
                return rc;
            cudaGraph_t graph;
            if ((rc = check_cuda(ctx, cudaStreamBeginCapture(dag->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture")))
                return rc;
            int n = enqueue_dispatch(ctx, dag, plan, wires, dag->cap_stream, tri_base, false, df_tag);
            cudaError_t ce = cudaStreamEndCapture(dag->cap_stream, &graph);
            if (n < 0) return -n;
            if ((rc = check_cuda(ctx, ce, "end capture"))) return rc;
            size_t nroots = 1;
            cudaGraphNode_t root;
            if ((rc = check_cuda(ctx, cudaGraphGetRootNodes(graph, &root, &nroots), "graph roots")) ||
                (rc = check_cuda(ctx, cudaGraphKernelNodeGetParams(root, &dag->gbegin_params), "begin node"))) {
                cudaGraphDestroy(graph);
                return rc;
            }
            rc = check_cuda(ctx, cudaGraphInstantiate(&dag->gexec, graph, 0), "graph instantiate");
            if (rc) {
                cudaGraphDestroy(graph);
                return rc;
            }
            dag->graph = graph;   // kept alive: the begin node is updated through it
            dag->gbegin = root;
            dag->gplan = plan;
            dag->gwires = *wires;
            dag->glaunches = n;
            dag->gtimed = dag->time_kernels;
        }
        DevState *ds = ctx->ds;
        uint64_t tb = tri_base;
        uint32_t tg = df_tag;
        void *args[3] = {&ds, &tb, &tg};
        cudaKernelNodeParams kp = dag->gbegin_params;
        kp.kernelParams = args;
        kp.extra = nullptr;
        if ((rc = check_cuda(ctx, cudaGraphExecKernelNodeSetParams(dag->gexec, dag->gbegin, &kp), "update begin node")) ||
            (rc = check_cuda(ctx, cudaGraphLaunch(dag->gexec, ctx->stream), "graph launch")))
            return rc;
        launches = dag->glaunches;
    } else {
        int n = enqueue_dispatch(ctx, dag, plan, wires, ctx->stream, tri_base, layer_events, df_tag);
        if (n < 0) return -n;
        launches = n;
    }
    ctx->tri_cursor += dag->n_mul;
    ctx->epoch += 1;
    if (!stats) return SPDZ_OK;
    cudaEventRecord(dag->ev1, ctx->stream);
    if ((rc = check_cuda(ctx, cudaMemcpyAsync(ctx->hres, ctx->ds, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream), "readback")) ||
        (rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "run sync")))
        return rc;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, dag->ev0, dag->ev1);
    stats->device_ms = ms;
    stats->passed = (int32_t)ctx->hres->res_passed;
    stats->launches = launches;
    stats->n_gates = dag->n_gates;
    stats->n_mul = dag->n_mul;
    if (layer_events) {
        if (plan.mode == SPDZ_SCHED_PER_LAYER) {
            for (int l = 0; l < dag->depth; ++l) cudaEventElapsedTime(&dag->layer_us[l], dag->lev[l], dag->lev[l + 1]);
            for (auto &v : dag->layer_us) v *= 1000.f;
        } else {
            for (int l = 0; l < dag->depth; ++l)
                dag->layer_us[l] = (float)((double)(ctx->hres->layer_ts[l + 1] - ctx->hres->layer_ts[l]) * 1e-3);
        }
    }
    if (ctx->hres->err_flags & ERR_TIMEOUT) return set_err(ctx, SPDZ_ERR_TIMEOUT, "run_dag: a device wait timed out");
    if (!stats->passed) return set_err(ctx, SPDZ_ERR_MAC, "run_dag: MAC check failed");
    return SPDZ_OK;
}

int spdz_run_dag_host(spdz_ctx *ctx, spdz_dag *dag, const spdz_plan *plan, const spdz_buf *wires,
                      const void *in_val_host, const void *in_mac_host, const void *const *tri_host, int64_t out_first,
                      int64_t out_count, void *out_val_host, void *out_mac_host) {
    if (!ctx || !dag || !wires) return set_err(ctx, SPDZ_ERR_ARG, "run_dag_host: null argument");
    if (ctx->field == SPDZ_F32)
        return set_err(ctx, SPDZ_ERR_ARG, "run_dag_host: host and device element formats differ for p = 2^32-5");
    const int n = ctx->n;
    const int64_t nin = dag->n_inputs, nm = dag->n_mul, W = dag->n_inputs + dag->n_gates;
    if (nin > 0 && (!in_val_host || !in_mac_host)) return set_err(ctx, SPDZ_ERR_ARG, "run_dag_host: no input shares");
    if (nm > 0) {
        if (!tri_host) return set_err(ctx, SPDZ_ERR_ARG, "run_dag_host: no triples");
        for (int k = 0; k < 6; ++k)
            if (!tri_host[k]) return set_err(ctx, SPDZ_ERR_ARG, "run_dag_host: triple array %d is null", k);
    }
    if (out_first < 0 || out_count < 0 || out_first + out_count > W ||
        (out_count > 0 && (!out_val_host || !out_mac_host)))
        return set_err(ctx, SPDZ_ERR_ARG, "run_dag_host: bad output range");
    int rc = validate_buf(ctx, wires, W, "run_dag_host.wires");
    if (rc) return rc;
    if (!ctx->alpha_loaded || !ctx->pool_ev) return set_err(ctx, SPDZ_ERR_STATE, "run_dag_host: preprocessing not loaded");
    if (ctx->opened != 0) return set_err(ctx, SPDZ_ERR_STATE, "run_dag_host: values opened since the last check");
    if (ctx->tri_total - ctx->tri_cursor < nm)
        return set_err(ctx, SPDZ_ERR_TRIPLES, "run_dag_host: need %lld triples, %lld left", (long long)nm,
                       (long long)(ctx->tri_total - ctx->tri_cursor));
    const size_t eb = elem_bytes(ctx->field);
    if (!ctx->copy_stream) {
        if ((rc = check_cuda(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "copy stream")))
            return rc;
        for (auto &e : ctx->copy_ev)
            if ((rc = check_cuda(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "copy event"))) return rc;
    }
    // the run's triples into the pool slots it consumes, on the copy stream
    // (so the next call's copy overlaps this run)
    if (nm > 0) {
        if ((rc = check_cuda(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->pool_ev, 0), "copy wait"))) return rc;
        const spdz_buf *tb[3] = {&ctx->ta, &ctx->tb, &ctx->tc};
        for (int k = 0; k < 6; ++k) {
            const spdz_buf &b = *tb[k / 2];
            char *dst = (char *)(k % 2 == 0 ? b.val : b.mac) + (size_t)ctx->tri_cursor * eb;
            if ((rc = check_cuda(ctx, cudaMemcpy2DAsync(dst, (size_t)b.stride * eb, tri_host[k], (size_t)nm * eb,
                                                         (size_t)nm * eb, (size_t)n, cudaMemcpyHostToDevice,
                                                         ctx->copy_stream), "triple copy")))
                return rc;
        }
    }
    cudaEvent_t ev = ctx->copy_ev[ctx->copy_k];
    ctx->copy_k = (ctx->copy_k + 1) % 4;
    if ((rc = check_cuda(ctx, cudaEventRecord(ev, ctx->copy_stream), "copy event"))) return rc;
    // the inputs, on the run's stream (after any earlier run that reads them)
    if (nin > 0) {
        if ((rc = check_cuda(ctx, cudaMemcpy2DAsync(wires->val, (size_t)wires->stride * eb, in_val_host, (size_t)nin * eb,
                                                     (size_t)nin * eb, (size_t)n, cudaMemcpyHostToDevice, ctx->stream),
                             "input copy")) ||
            (rc = check_cuda(ctx, cudaMemcpy2DAsync(wires->mac, (size_t)wires->stride * eb, in_mac_host, (size_t)nin * eb,
                                                     (size_t)nin * eb, (size_t)n, cudaMemcpyHostToDevice, ctx->stream),
                             "input copy")))
            return rc;
    }
    if ((rc = check_cuda(ctx, cudaStreamWaitEvent(ctx->stream, ev, 0), "copy wait"))) return rc;
    if ((rc = spdz_run_dag(ctx, dag, plan, wires, nullptr))) return rc;
    if (out_count > 0) {
        const size_t off = (size_t)out_first * eb;
        if ((rc = check_cuda(ctx, cudaMemcpy2DAsync(out_val_host, (size_t)out_count * eb, (const char *)wires->val + off,
                                                     (size_t)wires->stride * eb, (size_t)out_count * eb, (size_t)n,
                                                     cudaMemcpyDeviceToHost, ctx->stream), "output copy")) ||
            (rc = check_cuda(ctx, cudaMemcpy2DAsync(out_mac_host, (size_t)out_count * eb, (const char *)wires->mac + off,
                                                     (size_t)wires->stride * eb, (size_t)out_count * eb, (size_t)n,
                                                     cudaMemcpyDeviceToHost, ctx->stream), "output copy")))
            return rc;
    }
    return SPDZ_OK;
}

int spdz_check_result(spdz_ctx *ctx, int *passed, void *sigma_host) {
    if (!ctx || !passed) return set_err(ctx, SPDZ_ERR_ARG, "check_result: null argument");
    int rc;
    if ((rc = check_cuda(ctx, cudaMemcpyAsync(ctx->hres, ctx->ds, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream), "readback")) ||
        (rc = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync")))
        return rc;
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
    if (ctx->hres->err_flags & ERR_TIMEOUT) return set_err(ctx, SPDZ_ERR_TIMEOUT, "a device barrier wait timed out");
    return *passed ? SPDZ_OK : set_err(ctx, SPDZ_ERR_MAC, "MAC check failed");
}

int spdz_dag_layer_times(const spdz_dag *dag, float *us_out) {
    if (!dag || !us_out) return SPDZ_ERR_ARG;
    std::copy(dag->layer_us.begin(), dag->layer_us.end(), us_out);
    return SPDZ_OK;
}

int spdz_dag_layer_counts(const spdz_dag *dag, int32_t *counts_out) {
    if (!dag || !counts_out) return SPDZ_ERR_ARG;
    std::copy(dag->counts.begin(), dag->counts.end(), counts_out);
    return SPDZ_OK;
}

}  // extern "C"
