// sched.cu -- execution plans for circuit runs (the batch-size and slicing
// autotuning the paper leaves to future work, Sec. V-D).
//
// Two schedulers produce a spdz_plan for a circuit; neither changes any
// result bit (every plan computes the same shares):
//   * the autotuner runs the circuit under each candidate configuration as a
//     single group and keeps the fastest measured one;
//   * the learned planner predicts the device time of every layer under every
//     configuration with the cost model (an MLP trained on the GPU on
//     per-layer timings the pipeline records itself) and picks group
//     boundaries and a configuration per group by dynamic programming, with a
//     measured cost for each extra group (kernel switch).
// spdz_sched_choose measures the default, autotuned and learned plans (and,
// for p = 2^61-1, the tagged plan) and keeps the fastest: the
// autotuned plan is the learned plan's fallback and the judge of its
// makespan error.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "dag.cuh"

namespace spdz {

// Candidate configurations of one layer group.
struct GroupConfig {
    int cluster;   // 0: whole grid with device barriers; k: one cluster of k CTAs
    int block;     // threads per CTA
    int cpsm;      // CTAs per SM (grid groups)
    int tagged;    // 1: the tagged kernel (p = 2^61-1 only; fence-free barriers, slack 1/12 of the CTAs)
};
constexpr GroupConfig kConfigs[] = {
    {0, 256, 2, 0}, {0, 256, 1, 0}, {0, 128, 4, 0}, {0, 128, 2, 0}, {16, 256, 0, 0}, {8, 256, 0, 0}, {16, 128, 0, 0},
    {0, 256, 2, 1},
};
constexpr int NCFG = (int)(sizeof(kConfigs) / sizeof(kConfigs[0]));
constexpr int NFEAT = 6 + NCFG;
constexpr int DEFAULT_CFG = 0;

struct Sched {
    spdz_mlp *model = nullptr;
    bool trained = false;
    float train_loss = -1.f;
    std::vector<float> X, Y;          // samples: features, ln(layer microseconds)
    double switch_us = 3.0;           // measured cost of one extra group
    bool switch_measured = false;
    std::unordered_map<const spdz_dag *, spdz_plan> chosen;
    double last_tagged_ms = -1;       // the autotuner's measure of the uniform tagged configuration
    float *dX = nullptr, *dY = nullptr;
    int64_t dcap = 0;
};

static Sched *sched_of(spdz_ctx *ctx) {
    if (!ctx->sched) ctx->sched = new Sched();
    return (Sched *)ctx->sched;
}

void sched_destroy(spdz_ctx *ctx) {
    Sched *s = (Sched *)ctx->sched;
    if (!s) return;
    if (s->model) spdz_mlp_destroy(s->model);
    if (s->dX) cudaFree(s->dX);
    if (s->dY) cudaFree(s->dY);
    delete s;
    ctx->sched = nullptr;
}

static void layer_features(const spdz_dag *dag, int l, int cfg, float *f) {
    const int32_t *c = &dag->counts[(size_t)l * 5];
    const double w = std::max<int64_t>(1, (int64_t)c[0] + c[1] + c[2] + c[3] + c[4]);
    std::fill(f, f + NFEAT, 0.f);
    f[0] = (float)(std::log2(w) / 16.0);
    f[1] = (float)(c[0] / w);
    f[2] = (float)((c[1] + c[2]) / w);
    f[3] = (float)((c[3] + c[4]) / w);
    f[4] = dag->field == SPDZ_F127 ? 1.f : dag->field == SPDZ_F32 ? -1.f : 0.f;
    f[5] = (float)((dag->n - 2) / 6.0);
    f[6 + cfg] = 1.f;
}

// Configuration cfg is available for the circuit's field.
static bool config_ok(const spdz_dag *dag, int cfg) { return !kConfigs[cfg].tagged || dag->field == SPDZ_F61; }

// Barrier slack of tagged groups: a layer starts when all but 1/12 of the
// CTAs (2 per SM) have arrived.
static uint32_t tagged_slack(const spdz_dag *dag) {
    return (uint32_t)(2 * (dag->ctx ? dag->ctx->sm_count : 148) / 12);
}

static void uniform_plan(const spdz_dag *dag, int cfg, spdz_plan &p) {
    memset(&p, 0, sizeof p);
    p.mode = SPDZ_SCHED_FUSED;
    p.block = kConfigs[cfg].block;
    p.ctas_per_sm = kConfigs[cfg].cpsm;
    p.use_graph = 1;
    p.n_groups = 1;
    p.group_end[0] = dag->depth;
    p.group_cluster[0] = kConfigs[cfg].cluster;
    p.group_block[0] = kConfigs[cfg].block;
    p.group_ctas_per_sm[0] = kConfigs[cfg].cpsm;
    p.group_tagged[0] = kConfigs[cfg].tagged;
    if (kConfigs[cfg].tagged) p.barrier_slack = tagged_slack(dag);
}

// Two plans with the same groups and group configurations.
static bool same_groups(const spdz_plan &a, const spdz_plan &b) {
    if (a.mode != b.mode || a.n_groups != b.n_groups || a.barrier_slack != b.barrier_slack) return false;
    for (int g = 0; g < a.n_groups; ++g)
        if (a.group_end[g] != b.group_end[g] || a.group_cluster[g] != b.group_cluster[g] ||
            a.group_block[g] != b.group_block[g] || a.group_ctas_per_sm[g] != b.group_ctas_per_sm[g] ||
            a.group_tagged[g] != b.group_tagged[g] || a.group_flush[g] != b.group_flush[g])
            return false;
    return true;
}

// Median device time (ms) of `reps` runs of the plan, after one warm-up run.
static int measure(spdz_ctx *ctx, spdz_dag *dag, const spdz_plan &p, const spdz_buf *w, int reps, double *ms) {
    spdz_stats st{};
    std::vector<double> t;
    for (int r = 0; r <= reps; ++r) {
        int rc = spdz_run_dag(ctx, dag, &p, w, &st);
        if (rc) return rc;
        if (r > 0) t.push_back(st.device_ms);
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return SPDZ_OK;
}

static int ensure_dev(Sched *s, int64_t rows) {
    if (rows <= s->dcap) return SPDZ_OK;
    if (s->dX) cudaFree(s->dX);
    if (s->dY) cudaFree(s->dY);
    s->dX = s->dY = nullptr;
    if (cudaMalloc(&s->dX, (size_t)rows * NFEAT * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&s->dY, (size_t)rows * sizeof(float)) != cudaSuccess)
        return SPDZ_ERR_OOM;
    s->dcap = rows;
    return SPDZ_OK;
}

// Predicted per-layer microseconds for every configuration: pred[l*NCFG + c].
static int predict_layers(spdz_ctx *ctx, spdz_dag *dag, std::vector<double> &pred) {
    Sched *s = sched_of(ctx);
    if (!s->model || !s->trained) return SPDZ_ERR_STATE;
    const int64_t rows = (int64_t)dag->depth * NCFG;
    std::vector<float> X((size_t)rows * NFEAT), Y((size_t)rows);
    for (int l = 0; l < dag->depth; ++l)
        for (int c = 0; c < NCFG; ++c) layer_features(dag, l, c, &X[((size_t)l * NCFG + c) * NFEAT]);
    if (int rc = ensure_dev(s, rows)) return rc;
    cudaMemcpyAsync(s->dX, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (int rc = spdz_mlp_forward(s->model, s->dX, rows, s->dY)) return rc;
    cudaMemcpyAsync(Y.data(), s->dY, Y.size() * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return SPDZ_ERR_CUDA;
    pred.resize((size_t)rows);
    for (int64_t k = 0; k < rows; ++k) pred[(size_t)k] = std::exp((double)Y[(size_t)k]);
    return SPDZ_OK;
}

// Group boundaries and per-group configurations minimising the predicted
// makespan: dp[l] = min over j < l and c of dp[j] + sum_{k in [j,l)} pred[k][c]
// + switch_us * [j > 0].  At most SPDZ_MAX_GROUPS groups.
static int learned_plan(spdz_ctx *ctx, spdz_dag *dag, spdz_plan &p, double *pred_ms) {
    std::vector<double> pred;
    if (int rc = predict_layers(ctx, dag, pred)) return rc;
    Sched *s = sched_of(ctx);
    const int L = dag->depth;
    std::vector<double> pre((size_t)(L + 1) * NCFG, 0.0);
    for (int l = 0; l < L; ++l)
        for (int c = 0; c < NCFG; ++c) pre[(size_t)(l + 1) * NCFG + c] = pre[(size_t)l * NCFG + c] + pred[(size_t)l * NCFG + c];
    std::vector<double> dp((size_t)L + 1, 1e300);
    std::vector<int> from((size_t)L + 1, -1), cfg((size_t)L + 1, -1), ngr((size_t)L + 1, 0);
    dp[0] = 0.0;
    for (int l = 1; l <= L; ++l)
        for (int j = 0; j < l; ++j) {
            if (ngr[j] >= SPDZ_MAX_GROUPS) continue;
            for (int c = 0; c < NCFG; ++c) {
                if (!config_ok(dag, c)) continue;
                const double v = dp[j] + pre[(size_t)l * NCFG + c] - pre[(size_t)j * NCFG + c] + (j > 0 ? s->switch_us : 0.0);
                if (v < dp[l]) {
                    dp[l] = v;
                    from[l] = j;
                    cfg[l] = c;
                    ngr[l] = ngr[j] + 1;
                }
            }
        }
    std::vector<std::pair<int, int>> groups;   // (end, cfg)
    for (int l = L; l > 0; l = from[l]) groups.push_back({l, cfg[l]});
    std::reverse(groups.begin(), groups.end());
    // Several groups only when their predicted gain over the best single
    // group exceeds the model's error (the square root of its ln-space
    // training loss, at least 10 %): the switches between kernel kinds cost
    // more than the measured switch cost of one kind, and a predicted gain
    // inside the error is not one.
    {
        int best_c = -1;
        double best_uni = 1e300;
        for (int c = 0; c < NCFG; ++c)
            if (config_ok(dag, c) && pre[(size_t)L * NCFG + c] < best_uni) {
                best_uni = pre[(size_t)L * NCFG + c];
                best_c = c;
            }
        const double margin = std::max(0.10, std::sqrt(std::max(0.0, (double)s->train_loss)));
        if (groups.size() > 1 && best_c >= 0 && dp[L] > best_uni * (1.0 - margin)) {
            groups.assign(1, {L, best_c});
            dp[L] = best_uni;
        }
    }
    memset(&p, 0, sizeof p);
    p.mode = SPDZ_SCHED_FUSED;
    p.block = 256;
    p.use_graph = 1;
    p.n_groups = (int)groups.size();
    for (size_t g = 0; g < groups.size(); ++g) {
        const GroupConfig &gc = kConfigs[groups[g].second];
        p.group_end[g] = groups[g].first;
        p.group_cluster[g] = gc.cluster;
        p.group_block[g] = gc.block;
        p.group_ctas_per_sm[g] = gc.cpsm;
        p.group_tagged[g] = gc.tagged;
        if (gc.tagged) p.barrier_slack = tagged_slack(dag);
    }
    // one group: the block size and CTAs per SM of the plan as the autotuner
    // writes them, so that equal plans compare equal
    if (p.n_groups == 1) {
        p.block = p.group_block[0];
        p.ctas_per_sm = p.group_ctas_per_sm[0];
    }
    if (pred_ms) *pred_ms = dp[L] * 1e-3;
    return SPDZ_OK;
}

// Plan for a run without an explicit plan: the plan chosen for this circuit
// by spdz_sched_choose, else the learned plan, else none (the executor then
// uses its fused default).
int scheduler_plan(spdz_ctx *ctx, spdz_dag *dag, spdz_plan *out) {
    Sched *s = (Sched *)ctx->sched;
    if (!s) return SPDZ_ERR_STATE;
    auto it = s->chosen.find(dag);
    if (it != s->chosen.end()) {
        *out = it->second;
        return SPDZ_OK;
    }
    if (s->trained) return learned_plan(ctx, dag, *out, nullptr);
    return SPDZ_ERR_STATE;
}

// Helpers of the serving loop: per-layer predictions of one configuration
// for a circuit described only by its layer counts, and the configurations
// it compares (a single 16-CTA cluster vs the default whole-grid group).
int sched_predict_config(spdz_ctx *ctx, const spdz_dag *dag, int cfg, std::vector<double> &us) {
    std::vector<double> pred;
    if (int rc = predict_layers(ctx, const_cast<spdz_dag *>(dag), pred)) return rc;
    us.resize((size_t)dag->depth);
    for (int l = 0; l < dag->depth; ++l) us[(size_t)l] = pred[(size_t)l * NCFG + cfg];
    return SPDZ_OK;
}
int sched_cluster_config() { return 4; }   // {16, 256, 0}
int sched_cluster_width() { return kConfigs[sched_cluster_config()].cluster; }
int sched_grid_config() { return DEFAULT_CFG; }
double sched_switch_us(spdz_ctx *ctx) { return ctx->sched ? ((Sched *)ctx->sched)->switch_us : 3.0; }

void sched_forget(spdz_ctx *ctx, const spdz_dag *dag) {
    if (ctx && ctx->sched) ((Sched *)ctx->sched)->chosen.erase(dag);
}

}  // namespace spdz

using namespace spdz;

extern "C" {

int spdz_sched_num_configs(int32_t *count, int32_t *n_features) {
    if (count) *count = NCFG;
    if (n_features) *n_features = NFEAT;
    return SPDZ_OK;
}

int spdz_sched_config_plan(const spdz_dag *dag, int32_t cfg, spdz_plan *out) {
    if (!dag || !out || cfg < 0 || cfg >= NCFG) return SPDZ_ERR_ARG;
    uniform_plan(dag, cfg, *out);
    return SPDZ_OK;
}

int spdz_sched_record(spdz_ctx *ctx, spdz_dag *dag, const spdz_buf *wires, int32_t reps) {
    if (!ctx || !dag || !wires || reps < 1) return set_err(ctx, SPDZ_ERR_ARG, "sched_record: bad argument");
    Sched *s = sched_of(ctx);
    const int L = dag->depth;
    std::vector<float> f(NFEAT);
    for (int c = 0; c < NCFG; ++c) {
        if (!config_ok(dag, c)) continue;
        spdz_plan p;
        uniform_plan(dag, c, p);
        p.record_layer_times = 1;
        std::vector<std::vector<float>> t((size_t)L);
        for (int r = 0; r <= reps; ++r) {
            spdz_stats st{};
            if (int rc = spdz_run_dag(ctx, dag, &p, wires, &st)) return rc;
            if (r == 0) continue;   // warm-up
            std::vector<float> us((size_t)L);
            spdz_dag_layer_times(dag, us.data());
            for (int l = 0; l < L; ++l) t[(size_t)l].push_back(us[(size_t)l]);
        }
        for (int l = 0; l < L; ++l) {
            auto &v = t[(size_t)l];
            std::sort(v.begin(), v.end());
            const float med = std::max(0.05f, v[v.size() / 2]);
            layer_features(dag, l, c, f.data());
            s->X.insert(s->X.end(), f.begin(), f.end());
            s->Y.push_back(std::log(med));
        }
    }
    // cost of one extra group: every layer its own group vs one group
    if (!s->switch_measured && L >= 4) {
        spdz_plan one, split;
        uniform_plan(dag, DEFAULT_CFG, one);
        split = one;
        split.n_groups = L;
        for (int l = 0; l < L; ++l) {
            split.group_end[l] = l + 1;
            split.group_block[l] = one.group_block[0];
            split.group_ctas_per_sm[l] = one.group_ctas_per_sm[0];
            split.group_cluster[l] = 0;
        }
        double a = 0, b = 0;
        if (int rc = measure(ctx, dag, one, wires, reps, &a)) return rc;
        if (int rc = measure(ctx, dag, split, wires, reps, &b)) return rc;
        s->switch_us = std::max(0.0, (b - a) * 1e3 / (L - 1));
        s->switch_measured = true;
    }
    return SPDZ_OK;
}

int spdz_sched_samples(spdz_ctx *ctx, float *X_host, float *Y_host, int64_t *count, double *switch_us) {
    if (!ctx || !count) return SPDZ_ERR_ARG;
    Sched *s = sched_of(ctx);
    *count = (int64_t)s->Y.size();
    if (X_host) std::copy(s->X.begin(), s->X.end(), X_host);
    if (Y_host) std::copy(s->Y.begin(), s->Y.end(), Y_host);
    if (switch_us) *switch_us = s->switch_us;
    return SPDZ_OK;
}

int spdz_sched_add_samples(spdz_ctx *ctx, const float *X_host, const float *Y_host, int64_t count) {
    if (!ctx || count < 0 || (count > 0 && (!X_host || !Y_host))) return set_err(ctx, SPDZ_ERR_ARG, "sched_add_samples: bad argument");
    Sched *s = sched_of(ctx);
    s->X.insert(s->X.end(), X_host, X_host + count * NFEAT);
    s->Y.insert(s->Y.end(), Y_host, Y_host + count);
    return SPDZ_OK;
}

int spdz_sched_train(spdz_ctx *ctx, int32_t epochs, float lr, uint64_t seed, float *loss_out) {
    if (!ctx || epochs < 0) return set_err(ctx, SPDZ_ERR_ARG, "sched_train: bad argument");
    Sched *s = sched_of(ctx);
    const int64_t B = (int64_t)s->Y.size();
    if (B == 0) return set_err(ctx, SPDZ_ERR_STATE, "sched_train: no recorded samples");
    if (!s->model) {
        if (int rc = spdz_mlp_create(&s->model, NFEAT, 64, 3, seed, ctx->stream)) return set_err(ctx, rc, "sched_train: model");
    }
    // a fixed shuffle of the samples (counter PRG), so mini-batches mix configurations
    std::vector<int64_t> perm((size_t)B);
    for (int64_t k = 0; k < B; ++k) perm[(size_t)k] = k;
    for (int64_t k = B - 1; k > 0; --k) std::swap(perm[(size_t)k], perm[(size_t)(sm64(seed ^ 0xA5A5ull, (uint64_t)k) % (uint64_t)(k + 1))]);
    std::vector<float> X((size_t)B * NFEAT), Y((size_t)B);
    for (int64_t k = 0; k < B; ++k) {
        std::copy(&s->X[(size_t)perm[(size_t)k] * NFEAT], &s->X[(size_t)perm[(size_t)k] * NFEAT] + NFEAT, &X[(size_t)k * NFEAT]);
        Y[(size_t)k] = s->Y[(size_t)perm[(size_t)k]];
    }
    if (int rc = ensure_dev(s, B)) return set_err(ctx, rc, "sched_train: buffers");
    cudaMemcpyAsync(s->dX, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(s->dY, Y.data(), Y.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    float loss = 0.f;
    if (int rc = spdz_mlp_train(s->model, s->dX, s->dY, B, epochs, 128, lr, &loss)) return set_err(ctx, rc, "sched_train: training");
    s->trained = true;
    s->train_loss = loss;
    s->chosen.clear();
    if (loss_out) *loss_out = loss;
    return SPDZ_OK;
}

int spdz_sched_predict(spdz_ctx *ctx, spdz_dag *dag, int32_t cfg, float *us_out) {
    if (!ctx || !dag || !us_out || cfg < 0 || cfg >= NCFG) return SPDZ_ERR_ARG;
    std::vector<double> pred;
    if (int rc = predict_layers(ctx, dag, pred)) return set_err(ctx, rc, "sched_predict: model not trained");
    for (int l = 0; l < dag->depth; ++l) us_out[l] = (float)pred[(size_t)l * NCFG + cfg];
    return SPDZ_OK;
}

int spdz_sched_learned_plan(spdz_ctx *ctx, spdz_dag *dag, spdz_plan *out, double *predicted_ms) {
    if (!ctx || !dag || !out) return SPDZ_ERR_ARG;
    int rc = learned_plan(ctx, dag, *out, predicted_ms);
    return rc ? set_err(ctx, rc, "sched_learned_plan: model not trained") : SPDZ_OK;
}

int spdz_sched_autotune(spdz_ctx *ctx, spdz_dag *dag, const spdz_buf *wires, int32_t reps, spdz_plan *out,
                        double *best_ms) {
    if (!ctx || !dag || !wires || !out || reps < 1) return set_err(ctx, SPDZ_ERR_ARG, "sched_autotune: bad argument");
    double best = 1e300;
    Sched *s = sched_of(ctx);
    s->last_tagged_ms = -1;
    for (int c = 0; c < NCFG; ++c) {
        if (!config_ok(dag, c)) continue;
        spdz_plan p;
        uniform_plan(dag, c, p);
        double ms = 0;
        if (int rc = measure(ctx, dag, p, wires, reps, &ms)) return rc;
        if (kConfigs[c].tagged) s->last_tagged_ms = ms;
        if (ms < best) {
            best = ms;
            *out = p;
        }
    }
    if (best_ms) *best_ms = best;
    return SPDZ_OK;
}

int spdz_sched_choose(spdz_ctx *ctx, spdz_dag *dag, const spdz_buf *wires, int32_t reps, spdz_plan *out,
                      spdz_sched_report *rep) {
    if (!ctx || !dag || !wires || reps < 1) return set_err(ctx, SPDZ_ERR_ARG, "sched_choose: bad argument");
    Sched *s = sched_of(ctx);
    spdz_sched_report r{};
    spdz_plan def, tuned, learned;
    uniform_plan(dag, DEFAULT_CFG, def);
    if (int rc = measure(ctx, dag, def, wires, reps, &r.default_ms)) return rc;
    if (int rc = spdz_sched_autotune(ctx, dag, wires, reps, &tuned, &r.autotuned_ms)) return rc;
    r.tagged_ms = s->last_tagged_ms;
    // The winner's selection time is the least of several noisy medians,
    // biased low: its time is measured again, so that the default, the
    // autotuned and the learned plan are compared on fresh measurements alike.
    if (int rc = measure(ctx, dag, tuned, wires, reps, &r.autotuned_ms)) return rc;
    spdz_plan best = tuned;
    double best_ms = r.autotuned_ms;
    r.chosen = 1;
    if (r.default_ms < best_ms) {
        best = def;
        best_ms = r.default_ms;
        r.chosen = 0;
    }
    r.learned_ms = -1;
    r.predicted_ms = -1;
    if (s->trained && learned_plan(ctx, dag, learned, &r.predicted_ms) == SPDZ_OK) {
        r.learned_groups = learned.n_groups;
        if (same_groups(learned, tuned)) {
            // the model picked the plan the autotuner found by measuring
            // every configuration: nothing more to measure
            r.learned_is_autotuned = 1;
            r.learned_ms = r.autotuned_ms;
            if (r.chosen == 1) r.chosen = 2;
        } else {
            if (int rc = measure(ctx, dag, learned, wires, reps, &r.learned_ms)) return rc;
            if (r.learned_ms < best_ms) {
                best = learned;
                best_ms = r.learned_ms;
                r.chosen = 2;
            }
        }
    }
    r.samples = (int32_t)s->Y.size();
    r.train_loss = s->train_loss;
    r.switch_us = s->switch_us;
    s->chosen[dag] = best;
    if (out) *out = best;
    if (rep) *rep = r;
    return SPDZ_OK;
}

}  // extern "C"
