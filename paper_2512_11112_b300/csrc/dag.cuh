// dag.cuh -- host-side representation of an uploaded circuit, shared by the
// executor (dag.cu) and the scheduler (sched.cu).
#pragma once
#include <vector>

#include "common.cuh"

namespace spdz {

// One row per layer: record ranges of the five gate classes (MUL, ADD, SUB,
// CMUL, CADD, in that order) and the MUL rank of the layer's first MUL gate.
struct LayerRow {
    int32_t s[6];        // s[c] = first record of class c, s[5] = end of the layer
    int32_t mulbase;
    int32_t pad;
};

}  // namespace spdz

struct spdz_dag {
    spdz_ctx *ctx = nullptr;
    int field = 0, n = 0;
    int64_t n_inputs = 0, n_gates = 0, n_mul = 0;
    int depth = 0;
    std::vector<spdz::LayerRow> lay;            // host copy of the layer table
    std::vector<int32_t> counts;          // [depth][5] gates per class
    uint4 *d_rec = nullptr;
    spdz::LayerRow *d_lay = nullptr;
    void *d_kc = nullptr;
    // tagged mode: tagged wire-major copy of the wires, and the runs so far
    uint64_t *d_mir = nullptr;
    size_t mir_bytes = 0;
    uint64_t df_runs = 0;
    // captured run
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t gbegin = nullptr;
    cudaKernelNodeParams gbegin_params{};
    spdz_plan gplan{};
    spdz_buf gwires{};
    int glaunches = 0;
    bool gtimed = false;                  // the captured run records kev0 / kev1
    cudaStream_t cap_stream = nullptr;
    // timing
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaEvent_t> lev;
    std::vector<float> layer_us;
    // spdz_dag_time_kernels: events around the run's circuit kernels
    bool time_kernels = false;
    cudaEvent_t kev0 = nullptr, kev1 = nullptr;
};
