// mlp.cu -- the learned cost model: a small fully connected network
// (n_in -> H -> ... -> H -> 1, ReLU, FP32) with hand-written forward,
// backward (mean squared error) and Adam kernels.  It predicts the log
// device time of one circuit layer under one execution configuration from
// features of the layer; the scheduler trains it on timings the pipeline
// records itself.
//
// Parameters are one flat float array: for each layer l (input size I,
// output size O) the weights W_l[O][I] (row-major) followed by the biases
// b_l[O].  Every reduction runs in a fixed order (no atomics), so results
// are deterministic.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

struct spdz_mlp {
    int n_in = 0, hidden = 0, layers = 0;   // layers = number of weight layers
    std::vector<int> dims;                  // dims[0] = n_in, ..., dims[layers] = 1
    std::vector<int64_t> woff, boff;        // parameter offsets of W_l and b_l
    int64_t n_params = 0;
    cudaStream_t stream = nullptr;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // params, grads, Adam moments
    float *act = nullptr;                   // activations [layers+1][cap][maxdim]
    float *dz = nullptr, *dz2 = nullptr;    // backprop buffers [cap][maxdim]
    float *loss = nullptr;                  // [1]
    int64_t cap = 0;
    int maxdim = 0;
    int64_t adam_t = 0;
};

namespace spdz {

// out[b][o] = act(sum_i W[o][i] * in[b][i] + bias[o]), in row stride = ld.
__global__ void k_mlp_layer(const float *W, const float *bias, const float *in, float *out, int64_t B,
                            int I, int O, int ld, int relu) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= B * O) return;
    const int64_t b = t / O;
    const int o = (int)(t % O);
    float s = bias[o];
    const float *w = W + (int64_t)o * I;
    const float *x = in + b * ld;
    for (int i = 0; i < I; ++i) s = fmaf(w[i], x[i], s);
    out[b * ld + o] = relu ? fmaxf(s, 0.f) : s;
}

// dz[b] = 2 (y[b] - target[b]) / B and the loss sum (one block, fixed order).
__global__ void k_mlp_out_grad(const float *y, int ld, const float *target, float *dz, int dld, int64_t B,
                               float *loss) {
    __shared__ float part[256];
    float s = 0.f;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) {
        const float d = y[b * ld] - target[b];
        dz[b * dld] = 2.f * d / (float)B;
        s += d * d;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) part[threadIdx.x] += part[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / (float)B;
}

// dW[o][i] = sum_b dz[b][o] a[b][i] (i < I), db[o] = sum_b dz[b][o].
__global__ void k_mlp_wgrad(const float *dz, const float *a, float *dW, float *db, int64_t B, int I, int O,
                            int ld) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)O * (I + 1)) return;
    const int o = (int)(t / (I + 1)), i = (int)(t % (I + 1));
    float s = 0.f;
    if (i < I) {
        for (int64_t b = 0; b < B; ++b) s = fmaf(dz[b * ld + o], a[b * ld + i], s);
        dW[(int64_t)o * I + i] = s;
    } else {
        for (int64_t b = 0; b < B; ++b) s += dz[b * ld + o];
        db[o] = s;
    }
}

// dprev[b][i] = (sum_o W[o][i] dz[b][o]) * [a_prev[b][i] > 0].
__global__ void k_mlp_back(const float *W, const float *dz, const float *a_prev, float *dprev, int64_t B, int I,
                           int O, int ld) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= B * I) return;
    const int64_t b = t / I;
    const int i = (int)(t % I);
    float s = 0.f;
    for (int o = 0; o < O; ++o) s = fmaf(W[(int64_t)o * I + i], dz[b * ld + o], s);
    dprev[b * ld + i] = a_prev[b * ld + i] > 0.f ? s : 0.f;
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gg = g[t];
    const float mm = b1 * m[t] + (1.f - b1) * gg;
    const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
    m[t] = mm;
    v[t] = vv;
    p[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// Copies rows [b0, b0+B) of X ([*, n_in]) into activation slot 0 (stride ld).
__global__ void k_mlp_load(const float *X, int n_in, float *a0, int ld, int64_t B) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= B * n_in) return;
    const int64_t b = t / n_in;
    a0[b * ld + (t % n_in)] = X[t];
}

__global__ void k_mlp_store(const float *a, int ld, float *Y, int64_t B) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < B) Y[t] = a[t * ld];
}

static inline int nb(int64_t n) { return (int)((n + 255) / 256); }

static int mlp_reserve(spdz_mlp *m, int64_t B) {
    if (B <= m->cap) return SPDZ_OK;
    if (m->act) cudaFree(m->act);
    if (m->dz) cudaFree(m->dz);
    if (m->dz2) cudaFree(m->dz2);
    m->act = m->dz = m->dz2 = nullptr;
    const size_t per = (size_t)B * m->maxdim * sizeof(float);
    if (cudaMalloc(&m->act, per * (m->layers + 1)) != cudaSuccess || cudaMalloc(&m->dz, per) != cudaSuccess ||
        cudaMalloc(&m->dz2, per) != cudaSuccess)
        return SPDZ_ERR_OOM;
    m->cap = B;
    return SPDZ_OK;
}

static float *act_slot(spdz_mlp *m, int l) { return m->act + (size_t)l * m->cap * m->maxdim; }

static void mlp_forward(spdz_mlp *m, const float *X, int64_t B) {
    const int ld = m->maxdim;
    k_mlp_load<<<nb(B * m->n_in), 256, 0, m->stream>>>(X, m->n_in, act_slot(m, 0), ld, B);
    for (int l = 0; l < m->layers; ++l) {
        const int I = m->dims[l], O = m->dims[l + 1];
        k_mlp_layer<<<nb(B * O), 256, 0, m->stream>>>(m->p + m->woff[l], m->p + m->boff[l], act_slot(m, l),
                                                      act_slot(m, l + 1), B, I, O, ld, l + 1 < m->layers);
    }
}

// Forward and backward on one batch: gradient of the mean squared error into m->g.
static void mlp_grad(spdz_mlp *m, const float *X, const float *Tgt, int64_t B) {
    const int ld = m->maxdim;
    mlp_forward(m, X, B);
    k_mlp_out_grad<<<1, 256, 0, m->stream>>>(act_slot(m, m->layers), ld, Tgt, m->dz, ld, B, m->loss);
    float *cur = m->dz, *nxt = m->dz2;
    for (int l = m->layers - 1; l >= 0; --l) {
        const int I = m->dims[l], O = m->dims[l + 1];
        k_mlp_wgrad<<<nb((int64_t)O * (I + 1)), 256, 0, m->stream>>>(cur, act_slot(m, l), m->g + m->woff[l],
                                                                    m->g + m->boff[l], B, I, O, ld);
        if (l > 0) {
            k_mlp_back<<<nb(B * I), 256, 0, m->stream>>>(m->p + m->woff[l], cur, act_slot(m, l), nxt, B, I, O, ld);
            std::swap(cur, nxt);
        }
    }
}

}  // namespace spdz

using namespace spdz;

extern "C" {

int spdz_mlp_create(spdz_mlp **out, int32_t n_in, int32_t hidden, int32_t hidden_layers, uint64_t seed,
                    void *stream) {
    if (!out || n_in < 1 || n_in > 256 || hidden < 1 || hidden > 1024 || hidden_layers < 1 || hidden_layers > 8)
        return SPDZ_ERR_ARG;
    spdz_mlp *m = new spdz_mlp();
    m->n_in = n_in;
    m->hidden = hidden;
    m->layers = hidden_layers + 1;
    m->stream = (cudaStream_t)stream;
    m->dims.push_back(n_in);
    for (int k = 0; k < hidden_layers; ++k) m->dims.push_back(hidden);
    m->dims.push_back(1);
    m->maxdim = std::max(n_in, hidden);
    int64_t off = 0;
    for (int l = 0; l < m->layers; ++l) {
        m->woff.push_back(off);
        off += (int64_t)m->dims[l] * m->dims[l + 1];
        m->boff.push_back(off);
        off += m->dims[l + 1];
    }
    m->n_params = off;
    // He-uniform initial weights from the counter PRG, zero biases
    std::vector<float> init((size_t)off, 0.f);
    for (int l = 0; l < m->layers; ++l) {
        const int I = m->dims[l], O = m->dims[l + 1];
        const float lim = std::sqrt(6.f / (float)I);
        for (int64_t k = 0; k < (int64_t)I * O; ++k) {
            const uint64_t r = sm64(seed, (uint64_t)(m->woff[l] + k));
            const float u = (float)((r >> 40) * (1.0 / 16777216.0));   // [0, 1)
            init[(size_t)(m->woff[l] + k)] = (2.f * u - 1.f) * lim;
        }
    }
    const size_t bytes = (size_t)off * sizeof(float);
    if (cudaMalloc(&m->p, bytes) != cudaSuccess || cudaMalloc(&m->g, bytes) != cudaSuccess ||
        cudaMalloc(&m->m, bytes) != cudaSuccess || cudaMalloc(&m->v, bytes) != cudaSuccess ||
        cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess) {
        spdz_mlp_destroy(m);
        return SPDZ_ERR_OOM;
    }
    cudaMemcpy(m->p, init.data(), bytes, cudaMemcpyHostToDevice);
    cudaMemset(m->g, 0, bytes);
    cudaMemset(m->m, 0, bytes);
    cudaMemset(m->v, 0, bytes);
    *out = m;
    return SPDZ_OK;
}

int spdz_mlp_destroy(spdz_mlp *m) {
    if (!m) return SPDZ_OK;
    for (float *q : {m->p, m->g, m->m, m->v, m->act, m->dz, m->dz2, m->loss})
        if (q) cudaFree(q);
    delete m;
    return SPDZ_OK;
}

int spdz_mlp_num_params(const spdz_mlp *m, int64_t *count) {
    if (!m || !count) return SPDZ_ERR_ARG;
    *count = m->n_params;
    return SPDZ_OK;
}

int spdz_mlp_get_params(const spdz_mlp *m, float *host_out) {
    if (!m || !host_out) return SPDZ_ERR_ARG;
    cudaStreamSynchronize(m->stream);
    return cudaMemcpy(host_out, m->p, (size_t)m->n_params * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess
               ? SPDZ_OK : SPDZ_ERR_CUDA;
}

int spdz_mlp_set_params(spdz_mlp *m, const float *host_in) {
    if (!m || !host_in) return SPDZ_ERR_ARG;
    cudaStreamSynchronize(m->stream);
    if (cudaMemcpy(m->p, host_in, (size_t)m->n_params * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
        return SPDZ_ERR_CUDA;
    cudaMemset(m->m, 0, (size_t)m->n_params * sizeof(float));
    cudaMemset(m->v, 0, (size_t)m->n_params * sizeof(float));
    m->adam_t = 0;
    return SPDZ_OK;
}

int spdz_mlp_forward(spdz_mlp *m, const float *X_dev, int64_t B, float *Y_dev) {
    if (!m || !X_dev || !Y_dev || B < 0) return SPDZ_ERR_ARG;
    if (B == 0) return SPDZ_OK;
    if (int rc = mlp_reserve(m, B)) return rc;
    mlp_forward(m, X_dev, B);
    k_mlp_store<<<nb(B), 256, 0, m->stream>>>(act_slot(m, m->layers), m->maxdim, Y_dev, B);
    return cudaGetLastError() == cudaSuccess ? SPDZ_OK : SPDZ_ERR_CUDA;
}

int spdz_mlp_loss_grad(spdz_mlp *m, const float *X_dev, const float *T_dev, int64_t B, float *loss_host,
                       float *grad_host) {
    if (!m || !X_dev || !T_dev || B <= 0) return SPDZ_ERR_ARG;
    if (int rc = mlp_reserve(m, B)) return rc;
    mlp_grad(m, X_dev, T_dev, B);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return SPDZ_ERR_CUDA;
    if (loss_host) cudaMemcpy(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost);
    if (grad_host) cudaMemcpy(grad_host, m->g, (size_t)m->n_params * sizeof(float), cudaMemcpyDeviceToHost);
    return cudaGetLastError() == cudaSuccess ? SPDZ_OK : SPDZ_ERR_CUDA;
}

// One Adam step (the same kernel and step counter as spdz_mlp_train) with a
// gradient the caller supplies.
int spdz_mlp_adam_step(spdz_mlp *m, const float *grad_dev, float lr) {
    if (!m || !grad_dev) return SPDZ_ERR_ARG;
    const float b1 = 0.9f, b2 = 0.999f;
    ++m->adam_t;
    const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
    k_adam<<<nb(m->n_params), 256, 0, m->stream>>>(m->p, grad_dev, m->m, m->v, m->n_params, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? SPDZ_OK : SPDZ_ERR_CUDA;
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) over `epochs` passes of the data
// in consecutive mini-batches of `batch` rows (the caller shuffles).
int spdz_mlp_train(spdz_mlp *m, const float *X_dev, const float *T_dev, int64_t B, int32_t epochs, int32_t batch,
                   float lr, float *loss_host) {
    if (!m || !X_dev || !T_dev || B <= 0 || epochs < 0 || batch <= 0) return SPDZ_ERR_ARG;
    const int64_t mb = std::min<int64_t>(batch, B);
    if (int rc = mlp_reserve(m, mb)) return rc;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int e = 0; e < epochs; ++e) {
        for (int64_t b0 = 0; b0 < B; b0 += mb) {
            const int64_t n = std::min<int64_t>(mb, B - b0);
            mlp_grad(m, X_dev + b0 * m->n_in, T_dev + b0, n);
            ++m->adam_t;
            const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
            k_adam<<<nb(m->n_params), 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, m->n_params, lr, b1, b2, 1e-8f,
                                                           c1, c2);
        }
    }
    if (cudaGetLastError() != cudaSuccess) return SPDZ_ERR_CUDA;
    if (loss_host) {
        // loss over the whole set with the final parameters
        float total = 0.f;
        for (int64_t b0 = 0; b0 < B; b0 += mb) {
            const int64_t n = std::min<int64_t>(mb, B - b0);
            mlp_grad(m, X_dev + b0 * m->n_in, T_dev + b0, n);
            float l = 0.f;
            cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream);
            cudaStreamSynchronize(m->stream);
            total += l * (float)n;
        }
        *loss_host = total / (float)B;
    }
    return cudaGetLastError() == cudaSuccess ? SPDZ_OK : SPDZ_ERR_CUDA;
}

}  // extern "C"
