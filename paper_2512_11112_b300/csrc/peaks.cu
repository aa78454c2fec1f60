// peaks.cu -- integer issue-rate microbenchmarks: the denominators of the
// compute side of the roofline for kernels bound by integer arithmetic (the
// p = 2^127-1 Beaver products and inner products, whose 64-bit products are
// built from 32-bit multiply-adds).  Each thread runs eight independent
// dependency chains of one instruction kind, so the issue rate, not the
// latency, limits the loop; the chains' values are stored at the end so no
// work is removed.
#include "common.cuh"

namespace spdz {

template <int KIND>
__global__ void __launch_bounds__(256) k_int_peak(uint32_t m, uint32_t c, int64_t iters, uint32_t *out) {
    uint32_t v[8];
    uint64_t w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = threadIdx.x + 131u * k + blockIdx.x;
        w[k] = v[k];
    }
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (KIND == 0) {          // 32-bit multiply-add (low half)
                    asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(v[k]) : "r"(m), "r"(c));
                } else if constexpr (KIND == 1) {   // 32 x 32 + 64 -> 64 multiply-add
                    asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[k]) : "r"((uint32_t)w[k]), "r"(m));
                } else if constexpr (KIND == 2) {   // high half of a 32 x 32 product
                    asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(v[k]) : "r"(m));
                    asm volatile("add.u32 %0, %0, %1;" : "+r"(v[k]) : "r"(c));
                } else {                            // integer add / logic
                    asm volatile("add.u32 %0, %0, %1;" : "+r"(v[k]) : "r"(m));
                    asm volatile("xor.b32 %0, %0, %1;" : "+r"(v[k]) : "r"(c));
                }
            }
        }
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k] ^ (uint32_t)w[k] ^ (uint32_t)(w[k] >> 32);
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace spdz

using namespace spdz;

extern "C" int spdz_int_peak(int kind, int64_t iters, void *stream, void *scratch_dev, double *ops_per_s) {
    if (kind < 0 || kind > 3 || iters < 1 || !scratch_dev || !ops_per_s) return SPDZ_ERR_ARG;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = 8 * sms, block = 256;   // 64 warps per SM
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SPDZ_ERR_CUDA;
    auto launch = [&](int64_t n) {
        uint32_t *o = (uint32_t *)scratch_dev;
        switch (kind) {
            case 0: k_int_peak<0><<<grid, block, 0, st>>>(0x9E3779B9u, 7u, n, o); break;
            case 1: k_int_peak<1><<<grid, block, 0, st>>>(0x9E3779B9u, 7u, n, o); break;
            case 2: k_int_peak<2><<<grid, block, 0, st>>>(0x9E3779B9u, 7u, n, o); break;
            default: k_int_peak<3><<<grid, block, 0, st>>>(0x9E3779B9u, 7u, n, o); break;
        }
    };
    launch(16);   // warm-up
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || ms <= 0.f) return SPDZ_ERR_CUDA;
    // thread-level instructions of the measured kind (KIND 2 and 3 count both
    // instructions of their pair)
    const double per_iter = (kind >= 2 ? 2.0 : 1.0) * 32.0;
    *ops_per_s = (double)grid * block * (double)iters * per_iter / (ms * 1e-3);
    return SPDZ_OK;
}
