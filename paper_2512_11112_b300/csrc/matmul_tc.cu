// matmul_tc.cu -- the tensor-core path of the secret-shared matrix product.
#include "common.cuh"

namespace spdz {

int matmul_tensor(spdz_ctx *ctx, const uint64_t *E, const uint64_t *Fm, const uint64_t *Rfold, const spdz_buf *A,
                  const spdz_buf *C, const spdz_buf *Z, int64_t m, int64_t k, int64_t n) {
    (void)E; (void)Fm; (void)Rfold; (void)A; (void)C; (void)Z; (void)m; (void)k; (void)n;
    return set_err(ctx, SPDZ_ERR_ARG, "matmul: tensor path not built yet");
}

}  // namespace spdz
