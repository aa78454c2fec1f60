"""The allocation-free Beaver batch (spdz_mul_check_noalloc), for callers that
cannot allocate device memory, must give exactly what the context-based path
gives (spdz_mul_batch followed by spdz_mac_check) on the same inputs, call
after call, even though every call reuses the library's one fixed scratch
array.  Collected last on purpose (file name), so that a failure here comes
after every other test has run."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p,n,N", [(O.P61, 3, 5003), (O.P127, 2, 777), (O.P32, 3, 999)])
def test_noalloc_matches_context_path_two_calls(p, n, N):
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2512_11112_b300 import shares as SH
    from paper_2512_11112_b300 import spdz as S

    field = SH.field_of(p)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = S.spdz_ctx_create(n, field, stream)
    try:
        seed, chk = 23, 77
        ash = SH.zeros(field, n)
        S.spdz_deal_alpha(ctx, seed, ash)
        x, y = SH.alloc(field, n, N), SH.alloc(field, n, N)
        S.spdz_deal_shared(ctx, seed, S.SPDZ_KIND_INPUT, 0, 0, N, ash, None, x.buf())
        S.spdz_deal_shared(ctx, seed, S.SPDZ_KIND_INPUT, 1, 0, N, ash, None, y.buf())
        tri = [SH.alloc(field, n, 2 * N) for _ in range(3)]
        S.spdz_deal_triples(ctx, seed, 0, 2 * N, ash, *[t.buf() for t in tri])
        S.spdz_load_preproc(ctx, ash, *[t.buf() for t in tri], 2 * N)
        S.spdz_set_check_seed(ctx, chk)

        # context path: two batches, two checks (epochs 0 and 1)
        z_ctx = [SH.alloc(field, n, N) for _ in range(2)]
        sig_ctx = [O.zeros(p, n) for _ in range(2)]
        S.spdz_mul_batch(ctx, x.buf(), y.buf(), z_ctx[0].buf(), N)
        ok0 = S.spdz_mac_check(ctx, sig_ctx[0])
        S.spdz_mul_batch(ctx, y.buf(), x.buf(), z_ctx[1].buf(), N)
        ok1 = S.spdz_mac_check(ctx, sig_ctx[1])
        assert ok0 and ok1

        # allocation-free path: the same two batches, same triples and epochs
        z_na = [SH.alloc(field, n, N) for _ in range(2)]
        res = [SH.zeros(field, n + 1) for _ in range(2)]
        for k, (u, v) in enumerate(((x, y), (y, x))):
            S.spdz_mul_check_noalloc(n, field, stream, u.buf(), v.buf(), tri[0].buf(k * N),
                                     tri[1].buf(k * N), tri[2].buf(k * N), ash, z_na[k].buf(), N,
                                     chk, k, res[k])
        torch.cuda.synchronize()
        for k in range(2):
            assert np.array_equal(z_na[k].host()[0], z_ctx[k].host()[0]), f"call {k}: value shares differ"
            assert np.array_equal(z_na[k].host()[1], z_ctx[k].host()[1]), f"call {k}: MAC shares differ"
            r = SH.to_host(res[k])
            assert np.array_equal(r[:n], sig_ctx[k]), f"call {k}: sigma differs"
            assert O.to_ints(p, r[n:n + 1]) == [1], f"call {k}: check did not pass"

        # more parties than the scratch holds: a clear argument error
        with pytest.raises(S.SpdzError) as e:
            S.spdz_mul_check_noalloc(S.SPDZ_MAX_PARTIES + 1, field, stream, x.buf(), y.buf(), tri[0].buf(),
                                     tri[1].buf(), tri[2].buf(), ash, z_na[0].buf(), N, chk, 0, res[0])
        assert e.value.code == S.SPDZ_ERR_ARG
    finally:
        S.spdz_ctx_destroy(ctx)
