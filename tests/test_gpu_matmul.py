"""Secret-shared matrix products on the GPU against the CPU oracle: the
device dealer's matrix triple, the opened E and F, every share of Z and
gamma(Z), and the MAC check, bit-exact; at the benchmark size (2048^3,
3 parties) on sampled entries the oracle computes one by one."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

from gpu_helpers import assert_equal, ctx_for  # noqa: E402

P = O.P61
SEED, SUB, CHK = 44, 3, 12


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    global S, SH
    from paper_2512_11112_b300 import shares as SH  # noqa: F401
    from paper_2512_11112_b300 import spdz as S  # noqa: F401
    yield


def device_product(n, m, k, nn, path):
    ctx = ctx_for(n, P)
    f = S.SPDZ_F61
    ash = SH.zeros(f, n)
    S.spdz_deal_alpha(ctx, SEED, ash)
    X, Y = SH.alloc(f, n, m * k), SH.alloc(f, n, k * nn)
    S.spdz_deal_shared(ctx, SEED, S.SPDZ_KIND_INPUT, 10, 0, m * k, ash, None, X.buf())
    S.spdz_deal_shared(ctx, SEED, S.SPDZ_KIND_INPUT, 11, 0, k * nn, ash, None, Y.buf())
    A, B, Cm = SH.alloc(f, n, m * k), SH.alloc(f, n, k * nn), SH.alloc(f, n, m * nn)
    S.spdz_deal_matrix_triple(ctx, SEED, SUB, m, k, nn, ash, A.buf(), B.buf(), Cm.buf())
    S.spdz_load_preproc(ctx, ash, None, None, None, 0)
    S.spdz_set_check_seed(ctx, CHK)
    S.spdz_load_matrix_preproc(ctx, A.buf(), B.buf(), Cm.buf(), m, k, nn)
    Z = SH.alloc(f, n, m * nn)
    E, F = SH.zeros(f, m * k), SH.zeros(f, k * nn)
    S.spdz_matmul(ctx, X.buf(), Y.buf(), Z.buf(), m, k, nn, path, E, F)
    sig = O.zeros(P, n)
    passed = S.spdz_mac_check(ctx, sig)
    out = dict(A=A.host(), B=B.host(), C=Cm.host(), Z=Z.host(), E=SH.to_host(E), F=SH.to_host(F), sig=sig,
               passed=passed)
    # a second product without a new triple is refused
    with pytest.raises(S.SpdzError) as e:
        S.spdz_matmul(ctx, X.buf(), Y.buf(), Z.buf(), m, k, nn, path)
    assert e.value.code == S.SPDZ_ERR_TRIPLES
    S.spdz_ctx_destroy(ctx)
    return out


def oracle_inputs(n, m, k, nn):
    alpha, ash = O.deal_alpha(P, n, SEED)
    X = O.deal_shared(P, n, SEED, O.K_INPUT, 10, 0, m * k, alpha)
    Y = O.deal_shared(P, n, SEED, O.K_INPUT, 11, 0, k * nn, alpha)
    return alpha, ash, X, Y


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("n,m,k,nn", [(3, 64, 64, 64), (3, 100, 37, 50), (2, 5, 130, 7), (4, 33, 65, 129),
                                     (2, 1, 1, 1), (3, 1, 300, 1), (2, 257, 1, 3)])
def test_small_products_match_oracle(path, n, m, k, nn):
    if path == 1 and not _tensor_path_available():
        pytest.skip("tensor path not built")
    d = device_product(n, m, k, nn, path)
    alpha, ash, X, Y = oracle_inputs(n, m, k, nn)
    tri = O.deal_matrix_triple(P, n, SEED, SUB, m, k, nn, alpha)
    for name, (v, mm) in (("A", (tri.av, tri.am)), ("B", (tri.bv, tri.bm)), ("C", (tri.cv, tri.cm))):
        assert_equal(d[name][0], v, f"triple {name} values")
        assert_equal(d[name][1], mm, f"triple {name} MACs")
    E, F, Em, Fm = O.mat_open(P, m, k, nn, X[:2], Y[:2], tri)
    assert_equal(d["E"], E, "E")
    assert_equal(d["F"], F, "F")
    rows, cols = np.divmod(np.arange(m * nn), nn)
    Zv, Zm = O.mat_entries(P, m, k, nn, E, F, tri, ash, rows, cols)
    assert_equal(d["Z"][0], Zv, "Z values")
    assert_equal(d["Z"][1], Zm, "Z MACs")
    log = O.OpenLog(np.concatenate([E, F]), np.ascontiguousarray(np.concatenate([Em, Fm], axis=1)))
    ok, osig, _, _ = O.mac_check(P, [log], ash, CHK, 0)
    assert d["passed"] and ok
    assert_equal(d["sig"], osig, "sigma")


def _tensor_path_available():
    try:
        ctx = ctx_for(2, P)
    except Exception:
        return False
    S.spdz_ctx_destroy(ctx)
    return getattr(S, "TENSOR_PATH", False)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("dim", [512, 2048])
def test_benchmark_size_sampled_entries(path, dim):
    """X, Y of dim x dim, 3 parties: sampled entries of every party's Z and
    gamma(Z) against the oracle's own computation of those entries."""
    if path == 1 and not _tensor_path_available():
        pytest.skip("tensor path not built")
    n, m, k, nn = 3, dim, dim, dim
    d = device_product(n, m, k, nn, path)
    assert d["passed"]
    O.set_threads(8)
    alpha, ash, X, Y = oracle_inputs(n, m, k, nn)
    Av, Am, Asec = O.deal_shared(P, n, SEED, O.K_MTRIPLE_A, SUB, 0, m * k, alpha)
    Bv, Bm, Bsec = O.deal_shared(P, n, SEED, O.K_MTRIPLE_B, SUB, 0, k * nn, alpha)
    assert_equal(d["A"][0], Av, "A values")
    assert_equal(d["B"][1], Bm, "B MACs")
    # E, F from the oracle's own shares
    dummy = O.zeros(P, n, 1)
    tri_ab = O.Triples(Av, Am, Bv, Bm, dummy, dummy)
    E, F, _, _ = O.mat_open(P, m, k, nn, X[:2], Y[:2], tri_ab)
    assert_equal(d["E"], E, "E")
    assert_equal(d["F"], F, "F")
    rng = np.random.default_rng(dim)
    rows = rng.integers(0, m, 48)
    cols = rng.integers(0, nn, 48)
    rows[:2], cols[:2] = (0, m - 1), (nn - 1, 0)
    # C = A*B at the sampled entries, then its shares from the PRG at those indices
    Cv, Cm = O.zeros(P, n, m * nn), O.zeros(P, n, m * nn)   # only sampled columns are filled
    for r, c in zip(rows, cols):
        a = O.to_ints(P, Asec[r * k:(r + 1) * k])
        b = O.to_ints(P, Bsec[c::nn][:k])
        cval = sum(x * y for x, y in zip(a, b)) % P
        v, mm, _ = O.deal_shared(P, n, SEED, O.K_MTRIPLE_C, SUB, int(r * nn + c), 1, alpha, O.to_array(P, [cval]))
        Cv[:, r * nn + c], Cm[:, r * nn + c] = v[:, 0], mm[:, 0]
    tri = O.Triples(Av, Am, Bv, Bm, Cv, Cm)
    Zv, Zm = O.mat_entries(P, m, k, nn, E, F, tri, ash, rows, cols)
    idx = rows * nn + cols
    assert_equal(d["Z"][0][:, idx], Zv, "sampled Z values")
    assert_equal(d["Z"][1][:, idx], Zm, "sampled Z MACs")
    assert_equal(d["C"][0][:, idx], Cv[:, idx], "sampled C values")


def _worst_digit_value():
    """A value of [0, p) whose balanced base-2^8 digits are -128 in the seven
    low places (and 1 on top): every digit-pair product of two such values
    is 128 * 128 = 2^14, the largest a digit pair can give."""
    v = sum(-128 * 256**i for i in range(7)) + 256**7
    assert 0 < v < P
    t, digits = v, []
    for _ in range(7):
        d = t % 256
        d = d - 256 if d >= 128 else d
        digits.append(d)
        t = (t - d) // 256
    assert digits == [-128] * 7 and t == 1
    return v


@pytest.mark.parametrize("path", [0, 1])
def test_largest_digit_sums_stay_exact(path):
    """Shares built so that the opened E, and the right operand E is
    multiplied by in the value product of party 0 (B_0 + F), hold in every
    entry a value whose low digits are all -128: each digit-pair sum over an
    inner chunk of 1024 is then exactly 2^24, the largest the tensor path
    allows.  Every entry of Z and gamma(Z) equals the oracle, and the check
    over E and F passes."""
    if path == 1 and not _tensor_path_available():
        pytest.skip("tensor path not built")
    n, m, k, nn = 2, 64, 2048, 64
    f = S.SPDZ_F61
    ctx = ctx_for(n, P)
    try:
        ash_d = SH.zeros(f, n)
        S.spdz_deal_alpha(ctx, SEED, ash_d)
        A, B, Cm = SH.alloc(f, n, m * k), SH.alloc(f, n, k * nn), SH.alloc(f, n, m * nn)
        S.spdz_deal_matrix_triple(ctx, SEED, SUB, m, k, nn, ash_d, A.buf(), B.buf(), Cm.buf())
        alpha, ash = O.deal_alpha(P, n, SEED)
        al = O.to_ints(P, ash)
        (Av, Am), (Bv, Bm) = A.host(), B.host()
        w = _worst_digit_value()
        Ei = [w] * (m * k)
        B0 = O.to_ints(P, Bv[0])
        Fi = [(w - b) % P for b in B0]                    # B_0 + F = w everywhere
        Xv, Xm, Yv, Ym = (O.zeros(P, n, m * k), O.zeros(P, n, m * k), O.zeros(P, n, k * nn), O.zeros(P, n, k * nn))
        for i in range(n):
            ai, gai = O.to_ints(P, Av[i]), O.to_ints(P, Am[i])
            bi, gbi = O.to_ints(P, Bv[i]), O.to_ints(P, Bm[i])
            Xv[i] = O.to_array(P, [(a + (e if i == 0 else 0)) % P for a, e in zip(ai, Ei)])
            Xm[i] = O.to_array(P, [(g + al[i] * e) % P for g, e in zip(gai, Ei)])
            Yv[i] = O.to_array(P, [(b + (x if i == 0 else 0)) % P for b, x in zip(bi, Fi)])
            Ym[i] = O.to_array(P, [(g + al[i] * x) % P for g, x in zip(gbi, Fi)])
        X, Y = SH.alloc(f, n, m * k), SH.alloc(f, n, k * nn)
        X.val[:, :m * k] = SH.from_host(Xv)
        X.mac[:, :m * k] = SH.from_host(Xm)
        Y.val[:, :k * nn] = SH.from_host(Yv)
        Y.mac[:, :k * nn] = SH.from_host(Ym)
        S.spdz_load_preproc(ctx, ash_d, None, None, None, 0)
        S.spdz_set_check_seed(ctx, CHK)
        S.spdz_load_matrix_preproc(ctx, A.buf(), B.buf(), Cm.buf(), m, k, nn)
        Z = SH.alloc(f, n, m * nn)
        E, F = SH.zeros(f, m * k), SH.zeros(f, k * nn)
        S.spdz_matmul(ctx, X.buf(), Y.buf(), Z.buf(), m, k, nn, path, E, F)
        assert S.spdz_mac_check(ctx)
        assert O.to_ints(P, SH.to_host(E)) == Ei
        assert O.to_ints(P, SH.to_host(F)) == Fi
        Cv, Cmm = Cm.host()
        tri = O.Triples(Av, Am, Bv, Bm, Cv, Cmm)
        rows, cols = np.divmod(np.arange(m * nn), nn)
        Zv, Zm = O.mat_entries(P, m, k, nn, O.to_array(P, Ei), O.to_array(P, Fi), tri, ash, rows, cols)
        gv, gm = Z.host()
        assert_equal(gv, Zv, "Z values")
        assert_equal(gm, Zm, "Z MACs")
    finally:
        S.spdz_ctx_destroy(ctx)
