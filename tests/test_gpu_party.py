"""The library's party kernels (spdz_party_*) on the GPU against the oracle:
n parties, each with only its own shares on the device, run the protocol of
paper_2512_11112_b300.party; here the parties are threads of one process on
one GPU and the all-gather is an in-process exchange (no kernel of one party
waits on another's: the parties meet on the host).  Two Beaver batches in
two check epochs, three fields; every party's z shares, the opened values and
every sigma equal the oracle's all-party batch and check, bit for bit; a
party that sends a wrong eps_i row fails the check for everyone."""
import threading

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu

from gpu_helpers import assert_equal  # noqa: E402

SEED, CHK = 13, 6


@pytest.fixture(autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    yield
    torch.cuda.synchronize()


class ThreadComm:
    """All-gather between the party threads of this process."""

    def __init__(self, shared, rank):
        self.s, self.rank = shared, rank

    def _exchange(self, item):
        self.s["slots"][self.rank] = item
        self.s["bar"].wait()
        got = list(self.s["slots"])
        self.s["bar"].wait()
        return got

    def all_gather(self, t):
        torch.cuda.synchronize()
        return torch.stack(self._exchange(t))

    def all_gather_obj(self, obj):
        return self._exchange(obj)


def _party(rank, n, p, shared, data, out, tamper):
    from paper_2512_11112_b300 import shares as SH
    from paper_2512_11112_b300.party import DeviceParty, PartyProtocol, PartyRow
    try:
        f = SH.field_of(p)
        dev = lambda a: SH.from_host(np.ascontiguousarray(a), field=f)   # noqa: E731
        row = lambda v, m: PartyRow(dev(v[rank]), dev(m[rank]))          # noqa: E731  this party's rows only
        local = DeviceParty(rank, n, f, dev(data["ash"][rank:rank + 1]), CHK)
        proto = PartyProtocol(local, ThreadComm(shared, rank), p, rank, n)
        res = []
        for ep, (x, y, t) in enumerate(data["epochs"]):
            N = x[0].shape[1]
            X, Y = row(x[0], x[1]), row(y[0], y[1])
            A_, B_, C_ = row(t.av, t.am), row(t.bv, t.bm), row(t.cv, t.cm)
            Z = PartyRow.alloc(f, N)
            if tamper and ep == 1:
                # a cheating party: its eps_i row is shifted at element 5
                orig = local.mask

                def bad(*a, **k):
                    e, d = orig(*a, **k)
                    e = e.clone()
                    e.view(-1)[5 * (2 if f == SH.S.SPDZ_F127 else 1)] ^= 1
                    return e, d
                local.mask = bad
            eps, dlt = proto.mul_batch(X, Y, A_, B_, C_, Z, N)
            passed, sig = proto.mac_check()
            res.append({"zv": SH.to_host(Z.val[:N]), "zm": SH.to_host(Z.mac[:N]), "eps": SH.to_host(eps),
                        "dlt": SH.to_host(dlt), "passed": passed, "sig": sig})
        local.close()
        out[rank] = res
    except BaseException as e:   # noqa: BLE001
        out[rank] = e
        shared["bar"].abort()


def _run(n, p, sizes, tamper=False):
    alpha, ash = O.deal_alpha(p, n, SEED)
    epochs, j0 = [], 0
    for ep, N in enumerate(sizes):
        x = O.deal_shared(p, n, SEED, O.K_INPUT, 2 * ep, 0, N, alpha)
        y = O.deal_shared(p, n, SEED, O.K_INPUT, 2 * ep + 1, 0, N, alpha)
        t = O.deal_triples(p, n, SEED, j0, N, alpha)
        j0 += N
        epochs.append((x, y, t))
    shared = {"slots": [None] * n, "bar": threading.Barrier(n, timeout=120)}
    out = {}
    th = [threading.Thread(target=_party, args=(r, n, p, shared, {"ash": ash, "epochs": epochs}, out,
                                                tamper and r == 1)) for r in range(n)]
    for t_ in th:
        t_.start()
    for t_ in th:
        t_.join(300)
    for r in range(n):
        if isinstance(out.get(r), BaseException):
            raise out[r]
    return alpha, ash, epochs, out


@pytest.mark.parametrize("n,p,sizes", [(2, O.P61, [4099, 100]), (3, O.P127, [777, 2048]), (3, O.P32, [5003, 64]),
                                       (4, O.P61, [1, 33])])
def test_party_kernels_match_oracle(n, p, sizes):
    alpha, ash, epochs, out = _run(n, p, sizes)
    for ep, (x, y, t) in enumerate(epochs):
        zv, zm, eps, dlt, log = O.mul(p, x[0], x[1], y[0], y[1], t, ash)
        ok, sigma, _, _ = O.mac_check(p, [log], ash, CHK, ep)
        assert ok
        for r in range(n):
            got = out[r][ep]
            assert_equal(got["zv"], zv[r], f"epoch {ep} party {r} z values")
            assert_equal(got["zm"], zm[r], f"epoch {ep} party {r} z MACs")
            assert_equal(got["eps"], eps, f"epoch {ep} party {r} eps")
            assert_equal(got["dlt"], dlt, f"epoch {ep} party {r} delta")
            assert got["passed"]
            assert got["sig"] == O.to_ints(p, sigma)


def test_cheating_party_fails_on_the_gpu():
    p, n = O.P61, 3
    alpha, ash, epochs, out = _run(n, p, [300, 300], tamper=True)
    for r in range(n):
        assert out[r][0]["passed"] and not out[r][1]["passed"]
