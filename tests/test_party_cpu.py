"""The party-per-process online phase on CPU: 2 and 3 gloo ranks, one party
each, run the protocol's exchanges (all-gather of the eps_i, delta_i rows;
commitments, then the sigmas) with a host stand-in for the party's local
steps (HostParty below: the paper's per-party formulas on Python integers,
test infrastructure only; the library's party kernels are checked against
the oracle on the GPU in test_gpu_party.py).  Every party's z shares, the
public eps, delta and every sigma must equal the oracle's all-party batch
and check; a party that sends a wrong eps_i row makes the check fail."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O

SEED, CHK, N = 9, 5, 37


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class HostRow:
    def __init__(self, p, val, mac):
        self.p, self.val, self.mac = p, O.to_ints(p, val), O.to_ints(p, mac)


class HostParty:
    """One party's local steps on Python integers (stand-in for DeviceParty)."""

    def __init__(self, p, party, alpha_i, tamper=False):
        self.p, self.party, self.alpha, self.tamper = p, party, alpha_i, tamper
        self.key_epoch, self.opened = 0, 0
        self.A = self.S = 0

    def _t(self, ints):
        return torch.from_numpy(np.ascontiguousarray(O.to_array(self.p, ints)).view(np.int64))

    def _ints(self, t):
        return O.to_ints(self.p, t.numpy().view(np.uint64))

    def mask(self, x, y, a, b, n):
        p = self.p
        e = [(x.val[j] - a.val[j]) % p for j in range(n)]
        d = [(y.val[j] - b.val[j]) % p for j in range(n)]
        if self.tamper:
            e[5] = (e[5] + 1) % p
        return self._t(e), self._t(d)

    def open_sum(self, rows, n):
        k = rows.shape[0]
        parts = [self._ints(rows[r].contiguous()) for r in range(k)]
        return self._t([sum(col) % self.p for col in zip(*parts)])

    def combine(self, eps, dlt, x, y, a, b, c, z, n):
        p = self.p
        e, d = self._ints(eps), self._ints(dlt)
        r = O.to_ints(p, O.check_coeffs(p, CHK, self.key_epoch, self.opened, 2 * n))
        zv, zm = [], []
        for j in range(n):
            de = e[j] * d[j] % p
            zv.append((c.val[j] + e[j] * b.val[j] + d[j] * a.val[j] + (de if self.party == 0 else 0)) % p)
            zm.append((c.mac[j] + e[j] * b.mac[j] + d[j] * a.mac[j] + self.alpha * de) % p)
            self.A = (self.A + r[2 * j] * e[j] + r[2 * j + 1] * d[j]) % p
            self.S = (self.S + r[2 * j] * (x.mac[j] - a.mac[j]) + r[2 * j + 1] * (y.mac[j] - b.mac[j])) % p
        z.val, z.mac = zv, zm
        self.opened += 2 * n

    def sigma(self):
        s = (self.S - self.alpha * self.A) % self.p
        self.A = self.S = 0
        self.opened = 0
        self.key_epoch += 1
        return s


def _worker(rank, world, port, p, tamper_party, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2512_11112_b300.party import PartyProtocol, TorchComm
        alpha, ash = O.deal_alpha(p, world, SEED)
        x = O.deal_shared(p, world, SEED, O.K_INPUT, 0, 0, N, alpha)
        y = O.deal_shared(p, world, SEED, O.K_INPUT, 1, 0, N, alpha)
        t = O.deal_triples(p, world, SEED, 0, N, alpha)
        row = lambda v, m: HostRow(p, v[rank], m[rank])          # noqa: E731  this party's shares only
        X, Y = row(x[0], x[1]), row(y[0], y[1])
        A_, B_, C_ = row(t.av, t.am), row(t.bv, t.bm), row(t.cv, t.cm)
        Z = HostRow(p, O.zeros(p, N), O.zeros(p, N))
        local = HostParty(p, rank, O.to_ints(p, ash[rank:rank + 1])[0], tamper=(rank == tamper_party))
        proto = PartyProtocol(local, TorchComm(), p, rank, world)
        eps, dlt = proto.mul_batch(X, Y, A_, B_, C_, Z, N)
        passed, sigmas = proto.mac_check()
        out[rank] = {"zv": Z.val, "zm": Z.mac, "eps": local._ints(eps), "dlt": local._ints(dlt),
                     "passed": passed, "sigmas": sigmas}
    finally:
        dist.destroy_process_group()


def _run(world, p, tamper_party=-1):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, p, tamper_party, out)) for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(180)
            assert pr.exitcode == 0
        return dict(out)


@pytest.mark.parametrize("world,p", [(2, O.P61), (3, O.P61), (3, O.P127)])
def test_party_per_process_matches_oracle(world, p):
    out = _run(world, p)
    alpha, ash = O.deal_alpha(p, world, SEED)
    xv, xm, _ = O.deal_shared(p, world, SEED, O.K_INPUT, 0, 0, N, alpha)
    yv, ym, _ = O.deal_shared(p, world, SEED, O.K_INPUT, 1, 0, N, alpha)
    tri = O.deal_triples(p, world, SEED, 0, N, alpha)
    zv, zm, eps, dlt, log = O.mul(p, xv, xm, yv, ym, tri, ash)
    ok, sigma, _, _ = O.mac_check(p, [log], ash, CHK, 0)
    assert ok
    for r in range(world):
        assert out[r]["zv"] == O.to_ints(p, zv[r]) and out[r]["zm"] == O.to_ints(p, zm[r]), r
        assert out[r]["eps"] == O.to_ints(p, eps) and out[r]["dlt"] == O.to_ints(p, dlt), r
        assert out[r]["passed"] and out[r]["sigmas"] == O.to_ints(p, sigma), r


def test_cheating_party_fails_the_check():
    """Party 1 sends eps_1 + 1 at element 5: every party's check fails, and the
    sigmas sum to -alpha r_10 (the shift of the opened eps_5, index 2*5)."""
    p, world = O.P61, 3
    out = _run(world, p, tamper_party=1)
    alpha, _ = O.deal_alpha(p, world, SEED)
    a = O.to_ints(p, np.array([alpha]))[0]
    r10 = O.to_ints(p, O.check_coeffs(p, CHK, 0, 10, 1))[0]
    for k in range(world):
        assert not out[k]["passed"]
        assert sum(out[k]["sigmas"]) % p == (-a * r10) % p
