"""The online phase with one party per process and GPU.

Each process holds one party's shares on its own device; the parties meet
only at the two exchanges of the protocol (the paper runs its parties as
separate processes, Sec. IV-A, and names one GPU per party as future work,
Sec. V-B):

* the open of a Beaver batch (Sec. II-A.3): every party contributes its
  rows eps_i = x_i - a_i and delta_i = y_i - b_i, the rows are all-gathered
  and every party sums them into the public eps, delta;
* the batched MAC check (Sec. II-A.2/II-A.4): every party computes
  sigma_i = S_i - alpha_i A over the epoch's opened values, commits to it
  (SHA-256 of sigma_i and a fresh nonce), the commitments are all-gathered,
  then the sigmas and nonces; each party checks every commitment and accepts
  iff the sigmas sum to zero mod p.

The local steps run in the library's party kernels (``DeviceParty``); the
exchanges go through a communicator with ``all_gather`` (tensors) and
``all_gather_obj`` (small host objects) -- ``TorchComm`` over a
torch.distributed group (NCCL between GPUs).  No other data crosses between
parties, and a party never sees another party's shares of x, y or the
triples.
"""
from __future__ import annotations

import hashlib
import secrets

import torch
import torch.distributed as dist


def _lib():
    # the CUDA library is loaded by the device-side classes only: the
    # protocol and the communicator need none of it
    from . import shares as SH
    from . import spdz as S
    return S, SH


class TorchComm:
    """All-gathers over a torch.distributed process group (one rank per party,
    rank = party index)."""

    def __init__(self, group=None):
        self.group = group
        self.world = dist.get_world_size(group)

    def all_gather(self, t: torch.Tensor) -> torch.Tensor:
        out = [torch.empty_like(t) for _ in range(self.world)]
        dist.all_gather(out, t.contiguous(), group=self.group)
        return torch.stack(out)

    def all_gather_obj(self, obj):
        out = [None] * self.world
        dist.all_gather_object(out, obj, group=self.group)
        return out


class DeviceParty:
    """This party's local steps on its GPU through the library."""

    def __init__(self, party: int, n: int, field: int, alpha_share: torch.Tensor, check_seed: int, stream=None):
        S, _ = _lib()
        self.S = S
        self.party, self.n, self.field = party, n, field
        self.h = S.spdz_party_create(party, n, field, stream)
        S.spdz_party_load_alpha(self.h, alpha_share)
        S.spdz_party_set_check_seed(self.h, check_seed)

    def close(self):
        self.S.spdz_party_destroy(self.h)

    def _empty(self, N, like: torch.Tensor):
        shape = (N, 2) if self.field == self.S.SPDZ_F127 else (N,)
        return torch.empty(shape, dtype=like.dtype, device=like.device)

    def mask(self, x, y, a, b, N):
        eps_i, dlt_i = self._empty(N, x.val), self._empty(N, x.val)
        self.S.spdz_party_mask(self.h, x.buf(), y.buf(), a.buf(), b.buf(), eps_i, dlt_i, N)
        return eps_i, dlt_i

    def open_sum(self, rows, N):
        out = self._empty(N, rows)
        self.S.spdz_party_open_sum(self.h, rows.contiguous(), N, out)
        return out

    def combine(self, eps, dlt, x, y, a, b, c, z, N):
        self.S.spdz_party_combine(self.h, eps, dlt, x.buf(), y.buf(), a.buf(), b.buf(), c.buf(), z.buf(), N)

    def sigma(self) -> int:
        words, _ = self.S.spdz_party_sigma(self.h, 2 if self.field == self.S.SPDZ_F127 else 1)
        return int(words[0]) | (int(words[1]) << 64 if words.size > 1 else 0)


class PartyRow:
    """One party's row of a shared array on its device: value and MAC shares
    (the word layout of ``shares``), with the spdz_buf the party calls take."""

    def __init__(self, val: torch.Tensor, mac: torch.Tensor):
        self.val, self.mac = val, mac

    def buf(self):
        S, _ = _lib()
        return S.buf(self.val, self.mac, 0)

    @staticmethod
    def alloc(field: int, count: int, device="cuda") -> "PartyRow":
        _, SH = _lib()
        sh = SH.alloc(field, 1, count, device=device)
        return PartyRow(sh.val[0], sh.mac[0])


class PartyProtocol:
    """The exchanges of the online phase for party `party` of `n`, over a
    communicator; `local` does the party's own arithmetic."""

    def __init__(self, local, comm, p: int, party: int, n: int):
        self.local, self.comm, self.p, self.party, self.n = local, comm, p, party, n

    def mul_batch(self, x, y, a, b, c, z, N: int):
        """Beaver products of N pairs: z = x y with this party's triple rows.
        Returns the public eps, delta."""
        eps_i, dlt_i = self.local.mask(x, y, a, b, N)
        rows = self.comm.all_gather(torch.stack([eps_i, dlt_i]))       # [n, 2, N(, 2)]
        eps = self.local.open_sum(rows[:, 0].contiguous(), N)
        dlt = self.local.open_sum(rows[:, 1].contiguous(), N)
        self.local.combine(eps, dlt, x, y, a, b, c, z, N)
        return eps, dlt

    def mac_check(self):
        """Batched MAC check of the epoch: (passed, every party's sigma).
        Raises ValueError when a party's revealed sigma does not match its
        commitment."""
        sig = self.local.sigma()
        nonce = secrets.token_bytes(16)
        nb = 16 if self.p >= (1 << 64) else 8
        commit = hashlib.sha256(sig.to_bytes(nb, "little") + nonce).hexdigest()
        commits = self.comm.all_gather_obj(commit)
        revealed = self.comm.all_gather_obj((sig, nonce.hex()))
        for k, (s_k, n_k) in enumerate(revealed):
            if hashlib.sha256(int(s_k).to_bytes(nb, "little") + bytes.fromhex(n_k)).hexdigest() != commits[k]:
                raise ValueError(f"party {k}: revealed sigma does not match its commitment")
        sigmas = [int(s_k) for s_k, _ in revealed]
        return sum(sigmas) % self.p == 0, sigmas
