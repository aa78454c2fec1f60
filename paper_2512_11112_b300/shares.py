"""Device share tensors for the C ABI.

A shared array of ``count`` field elements for ``n`` parties is a pair of
torch tensors ``val`` and ``mac`` of shape [n, stride] (p61) or
[n, stride, 2] (p127), dtype int64 (the bit patterns of the uint64 words),
on the GPU.  The stride is rounded up to an even number of elements so every
party row stays 16-byte aligned.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import spdz as S


def words(field: int) -> int:
    return 1 if field == S.SPDZ_F61 else 2


def field_of(p: int) -> int:
    return S.SPDZ_F61 if p == S.P61 else S.SPDZ_F127


def empty(field: int, *dims, device="cuda") -> torch.Tensor:
    shape = tuple(dims) + ((2,) if words(field) == 2 else ())
    return torch.empty(shape, dtype=torch.int64, device=device)


def zeros(field: int, *dims, device="cuda") -> torch.Tensor:
    shape = tuple(dims) + ((2,) if words(field) == 2 else ())
    return torch.zeros(shape, dtype=torch.int64, device=device)


@dataclass
class Shared:
    field: int
    n: int
    count: int
    val: torch.Tensor
    mac: torch.Tensor

    @property
    def stride(self) -> int:
        return int(self.val.shape[1])

    def buf(self, offset: int = 0) -> S.spdz_buf:
        return S.buf(self.val, self.mac, self.stride, offset, words(self.field))

    def host(self):
        """(val, mac) as numpy uint64 arrays [n, count(, 2)]."""
        v = self.val[:, :self.count].cpu().numpy().view(np.uint64)
        m = self.mac[:, :self.count].cpu().numpy().view(np.uint64)
        return np.ascontiguousarray(v), np.ascontiguousarray(m)


def alloc(field: int, n: int, count: int, device="cuda", fill_zero: bool = False) -> Shared:
    stride = max(2, count + (count & 1))
    mk = zeros if fill_zero else empty
    return Shared(field, n, count, mk(field, n, stride, device=device), mk(field, n, stride, device=device))


def to_host(t: torch.Tensor) -> np.ndarray:
    return np.ascontiguousarray(t.cpu().numpy().view(np.uint64))


def from_host(a: np.ndarray, device="cuda") -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to(device)
