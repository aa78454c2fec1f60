"""Device share tensors for the C ABI.

A shared array of ``count`` field elements for ``n`` parties is a pair of
torch tensors ``val`` and ``mac`` of shape [n, stride] (p61: int64 holding the
uint64 words; p = 2^32-5: int32 holding the uint32 words) or [n, stride, 2]
(p127: int64 words, low first), on the GPU.  The stride is rounded up so
every party row stays 16-byte aligned.  Host copies are numpy uint64 arrays
in every field (p = 2^32-5 elements are widened), the oracle's format.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import spdz as S


def words(field: int) -> int:
    """64-bit words of a host element (2 for p127, else 1)."""
    return 2 if field == S.SPDZ_F127 else 1


def field_of(p: int) -> int:
    return {S.P61: S.SPDZ_F61, S.P127: S.SPDZ_F127, S.P32: S.SPDZ_F32}[p]


def _dtype(field: int):
    return torch.int32 if field == S.SPDZ_F32 else torch.int64


def _shape(field: int, dims):
    return tuple(dims) + ((2,) if field == S.SPDZ_F127 else ())


def empty(field: int, *dims, device="cuda") -> torch.Tensor:
    return torch.empty(_shape(field, dims), dtype=_dtype(field), device=device)


def zeros(field: int, *dims, device="cuda") -> torch.Tensor:
    return torch.zeros(_shape(field, dims), dtype=_dtype(field), device=device)


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
        return to_host(self.val[:, :self.count]), to_host(self.mac[:, :self.count])


def alloc(field: int, n: int, count: int, device="cuda", fill_zero: bool = False) -> Shared:
    q = 4 if field == S.SPDZ_F32 else 2          # elements per 16 bytes (p127: one per 16 B)
    stride = max(q, -(-count // q) * q)
    mk = zeros if fill_zero else empty
    return Shared(field, n, count, mk(field, n, stride, device=device), mk(field, n, stride, device=device))


def to_host(t: torch.Tensor) -> np.ndarray:
    """Device words -> numpy uint64 (int32 words are p = 2^32-5 elements, widened)."""
    a = t.contiguous().cpu().numpy()
    if a.dtype == np.int32:
        return np.ascontiguousarray(a.view(np.uint32).astype(np.uint64))
    return np.ascontiguousarray(a.view(np.uint64))


def from_host(a: np.ndarray, device="cuda", field: int | None = None) -> torch.Tensor:
    """numpy uint64 words -> device tensor (int32 words for field p = 2^32-5)."""
    a = np.ascontiguousarray(a)
    if field == S.SPDZ_F32:
        return torch.from_numpy(a.astype(np.uint32).view(np.int32)).to(device)
    return torch.from_numpy(a.view(np.int64)).to(device)
