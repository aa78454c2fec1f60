"""Shared helpers of the GPU parity tests: build a context on torch's
current stream, deal inputs on the device, and deal the same inputs with the
CPU oracle from the same seeds (each side with its own dealer)."""
from __future__ import annotations

import numpy as np
import torch

import oracle as O


def _mods():
    # imported lazily: collecting the GPU tests must not load the CUDA library
    from paper_2512_11112_b300 import shares as SH
    from paper_2512_11112_b300 import spdz as S
    return S, SH


def ctx_for(n: int, p: int):
    S, SH = _mods()
    stream = torch.cuda.current_stream().cuda_stream
    return S.spdz_ctx_create(n, SH.field_of(p), stream)


class DeviceWorld:
    """Device dealer: alpha shares, inputs x (sub 0), y (sub 1), a triple pool."""

    def __init__(self, ctx, p: int, n: int, seed: int, N: int, n_triples: int, input_subs=(0, 1)):
        S, SH = _mods()
        self.ctx, self.p, self.n, self.seed = ctx, p, n, seed
        self.field = SH.field_of(p)
        self.w = SH.words(self.field)
        self.alpha_sh = SH.zeros(self.field, n)
        S.spdz_deal_alpha(ctx, seed, self.alpha_sh)
        self.inputs = []
        for sub in input_subs:
            sh = SH.alloc(self.field, n, N)
            S.spdz_deal_shared(ctx, seed, S.SPDZ_KIND_INPUT, sub, 0, N, self.alpha_sh, None, sh.buf())
            self.inputs.append(sh)
        self.tri = [SH.alloc(self.field, n, max(n_triples, 1)) for _ in range(3)]
        if n_triples:
            S.spdz_deal_triples(ctx, seed, 0, n_triples, self.alpha_sh, *[t.buf() for t in self.tri])
        S.spdz_load_preproc(ctx, self.alpha_sh, *[t.buf() for t in self.tri], n_triples)


class OracleWorld:
    """The same world from the oracle's own dealer."""

    def __init__(self, p: int, n: int, seed: int, N: int, n_triples: int, input_subs=(0, 1)):
        self.p, self.n = p, n
        self.alpha, self.alpha_sh = O.deal_alpha(p, n, seed)
        self.inputs = [O.deal_shared(p, n, seed, O.K_INPUT, sub, 0, N, self.alpha) for sub in input_subs]
        self.tri = O.deal_triples(p, n, seed, 0, n_triples, self.alpha) if n_triples else None


def host(t: torch.Tensor, count: int | None = None) -> np.ndarray:
    S, SH = _mods()
    if count is not None:
        t = t[:, :count] if t.dim() >= 2 else t[:count]
    return SH.to_host(t.contiguous())


def assert_equal(got: np.ndarray, exp: np.ndarray, what: str):
    got = np.asarray(got, dtype=np.uint64)
    exp = np.asarray(exp, dtype=np.uint64)
    assert got.shape == exp.shape, (what, got.shape, exp.shape)
    if not np.array_equal(got, exp):
        bad = np.argwhere(got != exp)
        raise AssertionError(f"{what}: {len(bad)} mismatching words, first at {bad[0].tolist()}: "
                             f"got {got[tuple(bad[0])]} expected {exp[tuple(bad[0])]}")
