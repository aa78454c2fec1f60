"""Pins of the oracle's input sharing (mask, publish eps = x - r, [x] = [r] +
eps): the shares reconstruct to the clear inputs, the MAC relation holds,
eps is x - r, and the dealt masks reconstruct to the owner's clear masks."""
import numpy as np
import pytest

import oracle as O


@pytest.mark.parametrize("p,n", [(O.P61, 2), (O.P127, 3), (O.P32, 3), (101, 2)])
def test_input_sharing_reconstructs_and_authenticates(p, n):
    seed, owner, count = 9, n - 1, 57
    alpha, ash = O.deal_alpha(p, n, seed)
    rv, rm, r = O.deal_input_masks(p, n, seed, owner, 0, count, alpha)
    a = O.to_ints(p, np.asarray([alpha]))[0]
    assert O.reconstruct(p, rv) == O.to_ints(p, r)
    assert O.reconstruct(p, rm) == [(a * v) % p for v in O.to_ints(p, r)]
    rng = np.random.default_rng(p % 1000)
    xs = [int(v) % p for v in rng.integers(0, 2**62, count)]
    xs[:3] = [0, 1, p - 1]
    x = O.to_array(p, xs)
    xv, xm, eps = O.input_share(p, x, r, rv, rm, ash)
    assert O.to_ints(p, eps) == [(u - v) % p for u, v in zip(xs, O.to_ints(p, r))]
    assert O.reconstruct(p, xv) == xs
    assert O.reconstruct(p, xm) == [(a * v) % p for v in xs]
    # masks of another owner come from another stream
    rv2, _, r2 = O.deal_input_masks(p, n, seed, (owner + 1) % n, 0, count, alpha)
    assert O.to_ints(p, r2) != O.to_ints(p, r)
