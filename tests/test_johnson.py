"""Johnson's rule (Section 3.3 pipelining: copy, then decode) through the C ABI.

The rule is optimal for the two-machine flow shop, so the makespan of the
order zf_johnson_order returns must equal the brute-force minimum over all
permutations of small job sets.
"""
from __future__ import annotations

import itertools

import numpy as np
import pytest

import paper_2602_08190_gb300 as zf


def makespan(copy, dec, order) -> float:
    t_copy = t_dec = 0.0
    for i in order:
        t_copy += copy[i]
        t_dec = max(t_dec, t_copy) + dec[i]
    return t_dec


@pytest.mark.parametrize("n", range(1, 9))
def test_johnson_is_optimal_by_brute_force(n):
    rng = np.random.default_rng(100 + n)
    for trial in range(40 if n < 8 else 8):
        # float32 times (what the ABI takes); some equal pairs for ties
        copy = rng.integers(1, 50, n).astype(np.float32)
        dec = rng.integers(1, 50, n).astype(np.float32)
        if trial % 5 == 0:
            dec[: n // 2] = copy[: n // 2]
        order = zf.zf_johnson_order(copy, dec)
        assert sorted(order.tolist()) == list(range(n))
        best = min(makespan(copy, dec, p) for p in itertools.permutations(range(n)))
        assert makespan(copy, dec, order) == pytest.approx(best, abs=1e-3), (copy, dec, order)


def test_johnson_order_shape_of_the_rule():
    # copy-light jobs first by increasing copy, then copy-heavy ones by decreasing decode
    copy = np.array([5, 1, 9, 3, 7], np.float32)
    dec = np.array([2, 4, 8, 6, 1], np.float32)
    # copy < decode: jobs 1 (c=1), 3 (c=3); then the rest by decode 8 (2), 2 (0), 1 (4)
    assert zf.zf_johnson_order(copy, dec).tolist() == [1, 3, 2, 0, 4]
    assert zf.zf_johnson_order(np.zeros(0, np.float32), np.zeros(0, np.float32)).tolist() == []


def test_johnson_order_rejects_bad_times():
    with pytest.raises(zf.ZfError):
        zf.zf_johnson_order(np.array([1, -1], np.float32), np.array([1, 1], np.float32))
    with pytest.raises(zf.ZfError):
        zf.zf_johnson_order(np.array([1, np.nan], np.float32), np.array([1, 1], np.float32))
