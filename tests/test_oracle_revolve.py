"""Pins of the oracle's binomial checkpointing schedule (CPU only).

p(N, M) is fixed by the recursion of Sec. 3, Eq. "eqn:recompute"; it must
equal Griewank's closed form, and the schedule must be a valid reversal
(checked by executing it on an abstract machine) whose advance count is
p(N, M).  Stored values are in tests/golden/revolve_counts.txt.
"""
import os

import numpy as np
import pytest

from oracle import revolve as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "revolve_counts.txt")


def test_recursion_equals_closed_form():
    tab = R.p_table(150, 14)
    for m in range(1, 15):
        for n in range(1, 151):
            assert tab[m][n] == R.p_closed(n, m), (n, m)


def test_base_cases():
    assert R.p_closed(1, 5) == 0
    for n in range(1, 40):
        assert R.p_table(n, 1)[1][n] == n * (n - 1) // 2
        # with at least as many slots as steps the sweep is done once
        assert R.p_table(n, n)[n][n] == n - 1


@pytest.mark.parametrize("N,M", [(1, 1), (2, 1), (7, 1), (7, 2), (13, 3), (40, 4), (97, 5),
                                 (64, 64), (200, 7), (500, 10), (1000, 20)])
def test_schedule_is_valid_and_minimal(N, M):
    acts, c = R.schedule(N, M)
    adv = R.simulate(acts, N, M)
    assert adv == c["p"] == R.p_closed(N, M)
    assert sum(1 for a in acts if a[0] == R.YOUTURN) == N
    # every youturn but the first follows exactly one restore
    assert c["R"] == N - 1


def test_split_ties_take_smallest():
    # N = 6, M = 2: costs Nt + p(Nt,2) + p(6-Nt,1) = 1+0+10, 2+1+6, 3+2+3, 4+4+1, 5+6+0
    #             = 11, 9, 8, 9, 11 -> Nt = 3 is the unique minimum
    acts, _ = R.schedule(6, 2)
    assert acts[0] == (R.ADVANCE, 0, 3)
    # N = 5, M = 2: 1+0+6, 2+1+3, 3+2+1, 4+4+0 = 7, 6, 6, 8 -> tie 2 / 3, take 2
    acts, _ = R.schedule(5, 2)
    assert acts[0] == (R.ADVANCE, 0, 2)


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([int(v) for v in line.split()])
    return rows


def test_golden_counts():
    rows = _golden()
    assert rows
    for N, M, p, W in rows:
        assert R.p_closed(N, M) == p
        if N <= 1000:
            assert R.counts(N, M)["p"] == p and R.counts(N, M)["W"] == W
