"""Binomial (Revolve) checkpointing schedule — test infrastructure only.

Written from Sec. 3 ("Checkpointing performance model"): the minimal number
of forward steps p(N, M) to reverse N steps with M checkpoint slots,

    p(N, 1) = N (N - 1) / 2
    p(N, M) = min over 1 <= Nt <= N-1 of  Nt + p(Nt, M) + p(N - Nt, M - 1),

read with the split range 1..N-1 (the printed upper limit N makes the
Nt = N term refer to p(N, M) itself) and p(1, M) = 0.  M counts every slot,
including the one holding the initial state, as in p(N, 1).

The schedule Rev(s, n, M) reverses steps s..s+n-1 with the state s current
and stored in slot `slot`:
    n == 1 : youturn(s)
    M == 1 : for j = n-1 .. 1: [restore(s) unless j == n-1] advance(s, j),
             youturn(s+j); then restore(s), youturn(s)
    else   : split at the smallest Nt attaining the minimum above;
             advance(s, Nt), takeshot(s+Nt, slot+1),
             Rev(s+Nt, n-Nt, M-1, slot+1), restore(s, slot), Rev(s, Nt, M, slot)
youturn(s) is the reverse of step s (it needs the forward state s).
Actions are tuples (op, a, b):
    (ADVANCE, s, k)  (TAKESHOT, s, slot)  (RESTORE, s, slot)  (YOUTURN, s, 0)
"""
import sys
from functools import lru_cache
from math import comb

import numpy as np

ADVANCE, TAKESHOT, RESTORE, YOUTURN = 0, 1, 2, 3


def p_table(N, M):
    """tab[m][n] = p(n, m) for 1 <= m <= M, 0 <= n <= N, by the recursion."""
    tab = np.zeros((M + 1, N + 1), dtype=np.int64)
    n = np.arange(N + 1, dtype=np.int64)
    tab[1] = n * (n - 1) // 2
    tab[1][0] = 0
    for m in range(2, M + 1):
        prev = tab[m - 1]
        cur = tab[m]
        cur[0] = 0
        cur[1] = 0
        for nn in range(2, N + 1):
            nt = np.arange(1, nn, dtype=np.int64)
            cur[nn] = int(np.min(nt + cur[1:nn] + prev[nn - 1:0:-1]))
    return tab


def p_closed(N, M):
    """Griewank's closed form: with beta(s, r) = C(s + r, s) and r the smallest
    integer with beta(M, r) >= N, p = r N - beta(M + 1, r - 1)."""
    if N <= 1:
        return 0
    r = 0
    while comb(M + r, M) < N:
        r += 1
    b = comb(M + 1 + r - 1, M + 1) if r >= 1 else 0
    return r * N - b


def schedule(N, M):
    """Action list and counts {'p': advance steps, 'W': takeshots, 'R': restores}."""
    if N < 1 or M < 1:
        raise ValueError("N and M must be >= 1")
    tab = p_table(N, M)
    acts = []

    def split(n, m):
        nt = np.arange(1, n, dtype=np.int64)
        cost = nt + tab[m][1:n] + tab[m - 1][n - 1:0:-1]
        return int(np.argmin(cost)) + 1        # first minimum = smallest Nt

    def rev(s, n, m, slot):
        if n == 1:
            acts.append((YOUTURN, s, 0))
            return
        if m == 1:
            for j in range(n - 1, 0, -1):
                if j != n - 1:
                    acts.append((RESTORE, s, slot))
                acts.append((ADVANCE, s, j))
                acts.append((YOUTURN, s + j, 0))
            acts.append((RESTORE, s, slot))
            acts.append((YOUTURN, s, 0))
            return
        nt = split(n, m)
        acts.append((ADVANCE, s, nt))
        acts.append((TAKESHOT, s + nt, slot + 1))
        rev(s + nt, n - nt, m - 1, slot + 1)
        acts.append((RESTORE, s, slot))
        rev(s, nt, m, slot)

    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 4 * N + 100))
    try:
        rev(0, N, M, 0)
    finally:
        sys.setrecursionlimit(old)
    counts = {
        "p": sum(a[2] for a in acts if a[0] == ADVANCE),
        "W": sum(1 for a in acts if a[0] == TAKESHOT),
        "R": sum(1 for a in acts if a[0] == RESTORE),
    }
    return acts, counts


def simulate(acts, N, M):
    """Execute an action list on an abstract machine and check that it is a
    valid reversal: every youturn(s) sees the state s current, youturns run
    N-1..0 once each, restores read a slot holding that state, and at most
    M slots (slot 0 = the initial state) are used.  Returns the counts."""
    cur = 0
    slots = {0: 0}
    expect = N - 1
    adv = 0
    for op, a, b in acts:
        if op == ADVANCE:
            assert a == cur, "advance from %d but current state is %d" % (a, cur)
            assert b >= 1
            cur += b
            adv += b
            assert cur <= N - 1
        elif op == TAKESHOT:
            assert a == cur and 1 <= b < M, (a, b, cur)
            slots = {k: v for k, v in slots.items() if k < b}
            slots[b] = a
        elif op == RESTORE:
            assert slots.get(b) == a, "restore of state %d from slot %d" % (a, b)
            cur = a
        elif op == YOUTURN:
            assert a == cur == expect, (a, cur, expect)
            expect -= 1
        else:
            raise AssertionError(op)
    assert expect == -1
    return adv


def multistage_p(N, M, H):
    """Fewest forward steps to reverse N steps when slots 1..H are a second
    storage level written only in the first forward sweep (multistage
    checkpointing, Stumm and Walther, on which Sec. 3's model builds): the
    first sweep stores the starts of segments there, and each segment is
    reversed from its start by Revolve with the M - H remaining slots (its
    start included).  By the recursion over the first segment's length l,

        C(n, 0) = p(n, M - H)
        C(n, h) = min( C(n, h-1),  min over 1 <= l <= n-1 of
                       l + C(n - l, h - 1) + p(l, M - H) ),

    C(N, H) is returned (every segmentation is tried)."""
    md = M - H
    tab = p_table(N, md)[md]
    C = tab.copy()
    for h in range(1, H + 1):
        nxt = C.copy()
        for n in range(2, N + 1):
            l = np.arange(1, n)
            nxt[n] = min(nxt[n], int(np.min(l + C[n - l] + tab[l])))
        C = nxt
    return int(C[N])


@lru_cache(maxsize=None)
def counts(N, M):
    return schedule(N, M)[1]
