"""Writes tests/golden/revolve_counts.txt from the oracle alone.

p(N, M) comes from the oracle's closed form (Griewank), W(N, M) from the
oracle schedule (smallest split on ties) for N <= 1000.  Run from the
repository root:  python tests/golden/make_revolve_counts.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import revolve as R  # noqa: E402

CASES = [(500, 10), (1000, 20), (3000, 8), (3000, 16), (3000, 32), (3000, 64), (3000, 128),
         (3000, 256), (1500, 32), (2000, 16)]

HEADER = """# Binomial checkpointing counts for the workloads of the hot path.
# columns: N (steps)  M (slots incl. the initial state)  p(N, M)  W(N, M)
# p: Sec. 3, Eq. "eqn:recompute" (minimal forward steps), evaluated with
#    Griewank's closed form p = r N - C(M + r, M + 1), r the smallest
#    integer with C(M + r, M) >= N.  Hand check of the first row: r = 4
#    (C(14,10) = 1001 >= 500 > C(13,10) = 286), p = 2000 - C(14,11) = 1636.
# W: checkpoint writes of the smallest-split schedule (no value in the
#    paper; a regression value of the oracle schedule), -1 where N > 1000.
# Written by tests/golden/make_revolve_counts.py (calls oracle/ only).
"""


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "revolve_counts.txt")
    with open(path, "w") as f:
        f.write(HEADER)
        for N, M in CASES:
            W = R.schedule(N, M)[1]["W"] if N <= 1000 else -1
            f.write("%-5d %-4d %-6d %d\n" % (N, M, R.p_closed(N, M), W))


if __name__ == "__main__":
    main()
