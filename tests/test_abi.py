"""The C-ABI library: it loads without a GPU, exports every entry point that
include/ckfwi.h declares, and its host-only Revolve schedule is bit-exact
against the oracle's (Sec. 3, Eq. "eqn:recompute")."""
import os
import re

import numpy as np
import pytest

from oracle import revolve as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1810_05268_gb300 import build
    build.build()
    from paper_1810_05268_gb300 import _lib
    return _lib.lib()


def declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ckfwi_\w+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert "ckfwi_adjoint_gradient" in names and len(names) >= 11
    for n in names:
        assert hasattr(L, n), n


def test_error_strings(L):
    from paper_1810_05268_gb300 import ckfwi as C
    assert C.error_string(0) == "ok"
    assert "pool" in C.error_string(C.POOL_OVERFLOW)
    assert C.error_string(-99) == "unknown status"


@pytest.mark.parametrize("N,M", [(1, 1), (2, 1), (9, 1), (9, 2), (13, 3), (40, 4), (97, 5), (64, 64),
                                 (200, 7), (500, 10), (1000, 20), (300, 300), (257, 16)])
def test_revolve_schedule_bit_exact_vs_oracle(L, N, M):
    from paper_1810_05268_gb300 import ckfwi as C
    acts, (p, W, Rr) = C.revolve_schedule(N, M)
    ref, cnt = R.schedule(N, M)
    assert np.array_equal(acts, np.array(ref, dtype=np.int32).reshape(-1, 3))
    assert (p, W, Rr) == (cnt["p"], cnt["W"], cnt["R"])


@pytest.mark.parametrize("N,M", [(3000, 8), (3000, 32), (3000, 256), (1500, 32)])
def test_revolve_counts_large(L, N, M):
    from paper_1810_05268_gb300 import ckfwi as C
    acts, (p, W, Rr) = C.revolve_schedule(N, M)
    assert p == R.p_closed(N, M)
    assert R.simulate([tuple(a) for a in acts.tolist()], N, M) == p
    assert Rr == N - 1


def test_invalid_arguments_rejected_on_host(L):
    from paper_1810_05268_gb300 import ckfwi as C
    with pytest.raises(C.CkfwiError):
        C.revolve_schedule(0, 3)
    with pytest.raises(C.CkfwiError):
        C.codec_bound_words(4, 4, 4, 4)


@pytest.mark.parametrize("N,M,H", [(1, 3, 1), (2, 2, 1), (9, 3, 1), (9, 3, 2), (17, 4, 2), (30, 5, 3), (40, 3, 2),
                                   (25, 6, 5), (60, 8, 4), (12, 12, 11), (50, 2, 1), (200, 20, 12),
                                   (1000, 60, 40), (1000, 9, 4)])
def test_multistage_schedule_is_valid_and_takes_the_fewest_steps(L, N, M, H):
    """Two storage levels: a valid reversal that writes each host slot at
    most once, all in the first sweep, with the fewest forward steps of its
    family (every segmentation tried by the oracle)."""
    from paper_1810_05268_gb300 import ckfwi as C
    acts, (p, W, Rr) = C.multistage_schedule(N, M, H)
    trip = [tuple(a) for a in acts.tolist()]
    assert R.simulate(trip, N, M) == p
    assert p == R.multistage_p(N, M, H)
    assert W == sum(1 for a in trip if a[0] == R.TAKESHOT)
    assert Rr == sum(1 for a in trip if a[0] == R.RESTORE)
    first_turn = next(i for i, a in enumerate(trip) if a[0] == R.YOUTURN)
    host_w = [i for i, a in enumerate(trip) if a[0] == R.TAKESHOT and a[2] <= H]
    assert len(host_w) <= H and all(i < first_turn for i in host_w)
    assert len({trip[i][2] for i in host_w}) == len(host_w)
    # each segment's start is restored from the host once, then held on the device
    host_r = [a for a in trip if a[0] == R.RESTORE and 1 <= a[2] <= H]
    assert len({a[2] for a in host_r}) <= len(host_w)


def test_multistage_without_host_slots_is_revolve(L):
    from paper_1810_05268_gb300 import ckfwi as C
    a0, c0 = C.multistage_schedule(300, 12, 0)
    a1, c1 = C.revolve_schedule(300, 12)
    assert np.array_equal(a0, a1) and c0 == c1
    # the bench's two-level configuration: forty host checkpoints at most,
    # against 316 in the Revolve placement of the same slots
    _, (p, W, _) = C.multistage_schedule(1000, 60, 40)
    assert p <= 1.06 * R.p_closed(1000, 60)
    with pytest.raises(C.CkfwiError):
        C.multistage_schedule(100, 5, 5)
