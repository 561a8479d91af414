"""The time model of a checkpointed gradient (Sec. 3, Sec. 4) on the host:
schedule counts against the oracle's Revolve, and the choices the model
makes in the regimes the paper describes."""
import pytest

from oracle import revolve as R

P = pytest.importorskip("paper_1810_05268_gb300.perfmodel")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1810_05268_gb300 import build
    build.build()


@pytest.mark.parametrize("nt,slots", [(1000, 20), (500, 10), (300, 7), (60, 5), (40, 40)])
def test_counts_follow_revolve(nt, slots):
    nf, nc, nd = P.counts(nt, slots, "fp32")
    if slots >= nt:
        assert nf == nt
    else:
        acts, cnt = R.schedule(nt, slots)
        assert nf == cnt["p"] + 1 == R.p_closed(nt, slots) + 1
        nf2, nc2, nd2 = P.counts(nt, slots, "codec")
        assert nf2 == nf and nc2 == 2 * cnt["W"]
        r_slot = sum(1 for a in acts if a[0] == R.RESTORE and a[2] > 0)
        assert r_slot <= nd2 <= 2 * r_slot      # one or two fields per restore from a slot
    assert nc == nd == 0


def test_slots_at_equal_memory():
    assert P.slots_for(20, "fp32", 1000) == 20
    assert P.slots_for(20, "fp16", 1000) == 39
    assert P.slots_for(20, "codec", 1000, f_min=7.4) == 134
    assert P.slots_for(20, "codec", 100, f_min=50.0) == 100


def test_free_compression_wins_and_costly_compression_loses():
    base = dict(c_f=0.05, c_r=0.09, t_d=0.02, f_min=8.0)
    cheap = P.Costs(t_c=1e-4, **base)
    dear = P.Costs(t_c=0.5, **base)
    assert P.choose(cheap, 1000, 20, modes=("fp32", "codec"))[0] == "codec"
    assert P.choose(dear, 1000, 20, modes=("fp32", "codec"))[0] == "fp32"


def test_predicted_time_falls_with_memory_and_reaches_store_all():
    c = P.Costs(c_f=0.05, c_r=0.09, t_c=0.08, t_d=0.02, f_min=8.0)
    rows = P.sweep(c, 400, [2, 5, 20, 80, 400])
    t32 = [r["fp32"] for r in rows]
    assert all(a >= b for a, b in zip(t32, t32[1:]))
    assert rows[-1]["fp32"] == pytest.approx(400 * (0.05 + 0.09))


def test_regimes():
    """Little memory: compression pays; ample memory: plain checkpoints win."""
    c = P.Costs(c_f=0.05, c_r=0.09, t_c=0.03, t_d=0.01, f_min=10.0)
    low = P.choose(c, 1000, 3, modes=("fp32", "codec"))
    high = P.choose(c, 1000, 500, modes=("fp32", "codec"))
    assert low[0] == "codec"
    assert high[0] == "fp32"


def test_gradient_tolerance_excludes_modes():
    c = P.Costs(c_f=0.05, c_r=0.09, c_r16=0.09, t_c=1e-4, t_d=1e-4, f_min=8.0,
                grad_err={"bf16": 0.03, "fp16": 0.004, "codec": 0.0005})
    assert P.choose(c, 1000, 20, modes=("fp32", "bf16"), grad_tol=1e-2)[0] == "fp32"
    assert P.choose(c, 1000, 20, modes=("fp32", "bf16"))[0] == "bf16"


def test_working_field_restores_take_the_16_bit_reverse_cost():
    """Modes whose restores fill a working field (16-bit up-cast, codec
    decode) take the reverse cost measured in the 16-bit run; FP32 modes
    keep the FP32 run's; without a 16-bit measurement every mode uses C_R."""
    base = dict(c_f=0.05, c_r=0.09, t_c=0.03, t_d=0.01, f_min=10.0, t_d16=0.01)
    c0 = P.Costs(**base)
    c1 = P.Costs(c_r16=0.1, **base)
    nt = 300
    for mode, slots in (("fp16", 9), ("bf16", 9), ("codec", 20)):
        d = P.predict(c1, nt, slots, mode) - P.predict(c0, nt, slots, mode)
        assert d == pytest.approx(nt * (0.1 - 0.09), rel=1e-12), mode
    for slots in (5, nt):
        assert P.predict(c1, nt, slots, "fp32") == P.predict(c0, nt, slots, "fp32")


def _oracle_peak(nt, slots, size_of):
    # independent replay on the oracle's Revolve: the slots held at each takeshot
    acts, _ = R.schedule(nt, slots)
    held, peak = {}, 0.0
    for op, a, b in acts:
        if op == R.TAKESHOT:
            held = {k: v for k, v in held.items() if k < b}
            held[b] = size_of(a)
            peak = max(peak, sum(held.values()))
    return peak


@pytest.mark.parametrize("nt,slots", [(200, 5), (300, 17), (120, 60), (50, 50)])
def test_pool_peak_matches_an_independent_replay(nt, slots):
    import numpy as np
    rng = np.random.default_rng(nt + slots)
    sz = rng.uniform(1.0, 9.0, nt)
    f = lambda s: float(sz[s])
    assert P.pool_peak(nt, slots, f) == pytest.approx(_oracle_peak(nt, slots, f), rel=1e-12)


def test_uniform_sizes_give_the_worst_ratio_rule():
    # equal sizes S: the most slots is the budget over S, plus the initial state
    for nt, budget, S in ((1000, 20.0, 1.0), (300, 7.5, 0.5), (100, 1000.0, 1.0)):
        assert P.slots_for_sizes(nt, budget, lambda s: S, headroom=1.0) == min(nt, int(budget // S) + 1)


def test_growing_sizes_give_more_slots_than_the_worst_ratio():
    # states that compress better early (sizes growing with the step), as
    # for a wavefield spreading from a source
    nt, S = 1000, 1.0
    f = lambda s: S * min(1.0, 0.05 + s / 600.0)
    b = 20.0
    m = P.slots_for_sizes(nt, b, f)
    assert m > int(b // S) + 1
    assert P.pool_peak(nt, m, f) * 1.02 <= b
    assert P.pool_peak(nt, m + 1, f) * 1.02 > b or m == nt


def test_state_bytes_maps_words_to_states():
    import numpy as np
    nt, slots = 60, 7
    acts, (p, W, Rn) = __import__("paper_1810_05268_gb300.ckfwi", fromlist=["x"]).revolve_schedule(nt, slots)
    words = np.arange(2 * W) + 10
    sb = P.state_bytes(nt, slots, words)
    taken = [int(a[1]) for a in acts if a[0] == 1]
    assert list(sb) == taken
    assert sb[taken[0]] == 4 * (10 + 11)
    with pytest.raises(ValueError):
        P.state_bytes(nt, slots, words[:-2])


@pytest.mark.parametrize("nt,slots", [(1000, 39), (300, 9), (120, 5)])
def test_sixteen_bit_upcasts_follow_revolve(nt, slots):
    # a restore from a slot up-casts u^s before a reverse step, both fields
    # before a recomputation (the executor's 16-bit restore)
    acts, cnt = R.schedule(nt, slots)
    want = 0
    for i, a in enumerate(acts):
        if a[0] == R.RESTORE and a[2] > 0:
            nxt = acts[i + 1][0] if i + 1 < len(acts) else None
            want += 1 if nxt == R.YOUTURN else 2
    nf, nc, nd = P.counts(nt, slots, "fp16")
    assert nd == want and nc == 0 and nf == cnt["p"] + 1
    ev = P.events(nt, slots, "fp16")
    assert ev["takeshots"] == cnt["W"] and ev["decomp"] == want
