"""Host-side logic of bench.py (no GPU): the traffic lookup, the fixed-rate
slot count at a budget, and the time model fitted to a set of measured
modes (unit costs from store-all, FP32 and FP16 runs; choices at both
budgets)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

bench = pytest.importorskip("bench")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1810_05268_gb300 import build
    build.build()


def test_traffic_lookup_matches_kernel_shape_and_prefetch():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    e = d["fwd4_kernel"]
    t = list(e["tile"])
    assert bench.traffic_per_point("fwd4_kernel", t) == pytest.approx(e["dram_bytes_per_point"])
    t2 = list(t)
    t2[4] += 3                                         # another z-run length: same kernel
    assert bench.traffic_per_point("fwd4_kernel", t2) == pytest.approx(e["dram_bytes_per_point"])
    t3 = list(t)
    t3[3] = 2                                          # another vector width: another kernel
    assert bench.traffic_per_point("fwd4_kernel", t3) is None
    t4 = list(t) + [0] * (6 - len(t))
    t4[5] = 2 if t4[5] != 2 else 1                     # another prefetch depth
    assert bench.traffic_per_point("fwd4_kernel", t4) is None
    assert bench.traffic_per_point("no_such_kernel", t) is None


def test_rate_mode_slots_fill_the_budget_exactly():
    from paper_1810_05268_gb300 import ckfwi as C
    shape = (208, 208, 208)
    S = 2 * 208 ** 3 * 4
    for slots in (5, 20):
        kw = bench.rate_mode(C, 1000, shape, S, slots)
        per = 2 * 4 * C.codec_rate_words(3, *shape, bench.RATE)
        assert (kw["ckpt_slots"] - 1) * per <= kw["pool_bytes"] < kw["ckpt_slots"] * per
        assert kw["store_mode"] == "rate" and kw["rate"] == bench.RATE


def _mode(store, slots, nt, fwd_ms, fwd_n, adj_ms, comp=(0.0, 0), decomp=(0.0, 0), err=0.0, W=0, ms=None):
    return {"ms": ms or (fwd_ms + adj_ms + comp[0] + decomp[0]), "ckpt_slots": slots, "store_mode": store,
            "fwd_ms": fwd_ms, "fwd_launches": fwd_n, "adj_ms": adj_ms, "adj_launches": nt,
            "comp_ms": comp[0], "comp_calls": comp[1], "decomp_ms": decomp[0], "decomp_calls": decomp[1],
            "grad_rel_err_vs_storeall": err, "W": W, "host_slots": 0}


def test_time_model_fit_recovers_its_own_costs():
    from paper_1810_05268_gb300 import perfmodel as P
    nt, cf, cr, tck32, tck16, td16 = 400, 0.04, 0.08, 0.01, 0.012, 0.015
    res = {"storeall": _mode("fp32", nt, nt, cf * nt, nt, cr * nt)}
    for key, mode, slots in (("fp32", "fp32", 10), ("fp16", "fp16", 19)):
        ev = P.events(nt, slots, mode)
        tck = tck32 if mode == "fp32" else tck16
        fwd = ev["fwd"] * cf + ev["takeshots"] * tck
        dec = ev["decomp"] * td16 if mode == "fp16" else 0.0
        res[key] = _mode(mode, slots, nt, fwd, ev["fwd"], cr * nt, decomp=(dec, max(1, ev["decomp"] // 2)),
                         W=ev["takeshots"])
    out = bench.perf_model(res, nt, None)
    u = out["unit_ms"]
    assert u["C_F"] == pytest.approx(cf) and u["C_R"] == pytest.approx(cr)
    assert u["t_ck32"] == pytest.approx(tck32) and u["t_ck16"] == pytest.approx(tck16)
    assert u["t_d16"] == pytest.approx(td16)
    for k, m in out["modes"].items():
        assert m["predicted_ms"] == pytest.approx(m["measured_ms"], rel=1e-9), k
