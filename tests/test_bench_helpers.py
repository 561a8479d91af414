"""Host-side logic of bench.py (no GPU): the traffic lookup, the fixed-rate
slot count at a budget, the time model fitted to a set of measured modes
(unit costs from store-all, FP32 and FP16 runs; choices at both budgets),
and the bench line's roofline block."""
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


def _headline(**kw):
    H = {"ratio_mean": 0.0, "store_mode": "fp16", "ckpt_slots": 39, "W": 909, "fwd_launches": 2140,
         "fwd_ms": 2140 * 0.0433, "adj_launches": 1000, "adj_ms": 1000 * 0.0801, "comp_ms": 0.0, "comp_calls": 0,
         "decomp_ms": 30.0, "decomp_calls": 960, "fwd_kernel": [4, 32, 16, 4, 21, 1],
         "adj_kernel": [3, 32, 16, 4, 21]}
    H.update(kw)
    return H


def test_roofline_block_of_a_stencil_dominated_mode():
    npts, nt = 208 ** 3, 1000
    H = _headline()
    r = bench.roofline_block(H, nt, npts, 6686.1, "measured")
    assert r["class"] == "fwd" and r["kernel"] == "fwd4_kernel" and r["unit"] == "GB/s"
    # every forward launch moves 16 B/pt; the W launches that write a 16-bit
    # checkpoint pair move 4 more
    total = (16.0 * H["fwd_launches"] + 4.0 * H["W"]) * npts
    want = total / (H["fwd_ms"] * 1e-3) / 1e9
    assert r["achieved"] == pytest.approx(want)
    assert r["frac"] == pytest.approx(want / 6686.1)
    assert r["frac_of_nominal"] == pytest.approx(want / bench.NOMINAL_HBM_GBS)
    assert r["launches"] == H["fwd_launches"]
    assert r["algorithmic_bytes_per_launch"] * r["launches"] == pytest.approx(total)
    tpp = bench.traffic_per_point("fwd4_kernel", H["fwd_kernel"])
    assert tpp is not None and r["traffic"] == pytest.approx(tpp * npts)
    # the captured traffic is of a launch without a checkpoint write: the
    # basis names that launch's algorithmic bytes (16 B/pt)
    assert r["traffic_basis"] and ("%.0f" % (16.0 * npts)) in r["traffic_basis"]
    assert r["traffic_basis_bytes"] == pytest.approx(16.0 * npts)
    assert set(r["class_gbs"]) == {"fwd", "adj", "comp", "decomp"}
    json.dumps(r)


def test_every_step_kernel_generation_has_a_name_and_the_chosen_ones_a_traffic_entry():
    """The roofline names the kernel of every Tile generation the library
    reports, and the generations the autotuner picks on the bench grid (the
    tensor-copy forward step with one or two planes of prefetch, the lean
    reverse step and the split one) carry committed DRAM traffic for their
    tile."""
    assert set(bench.KERNEL_NAMES) == set(range(1, 9))
    npts = 208 ** 3
    H = _headline()
    H["fwd_kernel"] = [8, 32, 16, 4, 21, 1]
    r = bench.roofline_block(H, 1000, npts, 6686.1, "measured")
    assert r["kernel"] == "fwdq_kernel" and r["traffic"] is not None
    assert 15.0 < r["traffic"] / npts < 18.0
    assert bench.traffic_per_point("adj5_kernel", [7, 32, 16, 4, 21, 1]) is not None
    assert bench.traffic_per_point("fwdq_kernel", [8, 32, 16, 4, 25, 2]) is not None
    assert bench.traffic_per_point("fwdq_kernel+gradq_kernel", [8, 32, 16, 4, 25, 2]) is not None


def test_roofline_block_of_a_codec_dominated_mode():
    npts, nt = 208 ** 3, 1000
    H = _headline(store_mode="codec", ckpt_slots=232, ratio_mean=25.0, comp_ms=500.0, comp_calls=1692)
    r = bench.roofline_block(H, nt, npts, 6686.1, "measured")
    assert r["class"] == "comp" and r["traffic"] is None
    assert r["algorithmic_bytes_per_launch"] == pytest.approx((4.0 + 4.0 / 25.0) * npts)
    # no checkpoint bytes in the forward class of a codec mode
    assert r["class_gbs"]["fwd"] == pytest.approx(16.0 * npts * H["fwd_launches"] / (H["fwd_ms"] * 1e-3) / 1e9)


def test_bench_line_is_short_and_complete():
    """The driver keeps about 1.5 KB of stdout: a full-sized line (every key
    filled, long names) stays below that and keeps its required keys."""
    line = {
        "metric": "gradient point-updates per second (useful 2*N*npts/t)", "value": 102.512345678,
        "unit": "Gpt/s", "n_gpus": 1, "steps": 20, "warmup": 5, "ms_per_step": 175.61234567,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "3d-128cube-so8", "grid": [208, 208, 208], "nt": 1000, "space_order": 8,
                   "mode": "codec Revolve at the memory of 20 fp32 checkpoints, abs tol 0.0001",
                   "ckpt_slots": 232, "l2": "inputs > L2 (fields + checkpoints)", "parallelism": "single"},
        "roofline": {"bound": "hbm", "kernel": "codec compression (enc+compact)", "class": "comp",
                     "achieved": 3591.2, "peak": 6679.2, "unit": "GB/s", "frac": 0.5377, "peak_kind": "measured",
                     "algorithmic_bytes_per_launch": 159312345.123456, "traffic": 146312345.123456},
        "cpu_baseline": {"value": 0.4291965276, "unit": "Gpt/s", "cores": 16, "kind": "oracle",
                         "sample": "one FP64 oracle gradient of the whole workload (1000 steps, 123.4 s)"},
        "e2e": {"value": 99.123456789, "unit": "Gpt/s", "h2d_bytes_per_step": 16400000,
                "d2h_bytes_per_step": 35995656},
        "gpu_launches": 123456,
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]},
        "recompute_ratio": 2.1401, "gradients_per_hour": 20500.3,
        "oracle": {"grad_rel_err": 0.00331234567, "tol": 0.01},
    }
    out = bench.compact_line(dict(line))
    assert len(out) < 1500
    d = json.loads(out)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "roofline", "cpu_baseline",
              "e2e", "gpu_launches", "config"):
        assert k in d
    assert out == json.dumps(line)          # nothing had to be dropped
    # an over-long line drops optional keys, never the required ones
    line["config"]["mode"] = "x" * 1200
    d = json.loads(bench.compact_line(dict(line)))
    assert "value" in d and "roofline" in d and "oracle" not in d
