"""Benchmark of the checkpointed, compressed adjoint-state gradient.

One step = one full gradient (forward sweep, residual and FP64 misfit,
Revolve reverse sweep with recomputation, compression / decompression of
checkpoints, imaging condition) of one shot on the 3D workload: 128^3
interior + 40-cell damping layer (208^3 points) at 15 m, space order 8,
1000 steps of 1 ms, Gaussian-random-field velocity 1.5-4.5 km/s, 8 Hz
Ricker source, 64 x 64 receivers.

Headline (`value`): useful point-updates per second, 2 * N * npts / t, of
the gradient at the memory of 20 uncompressed checkpoints, with the fastest
storage choice whose gradient stays within 1e-2 (relative L2) of the FP64
oracle's: Revolve with 20 FP32 checkpoints, 39 FP16 / BF16 ones, or
checkpoints compressed in the same bytes by the fixed-tolerance codec (abs.
tol 1e-4, slots from the worst ratio) or by its fixed-rate mode (16 bits per
value) (Sec. 4); the one taken is named in `config.mode`.

stdout ends with ONE compact JSON line (the headline, its roofline, the
oracle baseline, the end-to-end rate, clocks).  Everything else -- every
storage mode at the memory of 20 and of 5 checkpoints, store-all, host
slots, the time model's predictions, the OT4 kernel's modes, a batch of 16
2D shots, and the tolerance -> gradient-error table against the FP64
oracle (the analogue of the paper's Table 2) -- goes to a side file whose
path is printed on stderr (`--detail` sets it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--detail PATH] [--modes M,...] [--sweep c3|c4|c5]

Under torchrun (N > 1) every rank computes the gradient of its own shot
(shots are independent, Sec. 1.2): weak scaling, no data-path collective.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "3d-128cube-so8"
BUDGET_SLOTS = 20          # memory of 20 uncompressed checkpoints
LOW_SLOTS = 5              # the low-memory comparison
HOST_SLOTS = 40            # second-level (host memory) slots of the two-level comparison
TOL = 1e-4                 # codec absolute tolerance
RATE = 16                  # fixed-rate codec: bits per value
FWD_BYTES = 16             # forward step: read u^n, u^{n-1}, w; write u^{n+1} (+4 with a fused checkpoint)
ADJ_BYTES = 28             # reverse step: read lam^j, lam^{j+1}, u^{j-1}, w, g; write lam^{j-1}, g
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal (the measured copy is the roofline's peak)
CPU_STEPS = 300            # time steps of the oracle sample (about 10-30 s on 16 cores)
GRAD_TOL = 1e-2            # gradient accuracy a storage mode must keep to be the headline
KERNEL_NAMES = {1: ("fwd_kernel", "adj_kernel"), 2: ("fwd_tma_kernel", "adj_tma_kernel"),
                3: ("fwd3_kernel", "adj3_kernel"), 4: ("fwd4_kernel", "adj4_kernel"),
                5: ("ot4_lap_kernel+ot4_fwd_kernel", "ot4_lap_kernel+ot4_adj_kernel"),
                6: ("ot4v_lap_kernel+ot4v_fwd_kernel", "ot4v_lap_kernel+ot4v_fwd_kernel+ot4v_grad_kernel"),
                7: ("fwd5_kernel", "adj5_kernel"), 8: ("fwdq_kernel", "fwdq_kernel+gradq_kernel")}
# OT4 forward step (two passes): reads u^n, w and writes Z = w lap u^n, then
# reads Z, u^n, u^{n-1}, w and writes u^{n+1}.  Reverse step (three passes):
# reads lam^j, u^{j-1}, w, the previous Z_u and g, writes Z_l, Z_u, g; reads
# Z_l, lam^j, lam^{j+1}, w, writes lam^{j-1}; reads u^{j-1}, Z_u, lam^{j-1}, g,
# writes g
OT4_FWD_BYTES = 32
OT4_ADJ_BYTES = 72


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "fallback"


def traffic_per_point(kernel, tile):
    """DRAM bytes per grid point per launch of `kernel` with `tile` from the
    committed ncu summary (taken on the same workload and tile shape), or
    None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        entries = d[kernel] if isinstance(d[kernel], list) else [d[kernel]]
        # the same kernel, tile shape (version, x, y, points per thread) and
        # prefetch depth; the z-run length moves the halo re-reads by a few
        # percent only
        t = list(tile) + [0] * (6 - len(tile))
        for e in entries:
            want = list(e["tile"]) + [0] * (6 - len(e["tile"]))
            if want[:4] == t[:4] and want[5] == t[5]:
                return float(e["dram_bytes_per_point"])
        return None
    except (OSError, ValueError, KeyError, TypeError, IndexError):
        return None


def roofline_block(H, nt, npts, peak, peak_kind, delta=0.0):
    """The bench line's `roofline`: the kernel class with the largest device
    time in the headline mode H (one mode's profiled stats), its algorithmic
    bytes per launch over its average launch time, against `peak`.  A
    profiled gradient brackets every kernel-class call with two events; the
    per-call overhead `delta` [ms] that adds (measured on the store-all
    gradient against its graph replay) is taken off each call's time."""
    F = max(1.0, H["ratio_mean"] or 1.0)
    # a step that writes an FP32 or 16-bit checkpoint writes 4 more B/pt
    # (u^{n-1} in FP32, or both levels in 16 bits), W of the launches
    ck_bytes = 4.0 if H["store_mode"] in ("fp32", "fp16", "bf16") and H["ckpt_slots"] < nt else 0.0
    fwd_b = (FWD_BYTES + ck_bytes * H["W"] / max(1, H["fwd_launches"])) * npts
    classes = {
        "fwd": (H["fwd_ms"], H["fwd_launches"], fwd_b),
        "adj": (H["adj_ms"], H["adj_launches"], ADJ_BYTES * npts),
        "comp": (H["comp_ms"], H["comp_calls"], (4.0 + 4.0 / F) * npts),
        "decomp": (H["decomp_ms"], H["decomp_calls"], (4.0 / F + 4.0) * npts),
    }
    per = {k: (max(1e-9, ms / n - delta) if ms > 0 and n > 0 else 0.0) for k, (ms, n, b) in classes.items()}
    gbs = {k: (b / (per[k] / 1e3) / 1e9 if per[k] > 0 else 0.0) for k, (ms, n, b) in classes.items()}
    dom = max(classes, key=lambda k: classes[k][0])
    _, n_d, b_d = classes[dom]
    if dom in ("fwd", "adj"):
        ver = H[dom + "_kernel"][0]
        kname = KERNEL_NAMES.get(ver, ("?", "?"))[0 if dom == "fwd" else 1]
        tpp = traffic_per_point(kname, H[dom + "_kernel"])
    else:
        kname = "codec compression (enc+compact)" if dom == "comp" else "dec_kernel"
        tpp = None
    return {"bound": "hbm", "kernel": kname, "class": dom, "achieved": gbs[dom], "peak": peak,
            "unit": "GB/s", "frac": gbs[dom] / peak, "peak_kind": peak_kind,
            "frac_of_nominal": gbs[dom] / NOMINAL_HBM_GBS,
            "algorithmic_bytes_per_launch": b_d, "launches": n_d, "launch_us": 1e3 * per[dom],
            "event_overhead_us_per_call": 1e3 * delta,
            "traffic": (tpp * npts) if tpp is not None else None,
            # the ncu figure is of a launch without a fused checkpoint write:
            # compare it with that launch's algorithmic bytes
            "traffic_basis": ("one launch without a checkpoint write (ncu), against %.0f algorithmic bytes"
                              % ((FWD_BYTES if dom == "fwd" else ADJ_BYTES) * npts)) if tpp is not None else None,
            "traffic_basis_bytes": (FWD_BYTES if dom == "fwd" else ADJ_BYTES) * npts if tpp is not None else None,
            "class_gbs": gbs}


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def perf_model(results, nt, fmin):
    """The paper's time model (Sec. 3-4; paper_1810_05268_gb300.perfmodel)
    with the unit costs measured in this run: its prediction for every timed
    mode against the measured time, the mode it chooses at each budget, and
    its prediction across memory budgets (the regimes of Sec. 4)."""
    from paper_1810_05268_gb300 import perfmodel as P

    def unit(cls, n, modes=None):
        v = [r[cls + "_ms"] / r[n] for k, r in results.items()
             if r[n] > 0 and r[cls + "_ms"] > 0 and (modes is None or r["store_mode"] in modes)]
        return float(np.min(v)) if v else None

    def named(k):
        return results.get(k)
    # plain step costs from store-all (no fused checkpoint writes); the extra
    # cost of a step that writes a checkpoint, and of a reverse step reading a
    # 16-bit one, from the FP32 / FP16 runs and their event counts
    sa = named("storeall")
    # the profiled gradients time every kernel-class call between two events;
    # the store-all gradient gives that overhead per call: its profiled class
    # times minus its un-profiled (graph replay) time, over its calls
    delta = 0.0
    if sa:
        calls = sa["fwd_launches"] + sa["adj_launches"]
        prof = sa["fwd_ms"] + sa["adj_ms"] + sa.get("other_ms", 0.0)
        delta = max(0.0, (prof - sa["ms"]) / calls) if calls else 0.0
    raw_unit = unit

    def unit(cls, n, modes=None):
        u = raw_unit(cls, n, modes)
        return None if u is None else max(0.0, u - delta)
    c_f = sa["fwd_ms"] / sa["fwd_launches"] - delta if sa else unit("fwd", "fwd_launches")
    c_r = sa["adj_ms"] / sa["adj_launches"] - delta if sa else (unit("adj", "adj_launches", ("fp32", "codec", "rate"))
                                                                or unit("adj", "adj_launches"))
    t_ck = {}
    c_r16 = t_d16 = None
    for key, mode in (("fp32", "fp32"), ("fp16", "fp16")):
        r = named(key)
        if r and r["fwd_launches"] > 0 and c_f is not None:
            ev = P.events(nt, r["ckpt_slots"], mode)
            if ev["takeshots"]:
                t_ck[mode] = max(0.0, (r["fwd_ms"] - ev["fwd"] * (c_f + delta)) / ev["takeshots"])
            if mode == "fp16":
                c_r16 = r["adj_ms"] / r["adj_launches"] - delta
                if ev["decomp"]:
                    t_d16 = max(0.0, r["decomp_ms"] / ev["decomp"] - delta)
    costs = P.Costs(c_f=c_f, c_r=c_r, c_r16=c_r16, t_c=unit("comp", "comp_calls", ("codec",)),
                    t_d=unit("decomp", "decomp_calls", ("codec",)), f_min=fmin,
                    t_c_rate=unit("comp", "comp_calls", ("rate",)), t_d_rate=unit("decomp", "decomp_calls", ("rate",)),
                    t_d16=t_d16,
                    t_ck32=t_ck.get("fp32", 0.0), t_ck16=t_ck.get("fp16", 0.0), rate=RATE,
                    grad_err={r["store_mode"]: r.get("grad_rel_err_vs_storeall", 0.0) for r in results.values()})
    out = {"event_overhead_ms_per_call": delta, "unit_ms": {"C_F": costs.c_f, "C_R": costs.c_r, "C_R16": costs.c_r16, "t_c": costs.t_c,
                       "t_d": costs.t_d, "t_c_rate": costs.t_c_rate, "t_d_rate": costs.t_d_rate,
                       "t_d16": costs.t_d16, "t_ck32": costs.t_ck32, "t_ck16": costs.t_ck16, "F_min": fmin},
           "modes": {}}
    for name, r in results.items():
        if r.get("host_slots"):
            continue          # slots in host memory have their own (link) costs; not modelled
        nf, nc, nd = P.counts(nt, r["ckpt_slots"], r["store_mode"])
        out["modes"][name] = {"predicted_ms": P.predict(costs, nt, r["ckpt_slots"], r["store_mode"]),
                              "measured_ms": r["ms"], "forward_steps": nf, "compressions": nc,
                              "decompressions": nd}
    for budget, slots, names in (("budget", BUDGET_SLOTS, ("codec", "fp32", "fp16", "bf16", "rate")),
                                 ("low", LOW_SLOTS, ("codec_low", "fp32_low", "fp16_low", "rate_low"))):
        # (the scheduled codec modes are the codec with per-state sizes: the
        # model's uniform-ratio choice is made among the others)
        c = [n for n in names if n in out["modes"]]
        if c:
            pick = P.choose(costs, nt, slots, modes=tuple(results[n]["store_mode"] for n in c), grad_tol=GRAD_TOL)
            meas = min((n for n in c if results[n].get("grad_rel_err_vs_storeall", 0.0) <= GRAD_TOL),
                       key=lambda n: out["modes"][n]["measured_ms"], default=None)
            out["choice_" + budget] = {"predicted": pick[0] if pick else None,
                                       "measured": results[meas]["store_mode"] if meas else None}
    if fmin and costs.t_c is not None:
        out["budget_sweep"] = P.sweep(costs, nt, [2, 3, 5, 8, 12, 20, 32, 50, 80, 128, 250, 500, nt],
                                      modes=("fp32", "fp16", "codec") + (("rate",) if costs.t_c_rate else ()))
    return out


def time_modes(C, torch, model, shot, d_obs, modes, nt, npts, args, ws, lr, full=None):
    """Time one gradient of every storage mode in `modes` (dict name ->
    adjoint_gradient keywords): W warm-ups, K timed graph replays (CUDA
    events, max over ranks, clocks sampled), then profiled gradients for the
    per-class device times.  Modes not in `full` (None: all) are timed over
    min(K, 5) replays.  Returns (results, last gradients, clocks, skipped
    modes)."""
    grads = {}

    def one(kw, profile, keep=None):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        phi, g, st = model.adjoint_gradient(shot, d_obs, profile=profile, use_graph=not profile, **kw)
        torch.cuda.synchronize()
        if keep is not None:
            grads[keep] = g
        return time.perf_counter() - t0, phi, st

    results = {}
    clocks = {}
    skipped = {}
    for name, kw in list(modes.items()):
        # retry with fewer codec slots if the pool overflowed at run time; a
        # 16-bit mode whose states overflow FP16 is reported and skipped
        ok = False
        for _ in range(4):
            try:
                for _ in range(args.warmup):
                    one(kw, False, keep=name)
                ok = True
                break
            except C.CkfwiError as e:
                if e.status == C.NONFINITE and kw.get("store_mode") in ("fp16", "bf16"):
                    skipped[name] = "checkpoint values overflow %s" % kw["store_mode"]
                    break
                if e.status != C.POOL_OVERFLOW or kw.get("store_mode") != "codec":
                    raise
                kw["ckpt_slots"] = max(2, int(kw["ckpt_slots"] * 0.8))
        if not ok:
            modes.pop(name)
            continue
        # profiled warm-up creates the library's timing events, so that the
        # profiled steps below do not include host-side event creation
        one(kw, True)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk = Clocks(lr)
        # timed region: K gradients replayed from the recorded graph, CUDA
        # events on torch's stream (the library launches on that stream), max
        # over ranks
        k_steps = args.steps if full is None or name in full else max(1, min(args.steps, 5))
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k_steps + 1)]
        evs[0].record()
        for i in range(k_steps):
            _, phi, st_plain = one(kw, False)
            evs[i + 1].record()
        torch.cuda.synchronize()
        clocks[name] = clk.stop()
        ms = max_over_ranks(evs[0].elapsed_time(evs[-1]) / k_steps, "cuda")
        # each replay's own time (this rank): the spread behind the mean
        replay = [evs[i].elapsed_time(evs[i + 1]) for i in range(k_steps)]
        # per-kernel-class device time from profiled gradients (same work)
        sts = []
        for _ in range(max(1, min(args.steps, 3))):
            _, _, st = one(kw, True)
            sts.append(st)
        st = sts[-1]
        avg = lambda k: float(np.mean([s[k] for s in sts]))
        results[name] = {
            "ms": ms, "gpts": 2.0 * nt * npts / (ms / 1e3) / 1e9 * ws, "timed_steps": k_steps,
            # executed rate: every forward (recomputations included) and reverse step
            "executed_gpts": (st["fwd_steps"] + nt) * npts / (ms / 1e3) / 1e9 * ws,
            "replay_ms": [round(r, 2) for r in replay], "replay_ms_median": float(np.median(replay)),
            "u_absmax": st["u_absmax"],
            "ckpt_slots": kw["ckpt_slots"], "store_mode": kw["store_mode"],
            "pool_bytes": kw.get("pool_bytes", st["pool_bytes_peak"]), "host_slots": kw.get("host_slots", 0),
            "recompute_ratio": st["fwd_steps"] / nt, "p": st["p"], "W": st["takeshots"], "R": st["restores"],
            "fwd_launches": st["fwd_launches"], "adj_launches": st["adj_launches"],
            "comp_calls": st["comp_calls"], "decomp_calls": st["decomp_calls"],
            "fwd_ms": avg("fwd_ms"), "adj_ms": avg("adj_ms"), "comp_ms": avg("comp_ms"),
            "decomp_ms": avg("decomp_ms"), "other_ms": avg("other_ms"),
            "kernel_launches": st_plain["kernel_launches"], "misfit": phi,
            "ratio_mean": st["ratio_mean"], "ratio_min": st["ratio_min"],
            "pool_bytes_peak": st["pool_bytes_peak"],
            "fwd_kernel": [st["fwd_ver"], st["fwd_bx"], st["fwd_by"], st["fwd_vec"], st["fwd_zlen"], st["fwd_pf"]],
            "adj_kernel": [st["adj_ver"], st["adj_bx"], st["adj_by"], st["adj_vec"], st["adj_zlen"], st["adj_pf"]],
        }
    return results, grads, clocks, skipped


def grad_errors(torch, results, grads):
    """Gradient error of every mode against store-all (bitwise the exact
    FP32 gradient: the schedule never changes values)."""
    if "storeall" in grads:
        ref = grads["storeall"].double()
        nref = float(torch.linalg.vector_norm(ref))
        for k, g in grads.items():
            results[k]["grad_rel_err_vs_storeall"] = float(torch.linalg.vector_norm(g.double() - ref)) / nref


def size_profile(C, model, shot, d_obs, nt, state_bytes):
    """A pilot gradient that compresses every state once (nt slots): the
    worst ratio F_min and each state's compressed bytes (Sec. 8:
    non-uniform ratios)."""
    from paper_1810_05268_gb300 import perfmodel as P
    pool = nt * state_bytes // 4
    for _ in range(4):
        try:
            st = model.adjoint_gradient(shot, d_obs, nt, store_mode="codec", tol=TOL, pool_bytes=pool)[2]
            break
        except C.CkfwiError as e:
            if e.status != C.POOL_OVERFLOW:
                raise
            pool *= 2
    return max(1.0, st["ratio_min"]), P.state_bytes(nt, nt, model.stream_words())


def codec_modes(C, nt, state_bytes, fmin, sizes, slots, sched):
    """Codec checkpoints in the memory of `slots` FP32 checkpoints: slots
    from the worst ratio with 10% headroom, or (sched) the most slots whose
    pool peak with every state's measured size fits."""
    from paper_1810_05268_gb300 import perfmodel as P
    b = slots * state_bytes
    if sched:
        m = P.slots_for_sizes(nt, b, P.size_function(sizes))
    else:
        m = b / (state_bytes / fmin * 1.1)
    return dict(ckpt_slots=int(min(nt, max(2, m))), store_mode="codec", tol=TOL, pool_bytes=b)


def rate_mode(C, nt, shape, state_bytes, slots):
    """Fixed-rate checkpoints (RATE bits per value) in the memory of `slots`
    FP32 checkpoints: their size is known, so the slots are exact."""
    b = slots * state_bytes
    per = 2 * 4 * C.codec_rate_words(3, *shape, RATE)
    return dict(ckpt_slots=int(min(nt, 1 + b // per)), store_mode="rate", rate=RATE, pool_bytes=b)


def ot4_block(C, torch, w, grid, shot, nt, npts, state_bytes, args, ws, lr, res2):
    """The same gradient with the OT4 kernel: store-all, and Revolve at the
    memory of BUDGET_SLOTS and LOW_SLOTS FP32 checkpoints with FP32, FP16 and
    codec storage; the time model's prediction against the measurement, the
    OT4 / OT2 step-cost ratio and the budget sweep (where compression pays)."""
    import dataclasses
    from paper_1810_05268_gb300 import perfmodel as P
    g4 = dataclasses.replace(grid, time_order=4)
    m4 = C.Model(g4)
    m4.set_model(torch.from_numpy(w.true.astype(np.float32)).cuda())
    d_obs = m4.forward_shot(shot).clone()
    m4.set_model(torch.from_numpy(w.start.astype(np.float32)).cuda())
    fmin, sizes = size_profile(C, m4, shot, d_obs, nt, state_bytes)
    codec = lambda slots, sched=False: codec_modes(C, nt, state_bytes, fmin, sizes, slots, sched)
    modes = {"storeall": dict(ckpt_slots=nt, store_mode="fp32"),
             "fp32": dict(ckpt_slots=BUDGET_SLOTS, store_mode="fp32"),
             "fp16": dict(ckpt_slots=2 * (BUDGET_SLOTS - 1) + 1, store_mode="fp16"),
             "codec": codec(BUDGET_SLOTS),
             "codec_sched": codec(BUDGET_SLOTS, True),
             "fp32_low": dict(ckpt_slots=LOW_SLOTS, store_mode="fp32"),
             "codec_low": codec(LOW_SLOTS),
             "codec_sched_low": codec(LOW_SLOTS, True)}
    results, grads, clocks, skipped = time_modes(C, torch, m4, shot, d_obs, modes, nt, npts, args, ws, lr,
                                                 full=())
    m4.close()
    grad_errors(torch, results, grads)
    mdl = perf_model(results, nt, fmin)
    u2 = perf_model(res2, nt, None)["unit_ms"]
    u4 = mdl["unit_ms"]
    gbs = {}
    for name, r in results.items():
        gbs[name] = {k: (b * npts * r[k + "_launches"] / (r[k + "_ms"] / 1e3) / 1e9 if r[k + "_ms"] > 0 else 0.0)
                     for k, b in (("fwd", OT4_FWD_BYTES), ("adj", OT4_ADJ_BYTES))}
    return {
        "time_order": 4, "workload": WORKLOAD, "nt": nt, "codec_tol": TOL, "F_min": fmin,
        "compare": {k: dict(v, clocks=clocks.get(k), hbm_gbs=gbs.get(k)) for k, v in results.items()},
        "skipped": skipped,
        "step_cost_ratio_ot4_vs_ot2": {"C_F": u4["C_F"] / u2["C_F"] if u2["C_F"] else None,
                                       "C_R": u4["C_R"] / u2["C_R"] if u2["C_R"] else None},
        "algorithmic_bytes_per_point": {"fwd": OT4_FWD_BYTES, "adj": OT4_ADJ_BYTES},
        "model": mdl,
    }


def batch_compare(C, torch, synth, nshots=16, slots=16):
    """Shots of the 2D 1104 x 464 x 2000 workload (order 8): one batched call
    (every stencil step one launch over all shots, recorded as a graph)
    against the same gradients one shot at a time."""
    w = synth.workload("2d-1024x384-so8")
    grid = C.GridSpec(2, w.shape, w.nbl, w.h, w.so, w.dt, w.nt, w.vmax)
    m = C.Model(grid)
    m.set_model(torch.from_numpy(w.start.astype(np.float32)).cuda())
    ext = (w.shape[1] - 2 * w.nbl - 1) * w.h
    shots = [C.ShotSpec(src=(20.0, 0.0, float(x)), rec=w.rec, f0=w.f0)
             for x in np.linspace(0.1 * ext, 0.9 * ext, nshots)]
    dobs = [m.forward_shot(s) * 1.01 for s in shots]
    m.batch_gradient(shots, dobs, slots, use_graph=True)
    m.adjoint_gradient(shots[0], dobs[0], slots)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, gb, st = m.batch_gradient(shots, dobs, slots, use_graph=True)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    for s, d in zip(shots, dobs):
        m.adjoint_gradient(s, d, slots)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t0
    npts = int(np.prod(w.shape))
    m.close()
    return {"workload": "2d-1024x384-so8", "grid": list(w.shape), "nt": w.nt, "shots": nshots, "slots": slots,
            "batched_ms": 1e3 * tb, "one_shot_at_a_time_ms": 1e3 * ts, "speedup": ts / tb,
            "batched_gpts": 2.0 * w.nt * npts * nshots / tb / 1e9,
            "stencil_launches_per_step": 1, "fwd_launches": st["fwd_launches"]}


def rank_source(src, rk, ws):
    """Source position of rank rk's shot: shots are independent (Sec. 1.2), so
    ranks take distinct sources along x and share nothing on the data path."""
    return (src[0], src[1], src[2] * (0.5 + 0.5 * (rk + 1) / max(ws, 1)))


def max_over_ranks(ms, device):
    """The step time of the slowest rank (the job's time); no-op on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rk = int(os.environ.get("RANK", "0"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rk, lr


def cpu_sample(w, nt_sample):
    """Oracle gradient over the first nt_sample steps of the workload (FP64, host cores)."""
    from oracle import propagator as O
    og = O.Grid(w.dims, tuple(w.shape), w.nbl, w.h, w.so, w.dt, nt_sample, w.vmax)
    s = O.ricker(nt_sample, w.dt, w.f0)
    vel = w.start.astype(np.float32).astype(np.float64)
    dobs = np.zeros((nt_sample + 1, w.rec.shape[0]))
    t = time.perf_counter()
    O.gradient(og, vel, [w.src], s, w.rec, dobs)
    dt = time.perf_counter() - t
    npts = int(np.prod(w.shape))
    return 2.0 * nt_sample * npts / dt / 1e9, dt


def oracle_reference(w):
    """The FP64 oracle's data of the true model and its gradient at the start
    model over the whole workload (host cores): the reference every GPU
    gradient's error is stated against.  Returns (d_obs as float32, oracle
    gradient, oracle misfit, seconds of the gradient)."""
    from oracle import propagator as O
    og = O.Grid(w.dims, tuple(w.shape), w.nbl, w.h, w.so, w.dt, w.nt, w.vmax)
    ser = O.ricker(w.nt, w.dt, w.f0)
    d_true = O.forward(og, w.true.astype(np.float32).astype(np.float64), [w.src], ser, w.rec)
    dobs = d_true.astype(np.float32)
    t = time.perf_counter()
    phi, g, _ = O.gradient(og, w.start.astype(np.float32).astype(np.float64), [w.src], ser, w.rec,
                           dobs.astype(np.float64))
    return dobs, g, phi, time.perf_counter() - t


def err_vs(g, g_ref):
    """(absolute, relative) L2 distance of a GPU gradient (torch) from the oracle's (numpy FP64)."""
    d = float(np.linalg.norm(g.detach().cpu().numpy().astype(np.float64) - g_ref))
    return d, d / float(np.linalg.norm(g_ref))


def timed_ms(model, shot, d_obs, kw, reps=2):
    """Mean wall time of `reps` graph replays of one gradient (after one warm-up), device-synchronised."""
    import torch
    model.adjoint_gradient(shot, d_obs, use_graph=True, **kw)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        phi, g, st = model.adjoint_gradient(shot, d_obs, use_graph=True, **kw)
    torch.cuda.synchronize()
    return (time.perf_counter() - t) * 1e3 / reps, g, st


def error_table(C, torch, model, shot, dobs_o, g_ref, nt, npts, state_bytes, shape):
    """The tolerance -> gradient-error table at the memory of BUDGET_SLOTS
    FP32 checkpoints (the analogue of the paper's Table 2, Sec. 7): every
    storage format's gradient against the FP64 oracle's, with the ratio,
    the slots the memory buys, the recompute ratio and the gradient time.
    Codec slots come from the worst ratio of a pilot with that tolerance."""
    dd = torch.from_numpy(dobs_o).cuda()
    rows = []
    base = [("fp32", dict(ckpt_slots=BUDGET_SLOTS, store_mode="fp32"), None),
            ("bf16", dict(ckpt_slots=2 * (BUDGET_SLOTS - 1) + 1, store_mode="bf16"), None),
            ("fp16", dict(ckpt_slots=2 * (BUDGET_SLOTS - 1) + 1, store_mode="fp16"), None),
            ("rate16", rate_mode(C, nt, shape, state_bytes, BUDGET_SLOTS), None)]
    for tol in (1e-2, 1e-3, 1e-4, 1e-5, 1e-6):
        base.append(("codec %g" % tol, None, tol))
    umax = None
    for name, kw, tol in base:
        try:
            if tol is not None:
                pool = nt * state_bytes // 4
                fmin = None
                for _ in range(5):
                    try:
                        st = model.adjoint_gradient(shot, dd, nt, store_mode="codec", tol=tol, pool_bytes=pool)[2]
                        fmin = max(1.0, st["ratio_min"])
                        break
                    except C.CkfwiError as e:
                        if e.status != C.POOL_OVERFLOW:
                            raise
                        pool *= 2
                b = BUDGET_SLOTS * state_bytes
                kw = dict(ckpt_slots=int(min(nt, max(2, b / (state_bytes / fmin * 1.1)))), store_mode="codec",
                          tol=tol, pool_bytes=b)
            for _ in range(4):
                try:
                    ms, g, st = timed_ms(model, shot, dd, kw)
                    break
                except C.CkfwiError as e:
                    if e.status != C.POOL_OVERFLOW or kw["store_mode"] != "codec":
                        raise
                    kw["ckpt_slots"] = max(2, int(kw["ckpt_slots"] * 0.8))
        except C.CkfwiError as e:
            rows.append({"storage": name, "error": str(e)})
            continue
        umax = st["u_absmax"] or umax
        ea, er = err_vs(g, g_ref)
        row = {"storage": name, "slots": kw["ckpt_slots"], "abs_err": ea, "rel_err": er,
               "recompute_ratio": st["fwd_steps"] / nt, "ms": ms,
               "gpts": 2.0 * nt * npts / (ms / 1e3) / 1e9}
        if kw["store_mode"] in ("codec", "rate"):
            row["F_mean"] = st["ratio_mean"]
            row["F_min"] = st["ratio_min"]
        if tol is not None:
            row["tol"] = tol
            row["tol_over_max_u"] = tol / st["u_absmax"] if st["u_absmax"] else None
        rows.append(row)
    # the paper's observation (Sec. 7): the error falls with the tolerance
    # until it meets the uncompressed gradient's own error
    codec = [r for r in rows if "tol" in r and "rel_err" in r]
    fp32 = next((r["rel_err"] for r in rows if r["storage"] == "fp32" and "rel_err" in r), None)
    mono = all(codec[i + 1]["rel_err"] <= codec[i]["rel_err"] * 1.05 for i in range(len(codec) - 1))
    return {"budget_fp32_slots": BUDGET_SLOTS, "max_abs_u_N": umax, "rows": rows,
            "codec_error_falls_with_tol": mono, "fp32_rel_err": fp32,
            "plateau": (codec[-1]["rel_err"] / fp32) if codec and fp32 else None}


def _timed(torch, fn):
    """(seconds, result) of fn() bracketed by device synchronisations and CUDA events."""
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, out


def _rel(torch, g, ref):
    d = float(torch.linalg.vector_norm(g.double() - ref))
    return d, d / float(torch.linalg.vector_norm(ref))


def sweep_c3(C, torch, synth, args):
    """The 300 x 600 x 600 workload (order 16, 3000 steps of 1.5 ms, 25 m,
    layered model with faults): store-all would need 1.3 TB, so the gradient
    runs at checkpoint budgets of M uncompressed states (M S bytes, S = 864
    MB) with FP32, BF16, FP16 and codec storage in the same bytes.  Each
    configuration runs once (un-profiled, CUDA events); the error is stated
    against the FP32 Revolve gradient, which every FP32 schedule gives bit
    for bit.  The FP64 oracle's rate on this grid is extrapolated from its
    first ORACLE_STEPS steps."""
    w = synth.workload("3d-300x600x600-so16", nt=args.nt)
    nt = w.nt
    npts = int(np.prod(w.shape))
    S = 2 * npts * 4
    grid = C.GridSpec(3, w.shape, w.nbl, w.h, w.so, w.dt, nt, w.vmax)
    model = C.Model(grid)
    shot = C.ShotSpec(src=w.src, rec=w.rec, f0=w.f0)
    model.set_model(torch.from_numpy(w.true.astype(np.float32)).cuda())
    d_obs = model.forward_shot(shot).clone()
    model.set_model(torch.from_numpy(w.start.astype(np.float32)).cuda())
    budgets = [int(b) for b in args.budgets.split(",")]
    tols = (1e-3, 1e-4, 1e-5)
    out = {"workload": "3d-300x600x600-so16", "grid": list(w.shape), "nt": nt, "space_order": w.so,
           "state_bytes": S, "rows": []}

    def grad(kw, profile=False):
        return model.adjoint_gradient(shot, d_obs, profile=profile, **kw)
    t, (phi, g_ref, st) = _timed(torch, lambda: grad(dict(ckpt_slots=32, store_mode="fp32")))
    g_ref = g_ref.double()
    _, (_, _, stp) = _timed(torch, lambda: grad(dict(ckpt_slots=32, store_mode="fp32"), True))
    out["kernels"] = {"fwd_us": 1e3 * stp["fwd_ms"] / stp["fwd_launches"], "adj_us": 1e3 * stp["adj_ms"] / stp["adj_launches"],
                      "fwd_kernel": [stp["fwd_ver"], stp["fwd_bx"], stp["fwd_by"], stp["fwd_vec"], stp["fwd_zlen"], stp["fwd_pf"]],
                      "adj_kernel": [stp["adj_ver"], stp["adj_bx"], stp["adj_by"], stp["adj_vec"], stp["adj_zlen"], stp["adj_pf"]]}
    out["kernels"]["fwd_gbs"] = FWD_BYTES * npts / (out["kernels"]["fwd_us"] * 1e-6) / 1e9
    out["kernels"]["adj_gbs"] = ADJ_BYTES * npts / (out["kernels"]["adj_us"] * 1e-6) / 1e9
    out["u_absmax"] = st["u_absmax"]
    # worst compression ratio per tolerance, from a pilot at the smallest budget
    fmin = {}
    for tol in tols:
        slots, pool = min(nt, 3 * budgets[0]), budgets[0] * S
        for _ in range(6):
            try:
                stc = grad(dict(ckpt_slots=slots, store_mode="codec", tol=tol, pool_bytes=pool))[2]
                fmin[tol] = max(1.0, stc["ratio_min"])
                break
            except C.CkfwiError as e:
                if e.status != C.POOL_OVERFLOW:
                    raise
                slots = max(2, slots // 2)
    out["F_min"] = {str(k): v for k, v in fmin.items()}
    for M in budgets:
        modes = [("fp32", dict(ckpt_slots=min(nt, M), store_mode="fp32")),
                 ("bf16", dict(ckpt_slots=min(nt, 2 * (M - 1) + 1), store_mode="bf16")),
                 ("fp16", dict(ckpt_slots=min(nt, 2 * (M - 1) + 1), store_mode="fp16"))]
        for tol in tols:
            if tol in fmin:
                modes.append(("codec %g" % tol, dict(ckpt_slots=int(min(nt, max(2, M * fmin[tol] / 1.1))),
                                                     store_mode="codec", tol=tol, pool_bytes=M * S)))
        for name, kw in modes:
            row = {"budget_fp32_states": M, "storage": name}
            try:
                for _ in range(4):
                    try:
                        t, (phi, g, st) = _timed(torch, lambda: grad(kw))
                        break
                    except C.CkfwiError as e:
                        if e.status != C.POOL_OVERFLOW or kw["store_mode"] != "codec":
                            raise
                        kw["ckpt_slots"] = max(2, int(kw["ckpt_slots"] * 0.8))
                ea, er = _rel(torch, g, g_ref)
                row.update(slots=kw["ckpt_slots"], seconds=t, gpts=2.0 * nt * npts / t / 1e9,
                           recompute_ratio=st["fwd_steps"] / nt, p=st["p"], W=st["takeshots"], R=st["restores"],
                           abs_err=ea, rel_err=er)
                if kw["store_mode"] == "codec":
                    row.update(F_mean=st["ratio_mean"], F_min=st["ratio_min"],
                               tol_over_max_u=kw["tol"] / st["u_absmax"] if st["u_absmax"] else None)
            except C.CkfwiError as e:
                row["skipped"] = str(e)
            out["rows"].append(row)
            print("c3", json.dumps(row), file=sys.stderr, flush=True)
    model.close()
    if not args.no_cpu:
        r, secs = cpu_sample(w, ORACLE_STEPS)
        out["oracle"] = {"gpts_extrapolated": r, "steps": ORACLE_STEPS, "seconds": secs, "cores": os.cpu_count(),
                         "gradient_seconds_extrapolated": 2.0 * nt * npts / (r * 1e9),
                         "note": "the oracle's rate over its first %d steps; its 3000-step gradient is not run" %
                                 ORACLE_STEPS}
    return out


ORACLE_STEPS = 50


def sweep_c4(C, torch, synth, args):
    """32 shots with uneven 3D apertures (128^3 to 256 x 320 x 320 windows of
    one survey model, order 8, 15 m, 1500 steps of 1 ms), every stencil step
    of a batch one launch over all its shots, recorded as a CUDA graph, at
    M = 32 checkpoints per shot with BF16, FP16 and codec (1e-4) storage; the
    FP16 batch against the same shots one at a time."""
    nt = args.nt or 1500
    vel, wins = synth.batched_apertures()
    nbl, h, so, dt = 40, 15.0, 8, 1.0
    models, shots, dobs, offs = [], [], [], []
    npts = 0
    for wn in wins:
        g = C.GridSpec(3, wn.shape, nbl, h, so, dt, nt, 4.5)
        m = C.Model(g)
        ext = [(n - 2 * nbl - 1) * h for n in wn.shape]
        rec = synth.receiver_grid(30.0, np.linspace(0, ext[1], 32), np.linspace(0, ext[2], 32))
        sh = C.ShotSpec(src=(30.0, ext[1] / 2, ext[2] / 2), rec=rec, f0=0.008)
        # observed data of a 3% faster medium, the gradient at the window's own
        m.set_model(torch.from_numpy((wn.vel * 1.03).astype(np.float32)).cuda())
        dobs.append(m.forward_shot(sh).clone())
        m.set_model(torch.from_numpy(wn.vel.astype(np.float32)).cuda())
        models.append(m)
        shots.append(sh)
        offs.append(wn.offset)
        npts += int(np.prod(wn.shape))
    out = {"shots": len(wins), "nt": nt, "space_order": so, "slots": 32, "points_all_shots": npts,
           "window_shapes": [list(wn.shape) for wn in wins], "survey": list(vel.shape), "modes": {}}
    M = 32
    for name, kw in (("bf16", dict(store_mode="bf16")), ("fp16", dict(store_mode="fp16")),
                     ("codec 1e-4", dict(store_mode="codec", tol=1e-4, pool_bytes=0))):
        run = lambda prof=False: C.batch_gradient_models(models, shots, dobs, offs, vel.shape, M, use_graph=not prof,
                                                         profile=prof, **kw)
        try:
            run()
            t, (phi, gs, st) = _timed(torch, run)
            _, (_, _, sp) = _timed(torch, lambda: run(True))
        except C.CkfwiError as e:
            out["modes"][name] = {"skipped": str(e)}
            continue
        nsh = len(shots)
        steps = st["fwd_steps"] / nsh            # the stats count every lane's steps
        row = {"seconds": t, "gpts": 2.0 * nt * npts / t / 1e9, "misfit": phi,
               "fwd_launches": sp["fwd_launches"], "adj_launches": sp["adj_launches"],
               "recompute_ratio": steps / nt, "u_absmax": st["u_absmax"]}
        # the batched kernels' aggregate algorithmic bandwidth: every lane's
        # forward steps move 16 B a point, reverse steps 28 B
        if sp["fwd_ms"] > 0:
            row["fwd_gbs"] = FWD_BYTES * npts * steps / (sp["fwd_ms"] / 1e3) / 1e9
        if sp["adj_ms"] > 0:
            row["adj_gbs"] = ADJ_BYTES * npts * nt / (sp["adj_ms"] / 1e3) / 1e9
        row["fwd_kernel"] = [sp["fwd_ver"], sp["fwd_bx"], sp["fwd_by"], sp["fwd_vec"], sp["fwd_zlen"], sp["fwd_pf"]]
        row["adj_kernel"] = [sp["adj_ver"], sp["adj_bx"], sp["adj_by"], sp["adj_vec"], sp["adj_zlen"], sp["adj_pf"]]
        if kw["store_mode"] == "codec":
            row.update(F_mean=st["ratio_mean"], F_min=st["ratio_min"])
        out["modes"][name] = row
        print("c4", name, json.dumps(row), file=sys.stderr, flush=True)
    # the same FP16 gradients one shot at a time
    def singles():
        for m, sh, d in zip(models, shots, dobs):
            m.adjoint_gradient(sh, d, M, store_mode="fp16", use_graph=True)
    singles()
    t1, _ = _timed(torch, singles)
    out["fp16_one_shot_at_a_time_seconds"] = t1
    if "fp16" in out["modes"] and "seconds" in out["modes"]["fp16"]:
        out["fp16_batch_speedup"] = t1 / out["modes"]["fp16"]["seconds"]
    for m in models:
        m.close()
    return out


def sweep_c5(C, torch, synth, args):
    """The FWI loop on the 2D 1104 x 464 workload (order 8, 2000 steps): 64
    shots evenly on the surface, observed data of the layered true model from
    the FP64 oracle, steepest descent from the smoothed start model through
    the torch.autograd wrapper (backward = the batched checkpointed adjoint
    with codec checkpoints, M = 16), for ITERATIONS iterations.  At the
    first and the last iteration the misfit and gradient of four of the shots
    are compared with the oracle's (with FP32 and with codec checkpoints), and
    at the first the gradient's directional derivative with central
    differences of the misfit."""
    from oracle import propagator as O
    from paper_1810_05268_gb300 import autograd as A
    w = synth.workload("2d-1024x384-so8", nt=args.nt)
    nt = w.nt
    og = O.Grid(2, tuple(w.shape), w.nbl, w.h, w.so, w.dt, nt, w.vmax)
    grid = C.GridSpec(2, w.shape, w.nbl, w.h, w.so, w.dt, nt, w.vmax)
    ext = (w.shape[1] - 2 * w.nbl - 1) * w.h
    srcs = [(20.0, 0.0, float(x)) for x in np.linspace(0.0, ext, 64)]
    ser = O.ricker(nt, w.dt, w.f0)
    true = w.true.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    dobs_np = [O.forward(og, true, [s], ser, w.rec).astype(np.float32) for s in srcs]
    oracle_data_s = time.perf_counter() - t0
    shots = [C.ShotSpec(src=s, rec=w.rec, f0=w.f0) for s in srcs]
    dobs = [torch.from_numpy(d).cuda() for d in dobs_np]
    model = C.Model(grid)
    m0 = torch.from_numpy((1.0 / w.start.astype(np.float64) ** 2).astype(np.float32)).cuda()
    # codec tolerance: 1e-3 of the wavefield's scale (max |u^N| of a first gradient)
    model.set_model(m0, kind=C.SLOWNESS2)
    _, _, st0 = model.batch_gradient(shots[:1], dobs[:1], 16)
    tol = 1e-3 * st0["u_absmax"]
    S = 2 * int(np.prod(w.shape)) * 4
    opts = dict(store_mode="codec", tol=tol, pool_bytes=16 * S)
    check_idx = [0, 21, 42, 63]

    def oracle_check(m):
        vel = 1.0 / np.sqrt(m.detach().cpu().numpy().astype(np.float64))
        phi_o, g_o, rr, dd = 0.0, np.zeros(w.shape), 0.0, 0.0
        for i in check_idx:
            p, g, dsim = O.gradient(og, vel, [srcs[i]], ser, w.rec, dobs_np[i].astype(np.float64))
            phi_o += p
            g_o += g
            rr += float(np.sum((dsim[1:] - dobs_np[i][1:]) ** 2))
            dd += float(np.sum(dobs_np[i][1:].astype(np.float64) ** 2))
        # the FP32 data's relative error (about 2e-6) over |r| / |d| bounds the
        # attainable accuracy of any FP32 gradient of these data
        res = {"residual_over_data": float(np.sqrt(rr / dd)),
               "fp32_attainable_rel_err": 2e-6 / float(np.sqrt(rr / dd))}
        model.set_model(m.detach(), kind=C.SLOWNESS2)
        for name, kw in (("fp32", dict(store_mode="fp32")), ("codec", opts)):
            phi, gs, _ = model.batch_gradient([shots[i] for i in check_idx], [dobs[i] for i in check_idx], 16, **kw)
            gg = gs.cpu().numpy()
            res[name] = {"misfit": phi, "misfit_oracle": phi_o, "misfit_rel_diff": abs(phi - phi_o) / phi_o,
                         "grad_rel_err": float(np.linalg.norm(gg - g_o) / np.linalg.norm(g_o))}
        return res

    out = {"workload": "2d-1024x384-so8", "grid": list(w.shape), "nt": nt, "shots": 64, "slots": 16,
           "codec_tol": tol, "iterations": ITERATIONS, "oracle_data_seconds": oracle_data_s,
           "checked_shots": check_idx}
    out["check_first"] = oracle_check(m0)
    # directional derivative at the start: central differences of the misfit
    # against the exact (FP32-checkpoint) adjoint gradient, at three step sizes
    # (small ones drown in the FP32 misfit's rounding, large ones in the
    # second-order term)
    dm = torch.from_numpy(synth.smooth_perturbation(tuple(w.shape), 10.0, 7).astype(np.float32)).cuda()
    x = m0.clone().requires_grad_(True)
    phi = A.misfit(x, model, shots, dobs, 16, store_mode="fp32")
    (g,) = torch.autograd.grad(phi, x)
    ad = float((g.double() * dm.double()).sum())
    out["fd_check"] = {"adjoint": ad, "steps": []}
    for rel in (3e-3, 1e-2, 3e-2):
        eps = rel * float(m0.abs().max())
        pp = float(A.misfit(m0 + eps * dm, model, shots, dobs, 16))
        pm = float(A.misfit(m0 - eps * dm, model, shots, dobs, 16))
        fd = (pp - pm) / (2 * eps)
        out["fd_check"]["steps"].append({"eps_rel": rel, "fd": fd, "rel_diff": abs(fd - ad) / abs(fd)})
    t, (m_fin, hist) = _timed(torch, lambda: A.steepest_descent(m0, model, shots, dobs, ITERATIONS, 16, step=0.02,
                                                               m_min=1.0 / 4.5 ** 2, m_max=1.0 / 1.5 ** 2,
                                                               backtrack=12, stop_on_stall=True, **opts))
    out["misfit_history"] = hist
    out["iterations_done"] = len(hist) - 1
    out["loop_seconds"] = t
    out["check_last"] = oracle_check(m_fin)
    model.close()
    return out


ITERATIONS = 20


def run_reference(args):
    ws, rk, _ = dist_env()
    if rk != 0:
        return 0
    from paper_1810_05268_gb300 import synth
    w = synth.workload(WORKLOAD)
    nt_sample = CPU_STEPS
    for _ in range(args.warmup):
        cpu_sample(w, nt_sample)
    rates, times = [], []
    for _ in range(args.steps):
        r, t = cpu_sample(w, nt_sample)
        rates.append(r)
        times.append(t)
    value = float(np.mean(rates))
    cores = os.cpu_count()
    # the small 2D workload on all cores and on one core, and the 3D one on
    # one core over a shorter sample (subprocesses: the oracle's OpenMP
    # thread count is fixed when its library loads)
    extra = {"cpu_model": cpu_model()}
    c1 = synth.workload("2d-201x201-so4")
    extra["c1_all_cores_gpts"] = cpu_sample(c1, c1.nt)[0]
    extra["c1_one_core_gpts"] = one_core("2d-201x201-so4", c1.nt)
    extra["c2_one_core_gpts"] = one_core(WORKLOAD, ONE_CORE_STEPS)
    line = {
        "impl": "reference", "metric": "gradient point-updates per second (useful 2*N*npts/t)",
        "value": value, "unit": "Gpt/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(w.shape), "nt": w.nt, "space_order": w.so,
                   "sample": "first %d of %d time steps per step" % (nt_sample, w.nt)},
        "cpu_baseline": {"value": value, "unit": "Gpt/s", "cores": cores, "kind": "oracle",
                         "sample": "FP64 oracle gradient, first %d of %d time steps" % (nt_sample, w.nt)},
        "e2e": {"value": value, "unit": "Gpt/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_timings": {"cpu": extra["cpu_model"],
                           "c1_2d_281sq_500_gpts": {"cores_%d" % cores: extra["c1_all_cores_gpts"],
                                                    "cores_1": extra["c1_one_core_gpts"]},
                           "c2_3d_208cube_gpts_1_core": extra["c2_one_core_gpts"],
                           "c2_1_core_sample": "first %d steps" % ONE_CORE_STEPS},
    }
    print(json.dumps(line), flush=True)
    return 0


ONE_CORE_STEPS = 40


def cpu_model():
    """The host CPU's model name (lscpu), or the architecture."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def one_core(name, steps):
    """The oracle gradient's rate on one host core (a subprocess with one OpenMP thread)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", "%s,%d" % (name, steps)],
                       capture_output=True, text=True, env=env, timeout=900)
    try:
        return float(r.stdout.strip().splitlines()[-1])
    except (ValueError, IndexError):
        return None


def compact_line(line, limit=1400):
    """The bench line as JSON of at most `limit` bytes: optional keys are
    dropped, in order, if it is longer."""
    optional = ["executed_gpts", "oracle", "gradients_per_hour", "recompute_ratio", "clocks"]
    out = json.dumps(line)
    for k in optional:
        if len(out) <= limit:
            break
        line.pop(k, None)
        out = json.dumps(line)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ckfwi")
    ap.add_argument("--nt", type=int, default=None, help="override the number of time steps (smaller runs)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle (baseline, errors, table)")
    ap.add_argument("--detail", default=os.path.join(ROOT, "gpurun_out", "bench_detail.json"),
                    help="side file for everything but the headline")
    ap.add_argument("--modes",
                    default="storeall,codec,codec_sched,rate,fp32,fp16,bf16,codec_low,rate_low,"
                            "fp32_low,fp16_low,fp32_host,fp32_eq,ot4,batch2d")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--sweep", default=None, choices=["c3", "c4", "c5"],
                    help="instead of the headline: the 300x600x600 budget sweep, the batched apertures, or the "
                         "FWI loop, into the side file")
    ap.add_argument("--budgets", default="8,16,32,64,128,256", help="c3: checkpoint budgets (uncompressed states)")
    args = ap.parse_args()
    if args.oracle_sample:
        from paper_1810_05268_gb300 import synth
        name, steps = args.oracle_sample.split(",")
        print(cpu_sample(synth.workload(name), int(steps))[0])
        return 0
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_1810_05268_gb300 import build, synth
    from paper_1810_05268_gb300 import ckfwi as C

    ws, rk, lr = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(lr)
    build.build()
    if args.sweep:
        fn = {"c3": sweep_c3, "c4": sweep_c4, "c5": sweep_c5}[args.sweep]
        res = fn(C, torch, synth, args)
        os.makedirs(os.path.dirname(os.path.abspath(args.detail)), exist_ok=True)
        with open(args.detail, "w") as f:
            json.dump({"sweep": args.sweep, "result": res}, f, indent=1)
        print("bench: %s sweep in %s" % (args.sweep, os.path.abspath(args.detail)), file=sys.stderr, flush=True)
        return 0

    w = synth.workload(WORKLOAD, nt=args.nt)
    nt = w.nt
    npts = int(np.prod(w.shape))
    grid = C.GridSpec(3, w.shape, w.nbl, w.h, w.so, w.dt, nt, w.vmax)
    # every rank its own shot: the source moves across the surface with the rank
    src = rank_source(w.src, rk, ws)
    shot = C.ShotSpec(src=src, rec=w.rec, f0=w.f0)
    model = C.Model(grid)
    model.set_model(torch.from_numpy(w.true.astype(np.float32)).cuda())
    d_obs = model.forward_shot(shot).clone()
    model.set_model(torch.from_numpy(w.start.astype(np.float32)).cuda())
    torch.cuda.synchronize()

    state_bytes = 2 * npts * 4
    modes = {}
    # codec slots at equal memory: from the worst ratio of a pilot run (the
    # last states compress worst, Sec. 7) with 10% headroom, or planned from
    # every state's measured size (non-uniform ratios, Sec. 8)
    want = args.modes.split(",")
    fmin, sizes = None, None
    if any(m.startswith("codec") for m in want):
        fmin, sizes = size_profile(C, model, shot, d_obs, nt, state_bytes)
    cm = lambda slots, sched=False: codec_modes(C, nt, state_bytes, fmin, sizes, slots, sched)
    rm = lambda slots: rate_mode(C, nt, w.shape, state_bytes, slots)
    if "codec" in want:
        modes["codec"] = cm(BUDGET_SLOTS)
    if "codec_sched" in want:
        modes["codec_sched"] = cm(BUDGET_SLOTS, True)
    if "rate" in want:
        modes["rate"] = rm(BUDGET_SLOTS)
    if "fp32" in want:
        modes["fp32"] = dict(ckpt_slots=BUDGET_SLOTS, store_mode="fp32")
    if "storeall" in want:
        modes["storeall"] = dict(ckpt_slots=nt, store_mode="fp32")
    # 16-bit slots in the same bytes: 2 (M - 1) + 1 slots (slot 0 is the initial state)
    for half in ("fp16", "bf16"):
        if half in want:
            modes[half] = dict(ckpt_slots=2 * (BUDGET_SLOTS - 1) + 1, store_mode=half)
    if "codec_low" in want:
        modes["codec_low"] = cm(LOW_SLOTS)
    if "codec_sched_low" in want:
        modes["codec_sched_low"] = cm(LOW_SLOTS, True)
    if "rate_low" in want:
        modes["rate_low"] = rm(LOW_SLOTS)
    if "fp32_low" in want:
        modes["fp32_low"] = dict(ckpt_slots=LOW_SLOTS, store_mode="fp32")
    if "fp16_low" in want:
        modes["fp16_low"] = dict(ckpt_slots=2 * (LOW_SLOTS - 1) + 1, store_mode="fp16")
    # a second storage level: the device budget plus HOST_SLOTS slots in pinned host memory
    if "fp32_host" in want:
        modes["fp32_host"] = dict(ckpt_slots=BUDGET_SLOTS + HOST_SLOTS, store_mode="fp32", host_slots=HOST_SLOTS)
    # the same slot count all in device memory: what the second level costs
    if "fp32_eq" in want:
        modes["fp32_eq"] = dict(ckpt_slots=BUDGET_SLOTS + HOST_SLOTS, store_mode="fp32")

    # the headline's candidates are timed over K replays, the rest over min(K, 5)
    cands = ("codec", "rate", "fp32", "fp16", "bf16")
    results, grads, clocks, skipped = time_modes(C, torch, model, shot, d_obs, modes, nt, npts, args, ws, lr,
                                                 full=cands)
    # gradient error of every mode against store-all (bitwise the exact
    # FP32 gradient: the schedule never changes values)
    grad_errors(torch, results, grads)
    model_block = perf_model(results, nt, fmin)

    # the FP64 oracle on the host cores: its data of the true model and its
    # gradient at the start model; every candidate's gradient from those data
    # against the oracle's (the headline must stay within GRAD_TOL of it)
    oracle = None
    cpu = None
    table = None
    if rk == 0 and not args.no_cpu:
        dobs_o, g_ref, phi_ref, secs = oracle_reference(w)
        cpu = {"value": 2.0 * nt * npts / secs / 1e9, "unit": "Gpt/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "one FP64 oracle gradient of the whole workload (%d steps, %.1f s)" % (nt, secs)}
        dd = torch.from_numpy(dobs_o).cuda()
        for name in cands:
            if name in results:
                _, g, _ = model.adjoint_gradient(shot, dd, use_graph=True, **modes[name])
                results[name]["grad_abs_err_vs_oracle"], results[name]["grad_rel_err_vs_oracle"] = err_vs(g, g_ref)
        table = error_table(C, torch, model, shot, dobs_o, g_ref, nt, npts, state_bytes, w.shape)
        oracle = {"misfit": phi_ref, "seconds": secs}
    key = "grad_rel_err_vs_oracle" if oracle else "grad_rel_err_vs_storeall"
    ok = [m for m in cands if m in results and results[m].get(key, 0.0) <= GRAD_TOL]
    headline = min(ok or list(results), key=lambda m: results[m]["ms"])
    H = results[headline]

    # end to end through the C-ABI with host buffers (pinned), same headline mode
    kw = modes[headline]
    dh = torch.empty(d_obs.shape, dtype=torch.float32, pin_memory=True)
    dh.copy_(d_obs)
    gh = torch.empty(tuple(w.shape), dtype=torch.float32, pin_memory=True)
    dh_np, gh_np = dh.numpy(), gh.numpy()
    model.adjoint_gradient(shot, dh_np, grad=gh_np, use_graph=True, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        model.adjoint_gradient(shot, dh_np, grad=gh_np, use_graph=True, **kw)
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    # the OT4 kernel on the same workload: its own unit costs and the time
    # model's break-even (Sec. 7: the costlier step favours compression)
    ot4 = None
    if "ot4" in want:
        model.close()
        ot4 = ot4_block(C, torch, w, grid, shot, nt, npts, state_bytes, args, ws, lr, results)

    batch = None
    if rk == 0 and "batch2d" in want:
        batch = batch_compare(C, torch, synth)

    if rk == 0:
        roof = roofline_block(H, nt, npts, *peaks(), delta=model_block.get("event_overhead_ms_per_call", 0.0))
        clk = clocks.get(headline) or {}
        line = {
            "metric": "gradient point-updates per second (useful 2*N*npts/t)",
            "value": H["gpts"], "unit": "Gpt/s", "n_gpus": ws, "steps": H["timed_steps"], "warmup": args.warmup,
            "ms_per_step": H["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(w.shape), "nt": nt, "space_order": w.so,
                       "mode": "%s Revolve at the memory of %d fp32 checkpoints%s" % (
                           H["store_mode"], BUDGET_SLOTS, ", abs tol %g" % TOL if H["store_mode"] == "codec" else ""),
                       "ckpt_slots": H["ckpt_slots"], "l2": "inputs > L2 (fields + checkpoints)",
                       "parallelism": "shots" if ws > 1 else "single"},
            "roofline": {"bound": "hbm", "kernel": roof["kernel"], "class": roof["class"],
                         "achieved": round(roof["achieved"], 1), "peak": roof["peak"], "unit": "GB/s",
                         "frac": round(roof["frac"], 4), "peak_kind": roof["peak_kind"],
                         "algorithmic_bytes_per_launch": roof["algorithmic_bytes_per_launch"],
                         "launch_us": round(roof["launch_us"], 2), "traffic": roof["traffic"],
                         "traffic_basis_bytes": roof["traffic_basis_bytes"]},
            "cpu_baseline": cpu,
            "e2e": {"value": 2.0 * nt * npts / e2e_s / 1e9, "unit": "Gpt/s",
                    "h2d_bytes_per_step": int(dh.numel() * 4), "d2h_bytes_per_step": int(gh.numel() * 4 + 8)},
            "gpu_launches": int(H["kernel_launches"] * H["timed_steps"]),
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons")} if clk else None,
            "recompute_ratio": round(H["recompute_ratio"], 4),
            "executed_gpts": round(H["executed_gpts"], 2),
            "gradients_per_hour": round(3.6e6 / H["ms"] * ws, 1),
            "oracle": {"grad_rel_err": H.get("grad_rel_err_vs_oracle"), "tol": GRAD_TOL} if oracle else None,
        }
        detail = {
            "headline": headline, "line": line, "roofline_all_classes": roof,
            "compare": {k: dict(v, clocks=clocks.get(k)) for k, v in results.items()},
            "skipped": skipped, "model": model_block, "oracle": oracle, "error_table": table,
            "ot4": ot4, "batch": batch,
        }
        try:
            os.makedirs(os.path.dirname(os.path.abspath(args.detail)), exist_ok=True)
            with open(args.detail, "w") as f:
                json.dump(detail, f, indent=1)
            print("bench: details in %s" % os.path.abspath(args.detail), file=sys.stderr, flush=True)
        except OSError as e:
            print("bench: could not write %s: %s" % (args.detail, e), file=sys.stderr, flush=True)
        sys.stderr.flush()
        print(compact_line(line), flush=True)
    model.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
