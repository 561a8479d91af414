"""Benchmark of the checkpointed, compressed adjoint-state gradient.

One step = one full gradient (forward sweep, residual and FP64 misfit,
Revolve reverse sweep with recomputation, compression / decompression of
checkpoints, imaging condition) of one shot on the 3D workload: 128^3
interior + 40-cell damping layer (208^3 points) at 15 m, space order 8,
1000 steps of 1 ms, Gaussian-random-field velocity 1.5-4.5 km/s, 8 Hz
Ricker source, 64 x 64 receivers.

Headline (`value`): useful point-updates per second, 2 * N * npts / t, of
the paper's method -- Revolve checkpointing with checkpoints compressed by
the fixed-tolerance codec (abs. tol 1e-4) -- at the memory of 20
uncompressed checkpoints.  Pure checkpointing (20 FP32 slots) and
store-all are timed beside it in the same run (`compare`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

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
TOL = 1e-4                 # codec absolute tolerance
FWD_BYTES = 16             # fwd kernel: read u^n, u^{n-1}, w; write u^{n+1}
ADJ_BYTES = 28             # reverse kernel: read lam^j, lam^{j+1}, u^{j-1}, w, g; write lam^{j-1}, g


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_per_point(kernel):
    """DRAM bytes per grid point per launch from the committed ncu summary, or None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d[kernel]["dram_bytes_per_point"])
    except Exception:
        return None


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
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
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


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rk = int(os.environ.get("RANK", "0"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rk, lr


def cpu_sample(w, nt_sample):
    """Oracle gradient over the first nt_sample steps of the workload (FP64, host cores)."""
    from oracle import propagator as O
    og = O.Grid(3, w.shape, w.nbl, w.h, w.so, w.dt, nt_sample, w.vmax)
    s = O.ricker(nt_sample, w.dt, w.f0)
    vel = w.start.astype(np.float32).astype(np.float64)
    dobs = np.zeros((nt_sample + 1, w.rec.shape[0]))
    t = time.perf_counter()
    O.gradient(og, vel, [w.src], s, w.rec, dobs)
    dt = time.perf_counter() - t
    npts = int(np.prod(w.shape))
    return 2.0 * nt_sample * npts / dt / 1e9, dt


def run_reference(args):
    ws, rk, _ = dist_env()
    if rk != 0:
        return 0
    from paper_1810_05268_gb300 import synth
    w = synth.workload(WORKLOAD)
    nt_sample = 6
    for _ in range(args.warmup):
        cpu_sample(w, nt_sample)
    rates, times = [], []
    for _ in range(args.steps):
        r, t = cpu_sample(w, nt_sample)
        rates.append(r)
        times.append(t)
    value = float(np.mean(rates))
    cores = os.cpu_count()
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
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ckfwi")
    ap.add_argument("--nt", type=int, default=None, help="override the number of time steps (smaller runs)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--modes", default="codec,fp32,storeall")
    args = ap.parse_args()
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

    w = synth.workload(WORKLOAD, nt=args.nt)
    nt = w.nt
    npts = int(np.prod(w.shape))
    grid = C.GridSpec(3, w.shape, w.nbl, w.h, w.so, w.dt, nt, w.vmax)
    # every rank its own shot: the source moves across the surface with the rank
    src = (w.src[0], w.src[1], w.src[2] * (0.5 + 0.5 * (rk + 1) / max(ws, 1)))
    shot = C.ShotSpec(src=src, rec=w.rec, f0=w.f0)
    model = C.Model(grid)
    model.set_model(torch.from_numpy(w.true.astype(np.float32)).cuda())
    d_obs = model.forward_shot(shot).clone()
    model.set_model(torch.from_numpy(w.start.astype(np.float32)).cuda())
    torch.cuda.synchronize()

    state_bytes = 2 * npts * 4
    budget = BUDGET_SLOTS * state_bytes
    modes = {}
    # codec slots at equal memory: size from the measured worst ratio of a
    # pilot run (the last states compress worst, Sec. 7), 10% headroom
    want = args.modes.split(",")
    if "codec" in want:
        pilot = model.adjoint_gradient(shot, d_obs, BUDGET_SLOTS, store_mode="codec", tol=TOL,
                                       pool_bytes=budget)[2]
        fmin = max(1.0, pilot["ratio_min"])
        m_codec = int(min(nt, max(2, budget / (state_bytes / fmin * 1.1))))
        modes["codec"] = dict(ckpt_slots=m_codec, store_mode="codec", tol=TOL, pool_bytes=budget)
    if "fp32" in want:
        modes["fp32"] = dict(ckpt_slots=BUDGET_SLOTS, store_mode="fp32")
    if "storeall" in want:
        modes["storeall"] = dict(ckpt_slots=nt, store_mode="fp32")
    headline = "codec" if "codec" in modes else list(modes)[0]

    def one(kw, profile):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        phi, g, st = model.adjoint_gradient(shot, d_obs, profile=profile, **kw)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, phi, st

    results = {}
    clocks = None
    for name, kw in modes.items():
        # retry with fewer codec slots if the pool overflowed at run time
        for _ in range(4):
            try:
                for _ in range(args.warmup):
                    one(kw, False)
                break
            except C.CkfwiError as e:
                if e.status != C.POOL_OVERFLOW or kw.get("store_mode") != "codec":
                    raise
                kw["ckpt_slots"] = max(2, int(kw["ckpt_slots"] * 0.8))
        # profiled warm-up creates the library's timing events, so that the
        # profiled steps below do not include host-side event creation
        one(kw, True)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if name == headline:
            clocks = Clocks(lr)
        # timed region: K un-profiled gradients, CUDA events on torch's stream
        # (the library launches on that stream), max over ranks
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            _, phi, st_plain = one(kw, False)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        if ws > 1:
            t = torch.tensor([ms], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        # per-kernel-class device time from profiled gradients (same work)
        sts = []
        for _ in range(max(1, min(args.steps, 3))):
            _, _, st = one(kw, True)
            sts.append(st)
        clk = clocks.stop() if name == headline else None
        st = sts[-1]
        fwd_ms = float(np.mean([s["fwd_ms"] for s in sts]))
        adj_ms = float(np.mean([s["adj_ms"] for s in sts]))
        results[name] = {
            "ms": ms, "gpts": 2.0 * nt * npts / (ms / 1e3) / 1e9 * ws,
            "ckpt_slots": kw["ckpt_slots"], "store_mode": kw["store_mode"],
            "recompute_ratio": st["fwd_steps"] / nt, "p": st["p"], "W": st["takeshots"], "R": st["restores"],
            "fwd_launches": st["fwd_launches"], "adj_launches": st["adj_launches"],
            "fwd_ms": fwd_ms, "adj_ms": adj_ms, "comp_ms": float(np.mean([s["comp_ms"] for s in sts])),
            "decomp_ms": float(np.mean([s["decomp_ms"] for s in sts])),
            "kernel_launches": st["kernel_launches"], "misfit": phi,
            "ratio_mean": st["ratio_mean"], "ratio_min": st["ratio_min"],
            "pool_bytes_peak": st["pool_bytes_peak"], "clocks": clk,
        }

    # end to end through the C-ABI with host buffers (pinned), same headline mode
    kw = modes[headline]
    dh = torch.empty(d_obs.shape, dtype=torch.float32, pin_memory=True)
    dh.copy_(d_obs)
    gh = torch.empty(tuple(w.shape), dtype=torch.float32, pin_memory=True)
    dh_np, gh_np = dh.numpy(), gh.numpy()
    model.adjoint_gradient(shot, dh_np, grad=gh_np, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        model.adjoint_gradient(shot, dh_np, grad=gh_np, **kw)
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    cpu = None
    if rk == 0 and not args.no_cpu:
        rate, secs = cpu_sample(w, 6)
        cpu = {"value": rate, "unit": "Gpt/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "FP64 oracle gradient on the same grid, first 6 of %d time steps (%.1f s)" % (nt, secs)}

    if rk == 0:
        H = results[headline]
        peak, peak_kind = peaks()
        # dominant kernel of the headline mode (largest share of device time)
        fwd_bytes = FWD_BYTES * npts * H["fwd_launches"]
        adj_bytes = ADJ_BYTES * npts * H["adj_launches"]
        fwd_gbs = fwd_bytes / (H["fwd_ms"] / 1e3) / 1e9 if H["fwd_ms"] > 0 else 0.0
        adj_gbs = adj_bytes / (H["adj_ms"] / 1e3) / 1e9 if H["adj_ms"] > 0 else 0.0
        if H["fwd_ms"] >= H["adj_ms"]:
            kname, ach, per, tkey = "fwd_kernel", fwd_gbs, FWD_BYTES, "fwd_kernel"
        else:
            kname, ach, per, tkey = "adj_kernel", adj_gbs, ADJ_BYTES, "adj_kernel"
        tpp = traffic_per_point(tkey)
        line = {
            "metric": "gradient point-updates per second (useful 2*N*npts/t)",
            "value": H["gpts"], "unit": "Gpt/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": H["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(w.shape), "nt": nt, "space_order": w.so,
                       "mode": "revolve+codec tol %g at the memory of %d fp32 checkpoints" % (TOL, BUDGET_SLOTS),
                       "ckpt_slots": H["ckpt_slots"], "l2": "working set (checkpoints + fields) > L2",
                       "parallelism": "shots" if ws > 1 else "single"},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_point": per,
                         "traffic": (tpp * npts) if tpp is not None else None,
                         "fwd_gbs": fwd_gbs, "adj_gbs": adj_gbs},
            "e2e": {"value": 2.0 * nt * npts / e2e_s / 1e9, "unit": "Gpt/s",
                    "h2d_bytes_per_step": int(dh.numel() * 4), "d2h_bytes_per_step": int(gh.numel() * 4 + 8)},
            "gpu_launches": int(H["kernel_launches"] * args.steps),
            "clocks": H["clocks"],
            "cpu_baseline": cpu,
            "compare": {k: {kk: vv for kk, vv in v.items() if kk != "clocks"} for k, v in results.items()},
        }
        print(json.dumps(line))
    model.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
