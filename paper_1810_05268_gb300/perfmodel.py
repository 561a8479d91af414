"""The paper's time model of a checkpointed gradient, with measured unit
costs, and the storage choice it implies (Sec. 3, Sec. 4).

A gradient with M slots runs p(N, M) + 1 forward steps (the extra one to
u^N), N reverse steps, and -- with compressed checkpoints -- 2 W
compressions and the decompressions of the restores (Sec. 3: the recompute
count p and the takeshots W of Revolve; Sec. 4: t_c and t_d per
checkpoint).  Its time is

    T(M, mode) = (p + 1) C_F + N C_R + n_c t_c + n_d t_d,

and at a memory budget of B bytes each storage mode gets the slots that fit:
FP32 checkpoints B / S, 16-bit ones 2 (B / S - 1) + 1 (slot 0 is the initial
state), codec ones B F / (S 1.1) with F the worst compression ratio seen.
`choose` takes the mode (and slot count) the model predicts fastest among
those whose gradient error is acceptable; `sweep` tabulates the prediction
over budgets, which shows the regimes of Sec. 4 (recomputation cheap,
compression paying, everything fitting).

The counts come from the library's own Revolve schedule; the unit costs from
profiled gradients (`measure`).
"""
from dataclasses import dataclass, field
from typing import Dict, Optional

from . import ckfwi as C


@dataclass
class Costs:
    c_f: float                     # forward step [ms]
    c_r: float                     # reverse step reading FP32 checkpoints [ms]
    c_r16: Optional[float] = None  # reverse step reading 16-bit checkpoints directly [ms]
    t_c: Optional[float] = None    # one field compression [ms]
    t_d: Optional[float] = None    # one field decompression [ms]
    f_min: Optional[float] = None  # worst compression ratio
    grad_err: Dict[str, float] = field(default_factory=dict)   # gradient error of each mode


def counts(nt, slots, mode):
    """(forward steps, compressions, decompressions) of one gradient."""
    if slots >= nt and mode == "fp32":
        return nt, 0, 0
    slots = min(slots, nt)
    acts, (p, W, R) = C.revolve_schedule(nt, slots)
    nc = 2 * W if mode == "codec" else 0
    nd = 0
    if mode == "codec":
        for i, a in enumerate(acts):
            if a[0] == 2 and a[2] > 0:           # restore from a slot
                nxt = acts[i + 1][0] if i + 1 < len(acts) else -1
                nd += 1 if nxt == 3 else 2        # a reverse step next needs u^s only
    return p + 1, nc, nd


def predict(costs: Costs, nt, slots, mode):
    """Predicted gradient time [ms] with `slots` slots of `mode` storage."""
    nf, nc, nd = counts(nt, slots, mode)
    c_r = costs.c_r16 if mode in ("fp16", "bf16") and costs.c_r16 is not None else costs.c_r
    t = nf * costs.c_f + nt * c_r
    if nc or nd:
        if costs.t_c is None or costs.t_d is None:
            raise ValueError("codec costs not measured")
        t += nc * costs.t_c + nd * costs.t_d
    return t


def slots_for(budget_fp32_slots, mode, nt, f_min=None):
    """Slots of `mode` that fit in the memory of `budget_fp32_slots` FP32 checkpoints."""
    b = budget_fp32_slots
    if mode == "fp32":
        return min(b, nt)
    if mode in ("fp16", "bf16"):
        return min(2 * (b - 1) + 1, nt)
    if mode == "codec":
        if not f_min:
            raise ValueError("codec needs the worst compression ratio")
        return int(min(nt, max(2, b * f_min / 1.1)))
    raise ValueError(mode)


def choose(costs: Costs, nt, budget_fp32_slots, modes=("fp32", "fp16", "bf16", "codec"), grad_tol=None):
    """(mode, slots, predicted ms) the model predicts fastest at the budget,
    among the modes whose measured gradient error is within grad_tol (all
    when grad_tol is None or the error was not measured)."""
    best = None
    for mode in modes:
        if grad_tol is not None and costs.grad_err.get(mode, 0.0) > grad_tol:
            continue
        if mode == "codec" and (costs.t_c is None or not costs.f_min):
            continue
        m = slots_for(budget_fp32_slots, mode, nt, costs.f_min)
        t = predict(costs, nt, m, mode)
        if best is None or t < best[2]:
            best = (mode, m, t)
    return best


def sweep(costs: Costs, nt, budgets, modes=("fp32", "fp16", "codec")):
    """Predicted time of every mode over budgets (in FP32 checkpoints)."""
    rows = []
    for b in budgets:
        row = {"budget_fp32_slots": b}
        for mode in modes:
            if mode == "codec" and (costs.t_c is None or not costs.f_min):
                continue
            row[mode] = predict(costs, nt, slots_for(b, mode, nt, costs.f_min), mode)
        row["best"] = min((k for k in row if k != "budget_fp32_slots"), key=lambda k: row[k])
        rows.append(row)
    return rows


def measure(model, shot, d_obs, nt, slots=20, tol=1e-4, state_bytes=None, reps=2):
    """Unit costs from profiled gradients on `model`: FP32, FP16 and codec
    checkpoints (the codec pool sized like `slots` FP32 checkpoints)."""
    def prof(**kw):
        best = None
        for _ in range(reps):
            _, _, st = model.adjoint_gradient(shot, d_obs, profile=True, **kw)
            best = st if best is None or st["fwd_ms"] + st["adj_ms"] < best["fwd_ms"] + best["adj_ms"] else best
        return best
    s32 = prof(ckpt_slots=slots, store_mode="fp32")
    s16 = prof(ckpt_slots=2 * (slots - 1) + 1, store_mode="fp16")
    kw = dict(ckpt_slots=slots, store_mode="codec", tol=tol)
    if state_bytes:
        kw["pool_bytes"] = int(slots * state_bytes)
    sc = prof(**kw)
    return Costs(c_f=s32["fwd_ms"] / s32["fwd_launches"], c_r=s32["adj_ms"] / s32["adj_launches"],
                 c_r16=s16["adj_ms"] / s16["adj_launches"],
                 t_c=sc["comp_ms"] / max(1, sc["comp_calls"]), t_d=sc["decomp_ms"] / max(1, sc["decomp_calls"]),
                 f_min=sc["ratio_min"])
