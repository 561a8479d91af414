"""The paper's time model of a checkpointed gradient, with measured unit
costs, and the storage choice it implies (Sec. 3, Sec. 4).

A gradient with M slots runs p(N, M) + 1 forward steps (the extra one to
u^N), N reverse steps, and -- with compressed checkpoints -- 2 W
compressions and the decompressions of the restores (Sec. 3: the recompute
count p and the takeshots W of Revolve; Sec. 4: t_c and t_d per
checkpoint).  Its time is

    T(M, mode) = (p + 1) C_F + N C_R + n_c t_c + n_d t_d,

where C_R is the reverse step of the FP32 run, or of the 16-bit run for the
modes whose restores land in a working field (a 16-bit up-cast or a codec
decode: the reverse step then reads u^s from that field),

and at a memory budget of B bytes each storage mode gets the slots that fit:
FP32 checkpoints B / S, 16-bit ones 2 (B / S - 1) + 1 (slot 0 is the initial
state), codec ones B F / (S 1.1) with F the worst compression ratio seen.
`choose` takes the mode (and slot count) the model predicts fastest among
those whose gradient error is acceptable; `sweep` tabulates the prediction
over budgets, which shows the regimes of Sec. 4 (recomputation cheap,
compression paying, everything fitting).

The counts come from the library's own Revolve schedule; the unit costs from
profiled gradients (`measure`).

Non-uniform ratios (Sec. 8 names them as the model's next step: early
wavefields are smoother and compress better).  The slot rule above sizes
every checkpoint by the worst ratio.  With the size of each state known (a
pilot gradient that compresses every state once, `state_bytes`),
`slots_for_sizes` instead replays the schedule's slot stack with those sizes
(`pool_peak`) and takes the most slots whose peak fits the budget.
"""
from dataclasses import dataclass, field
from typing import Callable, Dict, Optional

import numpy as np

from . import ckfwi as C


@dataclass
class Costs:
    c_f: float                     # forward step [ms]
    c_r: float                     # reverse step reading FP32 checkpoints [ms]
    c_r16: Optional[float] = None  # reverse step after a restore into a working field (a 16-bit
                                   # up-cast or a codec decode), measured in the 16-bit run [ms]
    t_d16: Optional[float] = None  # up-cast of one 16-bit checkpoint field [ms]
    t_ck32: float = 0.0            # extra cost of a forward step that writes an FP32 checkpoint [ms]
    t_ck16: float = 0.0            # extra cost of a forward step that writes a 16-bit checkpoint [ms]
    t_c: Optional[float] = None    # one field compression [ms]
    t_d: Optional[float] = None    # one field decompression [ms]
    f_min: Optional[float] = None  # worst compression ratio
    grad_err: Dict[str, float] = field(default_factory=dict)   # gradient error of each mode
    t_c_rate: Optional[float] = None   # fixed-rate mode: one field compression [ms]
    t_d_rate: Optional[float] = None   # fixed-rate mode: one field decompression [ms]
    rate: Optional[int] = None         # fixed-rate mode: bits per value


def counts(nt, slots, mode):
    """(forward steps, compressions, decompressions) of one gradient; for
    16-bit storage the third count is the fields up-cast by restores (a
    reverse step next needs u^s only)."""
    if slots >= nt and mode == "fp32":
        return nt, 0, 0
    slots = min(slots, nt)
    acts, (p, W, R) = C.revolve_schedule(nt, slots)
    comp = mode in ("codec", "rate")
    nc = 2 * W if comp else 0
    nd = 0
    for i, a in enumerate(acts):
        if a[0] == 2 and a[2] > 0:               # restore from a slot
            nxt = acts[i + 1][0] if i + 1 < len(acts) else -1
            if comp or mode in ("fp16", "bf16"):
                nd += 1 if nxt == 3 else 2        # a reverse step next needs u^s only
    return p + 1, nc, nd


def events(nt, slots, mode):
    """Every cost-bearing event of one gradient: forward steps, takeshots,
    compressions and decompressions (fields; 16-bit: fields up-cast)."""
    nf, nc, nd = counts(nt, slots, mode)
    ev = {"fwd": nf, "takeshots": 0, "comp": nc, "decomp": nd}
    if slots >= nt and mode == "fp32":
        return ev
    acts, (p, W, R) = C.revolve_schedule(nt, min(slots, nt))
    ev["takeshots"] = W
    return ev


def predict(costs: Costs, nt, slots, mode):
    """Predicted gradient time [ms] with `slots` slots of `mode` storage
    (Sec. 3-4: recomputation, storage writes and reads, compression)."""
    ev = events(nt, slots, mode)
    nf, nc, nd = ev["fwd"], ev["comp"], ev["decomp"]
    # a reverse step whose u^s was just up-cast or decoded into a working
    # field costs what the 16-bit run measured, where known
    c_rev = costs.c_r16 if (mode != "fp32" and costs.c_r16 is not None) else costs.c_r
    t = nf * costs.c_f + nt * c_rev
    if mode == "fp32":
        return t + ev["takeshots"] * costs.t_ck32
    if mode in ("fp16", "bf16"):
        return t + ev["takeshots"] * costs.t_ck16 + nd * (costs.t_d16 or 0.0)
    if nc or nd:
        tc, td = (costs.t_c_rate, costs.t_d_rate) if mode == "rate" else (costs.t_c, costs.t_d)
        if tc is None or td is None:
            raise ValueError("%s costs not measured" % mode)
        t += nc * tc + nd * td
    return t


def slots_for(budget_fp32_slots, mode, nt, f_min=None, rate=None):
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
    if mode == "rate":
        if not rate:
            raise ValueError("the fixed-rate mode needs its rate")
        return int(min(nt, 1 + b * 32 // rate))
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
        if mode == "rate" and (costs.t_c_rate is None or not costs.rate):
            continue
        m = slots_for(budget_fp32_slots, mode, nt, costs.f_min, costs.rate)
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
            if mode == "rate" and (costs.t_c_rate is None or not costs.rate):
                continue
            row[mode] = predict(costs, nt, slots_for(b, mode, nt, costs.f_min, costs.rate), mode)
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


def state_bytes(nt, slots, words):
    """{state: bytes} of the states a compressed-checkpoint gradient with
    `slots` slots stored, from its stream words (schedule order, two per
    takeshot: u^s then u^{s-1}; `ckfwi.stream_words`)."""
    acts, _ = C.revolve_schedule(nt, min(slots, nt))
    out, k = {}, 0
    if 2 * int(sum(1 for a in acts if a[0] == 1)) != len(words):
        raise ValueError("stream words do not match the schedule")
    for op, a, b in acts:
        if op == 1:
            out[int(a)] = 4 * int(words[k] + words[k + 1])
            k += 2
    if k != len(words):
        raise ValueError("stream words do not match the schedule (%d of %d used)" % (k, len(words)))
    return out


def size_function(sizes):
    """size_of(state) from measured {state: bytes}: linear interpolation
    between measured states, the nearest one outside them."""
    st = np.array(sorted(sizes), dtype=np.float64)
    by = np.array([sizes[k] for k in sorted(sizes)], dtype=np.float64)
    return lambda s: float(np.interp(float(s), st, by))


def pool_peak(nt, slots, size_of: Callable[[int], float]):
    """Peak bytes of the checkpoint pool when state s takes size_of(s) bytes.
    The slots form a stack (a takeshot into slot b drops the slots above
    it), so at a takeshot the pool holds slots 1..b."""
    acts, _ = C.revolve_schedule(nt, min(slots, nt))
    height = [0.0] * (min(slots, nt) + 2)
    peak = 0.0
    for op, a, b in acts:
        if op == 1:
            height[b] = height[b - 1] + size_of(int(a))
            peak = max(peak, height[b])
    return peak


def slots_for_sizes(nt, budget_bytes, size_of: Callable[[int], float], headroom=1.02):
    """The most slots (<= nt) whose pool peak, with these per-state sizes
    and a small headroom, fits the budget; 1 (the initial state only) if
    none does."""
    fits = lambda m: pool_peak(nt, m, size_of) * headroom <= budget_bytes
    lo, hi = 1, nt
    if fits(hi):
        return hi
    while hi - lo > 1:                   # the peak grows with the slots
        mid = (lo + hi) // 2
        if fits(mid):
            lo = mid
        else:
            hi = mid
    while lo > 1 and not fits(lo):       # guard a non-monotone step
        lo -= 1
    return lo
