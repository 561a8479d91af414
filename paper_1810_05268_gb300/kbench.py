"""Kernel-level driver: forward modelling, a store-all gradient and a codec
round trip on one synthetic 3D model, through the C-ABI; optionally a
gradient with FP16 checkpoints (the up-cast kernel) and a batched gradient
over several shots (the batched step kernels).  Used for timing and ncu
captures of single kernels on a chosen grid.

  python -m paper_1810_05268_gb300.kbench --shape 256,256,256 --so 8 --nt 12
  python -m paper_1810_05268_gb300.kbench --shape 128,128,128 --nt 12 --fp16 --batch 4
"""
import argparse
import json
import time

import numpy as np
import torch

from . import build, synth
from . import ckfwi as C


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", default="256,256,256")
    ap.add_argument("--so", type=int, default=8)
    ap.add_argument("--nt", type=int, default=12)
    ap.add_argument("--h", type=float, default=15.0)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--time-order", type=int, default=2, help="2: OT2 kernel, 4: OT4 kernel")
    ap.add_argument("--fp16", action="store_true", help="also a gradient with FP16 checkpoints (4 slots)")
    ap.add_argument("--batch", type=int, default=0, help="also a batched gradient over this many shots")
    args = ap.parse_args()
    build.build()
    shape = tuple(int(v) for v in args.shape.split(","))
    nbl = 20
    vel = synth.extend(synth.grf(tuple(n - 2 * nbl for n in shape), 8.0, 5, 1.5, 4.5), nbl).astype(np.float32)
    grid = C.GridSpec(3, shape, nbl, args.h, args.so, 1.0, args.nt, 4.5, time_order=args.time_order)
    ext = [(n - 2 * nbl - 1) * args.h for n in shape]
    rec = synth.receiver_grid(2 * args.h, np.linspace(0, ext[1], 32), np.linspace(0, ext[2], 32))
    shot = C.ShotSpec(src=(2 * args.h, ext[1] / 2, ext[2] / 2), rec=rec, f0=0.02, t0=25.0)
    m = C.Model(grid)
    m.set_model(torch.from_numpy(vel).cuda())
    out = {"shape": shape, "so": args.so, "nt": args.nt, "time_order": args.time_order}
    for _ in range(args.reps):
        d = m.forward_shot(shot)
    torch.cuda.synchronize()
    t = time.perf_counter()
    d = m.forward_shot(shot)
    torch.cuda.synchronize()
    out["forward_ms_per_step"] = (time.perf_counter() - t) * 1e3 / args.nt
    dobs = d * 1.01
    for _ in range(args.reps):
        _, g, st = m.adjoint_gradient(shot, dobs, ckpt_slots=args.nt, profile=True)
    out["fwd_us"] = st["fwd_ms"] * 1e3 / st["fwd_launches"]
    out["adj_us"] = st["adj_ms"] * 1e3 / st["adj_launches"]
    npts = int(np.prod(shape))
    # algorithmic bytes per point of a step (OT4: both passes)
    fb, ab = (32, 72) if args.time_order == 4 else (16, 28)
    out["fwd_gbs"] = fb * npts / (out["fwd_us"] * 1e-6) / 1e9
    out["adj_gbs"] = ab * npts / (out["adj_us"] * 1e-6) / 1e9
    # ver, bx, by, zlen, vec, pf: the CKFWI_TILE_FWD / CKFWI_TILE_ADJ form
    out["fwd_kernel"] = [st["fwd_ver"], st["fwd_bx"], st["fwd_by"], st["fwd_zlen"], st["fwd_vec"], st["fwd_pf"]]
    out["adj_kernel"] = [st["adj_ver"], st["adj_bx"], st["adj_by"], st["adj_zlen"], st["adj_vec"], st["adj_pf"]]
    if args.fp16:
        # Revolve with FP16 checkpoints: every restore up-casts u^s (and u^{s-1})
        _, _, st16 = m.adjoint_gradient(shot, dobs, ckpt_slots=min(4, args.nt), store_mode=C.STORE_FP16,
                                        profile=True)
        out["fp16_upcast_us"] = st16["decomp_ms"] * 1e3 / max(1, st16["decomp_calls"])
    if args.batch > 0:
        # shots along y; one launch per stencil step over all lanes
        shots = [C.ShotSpec(src=(2 * args.h, float(y), ext[2] / 2), rec=rec, f0=0.02, t0=25.0)
                 for y in np.linspace(0.2 * ext[1], 0.8 * ext[1], args.batch)]
        dl = [m.forward_shot(s) * 1.01 for s in shots]
        for _ in range(args.reps):
            _, _, stb = m.batch_gradient(shots, dl, min(4, args.nt), store_mode=C.STORE_FP16, profile=True)
        out["batch_fwd_us"] = stb["fwd_ms"] * 1e3 / stb["fwd_launches"]
        out["batch_adj_us"] = stb["adj_ms"] * 1e3 / stb["adj_launches"]
        out["batch_kernels"] = [stb["fwd_ver"], stb["adj_ver"]]
    # codec on a wavefield-like field: the last forward state of the shot
    x = torch.from_numpy((vel - vel.mean()) * 1e-2).cuda()
    for _ in range(args.reps):
        words, _ = C.codec_compress(x, args.tol)
        y = C.codec_decompress(words, shape)
    out["codec_ratio"] = npts / words.numel()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.reps):
        C.codec_compress(x, args.tol)
    torch.cuda.synchronize()
    out["compress_us"] = (time.perf_counter() - t) * 1e6 / args.reps
    t = time.perf_counter()
    for _ in range(args.reps):
        C.codec_decompress(words, shape)
    torch.cuda.synchronize()
    out["decompress_us"] = (time.perf_counter() - t) * 1e6 / args.reps
    # the fixed-rate mode at 16 bits per value
    for _ in range(args.reps):
        rw, _ = C.codec_compress_rate(x, 16)
        C.codec_decompress(rw, shape)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.reps):
        C.codec_compress_rate(x, 16)
    torch.cuda.synchronize()
    out["compress_rate16_us"] = (time.perf_counter() - t) * 1e6 / args.reps
    t = time.perf_counter()
    for _ in range(args.reps):
        C.codec_decompress(rw, shape)
    torch.cuda.synchronize()
    out["decompress_rate16_us"] = (time.perf_counter() - t) * 1e6 / args.reps
    print(json.dumps(out))


if __name__ == "__main__":
    main()
