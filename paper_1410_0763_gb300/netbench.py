"""Time the surrogate network on one grid: forward passes and training steps
(random inputs; weights as initialised).  ``python -m
paper_1410_0763_gb300.netbench --n 128 --reps 20`` prints one JSON line with
the per-pass time and the algorithmic TFLOP/s of each."""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128, help="cells per axis (cubic grid)")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--train", action="store_true", help="also time training steps")
    a = ap.parse_args(argv)
    import torch
    from . import art, build
    build.build()
    art.load()
    n, V = a.n, a.n ** 3
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn(4 * V, device="cuda", generator=g)
    t = torch.randn(V, device="cuda", generator=g)
    o = torch.empty(V, device="cuda")
    net = art.ArtNet()
    shape = (n, n, n)
    for _ in range(3):
        net.forward(X, o, shape)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        net.forward(X, o, shape)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    flops = 2.0 * 27 * V * (4 * 32 + 32 * 32 * 2 + 32 * 1)
    out = {"n": n, "forward_ms": round(ms, 4), "forward_tflops_algorithmic": round(flops / ms / 1e9, 1)}
    if a.train:
        for _ in range(2):
            net.train_step(X, t, shape, want_loss=False)
        e0.record()
        for _ in range(a.reps):
            net.train_step(X, t, shape, want_loss=False)
        e1.record()
        torch.cuda.synchronize()
        out["train_step_ms"] = round(e0.elapsed_time(e1) / a.reps, 4)
    net.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
