#!/usr/bin/env python
"""Benchmark of the diffuse-radiation parallel-ray sweep (Tanaka et al. 2014).

Metric: ray-segment updates per second -- the exact number of (ray, cell)
pairs with path length > 0 in one sweep (all directions, all bins), divided by
device time.  A step is one sweep of the whole hot path: the per-slab
transfer of Eq. (rt) along every ray of every HEALPix direction, the cell
averages of Eq. (averaged_intensity), the angle average J^in / J of
Eq. (mean_intensity) and the Gamma^diff epilogue of Eq. (gamma_diff).

Default workload (``grf64``): 64^3 cells, N_side = 4 (192 directions), one
frequency bin, FP32; kappa from a lognormal Gaussian random field (sigma = 1,
P(k) ~ k^-3) scaled to box optical depth 10, S proportional to density.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank sweeps its own independent
grid of the same size (weak scaling, no collective on the data path); the
value is all ranks' segments divided by the max over ranks of the timed device
time.  ``--impl reference`` times the FP64 CPU oracle on the host cores, on
rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "clumpy4": dict(n=256, nside=8, seed=5, bins=4, kind="clumpy", steps=12,
                    desc="256^3 clumpy medium (lognormal sigma 1.5, P(k)~k^-3, + 200 spheres x100), N_side 8 "
                         "(768 dirs), 4 bins of a 1e5 K blackbody (kappa_b ~ rho sigma_b, box tau 10 in bin 0; "
                         "S_b ~ rho)"),
    "grf64": dict(n=64, nside=4, seed=2, sigma=1.0,
                  desc="64^3 lognormal GRF (sigma 1, P(k)~k^-3, box tau 10), N_side 4 (192 dirs), 1 bin"),
    "grf128": dict(n=128, nside=8, seed=3, sigma=1.0,
                   desc="128^3 lognormal GRF (sigma 1, P(k)~k^-3, box tau 10), N_side 8 (768 dirs), 1 bin"),
    "grf256": dict(n=256, nside=8, seed=5, sigma=1.5,
                   desc="256^3 lognormal GRF (sigma 1.5, P(k)~k^-3, box tau 10), N_side 8 (768 dirs), 1 bin"),
}
METRIC = "ray-segment updates/sec"
UNIT = "segments/s"
L2_FLUSH_BYTES = 256 << 20      # > 129 MB L2
# MUFU ex2 results per clock per SM measured on GB300 (profiles/peaks_gb300.md);
# bench.py re-measures it on the box (art_measure_pipes) and uses the live value
EX2_PER_CLK_SM = 32
FFMA_PER_CLK_SM = 128
# FP32 operations of one segment, counted from Eq. (rt) and the deposit of
# Eq. (averaged_intensity): dtau = kappa ds; 1 - e^-dtau; I_in (1 - e) / kappa
# (two products) added to the cell sum; I_out = S + (I_in - S) e (two).
FP32_OPS_PER_SEG = 7
HERE = os.path.dirname(os.path.abspath(__file__))


def measured_hbm_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def measured_bf16_peak():
    """Sustained dense BF16 TFLOP/s measured on this machine (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"])
    except (OSError, KeyError, ValueError):
        return 1700.0


def kernel_source(variant: int) -> str:
    """The source file of the sweep kernel that a variant runs (wavefront variants are 16 and up)."""
    name = "art_wave.cuh" if variant >= 16 else "art_kernels.cuh"
    return os.path.join(HERE, "paper_1410_0763_gb300", "csrc", name)


def recorded_traffic(workload: str, variant: int, persistent: int):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on this workload, kernel variant and launch form with the kernel
    source as it is now; else None."""
    import hashlib
    path = os.path.join(HERE, "profiles", f"traffic_sweep_{workload}.txt")
    try:
        rec = dict(line.split(": ", 1) for line in open(path).read().splitlines() if ": " in line)
        digest = hashlib.sha256(open(kernel_source(variant), "rb").read()).hexdigest()
    except OSError:
        return None
    if rec.get("kernel_source_sha256") != digest or int(rec.get("variant", -1)) != variant or \
            int(rec.get("persistent", -1)) != persistent:
        return None
    return int(rec["dram_bytes_per_launch"])


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None, help="timed steps (default: per workload)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="clumpy4")
    p.add_argument("--paper-tests", action="store_true",
                   help="also run the paper's test problems as printed (Tests 1-3 with the energy equation, "
                        "Test 2's angular-resolution study) and the ray-grouping ablation")
    p.add_argument("--profile-case", choices=["sweep", "net", "hii", "clumpy", "thermal"], default=None,
                   help="run one small case for a profiler (ncu) instead of the benchmark")
    p.add_argument("--n", type=int, default=None, help="--profile-case: cells per axis")
    p.add_argument("--nside", type=int, default=None, help="--profile-case sweep: N_side")
    p.add_argument("--variant", type=int, default=0, help="--profile-case sweep: kernel variant (0: default)")
    p.add_argument("--reps", type=int, default=3, help="--profile-case: repetitions")
    p.add_argument("--bin", type=int, default=None, help="--profile-case sweep: one bin of a multi-bin workload")
    p.add_argument("--train", action="store_true", help="--profile-case net: also time training steps")
    p.add_argument("--myr", type=float, default=30.0, help="--profile-case thermal: evolve to this time")
    p.add_argument("--no-autotune", action="store_true", help="keep the default kernel variant")
    p.add_argument("--no-graph", action="store_true", help="plain launches instead of CUDA-graph replay")
    p.add_argument("--no-extra", action="store_true", help="skip the side measurements (128^3, 256^3, 48-grid batch, 128^3 ionization solve)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--shard", action="store_true",
                   help="strong scaling: one grid, its directions split over the ranks, the shares combined by "
                        "the rank-ordered reduce-scatter inside the timed region")
    a = p.parse_args()
    if a.steps is None:
        a.steps = WORKLOADS[a.workload].get("steps", 200)
    return a


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self, backend: str, always: bool = False):
        """One process per GPU (torchrun's environment); a process group when there are several
        ranks, or always (the sharded sweep's collectives run on a one-rank group too)."""
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1 or always:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", "29517")
            os.environ.setdefault("WORLD_SIZE", str(self.world))
            os.environ.setdefault("RANK", str(self.rank))
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max(self, x: float, device) -> float:
        if not self.dist:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(os.environ.get("ART_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def make_case(wl_name: str, rank: int):
    """The workload's seeded input (a different seed per rank: independent grids)."""
    from paper_1410_0763_gb300 import workloads as wl
    w = WORKLOADS[wl_name]
    if w.get("kind") == "clumpy":
        return wl.clumpy_sweep(w["n"], w["nside"], seed=w["seed"] + 1000 * rank, nbins=w["bins"])
    return wl.grf(w["n"], w["nside"], seed=w["seed"] + 1000 * rank, sigma=w["sigma"])


def case_bins(case) -> int:
    return 1 if case.kappa.ndim == 3 else int(case.kappa.shape[0])


def band_G(nbins: int = 1):
    """Band integrals of the Gamma epilogue: the recombination band [nu0, nu0 + k T / h] for one bin;
    for the blackbody bins of the clumpy workload, the integral over each bin."""
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    c = wl.chem_constants()
    if nbins == 1:
        return [art.art_band_integral(c["sigma0"], c["h"], c["nu0"], c["nu0"], c["nu0"] + c["dnu"])]
    _, _, edges = wl.blackbody_bins()
    return [art.art_band_integral(c["sigma0"], c["h"], c["nu0"], edges[b], edges[b + 1]) for b in range(nbins)]


def time_device(sw, J, Jin, gam, steps, flush, torch):
    """Per-step CUDA-event time (ms) of `steps` sweeps, L2 flushed between steps."""
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        sw.sweep(J, Jin, gam)
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def side_measure(wl_name, torch, dev, steps=5):
    from paper_1410_0763_gb300 import art
    c = make_case(wl_name, 0)
    k = torch.as_tensor(c.kappa, dtype=torch.float32, device=dev)
    s = torch.as_tensor(c.src, dtype=torch.float32, device=dev)
    sw = art.ArtSweep(c.shape, c.nside, case_bins(c))
    sw.set_fields(k, s)
    sw.set_band(band_G(case_bins(c)))
    J, Jin, gam = torch.empty_like(k), torch.empty_like(k), torch.empty(c.shape, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(2):
        sw.sweep(J, Jin, gam)
    ms = time_device(sw, J, Jin, gam, steps, flush, torch)
    seg = sw.stats.segments
    assert sw.check() == art.ART_OK
    sw.close()
    t = statistics.median(ms)
    return {"workload": WORKLOADS[wl_name]["desc"], "ms_per_step": round(t, 4),
            "segments_per_step": int(seg), "value": seg / (t * 1e-3)}


def batch_measure(torch, dev, steps=5):
    """48 grids of 32^3..96^3 cells and N_side 2..8 in one context: work-queue
    launches replayed as a CUDA graph, kernel variant picked by the autotuner
    (untimed), L2 flushed between timed steps."""
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    cases = wl.batch48()
    shapes = [c.kappa.shape for c in cases]
    k = torch.cat([torch.as_tensor(c.kappa.ravel(), dtype=torch.float32) for c in cases]).to(dev)
    s = torch.cat([torch.as_tensor(c.src.ravel(), dtype=torch.float32) for c in cases]).to(dev)
    sw = art.ArtSweep(shapes, [c.nside for c in cases], graph=True)
    sw.set_fields(k, s)
    t0 = time.perf_counter()
    best = sw.autotune(2)
    tune_s = time.perf_counter() - t0
    Jin = torch.empty_like(k)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(3):
        sw.sweep(J_in=Jin)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        sw.sweep(J_in=Jin)
        b.record(stream)
    torch.cuda.synchronize()
    t = statistics.median([a.elapsed_time(b) for a, b in evs])
    st = sw.stats
    sw.close()
    return {"workload": "48 grids, sizes from {32,48,64,96}^3, N_side from {2,4,8}, lognormal GRF "
                        "sigma in [0.5,1.5], one bin",
            "cells": int(sum(np.prod(x) for x in shapes)), "ms_per_step": round(t, 4),
            "segments_per_step": int(st.segments), "value": st.segments / (t * 1e-3),
            "variant": best, "autotune_s": round(tune_s, 3), "work_items": int(st.work_items),
            "ctas_per_launch": int(st.ctas_per_launch), "launches": int(st.launches), "graph": True}


def ionization_measure(torch, dev, tol=1e-6, n_setups=8, n_iter=24, train_steps=1500):
    """RT / ionization-balance solve of a 128^3 HII region (N_side 8, n_H 1e-3,
    Q 5e48 s^-1 at the centre, 6.6 kpc box) to residual tol: plain iteration
    from x = 1e-4, and warm-started (coarse-mesh solve, factor 4, N_side 4;
    then the surrogate phase with the network, or without it).  The network is
    first trained (untimed) on the iterates of n_setups random HII setups
    (lognormal density, 1-8 sources) that do not include this one."""
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    case = wl.hii_region()
    n = case.n
    V = n ** 3
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device=dev)

    def fresh():
        return torch.as_tensor(case.y0, dtype=torch.float64, device=dev).clone()

    def timed(fn, reps=3):
        best, out = None, None
        for _ in range(reps):
            y = fresh()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn(y)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        return best, out, y

    sw.iterate(nH, case.chem, srcs, fresh(), tol=tol, max_iter=300)        # warm-up (first-call allocations)
    t_plain, (rep, _), y_plain = timed(lambda y: sw.iterate(nH, case.chem, srcs, y, tol=tol, max_iter=300))
    y_plain = y_plain.cpu().numpy()
    out = {"workload": "128^3 HII region, N_side 8, uniform n_H 1e-3, T 1e4 K, Q 5e48 s^-1 central, 6.6 kpc, "
                       "FP32 sweep + FP64 balance", "tol": tol, "seconds_best_of": 3,
           "plain": {"iterations": int(rep.iterations), "seconds": round(t_plain, 4), "converged": bool(rep.converged)}}

    def warm(label, net, **kw):
        t, (wr, _), y = timed(lambda y: sw.iterate_warm(net, nH, case.chem, srcs, y, tol=tol, max_iter=300, **kw))
        dy = float(np.max(np.abs(y.cpu().numpy() - y_plain) / y_plain))
        out[label] = {"iterations": int(wr.total.iterations), "coarse_iterations": int(wr.coarse_iterations),
                      "surrogate_iterations": int(wr.surrogate_iterations), "full_sweeps": int(wr.plain_sweeps),
                      "judge_error": round(float(wr.judge_error), 5), "fell_back": bool(wr.fell_back),
                      "seconds": round(t, 4), "speedup_vs_plain": round(t_plain / t, 3),
                      "max_rel_dy_vs_plain": dy, "converged": bool(wr.total.converged)}

    warm("warm_coarse_solve", None, use_net=False, phase1_max_iter=0)
    warm("warm_coarse_solve_coarse_sweep_phase", None, use_net=False)
    # the on-the-spot approximation (alpha_A = alpha_B: no diffuse field, no sweep)
    otsa = dict(case.chem, alphaA=case.chem["alphaB"])
    sw.iterate(nH, otsa, srcs, fresh(), tol=tol, max_iter=300)
    t_otsa, (rep_o, _), y_otsa = timed(lambda y: sw.iterate(nH, otsa, srcs, y, tol=tol, max_iter=300))
    y_otsa = y_otsa.cpu().numpy()
    out["on_the_spot"] = {"iterations": int(rep_o.iterations), "seconds": round(t_otsa, 4),
                          "converged": bool(rep_o.converged),
                          "mean_neutral_fraction": float(np.mean(y_otsa)),
                          "mean_neutral_fraction_with_diffuse": float(np.mean(y_plain)),
                          "ionized_volume_ratio_diffuse_over_otsa": float(np.sum(1 - y_plain) / np.sum(1 - y_otsa))}
    # train the network on other setups (untimed)
    X = torch.empty((n_setups * n_iter, 4, V), device=dev)
    T = torch.empty((n_setups * n_iter, V), device=dev)
    W = torch.empty((n_setups * n_iter, V), device=dev)
    t0 = time.perf_counter()
    for k in range(n_setups):
        c = wl.hii_random(n, case.nside, seed=100 + k)
        sk = art.ArtSweep(c.nH.shape, c.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=c.chem["dx"])
        yk = torch.as_tensor(c.y0, dtype=torch.float64, device=dev).clone()
        sk.surrogate_collect(torch.as_tensor(c.nH, dtype=torch.float64, device=dev), c.chem,
                             [(p[0], p[1], p[2], q) for p, q in zip(c.pos, c.Q)], yk,
                             X[k * n_iter:(k + 1) * n_iter], T[k * n_iter:(k + 1) * n_iter], n_iter,
                             w=W[k * n_iter:(k + 1) * n_iter])
        sk.close()
    torch.cuda.synchronize()
    t_collect = time.perf_counter() - t0
    net = art.ArtNet(dilation=(1, 2, 4, 8), lr=3e-4, seed=1)
    t0 = time.perf_counter()
    hist = net.train(X, T, (n, n, n), n_setups * n_iter, train_steps, w=W, seed=1)
    t_train = time.perf_counter() - t0
    del X, T, W
    warm("warm_coarse_solve_net_phase", net)
    out["training"] = {"samples": n_setups * n_iter, "steps": train_steps, "collect_seconds": round(t_collect, 2),
                       "train_seconds": round(t_train, 2), "loss_first100": float(np.mean(hist[:100])),
                       "loss_last100": float(np.mean(hist[-100:]))}
    o = torch.empty(V, device=dev)
    xin = torch.zeros(4 * V, device=dev)
    for _ in range(3):
        net.forward(xin, o, (n, n, n))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        net.forward(xin, o, (n, n, n))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 20
    flops = 2.0 * 27 * V * (4 * 32 + 32 * 32 * 2 + 32 * 1)
    tflops = flops / (ms * 1e-3) / 1e12
    peak = measured_bf16_peak()
    out["network_forward"] = {"ms": round(ms, 4), "tflops_algorithmic": round(tflops, 1),
                              "roofline": {"bound": "tensor", "achieved": round(tflops, 1), "peak": peak,
                                           "unit": "TFLOP/s", "frac": round(tflops / peak, 4) if peak else None,
                                           "peak_basis": "measured sustained cuBLAS BF16 (MEASURED_PEAKS.json), "
                                                         "the kernel runs inside a long solve"},
                              "note": "4 layers, 128^3 cells, BF16 tcgen05 MMA, FP32 accumulation; "
                                      "algorithmic FLOPs 2 x 27 x c_in x c_out per cell and layer"}
    sw.close()
    clumpy = clumpy_measure(torch, dev, net, tol)
    net.close()
    return out, clumpy


def clumpy_measure(torch, dev, net, tol=1e-6):
    """The clumpy 256^3 medium (lognormal sigma 1.5 plus 200 clumps of
    overdensity 100, mean n_H 1e-3, 6.6 kpc, N_side 8) with 8 sources of
    5e48 s^-1 over 4 blackbody (1e5 K) bins above 13.6 eV: plain iteration and
    warm starts, one run each (the network is the one trained at 128^3)."""
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    case = wl.clumpy()
    frac, sig, _ = wl.blackbody_bins()
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    sw.set_source_spectrum(sig, frac)
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device=dev)
    out = {"workload": "256^3 clumpy (lognormal sigma 1.5 + 200 clumps x100, mean n_H 1e-3), N_side 8, 8 sources "
                       "x 5e48 s^-1, 4 blackbody bins (1e5 K) above 13.6 eV, 6.6 kpc", "tol": tol,
           "bins": {"frac": [round(float(v), 5) for v in frac], "sigma_over_sigma0": [round(float(v / wl.SIGMA0), 5)
                                                                                      for v in sig]}}

    def run(label, fn):
        y = torch.as_tensor(case.y0, dtype=torch.float64, device=dev).clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            res = fn(y)
        except Exception as ex:  # pragma: no cover
            out[label] = {"error": str(ex)}
            return None
        torch.cuda.synchronize()
        out[label] = {"seconds": round(time.perf_counter() - t0, 3)}
        return res, y

    r = run("plain", lambda y: sw.iterate(nH, case.chem, srcs, y, tol=tol, max_iter=400))
    if r:
        (rep, _), y_plain = r
        y_plain = y_plain.cpu().numpy()
        out["plain"].update(iterations=int(rep.iterations), converged=bool(rep.converged))
        for label, kw in (("warm_coarse_solve", dict(use_net=False, phase1_max_iter=0)),
                          ("warm_coarse_solve_net_phase", dict(use_net=True))):
            r2 = run(label, lambda y: sw.iterate_warm(net if kw["use_net"] else None, nH, case.chem, srcs, y,
                                                      tol=tol, max_iter=400, **kw))
            if r2:
                (wr, _), y = r2
                out[label].update(iterations=int(wr.total.iterations), coarse_iterations=int(wr.coarse_iterations),
                                  surrogate_iterations=int(wr.surrogate_iterations),
                                  full_sweeps=int(wr.plain_sweeps), judge_error=round(float(wr.judge_error), 5),
                                  converged=bool(wr.total.converged),
                                  speedup_vs_plain=round(out["plain"]["seconds"] / out[label]["seconds"], 3),
                                  max_rel_dy_vs_plain=float(np.max(np.abs(y.cpu().numpy() - y_plain) / y_plain)))
        # over-relaxed balance update (not in the paper; omega = 1.3), plain and after the coarse solve
        sw.set_relaxation(1.3)
        for label, fn in (("plain_relaxed_1.3", lambda y: sw.iterate(nH, case.chem, srcs, y, tol=tol, max_iter=400)),
                          ("warm_coarse_solve_relaxed_1.3",
                           lambda y: sw.iterate_warm(None, nH, case.chem, srcs, y, tol=tol, max_iter=400,
                                                     use_net=False, phase1_max_iter=0))):
            r2 = run(label, fn)
            if r2:
                res, y = r2
                rep = res[0].total if label.startswith("warm") else res[0]
                out[label].update(iterations=int(rep.iterations), converged=bool(rep.converged),
                                  speedup_vs_plain=round(out["plain"]["seconds"] / out[label]["seconds"], 3),
                                  max_rel_dy_vs_plain=float(np.max(np.abs(y.cpu().numpy() - y_plain) / y_plain)))
        sw.set_relaxation(1.0)
    sw.close()
    return out


def shadow_measure(torch, dev, tol=1e-6):
    """The geometry of the paper's Test 3 at 128^3, N_side 8: uniform n_H 2e-4
    with a clump of 200x density (radius 0.8 kpc, 1.7 kpc from the centre along
    x), lit by a plane-parallel flux of 1e6 photons/s/cm^2 through the x = 0
    face over 4 blackbody (1e5 K) bins; equilibrium solve at 1e4 K with the
    diffuse field and on the spot.  Reports the neutral fraction on the clump's
    axis just behind it and at the same depth off the shadow."""
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    case = wl.shadow_clump()
    frac, sig, _ = wl.blackbody_bins()
    n = case.n
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    sw.set_source_spectrum(sig, frac)
    sw.set_plane_source(*case.plane)
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device=dev)
    out = {"workload": "128^3 Test-3 geometry: n_H 2e-4, clump x200 (r 0.8 kpc, 1.7 kpc off centre along x), "
                       "plane-parallel flux 1e6 s^-1 cm^-2 through x = 0, 4 blackbody bins, N_side 8, 1e4 K",
           "tol": tol}
    mid = n // 2
    behind = (mid, mid, n - 2)          # (z, y, x): on the clump's axis, behind it
    beside = (mid, n // 8, n - 2)       # same depth, outside the shadow
    for label, chem in (("with_diffuse", case.chem), ("on_the_spot", dict(case.chem, alphaA=case.chem["alphaB"]))):
        y = torch.as_tensor(case.y0, dtype=torch.float64, device=dev).clone()
        sw.iterate(nH, chem, [], y, tol=tol, max_iter=400)       # first-call allocations
        y = torch.as_tensor(case.y0, dtype=torch.float64, device=dev).clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep, _ = sw.iterate(nH, chem, [], y, tol=tol, max_iter=400)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        yh = y.cpu().numpy()
        out[label] = {"iterations": int(rep.iterations), "seconds": round(dt, 4), "converged": bool(rep.converged),
                      "neutral_fraction_behind_clump": float(yh[behind]),
                      "neutral_fraction_beside_shadow": float(yh[beside]),
                      "mean_neutral_fraction": float(np.mean(yh))}
    sw.close()
    return out


def evolve_measure(torch, dev, F=1.0):
    """Time-dependent mode on the paper's Test-1 setup at 64^3, N_side 4: n_H
    1e-3, Q 5e48 s^-1 at a corner of a 6.6 kpc box, from x = 1e-4 to the
    paper's 30, 100 and 500 Myr, with the diffuse field and on the spot, at
    1e4 K (no energy equation).  Reports steps, iterations, sweeps, wall time
    and the ionized-volume radius against the on-the-spot Stromgren growth
    R_S (1 - e^{-t/t_rec})^{1/3}."""
    import math
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    nH0, Q = 1e-3, 5e48
    case = wl.hii_region(n=64, nside=4, box_kpc=6.6, nH=nH0, Q=Q, source_at="corner")
    aB, dx = case.chem["alphaB"], case.chem["dx"]
    t_rec = 1.0 / (aB * nH0)
    rs = (3 * Q / (4 * math.pi * nH0 * nH0 * aB)) ** (1 / 3)
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=dx)
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device=dev)
    out = {"workload": "Test-1 setup, 64^3, N_side 4: n_H 1e-3, Q 5e48 s^-1 at a corner, 6.6 kpc, 1e4 K, "
                       f"F = {F}, eps_iter 1e-3", "t_rec_myr": round(t_rec / wl.MYR, 2),
           "r_s_kpc": round(rs / wl.KPC, 3)}
    for label, chem in (("with_diffuse", case.chem), ("on_the_spot", dict(case.chem, alphaA=aB))):
        y = torch.as_tensor(case.y0, dtype=torch.float64, device=dev).clone()
        t, rows, tot = 0.0, [], {"steps": 0, "iterations": 0, "sweeps": 0, "seconds": 0.0}
        for t_myr in (30.0, 100.0, 500.0):
            rep = sw.evolve(nH, chem, srcs, y, t_myr * wl.MYR - t, F=F)
            t = t_myr * wl.MYR
            for k in ("steps", "iterations", "sweeps"):
                tot[k] += int(getattr(rep, k))
            tot["seconds"] += float(rep.seconds)
            vol = 8 * float(torch.sum(1 - y)) * dx ** 3
            r = (3 * vol / (4 * math.pi)) ** (1 / 3)
            rows.append({"t_myr": t_myr, "r_ion_over_r_s": round(r / rs, 4),
                         "stromgren_growth": round((1 - math.exp(-t / t_rec)) ** (1 / 3), 4)})
        out[label] = dict(tot, seconds=round(tot["seconds"], 3), radius=rows)
    sw.close()
    return out


def thermal_measure(torch, dev, F=1.0):
    """Time-dependent mode with the energy equation (App. C) on the paper's
    Test-1 setup as printed (Sec. 4.1): n_H 1e-3, initial T 100 K, a 1e5 K
    blackbody source of 5e48 photons/s (4 bins above 13.6 eV) at a corner of a
    6.6 kpc box, here 64^3 and N_side 4, to 30, 100 and 500 Myr, with the
    diffuse field and on the spot.  Reports steps, iterations, sweeps, wall
    time, the ionized-volume radius over R_S and the mean temperature of the
    ionized gas."""
    import math
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    nH0, Q = 1e-3, 5e48
    case = wl.hii_region(n=64, nside=4, box_kpc=6.6, nH=nH0, Q=Q, source_at="corner")
    frac, sig, _ = wl.blackbody_bins()
    dx = case.chem["dx"]
    rs = 5.4 * wl.KPC                          # the paper's printed Stromgren radius
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=dx)
    sw.set_source_spectrum(sig, frac)
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device=dev)
    th = {"e_bin": list(wl.blackbody_heat()), "e_diff": wl.diffuse_band_heat(case.chem)}
    out = {"workload": "Test-1 setup with the energy equation, 64^3, N_side 4: n_H 1e-3, T0 100 K, 1e5 K "
                       f"blackbody (4 bins) 5e48 s^-1 at a corner, 6.6 kpc, F = {F}, eps_iter 1e-3"}
    for label, otsa in (("with_diffuse", 0), ("on_the_spot", 1)):
        y = torch.as_tensor(case.y0, dtype=torch.float64, device=dev).clone()
        T = torch.full_like(y, 100.0)
        t, rows, tot = 0.0, [], {"steps": 0, "iterations": 0, "sweeps": 0, "seconds": 0.0}
        for t_myr in (30.0, 100.0, 500.0):
            rep = sw.evolve_thermal(nH, case.chem, dict(th, on_the_spot=otsa), srcs, y, T, t_myr * wl.MYR - t, F=F)
            t = t_myr * wl.MYR
            for k in ("steps", "iterations", "sweeps"):
                tot[k] += int(getattr(rep, k))
            tot["seconds"] += float(rep.seconds)
            x = 1 - y
            vol = 8 * float(torch.sum(x)) * dx ** 3
            r = (3 * vol / (4 * math.pi)) ** (1 / 3)
            rows.append({"t_myr": t_myr, "r_ion_over_r_s": round(r / rs, 4),
                         "mean_T_ionized_K": round(float(torch.sum(T * x) / torch.sum(x)), 1),
                         "max_T_K": round(float(T.max()), 1)})
        out[label] = dict(tot, seconds=round(tot["seconds"], 3), radius=rows)
    sw.close()
    return out


def test3_thermal_measure(torch, dev, n=64, nside=4, F=1.0):
    """The paper's Test 3 as printed (Sec. 4.3), with the energy equation:
    n_H 2e-4 at 8000 K, a clump of 200x density at 40 K (radius 0.8 kpc, 1.7
    kpc from the centre along x), a 1e5 K blackbody flux of 1e6 photons/s/cm^2
    (4 bins) through the x = 0 face, to the paper's 1, 3 and 15 Myr, with the
    diffuse field and on the spot.  Reports steps, iterations, wall time and y
    and T at the clump's centre, behind it on its axis, and at the same depth
    off the shadow."""
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    case = wl.shadow_clump(n=n, nside=nside)
    frac, sig, _ = wl.blackbody_bins()
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    sw.set_source_spectrum(sig, frac)
    sw.set_plane_source(*case.plane)
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device=dev)
    clump = case.nH > 1.5 * case.nH.min()
    T0 = np.where(clump, 40.0, 8000.0)
    th = {"e_bin": list(wl.blackbody_heat()), "e_diff": wl.diffuse_band_heat(case.chem)}
    mid = n // 2
    cz, cy, cx = [int(round(v)) for v in np.mean(np.argwhere(clump), axis=0)]
    cells = {"clump_centre": (cz, cy, cx), "behind_clump": (mid, mid, n - 2), "beside_shadow": (mid, n // 8, n - 2)}
    out = {"workload": f"Test 3 as printed with the energy equation, {n}^3, N_side {nside}: n_H 2e-4 at 8000 K, "
                       "clump x200 at 40 K (r 0.8 kpc, 1.7 kpc off centre along x), 1e5 K blackbody flux 1e6 s^-1 "
                       f"cm^-2 through x = 0 (4 bins), F = {F}, eps_iter 1e-3"}
    for label, otsa in (("with_diffuse", 0), ("on_the_spot", 1)):
        y = torch.as_tensor(case.y0, dtype=torch.float64, device=dev).clone()
        T = torch.as_tensor(T0, dtype=torch.float64, device=dev).clone()
        t, rows, tot = 0.0, [], {"steps": 0, "iterations": 0, "sweeps": 0, "seconds": 0.0}
        for t_myr in (1.0, 3.0, 15.0):
            rep = sw.evolve_thermal(nH, case.chem, dict(th, on_the_spot=otsa), [], y, T, t_myr * wl.MYR - t, F=F)
            t = t_myr * wl.MYR
            for k in ("steps", "iterations", "sweeps"):
                tot[k] += int(getattr(rep, k))
            tot["seconds"] += float(rep.seconds)
            yh, Th = y.cpu().numpy(), T.cpu().numpy()
            rows.append({"t_myr": t_myr, **{f"y_{k}": float(yh[c]) for k, c in cells.items()},
                         **{f"T_{k}_K": round(float(Th[c]), 1) for k, c in cells.items()}})
        out[label] = dict(tot, seconds=round(tot["seconds"], 3), at=rows)
    sw.close()
    return out


def test2_thermal_measure(torch, dev, n=64, nside=4, F=0.25):
    """The paper's Test 2 as printed (Sec. 4.2), with the energy equation: a
    1e5 K blackbody point source of 5e48 photons/s (4 bins) at the centre of
    the 6.6 kpc box, n_H 1e-3 at 100 K, a clump of 200x density at 100 K
    (radius 0.56 kpc, 0.8 kpc from the source along x), to 30, 100 and 500
    Myr, with the diffuse field and on the spot.  Reports steps, iterations,
    wall time and y and T at the clump's centre, in its shadow on the axis
    (halfway from its far side to the box face) and at the same distance from
    the source off the shadow."""
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    case = wl.point_clump(n=n, nside=nside)
    frac, sig, _ = wl.blackbody_bins()
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    sw.set_source_spectrum(sig, frac)
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device=dev)
    th = {"e_bin": list(wl.blackbody_heat()), "e_diff": wl.diffuse_band_heat(case.chem)}
    dx_kpc = 6.6 / n
    mid = n // 2
    far = int(round((0.8 + 0.56) / dx_kpc))                  # cells from the source to the clump's far side
    sh = min(n - 1, mid + (far + (n - mid)) // 2)            # halfway to the +x face
    d = sh - mid
    cells = {"clump_centre": (mid, mid, mid + int(round(0.8 / dx_kpc))), "shadow": (mid, mid, sh),
             "off_shadow": (mid, mid + d, mid)}
    # the shadow cone: cells behind the clump (farther along x than its far side) whose direction
    # from the source passes through it (half-angle asin(0.56 / 0.8))
    g = np.arange(n) + 0.5 - n / 2
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    rr = np.sqrt(xx * xx + yy * yy + zz * zz)
    cone = (xx > (0.8 + 0.56) / dx_kpc) & (xx / np.maximum(rr, 1e-9) > np.cos(np.arcsin(0.56 / 0.8)))
    out = {"workload": f"Test 2 as printed with the energy equation, {n}^3, N_side {nside}: 1e5 K blackbody point "
                       "source 5e48 s^-1 (4 bins) at the centre, n_H 1e-3 at 100 K, clump x200 at 100 K (r 0.56 kpc, "
                       f"0.8 kpc from the source along x), 6.6 kpc, F = {F}, eps_iter 1e-3"}
    for label, otsa in (("with_diffuse", 0), ("on_the_spot", 1)):
        y = torch.as_tensor(case.y0, dtype=torch.float64, device=dev).clone()
        T = torch.full_like(y, 100.0)
        t, rows, tot = 0.0, [], {"steps": 0, "iterations": 0, "sweeps": 0, "seconds": 0.0}
        for t_myr in (30.0, 100.0, 500.0):
            # at F = 1 and 0.5 some RT steps of this setup do not converge (App. D's
            # iteration stalls; the oracle's too, at 32^3); F = 0.25 takes 3-5 per step
            rep = sw.evolve_thermal(nH, case.chem, dict(th, on_the_spot=otsa), srcs, y, T, t_myr * wl.MYR - t, F=F,
                                    max_iter=300)
            t = t_myr * wl.MYR
            for k in ("steps", "iterations", "sweeps"):
                tot[k] += int(getattr(rep, k))
            tot["seconds"] += float(rep.seconds)
            yh, Th = y.cpu().numpy(), T.cpu().numpy()
            rows.append({"t_myr": t_myr, **{f"y_{k}": float(yh[c]) for k, c in cells.items()},
                         **{f"T_{k}_K": round(float(Th[c]), 1) for k, c in cells.items()},
                         "shadow_cone_neutral_fraction": round(float(yh[cone].mean()), 4)})
        out[label] = dict(tot, seconds=round(tot["seconds"], 3), at=rows)
    out["shadow_cone_cells"] = int(cone.sum())
    sw.close()
    return out


def test2_resolution_measure(torch, dev, n=64, F=0.25, nsides=(1, 2, 4, 8)):
    """The angular-resolution study of the paper's Test 2 (Sec. 4.2): the
    setup of test2_thermal_measure with the diffuse field, to 30 Myr, at
    several N_side.  Reports, per N_side, the mean and the maximum over cells
    of |y - y_ref| and |T - T_ref| / T_ref against the finest N_side."""
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    frac, sig, _ = wl.blackbody_bins()
    res = {}
    for ns in nsides:
        case = wl.point_clump(n=n, nside=ns)
        srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
        sw = art.ArtSweep(case.nH.shape, ns, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
        sw.set_source_spectrum(sig, frac)
        th = {"e_bin": list(wl.blackbody_heat()), "e_diff": wl.diffuse_band_heat(case.chem)}
        y = torch.as_tensor(case.y0, dtype=torch.float64, device=dev).clone()
        T = torch.full_like(y, 100.0)
        rep = sw.evolve_thermal(torch.as_tensor(case.nH, dtype=torch.float64, device=dev), case.chem, th, srcs, y, T,
                                30.0 * wl.MYR, F=F, max_iter=300)
        res[ns] = (y.cpu().numpy(), T.cpu().numpy(), float(rep.seconds), int(rep.iterations))
        sw.close()
    yr, Tr = res[nsides[-1]][0], res[nsides[-1]][1]
    out = {"workload": f"Test 2 with the energy equation and the diffuse field, {n}^3, to 30 Myr, F = {F}; "
                       f"differences against N_side {nsides[-1]}"}
    for ns in nsides:
        yh, Th, sec, it = res[ns]
        out[f"nside_{ns}"] = {"directions": 12 * ns * ns, "seconds": round(sec, 3), "iterations": it,
                              "mean_abs_dy": float(np.mean(np.abs(yh - yr))), "max_abs_dy": float(np.max(np.abs(yh - yr))),
                              "mean_rel_dT": float(np.mean(np.abs(Th - Tr) / Tr))}
    return out


def ablation_measure(torch, dev, reps=3):
    """The paper's ray-grouping comparison (Sec. 5) restated on GB300: the
    thread-per-ray layout of Sec. 3.1 with float atomics against the same
    layout with the four ray groups, both CUDA-graph replays of one launch
    (atomics) or four (groups) per direction, and the production tiled sweep,
    on the GRF workloads.  Milliseconds per sweep, best of reps after a
    warm-up."""
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import workloads as wl
    out = {"note": "benchmark only; the paper reports grouping > 2x faster than atomics on its GPUs"}
    for name, n, nside in (("grf64", 64, 4), ("grf128", 128, 8)):
        c = wl.grf(n, nside)
        k = torch.as_tensor(c.kappa, dtype=torch.float32, device=dev)
        s = torch.as_tensor(c.src, dtype=torch.float32, device=dev)
        sw = art.ArtSweep(k.shape, nside, 1, graph=True, variant=1)   # the slab-block tables it marches
        sw.set_fields(k, s)
        j = torch.empty_like(k)

        def best(fn):
            fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return min(ts)
        t_atomic = best(lambda: sw.ablation_sweep(0, j))
        t_group = best(lambda: sw.ablation_sweep(1, j))
        t_tiled = best(lambda: sw.sweep(J_in=j))
        segs = sw.stats.segments
        out[name] = {"ms_atomic": round(t_atomic, 3), "ms_ray_groups": round(t_group, 3),
                     "ms_tiled_sweep": round(t_tiled, 3), "groups_over_atomic_speedup": round(t_atomic / t_group, 3),
                     "tiled_over_groups_speedup": round(t_group / t_tiled, 3),
                     "gseg_per_s": {"atomic": round(segs / t_atomic / 1e6, 1), "ray_groups": round(segs / t_group / 1e6, 1),
                                    "tiled": round(segs / t_tiled / 1e6, 1)}}
        sw.close()
    return out


def cpu_baseline(case, seg_per_step: int, budget_s: float = 12.0) -> dict:
    """The FP64 oracle on the host cores: as many full sweeps of the workload as fit in budget_s
    when one takes less than that; else a bounded sample of directions (the oracle's cost is per
    segment, so segments per second carry over to the whole step)."""
    import oracle
    oracle.build()
    nt = oracle.default_threads()
    kap = case.kappa.astype(np.float32).astype(np.float64)
    src = case.src.astype(np.float32).astype(np.float64)
    k, s_ = (kap, src) if kap.ndim == 3 else (kap[0], src[0])
    nd = 12 * case.nside * case.nside
    # directions per chunk so that one chunk takes about a second
    t0 = time.perf_counter()
    oracle.sweep_range_count(k, s_, case.nside, 0, min(nd, nt), nthreads=nt)
    per_dir = (time.perf_counter() - t0) / min(nd, nt)
    chunk = int(max(1, min(nd, 1.0 / max(per_dir, 1e-9))))
    t0 = time.perf_counter()
    segs, d0 = 0, 0
    while True:
        d1 = min(nd, d0 + chunk)
        _, n = oracle.sweep_range_count(k, s_, case.nside, d0, d1, nthreads=nt)
        segs += n
        d0 = d1 % nd
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    d1 = max(1, nd // 64)
    t1 = time.perf_counter()
    segs1 = 0
    while True:
        _, n1 = oracle.sweep_range_count(k, s_, case.nside, 0, d1, nthreads=1)
        segs1 += n1
        if time.perf_counter() - t1 > budget_s / 4:
            break
    dt1 = time.perf_counter() - t1
    return {"value": segs / dt, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"bin 0 of the workload, {segs} segments in chunks of {chunk} of its {nd} directions "
                      f"({dt:.1f} s, FP64 oracle, OpenMP over directions); one step is {seg_per_step} segments",
            "single_core": {"value": segs1 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"directions 0-{d1 - 1} of bin 0 repeated ({segs1} segments, {dt1:.1f} s)"}}


def run_shard(args, d: Dist):
    """The workload's sweep with its directions split over the ranks (Sec. 3.2): each step is this
    rank's share (its RING-index block, all bins) and the rank-ordered reduce-scatter + all-gather
    that gives every rank J^in.  Strong scaling: the total work is fixed."""
    import torch
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import build as libbuild
    from paper_1410_0763_gb300 import dist as adist
    dev = torch.device("cuda", d.local)
    torch.cuda.set_device(dev)
    if d.rank == 0:
        libbuild.build()
    d.barrier()
    art.load()
    case = make_case(args.workload, 0)          # the same grid on every rank
    nb = case_bins(case)
    k = torch.as_tensor(case.kappa, dtype=torch.float32, device=dev)
    s = torch.as_tensor(case.src, dtype=torch.float32, device=dev)
    sh = adist.ShardedSweep(case.shape, case.nside, nb, group=None)
    sh.set_fields(k, s)
    seg_total = int(art.art_count_segments(case.shape, case.nside)) * nb
    part = torch.empty_like(k)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        jin = sh.jin(sh.share(part))
    torch.cuda.synchronize()
    if sh.check() != art.ART_OK:
        raise RuntimeError("sweep reported an error")
    clocks = ClockSampler(d.local)
    clocks.start()
    d.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        jin = sh.jin(sh.share(part))
        b.record(stream)
    torch.cuda.synchronize()
    d.barrier()
    ck = clocks.stop()
    total_ms = d.max(sum(a.elapsed_time(b) for a, b in evs), dev)
    st = sh.sw.stats if sh.sw is not None else None
    # per step: the sweep launches (one per bins_per_launch bins), one reduction per bin, the
    # rank-ordered sum of the exchanged blocks
    launches = (nb // max(1, int(st.bins_per_launch)) + nb + 1) if st is not None else 1
    sh.close()
    out = {
        "metric": METRIC, "value": seg_total * args.steps / (total_ms * 1e-3), "unit": UNIT, "n_gpus": d.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "n": int(case.shape[0]), "nside": case.nside,
                   "bins": nb, "segments_per_step": seg_total,
                   "parallelism": f"directions split over {d.world} ranks; rank-ordered reduce-scatter "
                                  f"(point-to-point) + all-gather of J^in"},
        "clocks": ck,
        "gpu_launches": int(args.steps * launches),
    }
    if d.rank == 0:
        print(json.dumps(out), flush=True)


def run_ours(args, d: Dist):
    import torch
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import build as libbuild

    dev = torch.device("cuda", d.local)
    torch.cuda.set_device(dev)
    if d.rank == 0:
        libbuild.build()
    d.barrier()
    art.load()
    case = make_case(args.workload, d.rank)
    nb = case_bins(case)
    k = torch.as_tensor(case.kappa, dtype=torch.float32, device=dev)
    s = torch.as_tensor(case.src, dtype=torch.float32, device=dev)
    sw = art.ArtSweep(case.shape, case.nside, nb, graph=not args.no_graph)
    sw.set_fields(k, s)
    sw.set_band(band_G(nb))
    t0 = time.perf_counter()
    if not args.no_autotune:
        sw.autotune(1)          # untimed: the library's own variant / launch-form choice
    tune_s = time.perf_counter() - t0
    st = sw.stats
    seg = int(st.segments)       # all bins
    J, Jin = torch.empty_like(k), torch.empty_like(k)
    gam = torch.empty(case.shape, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    clocks = ClockSampler(d.local)
    clocks.start()
    for _ in range(args.warmup):
        sw.sweep(J, Jin, gam)
    torch.cuda.synchronize()
    if sw.check() != art.ART_OK:
        raise RuntimeError("sweep reported an error: " + art.art_last_error(sw._ctx))
    d.barrier()
    torch.cuda.synchronize()
    ms = time_device(sw, J, Jin, gam, args.steps, flush, torch)
    torch.cuda.synchronize()
    d.barrier()
    ck = clocks.stop()
    if sw.check() != art.ART_OK:
        raise RuntimeError("sweep reported an error: " + art.art_last_error(sw._ctx))
    total_ms = d.max(sum(ms), dev)
    value = seg * d.world * args.steps / (total_ms * 1e-3)

    # kernel-level roofline: the same steps with per-kernel events inside the library
    # (events around each bin's sweep launch and around its reduction)
    prof_steps = min(args.steps, 50)
    sw.profile(True)
    time_device(sw, J, Jin, gam, prof_steps, flush, torch)
    sw.profile(False)
    pr = sw.profile_read()
    # algorithmic segments per sweep launch / average launch duration
    achieved_gseg = seg * prof_steps / (pr.sweep_ms * 1e-3) / 1e9
    sm_mhz = ck["sm_mhz"] or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    try:
        pipes = art.art_measure_pipes()
        ex2 = round(pipes["ex2"])
        # the FMA pipe's capacity: the faster of scalar and packed FP32x2 issue
        ffma = round(max(pipes["ffma"], pipes["ffma2"]))
    except Exception:  # pragma: no cover
        pipes, ex2, ffma = None, EX2_PER_CLK_SM, FFMA_PER_CLK_SM
    # two roofs for the algorithmic work of one segment (Eq. rt and the
    # path-averaged deposit): one exponential on the MUFU pipe, and
    # FP32_OPS_PER_SEG FP32 operations on the FMA pipe; the lower one binds
    peak_mufu = ex2 * n_sm * sm_mhz * 1e6 / 1e9
    peak_fp32 = ffma / FP32_OPS_PER_SEG * n_sm * sm_mhz * 1e6 / 1e9
    peak_gseg = min(peak_mufu, peak_fp32)
    sweep_share = pr.sweep_ms / max(pr.sweep_ms + pr.reduce_ms, 1e-9)
    # the DRAM side of the same kernel: recorded ncu bytes per launch over the live launch time
    traffic = recorded_traffic(args.workload, int(st.variant), int(st.persistent))
    launches_per_step = max(1, nb // max(1, int(st.bins_per_launch))) if st.variant >= 16 else st.launches - 1
    launch_ms = pr.sweep_ms / (prof_steps * max(1, launches_per_step))
    hbm = measured_hbm_gbs()
    dram_gbs = traffic / (launch_ms * 1e-3) / 1e9 if traffic else None
    wave = st.variant >= 16
    kname = "wave_kernel" if wave else ("sweep_queue_kernel" if st.persistent else "sweep_block_kernel")

    # end to end through the C ABI with host buffers (pinned): every step copies its kappa and
    # S in and its J out.  art_sweep_stream overlaps those copies with the neighbouring steps'
    # sweeps; the per-call form (art_set_fields + art_sweep, each synchronous) is reported beside it.
    kh = torch.as_tensor(case.kappa.astype(np.float32)).pin_memory()
    sh = torch.as_tensor(case.src.astype(np.float32)).pin_memory()
    Jh = [torch.empty(k.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    e2e_steps = max(3, min(args.steps, 50))
    sw.sweep_stream([kh] * 2, [sh] * 2, J=[Jh[i % 2] for i in range(2)])
    torch.cuda.synchronize()
    d.barrier()
    t0 = time.perf_counter()
    sw.sweep_stream([kh] * e2e_steps, [sh] * e2e_steps, J=[Jh[i % 2] for i in range(e2e_steps)])
    torch.cuda.synchronize()
    dt = d.max(time.perf_counter() - t0, dev)
    e2e = {"value": seg * d.world * e2e_steps / dt, "unit": UNIT,
           "h2d_bytes_per_step": int(2 * kh.numel() * 4), "d2h_bytes_per_step": int(Jh[0].numel() * 4),
           "api": "art_sweep_stream (copies overlap the neighbouring steps' sweeps)"}
    pc_steps = max(2, min(e2e_steps, 10))
    sw.set_fields(kh, sh)
    sw.sweep(Jh[0])
    torch.cuda.synchronize()
    d.barrier()
    t0 = time.perf_counter()
    for _ in range(pc_steps):
        sw.set_fields(kh, sh)
        sw.sweep(Jh[0])
    torch.cuda.synchronize()
    dt = d.max(time.perf_counter() - t0, dev)
    e2e["per_call"] = {"value": seg * d.world * pc_steps / dt, "unit": UNIT,
                       "api": "art_set_fields + art_sweep per step (each returns synchronized)"}
    sw.close()

    extra = {}
    if d.rank == 0 and d.world == 1 and not args.no_extra:
        for name in ("grf64", "grf128", "grf256"):
            if name != args.workload:
                try:
                    extra[name] = side_measure(name, torch, dev)
                except Exception as ex:  # pragma: no cover
                    extra[name] = {"error": str(ex)}
        try:
            extra["batch48"] = batch_measure(torch, dev)
        except Exception as ex:  # pragma: no cover
            extra["batch48"] = {"error": str(ex)}
        try:
            extra["rt_ionization_128"], extra["rt_ionization_256_clumpy"] = ionization_measure(torch, dev)
        except Exception as ex:  # pragma: no cover
            extra["rt_ionization_128"] = {"error": str(ex)}
        if args.paper_tests:
            try:
                extra["rt_ionization_128_plane_flux"] = shadow_measure(torch, dev)
            except Exception as ex:  # pragma: no cover
                extra["rt_ionization_128_plane_flux"] = {"error": str(ex)}
            for key, fn in (("time_dependent_64", evolve_measure), ("time_dependent_thermal_64", thermal_measure),
                            ("test3_thermal_64", test3_thermal_measure), ("test2_thermal_64", test2_thermal_measure),
                            ("test2_angular_resolution_64", test2_resolution_measure)):
                try:
                    extra[key] = fn(torch, dev)
                except Exception as ex:  # pragma: no cover
                    extra[key] = {"error": str(ex)}
            try:
                extra["ablation_ray_grouping"] = ablation_measure(torch, dev)
            except Exception as ex:  # pragma: no cover
                extra["ablation_ray_grouping"] = {"error": str(ex)}

    cpu = None
    if d.rank == 0 and d.world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(case, seg)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": d.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "n": int(case.shape[0]),
                   "nside": case.nside, "bins": nb, "segments_per_step": seg,
                   "kernel": (f"wavefront sweep, CTA tile {st.tile_b}x{st.tile_c} columns, "
                              f"{st.group} direction slots, {st.ctas_per_launch} units per bin, "
                              f"{st.bins_per_launch} bin(s) per launch"
                              if wave else
                              f"slab-block sweep, tile {st.tile_b}x{st.tile_c}, slab {st.slab}, "
                              f"dir groups {st.dir_split}, {st.ctas_per_launch} CTAs x {st.launches - 1} launches"),
                   "variant": int(st.variant), "autotune_s": round(tune_s, 2),
                   "l2": "inputs larger than L2; L2 also flushed between timed steps (256 MiB write)",
                   "parallelism": f"weak x{d.world} (independent grid per GPU)"},
        "roofline": {"bound": "alu", "achieved": achieved_gseg, "peak": peak_gseg, "unit": "Gseg/s",
                     "frac": achieved_gseg / peak_gseg,
                     "traffic": traffic,
                     "traffic_unit": "DRAM bytes per sweep launch (ncu)",
                     "dram_gbs": dram_gbs, "hbm_frac": dram_gbs / hbm if dram_gbs else None,
                     "hbm_peak_gbs": hbm, "binding": "FP32 pipe" if peak_fp32 <= peak_mufu else "MUFU",
                     "kernel": f"{kname} variant {st.variant} (tile {st.tile_b}x{st.tile_c})",
                     "kernel_share_of_step": sweep_share,
                     "peak_basis": f"binding roof = min(FP32: {ffma}/clk/SM (measured FMAs, scalar or packed FP32x2) / "
                                   f"{FP32_OPS_PER_SEG} ops per segment = {peak_fp32:.0f} Gseg/s, "
                                   f"MUFU: 1 ex2 per segment x {ex2}/clk/SM (measured) = {peak_mufu:.0f} Gseg/s), "
                                   f"x {n_sm} SMs x {sm_mhz:.0f} MHz (median SM clock under load)",
                     "peak_fp32_gseg": peak_fp32, "peak_mufu_gseg": peak_mufu,
                     "pipes_per_clk_sm": pipes},
        "e2e": e2e,
        # per step: one reduction per bin, one sweep launch per bins_per_launch bins
        "gpu_launches": int(args.steps * (nb + (st.launches - 1) * nb // max(1, int(st.bins_per_launch)))),
        "clocks": ck,
        "cpu_baseline": cpu,
    }
    if extra:
        out["extra"] = extra
    if d.rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, d: Dist):
    if d.rank != 0:
        return
    import oracle
    oracle.build()
    case = make_case(args.workload, 0)
    nb = case_bins(case)
    nt = oracle.default_threads()
    kap = case.kappa.astype(np.float32).astype(np.float64)
    src = case.src.astype(np.float32).astype(np.float64)
    nd = 12 * case.nside * case.nside
    # each step: a block of directions of one bin (bins in turn), sized so that warmup + steps
    # fit in about 2.5 minutes; the oracle's cost is per segment
    k0, s0 = (kap, src) if nb == 1 else (kap[0], src[0])
    t0 = time.perf_counter()
    oracle.sweep_range_count(k0, s0, case.nside, 0, min(nd, nt), nthreads=nt)
    per_dir = (time.perf_counter() - t0) / min(nd, nt)
    budget = 150.0 / max(args.steps + args.warmup, 1)
    ndir = int(max(1, min(nd, budget / max(per_dir, 1e-9))))
    pos = 0
    segs, tsum = 0, 0.0
    for i in range(args.warmup + args.steps):
        b = i % nb
        kb, sb = (kap, src) if nb == 1 else (kap[b], src[b])
        d0 = pos % nd
        d1 = min(nd, d0 + ndir)
        pos = d1
        t0 = time.perf_counter()
        _, n = oracle.sweep_range_count(kb, sb, case.nside, d0, d1, nthreads=nt)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            segs += n
            tsum += dt
    value = segs / tsum
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": d.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tsum / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "n": int(case.shape[0]),
                   "nside": case.nside, "bins": nb},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                         "sample": f"each step: {ndir} of the {nd} directions of one bin of the workload "
                                   f"(bins in turn; FP64 oracle)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# small cases for a profiler (ncu): one JSON line each, no benchmark line
# ---------------------------------------------------------------------------
def profile_case(args):
    import torch
    from paper_1410_0763_gb300 import art
    from paper_1410_0763_gb300 import build as libbuild
    from paper_1410_0763_gb300 import workloads as wl
    libbuild.build()
    art.load()
    out = {"profile_case": args.profile_case}
    if args.profile_case == "sweep":
        # a few sweeps of one workload: the GRF recipe at n^3 and N_side (one bin), or with
        # --workload given explicitly, that benchmark workload (all its bins; the clumpy medium at
        # n^3 when --n is given too, with the full workload's optical depth per cell); the kernel
        # variant given
        if "--workload" in sys.argv:
            w = WORKLOADS[args.workload]
            if args.n and w.get("kind") == "clumpy":
                c = wl.clumpy_sweep(args.n, args.nside or w["nside"], seed=w["seed"], nbins=w["bins"],
                                    tau_box=10.0 * args.n / w["n"])
            else:
                c = make_case(args.workload, 0)
            n, nside, nb = c.shape[-1], c.nside, case_bins(c)
        else:
            n, nside, nb = args.n or 128, args.nside or 8, 1
            c = wl.grf(n, nside, seed=3)
        kap, src = c.kappa, c.src
        if args.bin is not None and nb > 1:   # one bin of a multi-bin workload
            kap, src, nb = kap[args.bin], src[args.bin], 1
        k = torch.as_tensor(kap.astype(np.float32), device="cuda")
        s = torch.as_tensor(src.astype(np.float32), device="cuda")
        sw = art.ArtSweep(c.shape, nside, nb, variant=args.variant)
        sw.set_fields(k, s)
        Jin = torch.empty_like(k)
        for _ in range(args.reps):
            sw.sweep(None, Jin)
        torch.cuda.synchronize()
        if sw.check() != art.ART_OK:
            raise RuntimeError("sweep reported an error")
        st = sw.stats
        out.update(n=n, nside=nside, bins=nb, variant=int(st.variant), units=int(st.ctas_per_launch),
                   segments=int(st.segments))
        if int(st.variant) >= 16:
            cnt = sw.wave_counters()   # nonzero in ART_WAVE_STATS builds only
            if cnt["unit_cycles"]:
                out.update(barrier_fraction=round(cnt["barrier_cycles"] / cnt["unit_cycles"], 4),
                           poll_fraction=round(cnt["poll_cycles"] / cnt["unit_cycles"], 4),
                           polls=cnt["polls"])
        sw.close()
    elif args.profile_case == "net":
        # the surrogate network on one grid: forward passes (and training steps)
        n = args.n or 128
        V = n ** 3
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
        for _ in range(args.reps):
            net.forward(X, o, shape)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.reps
        flops = 2.0 * 27 * V * (4 * 32 + 32 * 32 * 2 + 32 * 1)
        out.update(n=n, forward_ms=round(ms, 4), forward_tflops_algorithmic=round(flops / ms / 1e9, 1))
        if args.train:
            for _ in range(2):
                net.train_step(X, t, shape, want_loss=False)
            e0.record()
            for _ in range(args.reps):
                net.train_step(X, t, shape, want_loss=False)
            e1.record()
            torch.cuda.synchronize()
            out["train_step_ms"] = round(e0.elapsed_time(e1) / args.reps, 4)
        net.close()
    elif args.profile_case in ("hii", "clumpy"):
        # point-source rates and RT / ionization-balance iterations
        case = wl.hii_region() if args.profile_case == "hii" else wl.clumpy()
        srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
        sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
        if args.profile_case == "clumpy":
            frac, sig, _ = wl.blackbody_bins()
            sw.set_source_spectrum(sig, frac)
        V = case.n ** 3
        kap = torch.as_tensor((case.y0 * case.nH * case.chem["sigma0"] * case.chem["dx"]).ravel(),
                              dtype=torch.float32, device="cuda")
        g = torch.empty(V, device="cuda")
        for _ in range(2):
            sw.point_sources(kap, [case.chem["sigma0"]], srcs, g)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.reps):
            sw.point_sources(kap, [case.chem["sigma0"]], srcs, g)
        torch.cuda.synchronize()
        t_pt = (time.perf_counter() - t0) / args.reps
        nH = torch.as_tensor(case.nH, dtype=torch.float64, device="cuda")
        y = torch.as_tensor(case.y0, dtype=torch.float64, device="cuda").clone()
        t0 = time.perf_counter()
        try:
            sw.iterate(nH, case.chem, srcs, y, tol=1e-300, max_iter=args.reps)
        except art.ArtError as ex:
            if ex.status != art.ART_E_NOT_CONVERGED:
                raise
        torch.cuda.synchronize()
        t_it = (time.perf_counter() - t0) / args.reps
        sw.close()
        out.update(n=case.n, sources=len(srcs), point_sources_ms_one_bin=round(1e3 * t_pt, 3),
                   iteration_ms=round(1e3 * t_it, 3))
    else:
        # the time-dependent mode with the energy equation on the Test-1 setup (64^3, N_side 4,
        # T0 100 K, a 1e5 K blackbody source in 4 bins) to args.myr
        case = wl.hii_region(n=64, nside=4, box_kpc=6.6, nH=1e-3, Q=5e48, source_at="corner")
        frac, sig, _ = wl.blackbody_bins()
        srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
        sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
        sw.set_source_spectrum(sig, frac)
        th = {"e_bin": list(wl.blackbody_heat()), "e_diff": wl.diffuse_band_heat(case.chem)}
        nH = torch.as_tensor(case.nH, dtype=torch.float64, device="cuda")
        y = torch.as_tensor(case.y0, dtype=torch.float64, device="cuda").clone()
        T = torch.full_like(y, 100.0)
        rep = sw.evolve_thermal(nH, case.chem, th, srcs, y, T, args.myr * wl.MYR, F=1.0)
        sw.close()
        out.update(n=case.n, myr=args.myr, steps=int(rep.steps), iterations=int(rep.iterations),
                   sweeps=int(rep.sweeps), seconds=round(float(rep.seconds), 4),
                   ms_per_iteration=round(1e3 * float(rep.seconds) / max(int(rep.iterations), 1), 3))
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
        return
    if args.impl == "reference":
        d = Dist("gloo")
        try:
            run_reference(args, d)
        finally:
            d.close()
        return
    d = Dist("nccl", always=args.shard)
    try:
        (run_shard if args.shard else run_ours)(args, d)
    finally:
        d.close()


if __name__ == "__main__":
    main()
