"""Time the point-source rates and one RT / ionization-balance iteration on a
grid: ``python -m paper_1410_0763_gb300.ionbench --case hii --reps 5`` (128^3
HII region, one source) or ``--case clumpy`` (256^3 clumpy medium, 8 sources,
4 bins); or, with ``--case thermal --myr 30``, the time-dependent mode with
the energy equation on the Test-1 setup (64^3, N_side 4, T0 100 K, a 1e5 K
blackbody source in 4 bins) to the given time.  Prints one JSON line."""
from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=("hii", "clumpy", "thermal"), default="hii")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--myr", type=float, default=30.0, help="thermal case: evolve to this time")
    a = ap.parse_args(argv)
    if a.case == "thermal":
        return thermal(a.myr)
    import torch
    from . import art, build
    from . import workloads as wl
    build.build()
    art.load()
    case = wl.hii_region() if a.case == "hii" else wl.clumpy()
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    if a.case == "clumpy":
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
    for _ in range(a.reps):
        sw.point_sources(kap, [case.chem["sigma0"]], srcs, g)
    torch.cuda.synchronize()
    t_pt = (time.perf_counter() - t0) / a.reps
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device="cuda")
    y = torch.as_tensor(case.y0, dtype=torch.float64, device="cuda").clone()
    t0 = time.perf_counter()
    try:
        sw.iterate(nH, case.chem, srcs, y, tol=1e-300, max_iter=a.reps)
    except art.ArtError as ex:
        if ex.status != art.ART_E_NOT_CONVERGED:
            raise
    torch.cuda.synchronize()
    t_it = (time.perf_counter() - t0) / a.reps
    sw.close()
    print(json.dumps({"case": a.case, "n": case.n, "sources": len(srcs),
                      "point_sources_ms_one_bin": round(1e3 * t_pt, 3),
                      "iteration_ms": round(1e3 * t_it, 3)}), flush=True)


def thermal(myr: float):
    import torch
    from . import art, build
    from . import workloads as wl
    build.build()
    art.load()
    case = wl.hii_region(n=64, nside=4, box_kpc=6.6, nH=1e-3, Q=5e48, source_at="corner")
    frac, sig, _ = wl.blackbody_bins()
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    sw.set_source_spectrum(sig, frac)
    th = {"e_bin": list(wl.blackbody_heat()), "e_diff": wl.diffuse_band_heat(case.chem)}
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device="cuda")
    y = torch.as_tensor(case.y0, dtype=torch.float64, device="cuda").clone()
    T = torch.full_like(y, 100.0)
    rep = sw.evolve_thermal(nH, case.chem, th, srcs, y, T, myr * wl.MYR, F=1.0)
    sw.close()
    print(json.dumps({"case": "thermal", "n": case.n, "myr": myr, "steps": int(rep.steps),
                      "iterations": int(rep.iterations), "sweeps": int(rep.sweeps),
                      "seconds": round(float(rep.seconds), 4),
                      "ms_per_iteration": round(1e3 * float(rep.seconds) / max(int(rep.iterations), 1), 3)}),
          flush=True)


if __name__ == "__main__":
    main()
