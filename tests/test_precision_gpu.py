"""Precision of the FP32 sweep against the FP64 oracle, per workload (the
bound asserted and the measured maximum printed, `pytest -s`):

* 16^3 lognormal, N_side 1: FP64 context, all cells;
* 64^3 GRF, N_side 4: FP32, all cells;
* 128^3 HII region at the converged ionization state, N_side 8, emissivity
  form: FP32, all cells;
* the 48-grid batch: FP32, sampled cells of every grid;
* 256^3 clumpy medium (sigma 1.5 + 200 clumps), N_side 8: FP32, sampled cells.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1410_0763_gb300 import art, build
from paper_1410_0763_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    art.load()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def gpu_jin(kap, src, nside, precision="fp32", form=0):
    dt = torch.float64 if precision == "fp64" else torch.float32
    k = torch.as_tensor(np.ascontiguousarray(kap), dtype=dt, device="cuda").reshape(-1)
    s = torch.as_tensor(np.ascontiguousarray(src), dtype=dt, device="cuda").reshape(-1)
    sw = art.ArtSweep(kap.shape, nside, 1, precision=precision, field_form=form)
    out = torch.empty_like(k)
    sw.set_fields(k, s)
    sw.sweep(J_in=out)
    torch.cuda.synchronize()
    sw.close()
    return out.cpu().numpy().astype(np.float64).reshape(kap.shape)


def report(name, err, bound):
    print(f"\nPRECISION {name}: max relative error of J^in {err:.3e} (bound {bound:.0e})")
    assert err < bound


def test_lognormal16_fp64(orc):
    c = wl.lognormal_iid(16, 1)
    want, _, _ = orc.sweep(c.kappa, c.src, 1)
    report("16^3 lognormal N_side 1 FP64", rel(gpu_jin(c.kappa, c.src, 1, "fp64"), want), 1e-12)


def test_grf64_fp32(orc):
    c = wl.grf(64, 4)
    want, _, _ = orc.sweep(f32(c.kappa), f32(c.src), 4)
    report("64^3 GRF N_side 4 FP32", rel(gpu_jin(c.kappa, c.src, 4), want), 1e-5)


def test_hii128_converged_state_fp32(orc):
    """kappa and eps of the converged 128^3 HII region (the fields the sweep
    sees in the last iterations of the solve)."""
    case = wl.hii_region()
    sw = art.ArtSweep(case.nH.shape, case.nside, 1, field_form=art.ART_FIELDS_EPS, dx_cm=case.chem["dx"])
    nH = torch.as_tensor(case.nH, dtype=torch.float64, device="cuda")
    y = torch.as_tensor(case.y0, dtype=torch.float64, device="cuda").clone()
    srcs = [(p[0], p[1], p[2], q) for p, q in zip(case.pos, case.Q)]
    sw.iterate(nH, case.chem, srcs, y, tol=1e-6, max_iter=200)
    sw.close()
    ch = case.chem
    yh = y.cpu().numpy()
    kap = f32(yh * case.nH * ch["sigma0"] * ch["dx"])
    eps = f32(((1.0 - yh) * case.nH) ** 2 * 1e-6)      # J^in is linear in eps: any positive scale
    want, _, _ = orc.sweep(kap, eps, case.nside, field_form=1)
    report("128^3 HII converged state N_side 8 FP32 (emissivity form)",
           rel(gpu_jin(kap, eps, case.nside, form=1), want), 1e-5)


def test_batch48_sampled_fp32(orc):
    cases = wl.batch48()
    shapes = [c.kappa.shape for c in cases]
    sw = art.ArtSweep(shapes, [c.nside for c in cases], 1)
    k = torch.cat([torch.as_tensor(c.kappa.ravel(), dtype=torch.float32) for c in cases]).cuda()
    s = torch.cat([torch.as_tensor(c.src.ravel(), dtype=torch.float32) for c in cases]).cuda()
    out = torch.empty_like(k)
    sw.set_fields(k, s)
    sw.sweep(J_in=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(6)
    worst = 0.0
    for c, off in zip(cases, sw.offsets):
        cells = rng.integers(0, c.kappa.size, 8)
        want = orc.jin_cells(f32(c.kappa), f32(c.src), c.nside, cells)
        worst = max(worst, rel(got[off + cells], want))
    sw.close()
    report("48-grid batch (8 sampled cells per grid) FP32", worst, 1e-5)


def test_clumpy256_sampled_fp32(orc):
    case = wl.clumpy()
    ch = case.chem
    kap = f32(case.nH * ch["sigma0"] * ch["dx"] * 0.5)    # half neutral everywhere: thick clumps, thin voids
    eps = f32((0.5 * case.nH) ** 2)
    got = gpu_jin(kap, eps, case.nside, form=1)
    rng = np.random.default_rng(7)
    cells = rng.integers(0, kap.size, 48)
    want = orc.jin_cells(kap, eps, case.nside, cells, field_form=1)
    report("256^3 clumpy N_side 8 (48 sampled cells) FP32", rel(got.ravel()[cells], want), 1e-4)
