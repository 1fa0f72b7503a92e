"""The wavefront kernel's series paths (CPU): the economized coefficients beta_k and the
thresholds in art_wave.cuh, read from the source, keep the deposit coefficient
g = ds phi(kappa ds), phi(x) = (1 - e^-x)/x, within its stated bound over each path's whole
range (every kappa below the threshold, every segment length up to sqrt(3)), against
phi from expm1 in float64 and with the kernel's FP32 evaluation order simulated."""
import math
import os
import re

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1410_0763_gb300", "csrc", "art_wave.cuh")


def source():
    with open(SRC) as f:
        return f.read()


def threshold(name):
    if not isinstance(name, str):
        return float(np.float32(name))
    m = re.search(r"constexpr float %s = ([0-9.eE+-]+)f;" % name, source())
    assert m, name
    return float(np.float32(float(m.group(1))))


def betas(K):
    m = re.search(r"constexpr float wv_beta<%d>\(int k\)[^{]*\{(.*?)\n\}" % K, source(), flags=re.S)
    assert m, K
    vals = [float(np.float32(float(v))) for v in re.findall(r"([0-9]*\.[0-9]+(?:[eE][+-]?[0-9]+)?)f", m.group(1))]
    assert len(vals) == K
    return vals


def g_fp32(beta, kap, ds):
    """The kernel's evaluation: c_k = (-kappa)^k beta_k by repeated products, Horner in ds,
    then ds + ds^2 q, every operation rounded to FP32."""
    f = np.float32
    kap, ds = kap.astype(f), ds.astype(f)
    ds2 = (ds * ds).astype(f)
    nk = (-kap).astype(f)
    pw, c = nk.copy(), []
    for b in beta:
        c.append((pw * f(b)).astype(f))
        pw = (pw * nk).astype(f)
    K = len(beta)
    q = (c[K - 1] * ds + c[K - 2]).astype(f)
    for k in range(K - 3, -1, -1):
        q = (q * ds + c[k]).astype(f)
    return (q * ds2 + ds).astype(f).astype(np.float64)


# (degree, top of its kappa range): the three series paths, and the mixed path's degree-4
# series, economized on x < X_SERIES (kappa up to X_SERIES / sqrt(3) with segments up to sqrt(3))
PATHS = [(2, "KAP_THIN2"), (3, "KAP_THIN"), (5, "KAP_THIN5"), (4, threshold("X_SERIES") / math.sqrt(3.0))]


@pytest.mark.parametrize("K,name", PATHS)
def test_economized_series_within_its_bound(K, name):
    beta = betas(K)
    kmax = threshold(name)
    h = math.sqrt(3.0) * kmax
    # each coefficient sits below its Taylor value 1/(k+1)!, the lower ones just below (the
    # highest absorbs most of the dropped terms); a transposed or missing coefficient fails here
    for k, b in enumerate(beta, start=1):
        t = 1.0 / math.factorial(k + 1)
        assert (0.5 if k == K else 0.95) * t < b <= t
    x = np.linspace(0.0, h, 400001)[1:]
    phi = -np.expm1(-x) / x
    a = [(-1) ** k * b for k, b in enumerate(beta, start=1)]   # psi(x) ~ sum a_k x^(k-1)
    approx = 1.0 + x * np.polyval(a[::-1], x)
    assert np.max(np.abs(approx - phi) / phi) < 2.0e-7


@pytest.mark.parametrize("K,name", PATHS)
def test_economized_series_in_fp32(K, name):
    beta = betas(K)
    kmax = threshold(name)
    rng = np.random.default_rng(K)
    kap = np.concatenate([rng.uniform(0.0, kmax, 300000), np.full(2000, np.nextafter(np.float32(kmax), 0))])
    ds = np.concatenate([rng.uniform(0.0, math.sqrt(3.0), 300000), np.linspace(1e-4, math.sqrt(3.0), 2000)])
    kap32, ds32 = kap.astype(np.float32).astype(np.float64), ds.astype(np.float32).astype(np.float64)
    g = g_fp32(beta, kap, ds)
    x = kap32 * ds32
    ge = np.where(x > 0, -np.expm1(-x) / np.where(kap32 > 0, kap32, 1.0), ds32)
    assert np.max(np.abs(g - ge) / ge) < 3.0e-7


def test_thresholds_order():
    """The series paths cover nested ranges up to the exponential-only path."""
    assert threshold("KAP_THIN2") < threshold("KAP_THIN") < threshold("KAP_THIN5") <= threshold("KAP_THICK")
    # the mixed path switches to the exponential where the series' range ends; the x-form mixed
    # path of the smaller shapes (the x^5 Taylor series) stops earlier
    assert threshold("X_SERIES_X") <= threshold("X_SERIES")
