"""FP64 CPU oracle of the 3D-convolution surrogate that warm-starts the RT /
ionization-balance iteration -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module; the product path never does.  Plain numpy in float64: a
convolution is a sum over the 27 taps of a shifted array times a channel
matrix, written out one tap at a time, with no blocking or fusion.

The surrogate is not in the paper (which iterates plain sweeps to
convergence, App. D); it is specified here:

* Inputs per cell (channels, in this order): 0.25 ln kappa, 0.1 ln(eps /
  eps_ref), x = 1 - y, 0.1 ln(J_c / eps_ref), each logarithm clamped at
  ln(1e-30) (-69) below its reference.
  kappa and eps are the sweep's absorption and emission per cell width
  (ART_FIELDS_EPS form), y the neutral fraction, eps_ref = max eps, J_c the
  mean intensity J^in of a sweep on the grid coarsened by a factor f (block
  means of kappa and eps times f, App. D's fields on a coarser mesh),
  prolonged to the fine cells by injection.
* Network: four 3x3x3 convolutions (zero padding, dilations d_l), 32 hidden
  channels, ReLU after the first three, one output channel o.
* Prediction J^in = J_c exp(o); training target t = ln(J^in / J_c) on the
  plain sweep's J^in (logarithms clamped at ln eps_ref - 69); loss
  mean(w (o - t)^2) with cell weights w = J^in / mean(J^in) (or 1).
* Optimizer: Adam (Kingma & Ba 2015), bias-corrected moments.

``bf16_mode=True`` rounds weights, activations and back-propagated gradients
(the output-layer gradient included) to bfloat16 (round to nearest even) where the GPU stores them in
bfloat16, so that the only remaining difference to the GPU is the order of
the FP32 sums.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
HIDDEN = 32
N_IN = 4
TINY = 1e-30


# ---------------------------------------------------------------------------
# bfloat16 rounding (round to nearest, ties to even, of the float32 value)
# ---------------------------------------------------------------------------
def bf16(a):
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


# ---------------------------------------------------------------------------
# convolution and its adjoints
# ---------------------------------------------------------------------------
def shifted(a, dz, dy, dx):
    """s[c, z, y, x] = a[c, z + dz, y + dy, x + dx], zero outside the grid."""
    C, nz, ny, nx = a.shape
    out = np.zeros_like(a)
    z0, z1 = max(0, -dz), min(nz, nz - dz)
    y0, y1 = max(0, -dy), min(ny, ny - dy)
    x0, x1 = max(0, -dx), min(nx, nx - dx)
    if z0 < z1 and y0 < y1 and x0 < x1:
        out[:, z0:z1, y0:y1, x0:x1] = a[:, z0 + dz:z1 + dz, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
    return out


def conv(a, W, b, d):
    """out[co, v] = b[co] + sum_t sum_ci W[t, co, ci] a[ci, v + d * off_t]."""
    C_out = W.shape[1]
    out = np.zeros((C_out,) + a.shape[1:])
    for t, (dz, dy, dx) in enumerate(TAPS):
        s = shifted(a, d * dz, d * dy, d * dx)
        out += np.einsum("oc,czyx->ozyx", W[t], s)
    return out + b[:, None, None, None]


def conv_grad_input(g, W, d):
    """Adjoint of conv in its input: ga[ci, v] = sum_t sum_co W[t, co, ci] g[co, v - d * off_t]."""
    C_in = W.shape[2]
    out = np.zeros((C_in,) + g.shape[1:])
    for t, (dz, dy, dx) in enumerate(TAPS):
        s = shifted(g, -d * dz, -d * dy, -d * dx)
        out += np.einsum("oc,ozyx->czyx", W[t], s)
    return out


def conv_grad_weight(g, a, d):
    """gW[t, co, ci] = sum_v g[co, v] a[ci, v + d * off_t];  gb[co] = sum_v g[co, v]."""
    C_out, C_in = g.shape[0], a.shape[0]
    gW = np.zeros((27, C_out, C_in))
    for t, (dz, dy, dx) in enumerate(TAPS):
        s = shifted(a, d * dz, d * dy, d * dx)
        gW[t] = np.einsum("ozyx,czyx->oc", g, s)
    return gW, g.sum(axis=(1, 2, 3))


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def layer_shapes(n_in=N_IN, hidden=HIDDEN):
    return [(n_in, hidden), (hidden, hidden), (hidden, hidden), (hidden, 1)]


def init_params(seed=0, n_in=N_IN, hidden=HIDDEN):
    """He-normal weights (std sqrt(2 / (27 c_in))), zero biases; the last layer scaled by 0.1."""
    rng = np.random.default_rng(seed)
    params = []
    for i, (ci, co) in enumerate(layer_shapes(n_in, hidden)):
        W = rng.standard_normal((27, co, ci)) * np.sqrt(2.0 / (27 * ci))
        if i == 3:
            W *= 0.1
        params.append((W, np.zeros(co)))
    return params


def forward(X, params, dil, bf16_mode=False):
    """X: (n_in, nz, ny, nx).  Returns (o, acts) with acts the layer inputs."""
    r = bf16 if bf16_mode else (lambda v: v)
    acts = [r(X)]
    h = acts[0]
    for i, (W, b) in enumerate(params):
        z = conv(h, r(W), b, dil[i])
        if i < 3:
            h = r(np.maximum(z, 0.0))
            acts.append(h)
        else:
            o = z[0]
    return o, acts


def loss(o, t, w=None):
    """mean(w (o - t)^2), w = 1 when not given."""
    d2 = (o - t) ** 2
    return float(np.mean(d2 if w is None else w * d2))


def weights(jin):
    """Per-cell loss weights J^in / mean(J^in): the loss then measures the
    intensity-weighted error that the surrogate's judge measures."""
    m = float(np.mean(jin))
    return jin / m if m > 0 else np.ones_like(jin)


def backward(o, t, acts, params, dil, bf16_mode=False, w=None):
    """Gradients of loss(o, t, w) in every weight and bias (list of (gW, gb))."""
    r = bf16 if bf16_mode else (lambda v: v)
    V = o.size
    g = (2.0 / V) * ((o - t) if w is None else w * (o - t))[None]
    grads = [None] * 4
    for i in range(3, -1, -1):
        W, _ = params[i]
        g_in = r(g)
        gW, gb = conv_grad_weight(g_in, acts[i], dil[i])
        grads[i] = (gW, gb)
        if i > 0:
            ga = conv_grad_input(g_in, r(W), dil[i])
            g = ga * (acts[i] > 0)
    return grads


def adam(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; state = (step, [(mW, vW, mb, vb)]) (created when None)."""
    if state is None:
        state = (0, [(np.zeros_like(W), np.zeros_like(W), np.zeros_like(b), np.zeros_like(b)) for W, b in params])
    step, mom = state
    step += 1
    out, new_mom = [], []
    for (W, b), (gW, gb), (mW, vW, mb, vb) in zip(params, grads, mom):
        res = []
        for p, gp, m, v in ((W, gW, mW, vW), (b, gb, mb, vb)):
            m = b1 * m + (1 - b1) * gp
            v = b2 * v + (1 - b2) * gp * gp
            mh = m / (1 - b1 ** step)
            vh = v / (1 - b2 ** step)
            res.append((p - lr * mh / (np.sqrt(vh) + eps), m, v))
        (W2, mW2, vW2), (b2_, mb2, vb2) = res
        out.append((W2, b2_))
        new_mom.append((mW2, vW2, mb2, vb2))
    return out, (step, new_mom)


# ---------------------------------------------------------------------------
# inputs, coarse sweep fields, target
# ---------------------------------------------------------------------------
def restrict(a, f):
    """Block means over f^3 cells times f (per-cell-width quantities on the coarse mesh)."""
    nz, ny, nx = a.shape
    b = a.reshape(nz // f, f, ny // f, f, nx // f, f)
    return f * b.mean(axis=(1, 3, 5))


def prolong(a, f):
    """Injection: every fine cell takes its coarse cell's value."""
    return np.repeat(np.repeat(np.repeat(a, f, axis=0), f, axis=1), f, axis=2)


LOG_FLOOR = -69.0     # ln(1e-30): logarithms are clamped this far below their reference


def _ln(a):
    a = np.asarray(a, dtype=np.float64)
    out = np.full(a.shape, -np.inf)
    np.log(a, out=out, where=a > 0)
    return out


def features(kappa, eps, y, jc_fine):
    """Input channels; eps_ref = max eps (0 gives the floor everywhere)."""
    eref = float(np.max(eps))
    lref = np.log(eref) if eref > 0 else 0.0
    X = np.zeros((N_IN,) + np.shape(kappa))
    X[0] = 0.25 * np.maximum(_ln(kappa), LOG_FLOOR)
    X[1] = 0.1 * np.maximum(_ln(eps) - lref, LOG_FLOOR)
    X[2] = 1.0 - np.asarray(y)
    X[3] = 0.1 * np.maximum(_ln(jc_fine) - lref, LOG_FLOOR)
    return X


def target(jin, jc_fine, eps):
    """t = ln J^in - ln J_c, each logarithm clamped at ln(eps_ref) + LOG_FLOOR."""
    eref = float(np.max(eps))
    floor = (np.log(eref) if eref > 0 else 0.0) + LOG_FLOOR
    return np.maximum(_ln(jin), floor) - np.maximum(_ln(jc_fine), floor)


def predict(jc_fine, o):
    return np.asarray(jc_fine) * np.exp(o)
