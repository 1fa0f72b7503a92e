"""Pins of the surrogate oracle (oracle/surrogate.py) against things other than
itself: the library's bfloat16 rounding and cross-correlation, adjoint
identities, central finite differences, Adam's closed-form first steps."""
import numpy as np
import pytest

from oracle import surrogate as sg

torch = pytest.importorskip("torch")
scipy_signal = pytest.importorskip("scipy.signal")


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-20, 20, 5000),
                        [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 65504.0, 3.0e38, 1e-40]])
    want = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(sg.bf16(x), want)
    # ties go to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert sg.bf16(np.array([1 + 2 ** -8]))[0] == 1.0
    assert sg.bf16(np.array([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6


def test_conv_center_delta_is_identity_and_off_center_is_a_shift():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((3, 5, 6, 7))
    W = np.zeros((27, 3, 3))
    W[13] = np.eye(3)                       # tap (0, 0, 0)
    b = np.array([0.5, -1.0, 2.0])
    assert np.allclose(sg.conv(a, W, b, 1), a + b[:, None, None, None], atol=0, rtol=0)
    W = np.zeros((27, 1, 3))
    t = sg.TAPS.index((1, -1, 1))
    W[t, 0, 2] = 1.0
    out = sg.conv(a, W, np.zeros(1), 2)[0]
    # out[z, y, x] = a[2, z + 2, y - 2, x + 2] inside, zero where that leaves the grid
    assert out[0, 2, 0] == a[2, 2, 0, 2]
    assert out[2, 5, 4] == a[2, 4, 3, 6]
    assert out[3, 1, 0] == 0.0 and out[0, 0, 0] == 0.0 and out[0, 2, 5] == 0.0


@pytest.mark.parametrize("d", [1, 2])
def test_conv_matches_scipy_correlate(d):
    rng = np.random.default_rng(2 + d)
    a = rng.standard_normal((2, 6, 7, 9))
    W = rng.standard_normal((27, 3, 2))
    b = rng.standard_normal(3)
    out = sg.conv(a, W, b, d)
    k = 2 * d + 1
    for co in range(3):
        want = np.full(a.shape[1:], b[co])
        for ci in range(2):
            K = np.zeros((k, k, k))
            for t, (dz, dy, dx) in enumerate(sg.TAPS):
                K[d + d * dz, d + d * dy, d + d * dx] = W[t, co, ci]
            want += scipy_signal.correlate(a[ci], K, mode="same", method="direct")
        assert np.allclose(out[co], want, rtol=1e-12, atol=1e-12)


def test_adjoints_by_dot_products():
    rng = np.random.default_rng(4)
    a = rng.standard_normal((3, 6, 5, 7))
    g = rng.standard_normal((4, 6, 5, 7))
    W = rng.standard_normal((27, 4, 3))
    for d in (1, 2, 4):
        lhs = np.sum(sg.conv(a, W, np.zeros(4), d) * g)
        assert lhs == pytest.approx(np.sum(a * sg.conv_grad_input(g, W, d)), rel=1e-12)
        gW, gb = sg.conv_grad_weight(g, a, d)
        assert lhs == pytest.approx(np.sum(W * gW), rel=1e-12)
        assert np.allclose(gb, g.sum(axis=(1, 2, 3)))


@pytest.mark.parametrize("weighted", [False, True])
def test_backward_matches_central_differences(weighted):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((2, 8, 8, 8))
    t = rng.standard_normal((8, 8, 8))
    w = sg.weights(rng.random((8, 8, 8)) ** 3) if weighted else None
    dil = (1, 2, 1, 2)
    params = sg.init_params(seed=3, n_in=2, hidden=4)
    params = [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]
    o, acts = sg.forward(X, params, dil)
    grads = sg.backward(o, t, acts, params, dil, w=w)
    h = 1e-6
    for li in range(4):
        W, b = params[li]
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in W.shape)
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = list(params)
            pp[li] = (Wp, b)
            lp = sg.loss(sg.forward(X, pp, dil)[0], t, w)
            pp[li] = (Wm, b)
            lm = sg.loss(sg.forward(X, pp, dil)[0], t, w)
            fd = (lp - lm) / (2 * h)
            assert grads[li][0][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)
        j = int(rng.integers(0, b.shape[0]))
        bp, bm = b.copy(), b.copy()
        bp[j] += h
        bm[j] -= h
        pp = list(params)
        pp[li] = (W, bp)
        lp = sg.loss(sg.forward(X, pp, dil)[0], t, w)
        pp[li] = (W, bm)
        lm = sg.loss(sg.forward(X, pp, dil)[0], t, w)
        assert grads[li][1][j] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)


def test_adam_first_steps_closed_form():
    W = np.array([[[1.0, -2.0]]]).repeat(27, axis=0)
    b = np.array([0.5])
    g = (np.full_like(W, 0.3), np.array([-4.0]))
    params, state = sg.adam([(W, b)], [g], None, lr=0.01, eps=0.0)
    # bias-corrected moments equal g and g^2 after one step: a step of lr * sign(g)
    assert np.allclose(params[0][0], W - 0.01)
    assert np.allclose(params[0][1], b + 0.01)
    # constant gradient: every step is lr * sign(g)
    params, state = sg.adam(params, [g], state, lr=0.01, eps=0.0)
    assert np.allclose(params[0][0], W - 0.02)
    assert state[0] == 2


def test_restrict_prolong_and_target_round_trip():
    rng = np.random.default_rng(6)
    c = rng.random((2, 3, 4))
    assert np.allclose(sg.restrict(sg.prolong(c, 4), 4), 4 * c)
    a = rng.random((8, 12, 16))
    assert sg.restrict(a, 4).sum() == pytest.approx(a.sum() / 16)
    jc = rng.random((8, 8, 8)) + 0.1
    jin = rng.random((8, 8, 8)) + 0.1
    eps = rng.random((8, 8, 8))
    assert np.allclose(sg.predict(jc, sg.target(jin, jc, eps)), jin, rtol=1e-14)
    # zero fields take the floors, not -inf
    X = sg.features(np.zeros((2, 2, 2)), np.zeros((2, 2, 2)), np.ones((2, 2, 2)), np.zeros((2, 2, 2)))
    assert np.all(np.isfinite(X)) and X[0].max() == 0.25 * sg.LOG_FLOOR


def test_features_are_scale_free_in_the_emissivity():
    rng = np.random.default_rng(7)
    kap, eps, y, jc = (rng.random((4, 4, 4)) + 0.01 for _ in range(4))
    f1 = sg.features(kap, eps, y, jc)
    f2 = sg.features(kap, 1e5 * eps, y, 1e5 * jc)   # J^in is linear in eps
    assert np.allclose(f1, f2, atol=1e-12)


def test_weights_have_unit_mean_and_follow_the_intensity():
    j = np.array([[[0.0, 1.0], [2.0, 5.0]]])
    w = sg.weights(j)
    assert w.mean() == pytest.approx(1.0) and w[0, 1, 1] == pytest.approx(2.5)
    assert np.all(sg.weights(np.zeros((2, 2, 2))) == 1.0)
