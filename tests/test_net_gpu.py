"""GPU parity of the 3D-convolution surrogate (tensor-core forward and input
gradient, weight gradients, Adam) against the FP64 oracle in its bfloat16
mode, which rounds weights, activations and gradients where the GPU stores
them in bfloat16; what remains is the order of FP32 sums (and, rarely, a
bfloat16 rounding that this order tips), so the bars are relative norms.

Shapes cover the three tile forms of the convolution kernel: nx < 128
(several x rows per tile), nx = 128, nx = 256 (two tiles per row).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import surrogate as sg
from paper_1410_0763_gb300 import art, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    art.load()


def relnorm(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


def random_case(shape, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((4,) + shape).astype(np.float32)
    X[2] = rng.random(shape)          # ionized fraction channel in [0, 1)
    t = (0.3 * rng.standard_normal(shape)).astype(np.float32)
    return X, t


def params_with_bias(seed):
    rng = np.random.default_rng(seed)
    layers = sg.init_params(seed=seed)
    layers = [(W, 0.05 * rng.standard_normal(b.shape)) for W, b in layers]
    # a last layer large enough that the output is not dominated by its bias
    W3, b3 = layers[3]
    layers[3] = (W3 * 10.0, b3)
    return layers


def oracle_params(flat32):
    return [(W.astype(np.float64), b.astype(np.float64)) for W, b in art.ArtNet.split_params(flat32)]


@pytest.mark.parametrize("shape,dil,planes", [((16, 16, 16), (1, 2, 4, 8), 0), ((4, 4, 128), (1, 2, 1, 2), 0),
                                               ((2, 3, 256), (1, 1, 2, 1), 0), ((16, 16, 16), (1, 2, 4, 8), 1),
                                               ((16, 16, 16), (1, 2, 4, 8), 2), ((13, 8, 16), (1, 2, 4, 1), 4)])
def test_forward_matches_oracle(shape, dil, planes):
    """planes: output planes per convolution work item (0 = automatic); 13 planes leave
    groups that run past the grid."""
    net = art.ArtNet(dilation=dil)
    net.set_plane_group(planes)
    flat = art.ArtNet.join_params(params_with_bias(3)).astype(np.float32)
    net.set_params(flat)
    X, _ = random_case(shape, 1)
    o = torch.empty(int(np.prod(shape)), dtype=torch.float32, device="cuda")
    net.forward(torch.as_tensor(X).cuda().reshape(-1), o, shape)
    torch.cuda.synchronize()
    got = o.cpu().numpy().astype(np.float64).reshape(shape)
    want, _ = sg.forward(X.astype(np.float64), oracle_params(flat), dil, bf16_mode=True)
    assert np.std(want) > 1e-2
    assert relnorm(got, want) < 2e-3, (relnorm(got, want), np.max(np.abs(got - want)))
    net.close()


@pytest.mark.parametrize("shape,dil,weighted,planes", [((16, 16, 16), (1, 2, 4, 8), False, 0),
                                                        ((4, 4, 128), (2, 1, 1, 3), False, 0),
                                                        ((16, 16, 16), (1, 2, 4, 8), True, 0),
                                                        ((13, 8, 16), (1, 2, 1, 3), True, 4)])
def test_gradients_match_oracle(shape, dil, weighted, planes):
    net = art.ArtNet(dilation=dil)
    net.set_plane_group(planes)
    flat = art.ArtNet.join_params(params_with_bias(4)).astype(np.float32)
    net.set_params(flat)
    X, t = random_case(shape, 2)
    w = sg.weights(np.random.default_rng(9).random(shape) ** 4).astype(np.float32) if weighted else None
    wd = torch.as_tensor(w).cuda().reshape(-1) if weighted else None
    loss, g = net.gradients(torch.as_tensor(X).cuda().reshape(-1), torch.as_tensor(t).cuda().reshape(-1), shape,
                            w=wd)
    P = oracle_params(flat)
    o, acts = sg.forward(X.astype(np.float64), P, dil, bf16_mode=True)
    w64 = None if w is None else w.astype(np.float64)
    want = sg.backward(o, t.astype(np.float64), acts, P, dil, bf16_mode=True, w=w64)
    assert loss == pytest.approx(sg.loss(o, t, w64), rel=1e-3)
    got = art.ArtNet.split_params(g)
    for li in range(4):
        assert relnorm(got[li][0], want[li][0]) < 1e-2, (li, relnorm(got[li][0], want[li][0]))
        assert relnorm(got[li][1], want[li][1]) < 1e-2, (li, relnorm(got[li][1], want[li][1]))
    net.close()


def test_adam_step_matches_oracle():
    shape, dil = (16, 16, 16), (1, 2, 4, 8)
    net = art.ArtNet(dilation=dil, lr=1e-3)
    flat = art.ArtNet.join_params(params_with_bias(5)).astype(np.float32)
    net.set_params(flat)
    X, t = random_case(shape, 3)
    Xd, td = torch.as_tensor(X).cuda().reshape(-1), torch.as_tensor(t).cuda().reshape(-1)
    _, g = net.gradients(Xd, td, shape)
    loss0 = net.train_step(Xd, td, shape)
    after = net.get_params()
    P = oracle_params(flat)
    G = [(gw.astype(np.float64), gb.astype(np.float64)) for gw, gb in art.ArtNet.split_params(g)]
    want, _ = sg.adam(P, G, None, lr=1e-3)
    want = art.ArtNet.join_params(want)
    close = np.abs(after - want) <= 1e-6 + 1e-6 * np.abs(want)
    assert close.mean() > 0.99
    # a few more steps lower the loss on this sample
    for _ in range(20):
        net.train_step(Xd, td, shape, want_loss=False)
    assert net.train_step(Xd, td, shape) < loss0
    net.close()


def test_bad_shapes_are_rejected():
    net = art.ArtNet()
    X = torch.zeros(4 * 10 * 10 * 10, device="cuda")
    o = torch.zeros(1000, device="cuda")
    with pytest.raises(art.ArtError) as e:
        net.forward(X, o, (10, 10, 10))
    assert e.value.status == art.ART_E_INVALID
    net.close()


def test_bounded_waits_report_a_timeout_and_the_network_recovers():
    """The test hook stops the TMA loads, so every convolution kernel's bounded
    waits run out (about a second each); the host sees ART_E_TIMEOUT, and
    the next passes are correct again (no GPU fault, context usable)."""
    shape, dil = (16, 16, 16), (1, 2, 4, 8)
    net = art.ArtNet(dilation=dil)
    flat = art.ArtNet.join_params(params_with_bias(3)).astype(np.float32)
    net.set_params(flat)
    X, _ = random_case(shape, 1)
    Xd = torch.as_tensor(X).cuda().reshape(-1)
    o = torch.empty(int(np.prod(shape)), dtype=torch.float32, device="cuda")
    net.set_test_stall(True)
    net.forward(Xd, o, shape)
    assert net.check() == art.ART_E_TIMEOUT
    assert net.check() == art.ART_OK            # the error word was cleared
    net.set_test_stall(False)
    net.forward(Xd, o, shape)
    assert net.check() == art.ART_OK
    got = o.cpu().numpy().astype(np.float64).reshape(shape)
    want, _ = sg.forward(X.astype(np.float64), oracle_params(flat), dil, bf16_mode=True)
    assert relnorm(got, want) < 2e-3
    net.close()
