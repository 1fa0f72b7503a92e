"""The allocation-free sweep entry point (art_sweep_noalloc) against the
context path (art_create / art_sweep).

Callers that cannot allocate device memory -- a simulation that reserves the
device memory budget for its own arrays, or code that must not trigger the
device-wide synchronization of cudaMalloc/cudaFree -- use art_sweep_noalloc,
whose working memory is a fixed file-scope device array.  This file runs last
(pytest collects it after the other test files) and also passes on its own in
a fresh process.
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


def test_noalloc_matches_context_sweep_twice():
    shape, nside = (24, 20, 28), 3          # ragged against the kernel tiles
    c = wl.grf(32, nside, seed=17)
    kap = np.ascontiguousarray(c.kappa[:shape[0], :shape[1], :shape[2]]).astype(np.float32)
    S = np.ascontiguousarray(c.src[:shape[0], :shape[1], :shape[2]]).astype(np.float32)
    k = torch.as_tensor(kap, device="cuda")
    s = torch.as_tensor(S, device="cuda")

    sw = art.ArtSweep(shape, nside)
    ref = torch.empty_like(k)
    sw.set_fields(k, s)
    sw.sweep(None, ref)
    torch.cuda.synchronize()
    sw.close()
    ref = ref.cpu().numpy().astype(np.float64)

    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):
        out = torch.full_like(k, float("nan"))
        st, msg = art.art_sweep_noalloc(shape, nside, k.data_ptr(), s.data_ptr(), out.data_ptr(), stream)
        assert st == art.ART_OK, msg
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy().astype(np.float64))
    for o in outs:
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - ref) / ref) < 1e-5
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_sizes_beyond_the_maximum():
    k = torch.zeros(1, device="cuda")
    for shape, nside in [((65, 8, 8), 1), ((40, 40, 40), 1), ((8, 8, 8), 5)]:
        st, msg = art.art_sweep_noalloc(shape, nside, k.data_ptr(), k.data_ptr(), k.data_ptr(), 0)
        assert st == art.ART_E_INVALID
        assert "maximum" in msg


def test_noalloc_allocates_nothing_and_matches_the_oracle_at_its_largest_sizes(orc):
    """At the largest accepted grid (64 x 64 x 8 = 32768 cells, N_side 4) the call matches the
    context sweep, and at 32^3, N_side 4 the FP64 oracle; after a first call, a second one leaves
    the device's free memory unchanged."""
    for shape, nside in [((8, 64, 64), 4), ((32, 32, 32), 4)]:
        rng = np.random.default_rng(21)
        kap = (0.3 * np.exp(rng.standard_normal(shape))).astype(np.float32)
        S = rng.random(shape).astype(np.float32)
        k = torch.as_tensor(kap, device="cuda")
        s = torch.as_tensor(S, device="cuda")
        outs = [torch.full_like(k, float("nan")) for _ in range(2)]
        stream = torch.cuda.current_stream().cuda_stream
        st, msg = art.art_sweep_noalloc(shape, nside, k.data_ptr(), s.data_ptr(), outs[0].data_ptr(), stream)
        assert st == art.ART_OK, msg
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st, msg = art.art_sweep_noalloc(shape, nside, k.data_ptr(), s.data_ptr(), outs[1].data_ptr(), stream)
        assert st == art.ART_OK, msg
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        got = outs[1].cpu().numpy().astype(np.float64)
        assert np.array_equal(got, outs[0].cpu().numpy().astype(np.float64))
        if shape == (32, 32, 32):
            jin_o, _, _ = orc.sweep(kap.astype(np.float64), S.astype(np.float64), nside)
            assert np.max(np.abs(got - jin_o) / jin_o) < 1e-5
        else:
            sw = art.ArtSweep(shape, nside)
            ref = torch.empty_like(k)
            sw.set_fields(k, s)
            sw.sweep(None, ref)
            torch.cuda.synchronize()
            sw.close()
            ref = ref.cpu().numpy().astype(np.float64)
            assert np.max(np.abs(got - ref) / ref) < 1e-5


def test_noalloc_refuses_a_capturing_stream_and_leaves_the_capture_valid():
    """The call synchronizes its stream, which a capture forbids: under capture it must return
    ART_E_INVALID before queuing anything, and the capture must still end with a valid graph."""
    shape, nside = (8, 8, 8), 1
    k = torch.ones(shape, device="cuda")
    out = torch.empty_like(k)
    warm = torch.empty_like(k)
    st, msg = art.art_sweep_noalloc(shape, nside, k.data_ptr(), k.data_ptr(), warm.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == art.ART_OK, msg        # the first call (device set-up) outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            out.copy_(k)
            st, msg = art.art_sweep_noalloc(shape, nside, k.data_ptr(), k.data_ptr(), out.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
            out.mul_(2.0)
    assert st == art.ART_E_INVALID and "captured" in msg
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, 2.0 * k)
