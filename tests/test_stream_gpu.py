"""art_sweep_stream: sweeps of several field sets held in host memory, with
the copies of neighbouring sets overlapping each sweep.  Its outputs are
bit-identical to art_set_fields + art_sweep per set (graph replay and plain
launches); an invalid set ends the call with ART_E_INVALID after the sets
before it are written, and leaves the later outputs untouched."""
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


def _sets(n, nsets):
    out = []
    for k in range(nsets):
        c = wl.grf(n, 2, seed=30 + k)
        out.append((np.ascontiguousarray(c.kappa, dtype=np.float32), np.ascontiguousarray(c.src, dtype=np.float32)))
    return out


@pytest.mark.parametrize("graph", [True, False])
def test_stream_matches_per_set_sweeps_bitwise(graph):
    n, nsets = 24, 5
    sets = _sets(n, nsets)
    shape = (n, n, n)
    want = []
    with art.ArtSweep(shape, 2, graph=graph) as sw:
        sw.set_band([0.7])
        for kap, src in sets:
            sw.set_fields(kap, src)
            J, Jin, g = (np.empty(shape, np.float32) for _ in range(3))
            sw.sweep(J, Jin, g)
            want.append((J, Jin, g))
    # pinned torch tensors for some inputs, numpy arrays for the others
    kaps = [torch.from_numpy(k).pin_memory() if i % 2 else k for i, (k, _) in enumerate(sets)]
    srcs = [s for _, s in sets]
    J = [np.full(shape, np.nan, np.float32) for _ in range(nsets)]
    Jin = [np.full(shape, np.nan, np.float32) for _ in range(nsets)]
    g = [np.full(shape, np.nan, np.float32) for _ in range(nsets)]
    with art.ArtSweep(shape, 2, graph=graph) as sw:
        sw.set_band([0.7])
        sw.sweep_stream(kaps, srcs, J, Jin, g)
        for k in range(nsets):
            assert np.array_equal(J[k], want[k][0]) and np.array_equal(Jin[k], want[k][1])
            assert np.array_equal(g[k], want[k][2])
        # the last set stays the context's fields
        J2 = np.empty(shape, np.float32)
        sw.sweep(J2)
        assert np.array_equal(J2, want[-1][0])
        # only J requested, twice in a row (slots and events reused)
        for _ in range(2):
            Jo = [np.empty(shape, np.float32) for _ in range(nsets)]
            sw.sweep_stream(kaps, srcs, J=Jo)
            assert all(np.array_equal(Jo[k], want[k][0]) for k in range(nsets))
        assert sw.sweep_stream([], [])[0] is None


def test_invalid_set_stops_the_stream():
    n = 16
    sets = _sets(n, 3)
    shape = (n, n, n)
    bad = sets[1][0].copy()
    bad[3, 4, 5] = -1.0
    kaps = [sets[0][0], bad, sets[2][0]]
    srcs = [s for _, s in sets]
    J = [np.full(shape, np.nan, np.float32) for _ in range(3)]
    with art.ArtSweep(shape, 2) as sw:
        with pytest.raises(art.ArtError) as ex:
            sw.sweep_stream(kaps, srcs, J=J)
        assert ex.value.status == art.ART_E_INVALID and "set 1" in str(ex.value)
        sw.set_fields(*sets[0])
        J0 = np.empty(shape, np.float32)
        sw.sweep(J0)
    assert np.array_equal(J[0], J0)
    assert np.all(np.isnan(J[1])) and np.all(np.isnan(J[2]))


@pytest.mark.parametrize("kind", ["fp64", "batch"])
def test_stream_fp64_and_batch_contexts(kind):
    if kind == "fp64":
        shape, nside, kw = (12, 10, 14), 2, dict(precision="fp64")
        dt = np.float64
        mk = lambda k: wl.grf(16, 2, seed=50 + k)
        cut = lambda a: np.ascontiguousarray(a[:12, :10, :14], dtype=dt)
        fields = [(cut(mk(k).kappa), cut(mk(k).src)) for k in range(3)]
        n = int(np.prod(shape))
    else:
        shape, nside, kw = [(8, 8, 8), (12, 10, 6)], [1, 2], {}
        dt = np.float32
        n = sum(int(np.prod(s)) for s in shape)
        rng = np.random.default_rng(7)
        fields = [(rng.uniform(0.05, 2.0, n).astype(dt), rng.uniform(0.0, 1.0, n).astype(dt)) for _ in range(3)]
    want = []
    with art.ArtSweep(shape, nside, **kw) as sw:
        for kap, src in fields:
            sw.set_fields(kap, src)
            J, Jin = np.empty(n, dt), np.empty(n, dt)
            sw.sweep(J.reshape(-1), Jin.reshape(-1))
            want.append((J, Jin))
    with art.ArtSweep(shape, nside, **kw) as sw:
        J = [np.empty(n, dt) for _ in fields]
        Jin = [np.empty(n, dt) for _ in fields]
        sw.sweep_stream([f[0].reshape(-1) for f in fields], [f[1].reshape(-1) for f in fields], J, Jin)
    for k in range(len(fields)):
        assert np.array_equal(J[k], want[k][0]) and np.array_equal(Jin[k], want[k][1])
