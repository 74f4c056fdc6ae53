"""oct_w2_noalloc: the roughness entry point for callers that cannot allocate.

Some callers hand the library only a device buffer and a stream, for example
a framework that owns all device memory, or a latency-critical loop that must
not call cudaMalloc.  oct_w2_noalloc serves them from a fixed array compiled
into the library.  This test calls it through the C ABI and checks that it
returns exactly what the allocating oct_measure_w2 returns.  The checks cover
calls in a row on different lattices, so that scratch left over from one call
cannot leak into the next.  It also checks that a lattice above the stated
maximum is refused.

This file is collected last, so that a run that stops at the first failure
has already run every other test; it also passes on its own in a fresh
process."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


def _same(a, b):
    assert (a.s1, a.s2_lo, a.s2_hi, a.hmax, a.n_sites) == (b.s1, b.s2_lo, b.s2_hi, b.hmax, b.n_sites)
    assert a.w2 == b.w2


def test_noalloc_matches_measure_on_calls_in_a_row(g):
    from paper_1705_01022_gb300 import _lib
    big = g.Simulation(1024, 0.95, 0.05, 3, Bx=256, By=64)
    small = g.Simulation(256, 1.0, 0.0, 4)
    try:
        for sim, n in ((big, 5), (small, 7), (big, 2), (small, 1)):
            sim.run(n)
            ref = sim.measure()
            info = _lib.oct_get_info(sim.h)
            got = _lib.oct_w2_noalloc(info.lattice, sim.L, info.stream)
            _same(got, ref)
            assert got.t == -1 and got.net_flips == 0
            # a second call in a row on the unchanged lattice gives the same answer
            _same(_lib.oct_w2_noalloc(info.lattice, sim.L, info.stream), ref)
    finally:
        big.close()
        small.close()


def test_noalloc_on_torch_memory_and_default_stream(g):
    """A caller that owns the buffer (a torch tensor) and passes no stream."""
    torch = pytest.importorskip("torch")
    from paper_1705_01022_gb300 import _lib
    L = 512
    buf = torch.empty(L * L // 4, dtype=torch.uint8, device="cuda")
    with g.Simulation(L, 0.7, 0.3, 9, Bx=128, By=64, lattice=buf) as sim:
        sim.run(4)
        ref = sim.measure()
        torch.cuda.synchronize()
        _same(_lib.oct_w2_noalloc(buf.data_ptr(), L, None), ref)
        sim.run(1)
        ref2 = sim.measure()
        torch.cuda.synchronize()
        _same(_lib.oct_w2_noalloc(buf.data_ptr(), L, None), ref2)
        assert ref2.s2 != ref.s2 or ref2.s1 != ref.s1


def test_noalloc_rejects_oversize_and_bad_arguments(g):
    from paper_1705_01022_gb300 import _lib
    with g.Simulation(256, 1.0, 0.0, 1) as sim:
        info = _lib.oct_get_info(sim.h)
        with pytest.raises(_lib.OctError) as e:
            _lib.oct_w2_noalloc(info.lattice, 2**18, info.stream)
        assert e.value.code == _lib.OCT_EINVAL
        assert "131072" in str(e.value)
        with pytest.raises(_lib.OctError) as e:
            _lib.oct_w2_noalloc(info.lattice, 100, info.stream)
        assert e.value.code == _lib.OCT_EINVAL
        with pytest.raises(_lib.OctError):
            _lib.oct_w2_noalloc(0, 256, info.stream)
        # the handle is unaffected by refused calls
        ref = sim.measure()
        _same(_lib.oct_w2_noalloc(info.lattice, 256, info.stream), ref)
