"""GPU strips of one lattice (the multi-GPU partition) run on one device: every
strip is a strip handle on its own buffer, the halo rows move by device
copies between device steps (strips.run_local), and no kernel waits for
another.  The strips together must equal the single-lattice run bit for bit
(and so the oracle), and the exactly combined W^2 must equal the
single-lattice measurement."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


CASES = [
    dict(L=256, nranks=2, By=32, Bx=64, p=0.95, q=0.05, scheme=0, cx=4, cy=4, n=4),
    dict(L=512, nranks=4, By=64, Bx=128, p=1.0, q=0.0, scheme=0, cx=4, cy=4, n=3),
    dict(L=1024, nranks=2, By=64, Bx=256, p=0.5, q=0.5, scheme=1, cx=4, cy=4, n=3),
    dict(L=512, nranks=2, By=32, Bx=64, p=0.6, q=0.3, scheme=2, cx=4, cy=4, n=3),
    dict(L=1024, nranks=4, By=64, Bx=256, p=0.95, q=0.05, scheme=0, cx=8, cy=8, n=2),
    dict(L=4096, nranks=8, By=64, Bx=256, p=0.95, q=0.05, scheme=0, cx=4, cy=4, n=2),
]


@pytest.mark.parametrize("c", CASES, ids=lambda c: "L{L}_n{nranks}_s{scheme}_TC{cx}x{cy}".format(**c))
def test_strips_equal_the_single_lattice_run(g, c):
    import torch

    from paper_1705_01022_gb300 import _lib, strips
    L, nr, By, Bx, seed = c["L"], c["nranks"], c["By"], c["Bx"], 31
    lays = [strips.StripLayout(L, By, nr, r) for r in range(nr)]
    engs = [strips.GpuStripEngine(lay, c["p"], c["q"], seed, Bx, cx=c["cx"], cy=c["cy"], scheme=c["scheme"])
            for lay in lays]
    try:
        with g.Simulation(L, c["p"], c["q"], seed, Bx=Bx, By=By, cx=c["cx"], cy=c["cy"], scheme=c["scheme"]) as ref:
            for step in range(c["n"]):
                strips.run_local(engs, lays, seed, 1)
                ref.run(1)
                torch.cuda.synchronize()
                whole = torch.cat([e.buf[:, :lay.H] for e, lay in zip(engs, lays)], dim=1).cpu().numpy()
                assert np.array_equal(whole.reshape(-1).view(np.uint32), ref.planes()), step
                got, want = strips.combine_local(engs), ref.measure()
                assert (got.s1, got.s2, got.hmax, got.net_flips, got.w2) == \
                    (want.s1, want.s2, want.hmax, want.net_flips, want.w2), step
    finally:
        for e in engs:
            e.close()


def test_device_steps_equal_run_mcs(g):
    """Four oct_device_step calls and oct_end_mcs equal oct_run_mcs(1)."""
    from paper_1705_01022_gb300 import _lib
    with g.Simulation(512, 0.95, 0.05, 3) as a, g.Simulation(512, 0.95, 0.05, 3) as b:
        for _ in range(3):
            a.run(1)
            for k in range(4):
                _lib.oct_device_step(b.h, k)
            _lib.oct_end_mcs(b.h)
        assert np.array_equal(a.planes(), b.planes()) and a.t == b.t == 3
        with pytest.raises(_lib.OctError):
            _lib.oct_device_step(b.h, 2)  # out of order
        with pytest.raises(_lib.OctError):
            _lib.oct_end_mcs(b.h)


def test_strip_handles_refuse_whole_lattice_calls(g):
    from paper_1705_01022_gb300 import _lib, strips
    lay = strips.StripLayout(256, 32, 2, 1)
    e = strips.GpuStripEngine(lay, 1.0, 0.0, 1, 64)
    try:
        for call in (lambda: _lib.oct_run_mcs(e.sim.h, 1), lambda: _lib.oct_measure_w2(e.sim.h),
                     lambda: e.sim.lattice()):
            with pytest.raises(_lib.OctError):
                call()
    finally:
        e.close()
    with pytest.raises(_lib.OctError):
        g.Simulation(256, 1.0, 0.0, 1, Bx=64, By=32, strip=(0, 96, 160))  # 96 is not a multiple of 2By
