"""Statistics of the GPU dynamics against what the paper fixes.

* KPZ (p = 1, q = 0): the effective growth exponent of Eq. (8) on W(t) lies
  near the paper's beta = 0.2414(2) (Sec. 2) at L = 4096 over t in [100, 1000]
  (finite-time corrections are expected, Sec. 4.2).
* EW (p = q = 0.5): roughening is logarithmic, so beta_eff is small.
* W^2(t) against true random-sequential updating (oracle O1): the paper
  reports that fine decomposition lowers the roughness prefactor (Sec. 4.2);
  with 4 x 4 thread cells the GPU's W^2 sits a few percent below RS at every
  t.  The test requires that band and prints the z-scores rather than
  requiring |z| < 3, which the method does not satisfy at high statistics.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


def _w2_series(g, L, p, q, seeds, ts):
    out = np.zeros((len(seeds), len(ts)))
    for i, s in enumerate(seeds):
        with g.Simulation(L, p, q, s) as sim:
            t = 0
            for j, tt in enumerate(ts):
                sim.run(tt - t)
                t = tt
                out[i, j] = sim.measure().w2
    return out


def test_kpz_growth_exponent(g):
    ts = [100, 1000]
    w2 = _w2_series(g, 4096, 1.0, 0.0, range(1, 5), ts).mean(axis=0)
    beta = 0.5 * math.log(w2[1] / w2[0]) / math.log(ts[1] / ts[0])
    print(f"beta_eff(100..1000, L=4096) = {beta:.4f}")
    assert 0.22 < beta < 0.26, beta


def test_ew_roughening_is_logarithmic(g):
    ts = [100, 1000]
    w2 = _w2_series(g, 2048, 0.5, 0.5, range(1, 5), ts).mean(axis=0)
    beta = 0.5 * math.log(w2[1] / w2[0]) / math.log(ts[1] / ts[0])
    print(f"EW beta_eff(100..1000, L=2048) = {beta:.4f}")
    assert 0.0 < beta < 0.12, beta
    # W^2 grows by about (1/(2*pi*sigma)) ln t: roughly linear in ln t
    w2s = _w2_series(g, 1024, 0.5, 0.5, range(1, 5), [10, 100, 1000]).mean(axis=0)
    d1, d2 = w2s[1] - w2s[0], w2s[2] - w2s[1]
    assert 0.5 < d2 / d1 < 1.5, (d1, d2)


def test_roughness_against_sequential_rs(g, oracle):
    L, n, ts = 512, 16, [4, 16, 48]
    gpu = _w2_series(g, L, 1.0, 0.0, range(100, 100 + n), ts)
    rs = np.zeros((n, len(ts)))
    for i in range(n):
        X, Y = oracle.flat(L)
        t = 0
        for j, tt in enumerate(ts):
            oracle.seq_rs(X, Y, 1.0, 0.0, 5000 + i, t, tt - t)
            t = tt
            rs[i, j] = oracle.w2(X, Y)
    ratio = gpu.mean(0) / rs.mean(0)
    z = (gpu.mean(0) - rs.mean(0)) / np.sqrt(gpu.var(0, ddof=1) / n + rs.var(0, ddof=1) / n)
    print("t", ts, "GPU/RS W^2 ratio", np.round(ratio, 4), "z", np.round(z, 2))
    assert np.all((ratio > 0.92) & (ratio < 1.0)), ratio
