"""The benchmark's CPU legs (the oracle on the host cores), on CPU: the
spawn-started pool replays one window per core, the reference arm prints its
JSON line with the cores it used, and O1 reports a rate."""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _args(**kw):
    d = dict(L=1024, p=0.95, q=0.05, seed=1, Bx=256, By=64, steps=2, warmup=1, ref_cores=2)
    d.update(kw)
    return argparse.Namespace(**d)


def test_host_cores_replay_every_core_once(oracle):
    import bench
    prm = oracle.Params(L=1024, p=0.95, q=0.05, seed=3, Bx=256, By=64)
    ox, oy, _ = oracle.mcs_draw(prm, 0)
    W, H = 512 + 1, 128 + 1
    xs, ys = (ox + np.arange(W)) % 1024, (oy + np.arange(H)) % 1024
    flat = ((xs[None, :] + ys[:, None]) & 1).astype(np.uint8)
    cores = bench.HostCores(2)
    try:
        total, wall, per = cores.replay(flat, flat, prm, 0, ox, oy, 512 * 128)
    finally:
        cores.close()
    assert total == 2 * 512 * 128 and len(per) == 2
    assert wall > 0 and all(s > 0 for s in per)
    # the window in the caller is untouched (each core replays its own copy)
    assert np.array_equal(flat, ((xs[None, :] + ys[:, None]) & 1).astype(np.uint8))


def test_reference_arm_line(oracle):
    import bench
    out = bench.run_reference(_args(), rank=0, world=1)
    assert out["impl"] == "reference" and out["value"] > 0
    assert out["cpu_baseline"]["cores"] == 2 and out["cpu_baseline"]["kind"] == "oracle"
    assert out["e2e"]["h2d_bytes_per_step"] == 0
    assert bench.run_reference(_args(), rank=1, world=2) is None


def test_sequential_rs_rate(oracle):
    import bench
    r = bench.cpu_sequential_rs(oracle, L=256, target_s=0.05)
    assert r["value"] > 0 and r["cores"] == 1 and "L=256" in r["sample"]
