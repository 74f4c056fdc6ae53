"""The C-ABI library loads and exports every entry point include/oct.h declares,
and rejects invalid arguments before touching a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_01022_gb300 import nvcc_build as b
    path = b.build()
    return ctypes.CDLL(path)


def _declared():
    src = open(os.path.join(ROOT, "include", "oct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(oct_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_1705_01022_gb300 import _lib
    assert sorted(_lib.exported_symbols()) == _declared()


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_1705_01022_gb300 import _lib
    _lib.load()
    with pytest.raises(_lib.OctError) as e:
        _lib.oct_create(100, 1.0, 0.0, 1)  # not a multiple of 64
    assert e.value.code == _lib.OCT_EINVAL
    with pytest.raises(_lib.OctError) as e:
        _lib.oct_create(256, 1.5, 0.0, 1)
    assert e.value.code == _lib.OCT_EINVAL
    prm = _lib.oct_params()
    prm.L, prm.p, prm.q, prm.seed, prm.cx, prm.cy = 256, 1.0, 0.0, 1, 64, 8
    with pytest.raises(_lib.OctError) as e:
        _lib.oct_create_ex(prm)
    assert e.value.code == _lib.OCT_EUNSUPPORTED
    prm.cx, prm.cy, prm.scheme = 8, 8, _lib.OCT_SCHEME_DB  # coarse cells run DTrDT only
    with pytest.raises(_lib.OctError) as e:
        _lib.oct_create_ex(prm)
    assert e.value.code == _lib.OCT_EUNSUPPORTED
    prm.scheme = 0
    prm.cx, prm.cy, prm.Bx, prm.By = 4, 4, 48, 16
    with pytest.raises(_lib.OctError) as e:
        _lib.oct_create_ex(prm)
    assert e.value.code == _lib.OCT_EINVAL
    assert _lib.oct_destroy(None) is None
    assert _lib.oct_strerror(0) == "success"


def test_null_handles_rejected_without_gpu(lib):
    """Entry points that take a handle reject NULL with OCT_EINVAL before any CUDA call."""
    from paper_1705_01022_gb300 import _lib
    _lib.load()
    calls = [
        lambda: _lib.oct_run_mcs(None, 1),
        lambda: _lib.oct_measure_w2(None),
        lambda: _lib.oct_measure_w2_async(None),
        lambda: _lib.oct_w2_wait(None),
        lambda: _lib.oct_get_planes_async(None, 0, 16),
        lambda: _lib.oct_measure_ac(None),
        lambda: _lib.oct_snapshot(None),
        lambda: _lib.oct_get_stats(None),
    ]
    for call in calls:
        with pytest.raises(_lib.OctError) as e:
            call()
        assert e.value.code == _lib.OCT_EINVAL


def test_batch_replicas_validated_without_gpu(lib):
    """oct_batch_create checks every replica before any CUDA call."""
    from paper_1705_01022_gb300 import _lib
    _lib.load()
    bad = [
        dict(L=96),                       # not a multiple of 64
        dict(L=32768),                    # above 16384
        dict(L=256, p=1.5),               # p outside [0, 1]
        dict(L=256, Bx=48, By=16),        # Bx not a multiple of 32
        dict(L=256, Bx=64, By=48),        # By not a multiple of 16
        dict(L=192, Bx=64, By=64),        # 2 Bx does not divide L
        dict(L=4096, Bx=1024, By=32),     # 64 groups: more than a warp
        dict(L=256, Bx=96, By=16),        # 3 group columns: not a power of two
    ]
    for kw in bad:
        r = _lib.oct_replica()
        r.L, r.p, r.q, r.seed = kw.get("L", 256), kw.get("p", 1.0), 0.0, 1
        r.Bx, r.By = kw.get("Bx", 0), kw.get("By", 0)
        with pytest.raises(_lib.OctError) as e:
            _lib.oct_batch_create([r], None)
        assert e.value.code == _lib.OCT_EINVAL, kw
