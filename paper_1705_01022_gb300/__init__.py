"""GB300-native octahedron-model (2+1-d KPZ) simulator under DTrDT decomposition.

The compute path is the CUDA library built from ``csrc/`` (sm_103a) behind the
C ABI of ``include/oct.h``; ``_lib`` binds it with ctypes.  ``Simulation`` is a
small convenience wrapper around one handle.  PyTorch is optional and only
supplies streams and device memory.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import OctError, oct_ac, oct_params, oct_w2  # noqa: F401


def build(force: bool = False) -> str:
    from .nvcc_build import build as _build
    return _build(force=force)


class Simulation:
    """One simulation handle.

    ``stream``: a ``torch.cuda.Stream`` (or raw cudaStream_t address) to run on;
    ``lattice``: an external device buffer (a torch tensor or raw address) of
    L*L/4 bytes (held_rows*L/4 for a strip) that the handle uses in place of
    its own allocation; ``strip``: (first row, rows owned, rows held) when the
    handle holds one row strip of a lattice split over devices."""

    def __init__(self, L: int, p: float, q: float, seed: int, Bx: int = 0, By: int = 0,
                 cx: int = 0, cy: int = 0, stream=None, lattice=None, no_init: bool = False,
                 scheme: int = 0, strip=None):
        prm = oct_params()
        if strip is not None:  # (first row, rows owned, rows held) of a row strip (see strips.py)
            prm.strip_row0, prm.strip_rows, prm.held_rows = strip
        prm.L, prm.p, prm.q, prm.seed = L, p, q, seed
        prm.Bx, prm.By, prm.cx, prm.cy = Bx, By, cx, cy
        prm.stream = _address(stream, "cuda_stream")
        prm.lattice = _address(lattice, "data_ptr")
        prm.no_init = 1 if no_init else 0
        prm.scheme = scheme
        self._keep = (stream, lattice)
        self.h = _lib.oct_create_ex(prm)
        info = _lib.oct_get_info(self.h)
        self.L, self.Bx, self.By, self.cx, self.cy = L, info.Bx, info.By, info.cx, info.cy
        self.p, self.q, self.seed = p, q, seed

    @property
    def t(self) -> int:
        return _lib.oct_get_info(self.h).t

    def run(self, n: int) -> None:
        _lib.oct_run_mcs(self.h, n)

    def measure(self) -> oct_w2:
        return _lib.oct_measure_w2(self.h)

    def measure_async(self) -> None:
        """Enqueues a W^2 measurement of the lattice as it stands; `w2_wait` returns it."""
        _lib.oct_measure_w2_async(self.h)

    def w2_wait(self) -> oct_w2:
        return _lib.oct_w2_wait(self.h)

    def snapshot(self) -> None:
        """Stores the current lattice as the state at the waiting time s = t."""
        _lib.oct_snapshot(self.h)

    def measure_ac(self) -> oct_ac:
        """C_h(t,s) and C_s(t,s) of the current lattice against the last snapshot."""
        return _lib.oct_measure_ac(self.h)

    def lattice(self) -> np.ndarray:
        w = np.empty(self.L * self.L // 16, dtype=np.uint32)
        _lib.oct_get_lattice(self.h, w, w.size)
        return w

    def set_lattice(self, words: np.ndarray, t: int) -> None:
        w = np.ascontiguousarray(words, dtype=np.uint32)
        _lib.oct_set_lattice(self.h, w, w.size, t)

    def planes(self) -> np.ndarray:
        w = np.empty(self.L * self.L // 16, dtype=np.uint32)
        _lib.oct_get_planes(self.h, w, w.size)
        return w

    def window(self, wx: int, wy: int, W: int, H: int):
        X = np.empty((H, W), dtype=np.uint8)
        Y = np.empty((H, W), dtype=np.uint8)
        _lib.oct_get_window(self.h, wx, wy, W, H, X, Y)
        return X, Y

    def sync(self) -> None:
        _lib.oct_sync(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            _lib.oct_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy: the legacy default stream


class Batch:
    """Many independent replicas advanced together (see oct_batch_* in include/oct.h).

    ``replicas``: iterable of (L, p, q, seed) or (L, p, q, seed, Bx, By)."""

    def __init__(self, replicas, stream=None):
        reps = []
        for r in replicas:
            o = _lib.oct_replica()
            o.L, o.p, o.q, o.seed = int(r[0]), float(r[1]), float(r[2]), int(r[3])
            if len(r) > 4:
                o.Bx, o.By = int(r[4]), int(r[5])
            reps.append(o)
        self.replicas = reps
        self._keep = stream
        self.h = _lib.oct_batch_create(reps, _address(stream, "cuda_stream"))

    def __len__(self):
        return len(self.replicas)

    def run(self, n: int) -> None:
        _lib.oct_batch_run(self.h, n)

    def measure(self):
        return _lib.oct_batch_measure_w2(self.h, len(self.replicas))

    def snapshot(self, r: int) -> None:
        """Stores replica r's current lattice as its state at the waiting time s."""
        _lib.oct_batch_snapshot(self.h, r)

    def measure_ac(self, r: int) -> oct_ac:
        """C_h(t,s), C_s(t,s) of replica r against its last snapshot."""
        return _lib.oct_batch_measure_ac(self.h, r)

    def planes(self, r: int) -> np.ndarray:
        L = self.replicas[r].L
        w = np.empty(L * L // 16, dtype=np.uint32)
        _lib.oct_batch_get_planes(self.h, r, w, w.size)
        return w

    def stats(self):
        return _lib.oct_batch_get_stats(self.h)

    def sync(self) -> None:
        _lib.oct_batch_sync(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            _lib.oct_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def two_time(lat_t, lat_s, L: int, stream=None) -> oct_ac:
    """C_h(t,s), C_s(t,s) of two planar device lattices (torch tensors or raw
    addresses of L*L/4 bytes each), e.g. a batched replica and a copy of it."""
    return _lib.oct_two_time_planes(_address(lat_t, "data_ptr"), _address(lat_s, "data_ptr"), L,
                                    _address(stream, "cuda_stream"))


def _address(obj, attr: str):
    if obj is None:
        return None
    if isinstance(obj, int):
        return obj
    v = getattr(obj, attr)
    v = v() if callable(v) else v
    if attr == "cuda_stream" and v == 0:
        # a torch stream object for the legacy default stream has handle 0,
        # which the C ABI reads as "no stream given"
        return _CUDA_STREAM_LEGACY
    return v


def planes_to_bits(words: np.ndarray, L: int):
    """Unpack the planar layout to per-site byte arrays X[y, x], Y[y, x]."""
    w = words.reshape(2, L, L // 32)
    bits = np.unpackbits(w.view(np.uint8).reshape(2, L, L // 32, 4), axis=-1, bitorder="little")
    bits = bits.reshape(2, L, L)
    return bits[0].copy(), bits[1].copy()
