"""ctypes binding of the C ABI in ``include/oct.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and raises
``OctError`` when that entry point returns a non-zero code.  There is no
fallback: if ``_build/liboct.so`` is missing the import of the library fails
loudly (build it with ``paper_1705_01022_gb300.build()``).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liboct.so")

OCT_OK, OCT_EINVAL, OCT_ENOMEM, OCT_ECUDA, OCT_ETIMEDOUT, OCT_EINTERNAL, OCT_EUNSUPPORTED = range(7)
OCT_SCHEME_DT, OCT_SCHEME_DB, OCT_SCHEME_DTR = 0, 1, 2


class OctError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func} failed with code {code}: {msg}")
        self.code = code


class oct_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("p", ctypes.c_double), ("q", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("Bx", ctypes.c_int32), ("By", ctypes.c_int32),
                ("cx", ctypes.c_int32), ("cy", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("lattice", ctypes.c_void_p), ("no_init", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("strip_row0", ctypes.c_int32), ("strip_rows", ctypes.c_int32),
                ("held_rows", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class oct_strip_sums(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("L", ctypes.c_int64), ("f", ctypes.c_int64), ("e_last", ctypes.c_int64),
                ("p1", ctypes.c_int64), ("p2_lo", ctypes.c_uint64), ("p2_hi", ctypes.c_uint64),
                ("lo", ctypes.c_int64), ("hi", ctypes.c_int64), ("t", ctypes.c_int64), ("net_flips", ctypes.c_int64)]


class oct_w2(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int64), ("n_sites", ctypes.c_int64), ("s1", ctypes.c_int64),
                ("s2_lo", ctypes.c_uint64), ("s2_hi", ctypes.c_uint64),
                ("net_flips", ctypes.c_int64), ("hmax", ctypes.c_int64), ("w2", ctypes.c_double)]

    @property
    def s2(self) -> int:
        return (int(self.s2_hi) << 64) | int(self.s2_lo)


class oct_info(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("t", ctypes.c_int64), ("Bx", ctypes.c_int32),
                ("By", ctypes.c_int32), ("cx", ctypes.c_int32), ("cy", ctypes.c_int32),
                ("p", ctypes.c_double), ("q", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("lattice", ctypes.c_void_p),
                ("lattice_bytes", ctypes.c_int64), ("scheme", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class oct_stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int64), ("net_flips", ctypes.c_int64), ("draws", ctypes.c_int64),
                ("tail_blocks", ctypes.c_int64)]


class oct_replica(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("p", ctypes.c_double), ("q", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("Bx", ctypes.c_int32), ("By", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]


class oct_ac(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int64), ("s", ctypes.c_int64), ("n_sites", ctypes.c_int64),
                ("sum_ht", ctypes.c_int64), ("sum_hs", ctypes.c_int64),
                ("cross_lo", ctypes.c_uint64), ("cross_hi", ctypes.c_int64),
                ("occ_x", ctypes.c_int64), ("occ_y", ctypes.c_int64),
                ("m_t", ctypes.c_int64), ("m_s", ctypes.c_int64),
                ("c_h", ctypes.c_double), ("c_s", ctypes.c_double),
                ("reserved", ctypes.c_int64 * 4)]

    @property
    def cross(self) -> int:
        """sum h(t) h(s) as a Python int (signed 128-bit)."""
        return (int(self.cross_hi) << 64) | int(self.cross_lo)


# (name, argtypes, restype) of every entry point declared in include/oct.h
_H = ctypes.c_void_p
_SIGNATURES = [
    ("oct_create", [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                    ctypes.POINTER(_H)], ctypes.c_int),
    ("oct_create_ex", [ctypes.POINTER(oct_params), ctypes.POINTER(_H)], ctypes.c_int),
    ("oct_run_mcs", [_H, ctypes.c_int64], ctypes.c_int),
    ("oct_device_step", [_H, ctypes.c_int], ctypes.c_int),
    ("oct_end_mcs", [_H], ctypes.c_int),
    ("oct_mcs_draw", [ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int64),
                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    ("oct_strip_measure", [_H, ctypes.POINTER(oct_strip_sums)], ctypes.c_int),
    ("oct_strip_combine", [ctypes.POINTER(oct_strip_sums), ctypes.c_int64, ctypes.POINTER(oct_w2)], ctypes.c_int),
    ("oct_measure_w2", [_H, ctypes.POINTER(oct_w2)], ctypes.c_int),
    ("oct_measure_w2_async", [_H], ctypes.c_int),
    ("oct_w2_wait", [_H, ctypes.POINTER(oct_w2)], ctypes.c_int),
    ("oct_get_lattice", [_H, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    ("oct_set_lattice", [_H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64], ctypes.c_int),
    ("oct_get_planes", [_H, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    ("oct_set_planes", [_H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int64], ctypes.c_int),
    ("oct_get_planes_async", [_H, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    ("oct_get_window", [_H, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                        ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    ("oct_get_info", [_H, ctypes.POINTER(oct_info)], ctypes.c_int),
    ("oct_sync", [_H], ctypes.c_int),
    ("oct_set_timing", [_H, ctypes.c_int], ctypes.c_int),
    ("oct_get_timing", [_H, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    ("oct_get_stats", [_H, ctypes.POINTER(oct_stats)], ctypes.c_int),
    ("oct_probe_int_rate", [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)],
     ctypes.c_int),
    ("oct_w2_noalloc", [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(oct_w2)],
     ctypes.c_int),
    ("oct_snapshot", [_H], ctypes.c_int),
    ("oct_measure_ac", [_H, ctypes.POINTER(oct_ac)], ctypes.c_int),
    ("oct_two_time_planes", [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                             ctypes.POINTER(oct_ac)], ctypes.c_int),
    ("oct_replica_seed", [ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)],
     ctypes.c_int),
    ("oct_batch_create", [ctypes.c_int64, ctypes.POINTER(oct_replica), ctypes.c_void_p,
                          ctypes.POINTER(_H)], ctypes.c_int),
    ("oct_batch_add", [_H, ctypes.POINTER(oct_replica), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    ("oct_batch_remove", [_H, ctypes.c_int64], ctypes.c_int),
    ("oct_batch_run", [_H, ctypes.c_int64], ctypes.c_int),
    ("oct_batch_measure_slot", [_H, ctypes.c_int64, ctypes.POINTER(oct_w2)], ctypes.c_int),
    ("oct_batch_measure_async", [_H, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    ("oct_batch_poll", [_H, ctypes.c_int64, ctypes.POINTER(oct_w2), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    ("oct_batch_wait", [_H, ctypes.c_int64, ctypes.POINTER(oct_w2)], ctypes.c_int),
    ("oct_batch_measure_w2", [_H, ctypes.POINTER(oct_w2), ctypes.c_int64], ctypes.c_int),
    ("oct_batch_get_planes", [_H, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
    ("oct_batch_snapshot", [_H, ctypes.c_int64], ctypes.c_int),
    ("oct_batch_measure_ac", [_H, ctypes.c_int64, ctypes.POINTER(oct_ac)], ctypes.c_int),
    ("oct_batch_get_stats", [_H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
     ctypes.c_int),
    ("oct_batch_sync", [_H], ctypes.c_int),
    ("oct_batch_mark", [_H, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    ("oct_batch_mark_done", [_H, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    ("oct_batch_mark_wait", [_H, ctypes.c_int64], ctypes.c_int),
    ("oct_batch_set_timing", [_H, ctypes.c_int], ctypes.c_int),
    ("oct_batch_get_timing", [_H, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
     ctypes.c_int),
    ("oct_batch_destroy", [_H], ctypes.c_int),
    ("oct_destroy", [_H], ctypes.c_int),
    ("oct_strerror", [ctypes.c_int], ctypes.c_char_p),
    ("oct_last_error", [], ctypes.c_char_p),
]

_lib = None


def load(path: str | None = None):
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"the CUDA library {p} is missing; build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        for name, args, res in _SIGNATURES:
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def exported_symbols():
    return [name for name, _, _ in _SIGNATURES]


def _check(rc: int, func: str):
    if rc != OCT_OK:
        msg = load().oct_last_error().decode(errors="replace")
        raise OctError(rc, func, msg)


def _ptr(buf) -> int:
    """Address of a numpy array or an integer address."""
    if isinstance(buf, int):
        return buf
    return buf.ctypes.data


# ---------------------------------------------------------------- wrappers --

def oct_create(L: int, p: float, q: float, seed: int) -> int:
    h = _H()
    _check(load().oct_create(L, p, q, seed, ctypes.byref(h)), "oct_create")
    return h.value


def oct_create_ex(prm: oct_params) -> int:
    h = _H()
    _check(load().oct_create_ex(ctypes.byref(prm), ctypes.byref(h)), "oct_create_ex")
    return h.value


def oct_run_mcs(h: int, n: int) -> None:
    _check(load().oct_run_mcs(h, n), "oct_run_mcs")


def oct_device_step(h: int, k: int) -> None:
    _check(load().oct_device_step(h, k), "oct_device_step")


def oct_end_mcs(h: int) -> None:
    _check(load().oct_end_mcs(h), "oct_end_mcs")


def oct_mcs_draw(seed: int, L: int, t: int):
    """(ox, oy, perm) of MCS t, as the kernels draw them."""
    ox, oy, perm = ctypes.c_int64(), ctypes.c_int64(), (ctypes.c_int32 * 4)()
    _check(load().oct_mcs_draw(seed, L, t, ctypes.byref(ox), ctypes.byref(oy), perm), "oct_mcs_draw")
    return ox.value, oy.value, list(perm)


def oct_strip_measure(h: int) -> oct_strip_sums:
    out = oct_strip_sums()
    _check(load().oct_strip_measure(h, ctypes.byref(out)), "oct_strip_measure")
    return out


def oct_strip_combine(parts) -> oct_w2:
    arr = (oct_strip_sums * len(parts))(*parts)
    out = oct_w2()
    _check(load().oct_strip_combine(arr, len(parts), ctypes.byref(out)), "oct_strip_combine")
    return out


def oct_measure_w2(h: int) -> oct_w2:
    out = oct_w2()
    _check(load().oct_measure_w2(h, ctypes.byref(out)), "oct_measure_w2")
    return out


def oct_measure_w2_async(h: int) -> None:
    _check(load().oct_measure_w2_async(h), "oct_measure_w2_async")


def oct_w2_wait(h: int) -> oct_w2:
    out = oct_w2()
    _check(load().oct_w2_wait(h, ctypes.byref(out)), "oct_w2_wait")
    return out


def oct_get_lattice(h: int, buf, words: int) -> None:
    _check(load().oct_get_lattice(h, _ptr(buf), words), "oct_get_lattice")


def oct_set_lattice(h: int, buf, words: int, t: int) -> None:
    _check(load().oct_set_lattice(h, _ptr(buf), words, t), "oct_set_lattice")


def oct_get_planes(h: int, buf, words: int) -> None:
    _check(load().oct_get_planes(h, _ptr(buf), words), "oct_get_planes")


def oct_get_planes_async(h: int, buf, words: int) -> None:
    """`buf` must stay alive, unread, until the handle's next synchronising call."""
    _check(load().oct_get_planes_async(h, _ptr(buf), words), "oct_get_planes_async")


def oct_set_planes(h: int, buf, words: int, t: int) -> None:
    _check(load().oct_set_planes(h, _ptr(buf), words, t), "oct_set_planes")


def oct_get_window(h: int, wx: int, wy: int, W: int, H: int, X, Y) -> None:
    _check(load().oct_get_window(h, wx, wy, W, H, _ptr(X), _ptr(Y)), "oct_get_window")


def oct_get_info(h: int) -> oct_info:
    out = oct_info()
    _check(load().oct_get_info(h, ctypes.byref(out)), "oct_get_info")
    return out


def oct_sync(h: int) -> None:
    _check(load().oct_sync(h), "oct_sync")


def oct_set_timing(h: int, enable: bool) -> None:
    _check(load().oct_set_timing(h, 1 if enable else 0), "oct_set_timing")


def oct_get_timing(h: int):
    ms, n, other = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    _check(load().oct_get_timing(h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(other)),
           "oct_get_timing")
    return ms.value, n.value, other.value


def oct_get_stats(h: int) -> oct_stats:
    out = oct_stats()
    _check(load().oct_get_stats(h, ctypes.byref(out)), "oct_get_stats")
    return out


def oct_probe_int_rate(op: int):
    r, mhz, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(load().oct_probe_int_rate(op, ctypes.byref(r), ctypes.byref(mhz), ctypes.byref(n)),
           "oct_probe_int_rate")
    return r.value, mhz.value, n.value


def oct_w2_noalloc(lattice: int, L: int, stream: int | None) -> oct_w2:
    out = oct_w2()
    _check(load().oct_w2_noalloc(lattice, L, stream, ctypes.byref(out)), "oct_w2_noalloc")
    return out


def oct_snapshot(h: int) -> None:
    _check(load().oct_snapshot(h), "oct_snapshot")


def oct_measure_ac(h: int) -> oct_ac:
    out = oct_ac()
    _check(load().oct_measure_ac(h, ctypes.byref(out)), "oct_measure_ac")
    return out


def oct_two_time_planes(lat_t: int, lat_s: int, L: int, stream: int | None) -> oct_ac:
    out = oct_ac()
    _check(load().oct_two_time_planes(lat_t, lat_s, L, stream, ctypes.byref(out)), "oct_two_time_planes")
    return out


def oct_replica_seed(master: int, r: int) -> int:
    out = ctypes.c_uint64()
    _check(load().oct_replica_seed(master, r, ctypes.byref(out)), "oct_replica_seed")
    return out.value


def oct_batch_create(reps, stream=None) -> int:
    arr = (oct_replica * max(1, len(reps)))(*reps)
    h = _H()
    _check(load().oct_batch_create(len(reps), arr, stream, ctypes.byref(h)), "oct_batch_create")
    return h.value


def oct_batch_add(h: int, rep: oct_replica) -> int:
    slot = ctypes.c_int64()
    _check(load().oct_batch_add(h, ctypes.byref(rep), ctypes.byref(slot)), "oct_batch_add")
    return slot.value


def oct_batch_remove(h: int, slot: int) -> None:
    _check(load().oct_batch_remove(h, slot), "oct_batch_remove")


def oct_batch_measure_slot(h: int, slot: int) -> oct_w2:
    out = oct_w2()
    _check(load().oct_batch_measure_slot(h, slot, ctypes.byref(out)), "oct_batch_measure_slot")
    return out


def oct_batch_measure_async(h: int, slot: int) -> int:
    t = ctypes.c_int64()
    _check(load().oct_batch_measure_async(h, slot, ctypes.byref(t)), "oct_batch_measure_async")
    return t.value


def oct_batch_poll(h: int, ticket: int):
    """The measurement of a ticket if it is done, else None."""
    out, ready = oct_w2(), ctypes.c_int()
    _check(load().oct_batch_poll(h, ticket, ctypes.byref(out), ctypes.byref(ready)), "oct_batch_poll")
    return out if ready.value else None


def oct_batch_wait(h: int, ticket: int) -> oct_w2:
    out = oct_w2()
    _check(load().oct_batch_wait(h, ticket, ctypes.byref(out)), "oct_batch_wait")
    return out


def oct_batch_run(h: int, n: int) -> None:
    _check(load().oct_batch_run(h, n), "oct_batch_run")


def oct_batch_measure_w2(h: int, n: int):
    out = (oct_w2 * n)()
    _check(load().oct_batch_measure_w2(h, out, n), "oct_batch_measure_w2")
    return list(out)


def oct_batch_snapshot(h: int, slot: int) -> None:
    _check(load().oct_batch_snapshot(h, slot), "oct_batch_snapshot")


def oct_batch_measure_ac(h: int, slot: int) -> oct_ac:
    out = oct_ac()
    _check(load().oct_batch_measure_ac(h, slot, ctypes.byref(out)), "oct_batch_measure_ac")
    return out


def oct_batch_get_planes(h: int, r: int, buf, words: int) -> None:
    _check(load().oct_batch_get_planes(h, r, _ptr(buf), words), "oct_batch_get_planes")


def oct_batch_get_stats(h: int):
    t, n, sites, draws = (ctypes.c_int64() for _ in range(4))
    _check(load().oct_batch_get_stats(h, ctypes.byref(t), ctypes.byref(n), ctypes.byref(sites),
                                      ctypes.byref(draws)), "oct_batch_get_stats")
    return t.value, n.value, sites.value, draws.value


def oct_batch_sync(h: int) -> None:
    _check(load().oct_batch_sync(h), "oct_batch_sync")


def oct_batch_mark(h: int) -> int:
    """Number of a mark at the point the batch's stream has reached."""
    m = ctypes.c_int64()
    _check(load().oct_batch_mark(h, ctypes.byref(m)), "oct_batch_mark")
    return m.value


def oct_batch_mark_done(h: int, mark: int) -> bool:
    done = ctypes.c_int()
    _check(load().oct_batch_mark_done(h, mark, ctypes.byref(done)), "oct_batch_mark_done")
    return bool(done.value)


def oct_batch_mark_wait(h: int, mark: int) -> None:
    _check(load().oct_batch_mark_wait(h, mark), "oct_batch_mark_wait")


def oct_batch_set_timing(h: int, enable: bool) -> None:
    _check(load().oct_batch_set_timing(h, 1 if enable else 0), "oct_batch_set_timing")


def oct_batch_get_timing(h: int):
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(load().oct_batch_get_timing(h, ctypes.byref(ms), ctypes.byref(n)), "oct_batch_get_timing")
    return ms.value, n.value


def oct_batch_destroy(h: int) -> None:
    _check(load().oct_batch_destroy(h), "oct_batch_destroy")


def oct_destroy(h: int) -> None:
    _check(load().oct_destroy(h), "oct_destroy")


def oct_strerror(code: int) -> str:
    return load().oct_strerror(code).decode()
