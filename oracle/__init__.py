"""CPU oracle for the octahedron-model DTrDT simulation -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product path (the CUDA
library in ``paper_1705_01022_gb300``) never imports it, and the two share no
code.

The arithmetic lives in ``oct_oracle.c`` (plain C, one site and one attempt at
a time); this module only compiles it with gcc and marshals numpy arrays.

Lattices are pairs of ``uint8`` arrays ``X, Y`` of shape ``(L, L)`` indexed
``[y, x]``: ``X[y, x] = 1`` iff ``h(x,y) - h(x-1,y) = +1`` and ``Y[y, x] = 1``
iff ``h(x,y) - h(x,y-1) = +1`` (the paper's on-site slope convention, Sec. 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oct_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboct_oracle.so")
_lib = None

TAG_MCS, TAG_SET, TAG_SITE, TAG_ACC, TAG_SEQ, TAG_REPLICA, TAG_TAIL, TAG_SITE_DB, TAG_BORG = 1, 2, 3, 4, 5, 6, 7, 8, 9
SCHEME_DT, SCHEME_DB, SCHEME_DB_IGNORE, SCHEME_DTR = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, C11, -O2)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oct_oracle.h")))
    if force or not fresh:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("Bx", ctypes.c_int64), ("By", ctypes.c_int64),
                ("cx", ctypes.c_int64), ("cy", ctypes.c_int64), ("p", ctypes.c_double),
                ("q", ctypes.c_double), ("seed", ctypes.c_uint64), ("scheme", ctypes.c_int64)]


@dataclass(frozen=True)
class Params:
    """DTrDT parameters: lattice L, sub-tile Bx x By, thread cell cx x cy (sites)."""
    L: int
    p: float
    q: float
    seed: int
    Bx: int = 64
    By: int = 64
    cx: int = 4
    cy: int = 4
    scheme: int = 0  # SCHEME_DT, SCHEME_DB, SCHEME_DB_IGNORE or SCHEME_DTR

    def c(self) -> _Params:
        return _Params(self.L, self.Bx, self.By, self.cx, self.cy, self.p, self.q, self.seed,
                       self.scheme)


_P_u8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_P_u32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_P_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i64, u32, u64, dbl = ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double
        P_i64 = ctypes.POINTER(ctypes.c_int64)
        P_u64 = ctypes.POINTER(ctypes.c_uint64)
        L.oo_philox4x32_10.argtypes = [_P_u32, _P_u32, _P_u32]
        L.oo_threshold32.argtypes = [dbl]
        L.oo_threshold32.restype = u64
        L.oo_init_flat.argtypes = [i64, _P_u8, _P_u8]
        L.oo_site_kind.argtypes = [i64, _P_u8, _P_u8, i64, i64]
        L.oo_attempt.argtypes = [i64, _P_u8, _P_u8, i64, i64, dbl, dbl, u32,
                                 ctypes.POINTER(ctypes.c_int)]
        L.oo_seq_rs.argtypes = [i64, dbl, dbl, u64, _P_u8, _P_u8, u32, u32, P_i64]
        L.oo_seq_rs_many.argtypes = [i64, dbl, dbl, u64, i64, u32, _P_u8, _P_u8]
        L.oo_check_params.argtypes = [ctypes.POINTER(_Params)]
        L.oo_mcs_draw.argtypes = [ctypes.POINTER(_Params), u32, P_i64, P_i64,
                                  ctypes.POINTER(ctypes.c_int)]
        L.oo_dtrdt_run.argtypes = [ctypes.POINTER(_Params), _P_u8, _P_u8, u32, u32, P_i64,
                                   ctypes.c_void_p, P_i64]
        L.oo_dtrdt_mcs_window.argtypes = [ctypes.POINTER(_Params), u32, i64, i64, i64, i64,
                                          _P_u8, _P_u8, P_i64]
        L.oo_w2_sums.argtypes = [i64, _P_u8, _P_u8, P_i64, P_u64, P_u64, P_i64]
        L.oo_w2_sums_colfirst.argtypes = [i64, _P_u8, _P_u8, P_i64, P_u64, P_u64]
        L.oo_w2_from_sums.argtypes = [i64, i64, u64, u64]
        L.oo_w2_from_sums.restype = dbl
        L.oo_invariants.argtypes = [i64, _P_u8, _P_u8]
        L.oo_pack_canonical.argtypes = [i64, _P_u8, _P_u8, _P_u32]
        L.oo_unpack_canonical.argtypes = [i64, _P_u32, _P_u8, _P_u8]
        L.oo_dtrdt_many.argtypes = [ctypes.POINTER(_Params), u64, i64, u32, _P_u8, _P_u8]
        L.oo_dtrdt_acc_prefix.argtypes = [u64, u32, u32, u32, u32, u32, ctypes.c_int]
        L.oo_dtrdt_acc_prefix.restype = u32
        L.oo_dtrdt_tail_word.argtypes = [u64, u32, u32, u32, u32, u32]
        L.oo_dtrdt_tail_word.restype = u32
        L.oo_w2_sums_planar.argtypes = [i64, _P_u32, P_i64, P_u64, P_u64, P_i64]
        L.oo_invariants_planar.argtypes = [i64, _P_u32, i64, i64]
        L.oo_replica_seed.argtypes = [u64, u32]
        L.oo_replica_seed.restype = u64
        L.oo_subtile_step_sites.argtypes = [ctypes.POINTER(_Params), u32, u32, u32, i64, _P_i64, _P_i64]
        L.oo_subtile_steps_many.argtypes = [ctypes.POINTER(_Params), u64, i64, u32, u32, u32, i64, i64,
                                            i64, _P_u8, _P_u8, _P_u8, _P_u8, _P_i64]
        L.oo_device_step_strip.argtypes = [ctypes.POINTER(_Params), u32, u32, i64, i64, i64, _P_u8, _P_u8, P_i64]
        L.oo_set_plant.argtypes = [ctypes.c_int]
        L.oo_set_tie_log.argtypes = [ctypes.c_void_p, i64]
        L.oo_tie_log_count.restype = i64
        L.oo_two_time_sums.argtypes = [i64, _P_u8, _P_u8, _P_u8, _P_u8, ctypes.POINTER(_TwoTime)]
        L.oo_ch_from_sums.argtypes = [i64, ctypes.POINTER(_TwoTime)]
        L.oo_ch_from_sums.restype = dbl
        L.oo_cs_from_sums.argtypes = [i64, ctypes.POINTER(_TwoTime)]
        L.oo_cs_from_sums.restype = dbl
        _lib = L
    return _lib


# ---------------------------------------------------------------- helpers ---

def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oo_philox4x32_10(c, k, out)
    return out


def threshold32(p: float) -> int:
    return int(lib().oo_threshold32(float(p)))


def flat(L: int):
    X = np.zeros((L, L), dtype=np.uint8)
    Y = np.zeros((L, L), dtype=np.uint8)
    lib().oo_init_flat(L, X, Y)
    return X, Y


def site_kind(X, Y, x: int, y: int) -> int:
    return int(lib().oo_site_kind(X.shape[0], X, Y, x, y))


def attempt(X, Y, x: int, y: int, p: float, q: float, u: int):
    kind = ctypes.c_int(0)
    r = lib().oo_attempt(X.shape[0], X, Y, x, y, p, q, u & 0xFFFFFFFF, ctypes.byref(kind))
    return int(r), int(kind.value)


def seq_rs(X, Y, p: float, q: float, seed: int, t0: int, n_mcs: int) -> int:
    """O1: sequential RS for n_mcs sweeps, in place.  Returns net flips."""
    net = ctypes.c_int64(0)
    lib().oo_seq_rs(X.shape[0], p, q, seed, X, Y, t0, n_mcs, ctypes.byref(net))
    return int(net.value)


def seq_rs_many(L: int, p: float, q: float, seed0: int, n_runs: int, n_mcs: int):
    X = np.zeros((n_runs, L, L), dtype=np.uint8)
    Y = np.zeros((n_runs, L, L), dtype=np.uint8)
    lib().oo_seq_rs_many(L, p, q, seed0, n_runs, n_mcs, X, Y)
    return X, Y


def check_params(prm: Params) -> bool:
    cp = prm.c()
    return lib().oo_check_params(ctypes.byref(cp)) == 0


def mcs_draw(prm: Params, t: int):
    cp = prm.c()
    ox, oy = ctypes.c_int64(), ctypes.c_int64()
    perm = (ctypes.c_int * 4)()
    lib().oo_mcs_draw(ctypes.byref(cp), t, ctypes.byref(ox), ctypes.byref(oy), perm)
    return int(ox.value), int(oy.value), list(perm)


def dtrdt_run(X, Y, prm: Params, t0: int, n_mcs: int, count_attempts: bool = False,
              check_conflicts: bool = False):
    """O2: DTrDT replay in place.  Returns (net_flips, attempts or None, conflicts or None)."""
    cp = prm.c()
    net = ctypes.c_int64(0)
    att = np.zeros((prm.L, prm.L), dtype=np.int64) if count_attempts else None
    conf = ctypes.c_int64(0)
    rc = lib().oo_dtrdt_run(ctypes.byref(cp), X, Y, t0, n_mcs, ctypes.byref(net),
                            att.ctypes.data_as(ctypes.c_void_p) if att is not None else None,
                            ctypes.byref(conf) if check_conflicts else None)
    if rc != 0:
        raise ValueError(f"invalid DTrDT parameters {prm}")
    return int(net.value), att, (int(conf.value) if check_conflicts else None)


def dtrdt_many(prm: Params, seed0: int, n_runs: int, n_mcs: int):
    """O2 from the flat start for seeds seed0 .. seed0+n_runs-1; returns final (X, Y) stacks."""
    cp = prm.c()
    X = np.zeros((n_runs, prm.L, prm.L), dtype=np.uint8)
    Y = np.zeros((n_runs, prm.L, prm.L), dtype=np.uint8)
    if lib().oo_dtrdt_many(ctypes.byref(cp), seed0, n_runs, n_mcs, X, Y) != 0:
        raise ValueError(f"invalid DTrDT parameters {prm}")
    return X, Y


def acc_prefix(seed: int, t: int, k: int, T: int, g: int, s: int, pos: int) -> int:
    """Bits 31..28 of the acceptance uniform of the thread cell at position pos of group g."""
    return int(lib().oo_dtrdt_acc_prefix(seed, t, k, T, g, s, pos))


def tail_word(seed: int, t: int, k: int, T: int, g: int, i: int) -> int:
    """Word i of group g's tail stream in device step k of MCS t (sub-tile T)."""
    return int(lib().oo_dtrdt_tail_word(seed, t, k, T, g, i))


def dtrdt_mcs_window(Xw, Yw, prm: Params, t: int, wx: int, wy: int) -> int:
    """O2 for one MCS on a window (H, W) whose corner is global site (wx, wy)."""
    cp = prm.c()
    H, W = Xw.shape
    net = ctypes.c_int64(0)
    rc = lib().oo_dtrdt_mcs_window(ctypes.byref(cp), t, wx, wy, W, H, Xw, Yw, ctypes.byref(net))
    if rc != 0:
        raise ValueError("invalid window replay arguments")
    return int(net.value)


def w2_sums(X, Y):
    """O3: (S1, S2, hmax) over heights relative to h(0,0) = 0 (exact Python ints)."""
    s1, lo, hi, hm = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int64()
    lib().oo_w2_sums(X.shape[0], X, Y, ctypes.byref(s1), ctypes.byref(lo), ctypes.byref(hi),
                     ctypes.byref(hm))
    return int(s1.value), (int(hi.value) << 64) | int(lo.value), int(hm.value)


def w2_sums_colfirst(X, Y):
    s1, lo, hi = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
    lib().oo_w2_sums_colfirst(X.shape[0], X, Y, ctypes.byref(s1), ctypes.byref(lo),
                              ctypes.byref(hi))
    return int(s1.value), (int(hi.value) << 64) | int(lo.value)


def w2_from_sums(L: int, s1: int, s2: int) -> float:
    return float(lib().oo_w2_from_sums(L, s1, s2 & ((1 << 64) - 1), s2 >> 64))


def w2(X, Y) -> float:
    s1, s2, _ = w2_sums(X, Y)
    return w2_from_sums(X.shape[0], s1, s2)


def subtile_step_sites(prm: "Params", t: int, k: int, T: int, s: int):
    """Local sites (lx, ly) of every thread cell's attempt in collective step s
    of sub-tile T (device step k of MCS t); index = TC row * (Bx/cx) + TC column."""
    n = (prm.Bx // prm.cx) * (prm.By // prm.cy)
    lx = np.zeros(n, dtype=np.int64)
    ly = np.zeros(n, dtype=np.int64)
    if lib().oo_subtile_step_sites(ctypes.byref(prm.c()), t, k, T, s, lx, ly) != 0:
        raise ValueError("invalid parameters")
    return lx, ly


def device_step_strip(Xs, Ys, prm: "Params", t: int, k: int, a: int, Hs: int) -> int:
    """Device step k of MCS t on the row strip [a, a + Hs) of the multi-GPU
    partition, in place on the held rows (Xs, Ys) (shape (rows, L), first row
    = global row a).  Returns the net flips."""
    net = ctypes.c_int64(0)
    rc = lib().oo_device_step_strip(ctypes.byref(prm.c()), t, k, a, Hs, Xs.shape[0], Xs, Ys, ctypes.byref(net))
    if rc != 0:
        raise ValueError(f"strip step failed ({rc})")
    return int(net.value)


def subtile_steps_many(prm: "Params", seed0: int, n_runs: int, t: int, k: int, T: int, x0: int, y0: int,
                       n_steps: int, X0, Y0):
    """The first n_steps collective steps of one sub-tile (at (x0, y0)) alone,
    once per seed seed0 + r from the lattice (X0, Y0).  Returns the stacks of
    resulting lattices (X, Y) and the net flips of each run."""
    L = prm.L
    X = np.zeros((n_runs, L, L), dtype=np.uint8)
    Y = np.zeros((n_runs, L, L), dtype=np.uint8)
    net = np.zeros(n_runs, dtype=np.int64)
    rc = lib().oo_subtile_steps_many(ctypes.byref(prm.c()), seed0, n_runs, t, k, T, x0, y0, n_steps,
                                     np.ascontiguousarray(X0, dtype=np.uint8),
                                     np.ascontiguousarray(Y0, dtype=np.uint8), X, Y, net)
    if rc != 0:
        raise ValueError("invalid parameters")
    return X, Y, net


class tie_log:
    """Context manager recording the tail words tied candidates take (rows of
    stream group, word index, candidate group, position) while it is open."""

    def __init__(self, cap: int = 1 << 16):
        self.buf = np.zeros((cap, 4), dtype=np.int64)

    def __enter__(self):
        lib().oo_set_tie_log(self.buf.ctypes.data_as(ctypes.c_void_p), self.buf.shape[0])
        return self

    def __exit__(self, *exc):
        self.n = int(lib().oo_tie_log_count())
        lib().oo_set_tie_log(None, 0)
        return False

    def rows(self):
        return self.buf[: self.n]


class planted:
    """Context manager that plants one of the oracle's known mistakes (1: cells
    2i and 2i+1 share site bits; 2: DTrDB corners before borders; 3: all groups
    take tail words from group 0's stream) for a negative control, and removes
    it on exit."""

    def __init__(self, which: int):
        self.which = which

    def __enter__(self):
        lib().oo_set_plant(self.which)
        return self

    def __exit__(self, *exc):
        lib().oo_set_plant(0)
        return False


class _TwoTime(ctypes.Structure):
    _fields_ = [("sum_ht", ctypes.c_int64), ("sum_hs", ctypes.c_int64),
                ("cross_lo", ctypes.c_uint64), ("cross_hi", ctypes.c_int64),
                ("occ_x", ctypes.c_int64), ("occ_y", ctypes.c_int64),
                ("m_t", ctypes.c_int64), ("m_s", ctypes.c_int64)]


def two_time(Xt, Yt, Xs, Ys) -> dict:
    """Two-time sums and C_h(t,s), C_s(t,s) of one sample (Sec. 2): lattice
    (Xt, Yt) at time t against (Xs, Ys) at the waiting time s.  Integer sums
    are exact Python ints; 'cross' = sum h(t) h(s)."""
    L = Xt.shape[0]
    a = _TwoTime()
    arrs = [np.ascontiguousarray(v, dtype=np.uint8) for v in (Xt, Yt, Xs, Ys)]
    lib().oo_two_time_sums(L, *arrs, ctypes.byref(a))
    cross = (int(a.cross_hi) << 64) | int(a.cross_lo)
    return {"sum_ht": int(a.sum_ht), "sum_hs": int(a.sum_hs), "cross": cross,
            "occ_x": int(a.occ_x), "occ_y": int(a.occ_y), "m_t": int(a.m_t), "m_s": int(a.m_s),
            "c_h": float(lib().oo_ch_from_sums(L, ctypes.byref(a))),
            "c_s": float(lib().oo_cs_from_sums(L, ctypes.byref(a)))}


def w2_sums_planar(words, L: int):
    """O3 on the bit-packed planar layout: (S1, S2, hmax)."""
    s1, lo, hi, hm = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int64()
    lib().oo_w2_sums_planar(L, np.ascontiguousarray(words, dtype=np.uint32), ctypes.byref(s1),
                            ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(hm))
    return int(s1.value), (int(hi.value) << 64) | int(lo.value), int(hm.value)


def invariants_planar(words, L: int, circ_rows=None) -> int:
    y0, y1 = (0, L) if circ_rows is None else circ_rows
    return int(lib().oo_invariants_planar(L, np.ascontiguousarray(words, dtype=np.uint32), y0, y1))


def pack_planar(X, Y) -> np.ndarray:
    """Byte arrays -> planar words (X plane then Y plane); numpy bit packing."""
    L = X.shape[0]
    bits = np.stack([X, Y]).astype(np.uint8)
    packed = np.packbits(bits.reshape(2, L, L // 8, 8), axis=-1, bitorder="little")
    return packed.reshape(-1).view(np.uint32).copy()


def invariants(X, Y) -> int:
    return int(lib().oo_invariants(X.shape[0], X, Y))


def pack_canonical(X, Y) -> np.ndarray:
    L = X.shape[0]
    w = np.zeros((L // 4) * (L // 4), dtype=np.uint32)
    lib().oo_pack_canonical(L, X, Y, w)
    return w


def unpack_canonical(words, L: int):
    X = np.zeros((L, L), dtype=np.uint8)
    Y = np.zeros((L, L), dtype=np.uint8)
    lib().oo_unpack_canonical(L, np.ascontiguousarray(words, dtype=np.uint32), X, Y)
    return X, Y


def replica_seed(master: int, r: int) -> int:
    return int(lib().oo_replica_seed(master, r))
