"""PRNGD oracle: test infrastructure only.

A ctypes wrapper around ``prngd_oracle.c``, the plain exact CPU implementation of the
extended-precision uniform construction of Demchik and Gulov (arXiv:1401.8230, Section 2:
Eq. 1, the discrete accept-reject rule, Eq. 4 and Algorithm 1).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The CUDA library never does, and this package imports nothing from it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prngd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FORM_A, FORM_B, FORM_C, FORM_N, FORM_L = 0, 1, 2, 3, 4
# Mode bits: Eq. (5)/(6) map, 1 - z, Algorithm 1's single-redraw rejects (0: Eq. (4), pairs).
MODE_EQ5, MODE_ONE_MINUS, MODE_SINGLE = 1, 2, 4

_U64P = ctypes.POINTER(ctypes.c_uint64)
_U32P = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into a shared library next to its source."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_splitmix64_output.restype = ctypes.c_uint64
            L.orc_splitmix64_output.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.orc_stream_seed.restype = None
            L.orc_stream_seed.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _U32P]
            L.orc_xorshift128_next.restype = ctypes.c_uint32
            L.orc_xorshift128_next.argtypes = [_U32P]
            L.orc_mrg32k3a_next.restype = ctypes.c_uint32
            L.orc_mrg32k3a_next.argtypes = [_U32P]
            L.orc_mrg_stream_seed.restype = None
            L.orc_mrg_stream_seed.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _U32P]
            L.orc_mrg_denominator.restype = ctypes.c_uint64
            L.orc_mrg_denominator.argtypes = []
            L.orc_fill_mrg.restype = ctypes.c_int
            L.orc_fill_mrg.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_skip.restype = None
            L.orc_skip.argtypes = [_U32P, ctypes.c_uint64]
            L.orc_stream_raw.restype = None
            L.orc_stream_raw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _U32P]
            L.orc_accept.restype = ctypes.c_int
            L.orc_accept.argtypes = [ctypes.c_uint32, ctypes.c_int]
            L.orc_denominator.restype = ctypes.c_uint64
            L.orc_denominator.argtypes = [ctypes.c_int]
            L.orc_numerator.restype = ctypes.c_uint64
            L.orc_numerator.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int]
            L.orc_rn_ratio.restype = ctypes.c_double
            L.orc_rn_ratio.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.orc_value_rn.restype = ctypes.c_double
            L.orc_value_rn.argtypes = [ctypes.c_uint64, ctypes.c_int]
            L.orc_scale_constant.restype = ctypes.c_double
            L.orc_scale_constant.argtypes = [ctypes.c_int]
            L.orc_value_form_a.restype = ctypes.c_double
            L.orc_value_form_a.argtypes = [ctypes.c_uint64, ctypes.c_int]
            L.orc_fill.restype = ctypes.c_int
            L.orc_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_fill_state.restype = ctypes.c_int
            L.orc_fill_state.argtypes = [_U32P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p]
            L.orc_fill_mode.restype = ctypes.c_int
            L.orc_fill_mode.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_fill_state_mode.restype = ctypes.c_int
            L.orc_fill_state_mode.argtypes = [_U32P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_void_p, ctypes.c_void_p]
            L.orc_values_mode.restype = ctypes.c_int
            L.orc_values_mode.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            L.orc_stats.restype = ctypes.c_int
            L.orc_stats.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_enumerate_pairs.restype = ctypes.c_int
            L.orc_enumerate_pairs.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            for name in ("orc_values_rn", "orc_values_form_a"):
                f = getattr(L, name)
                f.restype = None
                f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
            L.orc_values_form_c.restype = None
            L.orc_values_form_c.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
            L.orc_values_stat_terms.restype = None
            L.orc_values_stat_terms.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- base generators
def splitmix64_output(seed: int, i: int) -> int:
    return int(lib().orc_splitmix64_output(seed, i))


def stream_seed(seed: int, stream: int) -> np.ndarray:
    st = np.zeros(4, dtype=np.uint32)
    lib().orc_stream_seed(seed, stream, st.ctypes.data_as(_U32P))
    return st


def xorshift128_outputs(state, count: int) -> np.ndarray:
    """`count` outputs of xorshift128 continued from `state` (x, y, z, w)."""
    st = np.array(state, dtype=np.uint32).copy()
    p = st.ctypes.data_as(_U32P)
    L = lib()
    return np.array([L.orc_xorshift128_next(p) for _ in range(count)], dtype=np.uint32)


def skip(state, draws: int) -> np.ndarray:
    """The state after `draws` steps of the generator."""
    st = np.array(state, dtype=np.uint32).copy()
    lib().orc_skip(st.ctypes.data_as(_U32P), draws)
    return st


MRG_M1, MRG_M2 = 4294967087, 4294944443


def mrg_stream_seed(seed: int, stream: int) -> np.ndarray:
    st = np.zeros(6, dtype=np.uint32)
    lib().orc_mrg_stream_seed(seed, stream, st.ctypes.data_as(_U32P))
    return st


def mrg_outputs(state, count: int):
    """`count` MRG32k3a outputs z in [1, m1] continued from `state`, and the state after them."""
    st = np.array(state, dtype=np.uint32).copy()
    p = st.ctypes.data_as(_U32P)
    L = lib()
    return np.array([L.orc_mrg32k3a_next(p) for _ in range(count)], dtype=np.uint64), st


def mrg_denominator() -> int:
    return int(lib().orc_mrg_denominator())


def fill_mrg(seed: int, first_stream: int, n_streams: int, per_stream: int, form: int):
    """Stream-major fill over MRG32k3a streams; returns (out, rejects per stream)."""
    out = _out_array(n_streams * per_stream, form)
    rej = np.zeros(n_streams, dtype=np.uint64)
    rc = lib().orc_fill_mrg(seed, first_stream, n_streams, per_stream, form, _ptr(out), _ptr(rej))
    if rc != 0:
        raise ValueError(f"orc_fill_mrg rc={rc}")
    return out, rej


def stream_raw(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint32)
    lib().orc_stream_raw(seed, stream, count, out.ctypes.data_as(_U32P))
    return out


# ---------------------------------------------------------------- the method
def accept(u1: int, w: int) -> bool:
    return bool(lib().orc_accept(u1, w))


def numerator(u1: int, u2: int, w: int) -> int:
    return int(lib().orc_numerator(u1, u2, w))


def denominator(w: int) -> int:
    return int(lib().orc_denominator(w))


def rn_ratio(num: int, den: int) -> float:
    return float(lib().orc_rn_ratio(num, den))


def scale_constant(w: int) -> float:
    return float(lib().orc_scale_constant(w))


def enumerate_pairs(w: int):
    side = 1 << w
    acc = np.zeros(side * side, dtype=np.uint8)
    n = np.zeros(side * side, dtype=np.uint64)
    rc = lib().orc_enumerate_pairs(w, _ptr(acc), _ptr(n))
    assert rc == 0
    return acc.astype(bool), n


def values(n: np.ndarray, w: int, form: int) -> np.ndarray:
    """Per-element output of each form for an array of numerators n."""
    n = np.ascontiguousarray(n, dtype=np.uint64)
    if form == FORM_B:
        out = np.zeros(n.size, dtype=np.float64)
        lib().orc_values_rn(_ptr(n), n.size, w, _ptr(out))
    elif form == FORM_A:
        out = np.zeros(n.size, dtype=np.float64)
        lib().orc_values_form_a(_ptr(n), n.size, w, _ptr(out))
    elif form == FORM_C:
        out = np.zeros(2 * n.size, dtype=np.float32)
        lib().orc_values_form_c(_ptr(n), n.size, w, _ptr(out))
    elif form == FORM_N:
        out = n.copy()
    else:
        raise ValueError(form)
    return out


def stat_terms(n: np.ndarray, w: int) -> np.ndarray:
    """(count, 5) array of (t, bin, p2, p3, p4) for each numerator."""
    n = np.ascontiguousarray(n, dtype=np.uint64)
    out = np.zeros((n.size, 5), dtype=np.uint64)
    lib().orc_values_stat_terms(_ptr(n), n.size, w, _ptr(out))
    return out


def values_mode(u1: np.ndarray, u2: np.ndarray, w: int, form: int, mode: int) -> np.ndarray:
    """Output of each accepted attempt (u1[i], u2[i]) in `form` under `mode`."""
    u1 = np.ascontiguousarray(u1, dtype=np.uint32)
    u2 = np.ascontiguousarray(u2, dtype=np.uint32)
    out = _out_array(u1.size, form)
    rc = lib().orc_values_mode(_ptr(u1), _ptr(u2), u1.size, w, form, mode, _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_values_mode rc={rc}")
    return out


def _out_array(count: int, form: int) -> np.ndarray:
    if form == FORM_C:
        return np.zeros(2 * count, dtype=np.float32)
    if form == FORM_N:
        return np.zeros(count, dtype=np.uint64)
    return np.zeros(count, dtype=np.float64)


def fill(seed: int, first_stream: int, n_streams: int, per_stream: int, w: int, form: int, mode: int = 0):
    """Stream-major fill; returns (out, rejects per stream)."""
    out = _out_array(n_streams * per_stream, form)
    rej = np.zeros(n_streams, dtype=np.uint64)
    rc = lib().orc_fill_mode(seed, first_stream, n_streams, per_stream, w, form, mode, _ptr(out), _ptr(rej))
    if rc != 0:
        raise ValueError(f"orc_fill rc={rc}")
    return out, rej


def fill_state(state, count: int, w: int, form: int, mode: int = 0):
    """Continue one stream from `state`; returns (out, rejects, new_state)."""
    st = np.array(state, dtype=np.uint32).copy()
    out = _out_array(count, form)
    rej = np.zeros(1, dtype=np.uint64)
    rc = lib().orc_fill_state_mode(st.ctypes.data_as(_U32P), count, w, form, mode, _ptr(out), _ptr(rej))
    if rc != 0:
        raise ValueError(f"orc_fill_state rc={rc}")
    return out, int(rej[0]), st


def stats(seed: int, first_stream: int, n_streams: int, per_stream: int, w: int):
    """Fused statistics; returns (hist[65536] uint64, sums[4] as python ints, rejects)."""
    hist = np.zeros(65536, dtype=np.uint64)
    sums = np.zeros(8, dtype=np.uint64)
    rej = np.zeros(n_streams, dtype=np.uint64)
    rc = lib().orc_stats(seed, first_stream, n_streams, per_stream, w, _ptr(hist), _ptr(sums), _ptr(rej))
    if rc != 0:
        raise ValueError(f"orc_stats rc={rc}")
    s = [int(sums[2 * p]) | (int(sums[2 * p + 1]) << 64) for p in range(4)]
    return hist, s, rej
