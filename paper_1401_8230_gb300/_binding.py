"""ctypes declarations of include/prngd.h and argument marshalling (no computation)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

PRNG_OK, PRNG_EINVAL, PRNG_ENOMEM, PRNG_ECUDA, PRNG_ETIMEOUT, PRNG_EBUSY, PRNG_ENOTFOUND = range(7)
FORM_A_FP64, FORM_B_INTBITS, FORM_C_F32PAIR, FORM_L_ALGO1 = 0, 1, 2, 4
MODE_EQ5, MODE_ONE_MINUS, MODE_SINGLE_REDRAW, MODE_BALANCED = 1, 2, 4, 8
GEN_XORSHIFT128, GEN_MRG32K3A = 0, 1
REQ_FRESH, REQ_RESIDENT = 0, 1
MAX_BATCH_REQUESTS = 4096


class TraceItem(ctypes.Structure):
    """struct prng_trace_item of include/prngd.h."""
    _fields_ = [("t", ctypes.c_double), ("client", ctypes.c_uint64), ("length", ctypes.c_uint64),
                ("form", ctypes.c_int32), ("mode", ctypes.c_uint32)]


class Request(ctypes.Structure):
    """struct prng_request of include/prngd.h."""
    _fields_ = [("kind", ctypes.c_int32), ("form", ctypes.c_int32), ("length", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("first_stream", ctypes.c_uint64), ("n_streams", ctypes.c_uint64),
                ("chunk", ctypes.c_uint32), ("mode", ctypes.c_uint32), ("d_out", ctypes.c_void_p),
                ("d_rejects", ctypes.c_void_p)]


def fresh_request(out, length: int, seed: int, first_stream: int, form: int = 1, chunk: int = 0, rejects=None,
                  mode: int = 0):
    return Request(REQ_FRESH, form, length, seed & (2**64 - 1), first_stream, 0, chunk, mode, _ptr(out),
                   _ptr(rejects))


def resident_request(out, length: int, first_stream: int, n_streams: int, form: int = 1, rejects=None,
                     mode: int = 0):
    return Request(REQ_RESIDENT, form, length, 0, first_stream, n_streams, 0, mode, _ptr(out), _ptr(rejects))

_lock = threading.Lock()
_lib: ctypes.CDLL | None = None

_u64, _i32, _dbl, _vp, _sz = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_P = _vp  # opaque handle

# name -> (restype, argtypes); mirrors include/prngd.h
_SIGNATURES = {
    "prng_last_error": (ctypes.c_char_p, []),
    "prng_version": (_i32, []),
    "prng_create": (_i32, [ctypes.POINTER(_P), _u64, _u64, _i32, _dbl, _dbl, _dbl, _dbl]),
    "prng_destroy": (_i32, [_P]),
    "prng_create_mrg32k3a": (_i32, [ctypes.POINTER(_P), _u64, _u64]),
    "prng_generator": (_i32, [_P]),
    "prng_get_info": (_i32, [_P, ctypes.POINTER(_u64), ctypes.POINTER(_i32)]),
    "prng_fill_f64": (_i32, [_P, _vp, _u64, _i32, _vp, _vp]),
    "prng_fill_f32pair": (_i32, [_P, _vp, _u64, _vp, _vp]),
    "prng_fill_mode": (_i32, [_P, _vp, _u64, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "prng_fill_split": (_i32, [_P, _vp, _u64, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, _vp, _vp]),
    "prng_skip": (_i32, [_P, _u64, _vp]),
    "prng_convert_pairs": (_i32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _u64, _vp, _vp]),
    "prng_fill_f64_host": (_i32, [_P, _vp, _u64, _i32, _vp]),
    "prng_fill_f64_host_noalloc": (_i32, [_P, _vp, _u64, _i32, _vp, _vp]),
    "prng_fused_stats": (_i32, [_P, _u64, _vp, _vp, _vp, _vp]),
    "prng_stats_merge": (_i32, [_vp, _vp, _vp, _vp]),
    "prng_state_bytes": (_sz, [_P]),
    "prng_submit": (_i32, [_P, ctypes.c_void_p, _i32, ctypes.POINTER(_u64), _vp]),
    "prng_poll": (_i32, [_P, _u64, ctypes.POINTER(_i32)]),
    "prng_wait": (_i32, [_P, _u64, _dbl]),
    "prng_batch_get_shape": (_i32, [_P, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                    ctypes.POINTER(_i32)]),
    "prng_batch_set_shape": (_i32, [_P, _i32, _i32, _i32, _i32]),
    "prng_batch_autotune": (_i32, [_P, _i32, _u64, _u64, ctypes.c_char_p, _i32, ctypes.POINTER(_i32),
                                   ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                   ctypes.POINTER(_dbl)]),
    "prng_server_create": (_i32, [ctypes.POINTER(_P), _P, _u64, _u64, _sz]),
    "prng_server_destroy": (_i32, [_P]),
    "prng_server_submit": (_i32, [_P, _u64, _u64, _i32, ctypes.POINTER(_u64)]),
    "prng_server_submit_mode": (_i32, [_P, _u64, _u64, _i32, ctypes.c_uint32, ctypes.POINTER(_u64)]),
    "prng_server_step": (_i32, [_P]),
    "prng_server_poll": (_i32, [_P, _u64, ctypes.POINTER(_i32), ctypes.POINTER(_vp)]),
    "prng_server_read": (_i32, [_P, _u64, _vp, _sz]),
    "prng_server_release": (_i32, [_P, _u64]),
    "prng_server_cancel": (_i32, [_P, _u64]),
    "prng_server_drain": (_i32, [_P, _dbl]),
    "prng_server_info": (_i32, [_P, ctypes.POINTER(_u64), ctypes.POINTER(_u64), ctypes.POINTER(_u64),
                                ctypes.POINTER(_u64), ctypes.POINTER(_sz)]),
    "prng_server_run_trace": (_i32, [_P, _vp, _u64, _vp, ctypes.POINTER(_dbl), _dbl]),
    "prng_state_save": (_i32, [_P, _vp, _sz]),
    "prng_state_restore": (_i32, [_P, _vp, _sz]),
}


class PrngError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"prngd error {code}: {message}")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libprngd.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != PRNG_OK:
        raise PrngError(rc, prng_last_error())


def _ptr(x) -> int | None:
    """Device/host address of a tensor-like (data_ptr()), an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):  # numpy
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:  # pragma: no cover
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def prng_last_error() -> str:
    msg = lib().prng_last_error()
    return msg.decode() if msg else ""


def prng_version() -> int:
    return int(lib().prng_version())


def prng_create(seed: int, n_streams: int, w: int = 32, a0: float = 0.0, a: float | None = None,
                b0: float = 0.0, b: float | None = None) -> int:
    step = float((2**w - 1) * 2.0**-w)
    a = a0 + step if a is None else a
    b = b0 + step if b is None else b
    h = _P()
    _check(lib().prng_create(ctypes.byref(h), seed & (2**64 - 1), n_streams, w, a0, a, b0, b))
    return h.value


def prng_create_mrg32k3a(seed: int, n_streams: int) -> int:
    h = _P()
    _check(lib().prng_create_mrg32k3a(ctypes.byref(h), seed & (2**64 - 1), n_streams))
    return h.value


def prng_generator(h: int) -> int:
    return int(lib().prng_generator(h))


def prng_destroy(h: int) -> None:
    _check(lib().prng_destroy(h))


def prng_get_info(h: int) -> tuple[int, int]:
    n, w = _u64(), _i32()
    _check(lib().prng_get_info(h, ctypes.byref(n), ctypes.byref(w)))
    return int(n.value), int(w.value)


def prng_fill_f64(h: int, out, per_stream: int, form: int = FORM_B_INTBITS, rejects=None, stream=None) -> None:
    _check(lib().prng_fill_f64(h, _ptr(out), per_stream, form, _ptr(rejects), _stream(stream)))


def prng_fill_f32pair(h: int, out, per_stream: int, rejects=None, stream=None) -> None:
    _check(lib().prng_fill_f32pair(h, _ptr(out), per_stream, _ptr(rejects), _stream(stream)))


def prng_fill_mode(h: int, out, per_stream: int, form: int, mode: int, rejects=None, stream=None) -> None:
    _check(lib().prng_fill_mode(h, _ptr(out), per_stream, form, mode, _ptr(rejects), _stream(stream)))


def prng_fill_split(h: int, out, per_stream: int, form: int, mode: int = 0, segments: int = 0, rejects=None,
                    stream=None) -> None:
    _check(lib().prng_fill_split(h, _ptr(out), per_stream, form, mode, segments, _ptr(rejects), _stream(stream)))


def prng_convert_pairs(w: int, form: int, mode: int, u1, u2, n: int, out, stream=None) -> None:
    _check(lib().prng_convert_pairs(w, form, mode, _ptr(u1), _ptr(u2), n, _ptr(out), _stream(stream)))


def prng_skip(h: int, draws: int, stream=None) -> None:
    _check(lib().prng_skip(h, draws, _stream(stream)))


def prng_fill_f64_host(h: int, out, per_stream: int, form: int = FORM_B_INTBITS, rejects=None) -> None:
    _check(lib().prng_fill_f64_host(h, _ptr(out), per_stream, form, _ptr(rejects)))


def prng_fill_f64_host_noalloc(h: int, out, per_stream: int, form: int = FORM_B_INTBITS, rejects=None,
                               stream=None) -> None:
    _check(lib().prng_fill_f64_host_noalloc(h, _ptr(out), per_stream, form, _ptr(rejects), _stream(stream)))


def prng_fused_stats(h: int, per_stream: int, hist, sums, rejects=None, stream=None) -> None:
    _check(lib().prng_fused_stats(h, per_stream, _ptr(hist), _ptr(sums), _ptr(rejects), _stream(stream)))


def prng_stats_merge(hist_in, sums_in, hist_acc, sums_acc) -> None:
    """Add one fused-statistics result (host arrays of uint64: 65536 counts, 8 sum words) into
    an accumulator of the same layout."""
    _check(lib().prng_stats_merge(_ptr(hist_in), _ptr(sums_in), _ptr(hist_acc), _ptr(sums_acc)))


def prng_submit(h: int, reqs, stream=None) -> int:
    """Enqueue a batch of Request structs (a list or a ctypes array); returns the ticket."""
    if not isinstance(reqs, ctypes.Array):
        reqs = (Request * len(reqs))(*reqs)
    t = _u64()
    _check(lib().prng_submit(h, ctypes.addressof(reqs), len(reqs), ctypes.byref(t), _stream(stream)))
    return int(t.value)


def prng_poll(h: int, ticket: int) -> bool:
    done = _i32()
    _check(lib().prng_poll(h, ticket, ctypes.byref(done)))
    return bool(done.value)


def prng_wait(h: int, ticket: int, timeout_s: float = 60.0) -> None:
    _check(lib().prng_wait(h, ticket, timeout_s))


def prng_batch_get_shape(h: int) -> tuple[int, int, int, int]:
    a, b, c, d = _i32(), _i32(), _i32(), _i32()
    _check(lib().prng_batch_get_shape(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def prng_batch_set_shape(h: int, warps_per_block: int, blocks_per_sm: int, items_per_ticket: int,
                         outputs_per_chunk: int = 16) -> None:
    _check(lib().prng_batch_set_shape(h, warps_per_block, blocks_per_sm, items_per_ticket, outputs_per_chunk))


def prng_batch_autotune(h: int, form: int, length_lo: int, length_hi: int, table_path: str | None = None,
                        force: bool = False) -> dict:
    a, b, c, d, ms = _i32(), _i32(), _i32(), _i32(), _dbl()
    path = table_path.encode() if table_path else None
    _check(lib().prng_batch_autotune(h, form, length_lo, length_hi, path, int(force), ctypes.byref(a), ctypes.byref(b),
                                     ctypes.byref(c), ctypes.byref(d), ctypes.byref(ms)))
    return {"warps_per_block": a.value, "blocks_per_sm": b.value, "items_per_ticket": c.value,
            "outputs_per_chunk": d.value, "ms": ms.value}


def prng_server_create(h: int, streams_per_client: int, min_per_stream: int = 256, pool_bytes: int = 32 << 30) -> int:
    s = _P()
    _check(lib().prng_server_create(ctypes.byref(s), h, streams_per_client, min_per_stream, pool_bytes))
    return s.value


def prng_server_destroy(s: int) -> None:
    _check(lib().prng_server_destroy(s))


def prng_server_submit(s: int, client: int, length: int, form: int = FORM_B_INTBITS) -> int:
    i = _u64()
    _check(lib().prng_server_submit(s, client, length, form, ctypes.byref(i)))
    return int(i.value)


def prng_server_submit_mode(s: int, client: int, length: int, form: int, mode: int) -> int:
    i = _u64()
    _check(lib().prng_server_submit_mode(s, client, length, form, mode, ctypes.byref(i)))
    return int(i.value)


def prng_server_step(s: int) -> None:
    _check(lib().prng_server_step(s))


def prng_server_poll(s: int, rid: int) -> tuple[bool, int]:
    done, ptr = _i32(), _vp()
    _check(lib().prng_server_poll(s, rid, ctypes.byref(done), ctypes.byref(ptr)))
    return bool(done.value), int(ptr.value or 0)


def prng_server_read(s: int, rid: int, host) -> None:
    _check(lib().prng_server_read(s, rid, _ptr(host), host.nbytes))


def prng_server_release(s: int, rid: int) -> None:
    _check(lib().prng_server_release(s, rid))


def prng_server_cancel(s: int, rid: int) -> None:
    _check(lib().prng_server_cancel(s, rid))


def prng_server_drain(s: int, timeout_s: float = 60.0) -> None:
    _check(lib().prng_server_drain(s, timeout_s))


def prng_server_info(s: int) -> dict:
    a, b, c, d, e = _u64(), _u64(), _u64(), _u64(), _sz()
    _check(lib().prng_server_info(s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d),
                                  ctypes.byref(e)))
    return {"clients": a.value, "batches": b.value, "completed": c.value, "samples": d.value, "pool_used": e.value}


def prng_server_run_trace(s: int, items, timeout_s: float = 600.0):
    """Replay [(t, client, length, form), ...] or [(t, client, length, form, mode), ...] in real
    time; returns (latencies, makespan)."""
    import numpy as np

    arr = (TraceItem * len(items))(*[TraceItem(float(it[0]), int(it[1]), int(it[2]), int(it[3]),
                                               int(it[4]) if len(it) > 4 else 0) for it in items])
    lat = np.zeros(len(items), dtype=np.float64)
    mk = _dbl()
    _check(lib().prng_server_run_trace(s, ctypes.addressof(arr), len(items), lat.ctypes.data, ctypes.byref(mk),
                                       timeout_s))
    return lat, mk.value


def prng_state_bytes(h: int) -> int:
    return int(lib().prng_state_bytes(h))


def prng_state_save(h: int, buf) -> None:
    _check(lib().prng_state_save(h, _ptr(buf), prng_state_bytes(h)))


def prng_state_restore(h: int, buf) -> None:
    _check(lib().prng_state_restore(h, _ptr(buf), prng_state_bytes(h)))


class Generator:
    """Owning wrapper of a handle; methods forward to the prng_* functions."""

    def __init__(self, seed: int, n_streams: int, w: int = 32, generator: int = GEN_XORSHIFT128, **ranges):
        if generator == GEN_MRG32K3A:
            self.h = prng_create_mrg32k3a(seed, n_streams)
        else:
            self.h = prng_create(seed, n_streams, w, **ranges)
        self.n_streams, self.w = prng_get_info(self.h)
        self.generator = prng_generator(self.h)

    def close(self) -> None:
        if self.h:
            prng_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fill_f64(self, out, per_stream: int, form: int = FORM_B_INTBITS, rejects=None, stream=None):
        prng_fill_f64(self.h, out, per_stream, form, rejects, stream)
        return out

    def fill_f32pair(self, out, per_stream: int, rejects=None, stream=None):
        prng_fill_f32pair(self.h, out, per_stream, rejects, stream)
        return out

    def fill_mode(self, out, per_stream: int, form: int, mode: int, rejects=None, stream=None):
        prng_fill_mode(self.h, out, per_stream, form, mode, rejects, stream)
        return out

    def fill_split(self, out, per_stream: int, form: int = FORM_B_INTBITS, mode: int = 0, segments: int = 0,
                   rejects=None, stream=None):
        prng_fill_split(self.h, out, per_stream, form, mode, segments, rejects, stream)
        return out

    def skip(self, draws: int, stream=None) -> None:
        prng_skip(self.h, draws, stream)

    def fill_f64_host(self, out, per_stream: int, form: int = FORM_B_INTBITS, rejects=None):
        prng_fill_f64_host(self.h, out, per_stream, form, rejects)
        return out

    def fused_stats(self, per_stream: int, hist, sums, rejects=None, stream=None):
        prng_fused_stats(self.h, per_stream, hist, sums, rejects, stream)

    def state_save(self, buf):
        prng_state_save(self.h, buf)
        return buf

    def state_restore(self, buf):
        prng_state_restore(self.h, buf)
