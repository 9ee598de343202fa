"""CPU checks of the C ABI: the library builds, loads, exports every function declared in
include/prngd.h, and rejects bad arguments on the host (no GPU needed for those paths)."""
import os
import re

import pytest

from conftest import ROOT

import paper_1401_8230_gb300 as P


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(prng_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("prng_create", "prng_destroy", "prng_fill_f64", "prng_fill_f32pair",
                     "prng_state_save", "prng_state_restore"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = P.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert P.prng_version() >= 100


@pytest.mark.parametrize("kwargs, fragment", [
    (dict(seed=1, n_streams=64, w=1), "outside [2, 32]"),
    (dict(seed=1, n_streams=64, w=33), "outside [2, 32]"),
    (dict(seed=1, n_streams=0, w=32), "n_streams"),
    (dict(seed=1, n_streams=2**32 + 1, w=32), "n_streams"),
    (dict(seed=1, n_streams=8, w=32, a0=0.0, a=1.0), "a - a0"),
    (dict(seed=1, n_streams=8, w=24, b0=0.5, b=1.0), "a - a0"),
    (dict(seed=1, n_streams=8, w=16, a0=float("nan")), "finite"),
])
def test_create_rejects_bad_arguments_on_the_host(kwargs, fragment):
    with pytest.raises(P.PrngError) as ei:
        P.prng_create(**kwargs)
    assert ei.value.code == P.PRNG_EINVAL
    assert fragment in str(ei.value)


def test_null_handle_is_rejected():
    with pytest.raises(P.PrngError) as ei:
        P.prng_fill_f64(0, 0, 16, P.FORM_B_INTBITS)
    assert ei.value.code == P.PRNG_EINVAL
    assert P.prng_state_bytes(0) == 0
    P.prng_destroy(0)  # no-op


def test_c_caller_gets_argument_errors_without_python(tmp_path):
    """A C program that includes only include/prngd.h and links libprngd: the argument errors
    that need no GPU come back as PRNG_EINVAL with a message."""
    import subprocess

    from conftest import build_c_caller

    exe = build_c_caller(tmp_path)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and "bad 0" in out.stdout, out.stdout


def test_stats_merge_is_exact_128_bit_addition():
    """prng_stats_merge (host only) against Python integers: counts add, and each 128-bit sum
    carries from its low word into its high word."""
    import numpy as np

    rng = np.random.default_rng(8)
    acc_h = np.zeros(65536, dtype=np.uint64)
    acc_s = np.zeros(8, dtype=np.uint64)
    want_h = np.zeros(65536, dtype=object)
    want_s = [0] * 4
    for k in range(6):
        h = rng.integers(0, 2**40, 65536, dtype=np.uint64)
        lo = rng.integers(2**63, 2**64 - 1, 4, dtype=np.uint64, endpoint=True)  # large low words: carries
        hi = rng.integers(0, 2**20, 4, dtype=np.uint64)
        s = np.empty(8, dtype=np.uint64)
        s[0::2], s[1::2] = lo, hi
        P.prng_stats_merge(h, s, acc_h, acc_s)
        want_h += h.astype(object)
        for p in range(4):
            want_s[p] += int(lo[p]) + (int(hi[p]) << 64)
    assert [int(v) for v in acc_h] == [int(v) for v in want_h]
    assert [int(acc_s[2 * p]) + (int(acc_s[2 * p + 1]) << 64) for p in range(4)] == want_s
    with pytest.raises(P.PrngError) as ei:
        P.prng_stats_merge(None, acc_s, acc_h, acc_s)
    assert ei.value.code == P.PRNG_EINVAL


def test_binding_mirrors_every_declaration():
    """Every function include/prngd.h declares has a ctypes signature in the binding with the
    same number of parameters, and a Python function of the same name."""
    from paper_1401_8230_gb300 import _binding as B

    text = open(os.path.join(ROOT, "include", "prngd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    decls = dict(re.findall(r"\b(prng_\w+)\s*\(([^)]*)\)\s*;", text, flags=re.S))
    assert set(decls) == set(declared_functions())
    for name, params in decls.items():
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert name in B._SIGNATURES, name
        assert len(B._SIGNATURES[name][1]) == n, (name, n, len(B._SIGNATURES[name][1]))
        assert callable(getattr(B, name, None)), name
