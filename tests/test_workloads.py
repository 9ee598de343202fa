"""The seeded input recipes of the batched and serving workloads (paper_1401_8230_gb300/
workloads.py, inputs only): deterministic for a seed, lengths log-uniform inside their range,
stream offsets cumulative so that no two requests share a stream, and the totals the bench's
workloads are stated with (about 2.2e10 outputs for the batch, about 433 Gsamples/s offered
by the serving trace)."""
import math

import numpy as np

from paper_1401_8230_gb300 import workloads as WL


def test_batched_requests_recipe():
    a = WL.batched_requests()
    assert a == WL.batched_requests()  # the same seed gives the same requests
    assert a != WL.batched_requests(seed=2)
    assert len(a) == 4096
    L = np.array([r["length"] for r in a], dtype=np.float64)
    assert L.min() >= 2**8 and L.max() <= 2**26
    # log-uniform: log2 of the lengths is uniform on [8, 26] (mean 17, sd 18/sqrt(12))
    lg = np.log2(L)
    assert abs(lg.mean() - 17.0) < 4 * (18 / math.sqrt(12)) / math.sqrt(len(a))
    assert abs(np.median(lg) - 17.0) < 0.5
    # streams: each request's rows follow the previous request's, none shared
    first = 0
    for r in a:
        assert r["first_stream"] == first and r["chunk"] == 1024
        first += -(-r["length"] // r["chunk"])
    assert len({r["seed"] for r in a}) == len(a)  # independent 64-bit seeds
    total = L.sum()
    assert 2.0e10 < total < 2.4e10  # the batched workload's stated size (22.2G outputs measured)


def test_serving_arrivals_recipe():
    T, rate = 2.0, 20000.0
    tr = WL.serving_arrivals(T, rate)
    assert tr == WL.serving_arrivals(T, rate)
    n = len(tr)
    assert abs(n - rate * T) < 5 * math.sqrt(rate * T)  # Poisson count
    t = np.array([r["t"] for r in tr])
    assert np.all(np.diff(t) >= 0) and t[0] >= 0 and t[-1] <= T
    L = np.array([r["length"] for r in tr], dtype=np.float64)
    assert L.min() >= 2**10 and L.max() <= 2**28
    forms = np.bincount([r["form"] for r in tr], minlength=3)
    assert forms.shape == (3,) and np.all(np.abs(forms - n / 3) < 5 * math.sqrt(n / 3))
    clients = np.array([r["client"] for r in tr])
    assert clients.min() >= 0 and clients.max() < 2**16
    # offered load: E[L] = (hi - lo) / ln(hi / lo) for log-uniform lengths, 20k requests/s
    expect = rate * (2**28 - 2**10) / math.log(2**18)
    offered = L.sum() / T
    assert abs(offered / expect - 1) < 0.1
    assert 3.9e11 < expect < 4.8e11  # about 433 Gsamples/s, the serving workload's offered load
