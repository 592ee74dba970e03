"""Serving (continuous batching) through the C ABI: every result equals the
single-signal afd_decompose result (bitwise: same kernels, same work split),
requests of mixed N overlap on the device, and the host-side limits hold."""
import threading
import time

import numpy as np
import pytest

from paper_1711_08604_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

afd = pytest.importorskip("paper_1711_08604_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    afd._native.load()


def alone(G, radii, K, tol, prec=1):
    plan = afd.afd_plan_create(G.size, radii, precision=prec)
    r = afd.afd_decompose(plan, G, K, tol)
    plan.close()
    return r


def test_mix_equals_alone_small_stream():
    reqs = W.serving_requests(rate=2000.0, duration=0.1, Ns=(512, 1024, 2048, 4096), M=32, K=24,
                              tol=1e-4, seed_item=7)
    srv = afd.afd_serve_create(1 << 30)
    ids = [afd.afd_serve_submit(srv, s.G, s.radii, s.K, s.tol) for _, s in reqs]
    outs = [afd.afd_serve_wait(srv, i, 120.0) for i in ids]
    stats = afd.afd_serve_get_stats(srv)
    srv.close()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["ticks"] < sum(o["steps"] for o in outs)  # requests shared ticks
    assert stats["kernel_launches"] == stats["ticks"]  # one multi-signal launch per tick
    for (_, s), o in zip(reqs, outs):
        one = alone(s.G, s.radii, s.K, s.tol)
        assert o["steps"] == one["steps"]
        for k in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(o[k], one[k]), k


def test_poisson_arrivals_parity_and_latency():
    # arrivals paced in real time by a submitting thread; results checked
    # against the oracle for a sample
    reqs = W.serving_requests(rate=1000.0, duration=0.3, Ns=(512, 1024, 2048, 4096, 8192, 16384), M=64,
                              K=64, tol=1e-4, seed_item=3)
    srv = afd.afd_serve_create(2 << 30)
    ids = [None] * len(reqs)
    t0 = time.perf_counter()

    def submit():
        for n, (t, s) in enumerate(reqs):
            while time.perf_counter() - t0 < t:
                time.sleep(0.0002)
            ids[n] = afd.afd_serve_submit(srv, s.G, s.radii, s.K, s.tol)

    th = threading.Thread(target=submit)
    th.start()
    th.join()
    outs = [afd.afd_serve_wait(srv, i, 300.0) for i in ids]
    srv.close()
    lat = np.array([o["latency_ms"] for o in outs])
    assert np.all(lat > 0)
    # a sample of every N (up to 16384): the selection of every step against
    # the oracle's FFT-route grid, coefficients, delta and the stop step
    seen = {}
    for n, (_, s) in enumerate(reqs):
        seen.setdefault(s.N, []).append(n)
    sample = sorted(n for ns in seen.values() for n in (ns[0], ns[-1]))
    for n in sample:
        s, o = reqs[n][1], outs[n]
        r = {k: o[k] for k in ("a", "coeff", "delta", "idx")}
        r["steps"] = o["steps"]
        out = parity.check(s.G, s.radii, r, 1, full_grid="fft", energy_tol=s.tol)
        assert out["selection_checked"] == o["steps"]
    for (_, s), o in zip(reqs, outs):
        assert o["delta"][-1] <= s.tol or o["steps"] == s.K


def test_step_limits_inside_a_tick():
    # a tick runs several steps: requests whose step limit (1, 2, 3, 5, 6) or
    # stop rule falls inside a tick stop there, with the results they get alone
    limits = ((1, 0.0), (2, 0.0), (3, 0.0), (5, 0.0), (6, 1e-3))
    reqs = []
    for N in (512, 1024, 2048, 4096, 16384):
        for K, tol in limits:
            G = W.random_signal(N, 70 + len(reqs)) + W.szego_sum(N, np.array([0.7j, -0.5]), np.array([1.0, 0.3]))
            reqs.append((G, K, tol))
    radii = W.radii_linear(20)
    srv = afd.afd_serve_create(1 << 30)
    ids = [afd.afd_serve_submit(srv, G, radii, K, tol) for G, K, tol in reqs]
    outs = [afd.afd_serve_wait(srv, i, 120.0) for i in ids]
    srv.close()
    for (G, K, tol), o in zip(reqs, outs):
        one = alone(G, radii, K, tol)
        assert o["steps"] == one["steps"] <= K
        for k in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(o[k], one[k]), (G.size, K, k)


def test_per_class_launch_server_matches_multi_launch_server():
    # persistent=False serves each N-class with its own step kernels: the same
    # results bitwise as the one-launch ticks
    reqs = W.serving_requests(rate=2000.0, duration=0.05, Ns=(512, 2048, 16384), M=24, K=16, tol=1e-4,
                              seed_item=11)
    outs = []
    for persistent in (True, False):
        srv = afd.afd_serve_create(1 << 30, persistent=persistent)
        ids = [afd.afd_serve_submit(srv, s.G, s.radii, s.K, s.tol) for _, s in reqs]
        outs.append([afd.afd_serve_wait(srv, i, 120.0) for i in ids])
        st = afd.afd_serve_get_stats(srv)
        srv.close()
        assert (st["kernel_launches"] == st["ticks"]) == persistent
    for a, b in zip(*outs):
        assert a["steps"] == b["steps"]
        for k in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(a[k], b[k]), k


def test_fp64_server_matches_plan():
    # N = 256 and N = 16384 (two FP64 sub-transforms per radius) in one server
    reqs = [W.kernel_sum(item=6), W.kernel_sum(item=7, N=16384, M=64, K=6)]
    srv = afd.afd_serve_create(1 << 30, precision=afd.AFD_FP64_PLAIN)
    ids = [afd.afd_serve_submit(srv, s.G, s.radii, s.K, 0.0) for s in reqs]
    outs = [afd.afd_serve_wait(srv, i, 60.0) for i in ids]
    srv.close()
    for s, o in zip(reqs, outs):
        one = alone(s.G, s.radii, s.K, 0.0, prec=0)
        for k in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(o[k], one[k])


def test_host_side_limits():
    srv = afd.afd_serve_create(64 << 20)  # 64 MiB
    s = W.kernel_sum()
    with pytest.raises(afd.AfdError) as e:
        afd.afd_serve_submit(srv, np.ones(100, complex), s.radii, 5)
    assert e.value.status == -1                       # N not a power of two
    with pytest.raises(afd.AfdError) as e:
        afd.afd_serve_submit(srv, np.ones(16384, complex), np.arange(1000) / 1000, 5)
    assert e.value.status == -5                       # needs more than the budget
    with pytest.raises(afd.AfdError) as e:
        afd.afd_serve_poll(srv, 987654)
    assert e.value.status == -6                       # unknown id
    i = afd.afd_serve_submit(srv, s.G, s.radii, 10)
    o = afd.afd_serve_wait(srv, i, 60.0)
    assert o["steps"] == 10 and o["status"] == 0
    with pytest.raises(afd.AfdError) as e:
        afd.afd_serve_poll(srv, i)                    # results are handed out once
    assert e.value.status == -6
    srv.close()


def test_budget_admits_in_waves():
    # 48 MiB: the N = 16384, M = 128 plan tables take ~40 MiB, leaving room for
    # a few 1 MiB slots at a time; everything still completes, in waves
    reqs = [W.kernel_sum(item=i, N=16384, M=128, K=8) for i in range(12)]
    srv = afd.afd_serve_create(48 << 20)
    ids = [afd.afd_serve_submit(srv, s.G, s.radii, s.K) for s in reqs]
    outs = [afd.afd_serve_wait(srv, i, 120.0) for i in ids]
    st = afd.afd_serve_get_stats(srv)
    srv.close()
    assert st["completed"] == 12 and st["bytes_reserved"] <= 48 << 20
    # more than one wave of 8 steps: a tick runs four steps (one launch)
    assert st["ticks"] > 2
    for s, o in zip(reqs, outs):
        one = alone(s.G, s.radii, s.K, 0.0)
        assert np.array_equal(o["coeff"], one["coeff"])


def test_suspend_resume_is_bitwise():
    # a long request is moved to host memory mid-run and resumed while others
    # keep running; its result is the uninterrupted one
    radii = W.radii_linear(128)
    sigs = [W.random_signal(N, 900 + i) for i, N in enumerate([4096, 1024, 2048, 512])]
    K = [200, 30, 30, 30]
    alone = []
    for G, k in zip(sigs, K):
        plan = afd.afd_plan_create(G.size, radii)
        alone.append(afd.afd_decompose(plan, G, k))
        plan.close()
    srv = afd.afd_serve_create(512 << 20)
    ids = [afd.afd_serve_submit(srv, G, radii, k) for G, k in zip(sigs, K)]
    import time
    t0 = time.time()
    while afd.afd_serve_get_stats(srv)["ticks"] < 10 and time.time() - t0 < 60:
        time.sleep(0.001)  # running: 10 of its 200 steps at least
    afd.afd_serve_suspend(srv, ids[0])
    assert afd.afd_serve_poll(srv, ids[0]) is None  # pending while suspended
    others = [afd.afd_serve_wait(srv, i, 60.0) for i in ids[1:]]
    afd.afd_serve_resume(srv, ids[0])
    first = afd.afd_serve_wait(srv, ids[0], 60.0)
    stats = afd.afd_serve_get_stats(srv)
    srv.close()
    assert stats["suspended"] == 1
    for got, want in zip([first] + others, alone):
        assert got["steps"] == want["steps"]
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(got[key], want[key]), key


def test_suspend_queued_and_finished_requests():
    radii = W.radii_linear(32)
    srv = afd.afd_serve_create(64 << 20)
    G = W.random_signal(256, 5)
    i = afd.afd_serve_submit(srv, G, radii, 4)
    o = afd.afd_serve_wait(srv, i, 60.0)
    with pytest.raises(afd.AfdError) as e:
        afd.afd_serve_suspend(srv, i)            # handed out already: unknown
    assert e.value.status == -6
    with pytest.raises(afd.AfdError) as e:
        afd.afd_serve_resume(srv, 12345)
    assert e.value.status == -6
    j = afd.afd_serve_submit(srv, G, radii, 4)
    try:
        afd.afd_serve_suspend(srv, j)            # queued or running: leaves the device
    except afd.AfdError as err:                  # or it finished first
        assert err.status == -1
        assert afd.afd_serve_wait(srv, j, 60.0)["steps"] == 4
    else:
        with pytest.raises(afd.AfdError):
            afd.afd_serve_resume(srv, 999999)
        afd.afd_serve_resume(srv, j)
        r = afd.afd_serve_wait(srv, j, 60.0)
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(r[key], o[key]), key
    srv.close()
