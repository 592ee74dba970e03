"""Off-grid refinement of each step's point (afd_plan_opts.offgrid_iters):
the CUDA path against the oracle's refinement (the same damped Newton
iteration on the same discrete objective), on every plan path that takes it:
power-of-two and mixed-radix sizes in both precisions, the reproducing kernel
off the grid, the stop rule, and the argument checks."""
import numpy as np
import pytest

import oracle
from paper_1711_08604_gb300 import workloads as W

pytestmark = pytest.mark.gpu

afd = pytest.importorskip("paper_1711_08604_gb300")
PRECS = [afd.AFD_FP64_PLAIN, afd.AFD_FP32_GUARDED]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    afd._native.load()


def run(G, radii, K, prec, tol=0.0, **kw):
    plan = afd.afd_plan_create(G.size, radii, precision=prec, **kw)
    try:
        r = afd.afd_decompose(plan, G, K, tol)
        r["flags"] = afd.afd_plan_last_info(plan, r["steps"])["flags"]
        return r
    finally:
        plan.close()


def compare(G, radii, K, prec, iters=20, tol=0.0):
    """GPU vs oracle: the same grid starting points at every step (both sides
    select on the grid first; a near-tie there would resynchronise, which
    these signals do not have), refined points within 1e-9, coefficients within
    1e-8 relative (FP64 sums in different orders go through the same Newton
    iteration), delta within 1e-7 relative."""
    r = run(G, radii, K, prec, tol, offgrid_iters=iters)
    o = oracle.decompose(G, radii, K, energy_tol=tol, offgrid_iters=iters)
    assert r["steps"] == o["steps"]
    assert np.array_equal(r["idx"], o["idx"]), (r["idx"], o["idx"])
    assert np.max(np.abs(r["a"] - o["a"])) < 1e-9
    assert np.max(np.abs(r["coeff"] - o["coeff"]) / np.abs(o["coeff"])) < 1e-8
    assert np.all(np.abs(r["delta"] - o["delta"]) <= 1e-7 * o["delta"] + 1e-14)
    assert np.all((r["flags"] & 8) != 0)
    return r, o


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [256, 1024])
def test_offgrid_matches_oracle(prec, N):
    b = np.array([0.55 * np.exp(2j * np.pi * 0.123), 0.8 * np.exp(-2j * np.pi * 0.31), 0.3 + 0.2j])
    G = W.szego_sum(N, b, np.array([1.0, 0.6, 0.4j])) + 0.05 * W.random_signal(N, N + prec)
    compare(G, W.radii_linear(24), 8, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_offgrid_mixed_radix_size(prec):
    N = 3 * 5 * 64  # 960: radices 16, 4, 3, 5
    G = W.szego_sum(N, np.array([0.7 * np.exp(0.9j), -0.4 + 0.1j]), np.array([1.0, 0.5])) \
        + 0.02 * W.random_signal(N, 9)
    compare(G, W.radii_linear(20), 6, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_offgrid_recovers_a_kernel(prec):
    # e_b with b off the grid and |b|^N negligible: one refined step finds b
    # and leaves nothing
    N = 512
    b = 0.62 * np.exp(2j * np.pi * 0.2718)
    G = W.szego_sum(N, np.array([b]), np.array([1.0]))
    r = run(G, W.radii_linear(16), 2, prec, offgrid_iters=30)
    assert abs(r["a"][0] - b) < 1e-11
    assert abs(abs(r["coeff"][0]) - 1.0) < 1e-11
    assert r["delta"][1] < 1e-20


def test_offgrid_stop_rule_and_gain():
    # the refined path reaches the energy tolerance in no more steps than the
    # grid path, and each of its steps gains at least as much
    N = 1024
    s = W.tones(N=N, M=40, K=30)
    r_grid = run(s.G, s.radii, 30, afd.AFD_FP32_GUARDED, 1e-3)
    r, o = compare(s.G, s.radii, 30, afd.AFD_FP32_GUARDED, tol=1e-3)
    assert r["steps"] <= r_grid["steps"]
    assert r["delta"][1] <= r_grid["delta"][1]


def test_offgrid_argument_checks():
    G = W.random_signal(64, 1)
    radii = W.radii_linear(8)
    for kw in ({"offgrid_iters": -1}, {"offgrid_iters": 65}, {"offgrid_iters": 4, "renormalise": True}):
        with pytest.raises(afd.AfdError):
            afd.afd_plan_create(64, radii, **kw)
    with pytest.raises(afd.AfdError):
        afd.afd_batch_create([64, 128], radii, 4, offgrid_iters=4)
    with pytest.raises(afd.AfdError):
        afd.afd_serve_create(1 << 26, offgrid_iters=4)
    r = run(G, radii, 3, afd.AFD_FP32_GUARDED, offgrid_iters=0)
    assert np.all((r["flags"] & 8) == 0)
