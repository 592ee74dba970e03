"""Non-uniform samples (the remark after Step 2 of Sec. 3.2): the non-uniform
DFT route on the GPU against the oracle's weighted rectangle rule."""
import numpy as np
import pytest

import oracle
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


def run(theta, w, G, radii, L, K, **kw):
    plan = afd.afd_plan_create_nonuniform(theta, radii, L, weights=w, **kw)
    try:
        return afd.afd_decompose(plan, G, K)
    finally:
        plan.close()


def check_nu(theta, w, G, radii, L, res, full_grid=True, grid_steps=()):
    """The rules of tests/parity.py on the L-angle grid: the same pick unless a
    near-tie (1e-6 relative), FP64 coefficients, a_k and delta."""
    steps = int(res["steps"])
    idx = np.asarray(res["idx"]).reshape(steps, 2)
    ora = oracle.nu_decompose(G, theta, w, radii, L, steps, forced_idx=idx, compute_grid=full_grid)
    floor = parity.ABS_FLOOR * np.sqrt(ora["energy"][0])
    for k in range(steps):
        if full_grid and tuple(idx[k]) != tuple(ora["own_idx"][k]):
            assert ora["objused"][k] >= ora["objmax"][k] * (1 - parity.NEAR_TIE), (k, idx[k], ora["own_idx"][k])
        assert abs(res["coeff"][k] - ora["coeff"][k]) <= 1e-10 * abs(ora["coeff"][k]) + floor, k
        assert abs(res["a"][k] - ora["a"][k]) <= 1e-14, k
        assert abs(res["delta"][k + 1] - ora["delta"][k + 1]) <= 1e-10 * ora["delta"][k + 1] + 1e-14, k
    for k1 in grid_steps:
        k = k1 - 1
        Gk = G if k == 0 else oracle.nu_decompose(G, theta, w, radii, L, k, forced_idx=idx[:k],
                                                  compute_grid=False)["G_final"]
        one = oracle.nu_decompose(Gk, theta, w, radii, L, 1)
        if tuple(one["own_idx"][0]) != tuple(idx[k]):
            c = oracle.nu_inner(Gk, theta, w, res["a"][k])
            assert c.real ** 2 + c.imag ** 2 >= one["objmax"][0] * (1 - parity.NEAR_TIE), k1
    return ora


def test_equispaced_samples_match_the_uniform_path():
    s = W.kernel_sum(item=1)
    N = s.N
    theta = 2 * np.pi * np.arange(N) / N
    w = np.full(N, 1.0 / N)
    res = run(theta, w, s.G, s.radii, N, s.K)
    check_nu(theta, w, s.G, s.radii, N, res)
    plan = afd.afd_plan_create(N, s.radii)
    uni = afd.afd_decompose(plan, s.G, s.K)
    plan.close()
    assert np.array_equal(res["idx"], uni["idx"])
    assert np.max(np.abs(res["coeff"] - uni["coeff"])) <= 1e-12 * np.max(np.abs(uni["coeff"]))


@pytest.mark.parametrize("L", [32, 64, 256])
def test_jittered_samples_full_grid(L):
    x = W.nonuniform(item=1, N=300, L=L, M=40, K=8)
    res = run(x.theta, x.weights, x.G, x.radii, x.L, x.K)
    assert res["steps"] == x.K
    check_nu(x.theta, x.weights, x.G, x.radii, x.L, res)


def test_default_weights_are_the_trapezoid_rule():
    x = W.nonuniform(item=2, N=257, L=128, M=20, K=5)
    a = run(x.theta, None, x.G, x.radii, x.L, x.K)
    b = run(x.theta, x.weights, x.G, x.radii, x.L, x.K)
    for key in ("a", "coeff", "delta", "idx"):
        assert np.array_equal(a[key], b[key]), key


def test_nonuniform_workload_full_grid():
    # N = 3000 jittered samples, L = 1024, M = 64, K = 12: the oracle's own
    # direct grid (65,536 points x 3000 samples) at every step
    x = W.nonuniform()
    res = run(x.theta, x.weights, x.G, x.radii, x.L, x.K)
    assert res["steps"] == x.K
    check_nu(x.theta, x.weights, x.G, x.radii, x.L, res)
    assert np.all(np.diff(res["delta"]) <= 1e-12)


def test_radius_near_one_needs_folds():
    # r = 0.999 needs 43 folds of a 1024-angle grid, more than 64 of 256
    x = W.nonuniform(item=3, N=500, L=1024, M=8, K=4)
    radii = np.array([0.0, 0.5, 0.9, 0.99, 0.999])
    G = W.szego_sum_at(x.theta, np.array([0.999 * np.exp(2j * np.pi * 300 / 1024)]), np.array([1.0])) + x.G
    res = run(x.theta, x.weights, G, radii, 1024, 4)
    check_nu(x.theta, x.weights, G, radii, 1024, res)
    with pytest.raises(afd.AfdError) as e:
        afd.afd_plan_create_nonuniform(x.theta, radii, 256, weights=x.weights)
    assert e.value.status == -1


def test_nonuniform_resume_is_bitwise():
    x = W.nonuniform(item=4, N=700, L=512, M=32, K=10)
    plan = afd.afd_plan_create_nonuniform(x.theta, x.radii, x.L, weights=x.weights)
    full = afd.afd_decompose_from(plan, x.G, 10)
    p1 = afd.afd_decompose_from(plan, x.G, 3)
    p2 = afd.afd_decompose_from(plan, p1["G_final"], 7, E1=p1["E1"])
    plan.close()
    for key in ("a", "coeff", "idx"):
        assert np.array_equal(np.concatenate([p1[key], p2[key]]), full[key]), key
    assert np.array_equal(p2["G_final"], full["G_final"])


def test_nonuniform_invalid_arguments():
    th = W.nonuniform_angles(64, 1)
    r = np.array([0.0, 0.5])
    bad = [dict(theta=th[::-1], radii=r, L=64), dict(theta=np.append(th, 7.0), radii=r, L=64),
           dict(theta=th, radii=r, L=100), dict(theta=th, radii=r, L=4), dict(theta=th, radii=r, L=1 << 14),
           dict(theta=th, radii=r, L=64, precision=afd.AFD_FP64_PLAIN),
           dict(theta=th, radii=r, L=64, force_a1_zero=True), dict(theta=th, radii=r, L=64, renormalise=True),
           dict(theta=th, radii=r, L=64, weights=-np.ones(64))]
    for kw in bad:
        with pytest.raises(afd.AfdError) as e:
            afd.afd_plan_create_nonuniform(**kw)
        assert e.value.status == -1, kw
