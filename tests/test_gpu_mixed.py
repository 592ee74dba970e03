"""N = 2^a 3^b 5^c 7^d 11^e 13^f that is not a power of two: the mixed-radix path
against the oracle (the remark after Table 9, Sec. 4.2: the algorithm stays valid
for N = p^K with p prime)."""
import numpy as np
import pytest

import oracle
from paper_1711_08604_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

afd = pytest.importorskip("paper_1711_08604_gb300")
PRECS = [afd.AFD_FP64_PLAIN, afd.AFD_FP32_GUARDED]
RADII = np.array([0.0, 0.05, 0.3, 0.55, 0.8, 0.9, 0.97])


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    afd._native.load()


def run(G, radii, K, prec, **kw):
    plan = afd.afd_plan_create(G.size, radii, precision=prec, **kw)
    try:
        return afd.afd_decompose(plan, G, K)
    finally:
        plan.close()


# every radix (16, 8, 4, 2, 3, 5) as first, middle and last pass, ragged
# butterfly counts against the 256-thread CTA
SMALL = [9, 10, 12, 15, 24, 40, 48, 60, 80, 96, 160, 243, 625, 729, 1000, 1500]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", SMALL)
def test_mixed_sizes_full_grid_parity(prec, N):
    G = W.random_signal(N, 11 * N)
    res = run(G, RADII, 6, prec)
    assert res["steps"] == 6
    parity.check(G, RADII, res, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [2187, 3125, 6400])
def test_mixed_larger_sizes(prec, N):
    G = W.szego_sum(N, 0.85 * np.exp(2j * np.pi * np.array([0.123, 0.61])), np.array([1.0, 0.4 - 0.3j]))
    G = G + 0.05 * W.random_signal(N, N)
    radii = W.radii_linear(40)
    res = run(G, radii, 5, prec)
    assert parity.check(G, radii, res, prec, full_grid="fft")["selection_checked"] == 5


def test_mixed_largest_fp32_size():
    N = 12800
    G = W.random_signal(N, 3)
    res = run(G, RADII, 3, afd.AFD_FP32_GUARDED)
    assert parity.check(G, RADII, res, afd.AFD_FP32_GUARDED, full_grid="fft")["selection_checked"] == 3


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_reproducing_kernel(prec):
    # G = e_b with b on the grid: the first step must pick b with |c_1| = 1
    N, radii = 1000, W.radii_linear(50)
    b = radii[31] * np.exp(2j * np.pi * 377 / N)
    G = W.szego_sum(N, np.array([b]), np.array([1.0]))
    res = run(G, radii, 1, prec)
    assert tuple(res["idx"][0]) == (31, 377)
    assert abs(abs(res["coeff"][0]) - 1.0) <= 1e-13
    assert abs(res["coeff"][0] - oracle.inner(G, res["a"][0])) <= 1e-13


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_zero_radius_ties_lowest_index(prec):
    G = W.random_signal(729, 5)
    res = run(G, np.array([0.0]), 3, prec)
    for k in range(3):
        assert tuple(res["idx"][k]) == (0, 0)


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_and_power_of_two_batch_equals_single_runs(prec):
    Ns = [729, 1000, 1024, 1500, 1000, 96, 4096, 243]
    sigs = [W.random_signal(N, 40 + i) for i, N in enumerate(Ns)]
    radii = W.radii_linear(24)
    K = 5
    res = afd.afd_decompose_batch(sigs, radii, K, precision=prec)
    for i, G in enumerate(sigs):
        one = run(G, radii, K, prec)
        assert res["steps"][i] == one["steps"]
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(res[key][i], one[key]), (Ns[i], key)


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_resume_is_bitwise(prec):
    G = W.random_signal(1500, 8)
    radii = W.radii_linear(30)
    plan = afd.afd_plan_create(G.size, radii, precision=prec)
    full = afd.afd_decompose_from(plan, G, 10)
    p1 = afd.afd_decompose_from(plan, G, 4)
    p2 = afd.afd_decompose_from(plan, p1["G_final"], 6, E1=p1["E1"])
    plan.close()
    for key in ("a", "coeff", "idx"):
        assert np.array_equal(np.concatenate([p1[key], p2[key]]), full[key]), key
    assert np.array_equal(p2["G_final"], full["G_final"])


# N = p^K for the primes 7, 11 and 13 (the paper's remark), ragged products
# with 2, 3 and 5, and every odd prime as first, middle and last pass
PRIME = [49, 14, 26, 77, 91, 143, 343, 105, 616, 1001, 1331, 2197, 2401]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", PRIME)
def test_prime_power_sizes_full_grid_parity(prec, N):
    # every grid point of every step against the oracle's own direct grid
    G = W.random_signal(N, 13 * N) + W.szego_sum(N, np.array([0.9 * np.exp(1.3j)]), np.array([0.7]))
    res = run(G, RADII, 5, prec)
    assert res["steps"] == 5
    assert parity.check(G, RADII, res, prec)["selection_checked"] == 5


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [1331, 2197, 2401])
def test_prime_power_reproducing_kernel(prec, N):
    # G = e_b, b on the grid: the first step picks b with |c_1| = 1
    radii = W.radii_linear(40)
    j0 = N // 3 + 2
    b = radii[29] * np.exp(2j * np.pi * j0 / N)
    G = W.szego_sum(N, np.array([b]), np.array([1.0]))
    res = run(G, radii, 1, prec)
    assert tuple(res["idx"][0]) == (29, j0)
    assert abs(abs(res["coeff"][0]) - 1.0) <= 1e-12


def test_prime_power_batch_equals_single_runs():
    Ns = [2401, 1331, 2197, 1024, 1331, 343]
    sigs = [W.random_signal(N, 60 + i) for i, N in enumerate(Ns)]
    radii = W.radii_linear(16)
    res = afd.afd_decompose_batch(sigs, radii, 4)
    for i, G in enumerate(sigs):
        one = run(G, radii, 4, afd.AFD_FP32_GUARDED)
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(res[key][i], one[key]), (Ns[i], key)


def test_mixed_size_limits():
    r = np.array([0.0, 0.5])
    for N, prec in [(17 * 128, 1), (19 * 9, 1), (7, 1), (13500, 1), (7200, 0), (6, 1)]:
        with pytest.raises(afd.AfdError) as e:
            afd.afd_plan_create(N, r, precision=prec)
        assert e.value.status == -1, N
    srv = afd.afd_serve_create(64 << 20)
    with pytest.raises(afd.AfdError) as e:
        afd.afd_serve_submit(srv, np.ones(1000, complex), r, 2)  # serving: powers of two only
    assert e.value.status == -1
    srv.close()


def test_mixed_batch_in_one_persistent_launch():
    # persistent=2: the batch, mixed-radix classes included (each radius a grid
    # item, the forward transform split over items for even N), in one launch
    # of the multi-signal kernel, bitwise equal to the per-step kernels
    Ns = [729, 1000, 1024, 1500, 96, 4096, 243, 3000]
    sigs = [W.random_signal(N, 60 + i) for i, N in enumerate(Ns)]
    radii = W.radii_linear(20)
    K = 6
    res = afd.afd_decompose_batch(sigs, radii, K, persistent=2)
    for i, G in enumerate(sigs):
        one = run(G, radii, K, afd.AFD_FP32_GUARDED, persistent=False)
        assert res["steps"][i] == one["steps"]
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(res[key][i], one[key]), (Ns[i], key)
    # the stop rule inside the launch: a tolerance between deltas 3 and 4 of
    # one signal stops it after step 4 and leaves the others as they were
    tol = float(res["delta"][7][4]) * 1.0000001
    res2 = afd.afd_decompose_batch(sigs, radii, K, energy_tol=tol, persistent=2)
    for i, G in enumerate(sigs):
        plan = afd.afd_plan_create(G.size, radii, persistent=False)
        try:
            one = afd.afd_decompose(plan, G, K, tol)
        finally:
            plan.close()
        assert res2["steps"][i] == one["steps"]
        assert np.array_equal(res2["coeff"][i], one["coeff"]), Ns[i]
    assert res2["steps"][7] <= 4
