"""Batched decompositions of uneven N through the C ABI (afd_batch_*)."""
import numpy as np
import pytest

from paper_1711_08604_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

afd = pytest.importorskip("paper_1711_08604_gb300")
PRECS = [afd.AFD_FP64_PLAIN, afd.AFD_FP32_GUARDED]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    afd._native.load()


def small_batch(n=12, Ns=(256, 512, 1024, 2048, 4096, 8192), seed=0):
    sigs = []
    for i in range(n):
        N = Ns[i % len(Ns)]
        sigs.append(W.random_signal(N, 500 + seed + i) if i % 3 == 0
                    else W.szego_sum(N, 0.9 * np.exp(2j * np.pi * np.array([0.1 * i, 0.37 + 0.05 * i])),
                                     np.array([1.0, 0.5j])))
    return sigs


@pytest.mark.parametrize("prec", PRECS)
def test_batch_equals_single_signal_runs(prec):
    sigs = small_batch()
    radii = W.radii_linear(30)
    K = 8
    res = afd.afd_decompose_batch(sigs, radii, K, precision=prec)
    for i, G in enumerate(sigs):
        plan = afd.afd_plan_create(G.size, radii, precision=prec)
        one = afd.afd_decompose(plan, G, K)
        plan.close()
        assert res["steps"][i] == one["steps"]
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(res[key][i], one[key]), (i, key)


@pytest.mark.parametrize("prec", PRECS)
def test_batch_parity_with_oracle(prec):
    sigs = small_batch(n=6, Ns=(64, 256, 1024), seed=9)
    radii = W.radii_linear(20)
    res = afd.afd_decompose_batch(sigs, radii, 6, precision=prec)
    for i, G in enumerate(sigs):
        r = {k: res[k][i] for k in ("a", "coeff", "delta", "idx")}
        r["steps"] = int(res["steps"][i])
        parity.check(G, radii, r, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_batch_per_signal_energy_stop(prec):
    sigs = small_batch(n=6, Ns=(512, 1024), seed=3)
    radii = W.radii_linear(25)
    full = afd.afd_decompose_batch(sigs, radii, 10, precision=prec)
    tol = float(np.median([d[4] for d in full["delta"]]))
    res = afd.afd_decompose_batch(sigs, radii, 10, energy_tol=tol, precision=prec)
    for i in range(len(sigs)):
        d = full["delta"][i][1:]
        first = int(np.argmax(d <= tol)) + 1 if np.any(d <= tol) else 10
        assert res["steps"][i] == first
        assert np.array_equal(res["coeff"][i], full["coeff"][i][:first])


@pytest.mark.parametrize("prec,Ns", [(afd.AFD_FP64_PLAIN, (4096, 16384, 32768, 65536)),
                                     (afd.AFD_FP32_GUARDED, (16384, 32768))])
def test_batch_with_split_sizes(prec, Ns):
    # sizes split into resident sub-transforms share launches with other
    # signals of their N and give the single-signal results bitwise; the
    # selection of every step against the oracle's FFT-route grid
    sigs = [W.random_signal(N, 70 + N) for N in Ns for _ in range(2)]
    radii = W.radii_linear(12)
    res = afd.afd_decompose_batch(sigs, radii, 3, precision=prec)
    for i, G in enumerate(sigs):
        plan = afd.afd_plan_create(G.size, radii, precision=prec)
        one = afd.afd_decompose(plan, G, 3)
        plan.close()
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(res[key][i], one[key]), (i, key)
        r = {k: res[k][i] for k in ("a", "coeff", "delta", "idx")}
        r["steps"] = int(res["steps"][i])
        assert parity.check(G, radii, r, prec, full_grid="fft")["selection_checked"] == 3


def test_large_class_equals_single_runs():
    # twelve signals of one N share each launch (the guard then keeps one
    # candidate in flight per signal instead of four): the results are the
    # single-signal ones bitwise
    sigs = [W.tones(item=20 + i, N=2048, M=40, K=6).G for i in range(12)]
    radii = W.radii_linear(40)
    res = afd.afd_decompose_batch(sigs, radii, 6)
    for i, G in enumerate(sigs):
        plan = afd.afd_plan_create(G.size, radii)
        one = afd.afd_decompose(plan, G, 6)
        plan.close()
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(res[key][i], one[key]), (i, key)


@pytest.mark.parametrize("tol", [0.0, 3e-3])
def test_multi_signal_launch_equals_stream_path(tol):
    # every power of two the multi-signal persistent kernel takes (8 .. 16384),
    # several signals per N-class and a lone one, with and without the stop
    # rule: one cooperative launch per batch gives bitwise the per-kernel,
    # per-class sequence (persistent=False) and the single-signal runs
    Ns = [8, 16, 64, 256, 256, 512, 1024, 2048, 2048, 2048, 4096, 8192, 8192, 16384]
    sigs = [W.random_signal(N, 90 + i) + W.szego_sum(N, np.array([0.8 * np.exp(0.7j * (i + 1))]), np.array([1.0]))
            for i, N in enumerate(Ns)]
    radii = W.radii_linear(21)
    K = 7
    multi = afd.afd_batch_create([g.size for g in sigs], radii, K, persistent=2)
    r1 = afd.afd_batch_run(multi, np.concatenate(sigs), tol)
    launches = afd.afd_batch_counters(multi)["kernel_launches"]
    multi.close()
    assert launches == 1  # the whole batch: one launch
    r2 = afd.afd_decompose_batch(sigs, radii, K, energy_tol=tol, persistent=False)
    for i, G in enumerate(sigs):
        assert r1["steps"][i] == r2["steps"][i]
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(r1[key][i], r2[key][i]), (Ns[i], key)
        plan = afd.afd_plan_create(G.size, radii)
        one = afd.afd_decompose(plan, G, K, tol)
        plan.close()
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(r1[key][i], one[key]), (Ns[i], key)


def test_batch_reuse_and_counters():
    sigs = small_batch(n=5, Ns=(1024, 2048))
    radii = W.radii_linear(16)
    b = afd.afd_batch_create([g.size for g in sigs], radii, 5)
    packed = np.concatenate(sigs)
    r1 = afd.afd_batch_run(b, packed)
    r2 = afd.afd_batch_run(b, packed)
    assert afd.afd_batch_counters(b)["kernel_launches"] > 0
    b.close()
    for i in range(len(sigs)):
        assert np.array_equal(r1["coeff"][i], r2["coeff"][i])


def test_workload3_full_batch_parity():
    # 1024 signals, N in {1024..8192}, M = 100, K = 30, FP32 grid + FP64 guard.
    # Four signals of every N-class (the first, the last and two between):
    # the selection of all 30 steps against the oracle's FFT-route grid, and
    # coefficients and delta through the forced oracle
    sigs = W.batch()
    G = [s.G for s in sigs]
    radii = sigs[0].radii
    res = afd.afd_decompose_batch(G, radii, 30)
    assert np.all(res["steps"] == 30)
    by_n = {}
    for i, s in enumerate(sigs):
        by_n.setdefault(s.N, []).append(i)
    assert sorted(by_n) == [1024, 2048, 4096, 8192]
    for N, members in sorted(by_n.items()):
        pick = sorted({members[0], members[len(members) // 3], members[2 * len(members) // 3], members[-1]})
        for i in pick:
            r = {k: res[k][i] for k in ("a", "coeff", "delta", "idx")}
            r["steps"] = 30
            out = parity.check(sigs[i].G, radii, r, 1, full_grid="fft")
            assert out["selection_checked"] == 30, (N, i)


def test_grid_variants_are_bitwise_equivalent():
    # the autotuner's candidates (points per thread, CTA width) compute the
    # same values (on the per-class path, where the variants run): the paired
    # 32-points-per-thread transforms against the scalar ones at every first
    # radix (2: N = 32, 512, 8192, pass 0 in registers; 4: 64, 1024; 8: 128,
    # 2048; 16: 256, 4096)
    sigs = small_batch(n=20, Ns=(32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 512), seed=4)
    radii = W.radii_linear(24)
    ref = afd.afd_decompose_batch(sigs, radii, 5, autotune=False, persistent=False)
    for v in (0, 1, 2):
        r = afd.afd_decompose_batch(sigs, radii, 5, grid_variant=v, persistent=False)
        for i in range(len(sigs)):
            for key in ("a", "coeff", "delta", "idx"):
                assert np.array_equal(r[key][i], ref[key][i]), (v, i, key)


def test_autotuner_reports_choices_and_keeps_results():
    # the per-class path (persistent=False) is the one with grid-kernel variants
    sigs = small_batch(n=16, Ns=(1024, 2048, 4096, 8192), seed=6)
    radii = W.radii_linear(50)
    b = afd.afd_batch_create([g.size for g in sigs], radii, 6, persistent=False)
    r = afd.afd_batch_run(b, np.concatenate(sigs))
    tun = afd.afd_batch_tuning(b)
    b.close()
    assert [t["N"] for t in tun] == [1024, 2048, 4096, 8192]
    assert all(t["variant"] in (0, 1, 2) and t["us"] > 0 for t in tun)
    ref = afd.afd_decompose_batch(sigs, radii, 6, autotune=False, persistent=False)
    for i in range(len(sigs)):
        for key in ("a", "coeff", "delta", "idx"):
            assert np.array_equal(r[key][i], ref[key][i]), (i, key)
