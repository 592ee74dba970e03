"""CUDA path (through the C ABI) against the FP64 oracle on seeded inputs."""
import numpy as np
import pytest

import oracle
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


def run(G, radii, K, prec, tol=0.0, **kw):
    plan = afd.afd_plan_create(G.size, radii, precision=prec, **kw)
    try:
        return afd.afd_decompose(plan, G, K, tol), plan
    finally:
        pass


@pytest.mark.parametrize("prec", PRECS)
def test_workload1_kernel_sum_full_parity(prec):
    s = W.kernel_sum()
    res, _ = run(s.G, s.radii, s.K, prec)
    assert res["steps"] == s.K
    parity.check(s.G, s.radii, res, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("item", [1, 2, 3])
def test_workload1_more_items(prec, item):
    s = W.kernel_sum(item=item)
    res, _ = run(s.G, s.radii, 12, prec)
    parity.check(s.G, s.radii, res, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_reproducing_kernel(prec):
    N, radii = 256, W.radii_linear(50)
    b = radii[25] * np.exp(2j * np.pi * 17 / N)
    G = W.szego_sum(N, np.array([b]), np.array([1.0]))
    res, _ = run(G, radii, 1, prec)
    assert tuple(res["idx"][0]) == (25, 17)
    assert abs(abs(res["coeff"][0]) - 1.0) <= 1e-13
    assert res["delta"][1] <= 1e-24


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [8, 16, 32, 64, 128, 512, 1024, 2048])
def test_small_and_ragged_sizes(prec, N):
    G = W.random_signal(N, 7 * N)
    radii = np.array([0.0, 0.05, 0.3, 0.55, 0.8, 0.9, 0.97])
    res, _ = run(G, radii, 6, prec)
    parity.check(G, radii, res, prec)


@pytest.mark.parametrize("prec,N", [(afd.AFD_FP64_PLAIN, 8192), (afd.AFD_FP32_GUARDED, 8192),
                                    (afd.AFD_FP32_GUARDED, 16384)])
def test_largest_resident_sizes(prec, N):
    # the largest transforms held on chip: N = 8192 (the FP64 limit) and
    # N = 16384 (FP32, 32 points per thread); every grid point at every step
    G = W.random_signal(N, 11 * N)
    radii = np.array([0.0, 0.4, 0.9, 0.995])
    res, _ = run(G, radii, 3, prec)
    assert res["steps"] == 3
    parity.check(G, radii, res, prec)


SPLIT = [(afd.AFD_FP32_GUARDED, 32768), (afd.AFD_FP64_PLAIN, 16384), (afd.AFD_FP64_PLAIN, 32768),
         (afd.AFD_FP64_PLAIN, 65536)]


@pytest.mark.parametrize("prec,N", SPLIT)
def test_split_sizes_full_grid(prec, N):
    # transforms longer than one CTA holds on chip (2^14 FP32 points, 2^13
    # FP64), split by output index into 2, 4 or 8 resident sub-transforms: every
    # grid point of every step against the oracle's FFT-route grid, radii from
    # 0 (an N-way tie) to 0.999, coefficients and delta against the oracle
    G = W.random_signal(N, 13 * N) + W.szego_sum(N, np.array([0.95 * np.exp(2.0j), 0.6j]), np.array([1.0, 0.5]))
    radii = np.array([0.0, 0.3, 0.7, 0.9, 0.99, 0.999])
    res, _ = run(G, radii, 4, prec)
    assert res["steps"] == 4
    assert parity.check(G, radii, res, prec, full_grid="fft")["selection_checked"] == 4


@pytest.mark.parametrize("prec,N", SPLIT)
def test_split_sizes_reproducing_kernel(prec, N):
    # G = e_b, b on the grid: the split selection finds b (FP64: exactly; FP32:
    # b or, within the near-tie rule, a neighbouring angle) with |c_1| = 1
    radii = W.radii_linear(20)
    j0 = N // 3 + 1  # an index of every residue class mod 8 as N varies
    b = radii[17] * np.exp(2j * np.pi * j0 / N)
    G = W.szego_sum(N, np.array([b]), np.array([1.0]))
    res, _ = run(G, radii, 1, prec)
    s, j = (int(v) for v in res["idx"][0])
    if prec == afd.AFD_FP64_PLAIN:
        assert (s, j) == (17, j0)
        assert abs(abs(res["coeff"][0]) - 1.0) <= 1e-12
    else:
        assert s == 17 and abs(j - j0) <= 4
        assert abs(res["coeff"][0]) ** 2 >= 1.0 - parity.NEAR_TIE


@pytest.mark.parametrize("prec", PRECS)
def test_single_radius_and_zero_radius_ties(prec):
    # only r = 0: every angle ties exactly, the lowest index must win
    N = 64
    G = W.random_signal(N, 3)
    res, _ = run(G, np.array([0.0]), 3, prec)
    for k in range(3):
        assert tuple(res["idx"][k]) == (0, 0)
    parity.check(G, np.array([0.0]), res, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_constant_signal(prec):
    N = 128
    res, _ = run(np.ones(N, dtype=complex), np.array([0.0, 0.2, 0.5]), 1, prec)
    assert tuple(res["idx"][0]) == (0, 0)
    assert abs(res["coeff"][0] - 1.0) <= 1e-14
    assert res["delta"][1] <= 1e-28


@pytest.mark.parametrize("prec", PRECS)
def test_energy_tolerance_stop(prec):
    s = W.kernel_sum(item=5)
    full, _ = run(s.G, s.radii, 10, prec)
    tol = float(full["delta"][5]) * 1.0001
    res, _ = run(s.G, s.radii, 10, prec, tol=tol)
    assert res["steps"] == 5
    parity.check(s.G, s.radii, res, prec, energy_tol=tol)


@pytest.mark.parametrize("prec", PRECS)
def test_paper_table4_forced_a1(prec):
    G = W.paper_f1(1024)
    radii = W.radii_paper()
    res, _ = run(G, radii, 10, prec, force_a1_zero=True)
    parity.check(G, radii, res, prec, force_a1_zero=True)
    want = np.array([float(l.split()[1]) for l in open("tests/golden/table4_case1_delta.txt")
                     if l.strip() and not l.startswith("#")])
    assert np.max(np.abs(res["delta"][1:11] - want)) <= 2e-3


@pytest.mark.parametrize("prec", PRECS)
def test_workload2_tones_every_step(prec):
    # N = 4096, M = 200, K = 50: the selection of every step against the
    # oracle's own direct grid (all 819,200 points by Eq. (formula1), 3.4e9
    # complex terms per step; the oracle run is shared by the two precisions
    # when they pick the same points) and against the FFT-route grid;
    # coefficients and delta at every step
    s = W.tones()
    res, _ = run(s.G, s.radii, s.K, prec)
    assert res["steps"] == s.K
    out = parity.check(s.G, s.radii, res, prec, full_grid=True)
    assert out["selection_checked"] == s.K
    assert parity.check(s.G, s.radii, res, prec, full_grid="fft")["selection_checked"] == s.K


def test_determinism_and_graph_equivalence():
    s = W.tones(item=1, K=12)
    r1, _ = run(s.G, s.radii, s.K, 1)
    r2, _ = run(s.G, s.radii, s.K, 1)
    r3, _ = run(s.G, s.radii, s.K, 1, use_graph=False)
    for k in ("a", "coeff", "delta", "idx"):
        assert np.array_equal(r1[k], r2[k])
        assert np.array_equal(r1[k], r3[k])


def test_plan_reuse_with_different_K():
    s = W.kernel_sum(item=2)
    plan = afd.afd_plan_create(s.N, s.radii)
    a = afd.afd_decompose(plan, s.G, 4)
    b = afd.afd_decompose(plan, s.G, 9)
    c = afd.afd_decompose(plan, s.G, 4)
    assert np.array_equal(a["coeff"], b["coeff"][:4])
    assert np.array_equal(a["coeff"], c["coeff"])


def test_device_pointers():
    import torch
    s = W.kernel_sum(item=4)
    plan = afd.afd_plan_create(s.N, s.radii)
    host = afd.afd_decompose(plan, s.G, 8)
    Gd = torch.from_numpy(s.G).cuda()
    out = {"a": torch.zeros(16, dtype=torch.float64, device="cuda"),
           "coeff": torch.zeros(16, dtype=torch.float64, device="cuda"),
           "delta": torch.zeros(9, dtype=torch.float64, device="cuda"),
           "idx": torch.zeros(16, dtype=torch.int32, device="cuda")}
    dev = afd.afd_decompose(plan, Gd, 8, out=out)
    assert dev["steps"] == 8
    assert np.array_equal(out["coeff"].cpu().numpy().view(np.complex128), host["coeff"])
    assert np.array_equal(out["idx"].cpu().numpy().reshape(8, 2), host["idx"])
    assert np.array_equal(out["delta"].cpu().numpy(), host["delta"])
    # with every output on the device the step records stay there until
    # afd_plan_last_info asks for them; they are the host-output run's
    ref = afd.afd_plan_create(s.N, s.radii)
    afd.afd_decompose(ref, s.G, 8)
    want = afd.afd_plan_last_info(ref, 8)
    got = afd.afd_plan_last_info(plan, 8)
    for k in ("n_cand", "flags", "obj32"):
        assert np.array_equal(got[k], want[k]), k
    # a later host-output call on the same plan refreshes the records
    afd.afd_decompose(plan, s.G, 3)
    got3 = afd.afd_plan_last_info(plan, 3)
    assert np.array_equal(got3["obj32"], want["obj32"][:3])


def test_device_outputs_of_batches_and_resumed_runs():
    # outputs in device memory are written on the device by a gather kernel;
    # they must equal the host-output results bitwise, for batches (with
    # steps_out) and for resumed runs (steps_done, G_final and E_1 as well)
    import ctypes
    import torch
    lib = afd._lib()
    sigs = [W.kernel_sum(item=i, N=N).G for i, N in enumerate((256, 1024, 256))]
    radii = W.radii_linear(16)
    K = 6
    host = afd.afd_decompose_batch(sigs, radii, K)
    b = afd.afd_batch_create([g.size for g in sigs], radii, K)
    dev = {"a": torch.zeros(2 * 3 * K, dtype=torch.float64, device="cuda"),
           "c": torch.zeros(2 * 3 * K, dtype=torch.float64, device="cuda"),
           "d": torch.zeros(3 * (K + 1), dtype=torch.float64, device="cuda"),
           "ix": torch.zeros(2 * 3 * K, dtype=torch.int32, device="cuda"),
           "st": torch.zeros(3, dtype=torch.int32, device="cuda")}
    Gp = torch.from_numpy(np.concatenate(sigs)).cuda()
    st = lib.afd_batch_run(b.handle, Gp.data_ptr(), 0.0, dev["a"].data_ptr(), dev["c"].data_ptr(),
                           dev["d"].data_ptr(), dev["ix"].data_ptr(), dev["st"].data_ptr())
    b.close()
    assert st == 0
    assert np.array_equal(dev["st"].cpu().numpy(), host["steps"])
    for i in range(3):
        n = int(host["steps"][i])
        a = dev["a"].cpu().numpy()[2 * i * K: 2 * (i * K + n)].view(np.complex128)
        c = dev["c"].cpu().numpy()[2 * i * K: 2 * (i * K + n)].view(np.complex128)
        d = dev["d"].cpu().numpy()[i * (K + 1): i * (K + 1) + n + 1]
        ix = dev["ix"].cpu().numpy()[2 * i * K: 2 * (i * K + n)].reshape(n, 2)
        assert np.array_equal(a, host["a"][i]) and np.array_equal(c, host["coeff"][i])
        assert np.array_equal(d, host["delta"][i]) and np.array_equal(ix, host["idx"][i])
    # resumed single-signal run with every output on the device
    s = W.tones(item=2, K=10)
    plan = afd.afd_plan_create(s.N, s.radii)
    p1 = afd.afd_decompose_from(plan, s.G, 4)
    ref = afd.afd_decompose_from(plan, p1["G_final"], 6, E1=p1["E1"])
    o = {"a": torch.zeros(12, dtype=torch.float64, device="cuda"),
         "c": torch.zeros(12, dtype=torch.float64, device="cuda"),
         "d": torch.zeros(7, dtype=torch.float64, device="cuda"),
         "ix": torch.zeros(12, dtype=torch.int32, device="cuda"),
         "n": torch.zeros(1, dtype=torch.int32, device="cuda"),
         "gf": torch.zeros(s.N, dtype=torch.complex128, device="cuda"),
         "e1": torch.zeros(1, dtype=torch.float64, device="cuda")}
    G1 = torch.from_numpy(p1["G_final"]).cuda()
    st = lib.afd_decompose_from(plan.handle, G1.data_ptr(), p1["E1"], 6, 0.0, o["a"].data_ptr(), o["c"].data_ptr(),
                                o["d"].data_ptr(), o["ix"].data_ptr(), o["n"].data_ptr(), o["gf"].data_ptr(),
                                o["e1"].data_ptr())
    plan.close()
    assert st == 0 and int(o["n"].item()) == ref["steps"] == 6
    assert np.array_equal(o["a"].cpu().numpy().view(np.complex128), ref["a"])
    assert np.array_equal(o["c"].cpu().numpy().view(np.complex128), ref["coeff"])
    assert np.array_equal(o["d"].cpu().numpy(), ref["delta"])
    assert np.array_equal(o["ix"].cpu().numpy().reshape(6, 2), ref["idx"])
    assert np.array_equal(o["gf"].cpu().numpy(), ref["G_final"]) and o["e1"].item() == ref["E1"]


def test_invalid_arguments():
    with pytest.raises(afd.AfdError) as e:
        afd.afd_plan_create(272, [0.1, 0.2])  # 17 * 16: a prime factor above 13
    assert e.value.status == -1
    with pytest.raises(afd.AfdError):
        afd.afd_plan_create(64, [0.2, 0.1])
    with pytest.raises(afd.AfdError):
        afd.afd_plan_create(64, [0.1, 1.0])
    with pytest.raises(afd.AfdError):
        afd.afd_plan_create(1 << 17, [0.1])
    with pytest.raises(afd.AfdError):
        afd.afd_plan_create(1 << 17, [0.1], precision=0)
    with pytest.raises(afd.AfdError):
        afd.afd_plan_create(64, [0.1], guard_cap=0)
    with pytest.raises(afd.AfdError):
        afd.afd_plan_create(64, [0.1, 0.2], force_a1_zero=True)
    plan = afd.afd_plan_create(64, [0.0, 0.5])
    with pytest.raises(afd.AfdError):
        afd.afd_decompose(plan, np.ones(64, complex), 0)


@pytest.mark.parametrize("prec", PRECS)
def test_zero_signal(prec):
    res, _ = run(np.zeros(64, dtype=complex), np.array([0.0, 0.5]), 2, prec)
    assert res["steps"] == 2
    assert tuple(res["idx"][0]) == (0, 0)
    assert np.all(res["coeff"] == 0)
    assert np.all(res["delta"][1:] == 0)


@pytest.mark.parametrize("prec", PRECS)
def test_nan_input_reports_numeric_error(prec):
    G = W.random_signal(64, 1)
    G[5] = np.nan
    plan = afd.afd_plan_create(64, np.array([0.0, 0.5]), precision=prec)
    with pytest.raises(afd.AfdError) as e:
        afd.afd_decompose(plan, G, 3)
    assert e.value.status == -7


@pytest.mark.parametrize("N", [8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096])
def test_persistent_kernel_equals_kernel_sequence(N):
    # one cooperative launch per decomposition vs one launch per kernel per
    # step: the same FP64 arithmetic in the same order, so bitwise equal
    # results.  Every transform shape of the persistent kernel: groups
    # narrower than a warp (forward transform by all of warp 0), one warp,
    # and whole-warp groups on named barriers with the split input.
    s = W.tones(item=3, N=N, M=40, K=12) if N >= 1024 else W.kernel_sum(item=3, N=N, M=40, K=12)
    a, _ = run(s.G, s.radii, s.K, 1, persistent=True)
    b, _ = run(s.G, s.radii, s.K, 1, persistent=False)
    for k in ("a", "coeff", "delta", "idx"):
        assert np.array_equal(a[k], b[k]), k
    tol = float(a["delta"][6]) * 1.0000001
    if tol > 0.0 and float(a["delta"][5]) > tol:  # the stop rule fires at step 6
        c, _ = run(s.G, s.radii, s.K, 1, tol=tol, persistent=True)
        assert c["steps"] == 6 and np.array_equal(c["coeff"], a["coeff"][:6])


def test_persistent_kernel_several_tiles_per_cta():
    # more radius tiles than CTAs (one CTA per SM): CTAs loop over tiles, and
    # tiles after the first read their radial powers and weights from memory
    s = W.tones(item=6, N=4096, M=400, K=8)
    a, _ = run(s.G, s.radii, s.K, 1, persistent=True)
    b, _ = run(s.G, s.radii, s.K, 1, persistent=False)
    for k in ("a", "coeff", "delta", "idx"):
        assert np.array_equal(a[k], b[k]), k
    assert parity.check(s.G, s.radii, a, 1, full_grid="fft")["selection_checked"] == s.K


def test_persistent_kernel_profiled():
    s = W.tones(item=4, K=8)
    plan = afd.afd_plan_create(s.N, s.radii)
    afd.afd_plan_set_profiling(plan, True)
    r = afd.afd_decompose(plan, s.G, s.K)
    kt = afd.afd_plan_kernel_times(plan)
    assert r["steps"] == s.K
    assert kt["persistent"][1] == 1 and kt["persistent"][0] > 0
    assert parity.check(s.G, s.radii, r, 1, full_grid="fft")["selection_checked"] == s.K


@pytest.mark.parametrize("prec", PRECS)
def test_synthesis_recovers_energy_curve(prec):
    # Eq. (Sn): G - S_n = G_{n+1} times a unimodular Blaschke product on the
    # circle, so ||G - S_n||^2 / ||G||^2 = delta_n for every n
    s = W.kernel_sum(item=7)
    res, _ = run(s.G, s.radii, 10, prec)
    S = afd.afd_synthesize(s.N, res["a"], res["coeff"], all_prefixes=True)
    E1 = np.mean(np.abs(s.G) ** 2)
    for n in range(1, 11):
        d = np.mean(np.abs(s.G - S[n - 1]) ** 2) / E1
        assert abs(d - res["delta"][n]) <= 1e-12 + 1e-10 * res["delta"][n]
    # against the expansion written out with numpy
    z = W.sample_points(s.N)
    Sn = np.zeros_like(z)
    prod = np.ones_like(z)
    for a, c in zip(res["a"], res["coeff"]):
        Sn += c * np.sqrt(1 - abs(a) ** 2) / (1 - np.conj(a) * z) * prod
        prod *= (z - a) / (1 - np.conj(a) * z)
    assert np.max(np.abs(S[-1] - Sn)) <= 1e-12 * np.max(np.abs(s.G))
    last = afd.afd_synthesize(s.N, res["a"], res["coeff"])
    assert np.array_equal(last, S[-1])


@pytest.mark.parametrize("prec", PRECS)
def test_paper_table6_forced_a1(prec):
    G = W.paper_f2(1024)
    radii = W.radii_paper()
    res, _ = run(G, radii, 10, prec, force_a1_zero=True)
    parity.check(G, radii, res, prec, force_a1_zero=True)
    want = np.array([float(l.split()[1]) for l in open("tests/golden/table6_case2_delta.txt")
                     if l.strip() and not l.startswith("#")])
    assert np.max(np.abs(res["delta"][1:11] - want)) <= 3e-3


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [128, 256, 512, 1024, 2048, 4096])
def test_paper_table9_sweep(prec, N):
    # the N-sweep of Table 9: f1 sampled on N points, radii 0..0.8, 10 steps
    G = W.paper_f1(N)
    radii = W.radii_paper()
    res, _ = run(G, radii, 10, prec, force_a1_zero=True)
    parity.check(G, radii, res, prec, force_a1_zero=True)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("persistent", [True, False])
def test_checkpoint_resume_is_bitwise(prec, persistent):
    # a decomposition split into two calls (the state between calls is the
    # remainder and E_1) equals one call
    s = W.tones(item=5, K=30)
    plan = afd.afd_plan_create(s.N, s.radii, precision=prec, persistent=persistent)
    full = afd.afd_decompose_from(plan, s.G, 30)
    p1 = afd.afd_decompose_from(plan, s.G, 12)
    p2 = afd.afd_decompose_from(plan, p1["G_final"], 18, E1=p1["E1"])
    plan.close()
    assert p1["E1"] == full["E1"] and p2["E1"] == full["E1"]
    for key in ("a", "coeff", "idx"):
        assert np.array_equal(np.concatenate([p1[key], p2[key]]), full[key]), key
    assert np.array_equal(p1["delta"], full["delta"][:13])
    assert np.array_equal(p2["delta"], full["delta"][12:])
    assert np.array_equal(p2["G_final"], full["G_final"])
    # the remainder is the oracle's G_{k+1} to FP64 rounding
    ora = oracle.decompose(s.G, s.radii, 12, forced_idx=p1["idx"], compute_grid=False)
    assert np.max(np.abs(p1["G_final"] - ora["G_final"])) <= 1e-10 * np.max(np.abs(s.G))
