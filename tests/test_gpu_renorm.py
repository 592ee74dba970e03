"""The renormalised selection (objective divided by the discrete norm of the
kernel, (1 + r^N)/(1 - r^N)) on every path, against the oracle's renormalised
mode."""
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


def run(G, radii, K, prec, **kw):
    plan = afd.afd_plan_create(G.size, radii, precision=prec, **kw)
    try:
        return afd.afd_decompose(plan, G, K)
    finally:
        plan.close()


def two_kernel_signal(N=16):
    # e_b at r = 0.6 and a weaker e_b at r = 0.93: the plain objective prefers
    # the outer one (its discrete norm is 1.91 at N = 16), the renormalised one
    # the inner one
    b = np.array([0.6 * np.exp(2j * np.pi * 2 / N), 0.93 * np.exp(2j * np.pi * 10 / N)])
    return W.szego_sum(N, b, np.array([1.0, 0.5])), np.array([0.0, 0.3, 0.6, 0.85, 0.93])


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("persistent", [False, True])
def test_renormalised_pick_differs_and_matches_oracle(prec, persistent):
    G, radii = two_kernel_signal()
    ren = run(G, radii, 4, prec, renormalise=True, persistent=persistent)
    plain = run(G, radii, 4, prec, persistent=persistent)
    assert tuple(ren["idx"][0]) != tuple(plain["idx"][0])
    parity.check(G, radii, ren, prec, renormalise=True)
    parity.check(G, radii, plain, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("persistent", [False, True])
def test_renormalised_workload1(prec, persistent):
    # N = 256, radii up to 0.98: 0.98^256 = 0.0057, so the objective weights
    # differ by up to 1.1% between the two modes
    s = W.kernel_sum(item=2)
    res = run(s.G, s.radii, s.K, prec, renormalise=True, persistent=persistent)
    parity.check(s.G, s.radii, res, prec, renormalise=True)


@pytest.mark.parametrize("prec", PRECS)
def test_renormalised_persistent_equals_sequence(prec):
    s = W.kernel_sum(item=3)
    a = run(s.G, s.radii, 10, prec, renormalise=True, persistent=True)
    b = run(s.G, s.radii, 10, prec, renormalise=True, persistent=False)
    for key in ("a", "coeff", "delta", "idx"):
        assert np.array_equal(a[key], b[key]), key


def test_renormalised_batch_mixed_radix_and_serving():
    radii = W.radii_linear(40)
    sigs = [W.random_signal(N, 70 + i) for i, N in enumerate([64, 96, 256, 1000])]
    res = afd.afd_decompose_batch(sigs, radii, 5, renormalise=True)
    for i, G in enumerate(sigs):
        r = {k: res[k][i] for k in ("a", "coeff", "delta", "idx")}
        r["steps"] = int(res["steps"][i])
        parity.check(G, radii, r, afd.AFD_FP32_GUARDED, renormalise=True)
    srv = afd.afd_serve_create(256 << 20, renormalise=True)
    i = afd.afd_serve_submit(srv, sigs[2], radii, 5)
    o = afd.afd_serve_wait(srv, i, 60.0)
    srv.close()
    for key in ("a", "coeff", "delta", "idx"):
        assert np.array_equal(o[key], {k: res[k][2] for k in ("a", "coeff", "delta", "idx")}[key]), key


def test_renormalised_two_pass_equals_plain_when_rN_negligible():
    # N = 65536, r <= 0.999: r^N < 1e-28, the weights are 1 to FP64 rounding
    s = W.chirp(item=2, M=4, K=2)
    radii = np.array([0.0, 0.5, 0.9, 0.999])
    a = run(s.G, radii, 2, afd.AFD_FP32_GUARDED, renormalise=True)
    b = run(s.G, radii, 2, afd.AFD_FP32_GUARDED)
    assert np.array_equal(a["idx"], b["idx"]) and np.array_equal(a["coeff"], b["coeff"])
