"""Failure detection without a GPU fault: each kind of spin-wait in the
kernels is made to run out on purpose (a wait that nothing can satisfy); the
kernel flags the timeout and returns, the host reads AFD_ERR_TIMEOUT, and the
CUDA context stays usable for the next decomposition."""
import numpy as np
import pytest

from paper_1711_08604_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

afd = pytest.importorskip("paper_1711_08604_gb300")
AFD_ERR_TIMEOUT = -4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    afd._native.load()


@pytest.mark.parametrize("kind", [0, 1], ids=["grid_barrier", "mbarrier"])
def test_bounded_wait_runs_out_and_context_stays_usable(kind):
    status, seconds = afd.afd_selftest_wait_timeout(kind)
    print(f"wait kind {kind}: gave up after {seconds:.3f} s")
    assert status == AFD_ERR_TIMEOUT
    assert 0.0 < seconds < 60.0
    # the same context runs the next decomposition, equal to the oracle
    G = W.random_signal(256, 17)
    radii = np.array([0.0, 0.5, 0.9])
    for prec in (afd.AFD_FP64_PLAIN, afd.AFD_FP32_GUARDED):
        plan = afd.afd_plan_create(256, radii, precision=prec)
        res = afd.afd_decompose(plan, G, 3)
        plan.close()
        parity.check(G, radii, res, prec)
