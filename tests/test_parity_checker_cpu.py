"""The GPU-vs-oracle checker (tests/parity.py) on the CPU: a result that the
oracle itself produced passes in every selection mode with every step checked,
and a result with one wrong pick (planted in an oracle-made result) fails in
every mode that checks that step, even though its coefficients and delta are
the forced oracle's own."""
import numpy as np
import pytest

import oracle
from paper_1711_08604_gb300 import workloads as W
from tests import parity


def _as_result(d):
    return {"steps": d["steps"], "idx": d["idx"].copy(), "a": d["a"].copy(), "coeff": d["coeff"].copy(),
            "delta": d["delta"].copy()}


@pytest.fixture(scope="module")
def case():
    s = W.kernel_sum(item=1, N=128, M=12, K=6)
    return s, oracle.decompose(s.G, s.radii, s.K)


@pytest.mark.parametrize("mode", [True, "fft"])
def test_oracle_result_passes_every_step(case, mode):
    s, d = case
    out = parity.check(s.G, s.radii, _as_result(d), 0, full_grid=mode)
    assert out["selection_checked"] == s.K
    assert out["coeff_rel"] == 0.0 and out["delta_abs"] == 0.0


@pytest.mark.parametrize("mode,grid_steps,caught", [(True, (), True), ("fft", (), True),
                                                    (False, (3,), True), (False, (1, 2), False)])
def test_wrong_pick_is_caught(case, mode, grid_steps, caught):
    s, d = case
    # step 3 takes another grid point far from a tie: the forced oracle's
    # coefficients and delta then match, only a selection check can see it
    wrong = d["idx"].copy()
    k = 2
    sgood, jgood = wrong[k]
    wrong[k] = ((sgood + 5) % s.radii.size, (jgood + s.N // 2) % s.N)
    forced = oracle.decompose(s.G, s.radii, s.K, forced_idx=wrong, compute_grid=True)
    assert forced["objused"][k] < 0.99 * forced["objmax"][k]
    res = _as_result(forced)
    if caught:
        with pytest.raises(AssertionError, match="step 3"):
            parity.check(s.G, s.radii, res, 0, full_grid=mode, grid_steps=grid_steps)
    else:
        out = parity.check(s.G, s.radii, res, 0, full_grid=mode, grid_steps=grid_steps)
        assert out["selection_checked"] == len(grid_steps)
