"""GPU-vs-oracle comparison rules shared by the GPU tests.

Selection: the GPU's grid index must equal the oracle's argmax unless the
oracle's objective at the GPU's pick is within NEAR_TIE (relative) of the
oracle's maximum; in that case both are accepted and the oracle is
resynchronised to the GPU's pick (it is re-run forced to the GPU's index
sequence, so later steps compare like with like).

Coefficients: |c_gpu - c_ora| <= tol * |c_ora| + ABS_FLOOR * sqrt(E_1), where
ABS_FLOOR = 1000 eps (eps = 2^-52) is the FP64 rounding noise of an N-term sum
relative to the signal's RMS; it matters only for coefficients that are zero
or nearly so (e.g. a_1 = 0 imposed on a signal with zero mean).
Energy curve: |delta_gpu - delta_ora| <= 1e-5 * delta_ora + 1e-14.
"""
from __future__ import annotations

import hashlib

import numpy as np

import oracle

NEAR_TIE = 1e-6
DELTA_REL = 1e-5
COEFF_TOL = {0: 1e-11, 1: 1e-5}  # FP64 plain, FP32 guarded
ABS_FLOOR = 1e3 * np.finfo(np.float64).eps


_DIRECT_CACHE: dict = {}


def _oracle_forced(G, radii, idx, steps, force_a1_zero, renormalise, mode):
    """The oracle forced to the GPU's index sequence.  mode "direct" also
    computes its own O(M N^2) grid at every step (cached by inputs, so a second
    precision that picked the same points reuses it); "fft" keeps the
    remainders G_k for the FFT-route selection check."""
    if mode == "direct":
        key = hashlib.sha1(G.tobytes() + radii.tobytes() + idx.astype(np.int32).tobytes()
                           + bytes([force_a1_zero, renormalise])).hexdigest()
        if key not in _DIRECT_CACHE:
            _DIRECT_CACHE.clear()
            _DIRECT_CACHE[key] = oracle.decompose(G, radii, steps, force_a1_zero=force_a1_zero,
                                                  forced_idx=idx, compute_grid=True, renormalise=renormalise)
        return _DIRECT_CACHE[key]
    return oracle.decompose(G, radii, steps, force_a1_zero=force_a1_zero, forced_idx=idx,
                            compute_grid=False, renormalise=renormalise, keep_steps=(mode == "fft"))


def check(G, radii, res, prec: int, *, full_grid=True, grid_steps=(), force_a1_zero=False,
          energy_tol=0.0, coeff_tol=None, renormalise=False):
    """Compare a GPU result dict (afd_decompose output) with the oracle.

    Selection (the grid index of every step):
      full_grid=True   the oracle's own direct grid (Eq. (formula1) at every
                       grid point) at every step;
      full_grid="fft"  the oracle's FFT-route grid (Theorem 2.1 / Eq. (rcl),
                       ``oracle.select_fft``, pinned against the direct grid)
                       at every step, for sizes where the direct grid is too
                       slow;
      full_grid=False  the direct grid only at the steps listed in grid_steps.
    Coefficients, a_k and delta are checked at every step through the oracle
    forced to the GPU's picks.  Returns a dict of the largest observed errors
    and ``selection_checked``, the number of steps whose pick was checked
    against a whole grid.
    """
    G = np.asarray(G, dtype=np.complex128)
    radii = np.asarray(radii, dtype=np.float64)
    steps = int(res["steps"])
    assert steps >= 1
    idx = np.asarray(res["idx"]).reshape(steps, 2)
    tol = COEFF_TOL[prec] if coeff_tol is None else coeff_tol
    mode = "fft" if full_grid == "fft" else ("direct" if full_grid else "forced")
    ora = _oracle_forced(G, radii, idx, steps, bool(force_a1_zero), bool(renormalise), mode)
    E1 = ora["energy"][0]
    out = {"coeff_rel": 0.0, "delta_abs": 0.0, "a_abs": 0.0, "ties": 0, "selection_checked": 0}
    for k in range(steps):
        if mode != "forced" and not (force_a1_zero and k == 0):
            if mode == "direct":
                own, objmax, objpick = tuple(ora["own_idx"][k]), ora["objmax"][k], ora["objused"][k]
            else:
                sel = oracle.select_fft(ora["G_steps"][k], radii, pick=idx[k], renormalise=renormalise)
                own, objmax, objpick = sel["own"], sel["objmax"], sel["objpick"]
            if tuple(int(v) for v in idx[k]) != tuple(int(v) for v in own):
                assert objpick >= objmax * (1.0 - NEAR_TIE), (
                    f"step {k + 1}: GPU picked {tuple(idx[k])} (obj {objpick!r}), "
                    f"oracle {tuple(own)} (obj {objmax!r}) [{mode} grid]")
                out["ties"] += 1
            out["selection_checked"] += 1
        c_g, c_o = res["coeff"][k], ora["coeff"][k]
        err = abs(c_g - c_o)
        rel = err / max(abs(c_o), 1e-300)
        out["coeff_rel"] = max(out["coeff_rel"], rel if abs(c_o) > ABS_FLOOR * np.sqrt(E1) else 0.0)
        assert err <= tol * abs(c_o) + ABS_FLOOR * np.sqrt(E1), (
            f"step {k + 1}: coefficient {c_g} vs oracle {c_o} (rel {rel:.3e})")
        da = abs(res["a"][k] - ora["a"][k])
        out["a_abs"] = max(out["a_abs"], da)
        assert da <= 1e-14, f"step {k + 1}: a_k differs by {da}"
        dg, do = res["delta"][k + 1], ora["delta"][k + 1]
        out["delta_abs"] = max(out["delta_abs"], abs(dg - do))
        assert abs(dg - do) <= DELTA_REL * do + 1e-14, f"step {k + 1}: delta {dg} vs {do}"
    if mode == "forced":
        for k1 in grid_steps:
            k = k1 - 1
            if k >= steps or (force_a1_zero and k == 0):
                continue
            Gk = G if k == 0 else oracle.decompose(G, radii, k, force_a1_zero=force_a1_zero,
                                                    forced_idx=idx[:k], compute_grid=False)["G_final"]
            A = oracle.grid(Gk, radii).reshape(radii.size, G.size)
            obj = A.real ** 2 + A.imag ** 2
            if renormalise:
                obj = obj / np.array([oracle.kernel_norm2(G.size, r) for r in radii])[:, None]
            obj = obj.reshape(-1)
            f_own = int(np.argmax(obj))
            f_gpu = int(idx[k][0]) * G.size + int(idx[k][1])
            if f_gpu != f_own:
                assert obj[f_gpu] >= obj[f_own] * (1.0 - NEAR_TIE), (
                    f"step {k1}: GPU picked {tuple(idx[k])}, oracle {divmod(f_own, G.size)}")
                out["ties"] += 1
            out["selection_checked"] += 1
    if energy_tol > 0.0:
        # stopped exactly when the oracle's curve first reaches the tolerance
        d = ora["delta"][1:]
        first = int(np.argmax(d <= energy_tol)) + 1 if np.any(d <= energy_tol) else None
        if first is not None:
            assert steps == first or abs(d[steps - 1] - energy_tol) <= 1e-9 * energy_tol
    return out
