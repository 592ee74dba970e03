"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: an exact
identity the paper proves (the FFT route of Theorem 2.1 / Eq. (rcl)), closed
forms of the discrete Szego-kernel inner product, the reproducing property of
e_b, the decomposition identity Eq. (Sn) with the Takenaka-Malmquist system,
the energy identity of Sec. 2 in its exact discrete form, brute-force argmax
on small grids, and the relative errors printed in Tables 4 and 6.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1711_08604_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _discrete_szego_inner(a, b, N):
    """Closed form of the rectangle rule <e_b, e_a>~ on N points: summing the two
    geometric series and folding indices mod N gives
    sqrt(1-|a|^2) sqrt(1-|b|^2) (1 - (a conj b)^N) / ((1 - a conj b)(1 - a^N)(1 - conj(b)^N))."""
    bc = np.conj(b)
    return (np.sqrt(1 - abs(a) ** 2) * np.sqrt(1 - abs(b) ** 2) * (1 - (a * bc) ** N)
            / ((1 - a * bc) * (1 - a ** N) * (1 - bc ** N)))


@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_direct_sum_equals_fft_route(N):
    G = W.random_signal(N, 17 + N)
    radii = np.array([0.0, 0.1, 0.5, 0.9, 0.99])
    A = oracle.grid(G, radii)
    B = oracle.grid_fft(G, radii)
    assert np.max(np.abs(A - B)) <= 1e-13 * max(1.0, np.max(np.abs(B)))


def test_direct_sum_equals_fft_route_workload1():
    s = W.kernel_sum()
    A = oracle.grid(s.G, s.radii)
    B = oracle.grid_fft(s.G, s.radii)
    assert np.max(np.abs(A - B)) <= 1e-12 * np.max(np.abs(B))


@pytest.mark.parametrize("N,rows", [(4096, (0.0, 0.5, 0.995)), (65536, (0.3, 0.999)), (3000, (0.2, 0.97)),
                                    (2187, (0.9,))])
def test_fft_route_sampled_rows_at_large_N(N, rows):
    # the FFT route of Theorem 2.1 at the large transform sizes of the
    # workloads (and two sizes that are not powers of two), against the direct
    # rectangle rule at sampled grid points: whole rows at N = 4096, 512 angles
    # per row (a contiguous run and random ones) at the others
    G = W.random_signal(N, 5 + N) + W.szego_sum(N, np.array([0.97 * np.exp(0.3j)]), np.array([2.0]))
    radii = np.array(rows)
    B = oracle.grid_fft(G, radii)
    rng = np.random.default_rng(N)
    for s, r in enumerate(radii):
        js = np.arange(N) if N <= 4096 else np.unique(np.concatenate([np.arange(256), rng.integers(0, N, 256)]))
        A = oracle.inner_many(G, r * np.exp(2j * np.pi * js / N))
        assert np.max(np.abs(A - B[s, js])) <= 1e-12 * np.max(np.abs(B[s])), (N, r)


def test_fft_selection_equals_direct_selection():
    # select_fft (blocks of radii) picks the direct oracle's argmax, ties
    # included: G = 1 (every angle of r = 0 ties), random signals, one radius
    # per block and all radii in one block
    for G, radii in [(np.ones(32, complex), np.array([0.0, 0.5])),
                     (W.random_signal(64, 8), np.array([0.0, 0.2, 0.7, 0.95])),
                     (W.random_signal(48, 9), np.array([0.1, 0.6, 0.9]))]:
        d = oracle.decompose(G, radii, 1)
        for rows in (0, 1, 2):
            sel = oracle.select_fft(G, radii, pick=tuple(d["own_idx"][0]), rows_per_chunk=rows)
            assert sel["own"] == tuple(d["own_idx"][0])
            assert abs(sel["objmax"] - d["objmax"][0]) <= 1e-13 * d["objmax"][0]
            assert sel["objpick"] == sel["objmax"]
    # renormalised selection
    G, radii = W.random_signal(32, 2), np.array([0.0, 0.5, 0.9, 0.97])
    d = oracle.decompose(G, radii, 1, renormalise=True)
    assert oracle.select_fft(G, radii, renormalise=True)["own"] == tuple(d["own_idx"][0])


def test_keep_steps_are_the_remainders():
    # G_steps[k] is the remainder the (k+1)-th selection runs on: G_1 = G, and
    # each next one is the Sec. 2 update of the previous with that step's a_k, c_k
    s = W.kernel_sum(item=2)
    d = oracle.decompose(s.G, s.radii, 6, keep_steps=True)
    assert np.array_equal(d["G_steps"][0], s.G)
    for k in range(5):
        nxt = oracle.update(d["G_steps"][k], d["a"][k], d["coeff"][k])
        assert np.array_equal(nxt, d["G_steps"][k + 1])
        assert d["coeff"][k] == oracle.inner(d["G_steps"][k], d["a"][k])
    f = oracle.decompose(s.G, s.radii, 6, forced_idx=d["idx"], compute_grid=False, keep_steps=True)
    assert np.array_equal(f["G_steps"], d["G_steps"])


@pytest.mark.parametrize("N", [8, 64, 256])
def test_inner_matches_discrete_szego_closed_form(N):
    rng = np.random.default_rng(5 + N)
    for _ in range(6):
        a = 0.97 * np.sqrt(rng.random()) * np.exp(2j * np.pi * rng.random())
        b = 0.97 * np.sqrt(rng.random()) * np.exp(2j * np.pi * rng.random())
        G = W.szego_sum(N, np.array([b]), np.array([1.0]))
        got = oracle.inner(G, a)
        want = _discrete_szego_inner(a, b, N)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want))
    # a = b: the discrete norm ||e_b||^2 = (1 - |b|^{2N}) / |1 - b^N|^2
    b = 0.8 * np.exp(0.3j)
    G = W.szego_sum(N, np.array([b]), np.array([1.0]))
    want = (1 - abs(b) ** (2 * N)) / abs(1 - b ** N) ** 2
    assert abs(oracle.inner(G, b) - want) <= 1e-12 * want
    assert abs(oracle.energy(G) - want) <= 1e-12 * want


def test_inner_many_matches_closed_form_and_grid():
    N = 64
    rng = np.random.default_rng(8)
    b = 0.8 * np.exp(0.7j)
    G = W.szego_sum(N, np.array([b]), np.array([1.0]))
    pts = 0.95 * np.sqrt(rng.random(9)) * np.exp(2j * np.pi * rng.random(9))
    got = oracle.inner_many(G, pts)
    want = np.array([_discrete_szego_inner(a, b, N) for a in pts])
    assert np.max(np.abs(got - want)) <= 1e-12
    radii = np.array([0.3, 0.7])
    A = oracle.grid(G, radii)
    on_grid = np.array([r * np.exp(2j * np.pi * j / N) for r in radii for j in range(N)])
    assert np.max(np.abs(oracle.inner_many(G, on_grid) - A.reshape(-1))) <= 1e-13


def test_inner_at_zero_is_mean():
    G = W.random_signal(128, 3)
    assert abs(oracle.inner(G, 0.0) - G.mean()) <= 1e-15 * 128


def test_reproducing_kernel_selects_b():
    # b on the grid: radius index 25 of radii i/50 and angle index 17 of N = 256.
    N, radii = 256, W.radii_linear(50)
    s, j = 25, 17
    b = radii[s] * np.exp(2j * np.pi * j / N)
    G = W.szego_sum(N, np.array([b]), np.array([1.0]))
    d = oracle.decompose(G, radii, 1)
    assert tuple(d["idx"][0]) == (s, j)
    assert abs(abs(d["coeff"][0]) - 1.0) <= 1e-13
    assert abs(d["a"][0] - b) <= 1e-15
    assert np.max(np.abs(d["G_final"])) <= 1e-13
    assert d["delta"][1] <= 1e-25


def test_constant_signal_ties_go_to_lowest_index():
    # G = 1: <G, e_a>~ = sqrt(1-r^2)/(1 - a^N); at r = 0 all N angles tie exactly
    # at the largest value 1, so the lowest flat index (0, 0) wins.
    N, radii = 64, np.array([0.0, 0.2, 0.5])
    d = oracle.decompose(np.ones(N, dtype=complex), radii, 1)
    assert tuple(d["idx"][0]) == (0, 0)
    assert abs(d["coeff"][0] - 1.0) <= 1e-15
    assert np.max(np.abs(d["G_final"])) <= 1e-15


@pytest.mark.parametrize("seed", range(4))
def test_argmax_brute_force_small(seed):
    N = 16
    G = W.random_signal(N, 100 + seed)
    radii = np.array([0.0, 0.3, 0.6, 0.85])
    A = oracle.grid(G, radii)
    obj = A.real ** 2 + A.imag ** 2
    flat = int(np.argmax(obj.reshape(-1)))  # numpy returns the first maximum
    d = oracle.decompose(G, radii, 1)
    assert tuple(d["idx"][0]) == (flat // N, flat % N)
    assert abs(d["coeff"][0] - A.reshape(-1)[flat]) == 0.0
    assert d["objmax"][0] == obj.reshape(-1)[flat]


def test_energy_identity_exact_discrete_form():
    # E_{k+1} = ||G_k - c_k e_{a_k}||^2_N because the Blaschke factor is unimodular
    # on the circle; with <G_k, e_a>~ = c_k and ||e_a||^2_N = (1+r^N)/(1-r^N) for
    # a on the grid this is E_{k+1} = E_k - |c_k|^2 + |c_k|^2 2 r^N / (1 - r^N).
    s = W.kernel_sum()
    d = oracle.decompose(s.G, s.radii, 20)
    E, c, a = d["energy"], d["coeff"], d["a"]
    N = s.N
    for k in range(d["steps"]):
        r = abs(a[k])
        want = E[k] - abs(c[k]) ** 2 + abs(c[k]) ** 2 * 2 * r ** N / (1 - r ** N)
        assert abs(E[k + 1] - want) <= 1e-12 * E[0]


def test_energy_identity_plain_form_when_rN_negligible():
    # Sec. 2: ||G||^2 = sum_k |<G_k, e_{a_k}>|^2 + ||G_{n+1}||^2 when r_max^N <= 1e-14.
    s = W.kernel_sum()
    radii = np.arange(18) / 20.0  # r_max = 0.85, 0.85^256 ~ 8e-19
    d = oracle.decompose(s.G, radii, 20)
    lhs = d["energy"][0]
    rhs = np.sum(np.abs(d["coeff"]) ** 2) + d["energy"][-1]
    assert abs(lhs - rhs) <= 1e-12 * lhs


def test_decomposition_identity_Sn():
    # Eq. (Sn): G = sum_k c_k B_k + G_{n+1} prod_k (z - a_k)/(1 - conj(a_k) z) pointwise,
    # B_k = e_{a_k} prod_{l<k} (z - a_l)/(1 - conj(a_l) z) (without the 1/sqrt(2 pi)
    # factor, in the normalised measure); hence delta_n = ||G - S_n||^2_N / ||G||^2_N.
    s = W.kernel_sum()
    n = 8
    d = oracle.decompose(s.G, s.radii, n)
    z = W.sample_points(s.N)
    S = np.zeros_like(z)
    prod = np.ones_like(z)
    for a, c in zip(d["a"], d["coeff"]):
        e = np.sqrt(1 - abs(a) ** 2) / (1 - np.conj(a) * z)
        S += c * e * prod
        prod *= (z - a) / (1 - np.conj(a) * z)
    resid = s.G - S
    assert np.max(np.abs(resid - d["G_final"] * prod)) <= 1e-12 * np.max(np.abs(s.G))
    delta = np.mean(np.abs(resid) ** 2) / np.mean(np.abs(s.G) ** 2)
    assert abs(delta - d["delta"][n]) <= 1e-12


def test_forced_sequence_reproduces_free_run():
    s = W.kernel_sum(item=3)
    free = oracle.decompose(s.G, s.radii, 6)
    forced = oracle.decompose(s.G, s.radii, 6, forced_idx=free["idx"], compute_grid=False)
    assert np.array_equal(free["idx"], forced["idx"])
    assert np.array_equal(free["coeff"], forced["coeff"])
    assert np.array_equal(free["delta"], forced["delta"])


def test_stop_on_energy_tolerance():
    s = W.kernel_sum(item=1)
    full = oracle.decompose(s.G, s.radii, 10)
    tol = full["delta"][4] * 1.0000001
    d = oracle.decompose(s.G, s.radii, 10, energy_tol=tol)
    assert d["steps"] == 4


def test_bad_arguments_raise():
    with pytest.raises(ValueError):
        oracle.grid(np.ones(8), [0.0, 1.0])
    with pytest.raises(ValueError):
        oracle.decompose(np.ones(8), [0.5, 0.2], 2)
    with pytest.raises(ValueError):
        oracle.decompose(np.ones(8), [0.1, 0.2], 2, force_a1_zero=True)


def _golden(name):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and not ln.startswith("#")]
    return np.array([float(r[1]) for r in rows])


@pytest.mark.parametrize("fname,signal,tol", [
    ("table4_case1_delta.txt", W.paper_f1, 2e-3),
    ("table6_case2_delta.txt", W.paper_f2, 3e-3),
])
def test_paper_tables_soft_pin(fname, signal, tol):
    # Tables 4 and 6 (Sec. 4.1): delta after n steps, N = 1024, radii 0..0.8, a_1 = 0.
    want = _golden(fname)
    d = oracle.decompose(signal(1024), W.radii_paper(), 10, force_a1_zero=True)
    got = d["delta"][1:11]
    assert np.max(np.abs(got - want)) <= tol


# ----------------------------------------------- renormalised selection --
# The discrete objective |<G, e_a>~|^2 is inflated at small N with r -> 1
# because the discrete norm of e_a exceeds 1; the renormalised selection
# divides it by ||e_a||_N^2 (the paper follows the continuous norm; this is the
# optional reading of the discrete one).

@pytest.mark.parametrize("N,r", [(8, 0.0), (16, 0.5), (32, 0.97), (64, 0.99), (256, 0.98), (1024, 0.8)])
def test_kernel_norm_matches_geometric_series(N, r):
    # (1/N) sum_m |e_a(z_m)|^2 for a on the grid sums the aliased geometric
    # series of |e_a|^2 = (1 - r^2) sum_{l, l'} ...: (1 + r^N) / (1 - r^N)
    assert abs(oracle.kernel_norm2(N, r) - (1 + r ** N) / (1 - r ** N)) <= 1e-13 * (1 + r ** N) / (1 - r ** N)


def test_renormalised_selection_brute_force():
    # On a small grid with radii near 1 the renormalised pick is the argmax of
    # |A|^2 / ||e_a||^2 with the norm summed at every grid point, and differs
    # from the plain pick.
    N = 16
    radii = np.array([0.0, 0.3, 0.6, 0.85, 0.93])
    # e_b at r = 0.6 plus a weaker e_b at r = 0.93, whose plain objective is
    # inflated by ||e_b||^2 = 1.91 at N = 16
    b = np.array([0.6 * np.exp(2j * np.pi * 2 / N), 0.93 * np.exp(2j * np.pi * 10 / N)])
    G = W.szego_sum(N, b, np.array([1.0, 0.5]))
    A = oracle.grid(G, radii).reshape(radii.size, N)
    z = np.exp(2j * np.pi * np.arange(N) / N)
    norm2 = np.empty((radii.size, N))
    for s, r in enumerate(radii):
        for j in range(N):
            a = r * np.exp(2j * np.pi * j / N)
            e = np.sqrt(1 - r * r) / (1 - np.conj(a) * z)
            norm2[s, j] = np.mean(e.real ** 2 + e.imag ** 2)
    obj = (A.real ** 2 + A.imag ** 2) / norm2
    want = np.unravel_index(int(np.argmax(obj)), obj.shape)
    ren = oracle.decompose(G, radii, 1, renormalise=True)
    plain = oracle.decompose(G, radii, 1)
    assert tuple(ren["idx"][0]) == tuple(int(v) for v in want)
    assert abs(ren["objused"][0] - obj[want]) <= 1e-12 * obj[want]
    assert tuple(ren["idx"][0]) != tuple(plain["idx"][0])
    assert ren["coeff"][0] == A[want]  # the coefficient is <G, e_a>~ itself


def test_renormalised_equals_plain_when_rN_negligible():
    s = W.paper_f1(1024)
    radii = W.radii_paper()  # r <= 0.8: r^N ~ 1e-100
    ren = oracle.decompose(s, radii, 6, renormalise=True)
    plain = oracle.decompose(s, radii, 6)
    assert np.array_equal(ren["idx"], plain["idx"])
    assert np.allclose(ren["coeff"], plain["coeff"], rtol=1e-14, atol=0)


# ------------------------------------------------------ non-uniform samples --
# The weighted rectangle rule on z_m = exp(i theta_m) (the remark after Step 2
# of Sec. 3.2), a grid of L equispaced angles.

def test_nonuniform_oracle_reduces_to_uniform():
    s = W.kernel_sum(item=1)
    N = s.N
    theta = 2 * np.pi * np.arange(N) / N
    w = np.full(N, 1.0 / N)
    nu = oracle.nu_decompose(s.G, theta, w, s.radii, N, 6)
    un = oracle.decompose(s.G, s.radii, 6)
    assert np.array_equal(nu["idx"], un["idx"])
    assert np.max(np.abs(nu["coeff"] - un["coeff"])) <= 1e-13 * np.max(np.abs(un["coeff"]))
    assert np.max(np.abs(nu["delta"] - un["delta"])) <= 1e-13


@pytest.mark.parametrize("seed", [0, 1])
def test_nonuniform_inner_equals_series_route(seed):
    # 1/(1 - a conj(z)) = sum_l a^l conj(z)^l for |a| < 1: the inner product is
    # sqrt(1 - |a|^2) sum_l a^l c_l with c_l = sum_m w_m G(z_m) exp(-i l theta_m)
    # (the non-uniform DFT the GPU route folds onto L angles)
    N = 37
    theta = W.nonuniform_angles(N, 10 + seed)
    w = W.trapezoid_weights(theta)
    G = W.random_signal(N, 40 + seed)
    l = np.arange(4000)
    c = (np.exp(-1j * np.outer(l, theta)) * (w * G)[None, :]).sum(axis=1)
    for a in (0.0, 0.5 * np.exp(1j), 0.97 * np.exp(-2.5j)):
        series = np.sqrt(1 - abs(a) ** 2) * np.sum(a ** l * c)
        assert abs(oracle.nu_inner(G, theta, w, a) - series) <= 1e-12 * max(1.0, abs(series))


def test_nonuniform_weights_sum_to_one_and_update_keeps_modulus():
    N = 50
    theta = W.nonuniform_angles(N, 3)
    w = W.trapezoid_weights(theta)
    assert abs(w.sum() - 1.0) <= 1e-14
    G = W.random_signal(N, 4)
    a = 0.8 * np.exp(0.7j)
    c = oracle.nu_inner(G, theta, w, a)
    G1 = oracle.nu_update(G, theta, a, c)
    # |(1 - conj(a) z) / (z - a)| = 1 on the circle: the energy after the
    # update is that of G - c e_a
    z = np.exp(1j * theta)
    r = G - c * np.sqrt(1 - abs(a) ** 2) / (1 - np.conj(a) * z)
    assert abs(oracle.nu_energy(G1, w) - np.sum(w * np.abs(r) ** 2)) <= 1e-13 * np.sum(w * np.abs(r) ** 2)


def test_nonuniform_brute_force_argmax():
    N, L = 29, 16
    theta = W.nonuniform_angles(N, 8)
    w = W.trapezoid_weights(theta)
    G = W.random_signal(N, 9)
    radii = np.array([0.0, 0.4, 0.7, 0.9])
    best, arg = -1.0, None
    for s, r in enumerate(radii):
        for j in range(L):
            c = oracle.nu_inner(G, theta, w, r * np.exp(2j * np.pi * j / L))
            v = c.real * c.real + c.imag * c.imag
            if v > best:
                best, arg = v, (s, j)
    d = oracle.nu_decompose(G, theta, w, radii, L, 1)
    assert tuple(d["idx"][0]) == arg and d["objmax"][0] == best


# ----------------------------------------------- off-grid refinement (opt-in)
# The refinement is not in the paper; these pins tie it to closed forms: the
# reproducing kernel off the grid, the stationarity of the discrete objective
# (checked by finite differences of the oracle's own inner product, a
# different code path from the Newton sums), and the exact discrete energy
# identity at a point off the grid, ||e_a||_N^2 = Re((1 + conj(a)^N) / (1 - conj(a)^N)).

@pytest.mark.parametrize("b", [0.6 * np.exp(2j * np.pi * 0.1234), 0.2 + 0.05j, -0.45 - 0.3j])
def test_refinement_recovers_an_off_grid_kernel(b):
    # G = e_b with |b|^N negligible: <G, e_a>~ is maximal at a = b, with
    # |c| = 1, and the remainder vanishes
    N = 256
    G = W.szego_sum(N, np.array([b]), np.array([1.0]))
    radii = W.radii_linear(20)
    r = oracle.decompose(G, radii, 2, offgrid_iters=30)
    assert abs(r["a"][0] - b) < 1e-12
    assert abs(abs(r["coeff"][0]) - 1.0) < 1e-12
    assert r["delta"][1] < 1e-20
    # idx keeps the grid point the refinement started from: the grid argmax
    r0 = oracle.decompose(G, radii, 1)
    assert np.array_equal(r["idx"][0], r0["idx"][0])


def test_refinement_reaches_a_stationary_point_and_gains():
    N = 512
    G = W.random_signal(N, 21) + W.szego_sum(N, np.array([0.7 * np.exp(0.3j)]), np.array([2.0]))
    radii = W.radii_linear(16)
    r0 = oracle.decompose(G, radii, 1)
    a, c = oracle.refine(G, r0["a"][0], 30)
    f = lambda p: abs(oracle.inner(G, p)) ** 2  # noqa: E731
    assert f(a) >= f(r0["a"][0])
    assert abs(c - oracle.inner(G, a)) < 1e-12 * abs(c)
    h = 1e-5
    gx = (f(a + h) - f(a - h)) / (2 * h)
    gy = (f(a + 1j * h) - f(a - 1j * h)) / (2 * h)
    assert np.hypot(gx, gy) < 1e-6 * f(a)  # a maximum: zero gradient, and
    for d in (1e-3, 1e-3j, -1e-3, -1e-3j):
        assert f(a + d) < f(a)                # lower values around it


def test_refinement_energy_identity_off_the_grid():
    N = 64  # small N with radii near 1: the aliasing term matters
    G = W.random_signal(N, 5)
    radii = np.array([0.0, 0.5, 0.8, 0.9])
    r = oracle.decompose(G, radii, 6, offgrid_iters=20)
    assert r["steps"] == 6
    E = r["energy"]
    for k in range(6):
        a, c = r["a"][k], r["coeff"][k]
        norm2 = np.real((1 + np.conj(a) ** N) / (1 - np.conj(a) ** N))
        assert abs(E[k + 1] - (E[k] - 2 * abs(c) ** 2 + abs(c) ** 2 * norm2)) < 1e-12 * E[0]


def test_refinement_off_is_the_plain_decomposition():
    s = W.kernel_sum()
    r0 = oracle.decompose(s.G, s.radii, 5)
    r1 = oracle.decompose(s.G, s.radii, 5, offgrid_iters=0)
    for key in ("a", "coeff", "idx", "delta"):
        assert np.array_equal(r0[key], r1[key])
