"""The allocation-free entry point afd_inner_products_noalloc, called through the
C ABI.  It is meant for callers that cannot allocate device memory (inside stream
capture, in latency-critical loops, or under a host-imposed fixed memory pool);
its scratch is a static device array shared by all calls.

The check: its FP64 inner products at the points a_k that afd_decompose selected
must equal the coefficients afd_decompose returned for them, within the FP64
coefficient tolerance of the parity tests, on two calls in a row (so the second
call runs on scratch the first one left behind).  This file is named so pytest
collects it last; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1711_08604_gb300 import workloads as W

pytestmark = pytest.mark.gpu

COEFF_TOL = 1e-11                               # FP64 coefficient tolerance of tests/parity.py
ABS_FLOOR = 1e3 * np.finfo(np.float64).eps      # times sqrt(E_1), as in tests/parity.py


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1711_08604_gb300 as afd
    lib = ctypes.CDLL(afd._native.load()._name)
    f = lib.afd_inner_products_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p]
    lib.afd_last_error.restype = ctypes.c_char_p
    return torch, afd, lib


def _reference(afd, G, radii, K, prec):
    """a_k and c_k of the existing entry point on the remainders G_k it starts from:
    step 1 only, so c_1 = <G, e_{a_1}>~ for the original samples."""
    plan = afd.afd_plan_create(G.size, radii, precision=prec)
    r = afd.afd_decompose(plan, G, K)
    plan.close()
    return r["a"][:1], r["coeff"][:1]


def _noalloc(torch, lib, G, pts):
    Gd = torch.from_numpy(G).cuda()
    pd = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    out = torch.full_like(pd, complex(np.nan, np.nan))
    torch.cuda.synchronize()
    st = lib.afd_inner_products_noalloc(Gd.data_ptr(), G.size, pd.data_ptr(), pts.size,
                                        out.data_ptr(), None)
    assert st == 0, lib.afd_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_decompose_on_two_calls(env):
    torch, afd, lib = env
    cases = [(W.kernel_sum(), afd.AFD_FP32_GUARDED), (W.tones(item=2, K=3), afd.AFD_FP64_PLAIN)]
    for s, prec in cases:                       # two calls in a row
        a, c = _reference(afd, s.G, s.radii, 1, prec)
        got = _noalloc(torch, lib, s.G, a)
        E1 = np.mean(np.abs(s.G) ** 2)
        err = np.abs(got - c)
        assert np.all(err <= COEFF_TOL * np.abs(c) + ABS_FLOOR * np.sqrt(E1)), (got, c)


def test_noalloc_many_points_and_limits(env):
    torch, afd, lib = env
    s = W.kernel_sum(item=1)
    rng = np.random.default_rng(11)
    pts = 0.95 * np.sqrt(rng.random(64)) * np.exp(2j * np.pi * rng.random(64))
    first = _noalloc(torch, lib, s.G, pts)
    again = _noalloc(torch, lib, s.G, pts)
    assert np.array_equal(first, again)
    # every point against the existing entry point: a 1-radius plan whose only
    # grid circle passes through the point selects it when it is the circle's maximum
    for p in pts[:4]:
        r = abs(p)
        j = int(round(np.angle(p) / (2 * np.pi) * s.N)) % s.N
        on_grid = r * np.exp(2j * np.pi * j / s.N)
        got = _noalloc(torch, lib, s.G, np.array([on_grid]))[0]
        plan = afd.afd_plan_create(s.N, np.array([r]), precision=afd.AFD_FP32_GUARDED)
        res = afd.afd_decompose(plan, s.G, 1)
        plan.close()
        if tuple(res["idx"][0]) == (0, j):
            assert abs(got - res["coeff"][0]) <= COEFF_TOL * abs(res["coeff"][0]) + 1e-13
    Gd = torch.from_numpy(s.G).cuda()
    pd = torch.zeros(65, dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(pd)
    assert lib.afd_inner_products_noalloc(Gd.data_ptr(), s.N, pd.data_ptr(), 65, out.data_ptr(), None) == -1
    assert b"n_points" in lib.afd_last_error()
    assert lib.afd_inner_products_noalloc(Gd.data_ptr(), 65537, pd.data_ptr(), 1, out.data_ptr(), None) == -1
    host = np.zeros(2, dtype=np.complex128)
    assert lib.afd_inner_products_noalloc(Gd.data_ptr(), s.N, host.ctypes.data, 1, out.data_ptr(), None) == -1
