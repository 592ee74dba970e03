"""The allocation-free entry point afd_inner_products_noalloc, called through the
C ABI.  It is meant for callers that cannot allocate device memory: work issued
while a stream is being captured, latency-critical loops where an allocation
could synchronise the device, and hosts that give the library a fixed,
pre-reserved memory pool.  Its scratch is a static device array shared by all
calls, so each check below runs two calls in a row (the second one on the
scratch the first left behind).

The checks: its FP64 inner products at the points a_k that afd_decompose
selected equal the coefficients afd_decompose returned for them; and at 64
arbitrary points of the disc, for sizes from one partial 512-sample chunk to the
128 chunks of N = 65536 (with ragged last chunks), every value equals the
oracle's direct rectangle rule of Eq. (formula1), within the FP64 coefficient
tolerance of the parity tests.  This file is named so pytest collects it last;
it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
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


def _close(got, want, G):
    E1 = np.mean(np.abs(G) ** 2)
    err = np.abs(got - want)
    bound = COEFF_TOL * np.abs(want) + ABS_FLOOR * np.sqrt(E1)
    assert np.all(np.isfinite(got))
    assert np.all(err <= bound), (int(np.argmax(err / bound)), float(np.max(err / bound)))


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
    # against the existing entry point: c_1 = <G, e_{a_1}>~ as afd_decompose
    # returned it, at the a_1 it selected
    torch, afd, lib = env
    cases = [(W.kernel_sum(), afd.AFD_FP32_GUARDED), (W.tones(item=2, K=3), afd.AFD_FP64_PLAIN)]
    for s, prec in cases:                       # two calls in a row
        plan = afd.afd_plan_create(s.N, s.radii, precision=prec)
        r = afd.afd_decompose(plan, s.G, 1)
        plan.close()
        got = _noalloc(torch, lib, s.G, r["a"][:1])
        _close(got, r["coeff"][:1], s.G)


def _points(seed, n=64):
    rng = np.random.default_rng(seed)
    pts = 0.95 * np.sqrt(rng.random(n)) * np.exp(2j * np.pi * rng.random(n))
    pts[0], pts[1], pts[2] = 0.0, 0.999 * np.exp(0.25j), -0.5   # the centre, near the circle, on an axis
    return pts


@pytest.mark.parametrize("N", [100, 512, 1000, 4096, 5000, 65536])
def test_noalloc_every_point_against_oracle(env, N):
    # 64 points; N = 100 (one partial chunk), 1000 and 5000 (ragged last
    # chunk), 65536 (all 128 chunks of the scratch); two calls in a row with
    # different points, every value against the oracle
    torch, afd, lib = env
    G = W.random_signal(N, 31 + N) + W.szego_sum(N, np.array([0.9 * np.exp(1.0j)]), np.array([1.5]))
    for call in range(2):
        pts = _points(N + call)
        got = _noalloc(torch, lib, G, pts)
        _close(got, oracle.inner_many(G, pts), G)


def test_noalloc_binding_and_device_memory(env):
    # the Python binding checks its tensors before calling the library; the
    # calls themselves leave the device's free memory unchanged
    torch, afd, lib = env
    s = W.kernel_sum(item=1)
    Gd = torch.from_numpy(s.G).cuda()
    pd = torch.from_numpy(_points(5)).cuda()
    out = torch.empty_like(pd)
    afd.afd_inner_products_noalloc(Gd, pd, out)        # first call: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        afd.afd_inner_products_noalloc(Gd, pd, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    _close(out.cpu().numpy(), oracle.inner_many(s.G, pd.cpu().numpy()), s.G)
    bad = [dict(G=Gd.to(torch.complex64)), dict(points=pd[::2]), dict(out=out[:10]),
           dict(G=Gd.cpu()), dict(points=torch.zeros(65, dtype=torch.complex128, device="cuda"))]
    for kw in bad:
        args = {"G": Gd, "points": pd, "out": out, **kw}
        with pytest.raises(ValueError):
            afd.afd_inner_products_noalloc(args["G"], args["points"], args["out"])


def test_noalloc_limits(env):
    torch, afd, lib = env
    s = W.kernel_sum(item=1)
    Gd = torch.from_numpy(s.G).cuda()
    pd = torch.zeros(65, dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(pd)
    assert lib.afd_inner_products_noalloc(Gd.data_ptr(), s.N, pd.data_ptr(), 65, out.data_ptr(), None) == -1
    assert b"n_points" in lib.afd_last_error()
    assert lib.afd_inner_products_noalloc(Gd.data_ptr(), 65537, pd.data_ptr(), 1, out.data_ptr(), None) == -1
    assert lib.afd_inner_products_noalloc(Gd.data_ptr(), 0, pd.data_ptr(), 1, out.data_ptr(), None) == -1
    host = np.zeros(2, dtype=np.complex128)
    assert lib.afd_inner_products_noalloc(Gd.data_ptr(), s.N, host.ctypes.data, 1, out.data_ptr(), None) == -1
    assert lib.afd_inner_products_noalloc(None, s.N, pd.data_ptr(), 1, out.data_ptr(), None) == -1
