"""CPU-side checks of the C ABI library: it builds, loads without a GPU and
exports every function include/afd.h declares.  No compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for fn in sorted(os.listdir(HEADER_DIR)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(afd_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_08604_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("afd_plan_create", "afd_plan_destroy", "afd_decompose", "afd_decompose_batch",
                 "afd_batch_create", "afd_batch_run", "afd_batch_destroy", "afd_status_str"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    lib.afd_status_str.restype = ctypes.c_char_p
    lib.afd_version.restype = ctypes.c_char_p
    assert lib.afd_status_str(0) == b"AFD_OK"
    assert lib.afd_status_str(-7) == b"AFD_ERR_NUMERIC"
    assert re.match(rb"^\d+\.\d+\.\d+$", lib.afd_version())


def test_defaults_without_gpu(lib):
    import paper_1711_08604_gb300 as afd
    o = afd.afd_plan_opts_default()
    assert o.precision == afd.AFD_FP32_GUARDED
    assert o.guard_cap == 16 and abs(o.guard_tau - 1e-4) < 1e-18
    assert o.use_graph == 1 and o.device == -1


def test_binding_names_match_header():
    import paper_1711_08604_gb300 as afd
    from paper_1711_08604_gb300 import _native
    for n in declared_functions():
        assert n in _native.SIGNATURES, n
        if n not in ("afd_plan_opts_default",):
            assert hasattr(afd, n), n


def test_wait_selftest_checks_arguments_before_any_cuda_call(lib):
    st, sec = ctypes.c_int(), ctypes.c_double()
    assert lib.afd_selftest_wait_timeout(-1, 2, ctypes.byref(st), ctypes.byref(sec)) == -1
    assert lib.afd_selftest_wait_timeout(-1, 0, None, ctypes.byref(sec)) == -1


@pytest.mark.parametrize("N,radii,kw", [
    (272, [0.1, 0.2], {}),                # 17 x 16: a prime factor above 13
    (64, [0.2, 0.1], {}),                 # radii not ascending
    (64, [0.1, 1.0], {}),                 # a radius outside [0, 1)
    (1 << 17, [0.1], {}),                 # above the largest size of any path
    (1 << 17, [0.1], {"precision": 0}),
    (64, [0.1], {"guard_cap": 0}),
    (64, [0.1, 0.2], {"force_a1_zero": True}),  # needs radii[0] == 0
])
def test_plan_arguments_checked_before_any_cuda_call(lib, N, radii, kw):
    # AFD_ERR_INVALID on a machine without a GPU: no CUDA call comes first
    import paper_1711_08604_gb300 as afd
    with pytest.raises(afd.AfdError) as e:
        afd.afd_plan_create(N, radii, **kw)
    assert e.value.status == -1


def test_nonuniform_plan_arguments_checked_before_any_cuda_call(lib):
    import numpy as np
    import paper_1711_08604_gb300 as afd
    theta = 2 * np.pi * (np.arange(64) + 0.5) / 64
    for args in [(theta[::-1], [0.0, 0.5], 64),      # angles not ascending
                 (theta, [0.0, 0.5], 100),           # L not a power of two
                 (theta, [0.5, 0.0], 64)]:           # radii not ascending
        with pytest.raises(afd.AfdError) as e:
            afd.afd_plan_create_nonuniform(*args)
        assert e.value.status == -1


@pytest.mark.parametrize("N,prec,valid", [
    (8, 1, True), (4, 1, False),              # smallest size
    (16384, 1, True), (8192, 0, True),        # largest resident size per precision
    (32768, 1, True), (16384, 0, True),       # split into resident sub-transforms
    (32768, 0, True), (65536, 0, True),
    (65536, 1, True),                         # the two-pass size (FP32 path)
    (1 << 17, 1, False), (1 << 17, 0, False), # above every path
    (9, 1, True), (3000, 1, True),            # 2^a 3^b 5^c
    (21, 1, True), (112, 1, True),            # factors 7: N = p^K sizes (7, 11, 13)
    (2401, 0, True), (1331, 1, True), (2197, 0, True),
    (17, 1, False), (272, 1, False), (7, 1, False),  # a factor 17; a single pass
    (12800, 1, True), (13500, 1, False),      # largest mixed-radix sizes: 16 N and
    (6400, 0, True), (6480, 0, False),        # 32 N bytes of shared memory <= 204800
])
def test_size_rules(lib, N, prec, valid):
    # a valid size passes every argument check: without a GPU the call then
    # fails at the device lookup (AFD_ERR_CUDA), with one it makes a plan
    import paper_1711_08604_gb300 as afd
    try:
        plan = afd.afd_plan_create(N, [0.5], precision=prec)
    except afd.AfdError as e:
        assert e.status == (-3 if valid else -1), (N, prec, e.status)
    else:
        assert valid, (N, prec)
        plan.close()


def test_batch_and_server_arguments_checked_before_any_cuda_call(lib):
    import paper_1711_08604_gb300 as afd
    bad_batches = [([256, 272], [0.1, 0.5], 5),    # a size with a factor 17
                   ([256, 512], [0.5, 0.1], 5),    # radii not ascending
                   ([256], [0.1], 0),              # K_max below 1
                   ([65536], [0.1], 5)]            # the FP32 two-pass size: single-signal plans only
    for N, radii, K in bad_batches:
        with pytest.raises(afd.AfdError) as e:
            afd.afd_batch_create(N, radii, K)
        assert e.value.status == -1
    with pytest.raises(afd.AfdError) as e:
        afd.afd_serve_create(1 << 19)              # budget below 1 MiB
    assert e.value.status == -1
    with pytest.raises(afd.AfdError) as e:
        afd.afd_serve_create(1 << 30, guard_cap=0)  # an invalid option
    assert e.value.status == -1


def test_noalloc_binding_rejects_bad_tensors_before_the_library():
    # the binding refuses tensors the kernel would misread (wrong dtype,
    # strided, host memory, too many points, short output) with ValueError,
    # before any call into the library
    torch = pytest.importorskip("torch")
    import paper_1711_08604_gb300 as afd
    G = torch.zeros(64, dtype=torch.complex128)
    p = torch.zeros(4, dtype=torch.complex128)
    for args in [(G.to(torch.complex64), p, p.clone()), (G, p, p.clone()), (G[::2], p, p.clone()),
                 (G, torch.zeros(8, dtype=torch.complex128)[::2], p.clone()), ("G", p, p)]:
        with pytest.raises(ValueError):
            afd.afd_inner_products_noalloc(*args)
