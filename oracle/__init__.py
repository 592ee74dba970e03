"""Plain, slow FP64 CPU oracle of 1-D (Core) AFD (arXiv:1711.08604).

TEST INFRASTRUCTURE ONLY.  This package is imported by the test suite, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
product package ``paper_1711_08604_gb300`` never imports, links or runs it.
It shares no code with the CUDA path.

The arithmetic lives in ``afd_oracle.c`` (plain C99 complex, FP64, OpenMP over
grid points); this module only compiles it with gcc and marshals numpy arrays.
What each function computes, with the paper passage it follows:

* ``inner``   -- the rectangle-rule inner product <G, e_a>~, Sec. 3.1 Eq. (formula1).
* ``inner_many`` -- the same at a list of points.
* ``grid``    -- the same on the polar grid a_{s,j} = r_s exp(2 pi i j/N), Eq. (ku1)/(term81).
* ``update``  -- the reduced-remainder (Blaschke) update of Sec. 2.
* ``energy``  -- (1/N) sum |G(z_m)|^2, the discrete norm in the measure dt/2pi of Eq. (formula2).
* ``decompose`` -- the greedy loop of Sec. 2 with the grid selection of Sec. 3.2
  (Step 2) and the relative error delta of Eq. (er).
* ``kernel_norm2`` -- the discrete squared norm of e_a at a grid point (renormalised selection).
* ``grid_fft``, ``select_fft`` -- the same grid and selection by the FFT route of
  Theorem 2.1 / Eq. (rcl) with library FFTs in FP64 (fast enough to check the
  selection at every step of the large workloads; pinned against ``grid``).
* ``nu_inner``, ``nu_update``, ``nu_energy``, ``nu_decompose`` (``afd_oracle_nu.c``) --
  the same on non-uniform samples z_m = exp(i theta_m) with quadrature weights
  w_m (the remark after Step 2 of Sec. 3.2) and a grid of L equispaced angles.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "afd_oracle.c"), os.path.join(_HERE, "afd_oracle_nu.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle sources into ``liboracle.so`` (gcc -O2, OpenMP, no fast-math, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(f) for f in _SRCS)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.oracle_inner.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp]
        lib.oracle_grid.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
        lib.oracle_inner_many.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
        lib.oracle_update.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, _dp]
        lib.oracle_energy.argtypes = [ctypes.c_int, _dp]
        lib.oracle_energy.restype = ctypes.c_double
        lib.oracle_decompose.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int,
                                         _dp, _dp, _ip, _ip, _dp, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
        lib.oracle_refine.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      _dp, _dp]
        lib.oracle_kernel_norm2.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.oracle_kernel_norm2.restype = ctypes.c_double
        lib.oracle_nu_inner.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]
        lib.oracle_nu_energy.argtypes = [ctypes.c_int, _dp, _dp]
        lib.oracle_nu_energy.restype = ctypes.c_double
        lib.oracle_nu_update.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, _dp]
        lib.oracle_nu_decompose.argtypes = [ctypes.c_int, _dp, _dp, _dp, ctypes.c_int, _dp, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, _ip, ctypes.c_int,
                                            _dp, _dp, _ip, _ip, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _cvec(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


def _rvec(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    _load().oracle_set_num_threads(int(n))


def inner(G, a: complex) -> complex:
    """<G, e_a>~ by the rectangle rule of Eq. (formula1)."""
    g = _cvec(G)
    out = np.zeros(2)
    if _load().oracle_inner(g.size, _p(g), float(np.real(a)), float(np.imag(a)), _p(out)) != 0:
        raise ValueError("oracle_inner: bad arguments")
    return complex(out[0], out[1])


def inner_many(G, points) -> np.ndarray:
    """<G, e_a>~ at each of the given points (Eq. (formula1))."""
    g, pts = _cvec(G), _cvec(points)
    out = np.zeros_like(pts)
    if _load().oracle_inner_many(g.size, _p(g), pts.size, _p(pts), _p(out)) != 0:
        raise ValueError("oracle_inner_many: bad arguments")
    return out


def refine(G, a0: complex, iters: int) -> tuple:
    """Off-grid refinement of a point (not in the paper): damped Newton steps
    on log |<G, e_a>~|^2 over the open disc from a0, at most ``iters`` of
    them.  Returns (a, <G, e_a>~)."""
    g = _cvec(G)
    a = np.zeros(2)
    c = np.zeros(2)
    if _load().oracle_refine(g.size, _p(g), float(np.real(a0)), float(np.imag(a0)), int(iters), _p(a), _p(c)) != 0:
        raise ValueError("oracle_refine: bad arguments")
    return complex(a[0], a[1]), complex(c[0], c[1])


def grid(G, radii) -> np.ndarray:
    """(M, N) complex array of <G, e_{a_{s,j}}>~ over the polar grid, Eq. (term81)."""
    g, r = _cvec(G), _rvec(radii)
    A = np.zeros((r.size, g.size), dtype=np.complex128)
    if _load().oracle_grid(g.size, _p(g), r.size, _p(r), _p(A)) != 0:
        raise ValueError("oracle_grid: bad arguments")
    return A


def update(G, a: complex, c: complex) -> np.ndarray:
    """G_{k+1} from G_k, a_k and c_k = <G_k, e_{a_k}> (Sec. 2)."""
    g = _cvec(G)
    out = np.zeros_like(g)
    if _load().oracle_update(g.size, _p(g), float(np.real(a)), float(np.imag(a)),
                             float(np.real(c)), float(np.imag(c)), _p(out)) != 0:
        raise ValueError("oracle_update: bad arguments")
    return out


def energy(G) -> float:
    """(1/N) sum_m |G(z_m)|^2."""
    g = _cvec(G)
    return float(_load().oracle_energy(g.size, _p(g)))


def kernel_norm2(N: int, r: float) -> float:
    """(1/N) sum_m |e_a(z_m)|^2 at a grid point of radius r (direct sum)."""
    v = _load().oracle_kernel_norm2(int(N), float(r))
    if v < 0:
        raise ValueError("oracle_kernel_norm2: bad arguments")
    return v


def decompose(G, radii, K_max: int, energy_tol: float = 0.0, force_a1_zero: bool = False,
              forced_idx=None, compute_grid: bool = True, renormalise: bool = False,
              keep_steps: bool = False, offgrid_iters: int = 0) -> dict:
    """Core AFD: K_max greedy steps (or until delta <= energy_tol).

    ``renormalise`` selects by |<G_k, e_a>~|^2 / ||e_a||_N^2 (the discrete norm,
    ``kernel_norm2``) instead of |<G_k, e_a>~|^2.

    ``forced_idx`` is an optional (K_max, 2) int array of grid indices (s, j)
    to use instead of the argmax (rows with s < 0 are free).  With
    ``compute_grid=False`` every step must be forced and the O(M N^2) grid is
    skipped; the coefficient then comes from ``inner`` at the forced point.
    ``keep_steps`` adds ``G_steps``: (steps, N) array of G_k at the start of
    every step k (the remainder the step's selection runs on).
    ``offgrid_iters`` > 0 refines each step's point off the grid (``refine``)
    before its coefficient and update; ``idx`` keeps the grid starting point.
    """
    g, r = _cvec(G), _rvec(radii)
    K = int(K_max)
    fi = None
    if forced_idx is not None:
        fi = np.full((K, 2), -1, dtype=np.int32)
        f = np.asarray(forced_idx, dtype=np.int32).reshape(-1, 2)
        fi[: min(K, f.shape[0])] = f[:K]
        fi = np.ascontiguousarray(fi)
    a = np.zeros(K, dtype=np.complex128)
    c = np.zeros(K, dtype=np.complex128)
    idx = np.zeros((K, 2), dtype=np.int32)
    own = np.zeros((K, 2), dtype=np.int32)
    objmax = np.zeros(K)
    obj2 = np.zeros(K)
    objused = np.zeros(K)
    delta = np.zeros(K + 1)
    E = np.zeros(K + 1)
    Gf = np.zeros_like(g)
    Gs = np.zeros((K, g.size), dtype=np.complex128) if keep_steps else None
    steps = _load().oracle_decompose(
        g.size, _p(g), r.size, _p(r), K, float(energy_tol), int(bool(force_a1_zero)), int(bool(renormalise)),
        fi.ctypes.data_as(_ip) if fi is not None else None, int(bool(compute_grid)),
        _p(a), _p(c), idx.ctypes.data_as(_ip), own.ctypes.data_as(_ip), _p(objmax), _p(obj2),
        _p(objused), _p(delta), _p(E), _p(Gf), _p(Gs) if Gs is not None else None, int(offgrid_iters))
    if steps < 0:
        raise ValueError("oracle_decompose: bad arguments")
    out = {"steps": steps, "a": a[:steps], "coeff": c[:steps], "idx": idx[:steps],
           "own_idx": own[:steps], "objmax": objmax[:steps], "obj2": obj2[:steps],
           "objused": objused[:steps], "delta": delta[: steps + 1], "energy": E[: steps + 1],
           "G_final": Gf}
    if keep_steps:
        out["G_steps"] = Gs[:steps]
    return out


# ------------------------------------------- the FFT route of Theorem 2.1 --

def _fft_module():
    try:
        import scipy.fft as sf
        return sf, {"workers": max(1, os.cpu_count() or 1)}
    except ImportError:  # numpy's pocketfft, one thread
        return np.fft, {}


def grid_fft(G, radii, workers: int = 0) -> np.ndarray:
    """(M, N) grid of <G, e_{a_{s,j}}>~ by the FFT route of Theorem 2.1 / Eq. (rcl).

    Expanding 1/(1 - a conj(z_m)) = sum_l (a conj(z_m))^l and folding l mod N
    (z_m^N = 1) gives, with c_l = sum_m G(z_m) w^{-ml} (Eq. (term4)),
        <G, e_{a_{s,j}}>~ = sqrt(1 - r_s^2) / (N (1 - r_s^N)) sum_l r_s^l c_l w^{jl},
    one forward DFT of the samples and, per radius, one inverse DFT of the
    spectrum weighted by r_s^l.  The DFTs are library FFTs (scipy, else numpy)
    in FP64.  The identity is exact; it is pinned against the direct sum
    ``grid`` / ``inner_many`` by the test suite.
    """
    g, r = _cvec(G), _rvec(radii)
    N = g.size
    fft, kw = _fft_module()
    if workers and kw:
        kw = {"workers": workers}
    c = fft.fft(g, **kw)
    # r_s^l = r_s^(l mod B) * r_s^(B (l div B)): two short power tables and
    # one product per entry instead of M N calls of pow (relative error a few
    # ulp); the row scale sqrt(1 - r^2) / (1 - r^N) rides on the short table
    B = min(N, 256)
    scale = np.sqrt(1.0 - r * r) / (1.0 - r ** N)
    lo = scale[:, None] * r[:, None] ** np.arange(B, dtype=np.float64)[None, :]
    hi = r[:, None] ** (B * np.arange(-(-N // B), dtype=np.float64))[None, :]
    w = (hi[:, :, None] * lo[:, None, :]).reshape(r.size, -1)[:, :N]
    # the library's inverse DFT carries the 1/N of the formula
    return fft.ifft(w * c[None, :], axis=1, **kw)


def select_fft(G, radii, pick=None, renormalise: bool = False, rows_per_chunk: int = 0) -> dict:
    """Maximal selection of Step 2 (Sec. 3.2) on the grid computed by ``grid_fft``.

    Returns ``own`` = (s, j), the argmax of |<G, e_a>~|^2 (divided by the
    discrete norm ``kernel_norm2`` per radius when ``renormalise``), ties to
    the lowest flat index s N + j; ``objmax``, its value; and, when ``pick``
    = (s, j) is given, ``objpick``, the objective there.  The grid is formed
    in blocks of radii (host threads take blocks in parallel), so memory stays
    near 50 N rows_per_chunk bytes per thread.
    """
    from concurrent.futures import ThreadPoolExecutor

    g, r = _cvec(G), _rvec(radii)
    N, M = g.size, r.size
    if rows_per_chunk <= 0:
        rows_per_chunk = max(1, min(M, (1 << 21) // max(N, 1)))
    starts = list(range(0, M, rows_per_chunk))

    def block(s0):
        rr = r[s0:s0 + rows_per_chunk]
        A = grid_fft(g, rr, workers=1)
        obj = A.real ** 2 + A.imag ** 2
        if renormalise:
            obj /= np.array([kernel_norm2(N, x) for x in rr])[:, None]
        f = int(np.argmax(obj))  # first occurrence: the lowest flat index
        vp = None
        if pick is not None and s0 <= int(pick[0]) < s0 + rr.size:
            vp = float(obj[int(pick[0]) - s0, int(pick[1])])
        return float(obj.reshape(-1)[f]), (s0 + f // N, f % N), vp

    nthreads = max(1, min(len(starts), os.cpu_count() or 1, 16))
    if nthreads == 1:
        parts = [block(s0) for s0 in starts]
    else:
        with ThreadPoolExecutor(nthreads) as ex:
            parts = list(ex.map(block, starts))
    best, own, objpick = -1.0, None, None
    for v, o, vp in parts:  # blocks in ascending radius order: strict > keeps the lowest index
        if v > best:
            best, own = v, o
        if vp is not None:
            objpick = vp
    return {"own": own, "objmax": best, "objpick": objpick}


# ------------------------------------------------------- non-uniform samples --

def nu_inner(G, theta, w, a: complex) -> complex:
    """sqrt(1-|a|^2) sum_m w_m G(z_m) / (1 - a conj(z_m)), z_m = exp(i theta_m)."""
    g, t, ww = _cvec(G), _rvec(theta), _rvec(w)
    out = np.zeros(2)
    if _load().oracle_nu_inner(g.size, _p(g), _p(t), _p(ww), float(np.real(a)), float(np.imag(a)), _p(out)) != 0:
        raise ValueError("oracle_nu_inner: bad arguments")
    return complex(out[0], out[1])


def nu_energy(G, w) -> float:
    """sum_m w_m |G(z_m)|^2."""
    g, ww = _cvec(G), _rvec(w)
    return _load().oracle_nu_energy(g.size, _p(g), _p(ww))


def nu_update(G, theta, a: complex, c: complex) -> np.ndarray:
    """The Blaschke update of Sec. 2 at the points exp(i theta_m)."""
    g, t = _cvec(G), _rvec(theta)
    out = np.zeros_like(g)
    if _load().oracle_nu_update(g.size, _p(g), _p(t), float(np.real(a)), float(np.imag(a)),
                                float(np.real(c)), float(np.imag(c)), _p(out)) != 0:
        raise ValueError("oracle_nu_update: bad arguments")
    return out


def nu_decompose(G, theta, w, radii, L: int, K_max: int, energy_tol: float = 0.0, forced_idx=None,
                 compute_grid: bool = True) -> dict:
    """Core AFD on non-uniform samples with a grid of L equispaced angles (flat
    index s L + j); the same outputs as ``decompose``."""
    g, t, ww, r = _cvec(G), _rvec(theta), _rvec(w), _rvec(radii)
    K = int(K_max)
    fi = None
    if forced_idx is not None:
        fi = np.full((K, 2), -1, dtype=np.int32)
        f = np.asarray(forced_idx, dtype=np.int32).reshape(-1, 2)
        fi[: min(K, f.shape[0])] = f[:K]
        fi = np.ascontiguousarray(fi)
    a = np.zeros(K, dtype=np.complex128)
    c = np.zeros(K, dtype=np.complex128)
    idx = np.zeros((K, 2), dtype=np.int32)
    own = np.zeros((K, 2), dtype=np.int32)
    objmax, obj2, objused = np.zeros(K), np.zeros(K), np.zeros(K)
    delta, E = np.zeros(K + 1), np.zeros(K + 1)
    Gf = np.zeros_like(g)
    steps = _load().oracle_nu_decompose(
        g.size, _p(g), _p(t), _p(ww), r.size, _p(r), int(L), K, float(energy_tol),
        fi.ctypes.data_as(_ip) if fi is not None else None, int(bool(compute_grid)),
        _p(a), _p(c), idx.ctypes.data_as(_ip), own.ctypes.data_as(_ip), _p(objmax), _p(obj2),
        _p(objused), _p(delta), _p(E), _p(Gf))
    if steps < 0:
        raise ValueError("oracle_nu_decompose: bad arguments")
    return {"steps": steps, "a": a[:steps], "coeff": c[:steps], "idx": idx[:steps],
            "own_idx": own[:steps], "objmax": objmax[:steps], "obj2": obj2[:steps],
            "objused": objused[:steps], "delta": delta[: steps + 1], "energy": E[: steps + 1],
            "G_final": Gf}
