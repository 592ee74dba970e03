"""GB300 (sm_103a) FFT-accelerated 1-D (Core) AFD, after arXiv:1711.08604.

Thin Python binding of the C ABI in ``include/afd.h``: the functions below
carry the C names and only marshal arguments (numpy arrays or torch tensors,
host or CUDA) into ``lib/libafd.so``.  Every step of the decomposition runs
in the library's CUDA kernels; importing a function that needs the library
raises if it has not been built.

Quick use::

    import numpy as np, paper_1711_08604_gb300 as afd
    plan = afd.afd_plan_create(4096, np.arange(200) / 200)
    res = afd.afd_decompose(plan, G, K_max=50)      # G: complex128, N samples
    res["a"], res["coeff"], res["delta"], res["idx"], res["steps"]
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import PlanOpts

__all__ = [
    "afd_plan_create_nonuniform", "afd_batch_tuning",
    "AFD_FP64_PLAIN", "AFD_FP32_GUARDED", "AfdError", "PlanOpts", "afd_plan_opts_default",
    "afd_status_str", "afd_last_error", "afd_version", "afd_plan_create", "afd_plan_destroy",
    "afd_decompose", "afd_decompose_from", "afd_plan_last_info", "afd_plan_set_profiling", "afd_plan_counters",
    "afd_plan_reset_counters", "afd_plan_get_stream", "afd_plan_kernel_times", "afd_plan_phase_cycles", "afd_batch_create", "afd_batch_run", "afd_batch_counters",
    "afd_batch_destroy", "afd_decompose_batch", "afd_synthesize", "afd_serve_create", "afd_serve_submit",
    "afd_serve_poll", "afd_serve_wait", "afd_serve_suspend", "afd_serve_resume", "afd_serve_get_stats",
    "afd_serve_destroy",
    "afd_inner_products_noalloc", "library_path",
]

AFD_FP64_PLAIN = 0
AFD_FP32_GUARDED = 1
AFD_NOALLOC_MAX_N = 65536       # include/afd.h: limits of afd_inner_products_noalloc
AFD_NOALLOC_MAX_POINTS = 64
STATUS = {0: "AFD_OK", 1: "AFD_PENDING", -1: "AFD_ERR_INVALID", -2: "AFD_ERR_NOMEM",
          -3: "AFD_ERR_CUDA", -4: "AFD_ERR_TIMEOUT", -5: "AFD_ERR_BUDGET", -6: "AFD_ERR_NOT_FOUND",
          -7: "AFD_ERR_NUMERIC"}


class AfdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


def library_path() -> str:
    return _native.LIB_PATH


def _lib():
    return _native.load()


def _check(status: int, partial=None):
    if status != 0 and status != 1:
        err = AfdError(status, _lib().afd_last_error().decode())
        err.partial = partial
        raise err
    return status


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _in_ptr(x, dtype=np.complex128):
    """(pointer, keepalive) of an input array: numpy (host) or torch (host or CUDA)."""
    if _is_torch(x):
        import torch
        want = torch.complex128 if dtype == np.complex128 else torch.float64
        if x.dtype != want:
            raise TypeError(f"expected a {want} tensor, got {x.dtype}")
        x = x.contiguous()
        return x.data_ptr(), x
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    return a.ctypes.data, a


def _opts(opts=None, **kw) -> PlanOpts:
    o = PlanOpts()
    _lib().afd_plan_opts_default(ctypes.byref(o))
    if opts is not None:
        for f, _ in PlanOpts._fields_:
            setattr(o, f, getattr(opts, f))
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(getattr(v, "cuda_stream", v))
        if k in ("force_a1_zero", "use_graph", "renormalise", "autotune"):
            v = int(bool(v))
        if k == "persistent":  # False / True / 2 (a batch as one multi-signal launch)
            v = 2 if (not isinstance(v, bool) and v == 2) else int(bool(v))
        setattr(o, k, v)
    return o


def afd_plan_opts_default() -> PlanOpts:
    return _opts()


def afd_status_str(status: int) -> str:
    return _lib().afd_status_str(int(status)).decode()


def afd_last_error() -> str:
    return _lib().afd_last_error().decode()


def afd_version() -> str:
    return _lib().afd_version().decode()


class Plan:
    """Owning handle of an ``afd_plan``."""

    def __init__(self, handle, N: int, M: int, opts: PlanOpts):
        self.handle, self.N, self.M, self.opts = handle, N, M, opts

    def close(self):
        if self.handle:
            _lib().afd_plan_destroy(self.handle)
            self.handle = None

    __del__ = close


class Batch:
    """Owning handle of an ``afd_batch``."""

    def __init__(self, handle, N, M: int, K_max: int):
        self.handle, self.N, self.M, self.K_max = handle, list(N), M, K_max

    def close(self):
        if self.handle:
            _lib().afd_batch_destroy(self.handle)
            self.handle = None

    __del__ = close


def afd_plan_create(N: int, radii, opts: PlanOpts | None = None, **kw) -> Plan:
    """Plan for N samples and the given ascending radii; keyword options as in afd_plan_opts."""
    r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64))
    o = _opts(opts, **kw)
    h = ctypes.c_void_p()
    _check(_lib().afd_plan_create(ctypes.byref(h), int(N), r.ctypes.data, int(r.size), ctypes.byref(o)))
    return Plan(h, int(N), int(r.size), o)


def afd_plan_create_nonuniform(theta, radii, L: int, weights=None, opts: PlanOpts | None = None, **kw) -> Plan:
    """Plan for samples at exp(i theta_m) (ascending angles in [0, 2 pi)) with
    quadrature weights (None: the trapezoid rule) and a grid of L angles."""
    t = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64))
    w = None if weights is None else np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    o = _opts(opts, **kw)
    h = ctypes.c_void_p()
    _check(_lib().afd_plan_create_nonuniform(ctypes.byref(h), int(t.size), t.ctypes.data,
                                             None if w is None else w.ctypes.data, int(L), r.ctypes.data,
                                             int(r.size), ctypes.byref(o)))
    return Plan(h, int(t.size), int(r.size), o)


def afd_plan_destroy(plan: Plan) -> None:
    plan.close()


def afd_decompose(plan: Plan, G, K_max: int, energy_tol: float = 0.0, out: dict | None = None) -> dict:
    """Decompose one signal.  Returns numpy arrays a, coeff (complex), delta, idx and steps.

    ``out`` may supply caller buffers (numpy or torch, host or CUDA) for keys
    a (2K float64), coeff (2K float64), delta (K+1 float64), idx (2K int32);
    they are then filled in place and returned as given.
    """
    gp, keep = _in_ptr(G)
    K = int(K_max)
    out = out or {}
    bufs = {k: out[k] if k in out else np.zeros(n, dtype=dt)
            for k, n, dt in (("a", 2 * K, np.float64), ("coeff", 2 * K, np.float64),
                             ("delta", K + 1, np.float64), ("idx", 2 * K, np.int32))}
    ptrs = {k: (v.data_ptr() if _is_torch(v) else v.ctypes.data) for k, v in bufs.items()}
    steps = ctypes.c_int(0)
    st = _lib().afd_decompose(plan.handle, gp, K, float(energy_tol), ptrs["a"], ptrs["coeff"],
                              ptrs["delta"], ptrs["idx"], ctypes.byref(steps))
    n = steps.value
    res = {"steps": n}
    if out:
        res.update(bufs)
    else:
        res["a"] = bufs["a"][: 2 * n].view(np.complex128)
        res["coeff"] = bufs["coeff"][: 2 * n].view(np.complex128)
        res["delta"] = bufs["delta"][: n + 1]
        res["idx"] = bufs["idx"][: 2 * n].reshape(n, 2)
    _check(st, res)
    return res


def afd_decompose_from(plan: Plan, G, K_max: int, energy_tol: float = 0.0, E1: float = 0.0) -> dict:
    """Resumable decomposition: start from G (E1 = 0) or from a remainder returned
    earlier (E1 = that run's E_1).  The result dict adds "G_final" (the remainder
    to resume from) and "E1"."""
    gp, keep = _in_ptr(G)
    K = int(K_max)
    n_pts = int(G.numel()) if _is_torch(G) else int(np.asarray(G).size)
    a, c = np.zeros(2 * K), np.zeros(2 * K)
    d, ix = np.zeros(K + 1), np.zeros(2 * K, dtype=np.int32)
    gf = np.zeros(n_pts, dtype=np.complex128)
    steps, e1 = ctypes.c_int(0), ctypes.c_double(0.0)
    st = _lib().afd_decompose_from(plan.handle, gp, float(E1), K, float(energy_tol), a.ctypes.data,
                                   c.ctypes.data, d.ctypes.data, ix.ctypes.data, ctypes.byref(steps),
                                   gf.ctypes.data, ctypes.byref(e1))
    n = steps.value
    res = {"steps": n, "a": a[: 2 * n].view(np.complex128), "coeff": c[: 2 * n].view(np.complex128),
           "delta": d[: n + 1], "idx": ix[: 2 * n].reshape(n, 2), "G_final": gf, "E1": e1.value}
    _check(st, res)
    return res


def afd_plan_last_info(plan: Plan, steps: int) -> dict:
    n_cand = np.zeros(steps, dtype=np.int32)
    flags = np.zeros(steps, dtype=np.int32)
    obj32 = np.zeros(steps)
    _check(_lib().afd_plan_last_info(plan.handle, n_cand.ctypes.data, flags.ctypes.data, obj32.ctypes.data))
    return {"n_cand": n_cand, "flags": flags, "obj32": obj32}


def afd_plan_set_profiling(plan: Plan, on: bool) -> None:
    _check(_lib().afd_plan_set_profiling(plan.handle, int(bool(on))))


def afd_plan_counters(plan: Plan) -> dict:
    kl, gl, ms = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
    _check(_lib().afd_plan_counters(plan.handle, ctypes.byref(kl), ctypes.byref(gl), ctypes.byref(ms)))
    return {"kernel_launches": kl.value, "grid_launches": gl.value, "grid_ms": ms.value}


KERNEL_KINDS = ("grid", "guard", "update", "forward", "persistent")


def afd_plan_kernel_times(plan: Plan) -> dict:
    """Per kernel kind: {"grid": (ms, launches), ...} accumulated while profiling."""
    ms = np.zeros(len(KERNEL_KINDS))
    n = np.zeros(len(KERNEL_KINDS), dtype=np.int64)
    _check(_lib().afd_plan_kernel_times(plan.handle, ms.ctypes.data, n.ctypes.data))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


PHASES = ("transforms", "barrier1", "guard", "barrier2", "update", "barrier3", "energy")


def afd_plan_phase_cycles(plan: Plan) -> dict:
    """Average SM cycles per greedy step of each persistent-kernel phase (profiling on)."""
    v = np.zeros(len(PHASES))
    n = ctypes.c_longlong()
    _check(_lib().afd_plan_phase_cycles(plan.handle, v.ctypes.data, ctypes.byref(n)))
    out = {k: float(v[i]) for i, k in enumerate(PHASES)}
    out["steps"] = n.value
    return out


def afd_plan_get_stream(plan: Plan) -> int:
    """cudaStream_t (as an int) the plan's kernels run on."""
    sp = ctypes.c_void_p()
    _check(_lib().afd_plan_get_stream(plan.handle, ctypes.byref(sp)))
    return int(sp.value or 0)


def afd_plan_reset_counters(plan: Plan) -> None:
    _check(_lib().afd_plan_reset_counters(plan.handle))


def afd_batch_create(N, radii, K_max: int, opts: PlanOpts | None = None, **kw) -> Batch:
    n = np.ascontiguousarray(np.asarray(N, dtype=np.int32))
    r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64))
    o = _opts(opts, **kw)
    h = ctypes.c_void_p()
    _check(_lib().afd_batch_create(ctypes.byref(h), int(n.size), n.ctypes.data, r.ctypes.data,
                                   int(r.size), int(K_max), ctypes.byref(o)))
    return Batch(h, n.tolist(), int(r.size), int(K_max))


def afd_batch_run(batch: Batch, G_packed, energy_tol: float = 0.0) -> dict:
    """Run the batch on packed samples; returns per-signal lists of arrays."""
    gp, keep = _in_ptr(G_packed)
    n, K = len(batch.N), batch.K_max
    a = np.zeros(2 * n * K)
    c = np.zeros(2 * n * K)
    d = np.zeros(n * (K + 1))
    ix = np.zeros(2 * n * K, dtype=np.int32)
    steps = np.zeros(n, dtype=np.int32)
    st = _lib().afd_batch_run(batch.handle, gp, float(energy_tol), a.ctypes.data, c.ctypes.data,
                              d.ctypes.data, ix.ctypes.data, steps.ctypes.data)
    res = {"steps": steps, "a": [], "coeff": [], "delta": [], "idx": []}
    for i in range(n):
        s = int(steps[i])
        res["a"].append(a[2 * i * K: 2 * (i * K + s)].view(np.complex128))
        res["coeff"].append(c[2 * i * K: 2 * (i * K + s)].view(np.complex128))
        res["delta"].append(d[i * (K + 1): i * (K + 1) + s + 1])
        res["idx"].append(ix[2 * i * K: 2 * (i * K + s)].reshape(s, 2))
    _check(st, res)
    return res


def afd_batch_tuning(batch: Batch) -> list:
    """The autotuner's choice per N-class: dicts N, variant, us (time per grid launch)."""
    n = ctypes.c_int(0)
    _check(_lib().afd_batch_tuning(batch.handle, 0, ctypes.byref(n), None, None, None))
    k = n.value
    Ns, vs = np.zeros(k, dtype=np.int32), np.zeros(k, dtype=np.int32)
    us = np.zeros(k, dtype=np.float32)
    _check(_lib().afd_batch_tuning(batch.handle, k, ctypes.byref(n), Ns.ctypes.data, vs.ctypes.data,
                                   us.ctypes.data))
    return [{"N": int(a), "variant": int(b), "us": float(c)} for a, b, c in zip(Ns, vs, us)]


def afd_batch_counters(batch: Batch) -> dict:
    kl = ctypes.c_longlong()
    _check(_lib().afd_batch_counters(batch.handle, ctypes.byref(kl)))
    return {"kernel_launches": kl.value}


def afd_batch_destroy(batch: Batch) -> None:
    batch.close()


def afd_decompose_batch(signals, radii, K_max: int, energy_tol: float = 0.0,
                        opts: PlanOpts | None = None, **kw) -> dict:
    """One-shot batch over a list of sample arrays (numpy complex128)."""
    N = [int(np.asarray(g).size) for g in signals]
    packed = np.concatenate([np.asarray(g, dtype=np.complex128) for g in signals])
    b = afd_batch_create(N, radii, K_max, opts, **kw)
    try:
        return afd_batch_run(b, packed, energy_tol)
    finally:
        b.close()


def afd_synthesize(N: int, a, coeff, all_prefixes: bool = False) -> np.ndarray:
    """S_n (or S_1..S_n as rows) on the N sample points from a_k and coefficients."""
    av = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    cv = np.ascontiguousarray(np.asarray(coeff, dtype=np.complex128))
    n = int(av.size)
    out = np.zeros((n if all_prefixes else 1) * int(N), dtype=np.complex128)
    _check(_lib().afd_synthesize(int(N), av.ctypes.data, cv.ctypes.data, n, int(bool(all_prefixes)),
                                 out.ctypes.data))
    return out.reshape(n, int(N)) if all_prefixes else out


class Server:
    """Owning handle of an ``afd_server``."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            _lib().afd_serve_destroy(self.handle)
            self.handle = None

    __del__ = close


def afd_serve_create(mem_budget_bytes: int, opts: PlanOpts | None = None, **kw) -> Server:
    """Serving engine with a device memory budget (continuous batching)."""
    o = _opts(opts, **kw)
    h = ctypes.c_void_p()
    _check(_lib().afd_serve_create(ctypes.byref(h), int(mem_budget_bytes), ctypes.byref(o)))
    return Server(h)


def afd_serve_submit(server: Server, G, radii, K_max: int, energy_tol: float = 0.0) -> int:
    gp, keep = _in_ptr(G)
    r = np.ascontiguousarray(np.asarray(radii, dtype=np.float64))
    n = int(G.numel()) if _is_torch(G) else int(np.asarray(G).size)
    rid = ctypes.c_uint64()
    _check(_lib().afd_serve_submit(server.handle, n, r.ctypes.data, int(r.size), gp, int(K_max),
                                   float(energy_tol), ctypes.byref(rid)))
    return int(rid.value)


def _result_buffers(K_cap: int):
    a, c = np.zeros(2 * K_cap), np.zeros(2 * K_cap)
    d, ix = np.zeros(K_cap + 1), np.zeros(2 * K_cap, dtype=np.int32)
    res = _native.Result(K_cap, a.ctypes.data, c.ctypes.data, d.ctypes.data, ix.ctypes.data, 0, 0, 0.0)
    return res, (a, c, d, ix)


def _result_dict(res, bufs) -> dict:
    a, c, d, ix = bufs
    n = res.steps
    return {"steps": n, "status": res.status, "latency_ms": res.latency_ms,
            "a": a[: 2 * n].view(np.complex128), "coeff": c[: 2 * n].view(np.complex128),
            "delta": d[: n + 1], "idx": ix[: 2 * n].reshape(n, 2)}


def afd_serve_poll(server: Server, req_id: int, K_cap: int = 4096):
    """None while the request runs; its result dict once finished (then forgotten)."""
    res, bufs = _result_buffers(K_cap)
    st = _lib().afd_serve_poll(server.handle, int(req_id), ctypes.byref(res))
    if st == 1:
        return None
    out = _result_dict(res, bufs)
    _check(st, out)
    return out


def afd_serve_wait(server: Server, req_id: int, timeout_s: float = 60.0, K_cap: int = 4096) -> dict:
    res, bufs = _result_buffers(K_cap)
    st = _lib().afd_serve_wait(server.handle, int(req_id), float(timeout_s), ctypes.byref(res))
    out = _result_dict(res, bufs)
    _check(st, out)
    return out


def afd_serve_suspend(server: Server, req_id: int, timeout_s: float = 60.0) -> None:
    """Move a request out of the device (its state to host memory)."""
    _check(_lib().afd_serve_suspend(server.handle, int(req_id), float(timeout_s)))


def afd_serve_resume(server: Server, req_id: int) -> None:
    """Queue a suspended request again; it continues where it stopped."""
    _check(_lib().afd_serve_resume(server.handle, int(req_id)))


def afd_serve_get_stats(server: Server) -> dict:
    s = _native.ServeStats()
    _check(_lib().afd_serve_get_stats(server.handle, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in _native.ServeStats._fields_}


def afd_serve_destroy(server: Server) -> None:
    server.close()


def afd_inner_products_noalloc(G, points, out=None, stream=None):
    """<G, e_a>~ at each point of ``points`` (torch CUDA complex128 tensors), FP64,
    without any device allocation by the library (its scratch is a static device
    array).  ``out`` (complex128, same device, len(points)) is filled and returned.
    Asynchronous on ``stream`` (a torch stream or cudaStream_t int; default: the
    legacy default stream)."""
    import torch
    if out is None and isinstance(points, torch.Tensor):
        out = torch.empty_like(points)
    for name, t in (("G", G), ("points", points), ("out", out)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype != torch.complex128:
            raise ValueError(f"{name} must be complex128, not {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.device.type != "cuda":
            raise ValueError(f"{name} must be on a CUDA device, not {t.device}")
    if not (G.device == points.device == out.device):
        raise ValueError("G, points and out must be on the same CUDA device")
    if not 1 <= G.numel() <= AFD_NOALLOC_MAX_N:
        raise ValueError(f"len(G) must be in 1..{AFD_NOALLOC_MAX_N}")
    if not 1 <= points.numel() <= AFD_NOALLOC_MAX_POINTS:
        raise ValueError(f"len(points) must be in 1..{AFD_NOALLOC_MAX_POINTS}")
    if out.numel() != points.numel():
        raise ValueError("out must have one entry per point")
    s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(_lib().afd_inner_products_noalloc(G.data_ptr(), int(G.numel()), points.data_ptr(),
                                             int(points.numel()), out.data_ptr(), s or None))
    return out


def afd_selftest_wait_timeout(kind: int, device: int = -1) -> tuple[int, float]:
    """Make one bounded wait run out on purpose (kind 0: the persistent
    kernel's grid barrier; kind 1: the mbarrier wait of the TMA-staged
    passes).  Returns (status the kernel reported, seconds the wait polled);
    the expected status is AFD_ERR_TIMEOUT."""
    st, sec = ctypes.c_int(), ctypes.c_double()
    _check(_lib().afd_selftest_wait_timeout(int(device), int(kind), ctypes.byref(st), ctypes.byref(sec)))
    return st.value, sec.value
