"""Python binding of libipc_b300.so (argument marshalling only).

Every step of the solver runs in the library's CUDA kernels; this module
converts numpy / torch arrays to pointers and calls the C ABI declared in
include/ipc.h.  PyTorch provides device memory (through the caching
allocator, passed to the library as ipc_alloc_fns) and the CUDA stream.
The library must be built (``paper_2604_19892_b300.build.build()``); if it is
missing, loading fails with an error instead of falling back to anything.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libipc_b300.so")

IPC_OK = 0
IPC_NOT_CONVERGED = 1
IPC_PENDING = 2
IPC_ERR_INVALID = -1
IPC_ERR_INTERSECTING = -2
IPC_ERR_OOM = -3
IPC_ERR_NUMERIC = -4
IPC_ERR_TIMEOUT = -5
IPC_ERR_CUDA = -6
IPC_ERR_CAPACITY = -7
IPC_PREC_FP64 = 0
IPC_PREC_FP32 = 1
IPC_PREC_BF16_MAS = 2

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


class SceneDesc(C.Structure):
    _fields_ = [("n_verts", C.c_int), ("x_rest", _D), ("x0", _D), ("v0", _D), ("n_tets", C.c_int),
                ("tets", C.POINTER(C.c_int32)), ("E", _D), ("nu", _D), ("rho", _D),
                ("gravity", C.c_double * 3), ("has_ground", C.c_int), ("ground_normal", C.c_double * 3),
                ("ground_offset", C.c_double)]


class Params(C.Structure):
    _fields_ = [("h", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double), ("tol", C.c_double),
                ("delta", C.c_double), ("eps_rot_deg", C.c_double), ("ccd_shrink", C.c_double),
                ("eps_sing", C.c_double), ("eps_abs", C.c_double), ("K", C.c_int), ("iter_max", C.c_int),
                ("levels_max", C.c_int), ("ls_max", C.c_int), ("precision", C.c_int),
                ("contact_capacity", C.c_int), ("broad_phase", C.c_int), ("mas_mode", C.c_int),
                ("ccd_mode", C.c_int), ("graphs", C.c_int), ("fp32_pivot_floor", C.c_double),
                ("grid_pair_capacity", C.c_int), ("wait_polls", C.c_int), ("apply_ctas", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class ServerCfg(C.Structure):
    _fields_ = [("slots", C.c_int), ("min_free_bytes", C.c_size_t)]


class AllocFns(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class StepStats(C.Structure):
    _fields_ = [("steps", C.c_int), ("iters", C.c_int), ("restarts", C.c_int), ("ls_halvings", C.c_int),
                ("ls_failures", C.c_int), ("converged", C.c_int), ("n_contacts", C.c_int),
                ("ccd_fallbacks", C.c_int), ("energy", C.c_double), ("min_dist", C.c_double),
                ("znorm", C.c_double)]


class IterRecord(C.Structure):
    _fields_ = [("restart", C.c_int), ("n_contacts", C.c_int), ("n_update", C.c_int), ("ls_halvings", C.c_int),
                ("mu", C.c_double), ("nu", C.c_double), ("gz", C.c_double), ("znorm", C.c_double),
                ("energy_before", C.c_double), ("energy_after", C.c_double), ("alpha_min", C.c_double),
                ("alpha_max", C.c_double), ("r", C.c_double), ("pmax", C.c_double), ("ccd_passes", C.c_int),
                ("cached_pairs", C.c_int), ("ccd_passes_body", C.c_int), ("pad_", C.c_int)]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("launches", C.c_longlong * 8)]


STAGES = ["restart", "classify", "mas_blocks", "forms", "direction", "ccd", "trial_eval", "other"]

Q_POSITIONS, Q_VELOCITIES, Q_N_VERTS, Q_N_CONTACTS, Q_SUBDOMAIN_ALPHA, Q_N_SUBDOMAINS, Q_TRACE_LEN, Q_TRACE, \
    Q_SURFACE_COUNTS, Q_LEVEL_MAP, Q_BBOX_DIAG, Q_N_BODIES, Q_FP64_BLOCKS, Q_PIVOT_FIXES, Q_APPLY_CTAS = range(15)

_lib = None

EXPORTS = {
    "ipc_default_params": (None, [C.POINTER(Params)]),
    "ipc_scene_create": (C.c_int, [C.POINTER(SceneDesc), C.POINTER(Params), C.POINTER(AllocFns), C.POINTER(C.c_void_p)]),
    "ipc_scene_destroy": (None, [C.c_void_p]),
    "ipc_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(StepStats)]),
    "ipc_set_state": (C.c_int, [C.c_void_p, _D, _D, C.c_int, C.c_void_p]),
    "ipc_query": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "ipc_query_level": (C.c_int, [C.c_void_p, C.c_int, _I, _I, _I, _I]),
    "ipc_query_surface": (C.c_int, [C.c_void_p, _I, _I, _I]),
    "ipc_eval_energy_grad": (C.c_int, [C.c_void_p, _D, _D, _D, _D, C.c_void_p]),
    "ipc_eval_contacts": (C.c_int, [C.c_void_p, _D, C.c_int, _I, _I, _I, _I, _D, _D, _D, C.c_void_p]),
    "ipc_eval_precond": (C.c_int, [C.c_void_p, _D, _D, _D, _D, C.c_void_p]),
    "ipc_eval_forms": (C.c_int, [C.c_void_p, _D, _D, _D, _D, _D, C.c_void_p]),
    "ipc_eval_ccd": (C.c_int, [C.c_void_p, _D, _D, _D, _I, _D, _I, C.c_void_p]),
    "ipc_precond_apply_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ipc_profile_replay": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p,
                                     C.POINTER(C.c_double)]),
    "ipc_last_error": (C.c_char_p, []),
    "ipc_server_create": (C.c_int, [C.POINTER(ServerCfg), C.POINTER(AllocFns), C.POINTER(C.c_void_p)]),
    "ipc_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_ulonglong)]),
    "ipc_server_poll": (C.c_int, [C.c_void_p, C.c_ulonglong, C.POINTER(StepStats), C.POINTER(C.c_double)]),
    "ipc_server_wait": (C.c_int, [C.c_void_p, C.c_ulonglong, C.c_double, C.POINTER(StepStats),
                                  C.POINTER(C.c_double)]),
    "ipc_server_destroy": (None, [C.c_void_p]),
    "ipc_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "ipc_profile_read": (C.c_int, [C.c_void_p, C.POINTER(Profile)]),
    "ipc_kernel_launches": (C.c_longlong, []),
    "ipc_profile_fma_peak": (C.c_int, [C.c_int, C.c_double, C.POINTER(C.c_double)]),
}


def fma_peak_tflops(precision: int = IPC_PREC_FP32, target_ms: float = 20.0) -> float:
    """Measured FMA throughput of the SIMT pipes (ipc_profile_fma_peak)."""
    out = C.c_double()
    _check(load().ipc_profile_fma_peak(int(precision), float(target_ms), C.byref(out)))
    return out.value


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load().ipc_kernel_launches())


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2604_19892_b300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class IPCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ipc error {code}: {msg}")
        self.code = code


def _check(code):
    if code < 0:
        raise IPCError(code, load().ipc_last_error().decode())
    return code


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(n, ctx):
            try:
                return self.torch.cuda.caching_allocator_alloc(int(n), device=self.device)
            except Exception:
                return None

        def _free(p, ctx):
            self.torch.cuda.caching_allocator_delete(p)

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.fns = AllocFns(self._a, self._f, None)


def default_params(sc_params: dict, precision: int = IPC_PREC_FP64) -> Params:
    lib = load()
    p = Params()
    lib.ipc_default_params(C.byref(p))
    for k in ("h", "dhat", "kappa", "tol", "delta", "eps_rot_deg", "ccd_shrink", "eps_sing", "eps_abs", "K",
              "iter_max", "levels_max", "ls_max", "broad_phase", "mas_mode", "ccd_mode", "graphs",
              "fp32_pivot_floor", "grid_pair_capacity", "wait_polls", "apply_ctas"):
        if k in sc_params:
            setattr(p, k, type(getattr(p, k))(sc_params[k]))
    p.precision = precision
    if "contact_capacity" in sc_params:
        p.contact_capacity = int(sc_params["contact_capacity"])
    return p


class Scene:
    """One resident scene on the current CUDA device."""

    def __init__(self, sc: dict, params: dict | None = None, precision: int = IPC_PREC_FP64,
                 use_torch_allocator: bool = True, stream=None, alloc_fns: "AllocFns | None" = None):
        lib = load()
        self.lib = lib
        p = dict(sc["params"])
        if params:
            p.update(params)
        self.params = p
        self.nv = int(sc["x_rest"].shape[0])
        self.precision = precision
        keep = []

        def ptr(a, dt=np.float64):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data_as(C.POINTER(C.c_int32) if dt == np.int32 else _D)

        d = SceneDesc()
        d.n_verts = self.nv
        d.x_rest = ptr(sc["x_rest"])
        d.x0 = ptr(sc["x0"])
        d.v0 = ptr(sc["v0"])
        d.n_tets = int(sc["tets"].shape[0])
        d.tets = ptr(sc["tets"], np.int32)
        d.E = ptr(sc["E"])
        d.nu = ptr(sc["nu"])
        d.rho = ptr(sc["rho"])
        for i in range(3):
            d.gravity[i] = float(sc["gravity"][i])
        g = sc["ground"]
        d.has_ground = 0 if np.isnan(g[3]) else 1
        for i in range(3):
            d.ground_normal[i] = float(g[i]) if d.has_ground else 0.0
        d.ground_offset = float(g[3]) if d.has_ground else 0.0
        self._prm = default_params(p, precision)
        self._alloc = None
        fns = None
        if alloc_fns is not None:  # the caller's device allocator (kept alive with the scene)
            self._alloc = alloc_fns
            fns = C.byref(alloc_fns)
        elif use_torch_allocator:
            import torch
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            fns = C.byref(self._alloc.fns)
        h = C.c_void_p()
        _check(lib.ipc_scene_create(C.byref(d), C.byref(self._prm), fns, C.byref(h)))
        self.h = h
        self.stream = stream

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.ipc_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stepping ------------------------------------------------------------
    def step(self, n: int = 1, stream=None) -> dict:
        st = StepStats()
        code = _check(self.lib.ipc_step(self.h, int(n), _stream_handle(stream or self.stream), C.byref(st)))
        out = {f: getattr(st, f) for f, _ in StepStats._fields_}
        out["status"] = code
        return out

    def set_state(self, x, v=None, stream=None):
        import torch
        if isinstance(x, torch.Tensor) and x.is_cuda:
            xp = C.cast(C.c_void_p(x.data_ptr()), _D)
            vp = C.cast(C.c_void_p(v.data_ptr()), _D) if v is not None else None
            _check(self.lib.ipc_set_state(self.h, xp, vp, 1, _stream_handle(stream or self.stream)))
            return
        x = _f64(x)
        v = _f64(v) if v is not None else None
        _check(self.lib.ipc_set_state(self.h, _dp(x), _dp(v) if v is not None else None, 0,
                                      _stream_handle(stream or self.stream)))

    def _query_array(self, kind, n, dtype=np.float64):
        out = np.zeros(n, dtype=dtype)
        _check(self.lib.ipc_query(self.h, kind, out.ctypes.data_as(C.c_void_p), out.nbytes,
                                  _stream_handle(self.stream)))
        return out

    def positions(self):
        return self._query_array(Q_POSITIONS, 3 * self.nv).reshape(-1, 3)

    def velocities(self):
        return self._query_array(Q_VELOCITIES, 3 * self.nv).reshape(-1, 3)

    def n_subdomains(self):
        return int(self._query_array(Q_N_SUBDOMAINS, 1, np.int32)[0])

    def subdomain_alpha(self):
        return self._query_array(Q_SUBDOMAIN_ALPHA, self.n_subdomains())

    def bbox_diag(self):
        return float(self._query_array(Q_BBOX_DIAG, 1)[0])

    def fp64_blocks(self):
        """Subdomain blocks the last restart inverted in FP64 (FP32 bulk: the
        blocks whose FP32 factorisation would floor or raise a pivot)."""
        return int(self._query_array(Q_FP64_BLOCKS, 1, np.int32)[0])

    def apply_ctas(self):
        """CTAs per SM of the persistent block apply chosen by the library's
        autotuner at scene creation."""
        return int(self._query_array(Q_APPLY_CTAS, 1, np.int32)[0])

    def pivot_fixes(self):
        """Blocks of the last restart whose final (FP64) factorisation
        floored or raised a pivot (0: plain Cholesky inverses throughout)."""
        return int(self._query_array(Q_PIVOT_FIXES, 1, np.int32)[0])

    def trace(self):
        n = int(self._query_array(Q_TRACE_LEN, 1, np.int32)[0])
        rec = (IterRecord * max(n, 1))()
        _check(self.lib.ipc_query(self.h, Q_TRACE, C.cast(rec, C.c_void_p), C.sizeof(IterRecord) * n,
                                  _stream_handle(self.stream)))
        return [{f: getattr(rec[i], f) for f, _ in IterRecord._fields_} for i in range(n)]

    def surface(self):
        c = self._query_array(Q_SURFACE_COUNTS, 3, np.int32)
        sv = np.zeros(c[0], np.int32)
        sf = np.zeros((c[1], 3), np.int32)
        se = np.zeros((c[2], 2), np.int32)
        _check(self.lib.ipc_query_surface(self.h, sv.ctypes.data_as(_I), sf.ctypes.data_as(_I),
                                          se.ctypes.data_as(_I)))
        return sv, sf, se

    def levels(self):
        nl = _check(self.lib.ipc_query_level(self.h, 0, None, None, None, None))
        out = []
        for l in range(nl):
            n = C.c_int()
            g = C.c_int()
            self.lib.ipc_query_level(self.h, l, C.byref(n), C.byref(g), None, None)
            grp = np.zeros(n.value, np.int32)
            slot = np.zeros(n.value, np.int32)
            _check(self.lib.ipc_query_level(self.h, l, None, None, grp.ctypes.data_as(_I), slot.ctypes.data_as(_I)))
            out.append((grp, slot))
        return out

    def profile(self, enable: bool):
        _check(self.lib.ipc_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self) -> dict:
        p = Profile()
        _check(self.lib.ipc_profile_read(self.h, C.byref(p)))
        return {name: {"ms": p.ms[i], "launches": int(p.launches[i])} for i, name in enumerate(STAGES)}

    # -- evaluation entry points -----------------------------------------------
    def energy_grad(self, x, xt, grad=True):
        x, xt = _f64(x), _f64(xt)
        E = C.c_double()
        g = np.zeros((self.nv, 3)) if grad else None
        _check(self.lib.ipc_eval_energy_grad(self.h, _dp(x), _dp(xt), C.byref(E), _dp(g) if grad else None,
                                             _stream_handle(self.stream)))
        return (E.value, g) if grad else E.value

    def contacts(self, x):
        x = _f64(x)
        n = C.c_int()
        _check(self.lib.ipc_eval_contacts(self.h, _dp(x), 0, C.byref(n), None, None, None, None, None, None,
                                          _stream_handle(self.stream)))
        m = n.value
        typ = np.zeros(m, np.int32)
        ids = np.zeros((m, 2), np.int32)
        verts = np.zeros((m, 4), np.int32)
        dist = np.zeros(m)
        k = np.zeros(m)
        grad = np.zeros((m, 12))
        _check(self.lib.ipc_eval_contacts(self.h, _dp(x), m, C.byref(n), typ.ctypes.data_as(_I),
                                          ids.ctypes.data_as(_I), verts.ctypes.data_as(_I), _dp(dist), _dp(k),
                                          _dp(grad), _stream_handle(self.stream)))
        return {"type": typ, "ids": ids, "verts": verts, "dist": dist, "k": k, "grad": grad}

    def precond_apply(self, x_base, g, x_curr=None):
        xb, g = _f64(x_base), _f64(g)
        xc = _f64(x_curr) if x_curr is not None else None
        z = np.zeros((self.nv, 3))
        _check(self.lib.ipc_eval_precond(self.h, _dp(xb), _dp(xc) if xc is not None else None, _dp(g), _dp(z),
                                         _stream_handle(self.stream)))
        return z

    def profile_replay(self, stage: int, reps: int, flush=None, stream=None) -> float:
        """Mean device ms of one stage's kernels replayed on the current state
        (2 = MAS block apply, 3 = H~ quadratic forms); `flush` is a CUDA
        tensor overwritten before each replay to evict L2."""
        ms = C.c_double()
        fp = C.c_void_p(flush.data_ptr()) if flush is not None else None
        fb = flush.numel() * flush.element_size() if flush is not None else 0
        _check(self.lib.ipc_profile_replay(self.h, int(stage), int(reps), fp, fb, _stream_handle(stream or self.stream),
                                           C.byref(ms)))
        return ms.value

    def precond_apply_noalloc(self, g_dev, z_dev, stream=None):
        """z = P_base g on device tensors of shape (nv, 3) in the scene's bulk
        precision, through the allocation-free entry point; returns once z is
        complete (the call waits for the stream)."""
        import torch
        want = torch.float64 if self.precision == IPC_PREC_FP64 else torch.float32  # BF16_MAS: FP32 vectors
        for t in (g_dev, z_dev):
            if not (t.is_cuda and t.dtype == want and t.is_contiguous() and t.numel() == 3 * self.nv):
                raise ValueError(f"expected a contiguous CUDA {want} tensor of {3 * self.nv} values")
        _check(self.lib.ipc_precond_apply_noalloc(self.h, C.c_void_p(g_dev.data_ptr()), C.c_void_p(z_dev.data_ptr()),
                                                  _stream_handle(stream or self.stream)))

    def hess_forms(self, x_base, z, p, x_curr=None):
        xb, z, p = _f64(x_base), _f64(z), _f64(p)
        xc = _f64(x_curr) if x_curr is not None else None
        out = np.zeros(3)
        _check(self.lib.ipc_eval_forms(self.h, _dp(xb), _dp(xc) if xc is not None else None, _dp(z), _dp(p),
                                       _dp(out), _stream_handle(self.stream)))
        return out

    def n_bodies(self):
        return int(self._query_array(Q_N_BODIES, 1, np.int32)[0])

    def ccd(self, x, p, per_body=False):
        x, p = _f64(x), _f64(p)
        a = np.zeros(self.n_subdomains())
        passes = C.c_int()
        if not per_body:
            _check(self.lib.ipc_eval_ccd(self.h, _dp(x), _dp(p), _dp(a), C.byref(passes), None, None,
                                         _stream_handle(self.stream)))
            return a, passes.value
        ab = np.zeros(self.n_bodies())
        pb = C.c_int()
        _check(self.lib.ipc_eval_ccd(self.h, _dp(x), _dp(p), _dp(a), C.byref(passes), _dp(ab), C.byref(pb),
                                     _stream_handle(self.stream)))
        return a, passes.value, ab, pb.value


class Server:
    """Continuous batching of step requests over resident scenes
    (ipc_server_*): up to `slots` requests run at once, each on its own
    stream and host thread of the library. Scenes given to it should use the
    library's own allocator (Scene(..., use_torch_allocator=False)): their
    steps then run on the server's threads without calling back into Python.
    """

    def __init__(self, slots: int = 4, min_free_bytes: int = 0):
        self.lib = load()
        cfg = ServerCfg(int(slots), int(min_free_bytes))
        h = C.c_void_p()
        _check(self.lib.ipc_server_create(C.byref(cfg), None, C.byref(h)))
        self.h = h

    def submit(self, scene: "Scene", n: int = 1) -> int:
        t = C.c_ulonglong()
        _check(self.lib.ipc_server_submit(self.h, scene.h, int(n), C.byref(t)))
        return int(t.value)

    def _result(self, code, st, lat):
        if code == IPC_PENDING:
            return None
        _check(code)
        out = {f: getattr(st, f) for f, _ in StepStats._fields_}
        out["status"] = code
        out["latency_ms"] = lat.value
        return out

    def poll(self, ticket: int):
        """None while pending, else the step statistics and latency_ms."""
        st, lat = StepStats(), C.c_double()
        return self._result(self.lib.ipc_server_poll(self.h, C.c_ulonglong(ticket), C.byref(st), C.byref(lat)), st,
                            lat)

    def wait(self, ticket: int, timeout_s: float = 600.0):
        st, lat = StepStats(), C.c_double()
        code = self.lib.ipc_server_wait(self.h, C.c_ulonglong(ticket), float(timeout_s) * 1e3, C.byref(st),
                                        C.byref(lat))
        r = self._result(code, st, lat)
        if r is None:
            raise TimeoutError(f"request {ticket} still pending after {timeout_s} s")
        return r

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.ipc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
