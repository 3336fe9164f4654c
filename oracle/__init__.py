"""FP64 CPU oracle of MAS-PNCG (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference legs import this package.  The product path (the CUDA library and
its binding) never does.  The C sources next to this file restate the method
of the paper in plain FP64 C; this module compiles them with gcc and exposes
them through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ["o_mesh.c", "o_elastic.c", "o_contact.c", "o_broad.c", "o_mas.c", "o_ccd.c", "o_pncg.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, -O2, no fast-math)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    hdrs = [os.path.join(_HERE, h) for h in ("oracle.h", "o_internal.h")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(f) <= t for f in srcs + hdrs):
            return _LIB_PATH
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-Wall", "-Wno-unused-function",
           "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-o", _LIB_PATH + ".tmp"] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class OParams(C.Structure):
    _fields_ = [("h", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double), ("tol", C.c_double),
                ("delta", C.c_double), ("eps_rot_deg", C.c_double), ("ccd_shrink", C.c_double),
                ("eps_sing", C.c_double), ("eps_abs", C.c_double), ("K", C.c_int), ("iter_max", C.c_int),
                ("levels_max", C.c_int), ("ls_max", C.c_int), ("subdomain", C.c_int),
                ("brute_force", C.c_int)]


class OStepStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("ls_halvings", C.c_int),
                ("ls_failures", C.c_int), ("converged", C.c_int), ("n_contacts", C.c_int),
                ("energy", C.c_double), ("min_dist", C.c_double), ("znorm", C.c_double)]


class OIterRecord(C.Structure):
    _fields_ = [("restart", C.c_int), ("n_contacts", C.c_int), ("n_update", C.c_int),
                ("ls_halvings", C.c_int), ("mu", C.c_double), ("nu", C.c_double), ("gz", C.c_double),
                ("znorm", C.c_double), ("energy_before", C.c_double), ("energy_after", C.c_double),
                ("alpha_min", C.c_double), ("alpha_max", C.c_double), ("r", C.c_double),
                ("ccd_passes", C.c_int), ("ccd_passes_body", C.c_int)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def _lib_handle():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB_PATH)
        sig = {
            "o_scene_create": (C.c_void_p, [C.c_int, _D, C.c_int, _I, _D, _D, _D, _D, _D, C.POINTER(OParams)]),
            "o_scene_destroy": (None, [C.c_void_p]),
            "o_last_error": (C.c_char_p, []),
            "o_surface_counts": (None, [C.c_void_p, _I]),
            "o_surface_get": (None, [C.c_void_p, _I, _I, _I]),
            "o_mass_get": (None, [C.c_void_p, _D]),
            "o_bbox_diag": (C.c_double, [C.c_void_p]),
            "o_levels": (C.c_int, [C.c_void_p]),
            "o_level_info": (None, [C.c_void_p, C.c_int, _I, _I]),
            "o_level_map": (None, [C.c_void_p, C.c_int, _I, _I]),
            "o_barrier": (None, [C.c_double, C.c_double, _D]),
            "o_pt_distance": (C.c_double, [_D, _D, _D, _D, _D]),
            "o_ee_distance": (C.c_double, [_D, _D, _D, _D, _D]),
            "o_snh_tet": (None, [_D, C.c_double, C.c_double, C.c_double, _D, _D, _D, _D, C.c_int]),
            "o_snh_psi": (C.c_double, [_D, C.c_double, C.c_double]),
            "o_snh_dPdF": (None, [_D, C.c_double, C.c_double, _D]),
            "o_psd_project": (None, [C.c_int, _D]),
            "o_energy": (C.c_double, [C.c_void_p, _D, _D]),
            "o_gradient": (None, [C.c_void_p, _D, _D, _D]),
            "o_contacts": (C.c_int, [C.c_void_p, _D, C.c_int, _I, _I, _I, _D, _D, _D]),
            "o_hessian_apply": (None, [C.c_void_p, _D, _D, _D]),
            "o_precond_apply": (None, [C.c_void_p, _D, _D, _D, _D]),
            "o_hess_forms": (None, [C.c_void_p, _D, _D, _D, _D, _D]),
            "o_cubic_safe": (C.c_double, [_D, C.c_double]),
            "o_pair_safe": (C.c_double, [C.c_int, _D, _D, C.c_double, C.c_double]),
            "o_safe_bisect": (C.c_double, [_D, C.c_double, C.c_double, C.c_double, C.c_double]),
            "o_pt_cubic": (None, [_D, _D, _D]),
            "o_ee_cubic": (None, [_D, _D, _D]),
            "o_ltight_pt": (C.c_double, [_D]),
            "o_ltight_ee": (C.c_double, [_D]),
            "o_loriginal_pt": (C.c_double, [_D]),
            "o_ccd": (C.c_int, [C.c_void_p, _D, _D, _D, _D, _I]),
            "o_bodies": (C.c_int, [C.c_void_p, _I]),
            "o_solve2x2": (None, [C.c_double] * 7 + [_D, _D]),
            "o_step": (C.c_int, [C.c_void_p, _D, _D, C.POINTER(OStepStats)]),
            "o_trace": (C.c_int, [C.c_void_p, C.POINTER(OIterRecord), C.c_int]),
            "o_updates": (C.c_int, [C.c_void_p, C.c_int, _D, _I, _D]),
            "o_topk": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _I]),
            "o_chol_inverse": (C.c_int, [C.c_int, _D, _D]),
            "o_chol_floors": (C.c_longlong, [C.c_int]),
            "o_energy_tolerance": (C.c_double, [C.c_void_p, C.c_double]),
            "o_set_threads": (C.c_int, [C.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_I)


def make_params(p: dict, subdomain: int = 32) -> OParams:
    return OParams(h=p["h"], dhat=p["dhat"], kappa=p["kappa"], tol=p["tol"], delta=p["delta"],
                   eps_rot_deg=p["eps_rot_deg"], ccd_shrink=p["ccd_shrink"], eps_sing=p["eps_sing"],
                   eps_abs=p["eps_abs"], K=p["K"], iter_max=p["iter_max"], levels_max=p["levels_max"],
                   ls_max=p["ls_max"], subdomain=subdomain, brute_force=int(p.get("brute_force", 0)))


class Scene:
    """One oracle scene built from a scene dict of paper_2604_19892_b300.scenes."""

    def __init__(self, sc: dict, params: dict | None = None, subdomain: int = 32):
        lib = _lib_handle()
        self.lib = lib
        p = dict(sc["params"])
        if params:
            p.update(params)
        self.params = p
        self.nv = sc["x_rest"].shape[0]
        self._keep = []
        xr, xr_p = _d(sc["x_rest"])
        tt, tt_p = _i(sc["tets"])
        E, E_p = _d(sc["E"])
        nu, nu_p = _d(sc["nu"])
        rho, rho_p = _d(sc["rho"])
        g, g_p = _d(sc["gravity"])
        gr, gr_p = _d(sc["ground"])
        self._prm = make_params(p, subdomain)
        h = lib.o_scene_create(self.nv, xr_p, tt.shape[0], tt_p, E_p, nu_p, rho_p, g_p, gr_p, C.byref(self._prm))
        if not h:
            raise RuntimeError("oracle scene: " + lib.o_last_error().decode())
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.o_scene_destroy(self.h)
            self.h = None

    # --- topology ---------------------------------------------------------
    def surface(self):
        c = (C.c_int * 3)()
        self.lib.o_surface_counts(self.h, c)
        sv = np.zeros(c[0], np.int32)
        sf = np.zeros((c[1], 3), np.int32)
        se = np.zeros((c[2], 2), np.int32)
        self.lib.o_surface_get(self.h, sv.ctypes.data_as(_I), sf.ctypes.data_as(_I), se.ctypes.data_as(_I))
        return sv, sf, se

    def mass(self):
        m = np.zeros(self.nv)
        self.lib.o_mass_get(self.h, m.ctypes.data_as(_D))
        return m

    def bbox_diag(self):
        return self.lib.o_bbox_diag(self.h)

    def levels(self):
        out = []
        for l in range(self.lib.o_levels(self.h)):
            n = C.c_int()
            g = C.c_int()
            self.lib.o_level_info(self.h, l, C.byref(n), C.byref(g))
            grp = np.zeros(n.value, np.int32)
            slot = np.zeros(n.value, np.int32)
            self.lib.o_level_map(self.h, l, grp.ctypes.data_as(_I), slot.ctypes.data_as(_I))
            out.append((grp, slot))
        return out

    # --- evaluations ------------------------------------------------------
    def energy(self, x, xt):
        x, xp = _d(x)
        xt, xtp = _d(xt)
        return self.lib.o_energy(self.h, xp, xtp)

    def gradient(self, x, xt):
        x, xp = _d(x)
        xt, xtp = _d(xt)
        g = np.zeros((self.nv, 3))
        self.lib.o_gradient(self.h, xp, xtp, g.ctypes.data_as(_D))
        return g

    def contacts(self, x, cap=None):
        x, xp = _d(x)
        n = self.lib.o_contacts(self.h, xp, 0, None, None, None, None, None, None)
        cap = n
        typ = np.zeros(cap, np.int32)
        verts = np.zeros((cap, 4), np.int32)
        ids = np.zeros((cap, 2), np.int32)
        dist = np.zeros(cap)
        k = np.zeros(cap)
        grad = np.zeros((cap, 12))
        self.lib.o_contacts(self.h, xp, cap, typ.ctypes.data_as(_I), verts.ctypes.data_as(_I),
                            ids.ctypes.data_as(_I), dist.ctypes.data_as(_D), k.ctypes.data_as(_D),
                            grad.ctypes.data_as(_D))
        return {"type": typ, "verts": verts, "ids": ids, "dist": dist, "k": k, "grad": grad}

    def hessian_apply(self, x, v):
        x, xp = _d(x)
        v, vp = _d(v)
        out = np.zeros((self.nv, 3))
        self.lib.o_hessian_apply(self.h, xp, vp, out.ctypes.data_as(_D))
        return out

    def precond_apply(self, x_base, g, x_curr=None):
        xb, xbp = _d(x_base)
        g, gp = _d(g)
        if x_curr is None:
            xcp = None
        else:
            xc, xcp = _d(x_curr)
        z = np.zeros((self.nv, 3))
        self.lib.o_precond_apply(self.h, xbp, xcp, gp, z.ctypes.data_as(_D))
        return z

    def hess_forms(self, x_base, z, p, x_curr=None):
        xb, xbp = _d(x_base)
        z, zp = _d(z)
        p, pp = _d(p)
        if x_curr is None:
            xcp = None
        else:
            xc, xcp = _d(x_curr)
        out = np.zeros(3)
        self.lib.o_hess_forms(self.h, xbp, xcp, zp, pp, out.ctypes.data_as(_D))
        return out

    def bodies(self):
        b = np.zeros(self.nv, np.int32)
        n = self.lib.o_bodies(self.h, b.ctypes.data_as(_I))
        return n, b

    def ccd(self, x, p, per_body=False):
        x, xp = _d(x)
        p, pp = _d(p)
        n = C.c_int()
        g = C.c_int()
        self.lib.o_level_info(self.h, 0, C.byref(n), C.byref(g))
        a = np.zeros(g.value)
        if not per_body:
            passes = self.lib.o_ccd(self.h, xp, pp, a.ctypes.data_as(_D), None, None)
            return a, passes
        nb, _ = self.bodies()
        ab = np.zeros(nb)
        pb = C.c_int()
        passes = self.lib.o_ccd(self.h, xp, pp, a.ctypes.data_as(_D), ab.ctypes.data_as(_D), C.byref(pb))
        return a, passes, ab, pb.value

    def step(self, x, v):
        x = np.array(x, dtype=np.float64, copy=True)
        v = np.array(v, dtype=np.float64, copy=True)
        st = OStepStats()
        self.lib.o_step(self.h, x.ctypes.data_as(_D), v.ctypes.data_as(_D), C.byref(st))
        stats = {f: getattr(st, f) for f, _ in OStepStats._fields_}
        return x, v, stats

    def updates(self):
        """Classified updates of the last precond_apply / hess_forms with
        x_curr: dS, key (type, ida, idb) and u (12 values) of each."""
        n = self.lib.o_updates(self.h, 0, None, None, None)
        dS = np.zeros(n)
        key = np.zeros((n, 3), np.int32)
        u = np.zeros((n, 12))
        self.lib.o_updates(self.h, n, dS.ctypes.data_as(_D), key.ctypes.data_as(_I), u.ctypes.data_as(_D))
        return {"dS": dS, "key": key, "u": u}

    def topk(self, group):
        idx = np.zeros(64, np.int32)
        n = self.lib.o_topk(self.h, int(group), 64, idx.ctypes.data_as(_I))
        return idx[:min(n, 64)].copy()

    def energy_tolerance(self, E):
        return self.lib.o_energy_tolerance(self.h, float(E))

    def trace(self):
        n = self.lib.o_trace(self.h, None, 0)
        rec = (OIterRecord * max(n, 1))()
        self.lib.o_trace(self.h, rec, n)
        return [{f: getattr(rec[i], f) for f, _ in OIterRecord._fields_} for i in range(n)]


# --- stateless helpers ------------------------------------------------------

def barrier(d, dhat):
    out = (C.c_double * 3)()
    _lib_handle().o_barrier(d, dhat, out)
    return tuple(out)


def pt_distance(p, t0, t1, t2):
    w = (C.c_double * 3)()
    args = [_d(a)[0] for a in (p, t0, t1, t2)]
    d = _lib_handle().o_pt_distance(*[a.ctypes.data_as(_D) for a in args], w)
    return d, np.array(w)


def ee_distance(a0, a1, b0, b1):
    st = (C.c_double * 2)()
    args = [_d(a)[0] for a in (a0, a1, b0, b1)]
    d = _lib_handle().o_ee_distance(*[a.ctypes.data_as(_D) for a in args], st)
    return d, np.array(st)


def snh_tet(Dm_inv, vol, mu, lam, x12, project=True):
    B, Bp = _d(np.asarray(Dm_inv).reshape(9))
    x, xp = _d(np.asarray(x12).reshape(12))
    e = C.c_double()
    g = np.zeros(12)
    H = np.zeros((12, 12))
    _lib_handle().o_snh_tet(Bp, vol, mu, lam, xp, C.byref(e), g.ctypes.data_as(_D), H.ctypes.data_as(_D),
                            1 if project else 0)
    return e.value, g, H


def snh_psi(F, mu, lam):
    F, Fp = _d(np.asarray(F).reshape(9))
    return _lib_handle().o_snh_psi(Fp, mu, lam)


def snh_dPdF(F, mu, lam):
    F, Fp = _d(np.asarray(F).reshape(9))
    H = np.zeros((9, 9))
    _lib_handle().o_snh_dPdF(Fp, mu, lam, H.ctypes.data_as(_D))
    return H


def psd_project(A):
    A = np.array(A, dtype=np.float64, copy=True)
    _lib_handle().o_psd_project(A.shape[0], A.ctypes.data_as(_D))
    return A


def cubic_safe(coef, alpha_l):
    c, cp = _d(coef)
    return _lib_handle().o_cubic_safe(cp, alpha_l)


def pair_safe(kind, X, Q, shrink, dhat):
    """Safe fraction of a PT (kind 0) / EE (kind 1) pair: X, Q are 4 x 3."""
    x, xp = _d(np.asarray(X, dtype=np.float64).reshape(12))
    q, qp = _d(np.asarray(Q, dtype=np.float64).reshape(12))
    return _lib_handle().o_pair_safe(int(kind), xp, qp, shrink, dhat)


def safe_bisect(coef, xs, xu, ys, yu):
    c, cp = _d(coef)
    return _lib_handle().o_safe_bisect(cp, xs, xu, ys, yu)


def pt_cubic(x4, p4):
    x, xp = _d(x4)
    p, pp = _d(p4)
    c = np.zeros(4)
    _lib_handle().o_pt_cubic(xp, pp, c.ctypes.data_as(_D))
    return c


def ee_cubic(x4, p4):
    x, xp = _d(x4)
    p, pp = _d(p4)
    c = np.zeros(4)
    _lib_handle().o_ee_cubic(xp, pp, c.ctypes.data_as(_D))
    return c


def ltight_pt(p4):
    p, pp = _d(p4)
    return _lib_handle().o_ltight_pt(pp)


def ltight_ee(p4):
    p, pp = _d(p4)
    return _lib_handle().o_ltight_ee(pp)


def loriginal_pt(p4):
    p, pp = _d(p4)
    return _lib_handle().o_loriginal_pt(pp)


def solve2x2(A11, A12, A22, b1, b2, eps_sing=1e-12, eps_abs=1e-300):
    mu = C.c_double()
    nu = C.c_double()
    _lib_handle().o_solve2x2(A11, A12, A22, b1, b2, eps_sing, eps_abs, C.byref(mu), C.byref(nu))
    return mu.value, nu.value


def chol_inverse(A):
    """A^-1 by the oracle's Cholesky (with its pivot floor) and the number of
    floored pivots."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.zeros_like(A)
    f = _lib_handle().o_chol_inverse(A.shape[0], A.ctypes.data_as(_D), out.ctypes.data_as(_D))
    return out, f


def chol_floors(reset=False):
    """Pivots floored by every oracle Cholesky since the last reset."""
    return int(_lib_handle().o_chol_floors(1 if reset else 0))


def set_threads(n):
    """Host threads for the oracle's independent loops (0: query); returns the
    number now used.  Results do not depend on it."""
    return int(_lib_handle().o_set_threads(int(n)))
