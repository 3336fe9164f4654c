"""Brute-force geometric checks used by the tests (numpy, independent of
both the oracle and the CUDA path)."""
import numpy as np


def segment_triangle_hits(p0, p1, a, b, c):
    """Vectorised: does segment p0-p1 cross triangle abc (Moller-Trumbore)?"""
    d = p1 - p0
    e1 = b - a
    e2 = c - a
    h = np.cross(d, e2)
    det = np.einsum("...i,...i->...", e1, h)
    ok = np.abs(det) > 1e-300
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    s = p0 - a
    u = inv * np.einsum("...i,...i->...", s, h)
    q = np.cross(s, e1)
    v = inv * np.einsum("...i,...i->...", d, q)
    t = inv * np.einsum("...i,...i->...", e2, q)
    return ok & (u >= 0) & (v >= 0) & (u + v <= 1) & (t >= 0) & (t <= 1)


def any_intersection(x, sf, se):
    """True if any surface edge passes through a non-incident surface triangle."""
    A = x[sf[:, 0]]
    B = x[sf[:, 1]]
    Cc = x[sf[:, 2]]
    for (i, j) in se:
        hit = segment_triangle_hits(x[i][None], x[j][None], A, B, Cc)
        inc = (sf == i).any(axis=1) | (sf == j).any(axis=1)
        if np.any(hit & ~inc):
            return True
    return False


def _pt_dist(p, a, b, c):
    # sampled-free exact point-triangle distance via projection + edge clamps
    ab, ac = b - a, c - a
    n = np.cross(ab, ac)
    nn = np.einsum("...i,...i->...", n, n)
    t = np.einsum("...i,...i->...", p - a, n) / nn
    proj = p - t[..., None] * n
    # barycentric of proj
    v2 = proj - a
    d00 = np.einsum("...i,...i->...", ab, ab)
    d01 = np.einsum("...i,...i->...", ab, ac)
    d11 = np.einsum("...i,...i->...", ac, ac)
    d20 = np.einsum("...i,...i->...", v2, ab)
    d21 = np.einsum("...i,...i->...", v2, ac)
    den = d00 * d11 - d01 * d01
    v = (d11 * d20 - d01 * d21) / den
    w = (d00 * d21 - d01 * d20) / den
    inside = (v >= 0) & (w >= 0) & (v + w <= 1)
    best = np.where(inside, np.abs(t) * np.sqrt(nn), np.inf)
    for (s0, s1) in ((a, b), (b, c), (c, a)):
        e = s1 - s0
        tt = np.clip(np.einsum("...i,...i->...", p - s0, e) / np.einsum("...i,...i->...", e, e), 0, 1)
        q = s0 + tt[..., None] * e
        best = np.minimum(best, np.linalg.norm(p - q, axis=-1))
    return best


def min_surface_distance(x, sv, sf, se):
    """Minimum point-triangle distance over non-incident surface pairs."""
    A, B, Cc = x[sf[:, 0]], x[sf[:, 1]], x[sf[:, 2]]
    best = np.inf
    for p in sv:
        inc = (sf == p).any(axis=1)
        d = _pt_dist(x[p][None], A, B, Cc)
        d = np.where(inc, np.inf, d)
        best = min(best, d.min())
    return best


def contact_state(sc, frac=0.5):
    """Positions of a two-cube scene with point-triangle, edge-edge and
    point-ground contacts active: the upper cube lowered to within frac*dhat
    of the lower one, the lower one frac*dhat above the ground."""
    x = sc["x0"].copy()
    nv = x.shape[0] // 2
    dhat = sc["params"]["dhat"]
    x[:nv, 1] -= x[:nv, 1].min() - frac * dhat
    gap = x[nv:, 1].min() - x[:nv, 1].max()
    x[nv:, 1] -= gap - frac * dhat
    return x
