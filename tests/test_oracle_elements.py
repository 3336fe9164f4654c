"""Pins of the FP64 oracle's element-level pieces against mathematics that is
independent of the oracle's own code: closed forms, finite differences,
invariances, brute-force sampling, and independent library routines
(numpy.linalg.eigh, numpy polynomial roots, scipy.optimize)."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

import oracle as O

RNG = np.random.default_rng(1234)


# --------------------------------------------------------------------- barrier
# IPC log barrier (reading of Sec. 3.1): b(d) = -(d - dhat)^2 ln(d / dhat)

def test_barrier_vanishes_at_dhat_to_second_order():
    dhat = 1e-3
    for d in (dhat, dhat * (1 - 1e-9)):
        b, b1, b2 = O.barrier(d, dhat)
        assert abs(b) < 1e-24 and abs(b1) < 1e-15 and abs(b2) < 1e-6
    assert O.barrier(2 * dhat, dhat) == (0.0, 0.0, 0.0)


def test_barrier_closed_form_at_dhat_over_e():
    dhat = 2e-3
    d = dhat / math.e  # ln(d/dhat) = -1
    b, _, _ = O.barrier(d, dhat)
    assert b == pytest.approx(dhat * dhat * (1 - 1 / math.e) ** 2, rel=1e-14)


def test_barrier_derivatives_by_finite_differences():
    dhat = 1e-3
    for d in np.linspace(0.05, 0.95, 19) * dhat:
        e = 1e-6 * d
        bp = (O.barrier(d + e, dhat)[0] - O.barrier(d - e, dhat)[0]) / (2 * e)
        bpp = (O.barrier(d + e, dhat)[1] - O.barrier(d - e, dhat)[1]) / (2 * e)
        b, b1, b2 = O.barrier(d, dhat)
        assert b1 == pytest.approx(bp, rel=1e-7)
        assert b2 == pytest.approx(bpp, rel=1e-6)
        assert b > 0 and b1 < 0 and b2 > 0  # rank-1 stiffness k = kappa b'' > 0


# ------------------------------------------------------------------- distances

def _pt_brute(p, t0, t1, t2):
    """Minimise |p - (w0 t0 + w1 t1 + w2 t2)| over the simplex with SLSQP."""
    f = lambda uv: np.sum((p - ((1 - uv[0] - uv[1]) * t0 + uv[0] * t1 + uv[1] * t2)) ** 2)
    best = np.inf
    for start in ((1 / 3, 1 / 3), (0.0, 0.0), (1.0, 0.0), (0.0, 1.0)):
        r = minimize(f, start, method="SLSQP", bounds=[(0, 1), (0, 1)],
                     constraints=[{"type": "ineq", "fun": lambda uv: 1 - uv[0] - uv[1]}],
                     options={"ftol": 1e-16, "maxiter": 500})
        best = min(best, r.fun)
    return math.sqrt(max(best, 0.0))


def _ee_brute(a0, a1, b0, b1):
    f = lambda st: np.sum((a0 + st[0] * (a1 - a0) - b0 - st[1] * (b1 - b0)) ** 2)
    best = np.inf
    for start in ((0.5, 0.5), (0, 0), (1, 1), (0, 1), (1, 0)):
        r = minimize(f, start, method="L-BFGS-B", bounds=[(0, 1), (0, 1)],
                     options={"ftol": 1e-20, "gtol": 1e-14, "maxiter": 1000})
        best = min(best, r.fun)
    return math.sqrt(max(best, 0.0))


def test_pt_distance_matches_constrained_minimisation():
    for _ in range(200):
        t0, t1, t2, p = RNG.normal(size=(4, 3))
        d, w = O.pt_distance(p, t0, t1, t2)
        assert w.min() >= -1e-15 and abs(w.sum() - 1) < 1e-14
        q = w[0] * t0 + w[1] * t1 + w[2] * t2
        assert np.linalg.norm(p - q) == pytest.approx(d, rel=1e-12)
        assert d == pytest.approx(_pt_brute(p, t0, t1, t2), rel=1e-6, abs=1e-9)


def test_pt_distance_special_cases():
    t0, t1, t2 = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    d, w = O.pt_distance(np.array([0.25, 0.25, 0.7]), t0, t1, t2)  # above the interior
    assert d == pytest.approx(0.7, rel=1e-15) and w == pytest.approx([0.5, 0.25, 0.25])
    d, w = O.pt_distance(np.array([-1.0, -1.0, 0.0]), t0, t1, t2)  # beyond a vertex
    assert d == pytest.approx(math.sqrt(2)) and w == pytest.approx([1, 0, 0])
    d, w = O.pt_distance(np.array([0.5, -2.0, 0.0]), t0, t1, t2)  # beside an edge
    assert d == pytest.approx(2.0) and w == pytest.approx([0.5, 0.5, 0])


def test_ee_distance_matches_box_minimisation():
    for _ in range(200):
        a0, a1, b0, b1 = RNG.normal(size=(4, 3))
        d, st = O.ee_distance(a0, a1, b0, b1)
        assert 0 <= st[0] <= 1 and 0 <= st[1] <= 1
        pa = a0 + st[0] * (a1 - a0)
        pb = b0 + st[1] * (b1 - b0)
        assert np.linalg.norm(pa - pb) == pytest.approx(d, rel=1e-12)
        assert d == pytest.approx(_ee_brute(a0, a1, b0, b1), rel=1e-6, abs=1e-9)


def test_ee_distance_special_cases():
    # perpendicular crossing segments offset along z by 0.3
    d, st = O.ee_distance(np.array([-1.0, 0, 0]), np.array([1.0, 0, 0]),
                          np.array([0.0, -1, 0.3]), np.array([0.0, 1, 0.3]))
    assert d == pytest.approx(0.3) and st == pytest.approx([0.5, 0.5])
    # parallel overlapping segments at distance 0.2: any overlap point is a minimiser
    d, st = O.ee_distance(np.array([0.0, 0, 0]), np.array([1.0, 0, 0]),
                          np.array([0.5, 0.2, 0]), np.array([1.5, 0.2, 0]))
    assert d == pytest.approx(0.2)
    # collinear disjoint: endpoint gap
    d, _ = O.ee_distance(np.array([0.0, 0, 0]), np.array([1.0, 0, 0]),
                         np.array([3.0, 0, 0]), np.array([4.0, 0, 0]))
    assert d == pytest.approx(2.0)


# -------------------------------------------------------------------- SNH tet

def _rest_tet():
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.1 + RNG.normal(size=(4, 3)) * 0.01
    Dm = (X[1:] - X[0]).T
    B = np.linalg.inv(Dm)
    vol = np.linalg.det(Dm) / 6
    assert vol > 0
    return X, B, vol


def _rot(a, b, c):
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rx = np.array([[1, 0, 0], [0, math.cos(c), -math.sin(c)], [0, math.sin(c), math.cos(c)]])
    return Rz @ Ry @ Rx


def test_snh_rest_stable_and_rotation_invariant():
    mu, lam = 3.0e4, 1.5e5
    assert O.snh_psi(np.eye(3), mu, lam) == pytest.approx(0.0, abs=1e-10)
    X, B, vol = _rest_tet()
    e, g, _ = O.snh_tet(B, vol, mu, lam, X.reshape(-1))
    assert abs(e) < 1e-9 and np.abs(g).max() < 1e-9  # P(I) = 0
    F = np.eye(3) + 0.2 * RNG.normal(size=(3, 3))
    R = _rot(0.3, -1.1, 2.0)
    assert O.snh_psi(R @ F, mu, lam) == pytest.approx(O.snh_psi(F, mu, lam), rel=1e-12)
    # rigid motion of the whole tet keeps the energy and gives zero net force
    Y = X @ R.T + np.array([0.3, -0.2, 5.0])
    e2, g2, _ = O.snh_tet(B, vol, mu, lam, Y.reshape(-1))
    assert abs(e2) < 1e-9 and np.abs(g2).max() < 1e-8


def test_snh_closed_form_isochoric_stretch():
    mu, lam = 2.0, 7.0
    F = np.diag([2.0, 0.5, 1.0])  # J = 1: only the first term survives
    assert O.snh_psi(F, mu, lam) == pytest.approx(mu / 2 * (4 + 0.25 + 1 - 3), rel=1e-15)


def test_snh_gradient_and_hessian_by_finite_differences():
    mu, lam = 3.0e4, 1.5e5
    X, B, vol = _rest_tet()
    Y = (X + 0.01 * RNG.normal(size=X.shape)).reshape(-1)
    e, g, H = O.snh_tet(B, vol, mu, lam, Y, project=False)
    h = 1e-7
    gfd = np.zeros(12)
    Hfd = np.zeros((12, 12))
    for i in range(12):
        yp, ym = Y.copy(), Y.copy()
        yp[i] += h
        ym[i] -= h
        gfd[i] = (O.snh_tet(B, vol, mu, lam, yp)[0] - O.snh_tet(B, vol, mu, lam, ym)[0]) / (2 * h)
        Hfd[:, i] = (O.snh_tet(B, vol, mu, lam, yp)[1] - O.snh_tet(B, vol, mu, lam, ym)[1]) / (2 * h)
    assert np.linalg.norm(g - gfd) <= 1e-7 * np.linalg.norm(g)
    assert np.linalg.norm(H - Hfd) <= 1e-7 * np.linalg.norm(H)
    assert np.allclose(H, H.T, rtol=0, atol=1e-9 * np.abs(H).max())


def test_snh_dPdF_is_second_derivative_of_psi():
    mu, lam = 1.3, 4.1
    F = np.eye(3) + 0.3 * RNG.normal(size=(3, 3))
    D = O.snh_dPdF(F, mu, lam)

    def vec_to_F(v):  # vec is column-major: v[3c + r] = F[r, c]
        return v.reshape(3, 3).T

    v0 = F.T.reshape(-1)
    h = 1e-4
    Dfd = np.zeros((9, 9))
    for i in range(9):
        for j in range(9):
            def f(di, dj):
                v = v0.copy()
                v[i] += di
                v[j] += dj
                return O.snh_psi(vec_to_F(v), mu, lam)
            Dfd[i, j] = (f(h, h) - f(h, -h) - f(-h, h) + f(-h, -h)) / (4 * h * h)
    assert np.abs(D - Dfd).max() <= 1e-6 * np.abs(D).max()


def test_psd_projection_against_eigh():
    for n in (3, 9, 12):
        A = RNG.normal(size=(n, n))
        A = A + A.T
        P = O.psd_project(A)
        w, Q = np.linalg.eigh(A)
        Pref = (Q * np.maximum(w, 0)) @ Q.T
        assert np.abs(P - Pref).max() <= 1e-12 * np.abs(A).max()
        assert np.linalg.eigvalsh(P).min() >= -1e-12 * np.abs(A).max()
        S = A @ A.T  # already PSD: unchanged
        assert np.abs(O.psd_project(S) - S).max() <= 1e-12 * np.abs(S).max()


def test_projected_tet_hessian_is_psd():
    mu, lam = 3.0e4, 1.5e5
    X, B, vol = _rest_tet()
    for _ in range(10):
        Y = (X + 0.05 * RNG.normal(size=X.shape)).reshape(-1)
        _, _, H = O.snh_tet(B, vol, mu, lam, Y, project=True)
        assert np.linalg.eigvalsh(H).min() >= -1e-9 * np.abs(H).max()


# ----------------------------------------------------------------- CCD pieces

def _det_at(x4, p4, t, kind):
    X = (x4 + t * p4).reshape(4, 3)
    if kind == "pt":  # (t0, t1, t2, p)
        M = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    else:  # (a0, a1, b0, b1): det[b0 - a0, a1 - a0, b1 - a0]
        M = np.stack([X[2] - X[0], X[1] - X[0], X[3] - X[0]], axis=1)
    return np.linalg.det(M)


@pytest.mark.parametrize("kind", ["pt", "ee"])
def test_coplanarity_cubic_coefficients(kind):
    for _ in range(50):
        x4, p4 = RNG.normal(size=(2, 12))
        c = O.pt_cubic(x4, p4) if kind == "pt" else O.ee_cubic(x4, p4)
        for t in np.linspace(-1, 2, 7):
            val = ((c[3] * t + c[2]) * t + c[1]) * t + c[0]
            assert val == pytest.approx(_det_at(x4, p4, t, kind), rel=1e-9, abs=1e-12)


def test_ltight_bounds_and_frame_invariance():
    for _ in range(200):
        p4 = RNG.normal(size=12)
        lt = O.ltight_pt(p4)
        lo = O.loriginal_pt(p4)
        assert lt <= lo + 1e-15  # supplement Eq. 23 vs Eq. 29
        shift = np.tile(RNG.normal(size=3) * 10, 4)
        assert O.ltight_pt(p4 + shift) == pytest.approx(lt, rel=1e-12)
        assert O.ltight_ee(p4 + shift) == pytest.approx(O.ltight_ee(p4), rel=1e-12)
        # the bound dominates the relative displacement of any convex combination
        w = RNG.dirichlet(np.ones(3))
        P = p4.reshape(4, 3)
        rel = P[0] - (w[0] * P[1] + w[1] * P[2] + w[2] * P[3])
        assert np.linalg.norm(rel) <= lt + 1e-12
        s, t = RNG.uniform(size=2)
        rel = (1 - s) * P[0] + s * P[1] - (1 - t) * P[2] - t * P[3]
        assert np.linalg.norm(rel) <= O.ltight_ee(p4) + 1e-12
    same = np.tile(np.array([0.3, -2.0, 1.0]), 4)
    assert O.ltight_pt(same) == 0.0 and O.ltight_ee(same) == 0.0


def _first_root_after(coef, x0):
    """Smallest real root of the cubic in (x0, 1], in long double, or None."""
    d, c, b, a = [np.longdouble(v) for v in coef]
    roots = np.roots([float(a), float(b), float(c), float(d)]) if a != 0 else np.roots([float(b), float(c), float(d)])
    best = None
    for r in roots:
        if abs(r.imag) > 1e-9 * max(1.0, abs(r.real)):
            continue
        t = float(r.real)
        # polish in long double by Newton
        tt = np.longdouble(t)
        for _ in range(5):
            f = ((a * tt + b) * tt + c) * tt + d
            fp = (3 * a * tt + 2 * b) * tt + c
            if fp == 0:
                break
            tt = tt - f / fp
        t = float(tt)
        if x0 < t <= 1.0 and (best is None or t < best):
            best = t
    return best


def test_cubic_safe_is_safe_and_tight():
    for trial in range(3000):
        coef = RNG.normal(size=4)
        if trial % 3 == 0:
            # plant a root in (0, 1)
            r = RNG.uniform(0.05, 0.95)
            q = RNG.normal(size=3)
            coef = np.polynomial.polynomial.polymul([-r, 1.0], q[:2].tolist() + [q[2]])[:4]
        al = RNG.uniform(-0.2, 0.8)
        a = O.cubic_safe(coef, al)
        x0 = max(al, 0.0)
        assert x0 <= a <= 1.0
        f = lambda t: ((coef[3] * t + coef[2]) * t + coef[1]) * t + coef[0]
        y0 = f(x0)
        ts = np.linspace(x0, a, 2001)
        ys = f(ts)
        # no sign change of f on [x0, alpha]
        assert np.all(np.sign(ys) == np.sign(y0)) or y0 == 0
        r = _first_root_after(coef, x0)
        if r is None:
            assert a == 1.0
        else:
            assert a <= r + 1e-12
            # if the root is in the first monotone segment, bisection is tight
            fp = lambda t: (3 * coef[3] * t + 2 * coef[2]) * t + coef[1]
            crit = [t for t in np.roots([3 * coef[3], 2 * coef[2], coef[1]]) if abs(t.imag) < 1e-12
                    and x0 < t.real < r] if coef[3] != 0 else []
            if not crit:
                assert r - a <= 2.0 ** -16 * (1.0 - x0) * (1 + 1e-9) + 1e-15 or r - a <= 2.0 ** -16 * (r - x0) * 2


def test_cubic_safe_edge_cases():
    assert O.cubic_safe([1.0, 2.0, 3.0, 4.0], 1.0) == 1.0
    assert O.cubic_safe([1.0, 2.0, 3.0, 4.0], 5.0) == 1.0
    # f(alpha_l) = 0 returns alpha_l
    assert O.cubic_safe([-0.5, 1.0, 0.0, 0.0], 0.5) == 0.5
    # linear f with root 0.3: alpha in [0.3 - 2^-16, 0.3)
    a = O.cubic_safe([-0.3, 1.0, 0.0, 0.0], 0.0)
    assert 0.3 - 2.0 ** -16 <= a < 0.3


def test_safe_bisect_precision():
    for r in RNG.uniform(0.01, 0.99, size=50):
        coef = [-r, 1.0, 0.0, 0.0]
        a = O.safe_bisect(coef, 0.0, 1.0, -r, 1.0 - r)
        assert r - 2.0 ** -16 <= a < r


# ------------------------------------------------------------------- 2x2 solve

def test_solve2x2_closed_form_and_fallback():
    for _ in range(100):
        M = RNG.normal(size=(2, 2))
        A = M @ M.T + 0.1 * np.eye(2)
        A11, A12, A22 = A[0, 0], -A[0, 1], A[1, 1]  # system matrix [A11 -A12; -A12 A22]
        b = RNG.normal(size=2)
        mu, nu = O.solve2x2(A11, A12, A22, b[0], b[1])
        assert np.allclose(A @ [mu, nu], b, rtol=1e-12, atol=1e-12)
    # z parallel to p: singular, falls back to steepest descent (supplement Eq. 21)
    assert O.solve2x2(4.0, 2.0, 1.0, 1.0, 1.0) == (1.0, 0.0)
    assert O.solve2x2(0.0, 0.0, 0.0, 0.0, 0.0) == (1.0, 0.0)


def test_subspace_iteration_reproduces_pcg_on_a_quadratic():
    """On f(x) = x^T A x / 2 - b^T x with a fixed SPD preconditioner, the 2D
    subspace minimisation (Eq. 10) with unit steps generates the textbook PCG
    iterates (the minimiser over span{z, p} of a quadratic is the CG step)."""
    n = 30
    M = RNG.normal(size=(n, n))
    A = M @ M.T + n * np.eye(n)
    b = RNG.normal(size=n)
    Pm = np.diag(1.0 / np.diag(A))
    # ours
    x = np.zeros(n)
    p = np.zeros(n)
    ours = []
    for k in range(8):
        g = A @ x - b
        z = Pm @ g
        if k == 0:
            mu, nu = (g @ z) / (z @ A @ z), 0.0
        else:
            mu, nu = O.solve2x2(z @ A @ z, z @ A @ p, p @ A @ p, g @ z, -(g @ p))
        p = -mu * z + nu * p
        assert g @ p < 0  # descent, supplement Eq. 22
        x = x + p
        ours.append(x.copy())
    # textbook PCG
    x = np.zeros(n)
    r = b - A @ x
    zz = Pm @ r
    d = zz.copy()
    ref = []
    for k in range(8):
        al = (r @ zz) / (d @ A @ d)
        x = x + al * d
        rn = r - al * A @ d
        zn = Pm @ rn
        d = zn + (rn @ zn) / (r @ zz) * d
        r, zz = rn, zn
        ref.append(x.copy())
    for a, c in zip(ours, ref):
        assert np.linalg.norm(a - c) <= 1e-9 * np.linalg.norm(c)


def test_pair_safe_cuts_a_grazing_step_at_the_minimum_separation():
    """A point sliding over a triangle towards its plane never becomes
    coplanar, so the coplanarity walk alone would allow the whole step and
    leave a 1e-9 gap; the step is cut where the gap reaches s min(d0, dhat),
    to the bisection's resolution (the distance is linear in t there)."""
    s, dhat = 0.1, 1e-3
    X = np.array([[-0.5, 0.25, 1e-3], [0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float)
    Q = np.zeros((4, 3))
    Q[0] = [0.75, 0.0, -(1e-3 - 1e-9)]
    a = O.pair_safe(0, X, Q, s, dhat)
    d0 = math.sqrt(0.25 + 1e-6)
    thr = s * min(d0, dhat)
    t_star = (1e-3 - thr) / (1e-3 - 1e-9)          # over the interior, d(t) = z(t)
    al = (1 - s) * d0 / np.linalg.norm(Q[0])
    assert a < 1.0
    assert abs(a - t_star) <= (1.0 - al) * 2.0 ** -12 + 1e-12
    assert _brute_pt_distance(X + a * Q) >= thr * (1 - 1e-12)


def test_pair_safe_direct_approach_keeps_the_minimum_separation():
    """Falling straight onto a triangle: the plane is crossed at t = 0.5, the
    walk stops before it, and the step ends at least s min(d0, dhat) away."""
    s, dhat = 0.1, 1e-3
    X = np.array([[0.25, 0.25, 1e-3], [0, 0, 0], [1, 0, 0], [0, 1, 0]], dtype=float)
    Q = np.zeros((4, 3))
    Q[0] = [0, 0, -2e-3]
    a = O.pair_safe(0, X, Q, s, dhat)
    assert a < 0.5
    assert 1e-3 - 2e-3 * a >= s * 1e-3 * (1 - 1e-12)


def test_pair_safe_random_pairs_never_cross_and_end_apart():
    """Random PT and EE pairs and motions: no coplanarity sign change on
    [0, alpha] beyond alpha_l, and a step longer than alpha_l ends at least
    s min(d0, dhat) away."""
    s, dhat = 0.1, 0.05
    for trial in range(300):
        kind = trial % 2
        X = RNG.normal(size=(4, 3)) * 0.1
        Q = RNG.normal(size=(4, 3)) * 0.1
        a = O.pair_safe(kind, X, Q, s, dhat)
        assert 0.0 <= a <= 1.0
        dist = _brute_pt_distance if kind == 0 else _brute_ee_distance
        d0 = dist(X)
        l = (O.ltight_pt if kind == 0 else O.ltight_ee)(Q.reshape(12))
        al = (1 - s) * d0 / l if l > 0 else math.inf
        if a > al:
            assert dist(X + a * Q) >= s * min(d0, dhat) * (1 - 1e-6)


def _brute_pt_distance(X):
    return _pt_brute(X[0], X[1], X[2], X[3])


def _brute_ee_distance(X):
    return _ee_brute(X[0], X[1], X[2], X[3])
