"""Scene-level pins of the FP64 oracle: closed forms (surface counts, mass,
free fall), finite differences of the incremental potential (Eq. 1), MAS
exactness when one subdomain covers the mesh, the Woodbury identity of Eq. 7
checked against the H~ of Eq. 6, and the invariants of Algorithm 1 (energy
decrease, no intersection) on tiny scenes."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2604_19892_b300 import scenes as S
from tests.geometry import any_intersection, min_surface_distance

RNG = np.random.default_rng(99)


def _xt(sc, x, v):
    h = sc["params"]["h"]
    return x + h * v + h * h * sc["gravity"]


def test_surface_counts_closed_form():
    for n in (1, 2, 3, 5):
        sc = S.two_cubes(n=n, jitter=0.0)
        o = O.Scene(sc)
        sv, sf, se = o.surface()
        # a cube of n^3 cells: 6n^2 + 2 surface vertices, 12n^2 triangles, 18n^2 edges
        assert len(sv) == 2 * (6 * n * n + 2)
        assert len(sf) == 2 * 12 * n * n
        assert len(se) == 2 * 18 * n * n
        assert np.all(np.diff(sv) > 0)
        keys = np.sort(sf, axis=1)
        assert np.all(np.lexsort(keys.T[::-1]) == np.arange(len(keys)))


def test_lumped_mass_total():
    sc = S.two_cubes(n=3, jitter=0.0)
    o = O.Scene(sc)
    assert o.mass().sum() == pytest.approx(2 * 1000.0 * 0.1 ** 3, rel=1e-12)


def test_hierarchy_shape():
    sc = S.two_cubes(n=8)
    o = O.Scene(sc)
    lv = o.levels()
    n = sc["x0"].shape[0]
    for l, (grp, slot) in enumerate(lv):
        assert len(grp) == n
        ng = grp.max() + 1
        assert ng == math.ceil(n / 32)
        counts = np.bincount(grp)
        assert counts.max() <= 32 and counts.min() >= 1
        # slots are a bijection onto 0..size-1 within each group
        for g in range(ng):
            s = np.sort(slot[grp == g])
            assert np.all(s == np.arange(len(s)))
        n = ng
    assert n == 1 and len(lv[-1][0]) <= 32


def _contact_scene(n=2, gap_frac=0.5):
    sc = S.two_cubes(n=n, jitter=0.0, gap=1e-3)
    dhat = sc["params"]["dhat"]
    gap = gap_frac * dhat
    sc = S.two_cubes(n=n, jitter=1e-6, gap=gap, seed=3)
    sc["params"] = dict(sc["params"], dhat=dhat)
    return sc


def test_gradient_matches_finite_differences_with_contacts():
    sc = _contact_scene()
    o = O.Scene(sc)
    x = sc["x0"] + 2e-6 * RNG.normal(size=sc["x0"].shape)
    v = RNG.normal(size=x.shape) * 0.1
    xt = _xt(sc, x, v)
    C = o.contacts(x)
    assert (C["type"] == 0).sum() > 0 and (C["type"] == 1).sum() > 0 and (C["type"] == 2).sum() > 0
    g = o.gradient(x, xt)
    for _ in range(6):
        d = RNG.normal(size=x.shape)
        eps = 1e-8  # central differences settle to ~1e-6 relative here
        fd = (o.energy(x + eps * d, xt) - o.energy(x - eps * d, xt)) / (2 * eps)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-5)
    # per-coordinate on contact vertices (barrier gradient = kappa b'(d) grad d)
    verts = np.unique(C["verts"][C["verts"] >= 0])[:6]
    for vtx in verts:
        for r in range(3):
            e = np.zeros_like(x)
            e[vtx, r] = 1.0
            eps = 1e-8
            fd = (o.energy(x + eps * e, xt) - o.energy(x - eps * e, xt)) / (2 * eps)
            assert g[vtx, r] == pytest.approx(fd, rel=1e-5, abs=1e-7 * np.abs(g).max())


def test_hessian_apply_matches_finite_differences_where_exact():
    """H_base equals the true Hessian when the SNH Hessian is PSD (stretched
    state) and the only contacts are point-ground, whose distance is linear."""
    sc = S.two_cubes(n=2, jitter=0.0)
    # keep only the lower cube, resting dhat/2 above the ground, stretched 3 %
    nv = 27
    dhat = sc["params"]["dhat"]
    x_rest = sc["x_rest"][:nv].copy()
    tets = sc["tets"][: sc["tets"].shape[0] // 2]
    one = dict(sc, x_rest=x_rest, x0=x_rest.copy(), v0=np.zeros_like(x_rest), tets=tets,
               E=sc["E"][: len(tets)], nu=sc["nu"][: len(tets)], rho=sc["rho"][: len(tets)],
               body=sc["body"][:nv])
    one["params"] = dict(sc["params"], dhat=dhat)
    o = O.Scene(one)
    c = x_rest.mean(axis=0)
    x = c + 1.03 * (x_rest - c)
    x[:, 1] += 0.5 * dhat - x[:, 1].min()
    x += 1e-7 * RNG.normal(size=x.shape)
    mu = 1e5 / (2 * 1.4)
    lam = 1e5 * 0.4 / (1.4 * 0.2)
    for t in tets:
        Dm = (x_rest[t[1:]] - x_rest[t[0]]).T
        _, _, H = O.snh_tet(np.linalg.inv(Dm), np.linalg.det(Dm) / 6, mu, lam, x[t].reshape(-1), project=False)
        assert np.linalg.eigvalsh(H).min() > -1e-9 * np.abs(H).max()
    C = o.contacts(x)
    assert len(C["type"]) > 0 and np.all(C["type"] == 2)
    xt = x.copy()
    for _ in range(4):
        d = RNG.normal(size=x.shape)
        Hd = o.hessian_apply(x, d)
        eps = 1e-9
        fd = (o.gradient(x + eps * d, xt) - o.gradient(x - eps * d, xt)) / (2 * eps)
        assert np.linalg.norm(Hd - fd) <= 1e-6 * np.linalg.norm(Hd)


def test_single_subdomain_mas_is_exact_inverse():
    """One subdomain over all DOFs and no coarse level: P = H_base^-1
    (supplement Eq. 2 with D = 1)."""
    sc = _contact_scene(n=1)
    o = O.Scene(sc)
    assert len(o.levels()) == 1
    x = sc["x0"]
    g = RNG.normal(size=x.shape)
    z = o.precond_apply(x, g)
    assert np.linalg.norm(o.hessian_apply(x, z) - g) <= 1e-9 * np.linalg.norm(g)


def _dense_Htilde(o, x_base, x_curr, n):
    E = np.eye(3 * n)
    H = np.zeros((3 * n, 3 * n))
    for i in range(3 * n):
        for j in range(i, 3 * n):
            f = o.hess_forms(x_base, E[i].reshape(n, 3), E[j].reshape(n, 3), x_curr)
            H[i, j] = H[j, i] = f[1]
    return H


def test_woodbury_update_inverts_the_updated_hessian():
    """With one subdomain and K above the number of updates, the updated
    level-0 inverse is (H_base + U U^T)^-1 (Eq. 7), the H~ of Eq. 6."""
    sc = _contact_scene(n=1, gap_frac=0.9)
    o = O.Scene(sc, params={"K": 100000})
    n = sc["x0"].shape[0]
    xb = sc["x0"]
    xc = xb.copy()
    xc[8:, 1] -= 0.6 * sc["params"]["dhat"]  # top cube moves closer: stiffening + new pairs
    xc[8:, 0] += 0.3 * sc["params"]["dhat"]
    nb, nc = len(o.contacts(xb)["type"]), len(o.contacts(xc)["type"])
    assert nc > 0 and nb > 0
    Ht = _dense_Htilde(o, xb, xc, n)
    Hb = _dense_Htilde(o, xb, None, n)
    assert np.linalg.norm(Ht - Hb) > 1e-3 * np.linalg.norm(Hb)  # the update is not empty
    g = RNG.normal(size=(n, 3))
    z = o.precond_apply(xb, g, xc)
    zref = np.linalg.solve(Ht, g.reshape(-1))
    assert np.linalg.norm(z.reshape(-1) - zref) <= 1e-9 * np.linalg.norm(zref)
    # Woodbury form on the same data: B - B U (I + U^T B U)^-1 U^T B
    w, Q = np.linalg.eigh(Ht - Hb)
    keep = w > 1e-12 * w.max()
    U = Q[:, keep] * np.sqrt(w[keep])
    B = np.linalg.inv(Hb)
    Bg = B @ g.reshape(-1)
    W = B @ U
    lam = np.linalg.solve(np.eye(U.shape[1]) + U.T @ W, U.T @ Bg)
    assert np.linalg.norm((Bg - W @ lam) - zref) <= 1e-8 * np.linalg.norm(zref)


def test_multilevel_preconditioner_is_spd_and_matches_dense_form():
    """P = M0^-1 + sum_l C_l^T M_l^-1 C_l (supplement Eq. 4) rebuilt densely
    from the assembled H_base and the oracle's level maps."""
    sc = S.two_cubes(n=3)
    o = O.Scene(sc)
    x = sc["x0"] + 1e-5 * RNG.normal(size=sc["x0"].shape)
    n = x.shape[0]
    lv = o.levels()
    assert len(lv) >= 2
    H = np.zeros((3 * n, 3 * n))
    for i in range(3 * n):
        e = np.zeros(3 * n)
        e[i] = 1
        H[:, i] = o.hessian_apply(x, e.reshape(n, 3)).reshape(-1)
    node = np.arange(n)
    P = np.zeros_like(H)
    Cfine = np.eye(3 * n)
    for l, (grp, slot) in enumerate(lv):
        if l > 0:
            m = lv[l - 1][0].max() + 1  # nodes of level l = groups of level l-1
            Cl = np.zeros((3 * m, 3 * n))
            for v in range(n):
                for r in range(3):
                    Cl[3 * node[v] + r, 3 * v + r] = 1
        else:
            Cl = Cfine
        Al = Cl @ H @ Cl.T
        for gi in range(grp.max() + 1):
            idx = np.where(grp == gi)[0]
            idx = idx[np.argsort(slot[idx])]
            dof = (3 * idx[:, None] + np.arange(3)).reshape(-1)
            blk = np.linalg.inv(Al[np.ix_(dof, dof)])
            R = np.zeros((len(dof), Al.shape[0]))
            R[np.arange(len(dof)), dof] = 1
            P += Cl.T @ R.T @ blk @ R @ Cl
        node = grp[node]  # level-(l+1) node of each vertex
    g = RNG.normal(size=(n, 3))
    z = o.precond_apply(x, g)
    assert np.linalg.norm(z.reshape(-1) - P @ g.reshape(-1)) <= 1e-9 * np.linalg.norm(z)
    a, b = RNG.normal(size=(2, n, 3))
    Pa, Pb = o.precond_apply(x, a), o.precond_apply(x, b)
    assert np.sum(a * Pb) == pytest.approx(np.sum(b * Pa), rel=1e-10)
    assert np.sum(a * Pa) > 0


def test_free_fall_reaches_the_predictor():
    sc = S.free_fall_block(n=2)
    o = O.Scene(sc)
    x, v, st = o.step(sc["x0"], sc["v0"])
    h = sc["params"]["h"]
    assert st["converged"] == 1
    eps = sc["params"]["tol"] * h * o.bbox_diag()
    assert np.abs(x - (sc["x0"] + h * h * sc["gravity"])).max() <= eps
    assert np.abs(v - h * sc["gravity"]).max() <= eps / h


def test_steps_keep_energy_decreasing_and_no_intersection():
    sc = S.small_cubes(n=2, gap=0.004, drop_speed=0.6)
    o = O.Scene(sc)
    sv, sf, se = o.surface()
    x, v = sc["x0"].copy(), sc["v0"].copy()
    saw_contact = False
    for step in range(8):
        x, v, st = o.step(x, v)
        tr = o.trace()
        assert st["converged"] == 1
        for r in tr:
            assert r["energy_after"] <= r["energy_before"]
        saw_contact |= st["n_contacts"] > 0
        assert not any_intersection(x, sf, se)
        assert min_surface_distance(x, sv, sf, se) > 0
        assert x[:, 1].min() > 0
    assert saw_contact


def test_contact_set_matches_independent_brute_force():
    sc = _contact_scene(n=1, gap_frac=0.5)
    o = O.Scene(sc)
    x = sc["x0"] + 1e-6 * RNG.normal(size=sc["x0"].shape)
    dhat = sc["params"]["dhat"]
    sv, sf, se = o.surface()
    C = o.contacts(x)
    got = set()
    for t, (a, b) in zip(C["type"], C["ids"]):
        got.add((int(t), int(a), int(b)))
    from tests.test_oracle_elements import _ee_brute, _pt_brute
    want = set()
    amb = 1e-9 * dhat
    for fi, f in enumerate(sf):
        for p in sv:
            if p in f:
                continue
            d = _pt_brute(x[p], x[f[0]], x[f[1]], x[f[2]])
            if d < dhat - amb:
                want.add((0, int(p), fi))
            elif d < dhat + amb:
                got.discard((0, int(p), fi))
    for i in range(len(se)):
        for j in range(i + 1, len(se)):
            a, b = se[i], se[j]
            if len(set(a) & set(b)):
                continue
            u, w = x[a[1]] - x[a[0]], x[b[1]] - x[b[0]]
            if np.sum(np.cross(u, w) ** 2) < 1e-12 * np.sum(u * u) * np.sum(w * w):
                continue
            d = _ee_brute(x[a[0]], x[a[1]], x[b[0]], x[b[1]])
            if d < dhat - amb:
                want.add((1, i, j))
            elif d < dhat + amb:
                got.discard((1, i, j))
    for p in sv:
        if x[p, 1] < dhat:
            want.add((2, int(p), 0))
    assert got == want


def test_ccd_ground_only_closed_form():
    """Rigid translation toward the ground: PT/EE pairs have no relative
    motion (l_tight = 0), so only the point-ground bound acts and
    alpha_d = min(1, 0.9 min_{v in d} y_v / L)."""
    sc = S.free_fall_block(n=3)
    sc["x0"][:, 1] -= 10.0 - 0.01
    o = O.Scene(sc)
    x = sc["x0"]
    L = 0.05
    p = np.zeros_like(x)
    p[:, 1] = -L
    alpha, passes = o.ccd(x, p)
    grp, _ = o.levels()[0]
    sv, _, _ = o.surface()
    want = np.ones(grp.max() + 1)
    for v in sv:
        want[grp[v]] = min(want[grp[v]], 0.9 * x[v, 1] / L)
    assert passes >= 1
    np.testing.assert_allclose(alpha, want, rtol=1e-14)


def test_ccd_steps_are_intersection_free():
    sc = S.small_cubes(n=3, gap=0.003)
    o = O.Scene(sc)
    sv, sf, se = o.surface()
    x = sc["x0"]
    nv = x.shape[0]
    for trial in range(5):
        p = np.zeros_like(x)
        p[nv // 2:, 1] = -0.02  # upper cube drops through the gap
        p += 0.004 * RNG.normal(size=p.shape)
        alpha, passes = o.ccd(x, p)
        grp, _ = o.levels()[0]
        q = alpha[grp][:, None] * p
        assert alpha.min() < 1.0
        for t in np.linspace(0, 1, 41):
            assert not any_intersection(x + t * q, sf, se)


def test_per_body_ccd_steps_are_intersection_free():
    """The per-body steps (verified with connected bodies as the groups),
    which the energy check tries after the per-subdomain step and first when
    the per-subdomain verification fell back: the mixed motion alpha_b(v) p_v
    crosses no surface anywhere along it (brute force at 41 points)."""
    sc = S.small_cubes(n=3, gap=0.003)
    o = O.Scene(sc)
    sv, sf, se = o.surface()
    x = sc["x0"]
    nv = x.shape[0]
    _, body = o.bodies()
    for trial in range(5):
        p = np.zeros_like(x)
        p[nv // 2:, 1] = -0.02  # upper cube drops through the gap
        p += 0.004 * RNG.normal(size=p.shape)
        _, _, ab, pb = o.ccd(x, p, per_body=True)
        assert ab.min() < 1.0 and pb != 0
        q = ab[body][:, None] * p
        for t in np.linspace(0, 1, 41):
            assert not any_intersection(x + t * q, sf, se)


@pytest.mark.parametrize("K", [1, 3])
def test_topk_keeps_the_stiffest_new_contacts(K):
    """All contacts new (none at the restart point): classification gives
    u = sqrt(k) n, dS = k (Sec. 4.1.1 case 1); with one subdomain the updated
    inverse is (H_base + sum over the K largest k of k n n^T)^-1."""
    sc = _contact_scene(n=1, gap_frac=0.5)
    o = O.Scene(sc, params={"K": K})
    n = sc["x0"].shape[0]
    dhat = sc["params"]["dhat"]
    xb = sc["x0"].copy()
    xb[:, 1] += 0.01  # everything lifted: no contact at the restart point
    xb[8:, 1] += 0.01
    assert len(o.contacts(xb)["type"]) == 0
    xc = sc["x0"] + 1e-6 * RNG.normal(size=xb.shape)
    C = o.contacts(xc)
    assert len(C["k"]) > K
    E = np.eye(3 * n)
    P = np.stack([o.precond_apply(xb, E[i].reshape(n, 3), xc).reshape(-1) for i in range(3 * n)], axis=1)
    Hb = _dense_Htilde(o, xb, None, n)
    D = np.linalg.inv(P) - Hb
    order = np.argsort(-C["k"], kind="stable")[:K]
    want = np.zeros_like(D)
    for i in order:
        nvec = np.zeros(3 * n)
        for j, vtx in enumerate(C["verts"][i]):
            if vtx >= 0:
                nvec[3 * vtx:3 * vtx + 3] += C["grad"][i, 3 * j:3 * j + 3]
        want += C["k"][i] * np.outer(nvec, nvec)
    assert np.linalg.norm(D - want) <= 1e-7 * np.linalg.norm(want)


def test_grid_pair_search_equals_brute_force():
    """The oracle's grid pair search returns exactly the pairs of the
    all-pairs loop: identical contact sets and CCD step sizes."""
    sc = _contact_scene(n=3, gap_frac=0.5)
    ob = O.Scene(sc, params={"brute_force": 1})
    og = O.Scene(sc, params={"brute_force": 0})
    x = sc["x0"] + 1e-6 * RNG.normal(size=sc["x0"].shape)
    cb, cg = ob.contacts(x), og.contacts(x)
    assert len(cb["type"]) > 10
    for k in cb:
        np.testing.assert_array_equal(cb[k], cg[k])
    nv = x.shape[0]
    for trial in range(3):
        p = 0.003 * RNG.normal(size=x.shape)
        p[nv // 2:, 1] -= 0.01
        ab, pb = ob.ccd(x, p)
        ag, pg = og.ccd(x, p)
        np.testing.assert_array_equal(ab, ag)
        assert pb == pg
