"""Pins of oracle parts that a plausible slip would otherwise leave unseen:
the plain Cholesky of the MAS blocks and its pivot floor (supplement
Sec. 1.1), the rounding allowance of the energy check (Table 2's line-search
stage) and the convergence order of Algorithm 1, the three cases of the
contact classification (Sec. 4.1.1), the top-K tie-break, the restart ratio
r_k (Eq. 11) and the gradient by Richardson-extrapolated differences."""
import numpy as np
import pytest

import oracle as O
from paper_2604_19892_b300 import scenes as S
from tests.geometry import contact_state

RNG = np.random.default_rng(7)


# ---------------------------------------------------------------- Cholesky

def _spd(n, cond, rng):
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    ev = np.logspace(0.0, np.log10(cond), n)
    A = (Q * ev) @ Q.T
    return 0.5 * (A + A.T), (Q / ev) @ Q.T


@pytest.mark.parametrize("cond", [1e2, 1e6, 1e10])
def test_chol_inverse_is_exact_on_spd_blocks(cond):
    """A 96x96 SPD block of known spectrum: the inverse agrees with the
    spectral inverse to rounding times the condition number, and no pivot
    reaches the floor (the floor leaves such a block unchanged)."""
    A, ref = _spd(96, cond, RNG)
    inv, floored = O.chol_inverse(A)
    assert floored == 0
    assert np.linalg.norm(inv - ref) <= 64 * 2.0 ** -52 * cond * np.linalg.norm(ref)


def test_chol_floors_an_exactly_singular_pivot():
    """[[1, 1], [1, 1]] has a second pivot of exactly 0, floored at 1e-12 of
    its diagonal entry: the factorised matrix is [[1, 1], [1, 1 + 1e-12]],
    whose inverse is [[1 + 1e-12, -1], [-1, 1]] / 1e-12."""
    inv, floored = O.chol_inverse(np.array([[1.0, 1.0], [1.0, 1.0]]))
    assert floored == 1
    want = np.array([[1.0 + 1e-12, -1.0], [-1.0, 1.0]]) / 1e-12
    np.testing.assert_allclose(inv, want, rtol=1e-6)


def test_parity_states_never_reach_the_pivot_floor():
    """The contact states the GPU parity tests use (and a few timesteps of the
    impact scene) factorise every MAS block without a floored pivot: parity
    there compares plain Cholesky inverses."""
    O.chol_floors(reset=True)
    for sc in (S.two_cubes(n=3, gap=0.004), S.two_cubes(n=8)):
        o = O.Scene(sc)
        xb = contact_state(sc, 0.9)
        xc = contact_state(sc, 0.4) + 1e-6 * RNG.normal(size=xb.shape)
        g = RNG.normal(size=xb.shape)
        o.precond_apply(xb, g)
        o.precond_apply(xb, g, xc)
    sc = S.ground_drop(n=3, gap=0.003, drop_speed=0.5)
    o = O.Scene(sc, params={"tol": 1e-7})
    x, v = sc["x0"].copy(), sc["v0"].copy()
    for _ in range(3):
        x, v, st = o.step(x, v)
        assert st["converged"] == 1
    assert O.chol_floors() == 0


# ---------------------------------------------------------------- energy check

def _relabelled(sc, rng):
    """The same scene with vertices and tets renumbered and each tet's
    vertices rotated by an even permutation (orientation kept)."""
    nv, nt = sc["x0"].shape[0], sc["tets"].shape[0]
    perm = rng.permutation(nv)            # new id -> old id
    inv = np.empty(nv, np.int64)
    inv[perm] = np.arange(nv)
    tord = rng.permutation(nt)
    tets = inv[sc["tets"][tord]]
    even = np.array([[0, 1, 2, 3], [1, 2, 0, 3], [2, 0, 1, 3], [0, 2, 3, 1]])
    tets = np.take_along_axis(tets, even[rng.integers(0, 4, nt)], axis=1).astype(np.int32)
    out = dict(sc)
    for k in ("x_rest", "x0", "v0"):
        out[k] = sc[k][perm]
    out["body"] = sc["body"][perm]
    out["tets"] = tets
    for k in ("E", "nu", "rho"):
        out[k] = sc[k][tord]
    return out, perm


def test_energy_tolerance_covers_the_rounding_of_the_energy():
    """The same state summed in another order, with every tet's deformation
    gradient formed from other edge vectors, gives energies that differ by
    rounding only: within the allowance tau of the energy check, which is
    itself far below the energy (relative 1e-10 here)."""
    sc = S.small_cubes(n=3, gap=0.004)
    o = O.Scene(sc)
    x = contact_state(sc, 0.5) + 1e-5 * RNG.normal(size=sc["x0"].shape)
    h = sc["params"]["h"]
    xt = x + h * 0.3 * RNG.normal(size=x.shape) + h * h * sc["gravity"]
    assert len(o.contacts(x)["type"]) > 0
    E = o.energy(x, xt)
    tau = o.energy_tolerance(E)
    assert 0 < tau <= 1e-10 * abs(E)
    worst = 0.0
    for seed in range(4):
        sc2, perm = _relabelled(sc, np.random.default_rng(seed))
        E2 = O.Scene(sc2).energy(x[perm], xt[perm])
        worst = max(worst, abs(E2 - E))
    assert worst <= tau, (worst, tau)


def test_tight_tolerance_steps_converge():
    """At tol 1e-10 the last steps of a timestep change the energy by less
    than it can be resolved; every timestep of the impact scene still ends
    converged (accepted within tau, or the restart's own convergence test)
    and no accepted step raises the energy by more than tau."""
    sc = S.ground_drop(n=3, gap=0.003, drop_speed=0.5)
    o = O.Scene(sc, params={"tol": 1e-10})
    x, v = sc["x0"].copy(), sc["v0"].copy()
    for _ in range(3):
        x, v, st = o.step(x, v)
        assert st["converged"] == 1, st
        for r in o.trace():
            assert r["energy_after"] - r["energy_before"] <= o.energy_tolerance(r["energy_before"])


# ---------------------------------------------------------------- classification

def _two_tet_scene():
    """A lower tet with its top face in the plane y = 0 and an upper tet whose
    apex points down at that face, dhat/2 above its interior; no ground."""
    lo = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.0, 0.0, 0.1], [0.0, -0.1, 0.0]])
    up = np.array([[0.0, 0.0, 0.0], [0.05, 0.08, 0.0], [-0.03, 0.08, 0.04], [-0.03, 0.08, -0.04]])
    t = np.array([[0, 1, 2, 3]], np.int64)
    bodies = [(lo, S._orient(lo, t).astype(np.int32), 1e5, 0.4, 1000.0),
              (up, S._orient(up, t).astype(np.int32), 1e5, 0.4, 1000.0)]
    sc = S._assemble(bodies, ground=(0.0, 1.0, 0.0, np.nan))
    sc["params"] = S.default_params(0.2, 1.0 / 30, 1e5)   # dhat = 2e-4
    return sc


def _place(sc, apex):
    x = sc["x_rest"].copy()
    x[4:] += np.asarray(apex) - x[4]
    return x


def _pt_key(o, x):
    """Oracle contact list at x, indexed by (type, ida, idb)."""
    c = o.contacts(x)
    return {(int(t), int(a), int(b)): i for i, (t, (a, b)) in enumerate(zip(c["type"], c["ids"]))}, c


def _top_face_key(o):
    sv, sf, se = o.surface()
    tri = int(np.where((np.sort(sf, axis=1) == [0, 1, 2]).all(axis=1))[0][0])
    return (0, 4, tri)


def test_classification_stiffer_contact_adds_the_stiffness_difference():
    """Case 2 of Sec. 4.1.1, same normal and larger k: u = sqrt(k - k_base) n
    with dS = k - k_base."""
    sc = _two_tet_scene()
    dhat = sc["params"]["dhat"]
    o = O.Scene(sc)
    key = _top_face_key(o)
    xb = _place(sc, (0.02, 0.5 * dhat, 0.02))
    xc = _place(sc, (0.02, 0.3 * dhat, 0.02))
    kb, cb = _pt_key(o, xb)
    kc, cc = _pt_key(o, xc)
    assert list(kb) == [key] and list(kc) == [key]
    k_b, k_c = cb["k"][kb[key]], cc["k"][kc[key]]
    assert k_c > k_b
    o.precond_apply(xb, np.zeros_like(xb), xc)
    u = o.updates()
    assert u["dS"].shape == (1,) and tuple(u["key"][0]) == key
    assert u["dS"][0] == pytest.approx(k_c - k_b, rel=1e-12)
    np.testing.assert_allclose(u["u"][0], np.sqrt(k_c - k_b) * cc["grad"][kc[key]], rtol=1e-12, atol=1e-300)


def test_classification_softer_contact_adds_nothing():
    sc = _two_tet_scene()
    dhat = sc["params"]["dhat"]
    o = O.Scene(sc)
    key = _top_face_key(o)
    xb = _place(sc, (0.02, 0.5 * dhat, 0.02))
    xc = _place(sc, (0.02, 0.8 * dhat, 0.02))
    kc, _ = _pt_key(o, xc)
    assert list(kc) == [key]
    o.precond_apply(xb, np.zeros_like(xb), xc)
    assert o.updates()["dS"].shape == (0,)


def test_classification_rotated_contact_counts_as_new():
    """The apex moved past the face's edge x + z = 0.1: the closest point is
    on that edge and the direction has turned by atan(0.4 / 0.3) = 53 degrees
    (> 25), so the contact is treated as new, dS = k, even though it is
    softer than at the restart point."""
    sc = _two_tet_scene()
    dhat = sc["params"]["dhat"]
    o = O.Scene(sc)
    key = _top_face_key(o)
    xb = _place(sc, (0.02, 0.3 * dhat, 0.02))
    out = 0.4 * dhat / np.sqrt(2.0)       # outward along the edge normal (1, 0, 1)/sqrt(2)
    xc = _place(sc, (0.05 + out, 0.3 * dhat, 0.05 + out))
    kb, cb = _pt_key(o, xb)
    kc, cc = _pt_key(o, xc)
    assert key in kb and key in kc
    k_b, k_c = cb["k"][kb[key]], cc["k"][kc[key]]
    assert k_c < k_b                      # softer: case 2 alone would skip it
    o.precond_apply(xb, np.zeros_like(xb), xc)
    u = o.updates()
    keys = [tuple(k) for k in u["key"]]
    i = keys.index(key)
    assert u["dS"][i] == pytest.approx(k_c, rel=1e-12)
    np.testing.assert_allclose(u["u"][i], np.sqrt(k_c) * cc["grad"][kc[key]], rtol=1e-12, atol=1e-300)
    # every other update is a contact absent at the restart point: dS = k
    for j, kk in enumerate(keys):
        if kk != key:
            assert kk not in kb
            assert u["dS"][j] == pytest.approx(cc["k"][kc[kk]], rel=1e-12)


def test_topk_breaks_ties_by_ascending_key():
    """A jitter-free cube dhat/2 above the ground: every bottom vertex has the
    same point-ground distance, so all those new contacts tie on dS = k; each
    subdomain keeps the K of smallest key (vertex id)."""
    x, t = S.box_mesh(3, 0.1 / 3, (0.0, 0.5, 0.0))
    sc = S._assemble([(x, t, 1e5, 0.4, 1000.0)])
    sc["params"] = S.default_params(S.bbox_diag(x), 1.0 / 30, 1e5)
    dhat = sc["params"]["dhat"]
    K = 3
    o = O.Scene(sc, params={"K": K})
    xb = sc["x0"].copy()                         # 0.5 m up: no contact
    xc = sc["x0"] - [0.0, 0.5 - 0.5 * dhat, 0.0]
    c = o.contacts(xc)
    bottom = np.where(sc["x0"][:, 1] == 0.5)[0]
    assert len(c["type"]) == len(bottom) == 16 and np.all(c["type"] == 2)
    assert np.all(c["k"] == c["k"][0])   # exact ties
    o.precond_apply(xb, np.zeros_like(xb), xc)
    u = o.updates()
    grp, _ = o.levels()[0]
    for gi in range(grp.max() + 1):
        mine = sorted(int(v) for v in bottom if grp[v] == gi)
        picked = [int(u["key"][i][1]) for i in o.topk(gi)]
        assert picked == mine[:K], (gi, picked, mine)


# ---------------------------------------------------------------- restart ratio

def test_restart_ratio_vanishes_on_a_quadratic_potential():
    """With a negligible elastic modulus and no contact the incremental
    potential is the quadratic inertia term, H~ is its exact Hessian and P is
    fixed between restarts: the 2D subspace step is preconditioned CG, whose
    residuals are P-orthogonal, so r_k = |g_{k+1}^T z_k| / g_{k+1}^T z_{k+1}
    (Eq. 11) is at rounding level and no restart is triggered by it. A slip
    that used g_k in the numerator would make r_k ~ 1 and restart every
    iteration."""
    x, t = S.box_mesh(10, 0.01, (0.0, 5.0, 0.0))    # 1,331 vertices, three MAS levels
    sc = S._assemble([(x, t, 1e-6, 0.4, 1000.0)], ground=(0.0, 1.0, 0.0, np.nan))
    sc["params"] = S.default_params(S.bbox_diag(x), 1.0 / 30, 1e5)
    o = O.Scene(sc, params={"tol": 1e-6})
    assert len(o.levels()) == 3
    v = 0.005 * RNG.normal(size=x.shape)   # moves far less than any surface gap
    xn, vn, st = o.step(sc["x0"], v)
    tr = o.trace()
    assert st["converged"] == 1
    assert all(r["n_contacts"] == 0 and r["alpha_min"] == 1.0 for r in tr)
    # P M has the eigenvalues 1, 2, 3 (one per level), so CG needs three
    # iterations; the records before g^T z reaches rounding level
    live = [r for r in tr if r["gz"] > 1e-12 * tr[0]["gz"]]
    assert len(live) == 3 and tr[0]["restart"] == 1
    for r in live[1:]:
        assert r["restart"] == 0 and r["r"] <= 1e-8, r
    h = sc["params"]["h"]
    xt = sc["x0"] + h * v + h * h * sc["gravity"]
    assert np.abs(xn - xt).max() <= 1e-6 * h * o.bbox_diag()


def test_restart_follows_the_ratio_on_a_nonlinear_step():
    """On an impact step the ratio does exceed delta, and each iteration after
    one with r_k > delta restarts (Eq. 11)."""
    sc = S.ground_drop(n=3, gap=0.003, drop_speed=0.5)
    o = O.Scene(sc, params={"tol": 1e-7})
    x, v = sc["x0"].copy(), sc["v0"].copy()
    seen = 0
    for _ in range(2):
        x, v, st = o.step(x, v)
        tr = o.trace()
        for a, b in zip(tr[:-1], tr[1:]):
            if a["r"] > sc["params"]["delta"]:
                assert b["restart"] == 1
                seen += 1
    assert seen > 0


# ---------------------------------------------------------------- gradient

def test_gradient_matches_richardson_differences_to_1e7():
    """Central differences extrapolated (Richardson, error O(eps^4)) at a step
    where FP64 rounding of E stays far below the tolerance: every directional
    derivative of Eq. 1 with point-triangle, edge-edge and point-ground
    contacts agrees with the gradient to 1e-7 of |g| |d|. The upper cube is
    turned 30 degrees about the vertical so that facing edges cross at an
    angle: nearly parallel edge pairs have an edge-edge distance whose higher
    derivatives scale with 1 / sin(angle), which no small difference step
    resolves. The state is seeded; that the differences have converged there
    is checked too (the estimates from eps and 2 eps agree to 1e-7)."""
    rng = np.random.default_rng(0)
    sc = S.two_cubes(n=2, jitter=1e-6, seed=3)
    nv = sc["x0"].shape[0] // 2
    up = sc["x_rest"][nv:]
    c = up.mean(axis=0)
    a = np.radians(30.0)
    R = np.array([[np.cos(a), 0.0, np.sin(a)], [0.0, 1.0, 0.0], [-np.sin(a), 0.0, np.cos(a)]])
    sc["x_rest"][nv:] = (up - c) @ R.T + c
    sc["x0"] = sc["x_rest"].copy()
    o = O.Scene(sc)
    x = contact_state(sc, 0.5) + 2e-6 * rng.normal(size=sc["x0"].shape)
    v = rng.normal(size=x.shape) * 0.1
    h = sc["params"]["h"]
    xt = x + h * v + h * h * sc["gravity"]
    C = o.contacts(x)
    assert {0, 1, 2} <= set(int(t) for t in C["type"])
    g = o.gradient(x, xt)
    eps = 1e-3 * sc["params"]["dhat"]

    def cd(d, e):
        return (o.energy(x + e * d, xt) - o.energy(x - e * d, xt)) / (2 * e)

    for _ in range(8):
        d = rng.normal(size=x.shape)
        d /= np.abs(d).max()
        scale = np.linalg.norm(g) * np.linalg.norm(d)
        r1 = (4.0 * cd(d, eps / 2) - cd(d, eps)) / 3.0
        r2 = (4.0 * cd(d, eps) - cd(d, 2 * eps)) / 3.0
        assert abs(r1 - r2) <= 1e-7 * scale
        assert abs(np.sum(g * d) - r1) <= 1e-7 * scale


# ---------------------------------------------------------------- threads

def test_oracle_results_do_not_depend_on_the_thread_count():
    """Only loops with independent iterations run in parallel (per-tet
    Hessians, per-subdomain factorisations), so one timestep gives the same
    bits on one host thread and on four."""
    sc = S.small_cubes(n=3, gap=0.004, drop_speed=0.5)
    out = []
    for th in (1, 4):
        O.set_threads(th)
        o = O.Scene(sc)
        x, v, st = o.step(sc["x0"], sc["v0"])
        out.append((x, st["iters"]))
    O.set_threads(0)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_subdomain_fallback_takes_the_verified_body_steps_safely():
    """Thin spikes crossing several 32-vertex subdomains (two small spiky
    balls): in timestep 1 the per-subdomain verification of straddling pairs
    falls back on some iterations while the per-body one verifies, and the
    energy check then starts from the per-body steps. Every accepted step
    keeps the state separated (all active contacts at d > 0, which the
    oracle's own contact search checks), the energy never rises beyond the
    rounding allowance, and the timestep converges."""
    sc = S.spiky_balls(n_balls=2, cells=4, n_spikes=8, layers=64)
    o = O.Scene(sc)
    x, v, _ = o.step(sc["x0"].copy(), sc["v0"].copy())
    x, v, st = o.step(x, v)
    tr = o.trace()
    fb = [r for r in tr if r["ccd_passes"] < 0 and r["ccd_passes_body"] >= 0]
    assert fb, "the scene no longer exercises the fallback"
    assert st["converged"] and st["min_dist"] > 0.0
    for r in tr:
        assert r["energy_after"] <= r["energy_before"] + o.energy_tolerance(r["energy_before"])


def test_forms_are_the_quadratic_forms_of_the_patched_hessian():
    """Eq. 6: z^T H~ z, z^T H~ p and p^T H~ p, with H~ = H_base plus u u^T over
    the untruncated differential set (Sec. 4.1.1), equal the bilinear forms of
    the oracle's Hessian apply (pinned to finite differences) plus the sum of
    (u . z_c)(u . p_c) over its classified updates, each u placed on its
    contact's vertices."""
    sc = S.two_cubes(n=3, jitter=1e-4, seed=4)
    o = O.Scene(sc)
    xb, xc = contact_state(sc, 0.9), contact_state(sc, 0.4)
    rng = np.random.default_rng(11)
    z, p = rng.normal(size=(2,) + xb.shape)
    f0 = o.hess_forms(xb, z, p)
    Hz, Hp = o.hessian_apply(xb, z), o.hessian_apply(xb, p)
    ref0 = np.array([np.sum(z * Hz), np.sum(z * Hp), np.sum(p * Hp)])
    np.testing.assert_allclose(f0, ref0, rtol=1e-12, atol=1e-12 * np.abs(ref0).max())
    f1 = o.hess_forms(xb, z, p, xc)
    up = o.updates()
    assert len(up["dS"]) > 0 and np.all(up["dS"] > 0)
    C = o.contacts(xc)
    verts = {(int(t), int(a), int(b)): v for t, (a, b), v in zip(C["type"], C["ids"], C["verts"])}
    add = np.zeros(3)
    for key, u in zip(up["key"], up["u"]):
        v = verts[tuple(int(q) for q in key)]
        nvv = 1 if key[0] == 2 else 4
        zc = z[v[:nvv]].reshape(-1)
        pc = p[v[:nvv]].reshape(-1)
        zu, pu = float(u[:3 * nvv] @ zc), float(u[:3 * nvv] @ pc)
        add += [zu * zu, zu * pu, pu * pu]
    assert np.all(np.abs(add) > 0)
    np.testing.assert_allclose(f1, f0 + add, rtol=1e-10, atol=1e-10 * np.abs(f0).max())
