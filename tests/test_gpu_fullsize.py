"""Parity at the benchmarked size: the 64-sphere pile (46,656 vertices,
196,608 tets, 1,507 subdomain blocks) in the FP32-bulk mode that bench.py
times, against the FP64 oracle, element by element on one synthetic contact
state (the oracle finishes each of these in seconds at this size).

The state: the pile's balls (cube-to-ball meshes whose surface vertices lie
on the sphere and whose faces are chords inside it) with four balls moved
next to a neighbour along x, centres 2r + eps apart, so the two facing axis
vertices are eps apart and every other surface feature of the pair is
farther than dhat (the next ring of vertices is ~2 cm off the axis); the
pile lowered until its lowest vertex is eps above the ground; eps = dhat/2;
then 2e-6 m of noise. The meshes stay separated by about eps by
construction, which the oracle's contact distances confirm.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RADIUS = 0.1


def pile_contact_state(sc, n_pairs=4, eps_frac=0.5):
    x = sc["x0"].copy()
    dhat = sc["params"]["dhat"]
    body = np.asarray(sc["body"])
    nb = int(body.max()) + 1
    cen = np.array([x[body == b].mean(axis=0) for b in range(nb)])
    eps = eps_frac * dhat
    moved, pairs = set(), []
    for a in range(nb):
        if len(pairs) == n_pairs:
            break
        if a in moved:
            continue
        target = cen[a] + np.array([2 * RADIUS + eps, 0.0, 0.0])
        for b in range(nb):
            if b == a or b in moved:
                continue
            others = np.delete(np.arange(nb), [a, b])
            if np.min(np.linalg.norm(cen[others] - target, axis=1)) < 2 * RADIUS + 0.01:
                continue
            x[body == b] += target - cen[b]
            cen[b] = target
            moved |= {a, b}
            pairs.append((a, b))
            break
    x[:, 1] -= x[:, 1].min() - eps
    return x, pairs


@pytest.fixture(scope="module")
def pile():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_19892_b300 import build, ipc, scenes as S
    import oracle as O
    build.build()
    ipc.load()
    sc = S.sphere_pile()
    x, pairs = pile_contact_state(sc)
    assert len(pairs) == 4
    rng = np.random.default_rng(7)
    x = x + 2e-6 * rng.normal(size=x.shape)
    g = ipc.Scene(sc, precision=1)
    o = O.Scene(sc)
    return sc, x, pairs, g, o, rng


def test_fullsize_contact_set(pile):
    sc, x, pairs, g, o, rng = pile
    cg, co = g.contacts(x), o.contacts(x)
    dhat = sc["params"]["dhat"]
    assert {0, 1, 2} <= set(int(t) for t in co["type"])
    assert co["dist"].min() > 0.4 * dhat
    kg = {(int(t), int(a), int(b)): i for i, (t, (a, b)) in enumerate(zip(cg["type"], cg["ids"]))}
    ko = {(int(t), int(a), int(b)): i for i, (t, (a, b)) in enumerate(zip(co["type"], co["ids"]))}
    assert set(kg) == set(ko)
    for key, io in ko.items():
        ig = kg[key]
        assert cg["dist"][ig] == pytest.approx(co["dist"][io], rel=1e-12)
        assert cg["k"][ig] == pytest.approx(co["k"][io], rel=1e-8)
        np.testing.assert_array_equal(cg["verts"][ig], co["verts"][io])


def test_fullsize_energy_gradient(pile):
    sc, x, pairs, g, o, rng = pile
    h = sc["params"]["h"]
    v = 0.3 * rng.normal(size=x.shape)
    xt = x + h * v + h * h * sc["gravity"]
    Eg, gg = g.energy_grad(x, xt)
    Eo, go = o.energy(x, xt), o.gradient(x, xt)
    assert Eg == pytest.approx(Eo, rel=1e-10)
    assert np.linalg.norm(gg - go) <= 1e-5 * np.linalg.norm(go)


def test_fullsize_preconditioner(pile):
    sc, x, pairs, g, o, rng = pile
    grad = rng.normal(size=x.shape)
    zg = g.precond_apply(x, grad)
    zo = o.precond_apply(x, grad)
    assert np.linalg.norm(zg - zo) <= 1e-3 * np.linalg.norm(zo)
    assert float(np.sum(zg * grad)) > 0


def test_fullsize_ccd(pile):
    """Each moved ball pushed 1.5 dhat into its neighbour, every vertex
    jittered by 1e-4 m: per-subdomain and per-body step bounds."""
    sc, x, pairs, g, o, rng = pile
    body = np.asarray(sc["body"])
    p = 1e-4 * rng.normal(size=x.shape)
    for a, b in pairs:
        p[body == b, 0] -= 1.5 * sc["params"]["dhat"]
    ag, _, abg, _ = g.ccd(x, p, per_body=True)
    ao, _, abo, _ = o.ccd(x, p, per_body=True)
    assert ao.min() < 1.0
    np.testing.assert_allclose(ag, ao, rtol=0, atol=1e-6)
    np.testing.assert_allclose(abg, abo, rtol=0, atol=1e-6)


def test_fullsize_woodbury_preconditioner(pile):
    """The Woodbury-patched preconditioner (Eq. 7) of the benchmarked form:
    P_base at the state eps = 0.9 dhat, the contacts of the state eps = 0.4
    dhat (the same pairs, stiffer: dS = k - k_base) patched in per
    subdomain. The oracle rebuilds the level-0 inverses of H_base + U U^T
    instead."""
    sc, x, pairs, g, o, rng = pile
    xb, _ = pile_contact_state(sc, eps_frac=0.9)
    xc, _ = pile_contact_state(sc, eps_frac=0.4)
    kb, kc = o.contacts(xb)["k"], o.contacts(xc)["k"]
    assert len(kb) > 0 and len(kc) >= len(kb) and kc.max() > kb.max()
    grad = rng.normal(size=x.shape)
    zg = g.precond_apply(xb, grad, xc)
    zo = o.precond_apply(xb, grad, xc)
    assert np.linalg.norm(zg - zo) <= 1e-3 * np.linalg.norm(zo)
    assert float(np.sum(zg * grad)) > 0


def test_fullsize_forms(pile):
    """The three quadratic forms of H~ (Eq. 6) at full size in the FP32 bulk.
    zHz and pHp are sums of non-negative per-element terms: relative 2e-5.
    For zHp, sum_t |z_t H_t p_t| <= sqrt(zHz pHp) (Cauchy-Schwarz per element
    and over elements) bounds the summed magnitudes, so the FP32 rounding of
    the sum is within 2e-5 of that product."""
    sc, x, pairs, g, o, rng = pile
    xb, _ = pile_contact_state(sc, eps_frac=0.9)
    xc, _ = pile_contact_state(sc, eps_frac=0.4)
    z, p = rng.normal(size=(2,) + x.shape)
    for cur in (None, xc):
        fg = g.hess_forms(xb, z, p, cur)
        fo = o.hess_forms(xb, z, p, cur)
        assert fg[0] == pytest.approx(fo[0], rel=2e-5)
        assert fg[2] == pytest.approx(fo[2], rel=2e-5)
        assert abs(fg[1] - fo[1]) <= 2e-5 * np.sqrt(fo[0] * fo[2])
