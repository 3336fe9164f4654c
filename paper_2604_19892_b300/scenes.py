"""Seeded synthetic scene generators (inputs only).

This module builds tetrahedral meshes, materials and initial states shaped
like the paper's workloads (Table 1 scenes are not available, so synthetic
stand-ins are used).  It holds none of the solver's arithmetic: no energy,
no distance, no preconditioner.  Both the CUDA path and the FP64 oracle
consume what it returns.

Every scene is a plain dict of numpy arrays:

    x_rest  (nV,3) float64   rest positions (also the initial positions
                             unless x0 is given separately)
    x0      (nV,3) float64   initial positions
    v0      (nV,3) float64   initial velocities
    tets    (nT,4) int32     vertex indices, positively oriented
    E, nu, rho (nT,) float64 per-tet Young's modulus, Poisson ratio, density
    body    (nV,)  int32     body index of each vertex
    gravity (3,)   float64
    ground  (4,)   float64   plane normal (3) and offset; ground[3] = nan
                             means "no ground"
    params  dict             timestep, barrier width etc. (see default_params)
"""
from __future__ import annotations

import math
import numpy as np

# ----------------------------------------------------------------------------
# Elementary meshes
# ----------------------------------------------------------------------------

_CORNERS = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0],
                     [0, 0, 1], [1, 0, 1], [0, 1, 1], [1, 1, 1]], dtype=np.int64)

# Five-tet split of a hex cell; the odd-parity cells use the mirrored split so
# that neighbouring cells share face diagonals.
_FIVE_EVEN = [(0, 1, 2, 4), (3, 2, 1, 7), (5, 4, 7, 1), (6, 7, 4, 2), (1, 2, 4, 7)]
_FIVE_ODD = [(1, 0, 3, 5), (2, 3, 0, 6), (4, 5, 6, 0), (7, 6, 5, 3), (0, 3, 5, 6)]

# Six-tet (Kuhn) split along the 0-7 diagonal; conforming for every cell.
_SIX = [(0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7)]


def _orient(x, tets):
    """Flip tets with negative signed volume so every tet is positive."""
    a = x[tets[:, 1]] - x[tets[:, 0]]
    b = x[tets[:, 2]] - x[tets[:, 0]]
    c = x[tets[:, 3]] - x[tets[:, 0]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c))
    neg = vol < 0
    t = tets.copy()
    t[neg, 2], t[neg, 3] = tets[neg, 3], tets[neg, 2]
    return t


def hex_grid(nx, ny, nz, split=5):
    """Structured grid of nx*ny*nz unit cells split into tets.

    Returns (x, tets) with x on the integer lattice [0,nx]x[0,ny]x[0,nz].
    """
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    x = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    corner = np.stack([((ci + c[0]) * (ny + 1) + (cj + c[1])) * (nz + 1) + (ck + c[2])
                       for c in _CORNERS], axis=1)
    if split == 5:
        even = ((ci + cj + ck) % 2 == 0)[:, None, None]
        pe = corner[:, np.asarray(_FIVE_EVEN)]
        po = corner[:, np.asarray(_FIVE_ODD)]
        tets = np.where(even, pe, po).reshape(-1, 4)
    else:
        tets = corner[:, np.asarray(_SIX)].reshape(-1, 4)
    tets = tets.astype(np.int64)
    return x, _orient(x, tets).astype(np.int32)


def box_mesh(n, edge, origin, split=5, dims=None):
    """Cube (or box with cell counts dims) of cell size `edge` at `origin`."""
    nx, ny, nz = dims if dims is not None else (n, n, n)
    x, t = hex_grid(nx, ny, nz, split)
    return x * edge + np.asarray(origin, dtype=np.float64), t


def ball_mesh(n, radius, center, split=6):
    """Cube-to-ball mapped grid of n^3 cells (n even) of the given radius."""
    x, t = hex_grid(n, n, n, split)
    q = x / n * 2.0 - 1.0  # [-1,1]^3
    a, b, c = q[:, 0], q[:, 1], q[:, 2]
    a2, b2, c2 = a * a, b * b, c * c
    y = np.stack([
        a * np.sqrt(np.maximum(0.0, 1 - b2 / 2 - c2 / 2 + b2 * c2 / 3)),
        b * np.sqrt(np.maximum(0.0, 1 - c2 / 2 - a2 / 2 + c2 * a2 / 3)),
        c * np.sqrt(np.maximum(0.0, 1 - a2 / 2 - b2 / 2 + a2 * b2 / 3)),
    ], axis=1)
    y = y * radius + np.asarray(center, dtype=np.float64)
    return y, _orient(y, t.astype(np.int64)).astype(np.int32)


def torus_mesh(n_around, n_tube, R, r, center, axis=2, split=5):
    """Torus ring with square cross-section (side 2r) swept around a circle.

    A hex grid of n_around x n_tube x n_tube cells is bent around the axis;
    the seam is stitched so the ring is closed.
    """
    x, t = hex_grid(n_around, n_tube, n_tube, split)
    i, j, k = x[:, 0], x[:, 1], x[:, 2]
    theta = 2 * math.pi * i / n_around
    rad = R + (j / n_tube * 2 - 1) * r
    hgt = (k / n_tube * 2 - 1) * r
    pts = np.stack([rad * np.cos(theta), rad * np.sin(theta), hgt], axis=1)
    # stitch the seam: vertices with i == n_around coincide with i == 0
    nyz = (n_tube + 1) * (n_tube + 1)
    remap = np.arange(x.shape[0])
    seam = np.where(i == n_around)[0]
    remap[seam] = seam - n_around * nyz
    t = remap[t]
    keep = np.unique(t)
    newid = -np.ones(x.shape[0], dtype=np.int64)
    newid[keep] = np.arange(keep.size)
    t = newid[t]
    pts = pts[keep]
    if axis == 0:
        pts = pts[:, [2, 0, 1]]
    elif axis == 1:
        pts = pts[:, [0, 2, 1]]
    pts = pts + np.asarray(center, dtype=np.float64)
    return pts, _orient(pts, t).astype(np.int32)


# ----------------------------------------------------------------------------
# Scene assembly
# ----------------------------------------------------------------------------

def default_params(bbox_diag, h, E_max):
    """Solver parameters; the barrier width is 1e-3 of the bbox diagonal."""
    dhat = 1e-3 * bbox_diag
    return {
        "h": h,
        "dhat": dhat,
        "kappa": 10.0 * h * h * E_max * dhat,
        "tol": 1e-3,
        "iter_max": 10000,
        "delta": 0.3,
        "eps_rot_deg": 25.0,
        "K": 8,
        "levels_max": 6,
        "ls_max": 20,
        "ccd_shrink": 0.1,
        "eps_sing": 1e-12,
        "eps_abs": 1e-300,
    }


def _assemble(bodies, gravity=(0.0, -9.8, 0.0), ground=(0.0, 1.0, 0.0, 0.0)):
    xs, ts, Es, nus, rhos, body = [], [], [], [], [], []
    off = 0
    for b, (x, t, E, nu, rho) in enumerate(bodies):
        xs.append(x)
        ts.append(t + off)
        Es.append(np.full(t.shape[0], E))
        nus.append(np.full(t.shape[0], nu))
        rhos.append(np.full(t.shape[0], rho))
        body.append(np.full(x.shape[0], b, dtype=np.int32))
        off += x.shape[0]
    x = np.concatenate(xs).astype(np.float64)
    return {
        "x_rest": x.copy(),
        "x0": x.copy(),
        "v0": np.zeros_like(x),
        "tets": np.concatenate(ts).astype(np.int32),
        "E": np.concatenate(Es).astype(np.float64),
        "nu": np.concatenate(nus).astype(np.float64),
        "rho": np.concatenate(rhos).astype(np.float64),
        "body": np.concatenate(body),
        "gravity": np.asarray(gravity, dtype=np.float64),
        "ground": np.asarray(ground, dtype=np.float64),
    }


def bbox_diag(x):
    return float(np.linalg.norm(x.max(axis=0) - x.min(axis=0)))


def two_cubes(n=8, edge_len=0.1, gap=0.05, jitter=1e-4, seed=0, h=1.0 / 30):
    """Two n^3-cell cubes, 5 tets/cell, stacked `gap` apart above the ground.

    The lower cube sits `gap` above the plane y=0.  SNH E=1e5, nu=0.4,
    rho=1000.  Every vertex gets U(-jitter, jitter) noise per coordinate.
    """
    rng = np.random.default_rng(seed)
    c = edge_len / n
    lower = box_mesh(n, c, (0.0, gap, 0.0))
    upper = box_mesh(n, c, (0.0, gap + edge_len + gap, 0.0))
    sc = _assemble([(lower[0], lower[1], 1e5, 0.4, 1000.0),
                    (upper[0], upper[1], 1e5, 0.4, 1000.0)])
    sc["x_rest"] += rng.uniform(-jitter, jitter, size=sc["x_rest"].shape)
    sc["x0"] = sc["x_rest"].copy()
    sc["params"] = default_params(bbox_diag(sc["x0"]), h, 1e5)
    sc["name"] = f"two_cubes_{n}"
    return sc


def _rsa_centres(rng, count, radius, lo, hi, min_gap, max_tries=200000):
    """Random sequential placement of non-overlapping spheres in a box."""
    pts = np.zeros((0, 3))
    tries = 0
    while pts.shape[0] < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place spheres")
        c = rng.uniform(lo + radius, hi - radius)
        if pts.shape[0] == 0 or np.min(np.linalg.norm(pts - c, axis=1)) > 2 * radius + min_gap:
            pts = np.vstack([pts, c])
    return pts


def sphere_pile(n_balls=64, radius=0.1, cells=8, seed=1, h=1.0 / 60, nu=0.4, rho=1000.0, box=(1.0, 1.0, 1.0)):
    """Balls of the given radius at random non-overlapping centres in a box
    (1 m by default).

    Each ball is a cells^3 cube-to-ball mapped grid with 6 tets per cell; E is
    drawn log-uniform in [1e4, 1e6] per body.  The box spans y in
    [0.05, 0.05 + box[1]] above the ground plane y=0.
    """
    rng = np.random.default_rng(seed)
    lo = np.array([0.0, 0.05, 0.0])
    hi = np.array([box[0], 0.05 + box[1], box[2]])
    centres = _rsa_centres(rng, n_balls, radius, lo, hi, 0.01)
    Es = np.exp(rng.uniform(math.log(1e4), math.log(1e6), size=n_balls))
    bodies = []
    for b in range(n_balls):
        x, t = ball_mesh(cells, radius, centres[b])
        bodies.append((x, t, float(Es[b]), nu, rho))
    sc = _assemble(bodies)
    sc["params"] = default_params(bbox_diag(sc["x0"]), h, float(Es.max()))
    sc["name"] = f"sphere_pile_{n_balls}"
    return sc


def mixed_scene(target_nv, seed, h=1.0 / 60):
    """1-8 bodies (cube, ball, rod of aspect U(2,8)) totalling ~target_nv verts.

    Bodies are stacked in a loose column above the ground with small gaps so
    they collide within a few steps.
    """
    rng = np.random.default_rng(seed)
    nb = int(rng.integers(1, 9))
    per = max(target_nv / nb, 64.0)
    bodies = []
    y = 0.02
    Emax = 0.0
    for b in range(nb):
        kind = rng.integers(0, 3)
        E = float(np.exp(rng.uniform(math.log(1e4), math.log(1e6))))
        Emax = max(Emax, E)
        xz = rng.uniform(-0.03, 0.03, size=2)
        if kind == 0:
            n = max(2, int(round(per ** (1 / 3))) - 1)
            size = 0.1
            x, t = box_mesh(n, size / n, (xz[0] - size / 2, y, xz[1] - size / 2))
            y += size + 0.02
        elif kind == 1:
            n = max(2, 2 * (int(round(per ** (1 / 3))) // 2))
            r = 0.06
            x, t = ball_mesh(n, r, (xz[0], y + r, xz[1]))
            y += 2 * r + 0.02
        else:
            a = float(rng.uniform(2, 8))
            n = max(2, int(round((per / a) ** (1 / 3))) - 1)
            m = max(2, int(round(a * n)))
            size = 0.04
            c = size / n
            x, t = box_mesh(None, c, (xz[0] - m * c / 2, y, xz[1] - size / 2), dims=(m, n, n))
            y += size + 0.02
        bodies.append((x, t, E, 0.4, 1000.0))
    sc = _assemble(bodies)
    sc["x_rest"] += rng.uniform(-1e-5, 1e-5, size=sc["x_rest"].shape)
    # the jitter can flip a sliver tet of the mapped balls: orient again
    sc["tets"] = _orient(sc["x_rest"], sc["tets"].astype(np.int64)).astype(np.int32)
    sc["x0"] = sc["x_rest"].copy()
    sc["params"] = default_params(bbox_diag(sc["x0"]), h, Emax)
    sc["name"] = f"mixed_{target_nv}_{seed}"
    return sc


def batched_scenes(n_scenes=256, nv_lo=500, nv_hi=20000, seed=2):
    """Scene sizes drawn log-uniform in [nv_lo, nv_hi]."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(nv_lo), math.log(nv_hi), size=n_scenes))
    return [mixed_scene(int(s), seed * 100003 + i) for i, s in enumerate(sizes)]


def torus_stack(target_nv, seed, h=1.0 / 60, R=0.1, r=0.015, n_around=96, n_tube=7):
    """Interlocked chain of torus rings (square tube cross-section of side
    2r, ring radius R) along x: rings alternate between flat (in the xz
    plane) and upright (in the xy plane), centres R apart at one height, so
    that every ring passes through the holes of its two neighbours; enough
    rings for about target_nv vertices (6,144 per ring). The chain hangs
    2 cm above the ground; dhat is 1e-3 of one ring's diagonal."""
    rng = np.random.default_rng(seed)
    per_ring = n_around * (n_tube + 1) ** 2
    n_rings = max(2, int(round(target_nv / per_ring)))
    yc = R + r + 0.02
    bodies = []
    for q in range(n_rings):
        x, t = torus_mesh(n_around, n_tube, R, r, (0.0, 0.0, 0.0), axis=2)  # ring in the xy plane
        if q % 2 == 0:
            x = x[:, [0, 2, 1]]  # flat: into the xz plane
        x = x + np.array([q * R, yc, 0.0]) + rng.uniform(-1e-4, 1e-4, size=3)
        # swapping two axes (and the bend) can reverse the tets' orientation
        t = _orient(x, t.astype(np.int64)).astype(np.int32)
        bodies.append((x, t, 1e5, 0.4, 1000.0))
    sc = _assemble(bodies)
    # dhat from one ring's size: 1e-3 of the whole chain's diagonal (metres
    # long) would exceed the rings' own cells and put every ring in contact
    # with itself
    ring = bodies[0][0]
    sc["params"] = default_params(bbox_diag(ring), h, 1e5)
    sc["name"] = f"torus_stack_{n_rings}"
    return sc


def free_fall_block(n=2, edge_len=0.1, h=1.0 / 30):
    """A single block far above the ground (no contact within one step)."""
    x, t = box_mesh(n, edge_len / n, (0.0, 10.0, 0.0))
    sc = _assemble([(x, t, 1e5, 0.4, 1000.0)])
    sc["params"] = default_params(bbox_diag(sc["x0"]), h, 1e5)
    sc["name"] = "free_fall"
    return sc


def ground_drop(n=3, edge_len=0.1, gap=0.003, drop_speed=0.5, jitter=1e-4, seed=0, h=1.0 / 30):
    """One jittered n^3-cell cube `gap` above the ground plane moving down at
    `drop_speed`: plane contacts only, whose barrier is convex in x, so each
    step's incremental potential has a single minimiser near rest."""
    rng = np.random.default_rng(seed)
    x, t = box_mesh(n, edge_len / n, (0.0, gap, 0.0))
    sc = _assemble([(x, t, 1e5, 0.4, 1000.0)])
    sc["x_rest"] += rng.uniform(-jitter, jitter, size=sc["x_rest"].shape)
    sc["x0"] = sc["x_rest"].copy()
    sc["v0"][:, 1] = -drop_speed
    sc["params"] = default_params(bbox_diag(sc["x0"]), h, 1e5)
    sc["name"] = f"ground_drop_{n}"
    return sc


def small_cubes(n=2, gap=0.01, jitter=1e-4, seed=0, h=1.0 / 30, edge_len=0.1, drop_speed=0.0):
    """Tiny two-cube scene for brute-force invariant checks."""
    sc = two_cubes(n=n, edge_len=edge_len, gap=gap, jitter=jitter, seed=seed, h=h)
    sc["v0"][:, 1] = -drop_speed
    sc["name"] = f"small_cubes_{n}"
    return sc


def _prism_tets(p):
    """Three positively ordered tets of the prism with bottom (p0, p1, p2) and
    top (p3, p4, p5) (p3 above p0, ...), each quad face split along the
    diagonal from its smallest vertex id, so neighbouring prisms that share a
    quad face split it the same way (the usual id-based rule for conforming
    prism meshes)."""
    p = list(p)
    # rotate / flip so that the smallest id is p0
    k = int(np.argmin(p))
    rot = [[0, 1, 2, 3, 4, 5], [1, 2, 0, 4, 5, 3], [2, 0, 1, 5, 3, 4],
           [3, 5, 4, 0, 2, 1], [4, 3, 5, 1, 0, 2], [5, 4, 3, 2, 1, 0]][k]
    q = [p[i] for i in rot]
    if min(q[1], q[5]) < min(q[2], q[4]):
        return [(q[0], q[1], q[2], q[5]), (q[0], q[1], q[5], q[4]), (q[0], q[4], q[5], q[3])]
    return [(q[0], q[1], q[2], q[4]), (q[0], q[4], q[2], q[5]), (q[0], q[4], q[5], q[3])]


def spiky_ball_mesh(cells, radius, center, n_spikes=200, layers=132, spike_len=0.5, tip=0.15, seed=0):
    """A cube-to-ball mapped grid (cells^3, 6 tets per cell) with n_spikes
    conical spikes grown from surface quads: each spike extrudes the two
    boundary triangles of one surface quad outward in `layers` layers of
    prisms (3 tets each), tapering linearly to `tip` of its base size, to a
    length of spike_len * radius. The base triangles are the ball's own, so
    the mesh is conforming. Quads are picked at random without repetition,
    avoiding quads that share a vertex with an earlier pick."""
    x, t = ball_mesh(cells, radius, center)
    rng = np.random.default_rng(seed)
    # boundary triangles of the ball (faces used once)
    faces = np.concatenate([t[:, [0, 1, 2]], t[:, [0, 1, 3]], t[:, [0, 2, 3]], t[:, [1, 2, 3]]])
    key = np.sort(faces, axis=1)
    uniq, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    bnd = uniq[cnt == 1]
    # pair boundary triangles into quads: two triangles sharing an edge whose
    # four vertices lie on one cell face (the face diagonal)
    from collections import defaultdict
    edge_tris = defaultdict(list)
    for i, tr in enumerate(bnd):
        for a, b in ((tr[0], tr[1]), (tr[0], tr[2]), (tr[1], tr[2])):
            edge_tris[(min(a, b), max(a, b))].append(i)
    # the lattice index of each ball vertex tells which edges are face diagonals
    n1 = cells + 1
    ijk = np.stack(np.unravel_index(np.arange(n1 ** 3), (n1, n1, n1)), axis=1)
    quads = []
    for (a, b), tris in edge_tris.items():
        if len(tris) != 2:
            continue
        if np.count_nonzero(ijk[a] != ijk[b]) != 2:  # not a face diagonal
            continue
        tr0, tr1 = bnd[tris[0]], bnd[tris[1]]
        quads.append((tr0, tr1))
    order = rng.permutation(len(quads))
    used = set()
    picked = []
    for qi in order:
        tr0, tr1 = quads[qi]
        vs = set(tr0.tolist()) | set(tr1.tolist())
        if vs & used:
            continue
        picked.append((tr0, tr1))
        used |= vs
        if len(picked) == n_spikes:
            break
    pts = [x]
    tets = [t]
    nxt = x.shape[0]
    c = np.asarray(center, dtype=np.float64)
    for tr0, tr1 in picked:
        base = np.array(sorted(set(tr0.tolist()) | set(tr1.tolist())))
        bp = x[base]
        mid = bp.mean(axis=0)
        axis = mid - c
        axis /= np.linalg.norm(axis)
        ids = {int(v): int(v) for v in base}
        prev = ids
        for lay in range(1, layers + 1):
            f = lay / layers
            shrink = 1.0 - (1.0 - tip) * f
            layer_pts = mid + shrink * (bp - mid) + axis * (spike_len * radius * f)
            cur = {}
            for j, v in enumerate(base):
                cur[int(v)] = nxt
                nxt += 1
            pts.append(layer_pts)
            for tri in (tr0, tr1):
                pr = [prev[int(v)] for v in tri] + [cur[int(v)] for v in tri]
                tets.append(np.array(_prism_tets(pr), dtype=np.int64))
            prev = cur
    X = np.concatenate(pts)
    T = np.concatenate([np.asarray(q, dtype=np.int64).reshape(-1, 4) for q in tets])
    return X, _orient(X, T).astype(np.int32)


def spiky_balls(n_balls=8, cells=32, radius=0.1, n_spikes=200, layers=132, seed=5, h=1.0 / 30, E=5e4, nu=0.45,
                rho=1000.0):
    """Large-scene stand-in shaped like the paper's teaser (puffer balls):
    spiky balls (a 32^3-cell ball with 200 conical spikes of half its radius,
    about 141k vertices and 355k tets each) in two layers of four, spaced
    5 mm beyond their spike reach, the lower layer 5 mm above the ground;
    E = 5e4 Pa, nu = 0.45, dt = 1/30 s, dhat = 1e-4 of the bounding-box
    diagonal (the paper's value for this scene; the spike layers are 0.4 mm
    thick, so the default 1e-3 would put a spike's own faces within dhat)."""
    rng = np.random.default_rng(seed)
    reach = radius * 1.5
    sp = 2 * reach + 0.005
    bodies = []
    for b in range(n_balls):
        layer, k = divmod(b, 4)
        cx = (k % 2) * sp + rng.uniform(-0.01, 0.01)
        cz = (k // 2) * sp + rng.uniform(-0.01, 0.01)
        cy = 0.005 + reach + layer * (sp + 0.02)
        x, t = spiky_ball_mesh(cells, radius, (cx, cy, cz), n_spikes=n_spikes, layers=layers, seed=seed + b)
        bodies.append((x, t, E, nu, rho))
    sc = _assemble(bodies)
    bb = bbox_diag(sc["x0"])
    sc["params"] = default_params(bb, h, E)
    sc["params"]["dhat"] = 1e-4 * bb
    sc["params"]["kappa"] = 10.0 * h * h * E * sc["params"]["dhat"]
    sc["name"] = f"spiky_balls_{n_balls}"
    return sc
