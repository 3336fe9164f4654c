"""Serving (ipc_server_*): requests of several scenes run concurrently give
the same result as each scene stepped alone, and they overlap in time."""
import time

import numpy as np
import pytest

from paper_2604_19892_b300 import scenes as S

pytestmark = pytest.mark.gpu


def _bbox(x):
    return float(np.linalg.norm(x.max(0) - x.min(0)))


def _mix_vs_alone(sizes, steps):
    import torch
    from paper_2604_19892_b300 import ipc

    torch.cuda.set_device(0)
    scs = [S.mixed_scene(nv, seed) for nv, seed in sizes]
    scenes = [ipc.Scene(sc, precision=ipc.IPC_PREC_FP32, use_torch_allocator=False) for sc in scs]
    for g, sc in zip(scenes, scs):  # first-call setup outside the timings
        g.set_state(sc["x0"], sc["v0"])
        g.step(1)
    alone, alone_s = [], []
    for g, sc in zip(scenes, scs):
        g.set_state(sc["x0"], sc["v0"])
        t0 = time.perf_counter()
        st = g.step(steps)
        alone_s.append(time.perf_counter() - t0)
        assert st["converged"]
        alone.append(g.positions())
    for g, sc in zip(scenes, scs):
        g.set_state(sc["x0"], sc["v0"])
    srv = ipc.Server(slots=4)
    t0 = time.perf_counter()
    tickets = [srv.submit(g, steps) for g in scenes]
    res = [srv.wait(t) for t in tickets]
    wall = time.perf_counter() - t0
    srv.close()
    for g, sc, xa, r in zip(scenes, scs, alone, res):
        assert r["converged"] and r["steps"] == steps
        err = float(np.abs(g.positions() - xa).max()) / _bbox(sc["x0"])
        assert err <= 1e-6, err
    return wall, alone_s


def test_server_mix_matches_alone_small():
    # scenes of 800-12k vertices: each result as alone (their steps are
    # bound by host launches, so no speed-up is asserted)
    _mix_vs_alone(((800, 11), (3000, 12), (12000, 13), (1500, 14)), 2)


def test_server_mix_overlaps():
    # scenes of 5k-20k vertices: each result as alone, and the requests
    # overlap on the device: the mix takes less than the same requests run
    # one after another
    wall, alone_s = _mix_vs_alone(((20000, 31), (20000, 32), (10000, 33), (5000, 34)), 3)
    assert wall < 0.9 * sum(alone_s), (wall, alone_s)


def test_server_orders_requests_of_one_scene():
    import torch
    from paper_2604_19892_b300 import ipc

    torch.cuda.set_device(0)
    sc = S.mixed_scene(1000, 21)
    g = ipc.Scene(sc, precision=ipc.IPC_PREC_FP32, use_torch_allocator=False)
    g.set_state(sc["x0"], sc["v0"])
    g.step(3)
    x3 = g.positions()
    g.set_state(sc["x0"], sc["v0"])
    srv = ipc.Server(slots=3)
    ts = [srv.submit(g, 1) for _ in range(3)]  # must run one after another, in order
    for t in ts:
        assert srv.wait(t)["converged"]
    srv.close()
    assert float(np.abs(g.positions() - x3).max()) / _bbox(sc["x0"]) <= 1e-6


def test_numeric_failure_of_one_scene_leaves_the_others_as_alone():
    # one served scene gets velocities so large that its inertia energy
    # overflows: its request fails with IPC_ERR_NUMERIC, the requests of the
    # other scenes running beside it give their solo results, and the failed
    # scene steps normally again once its state is reset
    import torch
    from paper_2604_19892_b300 import ipc

    torch.cuda.set_device(0)
    scs = [S.mixed_scene(nv, seed) for nv, seed in ((1200, 41), (2500, 42), (1800, 43))]
    scenes = [ipc.Scene(sc, precision=ipc.IPC_PREC_FP32, use_torch_allocator=False) for sc in scs]
    alone = []
    for g, sc in zip(scenes, scs):
        g.set_state(sc["x0"], sc["v0"])
        assert g.step(2)["converged"]
        alone.append(g.positions())
        g.set_state(sc["x0"], sc["v0"])
    bad = 1
    scenes[bad].set_state(scs[bad]["x0"], np.full_like(scs[bad]["x0"], 1e200))
    srv = ipc.Server(slots=3)
    tickets = [srv.submit(g, 2) for g in scenes]
    for i, (t, g, sc, xa) in enumerate(zip(tickets, scenes, scs, alone)):
        if i == bad:
            with pytest.raises(ipc.IPCError) as e:
                srv.wait(t)
            assert e.value.code == ipc.IPC_ERR_NUMERIC
            assert np.array_equal(g.positions(), sc["x0"])  # x untouched
            continue
        assert srv.wait(t)["converged"]
        assert float(np.abs(g.positions() - xa).max()) / _bbox(sc["x0"]) <= 1e-6
    g, sc = scenes[bad], scs[bad]
    g.set_state(sc["x0"], sc["v0"])
    assert srv.wait(srv.submit(g, 2))["converged"]
    srv.close()
    assert float(np.abs(g.positions() - alone[bad]).max()) / _bbox(sc["x0"]) <= 1e-6


def test_scenes_are_created_and_destroyed_while_others_are_served():
    # scene creation and destruction wait on their own streams only: a host
    # thread builds and releases scenes while the server steps others (whose
    # first repeated launch sequences are captured as CUDA graphs meanwhile),
    # and every request and every creation succeeds
    import threading
    import torch
    from paper_2604_19892_b300 import ipc

    torch.cuda.set_device(0)
    scs = [S.mixed_scene(nv, seed) for nv, seed in ((3000, 61), (5000, 62), (2000, 63), (4000, 64))]
    scenes = [ipc.Scene(sc, precision=ipc.IPC_PREC_FP32, use_torch_allocator=False) for sc in scs]
    errors, made = [], []

    def builder():
        try:
            torch.cuda.set_device(0)
            for seed in range(71, 77):
                g = ipc.Scene(S.mixed_scene(6000, seed), precision=ipc.IPC_PREC_FP32, use_torch_allocator=False)
                made.append(g.nv)
                g.close()
        except Exception as e:  # reported below, in the test's thread
            errors.append(e)

    srv = ipc.Server(slots=4)
    th = threading.Thread(target=builder)
    th.start()
    tickets = [srv.submit(g, 4) for g in scenes]
    res = [srv.wait(t) for t in tickets]
    th.join()
    srv.close()
    assert not errors, errors
    assert len(made) == 6
    assert all(r["converged"] for r in res)
    for g in scenes:
        g.close()
