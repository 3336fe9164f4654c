"""Timestep-level GPU checks through the C ABI: checkpoint / resume, the FP32
bulk form against the FP64 oracle step by step, and the error path of the
bounded bulk-copy waits (made to run out by a zero poll budget, which needs
no fault: each CTA still drains its copy before it exits)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_19892_b300 import build, ipc
    build.build()
    ipc.load()
    torch.cuda.set_device(0)
    return ipc


def test_checkpoint_resume_equals_an_uninterrupted_run(lib):
    """N timesteps in one go equal k timesteps, a checkpoint (positions and
    velocities queried to the host), a fresh scene resumed from it by
    ipc_set_state, and N - k more timesteps: within 1e-6 of the bounding-box
    diagonal on a scene whose steps have one minimiser each (tol 1e-7)."""
    from paper_2604_19892_b300 import scenes as S
    sc = S.ground_drop(n=3, gap=0.003, drop_speed=0.5)
    prm = {"tol": 1e-7}
    N, k = 4, 2
    a = lib.Scene(sc, params=prm)
    sa = a.step(N)
    assert sa["converged"] == 1
    b = lib.Scene(sc, params=prm)
    b.step(k)
    x, v = b.positions(), b.velocities()
    b.close()
    c = lib.Scene(sc, params=prm)
    c.set_state(x, v)
    sc_ = c.step(N - k)
    assert sc_["converged"] == 1
    bbox = a.bbox_diag()
    assert np.abs(a.positions() - c.positions()).max() / bbox <= 1e-6
    assert np.abs(a.velocities() - c.velocities()).max() * sc["params"]["h"] / bbox <= 1e-6
    assert sa["n_contacts"] > 0


def test_fp32_bulk_steps_follow_the_fp64_oracle(lib):
    """The FP32 bulk form, fed the oracle's state each timestep, converges to
    the oracle's minimiser within 1e-5 of the bounding-box diagonal through an
    impact (tol 1e-5 for the FP32 form, 1e-8 for the oracle): FP32 gradients
    carry relative rounding of about 1e-7, so its converged iterate is known
    only to about tol h bbox plus that rounding mapped through P."""
    import oracle as O
    from paper_2604_19892_b300 import scenes as S
    sc = S.ground_drop(n=3, gap=0.003, drop_speed=0.5)
    o = O.Scene(sc, params={"tol": 1e-8})
    g = lib.Scene(sc, precision=lib.IPC_PREC_FP32, params={"tol": 1e-5})
    x, v = sc["x0"].copy(), sc["v0"].copy()
    errs = []
    for step in range(4):
        g.set_state(x, v)
        st = g.step(1)
        assert st["converged"] == 1, (step, st)
        xo, vo, so = o.step(x, v)
        assert so["converged"] == 1
        errs.append(float(np.abs(g.positions() - xo).max() / o.bbox_diag()))
        x, v = xo, vo
    assert max(errs) <= 1e-5, errs


def test_bf16_factor_steps_follow_the_fp64_oracle(lib):
    """With BF16 block factors the preconditioner changes, not the minimiser:
    fed the oracle's state each timestep, the BF16 form converges (tol 1e-5)
    to the oracle's positions within 1e-5 of the bounding-box diagonal."""
    import oracle as O
    from paper_2604_19892_b300 import scenes as S
    sc = S.ground_drop(n=3, gap=0.003, drop_speed=0.5)
    o = O.Scene(sc, params={"tol": 1e-8})
    g = lib.Scene(sc, precision=lib.IPC_PREC_BF16_MAS, params={"tol": 1e-5})
    x, v = sc["x0"].copy(), sc["v0"].copy()
    errs = []
    for step in range(4):
        g.set_state(x, v)
        st = g.step(1)
        assert st["converged"] == 1, (step, st)
        xo, vo, so = o.step(x, v)
        errs.append(float(np.abs(g.positions() - xo).max() / o.bbox_diag()))
        x, v = xo, vo
    assert max(errs) <= 1e-5, errs


def test_autotuned_apply_configuration_does_not_change_results(lib):
    """The autotuner picks the persistent apply's CTAs per SM among the
    candidates its shared memory allows; the preconditioner is the same
    whatever the choice (each block's arithmetic does not depend on the
    grid), here on a scene large enough to be tuned (46,656 vertices): every
    forced candidate gives the tuned result to the rounding of the restart's
    atomically summed assembly."""
    from paper_2604_19892_b300 import scenes as S
    sc = S.sphere_pile()
    rng = np.random.default_rng(4)
    grad = rng.normal(size=sc["x0"].shape)
    for prec, cands in ((lib.IPC_PREC_FP32, (2, 3, 4, 5)), (lib.IPC_PREC_BF16_MAS, (4, 6, 8, 10))):
        g = lib.Scene(sc, precision=prec)
        assert g.apply_ctas() in cands
        z0 = g.precond_apply(sc["x0"], grad)
        g.close()
        for c in cands:
            h = lib.Scene(sc, precision=prec, params={"apply_ctas": c})
            assert h.apply_ctas() == c
            z = h.precond_apply(sc["x0"], grad)
            assert np.linalg.norm(z - z0) <= 1e-5 * np.linalg.norm(z0), (prec, c)
            h.close()


def test_exhausted_copy_wait_reports_timeout_and_leaves_the_context_usable(lib):
    """wait_polls = 0: every bounded wait of the block-apply CTAs reports a
    timeout without polling; ipc_step stops with IPC_ERR_TIMEOUT before z is
    used. A second scene with the default budget then steps normally in the
    same process (the CTAs drained their copies, nothing faulted)."""
    from paper_2604_19892_b300 import scenes as S
    sc = S.ground_drop(n=3, gap=0.003, drop_speed=0.5)
    bad = lib.Scene(sc, params={"wait_polls": 0})
    with pytest.raises(lib.IPCError) as e:
        bad.step(1)
    assert e.value.code == lib.IPC_ERR_TIMEOUT and "bulk copy" in str(e.value)
    good = lib.Scene(sc)
    st = good.step(2)
    assert st["converged"] == 1


def test_allocation_failure_is_reported_and_everything_released(lib):
    # a caller allocator that refuses its 30th request: scene creation fails
    # with IPC_ERR_OOM, every block it was given is handed back, and a scene
    # created afterwards steps normally
    import torch
    from paper_2604_19892_b300 import scenes as S

    ipc = lib
    sc = S.mixed_scene(1500, 51)
    live, calls = {}, [0]

    def _alloc(n, ctx):
        calls[0] += 1
        if calls[0] >= 30:
            return None
        p = torch.cuda.caching_allocator_alloc(int(n), device=0)
        live[p] = int(n)
        return p

    def _free(p, ctx):
        assert live.pop(p, None) is not None
        torch.cuda.caching_allocator_delete(p)

    fns = ipc.AllocFns(ipc.ALLOC_FN(_alloc), ipc.FREE_FN(_free), None)
    with pytest.raises(ipc.IPCError) as e:
        ipc.Scene(sc, precision=ipc.IPC_PREC_FP32, alloc_fns=fns)
    assert e.value.code == ipc.IPC_ERR_OOM
    assert calls[0] == 30 and not live
    g = ipc.Scene(sc, precision=ipc.IPC_PREC_FP32)
    assert g.step(1)["converged"]
    g.close()


def test_non_finite_state_is_refused_and_the_state_kept(lib):
    # NaN or Inf in positions or velocities, from host or device buffers, is
    # refused before any kernel uses it; the scene keeps its state
    import torch
    from paper_2604_19892_b300 import scenes as S

    ipc = lib
    sc = S.mixed_scene(1200, 52)
    g = ipc.Scene(sc, precision=ipc.IPC_PREC_FP32)
    g.set_state(sc["x0"], sc["v0"])
    assert g.step(1)["converged"]
    x1, v1 = g.positions(), g.velocities()
    for on_device in (False, True):
        for which, bad in (("x", np.nan), ("v", np.inf)):
            x, v = x1.copy(), v1.copy()
            (x if which == "x" else v)[7, 1] = bad
            if on_device:
                x, v = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
            with pytest.raises(ipc.IPCError) as e:
                g.set_state(x, v)
            assert e.value.code == ipc.IPC_ERR_INVALID
            assert np.array_equal(g.positions(), x1) and np.array_equal(g.velocities(), v1)
    assert g.step(1)["converged"]
    g.close()


def test_fma_peak_measurement_is_plausible(lib):
    # the SIMT FMA throughput the inversion's roofline is read against: both
    # pipes measured, FP32 far above FP64 on this part and below the unit
    # count bound (lanes x 2 flops x the maximum clock)
    import torch
    ipc = lib
    f32 = ipc.fma_peak_tflops(ipc.IPC_PREC_FP32, 5.0)
    f64 = ipc.fma_peak_tflops(ipc.IPC_PREC_FP64, 5.0)
    props = torch.cuda.get_device_properties(0)
    bound = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    assert 0.25 * bound < f32 <= 1.05 * bound, (f32, bound)
    assert 0.0 < f64 < f32 / 10, (f64, f32)


def test_first_trial_takes_the_body_steps_after_a_subdomain_fallback(lib):
    """Per-subdomain steps on thin features (Sec. 4.4): two small spiky balls
    whose 64-layer spikes run through several 32-vertex subdomains. In
    timestep 1 the per-subdomain verification of the straddling pairs falls
    back to the uniform step on some iterations while the per-body one
    verifies; the first energy-check trial is then the per-body step, on both
    sides. From the oracle's state after timestep 0, the GPU's FP64 form
    follows the oracle iteration by iteration up to and including the first
    such iteration."""
    import oracle as O
    from paper_2604_19892_b300 import scenes as S

    ipc = lib
    sc = S.spiky_balls(n_balls=2, cells=4, n_spikes=8, layers=64)
    g = ipc.Scene(sc, precision=ipc.IPC_PREC_FP64)
    o = O.Scene(sc)
    x, v, _ = o.step(sc["x0"].copy(), sc["v0"].copy())
    g.set_state(x, v)
    g.step(1)
    o.step(x, v)
    tg, to = g.trace(), o.trace()
    k = next(i for i, r in enumerate(to) if r["ccd_passes"] < 0 and r["ccd_passes_body"] >= 0)
    assert len(tg) > k
    for i in range(k + 1):
        rg, ro = tg[i], to[i]
        assert rg["restart"] == ro["restart"], i
        assert rg["ccd_passes"] == ro["ccd_passes"] and rg["ccd_passes_body"] == ro["ccd_passes_body"], i
        assert rg["ls_halvings"] == ro["ls_halvings"], i
        assert rg["energy_after"] == pytest.approx(ro["energy_after"], rel=1e-8), i
    g.close()
