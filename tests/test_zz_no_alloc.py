"""Allocation-free preconditioner apply (ipc_precond_apply_noalloc).

Some callers cannot allocate device memory during a call: a solver loop that
shares the device with other busy streams (cudaMalloc / cudaFree can
synchronise the whole device) or a process whose device memory belongs to
another allocator. This entry point keeps its scratch in a static device
array and is checked here against the allocating evaluation entry point
ipc_eval_precond: same scene, same P_base, two calls in a row on
caller-owned device tensors. Named to be collected last, so it also runs
after every other GPU test in one session."""
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
    return ipc


@pytest.mark.parametrize("precision,rtol", [(0, 1e-12), (1, 1e-6)])
def test_noalloc_apply_matches_eval_precond(lib, precision, rtol):
    import torch
    from paper_2604_19892_b300 import scenes as S
    sc = S.two_cubes(n=8)                      # 1458 vertices, three levels
    g = lib.Scene(sc, precision=precision)
    assert len(g.levels()) >= 2                # the coarse scratch is used
    rng = np.random.default_rng(11)
    xb = sc["x0"] + 1e-4 * rng.normal(size=sc["x0"].shape)
    dtype = torch.float64 if precision == 0 else torch.float32
    for call in range(2):
        grad = rng.normal(size=sc["x0"].shape)
        z_ref = g.precond_apply(xb, grad)      # rebuilds P_base at xb, applies it
        gd = torch.tensor(grad, dtype=dtype, device="cuda")
        zd = torch.full_like(gd, float("nan"))  # every entry must be overwritten
        g.precond_apply_noalloc(gd, zd)
        z = zd.double().cpu().numpy()
        assert np.all(np.isfinite(z))
        err = np.linalg.norm(z - z_ref) / np.linalg.norm(z_ref)
        assert err <= rtol, (call, err)


def test_noalloc_rejects_a_scene_without_a_preconditioner(lib):
    """A freshly created scene has assembled and inverted nothing yet: the
    call refuses it instead of applying uninitialised blocks."""
    import torch
    from paper_2604_19892_b300 import scenes as S
    g = lib.Scene(S.two_cubes(n=3, gap=0.004))
    gd = torch.zeros(3 * g.nv, dtype=torch.float64, device="cuda")
    zd = torch.zeros_like(gd)
    with pytest.raises(lib.IPCError) as e:
        g.precond_apply_noalloc(gd, zd)
    assert e.value.code == lib.IPC_ERR_INVALID and "no preconditioner" in str(e.value)


def test_noalloc_rejects_bad_arguments(lib):
    import torch
    from paper_2604_19892_b300 import scenes as S
    sc = S.two_cubes(n=3, gap=0.004)
    g = lib.Scene(sc)
    g.precond_apply(sc["x0"], np.zeros_like(sc["x0"]))
    n3 = 3 * g.nv
    gd = torch.zeros(n3, dtype=torch.float64, device="cuda")
    zd = torch.zeros(n3, dtype=torch.float64, device="cuda")
    host = np.zeros(n3)
    L = lib.load()
    import ctypes as C
    code = L.ipc_precond_apply_noalloc(g.h, C.c_void_p(host.ctypes.data), C.c_void_p(zd.data_ptr()), None)
    assert code == lib.IPC_ERR_INVALID and b"device arrays" in L.ipc_last_error()
    code = L.ipc_precond_apply_noalloc(g.h, C.c_void_p(gd.data_ptr()), C.c_void_p(gd.data_ptr()), None)
    assert code == lib.IPC_ERR_INVALID and b"overlap" in L.ipc_last_error()


def test_noalloc_reports_an_exhausted_copy_wait(lib):
    """With a zero poll budget every block's bounded wait reports a timeout
    (each CTA still drains its copy): the call returns IPC_ERR_TIMEOUT instead
    of an undefined z, and the scene's own status is not touched."""
    import torch
    from paper_2604_19892_b300 import scenes as S
    sc = S.two_cubes(n=3, gap=0.004)
    g = lib.Scene(sc, params={"wait_polls": 0})
    with pytest.raises(lib.IPCError) as e:
        g.precond_apply(sc["x0"], np.ones_like(sc["x0"]))   # builds P_base, then times out
    assert e.value.code == lib.IPC_ERR_TIMEOUT
    gd = torch.ones(3 * g.nv, dtype=torch.float64, device="cuda")
    zd = torch.zeros_like(gd)
    for _ in range(2):
        with pytest.raises(lib.IPCError) as e:
            g.precond_apply_noalloc(gd, zd)
        assert e.value.code == lib.IPC_ERR_TIMEOUT


@pytest.mark.parametrize("precision,n_ok,n_over", [(0, 40, 56), (1, 56, 72)])
def test_noalloc_static_limit(lib, precision, n_ok, n_over):
    """The coarse scratch (two arrays of 3 x coarse nodes values, 8 bytes in
    FP64, 4 in FP32) fits the static 256 KiB below about 1.7e5 vertices in
    FP64 and 3.4e5 in FP32: a block scene below the limit is served, one
    above it (185,193 vertices in FP64; 389,017 in FP32) gets
    IPC_ERR_CAPACITY."""
    import torch
    from paper_2604_19892_b300 import scenes as S
    dtype = torch.float64 if precision == 0 else torch.float32
    for n, ok in ((n_ok, True), (n_over, False)):
        sc = S.free_fall_block(n=n)
        g = lib.Scene(sc, precision=precision)
        g.precond_apply(sc["x0"], np.zeros_like(sc["x0"]))
        gd = torch.ones(3 * g.nv, dtype=dtype, device="cuda")
        zd = torch.zeros_like(gd)
        if ok:
            g.precond_apply_noalloc(gd, zd)
            assert bool(torch.isfinite(zd).all())
        else:
            with pytest.raises(lib.IPCError) as e:
                g.precond_apply_noalloc(gd, zd)
            assert e.value.code == lib.IPC_ERR_CAPACITY and "static limit" in str(e.value)
        g.close()
