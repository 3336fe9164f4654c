"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(ipc_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ipc_scene_create", "ipc_scene_destroy", "ipc_step", "ipc_query", "ipc_last_error",
                 "ipc_set_state", "ipc_eval_energy_grad", "ipc_eval_contacts", "ipc_eval_precond",
                 "ipc_eval_forms", "ipc_eval_ccd"):
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2604_19892_b300 import build, ipc
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    # the binding's signature table covers the same set
    assert set(ipc.EXPORTS) <= _declared()
    ipc.load(path)


def test_library_is_built_for_sm_103a():
    from paper_2604_19892_b300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2604_19892_b300 import ipc
    with pytest.raises(RuntimeError):
        ipc.load.__wrapped__(str(tmp_path / "missing.so")) if hasattr(ipc.load, "__wrapped__") else \
            _load_missing(ipc, str(tmp_path / "missing.so"))


def _load_missing(ipc, path):
    saved = ipc._lib
    ipc._lib = None
    try:
        ipc.load(path)
    finally:
        ipc._lib = saved


def test_params_mirror_matches_the_header():
    """ipc_default_params (host code only) fills the binding's ctypes mirror of
    ipc_params: every field reads back its documented default, the last ones
    included, so the two layouts agree (a field added on one side only would
    shift the fields after it)."""
    from paper_2604_19892_b300 import build, ipc
    lib = ipc.load(build.build())
    p = ipc.Params()
    ctypes.memset(ctypes.byref(p), 0xAB, ctypes.sizeof(p))
    lib.ipc_default_params(ctypes.byref(p))
    assert (p.eps_rot_deg, p.ccd_shrink, p.eps_sing) == (25.0, 0.1, 1e-12)
    assert (p.K, p.iter_max, p.levels_max, p.ls_max) == (8, 10000, 6, 20)
    assert (p.precision, p.contact_capacity, p.broad_phase) == (ipc.IPC_PREC_FP64, 0, 0)
    assert (p.mas_mode, p.ccd_mode, p.graphs) == (0, 0, 1)
    assert p.fp32_pivot_floor == 1e-6
    assert p.grid_pair_capacity == 0
    assert p.wait_polls == 1 << 22
    assert p.apply_ctas == 0


def test_fma_peak_refuses_bad_arguments_before_any_cuda_call():
    # the argument checks come first, so this runs without a GPU
    import ctypes as C
    from paper_2604_19892_b300 import build, ipc
    lib = ipc.load(build.build())
    out = C.c_double(-1.0)
    for prec, ms in ((7, 10.0), (ipc.IPC_PREC_BF16_MAS, 10.0), (ipc.IPC_PREC_FP32, 0.0),
                     (ipc.IPC_PREC_FP32, 5000.0)):
        assert lib.ipc_profile_fma_peak(prec, ms, C.byref(out)) == ipc.IPC_ERR_INVALID
    assert lib.ipc_profile_fma_peak(ipc.IPC_PREC_FP32, 10.0, None) == ipc.IPC_ERR_INVALID
    assert out.value == -1.0
