"""The C ABI library builds, loads without a GPU and exports every entry
point that include/ehdg.h declares (no compute calls)."""
import ctypes
import os
import re

import numpy as np

from paper_1601_06681_gb300 import build, ehdg
from paper_1601_06681_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ehdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ehdg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared entry points
    assert sorted(ehdg.exported_names()) == names


def test_structured_mesh_matches_input_generator():
    build.build()
    for n in [(5, 4), (1, 7), (3, 2, 4)]:
        got = ehdg.ehdg_mesh_structured(n)
        want = W.structured_mesh(n)
        for k, v in want.items():
            if isinstance(v, np.ndarray):
                assert np.array_equal(got[k], v), (n, k)
        assert got["n_face"] == want["n_face"]


def test_structured_mesh_rejects_bad_sizes():
    build.build()
    try:
        ehdg.ehdg_mesh_structured((0, 3))
    except ehdg.EhdgError as e:
        assert e.status == 1
    else:
        raise AssertionError("expected EhdgError")


def test_new_entry_points_reject_null_handles_without_a_gpu():
    """The batch and tile autotuners validate their arguments before any CUDA
    call, so these return EHDG_ERR_INVALID (1) on a machine without a GPU."""
    import ctypes as C
    build.build()
    lib = ehdg.load()
    cands = (C.c_int * 2)(2, 4)
    best, ms = C.c_int(), C.c_double()
    assert lib.ehdg_batch_set_chains(None, 3) == 1
    assert lib.ehdg_batch_autotune_chains(None, cands, 2, C.byref(best), C.byref(ms)) == 1
    assert lib.ehdg_batch_autotune_sweep_tile(None, cands, 2, C.byref(best), C.byref(ms)) == 1
    assert lib.ehdg_batch_autotune_inner_sweeps(None, cands, 2, C.byref(best), C.byref(ms)) == 1
    assert lib.ehdg_batch_set_loop(None, 2) == 1      # NULL batch (mode 2: persistent)
    loop_on = C.c_int()
    assert lib.ehdg_batch_autotune_schedule(None, cands, 2, C.byref(loop_on), C.byref(best),
                                            C.byref(ms)) == 1
    assert lib.ehdg_autotune_sweep_tile(None, cands, 2, C.byref(best), C.byref(ms)) == 1
    assert b"NULL" in lib.ehdg_last_error() or b"bad argument" in lib.ehdg_last_error()


def test_without_a_usable_gpu_the_solver_fails_loudly():
    """On a machine without a usable GPU, creating a context raises EhdgError
    with EHDG_ERR_CUDA (3) and the CUDA runtime's message: there is no CPU
    fallback anywhere in the library or the binding."""
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    build.build()
    mesh = ehdg.ehdg_mesh_structured((4, 4))
    with pytest.raises(ehdg.EhdgError) as ei:
        ehdg.Solver(mesh, 2, scheme="be", dt=0.01, beta_const=[1.0, 0.5])
    assert ei.value.status == 3
    assert "cudaMalloc failed" in str(ei.value)
