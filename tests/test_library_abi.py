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


def test_structured_mesh_with_bounds_and_tag_matches_input_generator():
    """The library's mesh of a box [lo, hi] other than the unit box, with
    wall tags: the same connectivity and tags as the generator, and the same
    geometry to rounding (the two compute the corners in their own order)."""
    build.build()
    for n, lo, hi in [((5, 4), (-1.0, 2.0), (3.0, 2.5)),
                      ((3, 2, 4), (0.25, -0.5, 10.0), (1.0, 0.5, 10.2))]:
        got = ehdg.ehdg_mesh_structured(n, lo=lo, hi=hi, boundary_tag=W.TAG_WALL)
        want = W.structured_mesh(n, lo=lo, hi=hi, boundary_tag=W.TAG_WALL)
        for k in ("elem_face", "face_elem", "face_local", "face_tag"):
            assert np.array_equal(got[k], want[k]), (n, k)
        for k in ("elem_lo", "elem_h"):
            assert np.allclose(got[k], want[k], rtol=0, atol=1e-14 * max(map(abs, hi))), (n, k)


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


def _header_signatures():
    """{name: (return type, [parameter declarations])} of every function the
    header declares."""
    src = open(os.path.join(ROOT, "include", "ehdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#[^\n]*", "", src)
    out = {}
    for ret, name, params in re.findall(
            r"((?:const\s+)?[A-Za-z_][\w]*\s*\**)\s*\b(ehdg_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", src):
        ps = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        out[name] = (ret.replace(" ", ""), ps)
    return out


def _c_class(decl):
    """'ptr', 'i32', 'i64' or 'f64' for one C parameter declaration."""
    if "*" in decl or "[" in decl or re.match(r"(const\s+)?ehdg_(ctx|batch)\b", decl):
        return "ptr"
    t = decl.split()[0]
    return {"int": "i32", "int32_t": "i32", "int64_t": "i64", "double": "f64"}[t]


def _ctypes_class(t):
    import ctypes as C
    if t in (C.c_void_p, C.c_char_p) or hasattr(t, "_type_") and t.__name__.startswith("LP_"):
        return "ptr"
    return {C.c_int: "i32", C.c_int32: "i32", C.c_int64: "i64", C.c_double: "f64"}[t]


def test_binding_signatures_match_the_header():
    """Every ctypes signature of the binding has the header's parameter count,
    and each parameter the same class (pointer, 32- or 64-bit integer,
    double) and, where the binding names the pointee, the same pointee type;
    the return types agree (status int, void, or a C string)."""
    import ctypes as C
    hdr = _header_signatures()
    sigs = {n: (r, a) for n, r, a in ehdg._SIGS}
    assert sorted(hdr) == sorted(sigs)
    pointee = {"int": C.c_int, "int64_t": C.c_int64, "double": C.c_double}
    for name, (ret, params) in hdr.items():
        res, args = sigs[name]
        assert len(args) == len(params), name
        for decl, t in zip(params, args):
            assert _c_class(decl) == _ctypes_class(t), (name, decl, t)
            m = re.match(r"(?:const\s+)?(int|int64_t|double)\s*\*", decl)
            if m and t not in (C.c_void_p, C.c_char_p):
                assert t._type_ is pointee[m.group(1)], (name, decl, t)
        want_res = {"ehdg_status": C.c_int, "void": None, "constchar*": C.c_char_p}[ret]
        assert res is want_res, (name, ret, res)


def test_binding_structs_have_the_c_layout():
    """The ctypes structures of the binding (mesh, problem and info
    descriptors) have the layout the C compiler gives the header's structs:
    every field's offset and size, and the total size. A field added to one
    side only, or reordered, would otherwise corrupt every call silently."""
    import ctypes as C
    import shutil
    import subprocess
    import pytest
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"ehdg_mesh_desc": ehdg.MeshDesc, "ehdg_problem_desc": ehdg.ProblemDesc,
               "ehdg_info": ehdg.Info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ehdg.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f'sizeof((({cname}*)0)->{fname}));')
    lines += ["  return 0;", "}"]
    out_dir = os.path.join(ROOT, "paper_1601_06681_gb300", "_build", "abi_layout")
    os.makedirs(out_dir, exist_ok=True)
    src, exe = os.path.join(out_dir, "layout.c"), os.path.join(out_dir, "layout")
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                   check=True, capture_output=True)
    got = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {}
    for ln in filter(None, got):
        parts = ln.split()
        c_layout[tuple(parts[:-2]) if parts[1] != "size" else (parts[0],)] = (
            tuple(int(v) for v in parts[-2:]) if parts[1] != "size" else int(parts[2]))
    for cname, cls in structs.items():
        assert c_layout[(cname,)] == C.sizeof(cls), cname
        for fname, ftype in cls._fields_:
            assert c_layout[(cname, fname)] == (getattr(cls, fname).offset, C.sizeof(ftype)), \
                (cname, fname)


def test_create_validates_the_problem_before_any_cuda_call():
    """Invalid problems are rejected with EHDG_ERR_INVALID (1) or
    EHDG_ERR_UNSUPPORTED (7) and a message, before the library touches the
    GPU, so the checks hold on a machine without one."""
    import pytest
    build.build()
    mesh = ehdg.ehdg_mesh_structured((4, 4))
    base = dict(scheme="be", dt=0.01, beta_const=[1.0, 0.5])
    cases = [
        (dict(p=0), 7, "p must be"), (dict(p=7), 7, "p must be"),
        (dict(dt=0.0), 1, "dt must be positive"), (dict(dt=float("nan")), 1, "dt must be positive"),
        (dict(tol=-1e-10), 1, "bad tol"), (dict(tol=float("nan")), 1, "bad tol"),
        (dict(max_iter=0), 1, "max_iter"),
        (dict(precision="fp32", inner_sweeps=65), 1, "inner_sweeps must be 0..64"),
        (dict(beta_const=None), 1, "exactly one of beta_const and beta_nodes"),
        (dict(pde="sw", beta_const=None), 1, "tagged WALL"),
    ]
    for kw, status, msg in cases:
        args = dict(base, **kw)
        p = args.pop("p", 2)
        with pytest.raises(ehdg.EhdgError) as ei:
            ehdg.Solver(mesh, p, **args)
        assert ei.value.status == status, (kw, ei.value)
        assert msg in str(ei.value), (kw, str(ei.value))
