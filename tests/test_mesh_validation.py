"""Mesh validation of ehdg_create through the C ABI, which runs before any
CUDA call: every mesh the GPU tests hand to the library passes it, and
non-conforming meshes are rejected with EHDG_ERR_INVALID."""
import os
import re
import sys

import numpy as np
import pytest

from paper_1601_06681_gb300 import build, ehdg
from paper_1601_06681_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
PASSED_VALIDATION = (0, 3)    # created (a GPU is present) or stopped at the first CUDA call


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    ehdg.load()


def create_status(mesh, p, **kw):
    try:
        s = ehdg.Solver(mesh, p, **kw)
    except ehdg.EhdgError as e:
        return e.status, str(e)
    s.close()
    return 0, "created"


def _case_names(module_file):
    src = open(os.path.join(HERE, module_file)).read()
    return sorted(set(re.findall(r'name == "([^"]+)"', src)))


@pytest.mark.parametrize("module", ["test_gpu_parity", "test_gpu_edge_cases"])
def test_every_gpu_test_case_mesh_passes_validation(module):
    sys.path.insert(0, HERE)
    mod = __import__(module)
    names = _case_names(module + ".py")
    assert len(names) >= 10
    for name in names:
        mesh, p, kw, *_ = mod.make_case(name)
        st, msg = create_status(mesh, p, **kw)
        assert st in PASSED_VALIDATION, (name, msg)


@pytest.mark.parametrize("n,tag", [((64, 64, 64), W.TAG_DIRICHLET), ((256, 256), W.TAG_DIRICHLET),
                                   ((512, 512), W.TAG_WALL), ((97, 3), W.TAG_DIRICHLET)])
def test_large_structured_meshes_pass_validation(n, tag):
    mesh = ehdg.ehdg_mesh_structured(n, boundary_tag=tag)
    kw = (dict(pde="sw", scheme="be", dt=1e-3) if tag == W.TAG_WALL else
          dict(scheme="be", dt=0.01, beta_const=np.linspace(0.3, 0.9, len(n))))
    st, msg = create_status(mesh, 2, **kw)
    assert st in PASSED_VALIDATION, msg


def test_offset_and_graded_meshes_pass_validation():
    """Coordinates far from the origin relative to the element size, and a
    graded mesh whose element sizes are differences of node coordinates."""
    mesh = W.structured_mesh((6, 5), lo=(1.0e4, -3.0e3), hi=(1.0e4 + 6e-3, -3.0e3 + 5e-3))
    assert create_status(mesh, 2, scheme="be", dt=0.01, beta_const=[1.0, 0.5])[0] in \
        PASSED_VALIDATION
    rng = np.random.default_rng(5)
    xs = np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 1.5, 7))]) / 7.0
    ys = np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 1.5, 5))]) / 5.0
    g = W.structured_mesh((7, 5))
    i0, i1 = np.arange(g["n_elem"]) % 7, np.arange(g["n_elem"]) // 7
    g["elem_lo"] = np.stack([xs[i0], ys[i1]], -1)
    g["elem_h"] = np.stack([xs[i0 + 1] - xs[i0], ys[i1 + 1] - ys[i1]], -1)
    assert create_status(g, 2, scheme="be", dt=0.01, beta_const=[1.0, 0.5])[0] in \
        PASSED_VALIDATION


@pytest.mark.parametrize("what", ["size along the normal axis", "shift along the normal axis",
                                  "tangential extent"])
def test_non_conforming_meshes_are_rejected(what):
    """An element whose neighbour does not start where it ends, or whose face
    does not span its neighbour's face, makes a mesh whose faces do not match:
    EHDG_ERR_INVALID, before any CUDA call."""
    mesh = W.structured_mesh((4, 3))
    if what == "size along the normal axis":
        mesh["elem_h"][5, 0] *= 1.2
    elif what == "shift along the normal axis":
        mesh["elem_lo"][5, 0] += 0.01
    else:
        mesh["elem_h"][5, 1] *= 0.8
    st, msg = create_status(mesh, 2, scheme="be", dt=0.01, beta_const=[1.0, 0.5])
    assert st == 1 and "non-conforming" in msg, msg
