"""Failure detection without a GPU fault: every bounded device-side wait is
run against a condition that never holds, gives up within its poll limit and
reports EHDG_ERR_TIMEOUT, and the device keeps working afterwards."""
import numpy as np
import pytest

from oracle.ehdg import Problem
from paper_1601_06681_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ehdg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_06681_gb300 import build, ehdg as E
    build.build()
    E.load()
    return E


# 0: mbarrier waits, 1: grid barrier, 2: the persistent batched loop's work ring
@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_wait_gives_up_and_device_stays_usable(ehdg, which):
    import torch
    assert ehdg.ehdg_selftest_wait_timeout(which) == 6
    torch.cuda.synchronize()
    # the same process keeps solving correctly
    mesh, p = W.structured_mesh((7, 5)), 2
    beta = np.array([0.7, -0.4])
    rng = np.random.default_rng(99)
    prob = Problem(mesh, p, scheme="be", dt=0.05, beta_const=beta)
    u0 = rng.standard_normal((prob.nel, 1, prob.Np))
    g = rng.standard_normal((prob.nface, prob.Nqf))
    with ehdg.Solver(mesh, p, scheme="be", dt=0.05, tol=1e-12, max_iter=50,
                     beta_const=beta) as s:
        s.set_boundary(g)
        s.set_state(u0)
        s.step_fixed(3)
        u, _ = s.get_state()
    ou, _, _ = prob.solve_step(u0, None, g, fixed_iters=3)
    assert np.linalg.norm(u - ou) <= 1e-12 * np.linalg.norm(ou)
