"""The standalone FP64 trace residual (Algorithm 1's convergence check) on the
GPU against float64 numpy, including empty, single-element and ragged sizes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_06681_gb300 import build, ehdg
    build.build()
    ehdg.load()
    return ehdg


@pytest.mark.parametrize("n", [0, 1, 255, 257, 100003, 3_000_001])
def test_trace_residual_matches_numpy(E, n):
    import torch
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n)
    b = a + 1e-6 * rng.standard_normal(n)
    w = rng.uniform(0.1, 2.0, n)
    ta, tb, tw = (torch.from_numpy(x).cuda() for x in (a, b, w))
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    E.ehdg_trace_residual(ta, tb, tw, out)
    got = float(out.item())
    want = float(np.sqrt(np.sum(w * (a - b) ** 2)))
    if n == 0:
        assert got == 0.0
    else:
        assert abs(got - want) <= 1e-13 * want
    # deterministic: the same call gives the same bits
    out2 = torch.zeros(1, dtype=torch.float64, device="cuda")
    E.ehdg_trace_residual(ta, tb, tw, out2)
    assert out2.item() == got


def test_trace_residual_rejects_bad_arguments(E):
    import ctypes
    lib = E.load()
    st = lib.ehdg_trace_residual(None, None, None, 10, None, None)
    assert st == 1
    assert b"NULL" in lib.ehdg_last_error()
