"""The allocation-free residual entry point (for callers that cannot allocate
device memory) through the C ABI, against the allocating entry point.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
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


def _inputs(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(n)
    b = a + 1e-3 * rng.standard_normal(n)
    w = rng.uniform(0.05, 3.0, n)
    return [torch.from_numpy(x).cuda() for x in (a, b, w)]


@pytest.mark.parametrize("n", [1, 4097, 2_500_003])
def test_noalloc_matches_allocating_entry_point_twice(E, n):
    import torch
    a, b, w = _inputs(n, n)
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    E.ehdg_trace_residual(a, b, w, ref)
    for _ in range(2):   # two calls in a row share (and must reset) the fixed scratch
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        E.ehdg_trace_residual_noalloc(a, b, w, out)
        assert abs(out.item() - ref.item()) <= 1e-13 * abs(ref.item())


def test_noalloc_rejects_sizes_beyond_its_scratch(E):
    import torch
    n = E.EHDG_NOALLOC_MAX_N + 1
    # buffers of the full size, so nothing could be read out of bounds
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EhdgError) as ei:
        E.ehdg_trace_residual_noalloc(z, z, z, out)
    assert ei.value.status == 7
    assert "exceeds the maximum" in str(ei.value)


def test_noalloc_call_captures_into_a_cuda_graph_and_replays(E):
    """After a first call outside capture (which looks up the fixed array's
    address), a later call is captured: the capture allocates nothing and
    launches nothing, and each replay reads the inputs' current contents."""
    import torch
    n = 100_003
    a, b, w = _inputs(n, 11)
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    E.ehdg_trace_residual_noalloc(a, b, w, out)          # first call, outside capture
    torch.cuda.synchronize()
    out.fill_(-1.0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        E.ehdg_trace_residual_noalloc(a, b, w, out, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert out.item() == -1.0                              # captured, not run
    rng = np.random.default_rng(12)
    for rep in range(3):
        if rep:                                            # new values in the same buffers
            b.copy_(a + torch.from_numpy(1e-3 * rng.standard_normal(n)).cuda())
        E.ehdg_trace_residual(a, b, w, ref)
        out.fill_(-1.0)
        g.replay()
        torch.cuda.synchronize()
        assert abs(out.item() - ref.item()) <= 1e-13 * abs(ref.item())
