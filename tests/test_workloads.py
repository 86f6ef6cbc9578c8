"""The seeded input generators shared by the CUDA path's tests and bench and
by the oracle (no GPU): mesh connectivity invariants, determinism, and the
stated ranges of the batched mix."""
import numpy as np
import pytest

from paper_1601_06681_gb300 import workloads as W


@pytest.mark.parametrize("n", [(3, 4), (1, 5), (2, 3, 4), (1, 1, 1)])
def test_structured_mesh_connectivity_is_consistent(n):
    """Face counts, both directions of the element-face incidence, the local
    face numbering (2 axis for the lower side, 2 axis + 1 for the upper) and
    the boundary tags; the minus element of an interior face is the lower one
    along the face's normal axis and shares its lower corner but for that axis."""
    m = W.structured_mesh(n, lo=[0.5] * len(n), hi=[2.0] * len(n), boundary_tag=W.TAG_WALL)
    dim = len(n)
    assert m["n_elem"] == int(np.prod(n))
    n_face = sum((n[a] + 1) * int(np.prod([n[b] for b in range(dim) if b != a]))
                 for a in range(dim))
    assert m["n_face"] == n_face
    fe, fl, ef = m["face_elem"], m["face_local"], m["elem_face"]
    assert np.all(ef >= 0)                                   # every element face numbered
    interior = fe[:, 1] >= 0
    assert np.array_equal(m["face_tag"] == W.TAG_INTERIOR, interior)
    assert np.all(m["face_tag"][~interior] == W.TAG_WALL)
    for f in range(n_face):
        em, ep = fe[f]
        assert ef[em, fl[f, 0]] == f
        ax = fl[f, 0] // 2
        if ep >= 0:
            assert ef[ep, fl[f, 1]] == f
            assert fl[f, 0] == 2 * ax + 1 and fl[f, 1] == 2 * ax
            d = m["elem_lo"][ep] - m["elem_lo"][em]
            assert np.isclose(d[ax], m["elem_h"][em, ax])
            assert np.allclose(np.delete(d, ax), 0.0)
    # every element face appears exactly once in the face list
    seen = np.zeros(ef.shape, dtype=int)
    for f in range(n_face):
        for side in (0, 1):
            if fe[f, side] >= 0:
                seen[fe[f, side], fl[f, side]] += 1
    assert np.all(seen == 1)
    # the elements tile the box
    vol = np.prod(m["elem_h"], axis=1).sum()
    assert np.isclose(vol, 1.5 ** dim)


def test_generators_are_deterministic_in_their_seed():
    """The same seed gives the same inputs bit for bit; another seed other
    inputs."""
    def draw(seed):
        wl = W.transport_2d_variable(n=(6, 5), p=2, seed=seed)
        x = np.random.default_rng(0).uniform(0.0, 1.0, size=(40, 2))
        return np.concatenate([wl.beta_fn(x).ravel(), wl.initial(x[None]).ravel()])
    assert np.array_equal(draw(1002), draw(1002))
    assert not np.array_equal(draw(1002), draw(1003))
    a = W.batched_mix(n_inst=16, seed=7)
    b = W.batched_mix(n_inst=16, seed=7)
    assert [w.name for w in a] == [w.name for w in b]
    assert all(np.array_equal(u.beta_const, v.beta_const) for u, v in zip(a, b))


def test_batched_mix_stays_in_its_stated_ranges():
    """N in 8..128 (log-uniform), p in 1..5, |beta| in [0.5, 1.5], BE with
    dt 0.01 for 10 steps at tol 1e-10: the mix of 256 instances covers the
    range's ends."""
    mix = W.batched_mix()
    assert len(mix) == 256
    ns = np.array([w.n[0] for w in mix])
    ps = np.array([w.p for w in mix])
    sp = np.array([np.linalg.norm(w.beta_const) for w in mix])
    assert all(w.n[0] == w.n[1] for w in mix)
    assert ns.min() >= 8 and ns.max() <= 128
    assert ns.min() <= 10 and ns.max() >= 110          # both ends of the log-uniform range
    assert np.median(ns) < 40                           # log-uniform: median near 8 * 4 = 32
    assert set(ps.tolist()) == {1, 2, 3, 4, 5}
    assert sp.min() >= 0.5 and sp.max() <= 1.5
    assert all((w.scheme, w.dt, w.n_steps, w.tol) == ("be", 0.01, 10, 1e-10) for w in mix)
