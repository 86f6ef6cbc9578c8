"""Thin ctypes binding of libehdg (include/ehdg.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts numpy
arrays and torch CUDA tensors into the pointers and sizes the C ABI takes.
Loading fails loudly when libehdg.so has not been built (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

# A batch's graph runs its branches on the GPU's hardware work queues. CUDA
# creates 8 of them unless CUDA_DEVICE_MAX_CONNECTIONS says otherwise when
# the context is created, and a batch then runs at most 8 branches at once.
# Ask for the maximum, 32, unless the caller chose a value (this takes effect
# only if CUDA has not been initialised in the process yet).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libehdg.so")

EHDG_OK = 0
STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "NOT_CONVERGED", 5: "DIVERGED",
          6: "TIMEOUT", 7: "UNSUPPORTED"}
PDE = {"transport": 0, "sw": 1}
SCHEME = {"be": 0, "cn": 1, "steady": 2}
PRECISION = {"fp64": 0, "tf32": 1, "bf16": 2, "fp32": 3, "fp64_emulated": 4}
FACE_INTERIOR, FACE_DIRICHLET, FACE_WALL = 0, 1, 2


class EhdgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"ehdg status {STATUS.get(status, status)}: {msg}")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_elem", C.c_int64), ("n_face", C.c_int64),
                ("elem_lo", C.POINTER(C.c_double)), ("elem_h", C.POINTER(C.c_double)),
                ("elem_face", C.POINTER(C.c_int64)), ("face_elem", C.POINTER(C.c_int64)),
                ("face_local", C.POINTER(C.c_int8)), ("face_tag", C.POINTER(C.c_int32))]


class ProblemDesc(C.Structure):
    _fields_ = [("pde", C.c_int), ("p", C.c_int), ("scheme", C.c_int), ("dt", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int), ("precision", C.c_int),
                ("beta_const", C.POINTER(C.c_double)), ("beta_nodes", C.POINTER(C.c_double)),
                ("Phi", C.c_double), ("inner_sweeps", C.c_int),
                ("coriolis_f0", C.c_double), ("coriolis_beta", C.c_double),
                ("coriolis_ym", C.c_double), ("friction", C.c_double),
                ("emulated_outer", C.c_int)]


class Info(C.Structure):
    _fields_ = [("dim", C.c_int), ("p", C.c_int), ("nf", C.c_int), ("Np", C.c_int),
                ("q", C.c_int), ("Nqf", C.c_int), ("n_elem", C.c_int64), ("n_face", C.c_int64),
                ("state_len", C.c_int64), ("trace_len", C.c_int64),
                ("shared_operator", C.c_int), ("device_bytes", C.c_int64),
                ("sweep_rows", C.c_int64), ("sum_factorised", C.c_int),
                ("warm_start", C.c_int)]


_lib = None

# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("ehdg_mesh_structured", C.c_int, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.c_int32, C.POINTER(MeshDesc)]),
    ("ehdg_mesh_free", None, [C.POINTER(MeshDesc)]),
    ("ehdg_create", C.c_int, [C.POINTER(MeshDesc), C.POINTER(ProblemDesc), C.c_void_p,
                              C.POINTER(C.c_void_p)]),
    ("ehdg_get_info", C.c_int, [C.c_void_p, C.POINTER(Info)]),
    ("ehdg_destroy", None, [C.c_void_p]),
    ("ehdg_node_coords", C.c_int, [C.c_void_p, C.c_void_p]),
    ("ehdg_face_point_coords", C.c_int, [C.c_void_p, C.c_void_p]),
    ("ehdg_set_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    ("ehdg_set_forcing", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("ehdg_set_boundary", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("ehdg_step", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("ehdg_run", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    ("ehdg_step_fixed", C.c_int, [C.c_void_p, C.c_int]),
    ("ehdg_get_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    ("ehdg_get_residual_history", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64,
                                            C.POINTER(C.c_int64)]),
    ("ehdg_save", C.c_int, [C.c_void_p, C.c_char_p]),
    ("ehdg_load", C.c_int, [C.c_void_p, C.c_char_p]),
    ("ehdg_autotune_fp64_path", C.c_int, [C.c_void_p, C.POINTER(C.c_int),
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("ehdg_autotune_inner_sweeps", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int,
                                             C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("ehdg_autotune_sweep_tile", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int,
                                           C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("ehdg_set_profiling", C.c_int, [C.c_void_p, C.c_int]),
    ("ehdg_selftest_wait_timeout", C.c_int, [C.c_int, C.c_void_p]),
    ("ehdg_probe_fp64_rate", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("ehdg_kernel_stats", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64),
                                    C.POINTER(C.c_double)]),
    ("ehdg_batch_create", C.c_int, [C.c_int, C.POINTER(MeshDesc), C.POINTER(ProblemDesc),
                                    C.c_void_p, C.POINTER(C.c_void_p)]),
    ("ehdg_batch_instance", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    ("ehdg_batch_run", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("ehdg_batch_set_chains", C.c_int, [C.c_void_p, C.c_int]),
    ("ehdg_batch_set_loop", C.c_int, [C.c_void_p, C.c_int]),
    ("ehdg_batch_set_profiling", C.c_int, [C.c_void_p, C.c_int]),
    ("ehdg_batch_kernel_stats", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64),
                                          C.POINTER(C.c_double)]),
    ("ehdg_batch_autotune_chains", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int,
                                             C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("ehdg_batch_autotune_sweep_tile", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int,
                                                 C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("ehdg_batch_autotune_schedule", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int,
                                               C.POINTER(C.c_int), C.POINTER(C.c_int),
                                               C.POINTER(C.c_double)]),
    ("ehdg_batch_autotune_inner_sweeps", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int,
                                                   C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    ("ehdg_batch_destroy", None, [C.c_void_p]),
    ("ehdg_trace_residual", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                      C.c_void_p]),
    ("ehdg_trace_residual_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                              C.c_void_p, C.c_void_p]),
    ("ehdg_last_error", C.c_char_p, []),
]

EHDG_NOALLOC_MAX_N = 16777216

KERNEL_KINDS = ["assemble", "signs", "step", "elem", "face", "final", "aux", "corr"]


def load(path=LIB_PATH):
    """Load libehdg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1601_06681_gb300.build.build()")
    lib = C.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_names():
    return [s[0] for s in _SIGS]


def _check(status):
    if status != EHDG_OK:
        raise EhdgError(status, load().ehdg_last_error().decode())


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _buf(x, shape):
    """(pointer, on_device, keepalive) for a numpy array or a CUDA tensor."""
    if x is None:
        return None, 0, None
    if hasattr(x, "is_cuda") and x.is_cuda:
        import torch
        assert x.dtype == torch.float64 and x.is_contiguous() and x.numel() == int(np.prod(shape))
        return C.c_void_p(x.data_ptr()), 1, x
    a = np.ascontiguousarray(x, dtype=np.float64)
    assert a.size == int(np.prod(shape)), (a.shape, shape)
    return a.ctypes.data_as(C.c_void_p), 0, a


def _dev_ptr(t):
    import torch
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    return C.c_void_p(t.data_ptr())


def ehdg_trace_residual(a, b, w, out, stream=None):
    """sqrt(sum w (a - b)^2) of three float64 CUDA tensors into out (1 element)."""
    n = a.numel()
    assert b.numel() == n and w.numel() == n and out.numel() >= 1
    s = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(load().ehdg_trace_residual(_dev_ptr(a), _dev_ptr(b), _dev_ptr(w), n, _dev_ptr(out), s))
    return out


def ehdg_selftest_wait_timeout(which, stream=None):
    """Run a bounded device-side wait (0: mbarrier, 1: grid barrier) against a
    condition that never holds; returns the status (EHDG_ERR_TIMEOUT = 6 is
    the expected one)."""
    return load().ehdg_selftest_wait_timeout(int(which), _stream_ptr(stream))


def ehdg_probe_fp64_rate(stream=None):
    """(SM count, measured FP64 FMA rate in TFLOP/s) of the current device."""
    sms, tf = C.c_int(), C.c_double()
    _check(load().ehdg_probe_fp64_rate(_stream_ptr(stream), C.byref(sms), C.byref(tf)))
    return sms.value, tf.value


def ehdg_trace_residual_noalloc(a, b, w, out, stream=None):
    """As ehdg_trace_residual, with the scratch in the library's fixed device
    array (no allocation; calls must not overlap on the GPU)."""
    n = a.numel()
    assert b.numel() == n and w.numel() == n and out.numel() >= 1
    s = None if stream is None else C.c_void_p(stream.cuda_stream)
    _check(load().ehdg_trace_residual_noalloc(_dev_ptr(a), _dev_ptr(b), _dev_ptr(w), n,
                                              _dev_ptr(out), s))
    return out


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class Mesh:
    """A mesh descriptor that keeps its arrays alive (from a dict of arrays or
    from the library's structured-mesh builder)."""

    def __init__(self, d):
        self.dim = int(d["dim"])
        self.arrays = dict(
            elem_lo=np.ascontiguousarray(d["elem_lo"], dtype=np.float64),
            elem_h=np.ascontiguousarray(d["elem_h"], dtype=np.float64),
            elem_face=np.ascontiguousarray(d["elem_face"], dtype=np.int64),
            face_elem=np.ascontiguousarray(d["face_elem"], dtype=np.int64),
            face_local=np.ascontiguousarray(d["face_local"], dtype=np.int8),
            face_tag=np.ascontiguousarray(d["face_tag"], dtype=np.int32))
        a = self.arrays
        self.n_elem, self.n_face = int(d["n_elem"]), int(d["n_face"])
        self.desc = MeshDesc(self.dim, self.n_elem, self.n_face, _ptr(a["elem_lo"], C.c_double),
                             _ptr(a["elem_h"], C.c_double), _ptr(a["elem_face"], C.c_int64),
                             _ptr(a["face_elem"], C.c_int64), _ptr(a["face_local"], C.c_int8),
                             _ptr(a["face_tag"], C.c_int32))

    def as_dict(self):
        return dict(dim=self.dim, n_elem=self.n_elem, n_face=self.n_face, **self.arrays)


def ehdg_mesh_structured(n, lo=None, hi=None, boundary_tag=FACE_DIRICHLET):
    """The library's structured mesh, returned as a dict of numpy arrays."""
    lib = load()
    dim = len(n)
    nn = (C.c_int64 * 3)(*(list(n) + [1] * (3 - dim)))
    lo = [0.0] * dim if lo is None else list(lo)
    hi = [1.0] * dim if hi is None else list(hi)
    clo = (C.c_double * 3)(*(lo + [0.0] * (3 - dim)))
    chi = (C.c_double * 3)(*(hi + [1.0] * (3 - dim)))
    desc = MeshDesc()
    _check(lib.ehdg_mesh_structured(dim, nn, clo, chi, boundary_tag, C.byref(desc)))
    try:
        ne, nf = desc.n_elem, desc.n_face
        out = dict(dim=dim, n_elem=ne, n_face=nf,
                   elem_lo=np.ctypeslib.as_array(desc.elem_lo, (ne, dim)).copy(),
                   elem_h=np.ctypeslib.as_array(desc.elem_h, (ne, dim)).copy(),
                   elem_face=np.ctypeslib.as_array(desc.elem_face, (ne, 2 * dim)).copy(),
                   face_elem=np.ctypeslib.as_array(desc.face_elem, (nf, 2)).copy(),
                   face_local=np.ctypeslib.as_array(desc.face_local, (nf, 2)).copy(),
                   face_tag=np.ctypeslib.as_array(desc.face_tag, (nf,)).copy())
    finally:
        lib.ehdg_mesh_free(C.byref(desc))
    return out


class Solver:
    """One eHDG problem on the GPU (wraps an ehdg_ctx)."""

    def __init__(self, mesh, p, pde="transport", scheme="be", dt=1.0, tol=1e-10, max_iter=1000,
                 beta_const=None, beta_nodes=None, Phi=1.0, precision="fp64", inner_sweeps=0,
                 coriolis=(0.0, 0.0, 0.0), friction=0.0, emulated_outer=False, stream=None,
                 _handle=None):
        lib = load()
        self.mesh = mesh if isinstance(mesh, Mesh) else Mesh(mesh)
        self._beta_const = None if beta_const is None else np.ascontiguousarray(beta_const, np.float64)
        self._beta_nodes = None if beta_nodes is None else np.ascontiguousarray(beta_nodes, np.float64)
        self.prob = ProblemDesc(
            PDE[pde], int(p), SCHEME[scheme], float(dt), float(tol), int(max_iter),
            PRECISION[precision],
            None if self._beta_const is None else _ptr(self._beta_const, C.c_double),
            None if self._beta_nodes is None else _ptr(self._beta_nodes, C.c_double), float(Phi),
            int(inner_sweeps), float(coriolis[0]), float(coriolis[1]), float(coriolis[2]),
            float(friction), int(bool(emulated_outer)))
        self.max_iter = int(max_iter)
        self._owned = _handle is None
        if _handle is not None:          # an instance of a batch (owned by the batch)
            self._h = _handle
        else:
            s = _stream_ptr(stream)
            h = C.c_void_p()
            _check(lib.ehdg_create(C.byref(self.mesh.desc), C.byref(self.prob), s, C.byref(h)))
            self._h = h
        info = Info()
        _check(lib.ehdg_get_info(self._h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in Info._fields_}

    # sizes
    @property
    def state_shape(self):
        i = self.info
        return (i["n_elem"], i["nf"], i["Np"])

    @property
    def trace_shape(self):
        return (self.info["n_face"], self.info["Nqf"])

    def node_coords(self):
        i = self.info
        x = np.empty((i["n_elem"], i["Np"], i["dim"]))
        _check(load().ehdg_node_coords(self._h, x.ctypes.data_as(C.c_void_p)))
        return x

    def face_point_coords(self):
        i = self.info
        x = np.empty((i["n_face"], i["Nqf"], i["dim"]))
        _check(load().ehdg_face_point_coords(self._h, x.ctypes.data_as(C.c_void_p)))
        return x

    def set_state(self, u, uhat=None):
        pu, dev, ku = _buf(u, self.state_shape)
        ph, dev2, kh = _buf(uhat, self.trace_shape)
        if uhat is not None:
            assert dev == dev2
        _check(load().ehdg_set_state(self._h, pu, ph, dev))
        # device buffers are read on the context's stream after the call
        # returns: keep them alive until the next upload
        self._state_keep = (ku, kh)

    def set_forcing(self, f):
        pf, dev, kf = _buf(f, self.state_shape)
        _check(load().ehdg_set_forcing(self._h, pf, dev))
        self._forcing_keep = kf

    def set_boundary(self, g):
        pg, dev, kg = _buf(g, self.trace_shape)
        _check(load().ehdg_set_boundary(self._h, pg, dev))
        self._boundary_keep = kg

    def step(self, check=True):
        it, res = C.c_int(), C.c_double()
        st = load().ehdg_step(self._h, C.byref(it), C.byref(res))
        if check:
            _check(st)
        return it.value, res.value, st

    def step_fixed(self, n_iter):
        _check(load().ehdg_step_fixed(self._h, int(n_iter)))

    def run(self, n_steps):
        iters = (C.c_int * max(n_steps, 1))()
        _check(load().ehdg_run(self._h, int(n_steps), iters))
        return list(iters)[:n_steps]

    def get_state(self, u_out=None, uhat_out=None):
        """Host copies (numpy), or fills the given buffers: CUDA tensors, or
        host arrays / CPU tensors (pinned ones copy fastest)."""
        if u_out is None and uhat_out is None:
            u = np.empty(self.state_shape)
            uh = np.empty(self.trace_shape)
            _check(load().ehdg_get_state(self._h, u.ctypes.data_as(C.c_void_p),
                                         uh.ctypes.data_as(C.c_void_p), 0))
            return u, uh
        pu, dev, _ = _buf(u_out, self.state_shape)
        ph, dev2, _ = _buf(uhat_out, self.trace_shape)
        _check(load().ehdg_get_state(self._h, pu, ph, max(dev, dev2)))
        return u_out, uhat_out

    def residual_history(self):
        buf = np.empty(self.max_iter)
        n = C.c_int64()
        _check(load().ehdg_get_residual_history(self._h, buf.ctypes.data_as(C.c_void_p),
                                                buf.size, C.byref(n)))
        return buf[:min(n.value, buf.size)].copy()

    def save(self, path):
        _check(load().ehdg_save(self._h, os.fsencode(path)))

    def load_checkpoint(self, path):
        _check(load().ehdg_load(self._h, os.fsencode(path)))

    def autotune_fp64_path(self):
        """ehdg_autotune_fp64_path: (tensor cores chosen, ms per step DFMA, ms per
        step tensor cores)."""
        tc, md, mt = C.c_int(), C.c_double(), C.c_double()
        _check(load().ehdg_autotune_fp64_path(self._h, C.byref(tc), C.byref(md), C.byref(mt)))
        return bool(tc.value), md.value, mt.value

    def autotune_sweep_tile(self, candidates=(2, 4, 8)):
        """Row groups per 32-element tile of the fused FP64 sweep, timed one
        step each from the current state (restored): (best FT, ms)."""
        arr = (C.c_int * len(candidates))(*[int(k) for k in candidates])
        best, ms = C.c_int(), C.c_double()
        _check(load().ehdg_autotune_sweep_tile(self._h, arr, len(candidates), C.byref(best),
                                               C.byref(ms)))
        return best.value, ms.value

    def autotune_inner_sweeps(self, candidates=(2, 3, 4, 6, 8, 12)):
        """Fastest inner sweep count for one step from the current state (which
        is restored); the context keeps it. Returns (best, ms)."""
        arr = (C.c_int * len(candidates))(*candidates)
        best, ms = C.c_int(), C.c_double()
        _check(load().ehdg_autotune_inner_sweeps(self._h, arr, len(candidates), C.byref(best),
                                                 C.byref(ms)))
        return best.value, ms.value

    def tune_key(self):
        i = self.info
        return f"d{i['dim']}_p{i['p']}_nf{i['nf']}_q{i['q']}_shared{i['shared_operator']}_prec{self.prob.precision}"

    def set_profiling(self, on=True):
        _check(load().ehdg_set_profiling(self._h, 1 if on else 0))

    def kernel_stats(self):
        """{kind: (launches, total device ms)} since profiling was last switched."""
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            n, ms = C.c_int64(), C.c_double()
            _check(load().ehdg_kernel_stats(self._h, k, C.byref(n), C.byref(ms)))
            out[name] = (n.value, ms.value)
        return out

    def close(self):
        if getattr(self, "_owned", True) and getattr(self, "_h", None) is not None and self._h.value:
            load().ehdg_destroy(self._h)
        self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Independent problems stepped together: one CUDA graph launch per time
    step advances every instance (ehdg_batch_*). problems: list of dicts with
    the Solver keyword arguments (mesh, p, pde, scheme, dt, tol, ...)."""

    def __init__(self, problems, stream=None):
        lib = load()
        n = len(problems)
        self._keep = []
        meshes = (MeshDesc * n)()
        probs = (ProblemDesc * n)()
        self._specs = []
        for i, kw in enumerate(problems):
            kw = dict(kw)
            mesh = kw.pop("mesh")
            m = mesh if isinstance(mesh, Mesh) else Mesh(mesh)
            bc = kw.get("beta_const")
            bn = kw.get("beta_nodes")
            bc = None if bc is None else np.ascontiguousarray(bc, np.float64)
            bn = None if bn is None else np.ascontiguousarray(bn, np.float64)
            self._keep += [m, bc, bn]
            meshes[i] = m.desc
            probs[i] = ProblemDesc(
                PDE[kw.get("pde", "transport")], int(kw["p"]), SCHEME[kw.get("scheme", "be")],
                float(kw.get("dt", 1.0)), float(kw.get("tol", 1e-10)), int(kw.get("max_iter", 1000)),
                PRECISION[kw.get("precision", "fp64")],
                None if bc is None else _ptr(bc, C.c_double),
                None if bn is None else _ptr(bn, C.c_double), float(kw.get("Phi", 1.0)),
                int(kw.get("inner_sweeps", 0)), *[float(v) for v in kw.get("coriolis", (0, 0, 0))],
                float(kw.get("friction", 0.0)), int(bool(kw.get("emulated_outer", False))))
            self._specs.append((m, kw))
        h = C.c_void_p()
        _check(lib.ehdg_batch_create(n, meshes, probs, _stream_ptr(stream), C.byref(h)))
        self._h = h
        self.n = n
        self.instances = []
        for i in range(n):
            ih = C.c_void_p()
            _check(lib.ehdg_batch_instance(h, i, C.byref(ih)))
            m, kw = self._specs[i]
            args = {k: v for k, v in kw.items() if k not in ("p",)}
            self.instances.append(Solver(m, kw["p"], _handle=ih, **args))

    def run(self, n_steps):
        """(iters [n, n_steps], per-instance device seconds [n])."""
        iters = np.zeros((self.n, n_steps), dtype=np.int32)
        times = np.zeros(self.n)
        _check(load().ehdg_batch_run(self._h, int(n_steps), iters.ctypes.data_as(C.c_void_p),
                                     times.ctypes.data_as(C.c_void_p)))
        return iters, times

    def set_loop(self, on=True):
        """Batched iteration loop for the instances it supports (default on);
        off runs every instance's own loop on the graph's branches;
        "persistent" the loop's one-launch form (ehdg_batch_set_loop mode 2)."""
        mode = 2 if on == "persistent" else (1 if on else 0)
        _check(load().ehdg_batch_set_loop(self._h, mode))

    def set_profiling(self, on=True):
        """Kernel accounting of the batched loop (host-driven steps, every
        launch timed); resets the counters."""
        _check(load().ehdg_batch_set_profiling(self._h, 1 if on else 0))

    def kernel_stats(self):
        """{kind: (launches, total device ms)} of the batched loop's kernels."""
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            n, ms = C.c_int64(), C.c_double()
            _check(load().ehdg_batch_kernel_stats(self._h, k, C.byref(n), C.byref(ms)))
            out[name] = (n.value, ms.value)
        return out

    def set_chains(self, k):
        """Concurrent branches of the batch's graph (k <= 0: one per hardware
        work queue; k >= n: one per instance)."""
        _check(load().ehdg_batch_set_chains(self._h, int(k)))

    def autotune_chains(self, candidates=(8, 16, 32, 64, 256)):
        """Time one batch step per branch count from the current states
        (restored after each) and keep the fastest: (k, ms)."""
        arr = (C.c_int * len(candidates))(*[int(k) for k in candidates])
        best, ms = C.c_int(), C.c_double()
        _check(load().ehdg_batch_autotune_chains(self._h, arr, len(candidates), C.byref(best),
                                                 C.byref(ms)))
        return best.value, ms.value

    def autotune_schedule(self, chain_candidates=(16, 32, 64)):
        """Time the batched loop, its persistent form and the branch form
        with each branch count, from the current states (restored after
        each), and keep the fastest: (mode, k, ms), mode 0 branches, 1 loop,
        2 persistent."""
        arr = (C.c_int * len(chain_candidates))(*[int(k) for k in chain_candidates])
        loop_on, k, ms = C.c_int(), C.c_int(), C.c_double()
        _check(load().ehdg_batch_autotune_schedule(self._h, arr, len(chain_candidates),
                                                   C.byref(loop_on), C.byref(k), C.byref(ms)))
        return loop_on.value, k.value, ms.value

    def autotune_inner_sweeps(self, candidates=(2, 4, 6, 8, 12, 16)):
        """One inner sweep count m for every mixed-precision instance, timed
        as whole batch steps from the current states (restored): (m, ms)."""
        arr = (C.c_int * len(candidates))(*[int(k) for k in candidates])
        best, ms = C.c_int(), C.c_double()
        _check(load().ehdg_batch_autotune_inner_sweeps(self._h, arr, len(candidates),
                                                       C.byref(best), C.byref(ms)))
        return best.value, ms.value

    def autotune_sweep_tile(self, candidates=(2, 4, 8)):
        """One tile shape FT for every instance's fused FP64 sweep, timed as
        whole batch steps from the current states (restored): (FT, ms)."""
        arr = (C.c_int * len(candidates))(*[int(k) for k in candidates])
        best, ms = C.c_int(), C.c_double()
        _check(load().ehdg_batch_autotune_sweep_tile(self._h, arr, len(candidates),
                                                     C.byref(best), C.byref(ms)))
        return best.value, ms.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            for s in self.instances:
                s._h = C.c_void_p()
            load().ehdg_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def autotune_cached(solver, cache_path, candidates=(2, 3, 4, 6, 8, 12)):
    """Inner sweep count for this kind of problem from a JSON cache keyed by
    dimension, degree, fields, quadrature, operator sharing and precision;
    tuned (ehdg_autotune_inner_sweeps) and stored on a miss. Returns the count,
    which the solver is then configured with."""
    import json
    cache = {}
    if os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    key = solver.tune_key()
    if key in cache:
        best = int(cache[key]["inner_sweeps"])
        solver.autotune_inner_sweeps((best,))
        return best
    best, ms = solver.autotune_inner_sweeps(candidates)
    cache[key] = {"inner_sweeps": best, "ms_per_step": ms, "candidates": list(candidates)}
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return best
