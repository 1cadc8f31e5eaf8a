"""Thin ctypes binding of libstm.so (the C ABI declared in include/stm.h).

Functions keep the C names; ``Slab`` bundles one context.  Arrays are either
numpy arrays (host memory, copied inside the call) or CUDA torch tensors
(device memory, used in place on the context stream).  Every step of the
residual, the solve and the energy runs in the library's CUDA kernels; this
module only marshals arguments.  Loading fails loudly when the library has
not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstm.so")

STM_OK = 0
STM_EINVAL = -1
STM_ENOMEM = -2
STM_EDEVICE = -3
STM_ETIMEOUT = -4
STM_ENAN = -5
STM_EUNSUPPORTED = -6
STM_ENOTCONV = 1

STM_GEOM_BRICK = 0
STM_GEOM_AFFINE = 1
STM_GEOM_TRILINEAR = 2
STM_FP64 = 0
STM_FP32 = 1
STM_MIXED = 2
STM_MEM_HOST = 0
STM_MEM_DEVICE = 1

# Every exported entry point of include/stm.h.
EXPORTS = (
    "stm_create", "stm_destroy", "stm_last_error", "stm_sizes", "stm_residual_apply", "stm_operator_apply",
    "stm_set_state", "stm_get_state", "stm_set_initial", "stm_slab_solve", "stm_energy",
    "stm_launch_count", "stm_profile_enable", "stm_profile_read", "stm_residual_apply_noalloc",
    "stm_set_source_gauss", "stm_set_boundary", "stm_set_source", "stm_dof_layout", "stm_fp64_probe",
    "stm_server_create", "stm_server_submit", "stm_server_poll", "stm_server_wait", "stm_server_stats",
    "stm_server_destroy", "stm_autotune", "stm_host_alloc", "stm_host_free",
)


class stm_mesh(C.Structure):
    _fields_ = [
        ("n_elem", C.c_int64), ("n_vert", C.c_int64),
        ("vert", C.POINTER(C.c_double)), ("hex", C.POINTER(C.c_int64)), ("nbr", C.POINTER(C.c_int64)),
        ("n_hang", C.c_int64), ("hang", C.POINTER(C.c_int64)),
        ("p", C.POINTER(C.c_uint8)), ("q", C.POINTER(C.c_uint8)),
        ("eps", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double)),
        ("geometry", C.c_int32), ("nk", C.POINTER(C.c_uint8)),
    ]


class stm_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tol", C.c_double), ("restart", C.c_int32), ("max_it", C.c_int32),
                ("deterministic", C.c_int32), ("stream", C.c_int64), ("reorth", C.c_int32), ("graph", C.c_int32),
                ("eta_tol", C.c_double), ("t_final", C.c_double), ("c_diss", C.c_double),
                ("zero_guess", C.c_int32), ("no_tensor_cores", C.c_int32), ("cycles_per_launch", C.c_int32)]


class stm_solve_report(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("rel_residual", C.c_double),
                ("energy", C.c_double), ("eta2", C.c_double)]


class stm_gauss_src(C.Structure):
    _fields_ = [("centre", C.c_double * 3), ("dir", C.c_double * 3), ("sigma_x", C.c_double), ("t0", C.c_double),
                ("sigma_t", C.c_double), ("amp", C.c_double)]


class stm_server_opts(C.Structure):
    _fields_ = [("workers", C.c_int32), ("hbm_budget_bytes", C.c_int64), ("precision", C.c_int32),
                ("tol", C.c_double), ("restart", C.c_int32), ("max_it", C.c_int32)]


class stm_request(C.Structure):
    _fields_ = [("n", C.c_int32), ("p", C.c_int32), ("q", C.c_int32), ("n_slabs", C.c_int32), ("dt", C.c_double),
                ("kind", C.c_int32), ("n_boxes", C.c_int32), ("boxes", (C.c_double * 8) * 4),
                ("n_src", C.c_int32), ("src", stm_gauss_src * 8)]


class stm_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("energy", C.c_double), ("t_final", C.c_double),
                ("latency_ms", C.c_double), ("queue_ms", C.c_double), ("max_rel_residual", C.c_double),
                ("n_state", C.c_int64), ("footprint_bytes", C.c_int64)]


class stm_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("running", C.c_int64),
                ("queued", C.c_int64), ("peak_admitted_bytes", C.c_int64), ("hbm_budget_bytes", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("solves_per_s", C.c_double), ("wall_s", C.c_double)]


FIELD_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double))
ST_FIELD_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double))

_lib = None


def lib() -> C.CDLL:
    """Load libstm.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libstm.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.stm_create.argtypes = [C.POINTER(vp), C.POINTER(stm_mesh), C.POINTER(stm_opts)]
        L.stm_destroy.argtypes = [vp]
        L.stm_last_error.argtypes = [vp]
        L.stm_last_error.restype = C.c_char_p
        L.stm_sizes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
        L.stm_residual_apply.argtypes = [vp, d, d, vp, vp, i32, i32]
        L.stm_operator_apply.argtypes = [vp, d, vp, vp, i32, i32, i32]
        L.stm_set_state.argtypes = [vp, d, vp, i32]
        L.stm_get_state.argtypes = [vp, C.POINTER(d), vp, i32]
        L.stm_set_initial.argtypes = [vp, d, FIELD_FN, FIELD_FN, vp]
        L.stm_slab_solve.argtypes = [vp, d, C.POINTER(stm_solve_report)]
        L.stm_energy.argtypes = [vp, C.POINTER(d)]
        L.stm_launch_count.argtypes = [vp, C.POINTER(i64)]
        L.stm_profile_enable.argtypes = [vp, i32]
        L.stm_profile_read.argtypes = [vp, C.POINTER(d), C.POINTER(i64)]
        L.stm_residual_apply_noalloc.argtypes = [i64, i32, i32, d, vp, vp, vp, vp, vp, vp, i64]
        L.stm_set_source_gauss.argtypes = [vp, C.POINTER(stm_gauss_src), i32]
        L.stm_set_boundary.argtypes = [vp, ST_FIELD_FN, vp]
        L.stm_set_source.argtypes = [vp, ST_FIELD_FN, vp]
        L.stm_fp64_probe.argtypes = [C.POINTER(C.c_double)]
        L.stm_dof_layout.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
        L.stm_server_create.argtypes = [C.POINTER(vp), C.POINTER(stm_server_opts)]
        L.stm_server_submit.argtypes = [vp, C.POINTER(stm_request), C.POINTER(i64)]
        L.stm_server_poll.argtypes = [vp, i64, C.POINTER(stm_result), vp]
        L.stm_server_wait.argtypes = [vp, i64, C.POINTER(stm_result), vp]
        L.stm_server_stats.argtypes = [vp, C.POINTER(stm_stats)]
        L.stm_server_destroy.argtypes = [vp]
        L.stm_host_alloc.argtypes = [C.POINTER(vp), i64]
        L.stm_host_free.argtypes = [vp]
        L.stm_autotune.argtypes = [vp, d, i32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(d),
                                   C.POINTER(i32)]
        for name in EXPORTS:
            if name != "stm_last_error":
                getattr(L, name).restype = C.c_int32
        _lib = L
    return _lib


def residual_apply_noalloc(n_elem, p, q, dt, nbr, h, eps, mu, U, R, stream=None) -> int:
    """stm_residual_apply_noalloc with CUDA torch tensors (all device memory); returns the status."""
    import torch

    args = []
    for t, dt_ in ((nbr, torch.int32), (h, torch.float64), (eps, torch.float64), (mu, torch.float64),
                   (U, torch.float64), (R, torch.float64)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.dtype == dt_):
            raise TypeError("residual_apply_noalloc takes contiguous CUDA tensors of the documented types")
        args.append(C.c_void_p(t.data_ptr()))
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    return lib().stm_residual_apply_noalloc(n_elem, p, q, dt, *args, int(stream))


def fp64_probe() -> float:
    """Measured FP64 FMA throughput of the current device (TFLOP/s)."""
    v = C.c_double()
    rc = lib().stm_fp64_probe(C.byref(v))
    if rc != STM_OK:
        raise StmError(rc, "stm_fp64_probe failed")
    return v.value


class HostBuffer:
    """Page-locked host array from stm_host_alloc (numpy view in .array)."""

    def __init__(self, n, dtype=np.float64):
        dtype = np.dtype(dtype)
        p = C.c_void_p()
        rc = lib().stm_host_alloc(C.byref(p), int(n) * dtype.itemsize)
        if rc != STM_OK:
            raise StmError(rc, "stm_host_alloc failed")
        self._p = p
        self.array = np.ctypeslib.as_array(C.cast(p, C.POINTER(np.ctypeslib.as_ctypes_type(dtype))), shape=(int(n),))

    def close(self):
        if getattr(self, "_p", None):
            self.array = None
            lib().stm_host_free(self._p)
            self._p = None

    __del__ = close


class StmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"stm error {code}: {msg}")
        self.code = code


def _ptr(a, dtype=None):
    """(pointer, mem kind, keep-alive) for a numpy array or a CUDA torch tensor."""
    if isinstance(a, np.ndarray):
        if dtype is not None and a.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data_as(C.c_void_p), STM_MEM_HOST, a
    import torch

    if isinstance(a, torch.Tensor):
        if not a.is_cuda:
            return _ptr(a.numpy(), dtype)
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None and str(a.dtype).replace("torch.", "") != np.dtype(dtype).name:
            raise TypeError(f"expected {dtype}, got {a.dtype}")
        return C.c_void_p(a.data_ptr()), STM_MEM_DEVICE, a
    raise TypeError(f"unsupported array type {type(a)}")


class Slab:
    """One library context for a mesh (see include/stm.h)."""

    def __init__(self, mesh: dict, precision=STM_FP64, tol=1e-12, restart=10, max_it=500,
                 deterministic=True, stream=None, reorth=True, graph=True, eta_tol=0.0, t_final=0.0,
                 c_diss=0.0, zero_guess=False, tensor_cores=True, cycles_per_launch=1):
        L = lib()
        self._keep = {}
        ne = mesh["hex"].shape[0]
        arr = {
            "vert": np.ascontiguousarray(mesh["vert"], dtype=np.float64),
            "hex": np.ascontiguousarray(mesh["hex"], dtype=np.int64),
            "nbr": np.ascontiguousarray(mesh["nbr"], dtype=np.int64),
            "p": np.ascontiguousarray(np.asarray(mesh["p"]).reshape(ne), dtype=np.uint8),
            "q": np.ascontiguousarray(np.asarray(mesh["q"]).reshape(ne), dtype=np.uint8),
            "eps": np.ascontiguousarray(mesh["eps"], dtype=np.float64),
            "mu": np.ascontiguousarray(mesh["mu"], dtype=np.float64),
            "hang": np.ascontiguousarray(np.asarray(mesh.get("hang", np.zeros((0, 6)))).reshape(-1, 6),
                                         dtype=np.int64),
            "nk": np.ascontiguousarray(np.asarray(mesh.get("nk", np.ones(ne))).reshape(ne), dtype=np.uint8),
        }
        geom = {"brick": STM_GEOM_BRICK, "affine": STM_GEOM_AFFINE,
                "trilinear": STM_GEOM_TRILINEAR}[mesh.get("geometry", "brick")]
        m = stm_mesh(ne, arr["vert"].shape[0],
                     arr["vert"].ctypes.data_as(C.POINTER(C.c_double)),
                     arr["hex"].ctypes.data_as(C.POINTER(C.c_int64)),
                     arr["nbr"].ctypes.data_as(C.POINTER(C.c_int64)),
                     arr["hang"].shape[0], arr["hang"].ctypes.data_as(C.POINTER(C.c_int64)),
                     arr["p"].ctypes.data_as(C.POINTER(C.c_uint8)),
                     arr["q"].ctypes.data_as(C.POINTER(C.c_uint8)),
                     arr["eps"].ctypes.data_as(C.POINTER(C.c_double)),
                     arr["mu"].ctypes.data_as(C.POINTER(C.c_double)), geom,
                     arr["nk"].ctypes.data_as(C.POINTER(C.c_uint8)))
        if stream is None:
            import torch

            stream = torch.cuda.current_stream().cuda_stream
        o = stm_opts(precision, tol, restart, max_it, 1 if deterministic else 0, int(stream), 1 if reorth else 0,
                     1 if graph else 0, eta_tol, t_final, c_diss, 1 if zero_guess else 0,
                     0 if tensor_cores else 1, cycles_per_launch)
        h = C.c_void_p()
        rc = L.stm_create(C.byref(h), C.byref(m), C.byref(o))
        if rc != STM_OK:
            raise StmError(rc, "stm_create failed (see stderr)")
        self.ctx = h
        nt, ns, nst = C.c_int64(), C.c_int64(), C.c_int64()
        L.stm_sizes(h, C.byref(nt), C.byref(ns), C.byref(nst))
        self.n_trial, self.n_test, self.n_state = nt.value, ns.value, nst.value
        self.n_elem = ne

    def close(self):
        if getattr(self, "ctx", None):
            lib().stm_destroy(self.ctx)
            self.ctx = None

    __del__ = close

    def _check(self, rc, ok=(STM_OK,)):
        if rc not in ok:
            raise StmError(rc, lib().stm_last_error(self.ctx).decode())
        return rc

    def residual_apply(self, U, R, t0: float, dt: float, prec=STM_FP64):
        dt_ = np.float64 if prec == STM_FP64 else np.float32
        pu, mu_, _ = _ptr(U, dt_)
        pr, mr, _ = _ptr(R, dt_)
        if mu_ != mr:
            raise ValueError("U and R must both be host or both be device arrays")
        return self._check(lib().stm_residual_apply(self.ctx, t0, dt, pu, pr, prec, mu_))

    def operator_apply(self, V, W, dt: float, pre=True, prec=STM_FP64):
        """W = A P^{-1} V (pre) or A V: the operator of the slab's GMRES, test layout."""
        dt_ = np.float64 if prec == STM_FP64 else np.float32
        pv, mv, _ = _ptr(V, dt_)
        pw, mw, _ = _ptr(W, dt_)
        if mv != mw:
            raise ValueError("V and W must both be host or both be device arrays")
        return self._check(lib().stm_operator_apply(self.ctx, dt, pv, pw, 1 if pre else 0, prec, mv))

    def set_state(self, u, t=0.0):
        p, m, _ = _ptr(u, np.float64)
        return self._check(lib().stm_set_state(self.ctx, t, p, m))

    def get_state(self, out=None):
        out = np.empty(self.n_state) if out is None else out
        p, m, _ = _ptr(out, np.float64)
        t = C.c_double()
        self._check(lib().stm_get_state(self.ctx, C.byref(t), p, m))
        return out, t.value

    def set_initial(self, E0=None, H0=None, t=0.0):
        def wrap(fn):
            if fn is None:
                return C.cast(None, FIELD_FN)

            def cb(_user, n, x, out):
                xs = np.ctypeslib.as_array(x, shape=(n, 3))
                np.ctypeslib.as_array(out, shape=(n, 3))[:] = fn(xs)
            return FIELD_FN(cb)
        e, h = wrap(E0), wrap(H0)
        self._keep["cb"] = (e, h)
        return self._check(lib().stm_set_initial(self.ctx, t, e, h, None))

    def slab_solve(self, dt: float):
        rep = stm_solve_report()
        rc = self._check(lib().stm_slab_solve(self.ctx, dt, C.byref(rep)), ok=(STM_OK, STM_ENOTCONV))
        return rc, {"iterations": rep.iterations, "restarts": rep.restarts,
                    "rel_residual": rep.rel_residual, "energy": rep.energy, "eta2": rep.eta2}

    def energy(self) -> float:
        e = C.c_double()
        self._check(lib().stm_energy(self.ctx, C.byref(e)))
        return e.value

    def autotune(self, dt: float, reps: int = 3):
        """Pick the block size of every (p, q) class; returns [(p, q, block, ms)]."""
        n = 64
        P, Q, B = (C.c_int32 * n)(), (C.c_int32 * n)(), (C.c_int32 * n)()
        ms, cnt = (C.c_double * n)(), C.c_int32()
        self._check(lib().stm_autotune(self.ctx, dt, reps, n, P, Q, B, ms, C.byref(cnt)))
        return [(P[k], Q[k], B[k], ms[k]) for k in range(min(cnt.value, n))]

    def launch_count(self) -> int:
        n = C.c_int64()
        self._check(lib().stm_launch_count(self.ctx, C.byref(n)))
        return n.value

    def profile(self, on: bool):
        return self._check(lib().stm_profile_enable(self.ctx, 1 if on else 0))

    def profile_read(self):
        """{kernel: (total ms, launches)} for the residual kernels since profile(True)."""
        ms = (C.c_double * 4)()
        cnt = (C.c_int64 * 4)()
        self._check(lib().stm_profile_read(self.ctx, ms, cnt))
        names = ("k_prep_fp64", "k_apply_fp64", "k_prep_fp32", "k_apply_fp32")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(names)}

    def set_source_gauss(self, sources):
        """sources: list of dicts with centre, dir, sigma_x, t0, sigma_t, amp (at most 8)."""
        arr = (stm_gauss_src * max(1, len(sources)))()
        for k, sd in enumerate(sources):
            arr[k].centre[:] = list(sd["centre"])
            arr[k].dir[:] = list(sd["dir"])
            arr[k].sigma_x, arr[k].t0 = sd["sigma_x"], sd["t0"]
            arr[k].sigma_t, arr[k].amp = sd["sigma_t"], sd["amp"]
        return self._check(lib().stm_set_source_gauss(self.ctx, arr, len(sources)))

    def set_source(self, J=None):
        """J(x [n,3], t [n]) -> [n,3] current density, sampled on the host; None removes it."""
        if J is None:
            self._keep.pop("J", None)
            return self._check(lib().stm_set_source(self.ctx, C.cast(None, ST_FIELD_FN), None))

        def cb(_user, n, xt, out):
            a = np.ctypeslib.as_array(xt, shape=(n, 4))
            np.ctypeslib.as_array(out, shape=(n, 3))[:] = J(a[:, :3], a[:, 3])
        f = ST_FIELD_FN(cb)
        self._keep["J"] = f
        return self._check(lib().stm_set_source(self.ctx, f, None))

    def dof_layout(self):
        """(trial, test, state) per-element block offsets, each [n_elem + 1]."""
        n = self.n_elem + 1
        out = [np.empty(n, np.int64) for _ in range(3)]
        self._check(lib().stm_dof_layout(self.ctx, *[a.ctypes.data_as(C.POINTER(C.c_int64)) for a in out]))
        return tuple(out)

    def set_boundary(self, g=None):
        """g(x [n,3], t [n]) -> [n,3] boundary data of n x E = n x g; None = PEC."""
        if g is None:
            self._keep.pop("g", None)
            return self._check(lib().stm_set_boundary(self.ctx, C.cast(None, ST_FIELD_FN), None))

        def cb(_user, n, xt, out):
            a = np.ctypeslib.as_array(xt, shape=(n, 4))
            np.ctypeslib.as_array(out, shape=(n, 3))[:] = g(a[:, :3], a[:, 3])
        f = ST_FIELD_FN(cb)
        self._keep["g"] = f
        return self._check(lib().stm_set_boundary(self.ctx, f, None))


def _result_dict(r):
    return {k: getattr(r, k) for k, _ in stm_result._fields_}


class Server:
    """Request server of the C ABI (continuous batching of slab-solve requests)."""

    def __init__(self, workers=4, hbm_budget_bytes=0, precision=STM_FP64, tol=1e-9, restart=10, max_it=2000):
        o = stm_server_opts(workers, hbm_budget_bytes, precision, tol, restart, max_it)
        h = C.c_void_p()
        rc = lib().stm_server_create(C.byref(h), C.byref(o))
        if rc != STM_OK:
            raise StmError(rc, "stm_server_create failed")
        self.h = h

    def submit(self, n, p, q, n_slabs, dt, kind=0, boxes=(), sources=()) -> int:
        r = stm_request()
        r.n, r.p, r.q, r.n_slabs, r.dt, r.kind = n, p, q, n_slabs, dt, kind
        r.n_boxes = len(boxes)
        for k, b in enumerate(boxes):
            r.boxes[k][:] = list(b)
        r.n_src = len(sources)
        for k, sd in enumerate(sources):
            r.src[k].centre[:] = list(sd["centre"])
            r.src[k].dir[:] = list(sd["dir"])
            r.src[k].sigma_x, r.src[k].t0 = sd["sigma_x"], sd["t0"]
            r.src[k].sigma_t, r.src[k].amp = sd["sigma_t"], sd["amp"]
        t = C.c_int64()
        rc = lib().stm_server_submit(self.h, C.byref(r), C.byref(t))
        if rc != STM_OK:
            raise StmError(rc, "stm_server_submit failed")
        return t.value

    def wait(self, ticket, with_state=False):
        r = stm_result()
        lib().stm_server_wait(self.h, ticket, C.byref(r), None)
        state = None
        if with_state and r.n_state > 0 and r.status >= 0:
            state = np.empty(r.n_state)
            lib().stm_server_poll(self.h, ticket, C.byref(r), state.ctypes.data_as(C.c_void_p))
        return _result_dict(r), state

    def stats(self):
        st = stm_stats()
        lib().stm_server_stats(self.h, C.byref(st))
        return {k: getattr(st, k) for k, _ in stm_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().stm_server_destroy(self.h)
            self.h = None

    __del__ = close
