"""Thin ctypes binding of libcmrt (include/cmrt.h).

Argument marshalling only: every step of the lattice update runs in the CUDA
library.  Functions keep the C names; :class:`Lattice` is a convenience
wrapper that takes PyTorch CUDA tensors or NumPy arrays.  If the library has
not been built, loading fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcmrt.so")

CMRT_OK, CMRT_EINVAL, CMRT_ENOMEM, CMRT_ECUDA, CMRT_ENONFINITE, CMRT_ESTATE, CMRT_ETIMEOUT = range(7)
STATUS_NAMES = {0: "CMRT_OK", 1: "CMRT_EINVAL", 2: "CMRT_ENOMEM", 3: "CMRT_ECUDA", 4: "CMRT_ENONFINITE",
                5: "CMRT_ESTATE", 6: "CMRT_ETIMEOUT"}


class cmrt_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("wall_y", ctypes.c_int32),
        ("rho0_r", ctypes.c_double), ("rho0_b", ctypes.c_double),
        ("alpha_r", ctypes.c_double), ("alpha_b", ctypes.c_double),
        ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
        ("lambda3_r", ctypes.c_double), ("lambda3_b", ctypes.c_double),
        ("lambda6", ctypes.c_double), ("lambda7", ctypes.c_double),
        ("g_acc", ctypes.c_double * 2), ("g_vol", ctypes.c_double * 2),
        ("visc_mode", ctypes.c_int32), ("eta", ctypes.c_double),
        ("stencil_order", ctypes.c_int32), ("curvature_mode", ctypes.c_int32),
        ("fixed_K", ctypes.c_double), ("ghost_N_mode", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("diag_every", ctypes.c_int32),
        ("precision_reference", ctypes.c_int32), ("adjoint_fused", ctypes.c_int32),
    ]


# (name, restype, argtypes) of every exported symbol declared in include/cmrt.h
_SIGNATURES = [
    ("cmrt_abi_version", ctypes.c_int32, []),
    ("cmrt_params_size", ctypes.c_size_t, []),
    ("cmrt_params_default", ctypes.c_int, [ctypes.POINTER(cmrt_params), ctypes.c_int32, ctypes.c_int32]),
    ("cmrt_validate", ctypes.c_int, [ctypes.POINTER(cmrt_params)]),
    ("cmrt_init", ctypes.c_int, [ctypes.POINTER(cmrt_params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.POINTER(ctypes.c_void_p)]),
    ("cmrt_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    ("cmrt_set_graph_steps", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("cmrt_get_graph_steps", ctypes.c_int32, [ctypes.c_void_p]),
    ("cmrt_fields", ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 5),
    ("cmrt_diagnostics", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("cmrt_get_populations", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("cmrt_set_populations", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("cmrt_save_bytes", ctypes.c_size_t, [ctypes.c_void_p]),
    ("cmrt_save", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("cmrt_load", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("cmrt_synchronize", ctypes.c_int, [ctypes.c_void_p]),
    ("cmrt_time", ctypes.c_int64, [ctypes.c_void_p]),
    ("cmrt_launch_count", ctypes.c_int64, [ctypes.c_void_p]),
    ("cmrt_device_bytes", ctypes.c_size_t, [ctypes.c_void_p]),
    ("cmrt_diagnostics_noalloc", ctypes.c_int, [ctypes.POINTER(cmrt_params), ctypes.c_void_p,
                                                ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("cmrt_step_vjp", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_double)]),
    ("cmrt_adjoint", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.c_void_p]),
    ("cmrt_destroy", None, [ctypes.c_void_p]),
    ("cmrt_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("cmrt_batch_init", ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(cmrt_params), ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("cmrt_batch_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    ("cmrt_batch_tune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_double)]),
    ("cmrt_batch_set_rows", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32]),
    ("cmrt_batch_get_rows", ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    ("cmrt_batch_set_graph_steps", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    ("cmrt_batch_member", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    ("cmrt_batch_diagnostics", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("cmrt_batch_synchronize", ctypes.c_int, [ctypes.c_void_p]),
    ("cmrt_batch_size", ctypes.c_int32, [ctypes.c_void_p]),
    ("cmrt_batch_time", ctypes.c_int64, [ctypes.c_void_p]),
    ("cmrt_batch_launch_count", ctypes.c_int64, [ctypes.c_void_p]),
    ("cmrt_batch_work_items", ctypes.c_int64, [ctypes.c_void_p]),
    ("cmrt_batch_device_bytes", ctypes.c_size_t, [ctypes.c_void_p]),
    ("cmrt_batch_destroy", None, [ctypes.c_void_p]),
    ("cmrt_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
]

CMRT_TUNE_FORCE = 1

_lib = None
ABI_VERSION = 10  # the layout of cmrt_params and the calls this binding was written for


def load(path: str = LIB_PATH):
    """Load libcmrt.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libcmrt is not built ({path} missing): run __graft_entry__.build() "
                           "or python paper_2005_04642_gb300/build.py")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.cmrt_abi_version() != ABI_VERSION or lib.cmrt_params_size() != ctypes.sizeof(cmrt_params):
        raise RuntimeError(f"libcmrt at {path} has ABI version {lib.cmrt_abi_version()} "
                           f"(params {lib.cmrt_params_size()} B); this binding needs version {ABI_VERSION} "
                           f"({ctypes.sizeof(cmrt_params)} B): rebuild it")
    _lib = lib
    return lib


class CmrtError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status, ctx=None):
    if status != CMRT_OK:
        msg = load().cmrt_last_error(ctx)
        raise CmrtError(status, msg.decode() if msg else "")


def _bcheck(status, batch=None):
    if status != CMRT_OK:
        msg = load().cmrt_batch_last_error(batch)
        raise CmrtError(status, msg.decode() if msg else "")


def make_params(d: dict) -> cmrt_params:
    """cmrt_params from a plain dictionary (keys as in the C struct)."""
    lib = load()
    p = cmrt_params()
    _check(lib.cmrt_params_default(ctypes.byref(p), int(d["nx"]), int(d["ny"])))
    for k, v in d.items():
        if k in ("g_acc", "g_vol"):
            arr = getattr(p, k)
            arr[0], arr[1] = float(v[0]), float(v[1])
        elif k == "wall_y":
            p.wall_y = int(bool(v))
        elif k == "dtype":
            continue
        elif hasattr(p, k):
            ftype = dict(cmrt_params._fields_)[k]
            setattr(p, k, int(v) if ftype is ctypes.c_int32 else float(v))
    return p


# ---------------------------------------------------------------- C-named wrappers
def cmrt_abi_version():
    return load().cmrt_abi_version()


def cmrt_validate(params: cmrt_params):
    return load().cmrt_validate(ctypes.byref(params))


def cmrt_init(params: cmrt_params, rho_n0_ptr: int, u0_ptr: int, stream_ptr: int):
    h = ctypes.c_void_p()
    _check(load().cmrt_init(ctypes.byref(params), rho_n0_ptr or None, u0_ptr or None, stream_ptr or None,
                            ctypes.byref(h)))
    return h


def cmrt_step(ctx, n: int):
    _check(load().cmrt_step(ctx, int(n)), ctx)


def cmrt_fields(ctx, rho_r=0, rho_b=0, ux=0, uy=0, p=0):
    _check(load().cmrt_fields(ctx, rho_r or None, rho_b or None, ux or None, uy or None, p or None), ctx)


def cmrt_diagnostics(ctx):
    out = (ctypes.c_double * 6)()
    st = load().cmrt_diagnostics(ctx, out)
    vals = list(out)
    _check(st, ctx)
    return vals


def cmrt_get_populations(ctx, dst_ptr: int):
    _check(load().cmrt_get_populations(ctx, dst_ptr), ctx)


def cmrt_set_populations(ctx, src_ptr: int):
    _check(load().cmrt_set_populations(ctx, src_ptr), ctx)


def cmrt_synchronize(ctx):
    _check(load().cmrt_synchronize(ctx), ctx)


def cmrt_time(ctx):
    return load().cmrt_time(ctx)


def cmrt_launch_count(ctx):
    return load().cmrt_launch_count(ctx)


def cmrt_device_bytes(ctx):
    return load().cmrt_device_bytes(ctx)


def cmrt_diagnostics_noalloc(params: cmrt_params, pops_ptr: int, stream_ptr: int = 0):
    """Diagnostics of device populations without any allocation (six floats)."""
    out = (ctypes.c_double * 6)()
    st = load().cmrt_diagnostics_noalloc(ctypes.byref(params), pops_ptr, out, stream_ptr or None)
    vals = list(out)
    _check(st)
    return vals


ADJOINT_PARAMS = ("sigma", "beta", "lambda3_r", "lambda3_b", "g_acc_x", "g_acc_y")


def cmrt_step_vjp(ctx, lam_next_ptr: int, lam_ptr: int, grad_params=None):
    """One-step VJP; adds this step's parameter gradient to ``grad_params`` (list of 6) if given."""
    g = (ctypes.c_double * 6)(*(grad_params or [0.0] * 6))
    _check(load().cmrt_step_vjp(ctx, lam_next_ptr, lam_ptr, g), ctx)
    return list(g)


def cmrt_adjoint(ctx, nsteps: int, ckpt_every: int, target_ptr: int, grad_rho_n0_ptr: int = 0):
    """(J, [dJ/dtheta x 6]) of the colour-field mismatch; dJ/drho^N_0 into grad_rho_n0_ptr if given."""
    J = ctypes.c_double(0.0)
    g = (ctypes.c_double * 6)()
    _check(load().cmrt_adjoint(ctx, int(nsteps), int(ckpt_every), target_ptr, ctypes.byref(J), g,
                               grad_rho_n0_ptr or None), ctx)
    return J.value, list(g)


def cmrt_destroy(ctx):
    load().cmrt_destroy(ctx)


def cmrt_last_error(ctx=None):
    msg = load().cmrt_last_error(ctx)
    return msg.decode() if msg else ""


def cmrt_batch_init(params_list, rho_n0_ptrs, u0_ptrs, stream_ptr: int):
    """params_list: sequence of cmrt_params; *_ptrs: sequences of raw pointers (0 = NULL)."""
    n = len(params_list)
    arr = (cmrt_params * n)(*params_list)
    rn = (ctypes.c_void_p * n)(*[p or None for p in rho_n0_ptrs]) if rho_n0_ptrs is not None else None
    uu = (ctypes.c_void_p * n)(*[p or None for p in u0_ptrs]) if u0_ptrs is not None else None
    h = ctypes.c_void_p()
    _bcheck(load().cmrt_batch_init(n, arr, rn, uu, stream_ptr or None, ctypes.byref(h)))
    return h


def cmrt_batch_step(b, n: int):
    _bcheck(load().cmrt_batch_step(b, int(n)), b)


def cmrt_batch_tune(b, cache_path=None, flags: int = 0):
    us = ctypes.c_double(0.0)
    path = cache_path.encode() if cache_path else None
    _bcheck(load().cmrt_batch_tune(b, path, int(flags), ctypes.byref(us)), b)
    return us.value


def cmrt_batch_set_rows(b, nx, ny, wall_y, rows):
    _bcheck(load().cmrt_batch_set_rows(b, int(nx), int(ny), int(wall_y), int(rows)), b)


def cmrt_batch_get_rows(b, nx, ny, wall_y):
    return load().cmrt_batch_get_rows(b, int(nx), int(ny), int(wall_y))


def cmrt_batch_set_graph_steps(b, steps):
    _bcheck(load().cmrt_batch_set_graph_steps(b, int(steps)), b)


def cmrt_batch_member(b, k: int):
    h = ctypes.c_void_p()
    _bcheck(load().cmrt_batch_member(b, int(k), ctypes.byref(h)), b)
    return h


def cmrt_batch_diagnostics(b):
    n = load().cmrt_batch_size(b)
    out = (ctypes.c_double * (6 * n))()
    st = load().cmrt_batch_diagnostics(b, out)
    vals = np.array(list(out)).reshape(n, 6)
    _bcheck(st, b)
    return vals


def cmrt_batch_synchronize(b):
    _bcheck(load().cmrt_batch_synchronize(b), b)


def cmrt_batch_size(b):
    return load().cmrt_batch_size(b)


def cmrt_batch_time(b):
    return load().cmrt_batch_time(b)


def cmrt_batch_launch_count(b):
    return load().cmrt_batch_launch_count(b)


def cmrt_batch_work_items(b):
    return load().cmrt_batch_work_items(b)


def cmrt_batch_device_bytes(b):
    return load().cmrt_batch_device_bytes(b)


def cmrt_batch_destroy(b):
    load().cmrt_batch_destroy(b)


def cmrt_batch_last_error(b=None):
    msg = load().cmrt_batch_last_error(b)
    return msg.decode() if msg else ""


# ---------------------------------------------------------------- convenience wrapper
def _ptr(x):
    """Raw pointer of a torch tensor or NumPy array (must be contiguous float32)."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous() and str(x.dtype) == "torch.float32"
        return x.data_ptr()
    assert x.flags["C_CONTIGUOUS"] and x.dtype == np.float32
    return x.ctypes.data


class Lattice:
    """A two-colour lattice owned by libcmrt.

    ``params`` is a plain dictionary (see :mod:`paper_2005_04642_gb300.inputs`);
    ``rho_n0`` (ny, nx) and ``u0`` (2, ny, nx) are float32 NumPy arrays or CUDA
    tensors.  Work runs on ``stream`` (a torch.cuda.Stream, default: the current
    stream of the current device)."""

    def __init__(self, params: dict, rho_n0=None, u0=None, stream=None):
        import torch
        self.torch = torch
        self.params = dict(params)
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self._p = make_params(params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        keep = []

        def as_f32(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                a = a.to(torch.float32).contiguous()
            else:
                a = np.ascontiguousarray(a, dtype=np.float32)
            keep.append(a)
            return a

        rn = as_f32(rho_n0)
        uu = as_f32(u0)
        self.ctx = cmrt_init(self._p, _ptr(rn), _ptr(uu), self.stream.cuda_stream)
        self._keep = keep  # device inputs must outlive the queued init kernel

    @classmethod
    def _view(cls, ctx, params: dict, stream, owner):
        """A member of a :class:`Batch`: the batch owns the context."""
        self = cls.__new__(cls)
        import torch
        self.torch = torch
        self.params = dict(params)
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self._p = make_params(params)
        self.stream = stream
        self.ctx = ctx
        self._keep = []
        self._owner = owner  # keeps the batch (and so this context) alive
        return self

    def close(self):
        if getattr(self, "_owner", None) is not None:
            self.ctx = None  # a member view: freed with its batch
            self._owner = None
            return
        if getattr(self, "ctx", None):
            cmrt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        cmrt_step(self.ctx, n)

    def set_graph_steps(self, steps: int):
        """Steps per recorded CUDA graph in step() and adjoint() (0: none)."""
        _check(load().cmrt_set_graph_steps(self.ctx, steps), self.ctx)

    @property
    def graph_steps(self):
        return load().cmrt_get_graph_steps(self.ctx)

    def fields(self):
        """dict of (ny, nx) float32 CUDA tensors: rho_r, rho_b, ux, uy, p."""
        t = self.torch
        out = {k: t.empty((self.ny, self.nx), dtype=t.float32, device="cuda") for k in ("rho_r", "rho_b", "ux", "uy", "p")}
        cmrt_fields(self.ctx, *(out[k].data_ptr() for k in ("rho_r", "rho_b", "ux", "uy", "p")))
        return out

    def fields_host(self):
        """Same as :meth:`fields`, written straight into NumPy arrays."""
        out = {k: np.empty((self.ny, self.nx), dtype=np.float32) for k in ("rho_r", "rho_b", "ux", "uy", "p")}
        cmrt_fields(self.ctx, *(out[k].ctypes.data for k in ("rho_r", "rho_b", "ux", "uy", "p")))
        return out

    def diagnostics(self):
        v = cmrt_diagnostics(self.ctx)
        return {"mass_r": v[0], "mass_b": v[1], "mom_x": v[2], "mom_y": v[3], "umax": v[4], "nonfinite": v[5]}

    def populations(self):
        """(2, 9, ny, nx) float32 CUDA tensor of the pre-collision populations."""
        t = self.torch
        out = t.empty((2, 9, self.ny, self.nx), dtype=t.float32, device="cuda")
        cmrt_get_populations(self.ctx, out.data_ptr())
        return out

    def set_populations(self, pops):
        a = pops
        if hasattr(a, "data_ptr"):
            a = a.to(self.torch.float32).contiguous()
        else:
            a = np.ascontiguousarray(a, dtype=np.float32)
        cmrt_set_populations(self.ctx, _ptr(a))
        if hasattr(a, "data_ptr"):
            self.synchronize()

    def synchronize(self):
        cmrt_synchronize(self.ctx)

    def save(self):
        """Checkpoint of the state as stored, with its time (NumPy uint8 array)."""
        lib = load()
        buf = np.empty(lib.cmrt_save_bytes(self.ctx), dtype=np.uint8)
        _check(lib.cmrt_save(self.ctx, buf.ctypes.data, buf.nbytes), self.ctx)
        return buf

    def load(self, buf):
        """Restart from a checkpoint of save() (a NumPy array or a CUDA tensor)."""
        if hasattr(buf, "data_ptr"):
            ptr, n = buf.data_ptr(), buf.numel() * buf.element_size()
        else:
            buf = np.ascontiguousarray(buf, dtype=np.uint8)
            ptr, n = buf.ctypes.data, buf.nbytes
        _check(load().cmrt_load(self.ctx, ptr, n), self.ctx)

    def step_vjp(self, lam_next):
        """dJ/df(t) from dJ/df(t+1) for one step at the current state; returns
        (lam as a (2, 9, ny, nx) CUDA tensor, [dJ/dtheta of this step])."""
        t = self.torch
        a = lam_next.to(device="cuda", dtype=t.float32).contiguous() if hasattr(lam_next, "data_ptr") else \
            t.from_numpy(np.ascontiguousarray(lam_next, dtype=np.float32)).cuda()
        out = t.empty((2, 9, self.ny, self.nx), dtype=t.float32, device="cuda")
        g = cmrt_step_vjp(self.ctx, a.data_ptr(), out.data_ptr())
        return out, g

    def adjoint(self, nsteps: int, target, ckpt_every: int = 200, want_rho_n0: bool = False):
        """Advance nsteps and return (J, {theta: dJ/dtheta}, dJ/drho^N_0 or None) of
        J = 1/2 sum (rho^N - target)^2 at the end."""
        t = self.torch
        tg = target.to(device="cuda", dtype=t.float32).contiguous() if hasattr(target, "data_ptr") else \
            t.from_numpy(np.ascontiguousarray(target, dtype=np.float32)).cuda()
        grn = t.empty((self.ny, self.nx), dtype=t.float32, device="cuda") if want_rho_n0 else None
        J, g = cmrt_adjoint(self.ctx, nsteps, ckpt_every, tg.data_ptr(), grn.data_ptr() if grn is not None else 0)
        return J, dict(zip(ADJOINT_PARAMS, g)), grn

    @property
    def time(self):
        return cmrt_time(self.ctx)

    @property
    def launches(self):
        return cmrt_launch_count(self.ctx)


class Batch:
    """An ensemble of independent lattices stepped by one persistent launch
    per time step (include/cmrt.h, cmrt_batch_*).

    ``members`` is a sequence of (params dict, rho_n0, u0) triples, the arrays
    as for :class:`Lattice` (rho_n0 and u0 may be None)."""

    def __init__(self, members, stream=None):
        import torch
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.params = [dict(m[0]) for m in members]
        keep = []

        def as_f32(a):
            if a is None:
                return 0
            if hasattr(a, "data_ptr"):
                a = a.to(torch.float32).contiguous()
            else:
                a = np.ascontiguousarray(a, dtype=np.float32)
            keep.append(a)
            return _ptr(a)

        rn = [as_f32(m[1]) for m in members]
        uu = [as_f32(m[2]) for m in members]
        self.b = cmrt_batch_init([make_params(p) for p in self.params], rn, uu, self.stream.cuda_stream)
        self._keep = keep
        self._views = {}

    def close(self):
        if getattr(self, "b", None):
            for v in self._views.values():
                v.ctx = None
                v._owner = None
            self._views = {}
            cmrt_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return cmrt_batch_size(self.b)

    def step(self, n: int = 1):
        cmrt_batch_step(self.b, n)

    def tune(self, cache_path=None, force=False):
        """Autotune rows per size class; returns the best time of one batched step in us."""
        return cmrt_batch_tune(self.b, cache_path, CMRT_TUNE_FORCE if force else 0)

    def set_rows(self, nx, ny, wall_y, rows):
        cmrt_batch_set_rows(self.b, nx, ny, wall_y, rows)

    def get_rows(self, nx, ny, wall_y=0):
        return cmrt_batch_get_rows(self.b, nx, ny, wall_y)

    def set_graph_steps(self, steps):
        cmrt_batch_set_graph_steps(self.b, steps)

    def member(self, k: int) -> Lattice:
        """Lattice view of member k (fields, diagnostics, populations; no step)."""
        if k not in self._views:
            ctx = cmrt_batch_member(self.b, k)
            self._views[k] = Lattice._view(ctx, self.params[k], self.stream, self)
        return self._views[k]

    def diagnostics(self):
        """(n, 6) array: mass_r, mass_b, mom_x, mom_y, max|u|, non-finite count per member."""
        return cmrt_batch_diagnostics(self.b)

    def synchronize(self):
        cmrt_batch_synchronize(self.b)

    @property
    def time(self):
        return cmrt_batch_time(self.b)

    @property
    def launches(self):
        return cmrt_batch_launch_count(self.b)

    @property
    def work_items(self):
        return cmrt_batch_work_items(self.b)

    @property
    def device_bytes(self):
        return cmrt_batch_device_bytes(self.b)


def colour_mismatch(theta, rho_n0, params: dict, target, nsteps: int, ckpt_every: int = 200, u0=None):
    """J = 1/2 sum_r (rho^N(r, nsteps) - target(r))^2 as a differentiable torch
    function of theta = (sigma, beta, lambda3_r, lambda3_b, g_acc_x, g_acc_y)
    (float64 tensor) and of the initial colour field rho_n0 (float32 CUDA
    tensor).  The forward and the adjoint both run in libcmrt."""
    return _ColourMismatch.apply(theta, rho_n0, params, target, nsteps, ckpt_every, u0)


def _autograd_function():
    import torch

    class ColourMismatch(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, rho_n0, params, target, nsteps, ckpt_every, u0):
            th = [float(v) for v in theta.detach().cpu().tolist()]
            d = dict(params)
            d.update(sigma=th[0], beta=th[1], lambda3_r=th[2], lambda3_b=th[3], g_acc=(th[4], th[5]))
            lat = Lattice(d, rho_n0.detach(), u0)
            J, g, grn = lat.adjoint(nsteps, target, ckpt_every=ckpt_every, want_rho_n0=True)
            lat.close()
            ctx.save_for_backward(torch.tensor([g[k] for k in ADJOINT_PARAMS], dtype=torch.float64), grn)
            ctx.theta_device = theta.device
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            g, grn = ctx.saved_tensors
            gJ = gJ.detach().to(torch.float64).cpu()
            return (gJ * g).to(ctx.theta_device), (grn * float(gJ)), None, None, None, None, None

    return ColourMismatch


class _Lazy:
    fn = None

    def apply(self, *args):
        if _Lazy.fn is None:
            _Lazy.fn = _autograd_function()
        return _Lazy.fn.apply(*args)


_ColourMismatch = _Lazy()
