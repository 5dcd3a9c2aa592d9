"""Thin Python binding of the swm C ABI (include/swm.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Inputs may be NumPy arrays (host
memory) or CUDA torch tensors (device memory); outputs are written into caller-provided arrays or
tensors, or returned as new NumPy arrays by the ``swm_get_*`` helpers.  Negative status codes
raise :class:`SwmError`; SWM_ENOTCONV is returned as a warning code.  There is no fallback: if
the CUDA library cannot be built or loaded, every call fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SWM_OK, SWM_ENOTCONV = 0, 1
SWM_SOLVER_GMRES, SWM_SOLVER_GCR, SWM_SOLVER_BICGSTAB = 0, 1, 2
SWM_EINVAL, SWM_ENOMEM, SWM_ECUDA, SWM_ESTATE, SWM_ETIMEOUT = -1, -2, -3, -4, -5
SWM_HOST, SWM_DEVICE = 0, 1
SWM_C128, SWM_C64, SWM_BF16 = 0, 1, 2
SWM_MAX_SEG = 16
SWM_MAX_RESTART = 128

_lib = None


class SwmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"swm error {code}: {msg}")
        self.code = code


class swm_stats(C.Structure):
    _fields_ = [("nw", C.c_int64), ("n", C.c_int64), ("nb", C.c_int64), ("nnz", C.c_int64),
                ("n_rhs", C.c_int), ("iterations", C.c_int), ("restarts", C.c_int), ("converged", C.c_int),
                ("rel_residual", C.c_double), ("ms_neighbour", C.c_double), ("ms_fill", C.c_double),
                ("ms_precond", C.c_double), ("ms_rhs", C.c_double), ("ms_solve", C.c_double),
                ("ms_rcs", C.c_double), ("kernel_launches", C.c_int64), ("fill_evals", C.c_int64),
                ("nnz_offd", C.c_int64), ("ncm_offd", C.c_int64), ("prof_ms", C.c_double),
                ("prof_launches", C.c_int64), ("pattern_reused", C.c_int),
                ("step_rhs_block", C.c_int), ("nminv", C.c_int64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_P = C.c_void_p
_SIGS = {
    "swm_version": (C.c_char_p, []),
    "swm_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "swm_destroy": (None, [_P]),
    "swm_last_error": (C.c_char_p, [_P]),
    "swm_set_allocator": (C.c_int, [_P, ALLOC_FN, FREE_FN, _P]),
    "swm_set_cloud": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_int]),
    "swm_build": (C.c_int, [_P, C.c_double, C.c_double, C.c_int]),
    "swm_set_solver": (C.c_int, [_P, C.c_int]),
    "swm_solve": (C.c_int, [_P, C.c_int, _P, C.c_double, C.c_int, C.c_int, _P, C.c_int]),
    "swm_rcs_bistatic": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "swm_rcs_monostatic": (C.c_int, [_P, _P, C.c_int]),
    "swm_run": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, _P,
                          C.c_double, C.c_int, C.c_int, C.c_int, _P, _P, C.c_int]),
    "swm_get_stats": (C.c_int, [_P, C.POINTER(swm_stats)]),
    "swm_profile": (C.c_int, [_P, C.c_int]),
    "swm_get_pattern": (C.c_int, [_P, _P]),
    "swm_get_block": (C.c_int, [_P, C.c_int64, C.c_int64, _P]),
    "swm_get_rhs": (C.c_int, [_P, _P]),
    "swm_far_field": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_double, C.c_int, _P, C.c_int, _P, _P]),
    "swm_far_field_noalloc": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_double, C.c_int, _P, C.c_int, _P,
                                         _P]),
    "swm_stateless_error": (C.c_char_p, []),
    "swm_far_components": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_double, C.c_int, _P, C.c_int, _P, _P]),
    "swm_apply": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, C.c_int]),
    "swm_precond_apply": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, C.c_int]),
    "swm_rhs": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "swm_vec_dots": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, _P, _P, _P]),
    "swm_vec_axpy": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, _P, _P, _P]),
    "swm_vec_scale": (C.c_int, [_P, C.c_int64, C.c_int, _P, _P, _P]),
    "swm_vec_gram": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, _P, _P, _P]),
    "swm_vec_gemm": (C.c_int, [_P, C.c_int64, C.c_int, C.c_int, _P, _P, _P]),
    "swm_solve_guess": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, C.c_double, C.c_int, C.c_int, _P, C.c_int]),
    "swm_net_num_params": (C.c_int64, []),
    "swm_net_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "swm_net_destroy": (None, [_P]),
    "swm_net_last_error": (C.c_char_p, [_P]),
    "swm_net_set_params": (C.c_int, [_P, _P, C.c_int]),
    "swm_net_get_params": (C.c_int, [_P, _P, C.c_int]),
    "swm_net_predict": (C.c_int, [_P, _P, C.c_int, _P, _P, C.c_int]),
    "swm_net_train_step": (C.c_int, [_P, _P, C.c_int, _P, _P, C.c_int, C.c_float, _P, _P]),
}
EXPORTED = tuple(_SIGS)


def load(build: bool = True):
    """Load libswm.so (building it first when missing or stale)."""
    global _lib
    if _lib is None:
        if build:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: the CUDA library was not built")
        lib = C.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


# ------------------------------------------------------------------------------ marshalling
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype, shape=None, name="array"):
    """(pointer, mem_kind, keepalive) of a contiguous host NumPy array or CUDA torch tensor."""
    if _is_torch(x):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64,
               np.complex128: torch.complex128}[dtype]
        if x.dtype != tdt or not x.is_contiguous() or not x.is_cuda:
            raise TypeError(f"{name}: need a contiguous CUDA tensor of {tdt}")
        if shape is not None and tuple(x.shape) != tuple(shape):
            raise ValueError(f"{name}: shape {tuple(x.shape)} != {tuple(shape)}")
        return C.c_void_p(x.data_ptr()), SWM_DEVICE, x
    a = np.ascontiguousarray(x, dtype=dtype)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"{name}: shape {a.shape} != {tuple(shape)}")
    return a.ctypes.data_as(C.c_void_p), SWM_HOST, a


def _out_ptr(x, dtype, shape, name):
    if _is_torch(x):
        return _ptr(x, dtype, shape, name)
    if not (isinstance(x, np.ndarray) and x.dtype == dtype and x.flags.c_contiguous and x.shape == tuple(shape)):
        raise TypeError(f"{name}: need a C-contiguous {np.dtype(dtype).name} array of shape {tuple(shape)}")
    return x.ctypes.data_as(C.c_void_p), SWM_HOST, x


def _check(ctx, rc):
    if rc < 0:
        raise SwmError(rc, swm_last_error(ctx))
    return rc


def _torch_stream_handle():
    import torch
    return torch.cuda.current_stream().cuda_stream


# ------------------------------------------------------------------------------ context API
class Ctx:
    """Opaque context handle plus the Python objects that must outlive it."""

    def __init__(self, handle, device, stream):
        self.handle = handle
        self.device = device
        self.stream = stream
        self._keep = []

    @property
    def _as_parameter_(self):
        return self.handle


def swm_version() -> str:
    return load().swm_version().decode()


def swm_create(device: int = 0, stream=None, torch_allocator: bool = True) -> Ctx:
    """Create a context on ``device`` issuing work on ``stream`` (a cudaStream_t handle; default:
    torch's current stream).  With ``torch_allocator`` the device memory comes from torch's
    caching allocator."""
    lib = load()
    if stream is None:
        stream = _torch_stream_handle()
    h = C.c_void_p()
    rc = lib.swm_create(C.byref(h), int(device), C.c_void_p(stream))
    if rc < 0:
        raise SwmError(rc, "swm_create failed (no CUDA device?)")
    ctx = Ctx(h, device, stream)
    if torch_allocator:
        swm_set_allocator(ctx)
    return ctx


def swm_destroy(ctx: Ctx) -> None:
    if ctx is not None and ctx.handle:
        load().swm_destroy(ctx.handle)
        ctx.handle = None


def swm_last_error(ctx) -> str:
    h = ctx.handle if isinstance(ctx, Ctx) else ctx
    return load().swm_last_error(h).decode()


def swm_set_allocator(ctx: Ctx) -> int:
    """Route the context's device allocations through torch's caching allocator."""
    import torch

    dev = ctx.device

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
    ctx._keep += [fa, ff]
    return _check(ctx, load().swm_set_allocator(ctx.handle, fa, ff, None))


def swm_set_cloud(ctx: Ctx, centres, dirs, lengths, radii, nseg) -> int:
    nw = len(lengths)
    pc, k1, a1 = _ptr(centres, np.float64, (nw, 3), "centres")
    pt, k2, a2 = _ptr(dirs, np.float64, (nw, 3), "dirs")
    pl, k3, a3 = _ptr(lengths, np.float64, (nw,), "lengths")
    pr, k4, a4 = _ptr(radii, np.float64, (nw,), "radii")
    pn, k5, a5 = _ptr(nseg, np.int32, (nw,), "nseg")
    if len({k1, k2, k3, k4, k5}) != 1:
        raise TypeError("swm_set_cloud: all inputs must be host arrays or all device tensors")
    return _check(ctx, load().swm_set_cloud(ctx.handle, nw, pc, pt, pl, pr, pn, k1))


def swm_build(ctx: Ctx, k: float, r_c: float, precision: int = SWM_C128) -> int:
    return _check(ctx, load().swm_build(ctx.handle, float(k), float(r_c), int(precision)))


def swm_set_solver(ctx: Ctx, method) -> int:
    """Krylov method of the following solves: "gmres" / SWM_SOLVER_GMRES, "gcr" / SWM_SOLVER_GCR or
    "bicgstab" / SWM_SOLVER_BICGSTAB."""
    m = ({"gmres": SWM_SOLVER_GMRES, "gcr": SWM_SOLVER_GCR, "bicgstab": SWM_SOLVER_BICGSTAB}[method]
         if isinstance(method, str) else int(method))
    return _check(ctx, load().swm_set_solver(ctx.handle, m))


def swm_solve(ctx: Ctx, inc, tol: float = 1e-6, restart: int = 50, max_iter: int = 1000, currents_out=None) -> int:
    inc = np.ascontiguousarray(np.atleast_2d(inc), dtype=np.float64)
    n_inc = inc.shape[0]
    if currents_out is None:
        pc, kind = None, SWM_HOST
    else:
        n = swm_get_stats(ctx)["n"]
        pc, kind, _ = _out_ptr(currents_out, np.complex128, (n_inc, n), "currents_out")
    return _check(ctx, load().swm_solve(ctx.handle, n_inc, inc.ctypes.data_as(C.c_void_p), float(tol), int(restart),
                                        int(max_iter), pc, kind))


def swm_solve_guess(ctx: Ctx, inc, x0, tol: float = 1e-6, restart: int = 50, max_iter: int = 1000,
                    currents_out=None) -> int:
    """swm_solve starting from the initial guess x0 (n_inc x N complex128, caller order)."""
    inc = np.ascontiguousarray(np.atleast_2d(inc), dtype=np.float64)
    n_inc = inc.shape[0]
    n = swm_get_stats(ctx)["n"]
    if _is_torch(x0):
        px, xk, _ = _ptr(x0, np.complex128, (n_inc, n), "x0")
    else:
        x0 = np.ascontiguousarray(x0, dtype=np.complex128).reshape(n_inc, n)
        px, xk = x0.ctypes.data_as(C.c_void_p), SWM_HOST
    if currents_out is None:
        pc, kind = None, SWM_HOST
    else:
        pc, kind, _ = _out_ptr(currents_out, np.complex128, (n_inc, n), "currents_out")
    return _check(ctx, load().swm_solve_guess(ctx.handle, n_inc, inc.ctypes.data_as(C.c_void_p), px, xk, float(tol),
                                              int(restart), int(max_iter), pc, kind))


class Net:
    """Handle of the warm-start network (see swm_net_* in include/swm.h)."""

    def __init__(self, handle, device):
        self.handle = handle
        self.device = device


def _net_check(net, rc):
    if rc < 0:
        raise SwmError(rc, load().swm_net_last_error(net.handle).decode())
    return rc


def swm_net_num_params() -> int:
    return int(load().swm_net_num_params())


def swm_net_create(device: int = 0, stream=None) -> Net:
    lib = load()
    if stream is None:
        stream = _torch_stream_handle()
    h = C.c_void_p()
    rc = lib.swm_net_create(C.byref(h), int(device), C.c_void_p(stream))
    if rc < 0:
        raise SwmError(rc, "swm_net_create failed")
    return Net(h, device)


def swm_net_destroy(net: Net) -> None:
    if net is not None and net.handle:
        load().swm_net_destroy(net.handle)
        net.handle = None


def swm_net_set_params(net: Net, params) -> int:
    p = np.ascontiguousarray(params, dtype=np.float32).ravel()
    if p.size != swm_net_num_params():
        raise ValueError("wrong parameter count")
    return _net_check(net, load().swm_net_set_params(net.handle, p.ctypes.data_as(C.c_void_p), SWM_HOST))


def swm_net_get_params(net: Net) -> np.ndarray:
    p = np.zeros(swm_net_num_params(), dtype=np.float32)
    _net_check(net, load().swm_net_get_params(net.handle, p.ctypes.data_as(C.c_void_p), SWM_HOST))
    return p


def swm_net_predict(net: Net, ctx: Ctx, inc, x0_out=None):
    """Predicted currents (n_inc x N complex128, caller order); into x0_out if given."""
    inc = np.ascontiguousarray(np.atleast_2d(inc), dtype=np.float64)
    n_inc, n = inc.shape[0], swm_get_stats(ctx)["n"]
    if x0_out is None:
        x0_out = np.zeros((n_inc, n), dtype=np.complex128)
    px, kind, _ = _out_ptr(x0_out, np.complex128, (n_inc, n), "x0_out")
    _net_check(net, load().swm_net_predict(net.handle, ctx.handle, n_inc, inc.ctypes.data_as(C.c_void_p), px, kind))
    return x0_out


def swm_net_train_step(net: Net, ctx: Ctx, inc, x_true, lr: float = 0.0, want_grad: bool = False):
    """Loss of the prediction against x_true (n_inc x N complex128, caller order); with lr > 0 one
    Adam step.  Returns (loss, gradient or None)."""
    inc = np.ascontiguousarray(np.atleast_2d(inc), dtype=np.float64)
    n_inc, n = inc.shape[0], swm_get_stats(ctx)["n"]
    if _is_torch(x_true):
        pt, kind, _ = _ptr(x_true, np.complex128, (n_inc, n), "x_true")
    else:
        x_true = np.ascontiguousarray(x_true, dtype=np.complex128).reshape(n_inc, n)
        pt, kind = x_true.ctypes.data_as(C.c_void_p), SWM_HOST
    loss = C.c_double()
    g = np.zeros(swm_net_num_params(), dtype=np.float32) if want_grad else None
    pg = g.ctypes.data_as(C.c_void_p) if want_grad else None
    _net_check(net, load().swm_net_train_step(net.handle, ctx.handle, n_inc, inc.ctypes.data_as(C.c_void_p), pt, kind,
                                              float(lr), C.byref(loss), pg))
    return loss.value, g


def swm_rcs_bistatic(ctx: Ctx, obs, sigma_out) -> int:
    obs = np.ascontiguousarray(np.atleast_2d(obs), dtype=np.float64)
    n_inc = swm_get_stats(ctx)["n_rhs"]
    ps, kind, _ = _out_ptr(sigma_out, np.float64, (n_inc, obs.shape[0], 2), "sigma_out")
    return _check(ctx, load().swm_rcs_bistatic(ctx.handle, obs.shape[0], obs.ctypes.data_as(C.c_void_p), ps, kind))


def swm_rcs_monostatic(ctx: Ctx, sigma_out) -> int:
    n_inc = swm_get_stats(ctx)["n_rhs"]
    ps, kind, _ = _out_ptr(sigma_out, np.float64, (n_inc, 2), "sigma_out")
    return _check(ctx, load().swm_rcs_monostatic(ctx.handle, ps, kind))


def swm_run(ctx: Ctx, centres, dirs, lengths, radii, nseg, k: float, r_c: float, precision: int, inc, obs,
            sigma_out, tol: float = 1e-6, restart: int = 50, max_iter: int = 1000) -> int:
    """swm_set_cloud, swm_build, swm_solve and swm_rcs_bistatic in one call (synchronising only
    where the host needs device results); sigma_out as for swm_rcs_bistatic.  With ``obs`` None
    the RCS is monostatic and sigma_out is n_inc x 2, as for swm_rcs_monostatic."""
    nw = len(lengths)
    pc, k1, a1 = _ptr(centres, np.float64, (nw, 3), "centres")
    pt, k2, a2 = _ptr(dirs, np.float64, (nw, 3), "dirs")
    pl, k3, a3 = _ptr(lengths, np.float64, (nw,), "lengths")
    pr, k4, a4 = _ptr(radii, np.float64, (nw,), "radii")
    pn, k5, a5 = _ptr(nseg, np.int32, (nw,), "nseg")
    if len({k1, k2, k3, k4, k5}) != 1:
        raise TypeError("swm_run: all cloud inputs must be host arrays or all device tensors")
    inc = np.ascontiguousarray(np.atleast_2d(inc), dtype=np.float64)
    if obs is None:
        n_obs, pobs = 0, None
        ps, kind, _ = _out_ptr(sigma_out, np.float64, (inc.shape[0], 2), "sigma_out")
    else:
        obs = np.ascontiguousarray(np.atleast_2d(obs), dtype=np.float64)
        n_obs, pobs = obs.shape[0], obs.ctypes.data_as(C.c_void_p)
        ps, kind, _ = _out_ptr(sigma_out, np.float64, (inc.shape[0], n_obs, 2), "sigma_out")
    return _check(ctx, load().swm_run(ctx.handle, nw, pc, pt, pl, pr, pn, k1, float(k), float(r_c), int(precision),
                                      inc.shape[0], inc.ctypes.data_as(C.c_void_p), float(tol), int(restart),
                                      int(max_iter), n_obs, pobs, ps, kind))


def swm_get_stats(ctx: Ctx) -> dict:
    s = swm_stats()
    _check(ctx, load().swm_get_stats(ctx.handle, C.byref(s)))
    return {name: getattr(s, name) for name, _ in swm_stats._fields_}


SWM_K = {"none": 0, "pairs": 1, "fill_self": 2, "fill_mutual": 3, "invert": 4, "form_e": 5, "rhs": 6,
         "apply": 7, "dots": 8, "update": 9, "finish": 10, "far": 11, "gmres": 12, "transpose": 13}


def swm_profile(ctx: Ctx, kernel_class) -> int:
    """Time every launch of one kernel class (name from SWM_K or its number) with CUDA events."""
    kc = SWM_K[kernel_class] if isinstance(kernel_class, str) else int(kernel_class)
    return _check(ctx, load().swm_profile(ctx.handle, kc))


def swm_get_pattern(ctx: Ctx) -> np.ndarray:
    nb = swm_get_stats(ctx)["nb"]
    out = np.zeros((nb, 2), dtype=np.int64)
    _check(ctx, load().swm_get_pattern(ctx.handle, out.ctypes.data_as(C.c_void_p)))
    return out


def swm_get_block(ctx: Ctx, p: int, q: int, mp: int, mq: int) -> np.ndarray:
    out = np.zeros((mp, mq), dtype=np.complex128)
    _check(ctx, load().swm_get_block(ctx.handle, int(p), int(q), out.ctypes.data_as(C.c_void_p)))
    return out


def swm_get_rhs(ctx: Ctx) -> np.ndarray:
    st = swm_get_stats(ctx)
    out = np.zeros((st["n_rhs"], st["n"]), dtype=np.complex128)
    _check(ctx, load().swm_get_rhs(ctx.handle, out.ctypes.data_as(C.c_void_p)))
    return out


def swm_far_field(stream, centres, dirs, lengths, nseg, off, k, currents, obs, sigma_out, _entry="swm_far_field") -> int:
    """Stateless far-field RCS; every array a CUDA torch tensor (see include/swm.h).  Host arrays
    are refused (the C entry point takes device pointers only)."""
    nw = lengths.shape[0]
    n_rhs, n_obs = currents.shape[0], obs.shape[0]
    out_conv = (_ptr(sigma_out, np.complex128, (n_rhs, n_obs, 2), "comp_out") if _entry == "swm_far_components"
                else _ptr(sigma_out, np.float64, (n_rhs, n_obs, 2), "sigma_out"))
    conv = [_ptr(centres, np.float64, (nw, 3), "centres"), _ptr(dirs, np.float64, (nw, 3), "dirs"),
            _ptr(lengths, np.float64, (nw,), "lengths"), _ptr(nseg, np.int32, (nw,), "nseg"),
            _ptr(off, np.int64, (nw + 1,), "off"), _ptr(currents, np.complex128, None, "currents"),
            _ptr(obs, np.float64, (n_obs, 2), "obs"), out_conv]
    names = ("centres", "dirs", "lengths", "nseg", "off", "currents", "obs", "sigma_out")
    for name, (_, kind, _) in zip(names, conv):
        if kind != SWM_DEVICE:
            raise TypeError(f"{_entry}: {name} must be a CUDA tensor (device memory)")
    keep = [c[2] for c in conv]  # the converted objects stay alive until the call returns
    ptrs = [c[0] for c in conv]
    if stream is None:
        stream = _torch_stream_handle()
    lib = load()
    rc = getattr(lib, _entry)(C.c_void_p(stream), nw, *ptrs[:5], float(k), n_rhs, ptrs[5], n_obs, ptrs[6], ptrs[7])
    del keep
    if rc < 0:
        raise SwmError(rc, lib.swm_stateless_error().decode())
    return rc


def swm_far_components(stream, centres, dirs, lengths, nseg, off, k, currents, obs, comp_out) -> int:
    """Received far-field components theta_hat . F and phi_hat . F of the given currents
    (n_rhs x n_obs x 2 complex128, CUDA tensors throughout, see include/swm.h); they add over
    disjoint sets of wires."""
    return swm_far_field(stream, centres, dirs, lengths, nseg, off, k, currents, obs, comp_out,
                         _entry="swm_far_components")


def _dev_c128(x, shape, name):
    if not _is_torch(x):
        raise TypeError(f"{name}: need a CUDA tensor")
    return _ptr(x, np.complex128, shape, name)[0]


def swm_apply(ctx: Ctx, x, y) -> int:
    """y = (I + E) x = Z M^-1 x for every local row (n_rhs x N complex128, caller order)."""
    n = swm_get_stats(ctx)["n"]
    R = x.shape[0]
    px, kx, _ = _ptr(x, np.complex128, (R, n), "x")
    py, ky, _ = _out_ptr(y, np.complex128, (R, n), "y")
    return _check(ctx, load().swm_apply(ctx.handle, R, px, kx, py, ky))


def swm_precond_apply(ctx: Ctx, y, x) -> int:
    """x = M^-1 y, the self-block inverses wire by wire (n_rhs x N complex128, caller order)."""
    n = swm_get_stats(ctx)["n"]
    R = y.shape[0]
    py, ky, _ = _ptr(y, np.complex128, (R, n), "y")
    px, kx, _ = _out_ptr(x, np.complex128, (R, n), "x")
    return _check(ctx, load().swm_precond_apply(ctx.handle, R, py, ky, px, kx))


def swm_rhs(ctx: Ctx, inc, b_out) -> int:
    """Right-hand sides (Eq. (4)) of the built system for the given incidences, n_inc x N."""
    inc = np.ascontiguousarray(np.atleast_2d(inc), dtype=np.float64)
    n = swm_get_stats(ctx)["n"]
    pb, kb, _ = _out_ptr(b_out, np.complex128, (inc.shape[0], n), "b_out")
    return _check(ctx, load().swm_rhs(ctx.handle, inc.shape[0], inc.ctypes.data_as(C.c_void_p), pb, kb))


def swm_vec_dots(ctx: Ctx, Vb, k: int, w) -> np.ndarray:
    """(k x n_rhs) complex inner products Vb[i][r]^H w[r] for i < k; Vb (>= k, n_rhs, n) and w
    (n_rhs, n) CUDA complex128 tensors."""
    R, n = w.shape
    if Vb.shape[0] < k or tuple(Vb.shape[1:]) != (R, n) or not Vb.is_contiguous():
        raise ValueError("swm_vec_dots: basis shape")
    out = np.zeros((k, R), dtype=np.complex128)
    _check(ctx, load().swm_vec_dots(ctx.handle, n, int(k), R, C.c_void_p(Vb.data_ptr()), _dev_c128(w, (R, n), "w"),
                                    out.ctypes.data_as(C.c_void_p)))
    return out


def swm_vec_axpy(ctx: Ctx, Vb, k: int, coef, v) -> int:
    """v[r] -= sum over i < k of coef[i][r] Vb[i][r] (coef host k x n_rhs complex)."""
    R, n = v.shape
    if Vb.shape[0] < k or tuple(Vb.shape[1:]) != (R, n) or not Vb.is_contiguous():
        raise ValueError("swm_vec_axpy: basis shape")
    c = np.ascontiguousarray(coef, dtype=np.complex128).reshape(k, R)
    return _check(ctx, load().swm_vec_axpy(ctx.handle, n, int(k), R, C.c_void_p(Vb.data_ptr()),
                                           c.ctypes.data_as(C.c_void_p), _dev_c128(v, (R, n), "v")))


def swm_vec_scale(ctx: Ctx, a, v, out) -> int:
    """out[r] = a[r] v[r] (a host float64 per right-hand side)."""
    R, n = v.shape
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(R)
    return _check(ctx, load().swm_vec_scale(ctx.handle, n, R, a.ctypes.data_as(C.c_void_p), _dev_c128(v, (R, n), "v"),
                                            _dev_c128(out, (R, n), "out")))


def swm_vec_gram(ctx: Ctx, Vb, k: int, w) -> np.ndarray:
    """((k S) x S) complex inner products conj(Q[a]) . w[b] of the first k S vectors of Vb
    (a (>= k, S, n) CUDA complex128 tensor) with the S vectors of w (S, n)."""
    S, n = w.shape
    if Vb.shape[0] < k or tuple(Vb.shape[1:]) != (S, n) or not Vb.is_contiguous():
        raise ValueError("swm_vec_gram: basis shape")
    out = np.zeros((k * S, S), dtype=np.complex128)
    _check(ctx, load().swm_vec_gram(ctx.handle, n, int(k * S), S, C.c_void_p(Vb.data_ptr()), _dev_c128(w, (S, n), "w"),
                                    out.ctypes.data_as(C.c_void_p)))
    return out


def swm_vec_gemm(ctx: Ctx, Vb, k: int, coef, w) -> int:
    """w[b] -= sum over a < k S of Q[a] coef[a][b] (coef host (k S) x S complex)."""
    S, n = w.shape
    if Vb.shape[0] < k or tuple(Vb.shape[1:]) != (S, n) or not Vb.is_contiguous():
        raise ValueError("swm_vec_gemm: basis shape")
    c = np.ascontiguousarray(coef, dtype=np.complex128).reshape(k * S, S)
    return _check(ctx, load().swm_vec_gemm(ctx.handle, n, int(k * S), S, C.c_void_p(Vb.data_ptr()),
                                           c.ctypes.data_as(C.c_void_p), _dev_c128(w, (S, n), "w")))


def swm_far_field_noalloc(stream, centres, dirs, lengths, nseg, off, k, currents, obs, sigma_out) -> int:
    """Allocation-free far-field RCS for callers that cannot allocate device memory at call time;
    same arguments and results as :func:`swm_far_field`, scratch from a fixed 8 MiB array in the
    library (at most 174762 incidence-observation pairs per call; overlapping calls race)."""
    return swm_far_field(stream, centres, dirs, lengths, nseg, off, k, currents, obs, sigma_out,
                         _entry="swm_far_field_noalloc")
