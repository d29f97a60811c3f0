"""GB300-native Laplace-preconditioned CG / Chebyshev solver for the
axisymmetric elliptic equation of arXiv 1002.3094 (Terekhov).

A thin ctypes binding of ``libaxpcg.so`` (``include/axpcg.h``): the functions
below carry the C ABI's names and only marshal arguments; every step of the
solve runs in the library's CUDA kernels.  There is no CPU fallback: loading
fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

from .build import LIB, build  # noqa: F401

AX_OK = 0
AX_ERR_INVALID_ARG = 1
AX_ERR_NO_CONVERGENCE = 2
AX_ERR_BREAKDOWN = 3
AX_ERR_TIMEOUT = 4
AX_ERR_OOM = 5
AX_ERR_CUDA = 6
AX_ERR_UNSUPPORTED = 7

AX_PCG_FP64 = 0
AX_CHEB_FP64 = 1
AX_PCG_MIXED = 2
AX_CHEB_MIXED = 3

AX_FLAG_USE_GUESS = 1
AX_FLAG_HOST_BUFFERS = 4
AX_FLAG_CHECK_GUESS = 8
AX_FLAG_SERIAL_GROUPS = 16

AX_PREC_FP64 = 0
AX_PREC_FP32 = 1
AX_PREC_FP32_TC = 2
AX_PREC_FP32_TC3 = 3

METHODS = {"pcg64": AX_PCG_FP64, "cheb64": AX_CHEB_FP64, "pcg_mixed": AX_PCG_MIXED,
           "cheb_mixed": AX_CHEB_MIXED}

EXPORTED = ("ax_setup_operator", "ax_destroy_operator", "ax_operator_info", "ax_set_option", "ax_solve",
            "ax_apply_operator", "ax_apply_dst", "ax_apply_dst_inverse", "ax_apply_mode_solve",
            "ax_apply_preconditioner", "ax_status_string", "ax_version", "ax_kernel_launches", "ax_profile_read",
            "ax_apply_preconditioner_noalloc", "ax_laguerre_step", "ax_batch_create", "ax_batch_solve", "ax_batch_latency",
            "ax_batch_destroy", "ax_solve_batched", "ax_last_error",
            "ax_guessnet_create", "ax_guessnet_destroy", "ax_guessnet_num_params", "ax_guessnet_get_params",
            "ax_guessnet_set_params", "ax_guessnet_forward", "ax_guessnet_gradients", "ax_guessnet_train_step",
            "ax_guessnet_save", "ax_guessnet_load", "ax_guessnet_features", "ax_guessnet_lift",
            "ax_guessnet_set_loss", "ax_guessnet_features_pre", "ax_chebyshev_bounds", "ax_get_option",
            "ax_autotune", "ax_batch_autotune", "ax_batch_config", "ax_solve_learned")

PROFILE_KINDS = {"stencil": 0, "dst_forward": 1, "mode_solve": 2, "dst_inverse": 3, "scalar": 4,
                 "outer_residual": 5, "pcg_update": 6, "other": 7}


class AxGrid(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int32), ("nz", ctypes.c_int32), ("lr", ctypes.c_double),
                ("lz", ctypes.c_double), ("bc_z", ctypes.c_int32)]


class AxSolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer", ctypes.c_int32), ("rel_res", ctypes.c_double),
                ("guess_accepted", ctypes.c_int32), ("status", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AxError(RuntimeError):
    def __init__(self, status: int, what: str):
        extra = f" [{ax_last_error()}]" if status in (AX_ERR_CUDA, AX_ERR_OOM) else ""
        super().__init__(f"{what}: {ax_status_string(status)} (status {status}){extra}")
        self.status = status


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Loads libaxpcg.so (built in-tree by ``build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libaxpcg is not built ({path}); run paper_1002_3094_gb300.build()")
    lib = ctypes.CDLL(path)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    lib.ax_setup_operator.argtypes = [vp, vp, vp, ctypes.POINTER(AxGrid), vp, ctypes.POINTER(vp)]
    lib.ax_destroy_operator.argtypes = [vp]
    lib.ax_operator_info.argtypes = [vp] + [ctypes.POINTER(dbl)] * 4
    lib.ax_set_option.argtypes = [vp, ctypes.c_char_p, dbl]
    lib.ax_solve.argtypes = [vp, vp, vp, i32, dbl, i32, i32, i32, ctypes.POINTER(AxSolveInfo), vp]
    for name in ("ax_apply_operator", "ax_apply_dst", "ax_apply_dst_inverse", "ax_apply_mode_solve",
                 "ax_apply_preconditioner", "ax_apply_preconditioner_noalloc"):
        getattr(lib, name).argtypes = [vp, vp, vp, i32, i32, vp]
    lib.ax_last_error.argtypes = []
    lib.ax_status_string.argtypes = [ctypes.c_int]
    lib.ax_status_string.restype = ctypes.c_char_p
    lib.ax_version.restype = ctypes.c_char_p
    lib.ax_last_error.restype = ctypes.c_char_p
    pp = ctypes.POINTER(vp)
    lib.ax_batch_create.argtypes = [pp, i32, vp, ctypes.POINTER(vp)]
    lib.ax_batch_solve.argtypes = [vp, pp, pp, dbl, i32, i32, i32, ctypes.POINTER(AxSolveInfo), vp]
    lib.ax_batch_latency.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i32)]
    lib.ax_batch_destroy.argtypes = [vp]
    lib.ax_solve_batched.argtypes = [pp, pp, pp, i32, dbl, i32, i32, i32, ctypes.POINTER(AxSolveInfo), vp]
    f32p = ctypes.POINTER(ctypes.c_float)
    lib.ax_guessnet_create.argtypes = [i32, ctypes.POINTER(i32), i32, ctypes.c_uint64, ctypes.POINTER(vp)]
    lib.ax_guessnet_destroy.argtypes = [vp]
    lib.ax_guessnet_num_params.argtypes = [vp]
    lib.ax_guessnet_num_params.restype = ctypes.c_int64
    lib.ax_guessnet_get_params.argtypes = [vp, vp, ctypes.c_int64]
    lib.ax_guessnet_set_params.argtypes = [vp, vp, ctypes.c_int64]
    lib.ax_guessnet_forward.argtypes = [vp, vp, vp, i32, vp]
    lib.ax_guessnet_gradients.argtypes = [vp, vp, vp, i32, vp, ctypes.POINTER(dbl), vp]
    lib.ax_guessnet_train_step.argtypes = [vp, vp, vp, i32, ctypes.c_float, ctypes.POINTER(dbl), vp]
    lib.ax_guessnet_save.argtypes = [vp, ctypes.c_char_p]
    lib.ax_guessnet_load.argtypes = [vp, ctypes.c_char_p]
    lib.ax_guessnet_features.argtypes = [vp, vp, vp, i32, i32, i32, i32, vp, vp, vp]
    lib.ax_guessnet_lift.argtypes = [vp, i32, i32, vp, i32, i32, vp, vp]
    lib.ax_guessnet_set_loss.argtypes = [vp, dbl]
    lib.ax_guessnet_features_pre.argtypes = [vp, vp, vp, vp, i32, i32, vp, vp, vp]
    lib.ax_laguerre_step.argtypes = [vp, vp, vp, vp, vp, vp, dbl, dbl, dbl, vp, vp]
    lib.ax_kernel_launches.argtypes = []
    lib.ax_kernel_launches.restype = ctypes.c_int64
    lib.ax_profile_read.argtypes = [vp, i32] + [ctypes.POINTER(dbl)] * 3
    lib.ax_chebyshev_bounds.argtypes = [vp, i32, vp, vp, ctypes.POINTER(i32)]
    lib.ax_get_option.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(dbl)]
    lib.ax_autotune.argtypes = [vp, i32, i32, vp]
    lib.ax_batch_autotune.argtypes = [vp, i32, vp]
    lib.ax_batch_config.argtypes = [vp, i32] + [ctypes.POINTER(i32)] * 5
    lib.ax_solve_learned.argtypes = [vp, vp, vp, vp, vp, vp, i32, dbl, i32, i32, i32, i32, dbl,
                                     ctypes.POINTER(AxSolveInfo), vp]
    for name in EXPORTED:
        if name not in ("ax_status_string", "ax_version", "ax_kernel_launches", "ax_last_error",
                        "ax_guessnet_num_params"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(x) -> int:
    """Device (or host) address of a torch tensor, numpy array or int."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, what: str) -> int:
    if status != AX_OK:
        raise AxError(status, what)
    return status


def ax_status_string(status: int) -> str:
    return load_library().ax_status_string(status).decode()


def ax_last_error() -> str:
    return load_library().ax_last_error().decode()


def ax_version() -> str:
    return load_library().ax_version().decode()


def ax_setup_operator(kappa_r, kappa_z, q, nr: int, nz: int, lr: float = 1.0, lz: float = 1.0,
                      bc_z: int = 0, stream=None) -> int:
    """Returns an opaque operator handle (int).  kappa_r, kappa_z, q: FP64
    device tensors [nr][nz], [nr][nz+1], [nr][nz]."""
    lib = load_library()
    g = AxGrid(nr, nz, lr, lz, bc_z)
    out = ctypes.c_void_p()
    _check(lib.ax_setup_operator(_ptr(kappa_r), _ptr(kappa_z), _ptr(q), ctypes.byref(g), _stream(stream),
                                 ctypes.byref(out)), "ax_setup_operator")
    return out.value


def ax_destroy_operator(op: int) -> None:
    load_library().ax_destroy_operator(op)


def ax_operator_info(op: int):
    vals = [ctypes.c_double() for _ in range(4)]
    _check(load_library().ax_operator_info(op, *[ctypes.byref(v) for v in vals]), "ax_operator_info")
    return tuple(v.value for v in vals)


def ax_chebyshev_bounds(op: int, m: int):
    """(gamma1 [m], gamma2 [m], estimated) of the next Chebyshev solve of m
    right-hand sides (see include/axpcg.h)."""
    import numpy as np
    g1 = np.zeros(m)
    g2 = np.zeros(m)
    est = ctypes.c_int32()
    _check(load_library().ax_chebyshev_bounds(op, m, g1.ctypes.data, g2.ctypes.data, ctypes.byref(est)),
           "ax_chebyshev_bounds")
    return g1, g2, bool(est.value)


def ax_get_option(op: int, name: str) -> float:
    v = ctypes.c_double()
    _check(load_library().ax_get_option(op, name.encode(), ctypes.byref(v)), f"ax_get_option({name})")
    return v.value


def ax_autotune(op: int, m: int, reps: int = 5, stream=None) -> None:
    _check(load_library().ax_autotune(op, m, reps, _stream(stream)), "ax_autotune")


def ax_batch_autotune(batch: int, reps: int = 5, stream=None) -> None:
    _check(load_library().ax_batch_autotune(batch, reps, _stream(stream)), "ax_batch_autotune")


def ax_batch_config(batch: int, group: int) -> dict:
    vals = [ctypes.c_int32() for _ in range(5)]
    _check(load_library().ax_batch_config(batch, group, *[ctypes.byref(v) for v in vals]), "ax_batch_config")
    return dict(zip(("nr", "nz", "members", "dst_tensor", "mode_kernel"), (v.value for v in vals)))


def ax_set_option(op: int, name: str, value: float, raise_on_error: bool = True) -> int:
    st = load_library().ax_set_option(op, name.encode(), float(value))
    if raise_on_error:
        _check(st, f"ax_set_option({name})")
    return st


def ax_solve(op: int, f, u, m: int, tol: float, max_iter: int = 10000, method: int = AX_PCG_FP64,
             flags: int = 0, stream=None, raise_on_error: bool = True):
    """Solves for m right-hand sides; returns (status, [info dicts])."""
    infos = (AxSolveInfo * m)()
    st = load_library().ax_solve(op, _ptr(f), _ptr(u), m, tol, max_iter, method, flags, infos,
                                 _stream(stream) if not (flags & AX_FLAG_HOST_BUFFERS) or stream else
                                 _stream(None))
    if raise_on_error and st not in (AX_OK, AX_ERR_NO_CONVERGENCE):
        raise AxError(st, "ax_solve")
    return st, [i.as_dict() for i in infos]


def ax_solve_learned(op: int, net: int, kappa, q, f, u, m: int, tol: float, max_iter: int = 10000,
                     method: int = AX_PCG_MIXED, flags: int = 0, pre: bool = True, target_scale: float = 1.0,
                     stream=None, raise_on_error: bool = True):
    """Solve from the network's guess (features, forward, lift, gated solve in
    one library call); returns (status, [info dicts])."""
    infos = (AxSolveInfo * m)()
    st = load_library().ax_solve_learned(op, net, _ptr(kappa), _ptr(q), _ptr(f), _ptr(u), m, tol, max_iter, method,
                                         flags, 1 if pre else 0, target_scale, infos, _stream(stream))
    if raise_on_error and st not in (AX_OK, AX_ERR_NO_CONVERGENCE):
        raise AxError(st, "ax_solve_learned")
    return st, [i.as_dict() for i in infos]


def _apply(name: str, op: int, x, y, count: int, precision: int, stream=None) -> None:
    _check(getattr(load_library(), name)(op, _ptr(x), _ptr(y), count, precision, _stream(stream)), name)


def ax_apply_operator(op, x, y, m, precision=AX_PREC_FP64, stream=None):
    _apply("ax_apply_operator", op, x, y, m, precision, stream)


def ax_apply_dst(op, x, y, rows, precision=AX_PREC_FP64, stream=None):
    _apply("ax_apply_dst", op, x, y, rows, precision, stream)


def ax_apply_dst_inverse(op, x, y, rows, precision=AX_PREC_FP64, stream=None):
    _apply("ax_apply_dst_inverse", op, x, y, rows, precision, stream)


def ax_apply_mode_solve(op, x, y, m, precision=AX_PREC_FP64, stream=None):
    _apply("ax_apply_mode_solve", op, x, y, m, precision, stream)


def ax_apply_preconditioner(op, x, y, m, precision=AX_PREC_FP64, stream=None):
    _apply("ax_apply_preconditioner", op, x, y, m, precision, stream)


def ax_apply_preconditioner_noalloc(op, x, y, m, precision=AX_PREC_FP64, stream=None):
    """B^-1 without device allocation: stages through the library's fixed
    32 MiB array (see include/axpcg.h)."""
    _apply("ax_apply_preconditioner_noalloc", op, x, y, m, precision, stream)


def ax_laguerre_step(op, Q, T, S, c2, src, w_m: float, a_next: float, f_next: float, f_out, stream=None) -> None:
    """T += w_m Q, S += T, f_out = f_next src - c2 a_next S (dense FP64 device
    arrays [nr][nz]; see include/axpcg.h)."""
    _check(load_library().ax_laguerre_step(op, _ptr(Q), _ptr(T), _ptr(S), _ptr(c2), _ptr(src), w_m, a_next, f_next,
                                           _ptr(f_out), _stream(stream)), "ax_laguerre_step")


def ax_kernel_launches() -> int:
    return int(load_library().ax_kernel_launches())


def ax_profile_read(op: int, kind) -> dict:
    """{'ms', 'launches', 'units'} of one kernel class (name or number)."""
    k = PROFILE_KINDS[kind] if isinstance(kind, str) else int(kind)
    vals = [ctypes.c_double() for _ in range(3)]
    _check(load_library().ax_profile_read(op, k, *[ctypes.byref(v) for v in vals]), "ax_profile_read")
    return {"ms": vals[0].value, "launches": vals[1].value, "units": vals[2].value}


def _ptr_array(xs):
    arr = (ctypes.c_void_p * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = _ptr(x)
    return arr


def ax_batch_create(ops, stream=None) -> int:
    out = ctypes.c_void_p()
    _check(load_library().ax_batch_create(_ptr_array(ops), len(ops), _stream(stream), ctypes.byref(out)),
           "ax_batch_create")
    return out.value


def ax_batch_solve(batch: int, fs, us, tol: float, max_iter: int = 10000, method: int = AX_PCG_MIXED,
                   flags: int = 0, stream=None, raise_on_error: bool = True):
    n = len(fs)
    infos = (AxSolveInfo * n)()
    st = load_library().ax_batch_solve(batch, _ptr_array(fs), _ptr_array(us), tol, max_iter, method, flags, infos,
                                       _stream(stream))
    if raise_on_error and st not in (AX_OK, AX_ERR_NO_CONVERGENCE):
        raise AxError(st, "ax_batch_solve")
    return st, [i.as_dict() for i in infos]


def ax_batch_latency(batch: int, n: int):
    ms = (ctypes.c_double * n)()
    g = ctypes.c_int32()
    _check(load_library().ax_batch_latency(batch, ms, ctypes.byref(g)), "ax_batch_latency")
    return list(ms), g.value


def ax_batch_destroy(batch: int) -> None:
    load_library().ax_batch_destroy(batch)


def ax_solve_batched(ops, fs, us, tol: float, max_iter: int = 10000, method: int = AX_PCG_MIXED, flags: int = 0,
                     stream=None, raise_on_error: bool = True):
    n = len(ops)
    infos = (AxSolveInfo * n)()
    st = load_library().ax_solve_batched(_ptr_array(ops), _ptr_array(fs), _ptr_array(us), n, tol, max_iter, method,
                                         flags, infos, _stream(stream))
    if raise_on_error and st not in (AX_OK, AX_ERR_NO_CONVERGENCE):
        raise AxError(st, "ax_solve_batched")
    return st, [i.as_dict() for i in infos]


# ---- learned initial guess ---------------------------------------------------
def ax_guessnet_create(hw: int, channels=None, batch_capacity: int = 16, seed: int = 0) -> int:
    out = ctypes.c_void_p()
    ch = (ctypes.c_int32 * 4)(*channels) if channels is not None else None
    _check(load_library().ax_guessnet_create(hw, ch, batch_capacity, seed, ctypes.byref(out)), "ax_guessnet_create")
    return out.value


def ax_guessnet_destroy(net: int) -> None:
    load_library().ax_guessnet_destroy(net)


def ax_guessnet_num_params(net: int) -> int:
    return int(load_library().ax_guessnet_num_params(net))


def ax_guessnet_get_params(net: int):
    import numpy as np
    n = ax_guessnet_num_params(net)
    h = np.zeros(n, dtype=np.float32)
    _check(load_library().ax_guessnet_get_params(net, h.ctypes.data, n), "ax_guessnet_get_params")
    return h


def ax_guessnet_set_params(net: int, flat) -> None:
    import numpy as np
    h = np.ascontiguousarray(flat, dtype=np.float32)
    _check(load_library().ax_guessnet_set_params(net, h.ctypes.data, h.size), "ax_guessnet_set_params")


def ax_guessnet_forward(net: int, x, y, batch: int, stream=None) -> None:
    _check(load_library().ax_guessnet_forward(net, _ptr(x), _ptr(y), batch, _stream(stream)), "ax_guessnet_forward")


def ax_guessnet_gradients(net: int, x, target, batch: int, stream=None):
    """(loss, flat FP32 gradient as numpy)."""
    import numpy as np
    g = np.zeros(ax_guessnet_num_params(net), dtype=np.float32)
    loss = ctypes.c_double()
    _check(load_library().ax_guessnet_gradients(net, _ptr(x), _ptr(target), batch, g.ctypes.data, ctypes.byref(loss),
                                                _stream(stream)), "ax_guessnet_gradients")
    return loss.value, g


def ax_guessnet_train_step(net: int, x, target, batch: int, lr: float, stream=None) -> float:
    loss = ctypes.c_double()
    _check(load_library().ax_guessnet_train_step(net, _ptr(x), _ptr(target), batch, lr, ctypes.byref(loss),
                                                 _stream(stream)), "ax_guessnet_train_step")
    return loss.value


def ax_guessnet_save(net: int, path: str) -> None:
    _check(load_library().ax_guessnet_save(net, path.encode()), "ax_guessnet_save")


def ax_guessnet_load(net: int, path: str) -> None:
    _check(load_library().ax_guessnet_load(net, path.encode()), "ax_guessnet_load")


def ax_guessnet_features(kappa, q, f, m: int, nr: int, nz: int, hw: int, x, scale, stream=None) -> None:
    _check(load_library().ax_guessnet_features(_ptr(kappa), _ptr(q), _ptr(f), m, nr, nz, hw, _ptr(x), _ptr(scale),
                                               _stream(stream)), "ax_guessnet_features")


def ax_guessnet_set_loss(net: int, h1_weight: float) -> None:
    _check(load_library().ax_guessnet_set_loss(net, float(h1_weight)), "ax_guessnet_set_loss")


def ax_guessnet_features_pre(op, kappa, q, f, m: int, hw: int, x, scale, stream=None) -> None:
    _check(load_library().ax_guessnet_features_pre(op, _ptr(kappa), _ptr(q), _ptr(f), m, hw, _ptr(x), _ptr(scale),
                                                   _stream(stream)), "ax_guessnet_features_pre")


def ax_guessnet_lift(y, m: int, hw: int, scale, nr: int, nz: int, u, stream=None) -> None:
    _check(load_library().ax_guessnet_lift(_ptr(y), m, hw, _ptr(scale), nr, nz, _ptr(u), _stream(stream)),
           "ax_guessnet_lift")
