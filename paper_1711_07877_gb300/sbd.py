"""Thin Python binding of libsbd.so (argument marshalling only).

Every function has the name of the C entry point it wraps (include/sbd.h) and
passes raw pointers and sizes through ctypes; every step of the computation runs
in the library's CUDA kernels.  Device buffers are torch CUDA tensors (their
data_ptr() is passed); streams default to torch's current CUDA stream.  A
missing library is an ImportError: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsbd.so")

SBD_OK, SBD_EINVAL, SBD_ENOMEM, SBD_ECUDA, SBD_EFIT, SBD_ETIMEOUT, SBD_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
SBD_LAPLACE, SBD_HELMHOLTZ, SBD_RADIAL = 0, 1, 2
SBD_FORM_FP64, SBD_FORM_FP32 = 0, 1


class SbdError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {code} ({detail})")
        self.code = code


class sbd_kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("kappa", ctypes.c_double)]


RADIAL_VALUE = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_void_p)
RADIAL_LAPLACIAN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p)


class sbd_radial_kernel(ctypes.Structure):
    _fields_ = [("value", RADIAL_VALUE), ("deriv", RADIAL_VALUE), ("laplacian", RADIAL_LAPLACIAN),
                ("ctx", ctypes.c_void_p), ("log_coef", ctypes.c_double), ("n_enforce", ctypes.c_int32)]


def radial_kernel(value, deriv, laplacian=None, log_coef: float = 0.0, n_enforce: int = 0) -> sbd_radial_kernel:
    """sbd_radial_kernel from Python callables value(r), deriv(r), laplacian(j, r) (floats in, float
    out).  Keep the returned object alive while a plan is built with it."""
    k = sbd_radial_kernel()
    k._keep = (RADIAL_VALUE(lambda r, _c: float(value(r))), RADIAL_VALUE(lambda r, _c: float(deriv(r))),
               RADIAL_LAPLACIAN(lambda j, r, _c: float(laplacian(j, r))) if laplacian is not None
               else RADIAL_LAPLACIAN())
    k.value, k.deriv, k.laplacian = k._keep
    k.ctx = None
    k.log_coef = log_coef
    k.n_enforce = n_enforce
    return k


class sbd_options(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("fixed_P", ctypes.c_int32), ("nufft_tol", ctypes.c_double),
                ("max_nrhs", ctypes.c_int32), ("flags", ctypes.c_int32), ("delta_max", ctypes.c_double),
                ("host_threads", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class sbd_transform_stats(ctypes.Structure):
    _fields_ = [("sigma_s", ctypes.c_double), ("h", ctypes.c_double), ("deta", ctypes.c_double),
                ("nufft_tol", ctypes.c_double), ("grid_x", ctypes.c_int32), ("grid_k", ctypes.c_int32),
                ("fft_n", ctypes.c_int32), ("stencil_x", ctypes.c_int32), ("stencil_k", ctypes.c_int32),
                ("spread_window", ctypes.c_int32), ("P", ctypes.c_int64), ("n_circles", ctypes.c_int64),
                ("n_xi", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class sbd_gmres_options(ctypes.Structure):
    _fields_ = [("shift_re", ctypes.c_double), ("shift_im", ctypes.c_double), ("scale_re", ctypes.c_double),
                ("scale_im", ctypes.c_double), ("tol", ctypes.c_double), ("restart", ctypes.c_int32),
                ("max_iter", ctypes.c_int32)]


class sbd_plan_stats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("P", ctypes.c_int64), ("n_circles", ctypes.c_int64),
                ("n_xi", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_coincident", ctypes.c_int64),
                ("grid_x", ctypes.c_int32), ("grid_k", ctypes.c_int32), ("fft_n", ctypes.c_int32),
                ("stencil_x", ctypes.c_int32), ("stencil_k", ctypes.c_int32), ("form", ctypes.c_int32),
                ("kind", ctypes.c_int32),
                ("delta_max", ctypes.c_double), ("delta_min", ctypes.c_double), ("scale_R", ctypes.c_double),
                ("a", ctypes.c_double), ("fit_err", ctypes.c_double), ("nufft_tol", ctypes.c_double),
                ("w0_re", ctypes.c_double), ("w0_im", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("plan_seconds", ctypes.c_double), ("n_records", ctypes.c_int64), ("node_acc", ctypes.c_int32),
                ("node_sched", ctypes.c_int32), ("fft_split", ctypes.c_int32), ("node_binned", ctypes.c_int32),
                ("n_targets", ctypes.c_int64), ("separate_targets", ctypes.c_int32), ("uniform_grid", ctypes.c_int32),
                ("point_chunk", ctypes.c_int32), ("tuned", ctypes.c_int32), ("robin", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1711_07877_gb300.build` "
                          "(nvcc for sm_103a); there is no CPU fallback")
    return ctypes.CDLL(LIB_PATH)


lib = _load()
_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "sbd_fit_cache_stats": ([_P, _P, _P], ctypes.c_int),
    "sbd_tune": ([_P, _I32, _P, _P], ctypes.c_int),
    "sbd_set_tuning": ([_P, _I32, _I32, _I32], ctypes.c_int),
    "sbd_tune_points": ([_P, _I32, _P, _P], ctypes.c_int),
    "sbd_set_point_chunk": ([_P, _I32], ctypes.c_int),
    "sbd_tune_cache_stats": ([_P, _P, _P], ctypes.c_int),
    "sbd_tune_cache_save": ([ctypes.c_char_p], ctypes.c_int),
    "sbd_tune_cache_load": ([ctypes.c_char_p], ctypes.c_int),
    "sbd_tune_cache_clear": ([], ctypes.c_int),
    "sbd_plan_balanced": ([_P, _I64, sbd_kernel, _D, _P, _I32, _I32, _I32, ctypes.POINTER(sbd_options), _P,
                           ctypes.POINTER(_P), _P, ctypes.POINTER(_I32)], ctypes.c_int),
    "sbd_fit_cache_clear": ([], ctypes.c_int),
    "sbd_set_fit_device": ([_I32], ctypes.c_int),
    "sbd_fit_last_factorisation": ([_P, _P], ctypes.c_int),
    "sbd_y0_root": ([_I32, _P], ctypes.c_int),
    "sbd_plan": ([_P, _I64, sbd_kernel, _D, _D, ctypes.POINTER(sbd_options), _P, ctypes.POINTER(_P)], ctypes.c_int),
    "sbd_plan_st": ([_P, _I64, _P, _I64, sbd_kernel, _D, _D, ctypes.POINTER(sbd_options), _P, ctypes.POINTER(_P)],
                    ctypes.c_int),
    "sbd_plan_radial": ([_P, _I64, ctypes.POINTER(sbd_radial_kernel), _D, _D, ctypes.POINTER(sbd_options), _P,
                         ctypes.POINTER(_P)], ctypes.c_int),
    "sbd_offline_fit_radial": ([ctypes.POINTER(sbd_radial_kernel), _D, _D, _D, _I32, _I64, _P, _P, _P, _P, _P,
                                _P, _P], ctypes.c_int),
    "sbd_matvec": ([_P, _P, _P, _I32, _P], ctypes.c_int),
    "sbd_matvec_graph": ([_P, _P, _P, _I32, _P], ctypes.c_int),
    "sbd_batch_create": ([_P, _P, _I32, _P, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "sbd_batch_launch": ([_P, _P], ctypes.c_int),
    "sbd_matvec_batched": ([_P, _P, _P, _P, _I32, _P], ctypes.c_int),
    "sbd_set_device_wait": ([_D, _I32], ctypes.c_int),
    "sbd_device_status": ([_P], ctypes.c_int),
    "sbd_batch_destroy": ([_P], ctypes.c_int),
    "sbd_far": ([_P, _P, _P, _I32, _P], ctypes.c_int),
    "sbd_close": ([_P, _P, _P, _I32, _P], ctypes.c_int),
    "sbd_nufft_minus": ([_P, _P, _P, _P], ctypes.c_int),
    "sbd_nufft_plus": ([_P, _P, _P, _P], ctypes.c_int),
    "sbd_plan_info": ([_P, ctypes.POINTER(sbd_plan_stats)], ctypes.c_int),
    "sbd_plan_export": ([_P, _I64, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "sbd_close_export": ([_P, _P, _P, _P], ctypes.c_int),
    "sbd_destroy": ([_P], ctypes.c_int),
    "sbd_destroy_async": ([_P, _P], ctypes.c_int),
    "sbd_offline_fit": ([sbd_kernel, _D, _D, _D, _I32, _I64, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "sbd_transform_params": ([sbd_kernel, _D, _D, _D, _I64, _D, ctypes.POINTER(sbd_options),
                              ctypes.POINTER(sbd_transform_stats)], ctypes.c_int),
    "sbd_fft2": ([_P, _P, _I32, _I32, _I32, _I32, _P], ctypes.c_int),
    "sbd_fft2_noalloc": ([_P, _P, _I32, _I32, _I32, _I32, _P], ctypes.c_int),
    "sbd_gmres": ([_P, _P, _P, ctypes.POINTER(sbd_gmres_options), ctypes.POINTER(_I32), ctypes.POINTER(_D), _P],
                  ctypes.c_int),
    "sbd_gmres_begin": ([_P, _P, _P, ctypes.POINTER(sbd_gmres_options), _P, ctypes.POINTER(_P)], ctypes.c_int),
    "sbd_gmres_next": ([_P, ctypes.POINTER(_P), ctypes.POINTER(_P)], ctypes.c_int),
    "sbd_gmres_advance": ([_P], ctypes.c_int),
    "sbd_gmres_end": ([_P, ctypes.POINTER(_I32), ctypes.POINTER(_D)], ctypes.c_int),
    "sbd_profile": ([_P, _I32], ctypes.c_int),
    "sbd_profile_read": ([_P, _P, _P], ctypes.c_int),
    "sbd_error_string": ([ctypes.c_int], ctypes.c_char_p),
    "sbd_last_error_message": ([], ctypes.c_char_p),
    "sbd_version": ([], ctypes.c_char_p),
}
EXPORTED = tuple(_SIGS)
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


def _check(rc: int, where: str) -> None:
    if rc != SBD_OK:
        raise SbdError(rc, where, f"{lib.sbd_error_string(rc).decode()}: {lib.sbd_last_error_message().decode()}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(type(x))


def sbd_error_string(code: int) -> str:
    return lib.sbd_error_string(code).decode()


def sbd_last_error_message() -> str:
    return lib.sbd_last_error_message().decode()


def sbd_version() -> str:
    return lib.sbd_version().decode()


SBD_FLAG_GAUSSIAN_NODES = 1
SBD_FLAG_GAUSSIAN_SPREAD = 2
SBD_FLAG_SPREAD_SIGMA_2 = 4
SBD_FLAG_SPREAD_SIGMA_15 = 8
SBD_FLAG_NEAR_FP32 = 16
SBD_FLAG_UNIFORM_GRID = 32
SBD_FLAG_SPREAD_SIGMA_125 = 64


def make_options(form: int = SBD_FORM_FP64, fixed_P: int = 0, nufft_tol: float = 0.0, max_nrhs: int = 1,
                 flags: int = 0, delta_max: float = 0.0, host_threads: int = 0):
    return sbd_options(form, fixed_P, nufft_tol, max_nrhs, flags, delta_max, host_threads, 0)


def sbd_plan(points, n: int, kernel_kind: int, kappa: float, delta_min: float, eps: float,
             options: sbd_options | None = None, stream=None) -> int:
    """points: device (N, 2) float64 tensor or pointer.  Returns the plan handle (int)."""
    out = _P()
    rc = lib.sbd_plan(_ptr(points), n, sbd_kernel(kernel_kind, kappa), delta_min, eps,
                      ctypes.byref(options) if options is not None else None, _stream(stream), ctypes.byref(out))
    _check(rc, "sbd_plan")
    return out.value


def sbd_plan_radial(points, n: int, kernel: sbd_radial_kernel, delta_min: float, eps: float,
                    options: sbd_options | None = None, stream=None) -> int:
    """A plan for a general real radial kernel (Sec. 4.3), kernel from radial_kernel()."""
    out = _P()
    rc = lib.sbd_plan_radial(_ptr(points), n, ctypes.byref(kernel), delta_min, eps,
                             ctypes.byref(options) if options is not None else None, _stream(stream),
                             ctypes.byref(out))
    _check(rc, "sbd_plan_radial")
    return out.value


def sbd_offline_fit_radial(kernel: sbd_radial_kernel, delta_min: float, delta_max: float, eps: float,
                           fixed_P: int = 0, cap: int = 40000) -> dict:
    """Host-only fit of a general radial kernel: dict(P, n_circles, rho, alpha, M, fit_err, w0); the
    circles after the first P are the correction's terms (rho = omega_t, alpha = mu_t / J0(omega_t))."""
    import numpy as np
    rho, alpha = np.zeros(cap), np.zeros(cap)
    M = np.zeros(cap, dtype=np.int32)
    P, nc, err, w0 = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _check(lib.sbd_offline_fit_radial(ctypes.byref(kernel), delta_min, delta_max, eps, fixed_P, cap, rho.ctypes.data,
                                      alpha.ctypes.data, M.ctypes.data, ctypes.byref(P), ctypes.byref(nc),
                                      ctypes.byref(err), ctypes.byref(w0)), "sbd_offline_fit_radial")
    k = nc.value
    return {"P": P.value, "n_circles": k, "rho": rho[:k].copy(), "alpha": alpha[:k].copy(), "M": M[:k].copy(),
            "fit_err": err.value, "w0": w0.value}


def sbd_plan_st(targets, n_targets: int, sources, n_sources: int, kernel_kind: int, kappa: float,
                delta_min: float, eps: float, options: sbd_options | None = None, stream=None) -> int:
    """targets, sources: device (N, 2) float64 tensors or pointers.  Returns the plan handle (int)."""
    out = _P()
    rc = lib.sbd_plan_st(_ptr(targets), n_targets, _ptr(sources), n_sources, sbd_kernel(kernel_kind, kappa),
                         delta_min, eps, ctypes.byref(options) if options is not None else None, _stream(stream),
                         ctypes.byref(out))
    _check(rc, "sbd_plan_st")
    return out.value


def sbd_matvec(plan: int, f, q, nrhs: int = 1, stream=None) -> None:
    _check(lib.sbd_matvec(plan, _ptr(f), _ptr(q), nrhs, _stream(stream)), "sbd_matvec")


def sbd_matvec_graph(plan: int, f, q, nrhs: int = 1, stream=None) -> None:
    _check(lib.sbd_matvec_graph(plan, _ptr(f), _ptr(q), nrhs, _stream(stream)), "sbd_matvec_graph")


def sbd_batch_create(plans, f, q, nrhs=None) -> int:
    """One CUDA graph with the matvecs of several plans (f[i], q[i] device tensors that stay put)."""
    k = len(plans)
    nrhs = nrhs or [1] * k
    P = (_P * k)(*plans)
    R = (_I32 * k)(*nrhs)
    F = (_P * k)(*[_ptr(x) for x in f])
    Qp = (_P * k)(*[_ptr(x) for x in q])
    out = _P()
    _check(lib.sbd_batch_create(P, R, k, F, Qp, ctypes.byref(out)), "sbd_batch_create")
    return out.value


def sbd_matvec_batched(plans, f, q, nrhs=None, stream=None) -> None:
    """q[i] = matvec of plans[i] on f[i] (device tensors) for every i, in one batched call."""
    k = len(plans)
    nrhs = nrhs or [1] * k
    P = (_P * k)(*plans)
    F = (_P * k)(*[_ptr(x) for x in f])
    Qp = (_P * k)(*[_ptr(x) for x in q])
    R = (_I32 * k)(*nrhs)
    _check(lib.sbd_matvec_batched(P, F, Qp, R, k, _stream(stream)), "sbd_matvec_batched")


def sbd_set_device_wait(limit_seconds: float, phantom_arrivals: int = 0) -> None:
    _check(lib.sbd_set_device_wait(limit_seconds, phantom_arrivals), "sbd_set_device_wait")


def sbd_device_status(stream=None) -> int:
    """Synchronise the stream; return (and clear) the status of the bounded device waits."""
    return lib.sbd_device_status(_stream(stream))


def sbd_batch_launch(batch: int, stream=None) -> None:
    _check(lib.sbd_batch_launch(batch, _stream(stream)), "sbd_batch_launch")


def sbd_batch_destroy(batch: int) -> None:
    _check(lib.sbd_batch_destroy(batch), "sbd_batch_destroy")


def sbd_far(plan: int, f, q, nrhs: int = 1, stream=None) -> None:
    _check(lib.sbd_far(plan, _ptr(f), _ptr(q), nrhs, _stream(stream)), "sbd_far")


def sbd_close(plan: int, f, q, nrhs: int = 1, stream=None) -> None:
    _check(lib.sbd_close(plan, _ptr(f), _ptr(q), nrhs, _stream(stream)), "sbd_close")


def sbd_nufft_minus(plan: int, f, fhat, stream=None) -> None:
    _check(lib.sbd_nufft_minus(plan, _ptr(f), _ptr(fhat), _stream(stream)), "sbd_nufft_minus")


def sbd_nufft_plus(plan: int, ghat, q, stream=None) -> None:
    _check(lib.sbd_nufft_plus(plan, _ptr(ghat), _ptr(q), _stream(stream)), "sbd_nufft_plus")


def sbd_plan_info(plan: int) -> dict:
    st = sbd_plan_stats()
    _check(lib.sbd_plan_info(plan, ctypes.byref(st)), "sbd_plan_info")
    return st.as_dict()


def sbd_plan_export(plan: int):
    """Returns dict of numpy arrays rho, alpha, M, radius, weight (complex), one entry per circle."""
    import numpy as np
    nc = sbd_plan_info(plan)["n_circles"]
    rho, alpha, radius, wr, wi = (np.zeros(nc) for _ in range(5))
    M = np.zeros(nc, dtype=np.int32)
    _check(lib.sbd_plan_export(plan, nc, rho.ctypes.data, alpha.ctypes.data, M.ctypes.data, radius.ctypes.data,
                               wr.ctypes.data, wi.ctypes.data), "sbd_plan_export")
    return {"rho": rho, "alpha": alpha, "M": M, "radius": radius, "weight": wr + 1j * wi}


def sbd_close_export(plan: int):
    """Returns (rowptr int64, col int32, val float64 or complex128) host arrays of D."""
    import numpy as np
    info = sbd_plan_info(plan)
    n, nnz = info["n_targets"], info["nnz"]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    cplx = info["kind"] == SBD_HELMHOLTZ
    val = np.zeros(nnz, dtype=np.complex128 if cplx else np.float64)
    _check(lib.sbd_close_export(plan, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data), "sbd_close_export")
    return rowptr, col, val


def sbd_gmres(plan: int, b, x, shift=1.0, scale=1.0, tol: float = 1e-6, restart: int = 30,
              max_iter: int = 300, stream=None):
    """Solve (shift I + scale A) x = b in place of x (x holds the initial guess).
    Returns (iterations, relative residual)."""
    shift, scale = complex(shift), complex(scale)
    opt = sbd_gmres_options(shift.real, shift.imag, scale.real, scale.imag, tol, restart, max_iter)
    it, res = _I32(), _D()
    _check(lib.sbd_gmres(plan, _ptr(b), _ptr(x), ctypes.byref(opt), ctypes.byref(it), ctypes.byref(res),
                         _stream(stream)), "sbd_gmres")
    return it.value, res.value


STAGES = ("sum", "spread", "fft_fwd", "node", "fft_inv", "interp", "spmv")


def sbd_gmres_begin(plan: int, b, x, shift=1.0, scale=1.0, tol: float = 1e-6, restart: int = 30,
                    max_iter: int = 300, stream=None) -> int:
    """A resumable GMRES session on (shift I + scale A) x = b; returns its handle."""
    sh, sc = complex(shift), complex(scale)
    opt = sbd_gmres_options(sh.real, sh.imag, sc.real, sc.imag, tol, restart, max_iter)
    out = _P()
    _check(lib.sbd_gmres_begin(plan, _ptr(b), _ptr(x), ctypes.byref(opt), _stream(stream), ctypes.byref(out)),
           "sbd_gmres_begin")
    return out.value


def sbd_gmres_next(session: int):
    """(in, out) device pointers of the matvec the session needs, or None when it has finished."""
    pi, po = _P(), _P()
    rc = lib.sbd_gmres_next(session, ctypes.byref(pi), ctypes.byref(po))
    if rc < 0:
        _check(rc, "sbd_gmres_next")
    return (pi.value, po.value) if rc == 1 else None


def sbd_gmres_advance(session: int) -> None:
    _check(lib.sbd_gmres_advance(session), "sbd_gmres_advance")


def sbd_gmres_end(session: int):
    """Frees the session; returns (iterations, relative residual)."""
    it, res = _I32(), _D()
    _check(lib.sbd_gmres_end(session, ctypes.byref(it), ctypes.byref(res)), "sbd_gmres_end")
    return it.value, res.value


def sbd_profile(plan: int, enable: bool) -> None:
    _check(lib.sbd_profile(plan, 1 if enable else 0), "sbd_profile")


def sbd_profile_read(plan: int) -> dict:
    """{stage: (total_ms, count)} for the steps timed since sbd_profile(plan, True)."""
    import numpy as np
    ms = np.zeros(len(STAGES))
    cnt = np.zeros(len(STAGES), dtype=np.int64)
    _check(lib.sbd_profile_read(plan, ms.ctypes.data, cnt.ctypes.data), "sbd_profile_read")
    return {s: (float(ms[i]), int(cnt[i])) for i, s in enumerate(STAGES)}


def sbd_destroy(plan: int) -> None:
    _check(lib.sbd_destroy(plan), "sbd_destroy")


def sbd_destroy_async(plan: int, stream=None) -> None:
    _check(lib.sbd_destroy_async(plan, _stream(stream)), "sbd_destroy_async")


def sbd_offline_fit(kernel_kind: int, kappa: float, delta_min: float, delta_max: float, eps: float,
                    fixed_P: int = 0, cap: int = 40000):
    """Host-only SBD fit: returns dict(P, n_circles, rho, alpha, M, fit_err)."""
    import numpy as np
    rho, alpha = np.zeros(cap), np.zeros(cap)
    M = np.zeros(cap, dtype=np.int32)
    P, nc, err = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(lib.sbd_offline_fit(sbd_kernel(kernel_kind, kappa), delta_min, delta_max, eps, fixed_P, cap,
                               rho.ctypes.data, alpha.ctypes.data, M.ctypes.data, ctypes.byref(P),
                               ctypes.byref(nc), ctypes.byref(err)), "sbd_offline_fit")
    k = nc.value
    return {"P": P.value, "n_circles": k, "rho": rho[:k].copy(), "alpha": alpha[:k].copy(), "M": M[:k].copy(),
            "fit_err": err.value}


def sbd_transform_params(kernel_kind: int, kappa: float, delta_min: float, delta_max: float, eps: float,
                         n_points: int, half_extent: float, options: sbd_options | None = None) -> dict:
    """Host only: the transform sizes sbd_plan would choose (no GPU needed)."""
    out = sbd_transform_stats()
    _check(lib.sbd_transform_params(sbd_kernel(kernel_kind, kappa), delta_min, delta_max, eps, n_points, half_extent,
                                    ctypes.byref(options) if options is not None else None, ctypes.byref(out)),
           "sbd_transform_params")
    return out.as_dict()


def sbd_fit_cache_stats() -> dict:
    h, m, e = _I64(), _I64(), _I64()
    _check(lib.sbd_fit_cache_stats(ctypes.byref(h), ctypes.byref(m), ctypes.byref(e)), "sbd_fit_cache_stats")
    return {"hits": h.value, "misses": m.value, "entries": e.value}


def sbd_tune(plan: int, reps: int = 3, stream=None) -> list:
    """Time the node-kernel and row-FFT variants, keep the fastest; returns ms per node variant
    (index acc * 2 + sched for acc <= 3, 10 + sched for acc 4, -1 where not applicable) and, at 8
    and 9, per FFT split (0, 2)."""
    import numpy as np
    ms = np.zeros(12)
    _check(lib.sbd_tune(plan, reps, ms.ctypes.data, _stream(stream)), "sbd_tune")
    return ms.tolist()


def sbd_plan_balanced(points, n: int, kernel_kind: int, kappa: float, eps: float, alphas, nrhs: int = 1,
                      reps: int = 5, options: sbd_options | None = None, stream=None):
    """Plan with delta_min from Theorem 1 at the fastest of the candidate alphas.
    Returns (plan, ms per candidate (-1 where it could not be planned), chosen index)."""
    import numpy as np
    al = np.ascontiguousarray(alphas, dtype=np.float64)
    ms = np.zeros(len(al))
    out, chosen = _P(), _I32()
    rc = lib.sbd_plan_balanced(_ptr(points), n, sbd_kernel(kernel_kind, kappa), eps, al.ctypes.data, len(al), nrhs,
                               reps, ctypes.byref(options) if options is not None else None, _stream(stream),
                               ctypes.byref(out), ms.ctypes.data, ctypes.byref(chosen))
    _check(rc, "sbd_plan_balanced")
    return out.value, ms.tolist(), chosen.value


def sbd_tune_points(plan: int, reps: int = 3, stream=None) -> list:
    """Times spreading + interpolation per point chunk (128 .. 2048), keeps the fastest."""
    import numpy as np
    ms = np.zeros(5)
    _check(lib.sbd_tune_points(plan, reps, ms.ctypes.data, _stream(stream)), "sbd_tune_points")
    return ms.tolist()


def sbd_set_point_chunk(plan: int, chunk: int) -> None:
    _check(lib.sbd_set_point_chunk(plan, chunk), "sbd_set_point_chunk")


def sbd_tune_cache_stats() -> dict:
    h, m, e = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib.sbd_tune_cache_stats(ctypes.byref(h), ctypes.byref(m), ctypes.byref(e)), "sbd_tune_cache_stats")
    return {"hits": h.value, "misses": m.value, "entries": e.value}


def sbd_tune_cache_save(path: str) -> None:
    _check(lib.sbd_tune_cache_save(path.encode()), "sbd_tune_cache_save")


def sbd_tune_cache_load(path: str) -> None:
    _check(lib.sbd_tune_cache_load(path.encode()), "sbd_tune_cache_load")


def sbd_tune_cache_clear() -> None:
    _check(lib.sbd_tune_cache_clear(), "sbd_tune_cache_clear")


def sbd_set_tuning(plan: int, acc: int, sched: int, fft_split: int = 0) -> None:
    _check(lib.sbd_set_tuning(plan, acc, sched, fft_split), "sbd_set_tuning")


def sbd_y0_root(k: int) -> float:
    r = _D()
    _check(lib.sbd_y0_root(k, ctypes.byref(r)), "sbd_y0_root")
    return r.value


def sbd_fit_cache_clear() -> None:
    _check(lib.sbd_fit_cache_clear(), "sbd_fit_cache_clear")


def sbd_set_fit_device(mode: int) -> None:
    """Where the fit's full Cholesky runs: 0 auto (device for P >= 3000), 1 host, 2 device."""
    _check(lib.sbd_set_fit_device(mode), "sbd_set_fit_device")


def sbd_fit_last_factorisation() -> tuple[float, int]:
    """(seconds, where) of the last full factorisation; where 0 none, 1 host, 2 device."""
    sec, w = ctypes.c_double(), ctypes.c_int32()
    _check(lib.sbd_fit_last_factorisation(ctypes.byref(sec), ctypes.byref(w)), "sbd_fit_last_factorisation")
    return sec.value, w.value


def sbd_fft2(x, out, n0: int, n1: int, sign: int, form: int, stream=None) -> None:
    _check(lib.sbd_fft2(_ptr(x), _ptr(out), n0, n1, sign, form, _stream(stream)), "sbd_fft2")


SBD_NOALLOC_FFT_MAX_BYTES = 4 * 1024 * 1024
SBD_NOALLOC_FFT_MAX_SIDE = 4096


def sbd_fft2_noalloc(x, out, n0: int, n1: int, sign: int, form: int, stream=None) -> None:
    """sbd_fft2 with its scratch in the library's fixed device array (no allocation)."""
    _check(lib.sbd_fft2_noalloc(_ptr(x), _ptr(out), n0, n1, sign, form, _stream(stream)), "sbd_fft2_noalloc")
