"""ctypes declarations of ``include/tm.h`` (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_longlong, c_size_t, c_void_p, c_char_p

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libtmamg.so")

TM_OK, TM_ERR_ARG, TM_ERR_CUDA, TM_ERR_OOM = 0, -1, -2, -3
TM_ERR_NOT_CONVERGED, TM_ERR_TIMEOUT, TM_ERR_NOT_SU3 = -4, -5, -6
TM_ERR_NONFINITE, TM_ERR_STATE = -7, -8
TM_F64, TM_F32, TM_F16, TM_BF16, TM_F32X2 = 0, 1, 2, 3, 4
TM_EXPORT_P, TM_EXPORT_DC, TM_EXPORT_CLOVER, TM_EXPORT_TV = 0, 1, 2, 3
TM_EXPORT_P2, TM_EXPORT_DC2, TM_EXPORT_TV1 = 4, 5, 6


class tm_params(ctypes.Structure):
    _fields_ = [
        ("L", c_int * 4), ("m0", c_double), ("c_sw", c_double), ("mu", c_double),
        ("delta", c_double), ("bc_t", c_double), ("nv", c_int), ("agg", c_int * 4),
        ("sap_block", c_int * 4), ("mr_iters", c_int), ("pre_smooth", c_int),
        ("post_smooth", c_int), ("init_sweeps", c_int), ("setup_iters", c_int),
        ("coarse_tol", c_double), ("coarse_restart", c_int), ("coarse_maxit", c_int),
        ("restart", c_int), ("maxit", c_int), ("cycle_prec", c_int), ("max_rhs", c_int),
        ("levels", c_int), ("nv2", c_int), ("agg2", c_int * 4), ("sap_block1", c_int * 4),
        ("mr_iters1", c_int), ("pre_smooth1", c_int), ("post_smooth1", c_int), ("init_sweeps1", c_int),
        ("coarse_setup_iters", c_int), ("coarsest_tol", c_double), ("coarsest_maxit", c_int),
        ("coarse_mma", c_int), ("nn_mode", c_int), ("nn_prec", c_int), ("sap1_prec", c_int),
        ("outer_apply", c_int), ("block_oe", c_int), ("tc_spin_limit", c_int), ("transfer_prec", c_int),
        ("sap_prec", c_int), ("coarsest_steps", c_int),
    ]


class tm_solve_info(ctypes.Structure):
    _fields_ = [
        ("iters", c_int), ("restarts", c_int), ("converged", c_int),
        ("true_relres", c_double), ("coarse_iters", c_longlong), ("kcycles", c_int),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class TMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{tm_status_string(status)} ({status}): {message}")
        self.status = status


_lib = None

_SIGS = {
    "tm_params_default": (None, [POINTER(tm_params)]),
    "tm_create": (c_int, [POINTER(c_void_p), POINTER(tm_params), c_void_p]),
    "tm_destroy": (None, [c_void_p]),
    "tm_status_string": (c_char_p, [c_int]),
    "tm_last_error": (c_char_p, [c_void_p]),
    "tm_load_gauge": (c_int, [c_void_p, c_void_p]),
    "tm_setup": (c_int, [c_void_p, c_void_p]),
    "tm_setup_from_vectors": (c_int, [c_void_p, c_void_p]),
    "tm_set_mu": (c_int, [c_void_p, c_double, c_double]),
    "tm_set_mu_eo": (c_int, [c_void_p, c_double, c_double, c_double]),
    "tm_solve_odd": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, POINTER(tm_solve_info)]),
    "tm_solve_hasenbusch": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_double, c_double,
                                    POINTER(tm_solve_info)]),
    "tm_solve_oecg": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_int, POINTER(tm_solve_info)]),
    "tm_autotune_build": (c_int, [c_void_p, c_char_p, c_int, POINTER(c_double)]),
    "tm_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, POINTER(tm_solve_info)]),
    "tm_solve_squared": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, POINTER(tm_solve_info)]),
    "tm_field_bytes": (c_size_t, [c_void_p, c_int, c_int, c_int]),
    "tm_workspace_bytes": (c_size_t, [POINTER(tm_params), c_int]),
    "tm_save_setup": (c_int, [c_void_p, c_char_p]),
    "tm_load_setup": (c_int, [c_void_p, c_char_p]),
    "tm_pack": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int]),
    "tm_unpack": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int]),
    "tm_apply": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int]),
    "tm_sap": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int]),
    "tm_restrict": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int]),
    "tm_prolong": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int]),
    "tm_coarse_solve": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_int, POINTER(c_int)]),
    "tm_coarse_solve_noalloc": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_double, c_int, POINTER(c_int)]),
    "tm_kcycle": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int]),
    "tm_schur": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int]),
    "tm_setup_update": (c_int, [c_void_p, c_int, c_int]),
    "tm_nn_set_weights": (c_int, [c_void_p, c_void_p]),
    "tm_nn_get_weights": (c_int, [c_void_p, c_void_p]),
    "tm_nn_apply": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int]),
    "tm_nn_pairs": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int]),
    "tm_nn_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, POINTER(c_double)]),
    "tm_nn_train": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_double, c_void_p]),
    "tm_sap1": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int]),
    "tm_restrict1": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int]),
    "tm_prolong1": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int, c_int]),
    "tm_kcycle1": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_int]),
    "tm_export": (c_int, [c_void_p, c_int, c_void_p, c_size_t]),
    "tm_synchronize": (c_int, [c_void_p]),
    "tm_profile": (c_int, [c_void_p, c_int]),
    "tm_profile_kinds": (c_int, []),
    "tm_profile_name": (c_char_p, [c_int]),
    "tm_profile_read": (c_int, [c_void_p, POINTER(c_longlong), POINTER(c_longlong), POINTER(c_double), c_int]),
}


def exported_symbols() -> list[str]:
    """Names of the C ABI entry points this binding declares."""
    return list(_SIGS)


def lib() -> ctypes.CDLL:
    """Load ``libtmamg.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise RuntimeError(
                f"{library_path} is missing: build it with "
                "`python -m paper_1611_01034_gb300.build` (there is no CPU fallback)")
        L = ctypes.CDLL(library_path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    """Address of a torch tensor, numpy array, ctypes object or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "__array_interface__"):
        return x.__array_interface__["data"][0]
    if isinstance(x, ctypes.c_void_p):
        return x.value
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, h=None) -> None:
    if status != TM_OK:
        msg = tm_last_error(h) if h is not None else ""
        raise TMError(status, msg)


def tm_status_string(status: int) -> str:
    return lib().tm_status_string(status).decode()


def tm_last_error(h) -> str:
    return lib().tm_last_error(h).decode()


def tm_params_default() -> tm_params:
    p = tm_params()
    lib().tm_params_default(ctypes.byref(p))
    return p


def params(**kw) -> tm_params:
    """tm_params_default() with the given fields replaced (sequences for arrays)."""
    p = tm_params_default()
    for k, v in kw.items():
        if k in ("L", "agg", "sap_block"):
            getattr(p, k)[:] = [int(t) for t in v]
        else:
            setattr(p, k, v)
    return p


def tm_create(p: tm_params, stream=None):
    h = c_void_p()
    _check(lib().tm_create(ctypes.byref(h), ctypes.byref(p), _stream(stream)))
    return h


def tm_destroy(h) -> None:
    lib().tm_destroy(h)


def tm_load_gauge(h, gauge) -> None:
    _check(lib().tm_load_gauge(h, _ptr(gauge)), h)


def tm_setup(h, test_vectors) -> None:
    _check(lib().tm_setup(h, _ptr(test_vectors)), h)


def tm_setup_from_vectors(h, test_vectors) -> None:
    _check(lib().tm_setup_from_vectors(h, _ptr(test_vectors)), h)


def tm_set_mu(h, mu: float, delta: float) -> None:
    _check(lib().tm_set_mu(h, mu, delta), h)


def tm_autotune_build(h, cache_path=None, reps: int = 3) -> dict:
    out = (c_double * 4)()
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(lib().tm_autotune_build(h, path, reps, out), h)
    return {"ts": int(out[0]), "ktc": int(out[1]), "us": out[2], "timed": int(out[3])}


def tm_solve(h, b, x, nrhs: int, tol: float):
    info = tm_solve_info()
    st = lib().tm_solve(h, _ptr(b), _ptr(x), nrhs, tol, ctypes.byref(info))
    if st not in (TM_OK, TM_ERR_NOT_CONVERGED):
        _check(st, h)
    return st, info


def tm_set_mu_eo(h, mu_even: float, mu_odd: float, delta: float) -> None:
    _check(lib().tm_set_mu_eo(h, mu_even, mu_odd, delta), h)


def tm_solve_odd(h, b, x, nrhs: int, tol: float):
    info = tm_solve_info()
    st = lib().tm_solve_odd(h, _ptr(b), _ptr(x), nrhs, tol, ctypes.byref(info))
    if st not in (TM_OK, TM_ERR_NOT_CONVERGED):
        _check(st, h)
    return st, info


def tm_solve_hasenbusch(h, b, x, nrhs: int, mu: float, rho: float, tol: float):
    info = tm_solve_info()
    st = lib().tm_solve_hasenbusch(h, _ptr(b), _ptr(x), nrhs, mu, rho, tol, ctypes.byref(info))
    if st not in (TM_OK, TM_ERR_NOT_CONVERGED):
        _check(st, h)
    return st, info


def tm_solve_oecg(h, b, x, nrhs: int, tol: float, maxit: int = 100000):
    info = tm_solve_info()
    st = lib().tm_solve_oecg(h, _ptr(b), _ptr(x), nrhs, tol, maxit, ctypes.byref(info))
    if st not in (TM_OK, TM_ERR_NOT_CONVERGED):
        _check(st, h)
    return st, info


def tm_solve_squared(h, b, x, nrhs: int, tol: float):
    info = tm_solve_info()
    st = lib().tm_solve_squared(h, _ptr(b), _ptr(x), nrhs, tol, ctypes.byref(info))
    if st not in (TM_OK, TM_ERR_NOT_CONVERGED):
        _check(st, h)
    return st, info


def tm_field_bytes(h, level: int, prec: int, nrhs: int) -> int:
    return int(lib().tm_field_bytes(h, level, prec, nrhs))


def tm_workspace_bytes(p: tm_params, nrhs: int = 1) -> int:
    return int(lib().tm_workspace_bytes(ctypes.byref(p), nrhs))


def tm_save_setup(h, path: str) -> None:
    _check(lib().tm_save_setup(h, os.fsencode(path)), h)


def tm_load_setup(h, path: str) -> None:
    _check(lib().tm_load_setup(h, os.fsencode(path)), h)


def tm_pack(h, level, prec, natural, field, nrhs) -> None:
    _check(lib().tm_pack(h, level, prec, _ptr(natural), _ptr(field), nrhs), h)


def tm_unpack(h, level, prec, field, natural, nrhs) -> None:
    _check(lib().tm_unpack(h, level, prec, _ptr(field), _ptr(natural), nrhs), h)


def tm_apply(h, level, prec, inp, out, nrhs) -> None:
    _check(lib().tm_apply(h, level, prec, _ptr(inp), _ptr(out), nrhs), h)


def tm_sap(h, prec, b, x, sweeps, nrhs) -> None:
    _check(lib().tm_sap(h, prec, _ptr(b), _ptr(x), sweeps, nrhs), h)


def tm_restrict(h, prec, fine, coarse, nrhs) -> None:
    _check(lib().tm_restrict(h, prec, _ptr(fine), _ptr(coarse), nrhs), h)


def tm_prolong(h, prec, coarse, fine, nrhs, accumulate) -> None:
    _check(lib().tm_prolong(h, prec, _ptr(coarse), _ptr(fine), nrhs, int(accumulate)), h)


def tm_coarse_solve(h, prec, b, x, tol, maxit) -> int:
    it = c_int(0)
    _check(lib().tm_coarse_solve(h, prec, _ptr(b), _ptr(x), tol, maxit, ctypes.byref(it)), h)
    return it.value


def tm_coarse_solve_noalloc(h, prec, b, x, tol, maxit) -> int:
    """Same as tm_coarse_solve, with all workspaces in the library's fixed
    8 MiB device array instead of device allocations (see include/tm.h)."""
    it = c_int(0)
    _check(lib().tm_coarse_solve_noalloc(h, prec, _ptr(b), _ptr(x), tol, maxit, ctypes.byref(it)), h)
    return it.value


def tm_kcycle(h, prec, v, z, nrhs) -> None:
    _check(lib().tm_kcycle(h, prec, _ptr(v), _ptr(z), nrhs), h)


def tm_setup_update(h, fine_iters, coarse_iters=0) -> None:
    _check(lib().tm_setup_update(h, fine_iters, coarse_iters), h)


def tm_schur(h, prec, ve, ye, nrhs) -> None:
    _check(lib().tm_schur(h, prec, _ptr(ve), _ptr(ye), nrhs), h)


def tm_nn_set_weights(h, w) -> None:
    """w: 2304 complex weights (W1 [8,1,9,4,4] then W2 [1,8,9,4,4])."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(w, dtype=np.complex128).ravel())
    if a.size != 2304:
        raise ValueError("expected 2304 complex weights")
    _check(lib().tm_nn_set_weights(h, _ptr(a)), h)


def tm_nn_get_weights(h):
    import numpy as np
    a = np.zeros(2304, dtype=np.complex128)
    _check(lib().tm_nn_get_weights(h, _ptr(a)), h)
    return a


def tm_nn_apply(h, prec, inp, out, nrhs, accumulate=False) -> None:
    _check(lib().tm_nn_apply(h, prec, _ptr(inp), _ptr(out), nrhs, int(accumulate)), h)


def tm_nn_pairs(h, e0, r, e, npairs) -> None:
    _check(lib().tm_nn_pairs(h, _ptr(e0), _ptr(r), _ptr(e), npairs), h)


def tm_nn_grad(h, r, e, npairs):
    """(loss, gradient dL/d conj(W) as 2304 complex)."""
    import numpy as np
    g = np.zeros(2304, dtype=np.complex128)
    loss = c_double(0)
    _check(lib().tm_nn_grad(h, _ptr(r), _ptr(e), npairs, _ptr(g), ctypes.byref(loss)), h)
    return loss.value, g


def tm_nn_train(h, r, e, npairs, epochs, batch, lr):
    """Adam training; returns the mean loss of every epoch."""
    import numpy as np
    losses = np.zeros(epochs, dtype=np.float64)
    _check(lib().tm_nn_train(h, _ptr(r), _ptr(e), npairs, epochs, batch, lr, _ptr(losses)), h)
    return losses


def tm_sap1(h, prec, b, x, sweeps, nrhs) -> None:
    _check(lib().tm_sap1(h, prec, _ptr(b), _ptr(x), sweeps, nrhs), h)


def tm_restrict1(h, prec, c1, c2, nrhs) -> None:
    _check(lib().tm_restrict1(h, prec, _ptr(c1), _ptr(c2), nrhs), h)


def tm_prolong1(h, prec, c2, c1, nrhs, accumulate) -> None:
    _check(lib().tm_prolong1(h, prec, _ptr(c2), _ptr(c1), nrhs, int(accumulate)), h)


def tm_kcycle1(h, prec, v, z, nrhs) -> None:
    _check(lib().tm_kcycle1(h, prec, _ptr(v), _ptr(z), nrhs), h)


def tm_export(h, what, out, nbytes) -> None:
    _check(lib().tm_export(h, what, _ptr(out), nbytes), h)


def tm_synchronize(h) -> None:
    _check(lib().tm_synchronize(h), h)


def tm_profile(h, enable) -> None:
    """enable: False/0 off, True/-1 time every class, or a bit mask of classes to time."""
    mask = -1 if enable is True else int(enable)
    _check(lib().tm_profile(h, mask), h)


def tm_profile_kinds() -> int:
    return int(lib().tm_profile_kinds())


def tm_profile_name(kind: int) -> str:
    return lib().tm_profile_name(kind).decode()


def tm_profile_read(h) -> dict:
    """{name: {"launches", "units", "ms"}} since the last tm_profile()."""
    n = tm_profile_kinds()
    la = (c_longlong * n)()
    un = (c_longlong * n)()
    ms = (c_double * n)()
    _check(lib().tm_profile_read(h, la, un, ms, n), h)
    return {tm_profile_name(k): {"launches": la[k], "units": un[k], "ms": ms[k]} for k in range(n)}
