"""Thin ctypes binding over liblogdet.so (argument marshalling only).

Every computation runs inside the CUDA library; this module converts Python
arguments to the C-ABI declared in ``include/logdet.h`` and back.  PyTorch is
used only to hold device memory and streams for the step-level entry points.
There is no CPU fallback: if the library is missing, importing this module
raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LOGDET_LIB", os.path.join(_HERE, "liblogdet.so"))

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"liblogdet.so not found at {LIB_PATH}: build it with "
        "`python -m paper_2606_07004_gb300.build` (needs nvcc); there is no CPU fallback")
_lib = C.CDLL(LIB_PATH)

# ---- constants (logdet.h) --------------------------------------------------
OK, PENDING = 0, 1
EINVAL, ENOMEM, ENOTSPD, ETIMEOUT, ECUDA, ENOENT, ECANCEL = -1, -2, -3, -4, -5, -6, -7
VALS_F64, VALS_F32 = 0, 1
FP64, MIXED_FP32, MIXED_BF16VEC, MIXED_F32X2 = 0, 1, 2, 3
METHOD_OSLQ, METHOD_OSAIOP = 0, 1
ST_BREAKDOWN, ST_NONPOS_RITZ, ST_RANK_DEFICIENT, ST_LOG_FAILED = 1, 2, 4, 8

# The symbols the header declares (checked by the CPU test suite).
EXPORTED = [
    "logdet_opts_default", "logdet_strerror", "logdet_last_error",
    "logdet_create", "logdet_create_device", "logdet_create_grid", "logdet_destroy", "logdet_info",
    "logdet_grid_structure", "logdet_grid_structure_csr", "logdet_oslq", "logdet_osaiop",
    "logdet_probe_fill", "logdet_probe_fill_gaussian", "logdet_spmm", "logdet_quadform",
    "logdet_orth", "logdet_orth_f32",
    "logdet_gauss_quadrature_log", "logdet_hessenberg_log_e1",
    "logdet_launch_count", "logdet_autotune_clear", "logdet_profile_enable", "logdet_profile_reset", "logdet_profile_read",
    "logdet_hessenberg_log_e1_noalloc", "logdet_hessenberg_log_e1_banded",
    "logdet_estimate_bytes", "logdet_server_create", "logdet_server_destroy", "logdet_submit", "logdet_poll",
    "logdet_wait", "logdet_cancel", "logdet_release", "logdet_server_stats",
    "logdet_plan_create", "logdet_plan_run", "logdet_plan_kernels", "logdet_plan_destroy",
    "logdet_oslq_shifts", "logdet_osaiop_shifts", "logdet_suspend", "logdet_resume",
    "logdet_checked_report", "logdet_server_set_log", "logdet_submit_shifts",
]
KC_NAMES = ["spmm", "update", "scalar", "qr", "project", "small", "other", "grid", "krylov_run"]


class logdet_result(C.Structure):
    _fields_ = [
        ("logdet", C.c_double), ("tr_sub", C.c_double), ("tr_res", C.c_double),
        ("log_alpha", C.c_double), ("log_gamma", C.c_double),
        ("s", C.c_int32), ("r", C.c_int32), ("s_eff", C.c_int32),
        ("steps_min", C.c_int32), ("steps_max", C.c_int32),
        ("status_bits", C.c_uint32), ("device_ms", C.c_double),
        ("latency_ms", C.c_double), ("queue_ms", C.c_double),
    ]


class logdet_server_stats(C.Structure):
    _fields_ = [
        ("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
        ("failed", C.c_int64), ("cancelled", C.c_int64), ("queued", C.c_int64),
        ("resident", C.c_int64), ("max_resident", C.c_int64), ("ticks", C.c_int64),
        ("batched_steps", C.c_int64), ("bytes_in_use", C.c_size_t), ("bytes_budget", C.c_size_t),
        ("busy_ms", C.c_double), ("suspended", C.c_int64), ("suspensions", C.c_int64),
        ("suspended_in_krylov", C.c_int64),
    ]


class logdet_opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("tol", C.c_double),
        ("lambda_lo", C.c_double), ("lambda_hi", C.c_double),
        ("autotune", C.c_int32),
        ("per_probe", C.POINTER(C.c_double)), ("z_norm2", C.POINTER(C.c_double)),
        ("stream", C.c_void_p), ("shift", C.c_double),
        ("plain_slq", C.c_int32), ("gaussian_probes", C.c_int32),
        ("block_width", C.c_int32),
    ]


_P = C.c_void_p
_i32, _i64, _u64, _u32, _dbl = C.c_int32, C.c_int64, C.c_uint64, C.c_uint32, C.c_double


def _sig(name, restype, argtypes):
    f = getattr(_lib, name)
    f.restype = restype
    f.argtypes = argtypes
    return f


_sig("logdet_opts_default", None, [C.POINTER(logdet_opts)])
_sig("logdet_strerror", C.c_char_p, [C.c_int])
_sig("logdet_last_error", C.c_char_p, [])
_sig("logdet_create", C.c_int, [_i32, _P, _P, _P, _i32, C.POINTER(_P)])
_sig("logdet_create_device", C.c_int, [_i32, _P, _P, _P, _i32, C.POINTER(_P)])
_sig("logdet_create_grid", C.c_int, [_i32, _i32, _i32, _P, C.POINTER(_P)])
_sig("logdet_destroy", None, [_P])
_sig("logdet_info", C.c_int, [_P, C.POINTER(_i32), C.POINTER(_i64), C.POINTER(_dbl), C.POINTER(_dbl)])
_sig("logdet_grid_structure", C.c_int, [_P, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32)])
_sig("logdet_grid_structure_csr", C.c_int, [_i32, _P, _P, C.POINTER(_i32), C.POINTER(_i32),
                                            C.POINTER(_i32)])
for _n in ("logdet_oslq", "logdet_osaiop"):
    _sig(_n, C.c_int, [_P, _i32, _i32, _i32, _u64, C.POINTER(logdet_opts), C.POINTER(logdet_result)])
for _n in ("logdet_oslq_shifts", "logdet_osaiop_shifts"):
    _sig(_n, C.c_int, [_P, _i32, _P, _i32, _i32, _i32, _u64, C.POINTER(logdet_opts),
                       C.POINTER(logdet_result)])
_sig("logdet_probe_fill", C.c_int, [_u64, _i32, _i32, _i32, _i32, _P, _i32, _P])
_sig("logdet_probe_fill_gaussian", C.c_int, [_u64, _i32, _i32, _i32, _i32, _P, _i32, _P])
_sig("logdet_spmm", C.c_int, [_P, _P, _P, _i32, _i32, _P])
_sig("logdet_quadform", C.c_int, [_P, _P, _dbl, C.POINTER(_dbl), _P])
_sig("logdet_orth", C.c_int, [_i32, _i32, _P, _i32, _P, _i32, C.POINTER(_i32), _P])
_sig("logdet_orth_f32", C.c_int, [_i32, _i32, _P, _i32, _P, _i32, C.POINTER(_i32), _P])
_sig("logdet_gauss_quadrature_log", C.c_int, [_P, _P, _P, _i32, _i32, _dbl, _P, C.POINTER(_u32), _P])
_sig("logdet_hessenberg_log_e1", C.c_int, [_P, _i32, _P, _i32, _i32, _P, C.POINTER(_u32), _P])
_sig("logdet_hessenberg_log_e1_banded", C.c_int,
     [_P, _i32, _P, _i32, _i32, _i32, _P, C.POINTER(_u32), _P])
_sig("logdet_hessenberg_log_e1_noalloc", C.c_int,
     [_P, _i32, _P, _i32, _i32, _P, C.POINTER(_u32), _P])
_sig("logdet_estimate_bytes", C.c_int, [_P, _i32, _i32, _i32, _i32, C.POINTER(logdet_opts),
                                        C.POINTER(C.c_size_t)])
_sig("logdet_server_create", C.c_int, [C.c_size_t, _i32, _P, C.POINTER(_P)])
_sig("logdet_server_destroy", None, [_P])
_sig("logdet_submit", C.c_int, [_P, _P, _i32, _i32, _i32, _i32, _u64, C.POINTER(logdet_opts),
                                C.POINTER(_u64)])
_sig("logdet_poll", C.c_int, [_P, _u64, C.POINTER(logdet_result)])
_sig("logdet_wait", C.c_int, [_P, _u64, _i64, C.POINTER(logdet_result)])
_sig("logdet_cancel", C.c_int, [_P, _u64])
_sig("logdet_suspend", C.c_int, [_P, _u64])
_sig("logdet_server_set_log", C.c_int, [_P, C.c_char_p])
_sig("logdet_submit_shifts", C.c_int, [_P, _P, _i32, _i32, _P, _i32, _i32, _i32, _u64,
                                       C.POINTER(logdet_opts), _P])
_sig("logdet_checked_report", C.c_int, [C.POINTER(_i32), C.POINTER(_u32), C.POINTER(_u64)])
_sig("logdet_resume", C.c_int, [_P, _u64])
_sig("logdet_release", C.c_int, [_P, _u64])
_sig("logdet_server_stats", C.c_int, [_P, C.POINTER(logdet_server_stats)])
_sig("logdet_plan_create", C.c_int, [_P, _i32, _i32, _i32, _i32, C.POINTER(logdet_opts),
                                     C.POINTER(_P)])
_sig("logdet_plan_run", C.c_int, [_P, _u64, C.POINTER(logdet_result), _P, _P])
_sig("logdet_plan_kernels", C.c_int, [_P, C.POINTER(_i64)])
_sig("logdet_plan_destroy", None, [_P])
_sig("logdet_launch_count", C.c_int64, [])
_sig("logdet_autotune_clear", C.c_int, [])
_sig("logdet_profile_enable", C.c_int, [C.c_int])
_sig("logdet_profile_reset", C.c_int, [])
_sig("logdet_profile_read", C.c_int, [_i32, C.POINTER(_i64), C.POINTER(_dbl), C.POINTER(_dbl),
                                      C.POINTER(_dbl)])


def grid_structure_csr(A):
    """(dim, L, reach) of host CSR arrays (object with n, rowptr, colind), as
    a handle would report it (logdet_grid_structure_csr; host only)."""
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.colind, dtype=np.int32)
    dim, L, R = _i32(), _i32(), _i32()
    _check(_lib.logdet_grid_structure_csr(int(A.n), rp.ctypes.data, ci.ctypes.data,
                                          C.byref(dim), C.byref(L), C.byref(R)),
           "logdet_grid_structure_csr")
    return dim.value, L.value, R.value


class LogdetError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.logdet_strerror(code).decode()
        detail = _lib.logdet_last_error().decode()
        super().__init__(f"{where}: {msg} ({code}): {detail}")


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise LogdetError(rc, where)
    return rc


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        return 0
    return getattr(stream, "cuda_stream", stream)


def _make_opts(precision, tol, lam, stream, shift, per, zn, autotune=0, plain=0, gaussian=0,
               block_width=0):
    o = logdet_opts()
    _lib.logdet_opts_default(C.byref(o))
    o.precision = precision
    if tol is not None:
        o.tol = tol
    if lam is not None:
        o.lambda_lo, o.lambda_hi = lam
    o.per_probe = per.ctypes.data_as(C.POINTER(C.c_double))
    o.z_norm2 = zn.ctypes.data_as(C.POINTER(C.c_double))
    o.stream = _stream(stream) or None
    o.shift = shift
    o.autotune = int(autotune)
    o.plain_slq = int(plain)
    o.gaussian_probes = int(gaussian)
    o.block_width = int(block_width)
    return o


def _result(res, per, zn, s, r):
    return Result(res.logdet, res.tr_sub, res.tr_res, res.log_alpha, res.log_gamma,
                  res.s, res.r, res.s_eff, res.steps_min, res.steps_max, res.status_bits,
                  res.device_ms, per[: s + r].copy(), zn[:r].copy(), res.latency_ms, res.queue_ms)


@dataclass
class Result:
    logdet: float
    tr_sub: float
    tr_res: float
    log_alpha: float
    log_gamma: float
    s: int
    r: int
    s_eff: int
    steps_min: int
    steps_max: int
    status_bits: int
    device_ms: float
    per_probe: np.ndarray
    z_norm2: np.ndarray
    latency_ms: float = 0.0
    queue_ms: float = 0.0


class Handle:
    """A CSR matrix resident on the GPU (logdet_create / logdet_create_device)."""

    def __init__(self, n, rowptr, colind, vals, device: bool = False):
        self._h = _P()
        if device:
            dt = VALS_F64 if str(vals.dtype) == "torch.float64" else VALS_F32
            self._keep = (rowptr, colind, vals)
            _check(_lib.logdet_create_device(n, _ptr(rowptr), _ptr(colind), _ptr(vals), dt,
                                             C.byref(self._h)), "logdet_create_device")
        else:
            rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
            colind = np.ascontiguousarray(colind, dtype=np.int32)
            if vals.dtype == np.float32:
                vals = np.ascontiguousarray(vals)
                dt = VALS_F32
            else:
                vals = np.ascontiguousarray(vals, dtype=np.float64)
                dt = VALS_F64
            _check(_lib.logdet_create(n, _ptr(rowptr), _ptr(colind), _ptr(vals), dt,
                                      C.byref(self._h)), "logdet_create")

    @classmethod
    def grid(cls, nx: int, ny: int, table) -> "Handle":
        """Matrix-free gridded operator (logdet_create_grid); table is the
        (R + 1) x (R + 1) quadrant table W(|dy|, |dx|)."""
        w = np.ascontiguousarray(table, dtype=np.float64)
        if w.ndim != 2 or w.shape[0] != w.shape[1]:
            raise ValueError("table must be (R + 1) x (R + 1)")
        h = cls.__new__(cls)
        h._h = _P()
        h._keep = None
        _check(_lib.logdet_create_grid(nx, ny, w.shape[0] - 1, _ptr(w), C.byref(h._h)),
               "logdet_create_grid")
        return h

    @classmethod
    def from_csr(cls, A) -> "Handle":
        """From any object with n, rowptr, colind, vals (host arrays)."""
        return cls(A.n, A.rowptr, A.colind, A.vals)

    def close(self):
        if getattr(self, "_h", None):
            _lib.logdet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def raw(self):
        return self._h

    def info(self):
        n, nnz, lo, hi = _i32(), _i64(), _dbl(), _dbl()
        _check(_lib.logdet_info(self._h, C.byref(n), C.byref(nnz), C.byref(lo), C.byref(hi)),
               "logdet_info")
        return n.value, nnz.value, lo.value, hi.value

    def grid_structure(self):
        """(dim, L, reach): 2 = line sweep (line stride L, lines -reach..reach),
        3 = plane sweep (grid row length L, planes -reach..reach), (0, 0, 0)
        when the matrix has no grid structure (logdet_grid_structure)."""
        dim, L, A = _i32(), _i32(), _i32()
        _check(_lib.logdet_grid_structure(self._h, C.byref(dim), C.byref(L), C.byref(A)),
               "logdet_grid_structure")
        return dim.value, L.value, A.value

    def _run(self, fn, name, num_probes, krylov_steps, iop_window, seed, precision, tol,
             lam, stream, shift=0.0, autotune=0, plain=0, gaussian=0, block_width=0):
        s = 0 if plain else num_probes // 3
        r = num_probes - 2 * s
        per = np.zeros(max(s + r, 1))
        zn = np.zeros(max(r, 1))
        o = _make_opts(precision, tol, lam, stream, shift, per, zn, autotune, plain, gaussian,
                       block_width)
        res = logdet_result()
        _check(fn(self._h, num_probes, krylov_steps, iop_window, seed, C.byref(o), C.byref(res)),
               name)
        return _result(res, per, zn, s, r)

    def oslq(self, num_probes, krylov_steps, seed=0, iop_window=0, precision=FP64, tol=None,
             lam=None, stream=None, shift=0.0, autotune=0, plain=0, gaussian=0,
             block_width=0) -> Result:
        return self._run(_lib.logdet_oslq, "logdet_oslq", num_probes, krylov_steps, iop_window,
                         seed, precision, tol, lam, stream, shift, autotune, plain, gaussian,
                         block_width)

    def osaiop(self, num_probes, krylov_steps, iop_window=2, seed=0, precision=FP64, tol=None,
               lam=None, stream=None, shift=0.0, autotune=0, plain=0, gaussian=0,
               block_width=0) -> Result:
        return self._run(_lib.logdet_osaiop, "logdet_osaiop", num_probes, krylov_steps,
                         iop_window, seed, precision, tol, lam, stream, shift, autotune, plain,
                         gaussian, block_width)

    def _run_shifts(self, fn, name, shifts, num_probes, krylov_steps, iop_window, seed0,
                    precision, tol, lam, stream, autotune, plain, gaussian, block_width):
        sh = np.ascontiguousarray(shifts, dtype=np.float64).ravel()
        s = 0 if plain else num_probes // 3
        r = num_probes - 2 * s
        empty_p, empty_z = np.zeros(0), np.zeros(0)
        o = _make_opts(precision, tol, lam, stream, 0.0, empty_p, empty_z, autotune, plain,
                       gaussian, block_width)
        o.per_probe = None
        o.z_norm2 = None
        res = (logdet_result * max(len(sh), 1))()
        _check(fn(self._h, len(sh), sh.ctypes.data_as(C.c_void_p), num_probes, krylov_steps,
                  iop_window, seed0, C.byref(o), res), name)
        return [_result(res[t], empty_p, empty_z, 0, 0) for t in range(len(sh))]

    def oslq_shifts(self, shifts, num_probes, krylov_steps, seed0=0, iop_window=0,
                    precision=FP64, tol=None, lam=None, stream=None, autotune=0, plain=0,
                    gaussian=0, block_width=0) -> list:
        """log det(Q + shifts[t] I) for every t in one lockstep group
        (logdet_oslq_shifts); member t is oslq(..., seed=seed0 + t, shift=shifts[t])."""
        return self._run_shifts(_lib.logdet_oslq_shifts, "logdet_oslq_shifts", shifts,
                                num_probes, krylov_steps, iop_window, seed0, precision, tol, lam,
                                stream, autotune, plain, gaussian, block_width)

    def osaiop_shifts(self, shifts, num_probes, krylov_steps, iop_window=2, seed0=0,
                      precision=FP64, tol=None, lam=None, stream=None, autotune=0, plain=0,
                      gaussian=0, block_width=0) -> list:
        """The OSA-IOP counterpart (logdet_osaiop_shifts)."""
        return self._run_shifts(_lib.logdet_osaiop_shifts, "logdet_osaiop_shifts", shifts,
                                num_probes, krylov_steps, iop_window, seed0, precision, tol, lam,
                                stream, autotune, plain, gaussian, block_width)

    def estimate_bytes(self, method, num_probes, krylov_steps, iop_window=0, precision=FP64,
                       shift=0.0) -> int:
        o = logdet_opts()
        _lib.logdet_opts_default(C.byref(o))
        o.precision = precision
        o.shift = shift
        out = C.c_size_t()
        _check(_lib.logdet_estimate_bytes(self._h, method, num_probes, krylov_steps, iop_window,
                                          C.byref(o), C.byref(out)), "logdet_estimate_bytes")
        return out.value

    def quadform(self, x, shift: float = 0.0, stream=None) -> float:
        """x^T (Q + shift I) x for a device vector x of n doubles (logdet_quadform)."""
        out = _dbl()
        _check(_lib.logdet_quadform(self._h, _ptr(x), float(shift), C.byref(out), _stream(stream)),
               "logdet_quadform")
        return out.value

    def spmm(self, x, y, b, ld, stream=None):
        _check(_lib.logdet_spmm(self._h, _ptr(x), _ptr(y), b, ld, _stream(stream)), "logdet_spmm")


class Plan:
    """A solve of fixed shape captured into a CUDA graph (logdet_plan_create);
    run(seed) replays it (logdet_plan_run).  Keep the Handle open while the
    plan lives."""

    def __init__(self, handle: Handle, method: int, num_probes: int, krylov_steps: int,
                 iop_window: int = 0, precision=FP64, tol=None, lam=None, stream=None,
                 shift=0.0, autotune=0, plain=0, gaussian=0, block_width=0):
        self._p = _P()
        self._handle = handle
        self.s = 0 if plain else num_probes // 3
        self.r = num_probes - 2 * self.s
        dummy = np.zeros(1)
        o = _make_opts(precision, tol, lam, stream, shift, dummy, dummy, autotune, plain, gaussian,
                       block_width)
        o.per_probe = None
        o.z_norm2 = None
        _check(_lib.logdet_plan_create(handle.raw, method, num_probes, krylov_steps, iop_window,
                                       C.byref(o), C.byref(self._p)), "logdet_plan_create")

    def run(self, seed: int) -> Result:
        per = np.zeros(max(self.s + self.r, 1))
        zn = np.zeros(max(self.r, 1))
        res = logdet_result()
        _check(_lib.logdet_plan_run(self._p, seed, C.byref(res), _ptr(per), _ptr(zn)),
               "logdet_plan_run")
        return _result(res, per, zn, self.s, self.r)

    def kernels(self) -> int:
        k = _i64()
        _check(_lib.logdet_plan_kernels(self._p, C.byref(k)), "logdet_plan_kernels")
        return k.value

    def close(self):
        if getattr(self, "_p", None):
            _lib.logdet_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching server (logdet_server_create / submit / poll / wait)."""

    def __init__(self, budget_bytes: int, max_slots: int = 64, stream=None):
        self._s = _P()
        _check(_lib.logdet_server_create(int(budget_bytes), max_slots, _stream(stream) or None,
                                         C.byref(self._s)), "logdet_server_create")
        self._pending = {}

    def submit(self, handle: Handle, method: int, num_probes: int, krylov_steps: int,
               iop_window: int = 0, seed: int = 0, precision=FP64, tol=None, lam=None,
               shift=0.0, autotune=0, block_width=0) -> int:
        s = num_probes // 3
        r = num_probes - 2 * s
        per = np.zeros(max(s + r, 1))
        zn = np.zeros(max(r, 1))
        o = _make_opts(precision, tol, lam, None, shift, per, zn, autotune, block_width=block_width)
        rid = _u64()
        _check(_lib.logdet_submit(self._s, handle.raw, method, num_probes, krylov_steps, iop_window,
                                  seed, C.byref(o), C.byref(rid)), "logdet_submit")
        self._pending[rid.value] = (per, zn, s, r, handle)
        return rid.value

    def submit_shifts(self, handle: Handle, method: int, shifts, num_probes: int,
                      krylov_steps: int, iop_window: int = 0, seed0: int = 0, precision=FP64,
                      tol=None, lam=None, autotune=0, block_width=0) -> list:
        """A shift group through the server (logdet_submit_shifts): one id per shift."""
        sh = np.ascontiguousarray(shifts, dtype=np.float64).ravel()
        e = np.zeros(0)
        o = _make_opts(precision, tol, lam, None, 0.0, e, e, autotune, block_width=block_width)
        o.per_probe = None
        o.z_norm2 = None
        ids = np.zeros(max(len(sh), 1), dtype=np.uint64)
        _check(_lib.logdet_submit_shifts(self._s, handle.raw, method, len(sh),
                                         sh.ctypes.data_as(C.c_void_p), num_probes, krylov_steps,
                                         iop_window, seed0, C.byref(o),
                                         ids.ctypes.data_as(C.c_void_p)), "logdet_submit_shifts")
        out = [int(x) for x in ids[:len(sh)]]
        for rid in out:
            self._pending[rid] = (e, e, 0, 0, handle)
        return out

    def poll(self, rid: int):
        """None while pending, else the Result (raises LogdetError on failure)."""
        res = logdet_result()
        rc = _lib.logdet_poll(self._s, rid, C.byref(res))
        if rc == PENDING:
            return None
        _check(rc, "logdet_poll")
        per, zn, s, r, _ = self._pending[rid]
        return _result(res, per, zn, s, r)

    def wait(self, rid: int, timeout_us: int = -1):
        res = logdet_result()
        _check(_lib.logdet_wait(self._s, rid, timeout_us, C.byref(res)), "logdet_wait")
        per, zn, s, r, _ = self._pending[rid]
        return _result(res, per, zn, s, r)

    def cancel(self, rid: int):
        _check(_lib.logdet_cancel(self._s, rid), "logdet_cancel")

    def set_log(self, path):
        """Append one JSON line per finished request to `path` (None stops)."""
        p = None if path is None else str(path).encode()
        _check(_lib.logdet_server_set_log(self._s, p), "logdet_server_set_log")

    def suspend(self, rid: int):
        """Preempt a request: its device state moves to host memory (logdet_suspend)."""
        _check(_lib.logdet_suspend(self._s, rid), "logdet_suspend")

    def resume(self, rid: int):
        """Re-queue a suspended request at the front (logdet_resume)."""
        _check(_lib.logdet_resume(self._s, rid), "logdet_resume")

    def release(self, rid: int):
        _check(_lib.logdet_release(self._s, rid), "logdet_release")
        self._pending.pop(rid, None)

    def stats(self) -> dict:
        st = logdet_server_stats()
        _check(_lib.logdet_server_stats(self._s, C.byref(st)), "logdet_server_stats")
        return {f[0]: getattr(st, f[0]) for f in st._fields_}

    def close(self):
        if getattr(self, "_s", None):
            _lib.logdet_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def logdet_create(n, rowptr, colind, vals) -> Handle:
    return Handle(n, rowptr, colind, vals)


def logdet_create_device(n, rowptr, colind, vals) -> Handle:
    return Handle(n, rowptr, colind, vals, device=True)


def logdet_oslq(h: Handle, num_probes, krylov_steps, iop_window=0, seed=0, **kw) -> Result:
    return h.oslq(num_probes, krylov_steps, seed=seed, iop_window=iop_window, **kw)


def logdet_osaiop(h: Handle, num_probes, krylov_steps, iop_window=2, seed=0, **kw) -> Result:
    return h.osaiop(num_probes, krylov_steps, iop_window=iop_window, seed=seed, **kw)


def logdet_probe_fill(seed, stream_id, n, ncols, col0, out, ld, stream=None):
    _check(_lib.logdet_probe_fill(seed, stream_id, n, ncols, col0, _ptr(out), ld, _stream(stream)),
           "logdet_probe_fill")


def logdet_probe_fill_gaussian(seed, stream_id, n, ncols, col0, out, ld, stream=None):
    _check(_lib.logdet_probe_fill_gaussian(seed, stream_id, n, ncols, col0, _ptr(out), ld,
                                           _stream(stream)), "logdet_probe_fill_gaussian")


def logdet_spmm(h: Handle, x, y, b, ld, stream=None):
    h.spmm(x, y, b, ld, stream)


def logdet_orth(n, s, y, ldy, a, lda, stream=None) -> int:
    se = _i32()
    _check(_lib.logdet_orth(n, s, _ptr(y), ldy, _ptr(a), lda, C.byref(se), _stream(stream)),
           "logdet_orth")
    return se.value


def logdet_orth_f32(n, s, y, ldy, a, lda, stream=None) -> int:
    se = _i32()
    _check(_lib.logdet_orth_f32(n, s, _ptr(y), ldy, _ptr(a), lda, C.byref(se), _stream(stream)),
           "logdet_orth_f32")
    return se.value


def logdet_gauss_quadrature_log(alpha, beta, msteps, m, nprobe, clamp_lo, out, stream=None) -> int:
    st = _u32()
    _check(_lib.logdet_gauss_quadrature_log(_ptr(alpha), _ptr(beta), _ptr(msteps), m, nprobe,
                                            clamp_lo, _ptr(out), C.byref(st), _stream(stream)),
           "logdet_gauss_quadrature_log")
    return st.value


def logdet_hessenberg_log_e1(H, ldh, msteps, m, nprobe, c, stream=None) -> int:
    st = _u32()
    _check(_lib.logdet_hessenberg_log_e1(_ptr(H), ldh, _ptr(msteps), m, nprobe, _ptr(c),
                                         C.byref(st), _stream(stream)),
           "logdet_hessenberg_log_e1")
    return st.value


def logdet_hessenberg_log_e1_banded(H, ldh, msteps, m, nprobe, band, c, stream=None) -> int:
    st = _u32()
    _check(_lib.logdet_hessenberg_log_e1_banded(_ptr(H), ldh, _ptr(msteps), m, nprobe, band,
                                                _ptr(c), C.byref(st), _stream(stream)),
           "logdet_hessenberg_log_e1_banded")
    return st.value


def logdet_hessenberg_log_e1_noalloc(H, ldh, msteps, m, nprobe, c, stream=None) -> int:
    """Allocation-free variant of logdet_hessenberg_log_e1 (static scratch in the library)."""
    st = _u32()
    _check(_lib.logdet_hessenberg_log_e1_noalloc(_ptr(H), ldh, _ptr(msteps), m, nprobe, _ptr(c),
                                                 C.byref(st), _stream(stream)),
           "logdet_hessenberg_log_e1_noalloc")
    return st.value


def logdet_launch_count() -> int:
    return int(_lib.logdet_launch_count())


def logdet_profile_enable(on: bool = True):
    _check(_lib.logdet_profile_enable(1 if on else 0), "logdet_profile_enable")


def logdet_profile_reset():
    _check(_lib.logdet_profile_reset(), "logdet_profile_reset")


def logdet_profile_read(kclass: int) -> dict:
    n, ms, fl, by = _i64(), _dbl(), _dbl(), _dbl()
    _check(_lib.logdet_profile_read(kclass, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)),
           "logdet_profile_read")
    return {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}


def profile_snapshot() -> dict:
    return {name: logdet_profile_read(i) for i, name in enumerate(KC_NAMES)}


def exported_symbols() -> list[str]:
    return [name for name in EXPORTED if hasattr(_lib, name)]


def checked_report() -> dict:
    """State of the checks of a checked build (logdet_checked_report)."""
    c, v, b = _i32(), _u32(), _u64()
    _check(_lib.logdet_checked_report(C.byref(c), C.byref(v), C.byref(b)), "logdet_checked_report")
    return {"checked": bool(c.value), "device_violations": v.value, "canary_bytes": b.value}
