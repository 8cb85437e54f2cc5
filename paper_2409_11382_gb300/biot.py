"""Thin Python binding of the C ABI declared in ``include/biot.h``.

Argument marshalling only: every step of the solver runs in the sm_103a
kernels of ``libbiot_gb300.so``.  There is no CPU fallback -- loading fails
with an error if the shared library has not been built, and creating an
instance fails if no CUDA device is visible.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbiot_gb300.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_DIVERGED, ERR_NOT_CONVERGED, ERR_CUDA, ERR_TIMEOUT, ERR_NO_DEVICE = (
    0, -1, -2, -3, -4, -5, -6, -7)
FP64, FP32, FP32_COARSE64, FP32_DEV16, FP32_DEVBF16 = 0, 1, 2, 3, 4
CYCLE_V, CYCLE_W, CYCLE_F = 0, 1, 2
# biot_params.options (include/biot.h)
OPT_COARSEST_STORAGE, OPT_COLD_FP64, OPT_COLD_FP32, OPT_COARSE_LO_ALL, OPT_COARSE_LO_OFF = 1, 2, 4, 8, 16
OPT_SEGMENTS = 32
PERIODIC, SYMMETRY, DIRICHLET, NEUMANN = 0, 1, 2, 3
BOTTOM, RIGHT, TOP, LEFT = 0, 1, 2, 3

# Every function the header declares (checked by the tests against include/biot.h).
API_FUNCTIONS = (
    "biot_create", "biot_destroy", "biot_set_stream", "biot_set_sources", "biot_set_side_profile",
    "biot_step", "biot_solve_to", "biot_read_u", "biot_read_p", "biot_read_stress",
    "biot_stats_get", "biot_error_string", "biot_last_error", "biot_sweep_timing",
    "biot_sweep_timing_get", "biot_read_u_noalloc", "biot_read_async", "biot_read_wait",
    "biot_step_async", "biot_sync", "biot_batch_step_async", "biot_batch_sync",
    "biot_batch_create", "biot_batch_destroy", "biot_batch_size", "biot_batch_instance",
    "biot_batch_step", "biot_batch_stats_get", "biot_batch_read_async", "biot_batch_read_wait",
    "biot_estimate_bytes", "biot_server_create", "biot_server_submit", "biot_server_poll",
    "biot_server_wait", "biot_server_fetch", "biot_server_release", "biot_server_stats_get",
    "biot_server_destroy", "biot_autotune", "biot_checkpoint_size", "biot_save", "biot_load",
    "biot_autotune_sweeps",
)
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3
NOALLOC_MAX_CELLS = 262144  # BIOT_NOALLOC_MAX_CELLS of include/biot.h


class BiotError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where} failed with code {code}: {detail}")
        self.code = code


class biot_params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("lambda_", C.c_double), ("mu", C.c_double), ("alpha", C.c_double),
                ("c0", C.c_double), ("kappa", C.c_double), ("dt", C.c_double),
                ("r_coupling", C.c_double), ("mg_levels", C.c_int), ("K", C.c_int),
                ("gamma", C.c_double), ("tol", C.c_double), ("ne_max", C.c_int),
                ("ne_fixed", C.c_int), ("precision", C.c_int), ("options", C.c_int),
                ("cycle", C.c_int), ("fmg", C.c_int), ("pgrad", C.c_int), ("K_level", C.c_int * 16)]


class biot_side(C.Structure):
    _fields_ = [("eta_type", C.c_int), ("p_type", C.c_int),
                ("eta_profile", C.POINTER(C.c_double)), ("p_profile", C.POINTER(C.c_double))]


class biot_request_info(C.Structure):
    _fields_ = [("state", C.c_int), ("status", C.c_int), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double), ("nx", C.c_int), ("ny", C.c_int),
                ("steps", C.c_long), ("device_bytes", C.c_size_t)]


class biot_server_stats(C.Structure):
    _fields_ = [("queued", C.c_int), ("peak_resident", C.c_int), ("used_bytes", C.c_size_t),
                ("peak_bytes", C.c_size_t), ("ticks", C.c_long), ("graph_launches", C.c_long),
                ("graphs_reused", C.c_long)]


class biot_stats(C.Structure):
    _fields_ = [("last_ne", C.c_int), ("last_res", C.c_double), ("total_cycles", C.c_long),
                ("notconv_steps", C.c_int), ("diverged", C.c_int), ("nstep", C.c_long),
                ("t", C.c_double), ("omega", C.c_double), ("omega_s", C.c_double),
                ("omega_d", C.c_double), ("kernel_launches", C.c_long),
                ("device_bytes", C.c_size_t), ("last_res_l2", C.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load ``libbiot_gb300.so``; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    P = C.POINTER(C.c_double)
    H = C.c_void_p
    lib.biot_create.argtypes = [C.POINTER(biot_params), C.POINTER(biot_side), C.POINTER(H)]
    lib.biot_destroy.argtypes = [H]
    lib.biot_set_stream.argtypes = [H, C.c_void_p]
    lib.biot_set_sources.argtypes = [H, P, P]
    lib.biot_set_side_profile.argtypes = [H, C.c_int, P, P]
    lib.biot_step.argtypes = [H, C.c_int]
    lib.biot_solve_to.argtypes = [H, C.c_double]
    lib.biot_read_u.argtypes = [H, P, P]
    lib.biot_read_p.argtypes = [H, P, P]
    lib.biot_read_stress.argtypes = [H, P]
    lib.biot_stats_get.argtypes = [H, C.POINTER(biot_stats)]
    lib.biot_error_string.argtypes = [C.c_int]
    lib.biot_error_string.restype = C.c_char_p
    lib.biot_last_error.argtypes = []
    lib.biot_last_error.restype = C.c_char_p
    lib.biot_sweep_timing.argtypes = [H, C.c_int]
    lib.biot_sweep_timing_get.argtypes = [H, P, C.POINTER(C.c_long)]
    lib.biot_read_u_noalloc.argtypes = [H, P, P]
    lib.biot_read_async.argtypes = [H, P, P, P, P]
    lib.biot_read_wait.argtypes = [H]
    lib.biot_step_async.argtypes = [H, C.c_int]
    lib.biot_sync.argtypes = [H]
    lib.biot_batch_step_async.argtypes = [H, C.c_int]
    lib.biot_batch_sync.argtypes = [H]
    lib.biot_batch_create.argtypes = [C.c_int, C.POINTER(biot_params), C.POINTER(biot_side), C.POINTER(H)]
    lib.biot_batch_destroy.argtypes = [H]
    lib.biot_batch_size.argtypes = [H, C.POINTER(C.c_int)]
    lib.biot_batch_instance.argtypes = [H, C.c_int, C.POINTER(H)]
    lib.biot_batch_step.argtypes = [H, C.c_int]
    lib.biot_batch_stats_get.argtypes = [H, C.POINTER(C.c_long), C.POINTER(C.c_long), C.POINTER(C.c_long)]
    PP = C.POINTER(C.POINTER(C.c_double))
    lib.biot_batch_read_async.argtypes = [H, PP, PP, PP, P]
    lib.biot_batch_read_wait.argtypes = [H]
    lib.biot_autotune.argtypes = [H, C.POINTER(C.c_int), P, C.c_int]
    lib.biot_autotune_sweeps.argtypes = [H, C.c_int, C.POINTER(C.c_int), P, P]
    lib.biot_checkpoint_size.argtypes = [H, C.POINTER(C.c_size_t)]
    lib.biot_save.argtypes = [H, C.c_void_p, C.c_size_t]
    lib.biot_load.argtypes = [H, C.c_void_p, C.c_size_t]
    lib.biot_estimate_bytes.argtypes = [C.POINTER(biot_params), C.POINTER(biot_side), C.POINTER(C.c_size_t)]
    lib.biot_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(H)]
    lib.biot_server_submit.argtypes = [H, C.POINTER(biot_params), C.POINTER(biot_side), C.c_double,
                                       C.POINTER(C.c_uint64)]
    lib.biot_server_poll.argtypes = [H, C.c_uint64, C.POINTER(biot_request_info)]
    lib.biot_server_wait.argtypes = [H, C.c_uint64, C.c_double]
    lib.biot_server_fetch.argtypes = [H, C.c_uint64, P, P, P]
    lib.biot_server_release.argtypes = [H, C.c_uint64]
    lib.biot_server_stats_get.argtypes = [H, C.POINTER(biot_server_stats)]
    lib.biot_server_destroy.argtypes = [H]
    for name in API_FUNCTIONS:
        if name not in ("biot_error_string", "biot_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return C.POINTER(C.c_double)()
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> Optional[np.ndarray]:
    if a is None:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


def _fill_params(p: "biot_params", params: dict) -> "biot_params":
    p.nx, p.ny = int(params["nx"]), int(params["ny"])
    p.lx, p.ly = float(params["lx"]), float(params["ly"])
    p.lambda_, p.mu = float(params["lam"]), float(params["mu"])
    p.alpha, p.c0, p.kappa = float(params["alpha"]), float(params["c0"]), float(params["kappa"])
    p.dt, p.r_coupling = float(params["dt"]), float(params.get("r", 0.5))
    p.mg_levels, p.K = int(params["levels"]), int(params["K"])
    p.gamma, p.tol = float(params["gamma"]), float(params["tol"])
    p.ne_max, p.ne_fixed = int(params["ne_max"]), int(params["ne_fixed"])
    p.precision = int(params.get("precision", FP64))
    p.options = int(params.get("options", 0))
    p.cycle = int(params.get("cycle", CYCLE_V))
    p.fmg = int(params.get("fmg", 0))
    p.pgrad = int(params.get("pgrad", 0))
    ks = [int(k) for k in params.get("K_level", ())] + [0] * 16
    p.K_level = (C.c_int * 16)(*ks[:16])
    return p


def _fill_sides(arr, base: int, sides: Sequence[dict]) -> list:
    """Fill arr[base .. base+3] from four side dicts; returns the arrays to keep alive."""
    keep = []
    for i, s in enumerate(sides):
        arr[base + i].eta_type = int(s["eta_type"])
        arr[base + i].p_type = int(s["p_type"])
        for key in ("eta_profile", "p_profile"):
            v = _f64(s.get(key))
            if v is not None:
                keep.append(v)
            setattr(arr[base + i], key, _dptr(v))
    return keep


class Solver:
    """One instance of the coupled problem on the current CUDA device.

    ``params`` uses the keys of ``biot_params`` (``lam`` for lambda); ``sides``
    is a list of four dicts (bottom, right, top, left) with ``eta_type``,
    ``p_type`` and optional ``eta_profile`` / ``p_profile`` arrays.
    Methods map one-to-one onto the C entry points.
    """

    def __init__(self, params: dict, sides: Sequence[dict], stream: Optional[int] = None,
                 _handle: Optional[C.c_void_p] = None, _owner=None):
        self._lib = load_library()
        self._owner = _owner  # a Batch that owns this instance (not destroyed here)
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        if _handle is not None:
            self._h = _handle
            return
        p = _fill_params(biot_params(), params)
        arr = (biot_side * 4)()
        keep = _fill_sides(arr, 0, sides)
        h = C.c_void_p()
        self._check(self._lib.biot_create(C.byref(p), arr, C.byref(h)), "biot_create")
        del keep
        self._h = h
        if stream is not None:
            self.set_stream(stream)

    # -- helpers --------------------------------------------------------------------
    def _check(self, code: int, where: str, allow=(OK,)):
        if code not in allow:
            detail = self._lib.biot_last_error().decode(errors="replace")
            raise BiotError(code, where, detail)
        return code

    def close(self):
        if getattr(self, "_owner", None) is not None:
            self._h = None
            return
        if getattr(self, "_h", None):
            self._lib.biot_destroy(self._h)
            self._h = None

    destroy = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API --------------------------------------------------------------------------
    def set_stream(self, stream: Optional[int]):
        self._check(self._lib.biot_set_stream(self._h, C.c_void_p(stream or 0)), "biot_set_stream")

    def set_sources(self, f_body=None, s=None):
        fb, sr = _f64(f_body), _f64(s)
        self._check(self._lib.biot_set_sources(self._h, _dptr(fb), _dptr(sr)), "biot_set_sources")

    def set_side_profile(self, side: int, eta_profile=None, p_profile=None):
        e, p = _f64(eta_profile), _f64(p_profile)
        self._check(self._lib.biot_set_side_profile(self._h, side, _dptr(e), _dptr(p)),
                    "biot_set_side_profile")

    def step(self, n: int = 1, allow_not_converged: bool = True) -> int:
        allow = (OK, ERR_NOT_CONVERGED) if allow_not_converged else (OK,)
        return self._check(self._lib.biot_step(self._h, int(n)), "biot_step", allow)

    def step_async(self, n: int = 1):
        """biot_step_async: queue n steps and return without waiting for them."""
        self._check(self._lib.biot_step_async(self._h, int(n)), "biot_step_async")

    def sync(self, allow_not_converged: bool = True) -> int:
        """biot_sync: wait for the queued steps and reads; their status."""
        allow = (OK, ERR_NOT_CONVERGED) if allow_not_converged else (OK,)
        code = self._check(self._lib.biot_sync(self._h), "biot_sync", allow)
        self._inflight = []
        return code

    def solve_to(self, T: float, allow_not_converged: bool = True) -> int:
        allow = (OK, ERR_NOT_CONVERGED) if allow_not_converged else (OK,)
        return self._check(self._lib.biot_solve_to(self._h, float(T)), "biot_solve_to", allow)

    def read_u(self, out: Optional[np.ndarray] = None):
        out = np.empty((2, self.ny, self.nx)) if out is None else out
        t = C.c_double()
        self._check(self._lib.biot_read_u(self._h, _dptr(out), C.byref(t)), "biot_read_u")
        return out, t.value

    def read_u_noalloc(self, out: Optional[np.ndarray] = None):
        """biot_read_u_noalloc: the displacement staged through the library's
        static device array instead of an allocated buffer."""
        out = np.empty((2, self.ny, self.nx)) if out is None else out
        t = C.c_double()
        self._check(self._lib.biot_read_u_noalloc(self._h, _dptr(out), C.byref(t)), "biot_read_u_noalloc")
        return out, t.value

    def read_p(self, out: Optional[np.ndarray] = None):
        out = np.empty((self.ny, self.nx)) if out is None else out
        t = C.c_double()
        self._check(self._lib.biot_read_p(self._h, _dptr(out), C.byref(t)), "biot_read_p")
        return out, t.value

    def read_async(self, eta: Optional[np.ndarray] = None, p: Optional[np.ndarray] = None,
                   sigma: Optional[np.ndarray] = None) -> float:
        """biot_read_async: enqueue the read-out of the given fields into these
        host arrays and return their time; the arrays are filled once read_wait
        returns (page-locked arrays make the copy overlap later steps)."""
        shapes = ((eta, (2, self.ny, self.nx)), (p, (self.ny, self.nx)), (sigma, (3, self.ny, self.nx)))
        for a, shape in shapes:
            if a is not None and (a.dtype != np.float64 or a.shape != shape or not a.flags.c_contiguous
                                  or not a.flags.writeable):
                raise ValueError(f"read_async needs a writeable C-contiguous float64 array of shape {shape}")
        t = C.c_double()
        self._check(self._lib.biot_read_async(self._h, _dptr(eta), _dptr(p), _dptr(sigma), C.byref(t)),
                    "biot_read_async")
        self._inflight = getattr(self, "_inflight", []) + [a for a, _ in shapes if a is not None]
        return t.value

    def read_wait(self):
        """biot_read_wait: every read_async issued so far has reached its arrays."""
        self._check(self._lib.biot_read_wait(self._h), "biot_read_wait")
        self._inflight = []

    def read_stress(self, out: Optional[np.ndarray] = None):
        out = np.empty((3, self.ny, self.nx)) if out is None else out
        self._check(self._lib.biot_read_stress(self._h, _dptr(out)), "biot_read_stress")
        return out

    def save(self) -> bytes:
        """biot_save: the resumable state as bytes."""
        n = C.c_size_t()
        self._check(self._lib.biot_checkpoint_size(self._h, C.byref(n)), "biot_checkpoint_size")
        buf = C.create_string_buffer(n.value)
        self._check(self._lib.biot_save(self._h, buf, n), "biot_save")
        return buf.raw

    def load(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        self._check(self._lib.biot_load(self._h, buf, len(data)), "biot_load")

    def autotune(self, levels: int = 16) -> dict:
        """biot_autotune: strip height and time per level and sweep mode."""
        rows = (C.c_int * (2 * levels))()
        ms = (C.c_double * (2 * levels))()
        self._check(self._lib.biot_autotune(self._h, rows, ms, levels), "biot_autotune")
        out = {}
        for l in range(levels):
            for m, name in ((0, "smooth"), (1, "restrict")):
                if rows[2 * l + m]:
                    out[f"L{l}_{name}"] = (rows[2 * l + m], round(ms[2 * l + m], 5))
        return out

    def autotune_sweeps(self, apply: bool = True) -> dict:
        """biot_autotune_sweeps: smoothing sweeps per level (finest first), the
        residual contraction per V-cycle and the time of a V-cycle they give."""
        k = (C.c_int * 16)()
        rho, ms = C.c_double(), C.c_double()
        self._check(self._lib.biot_autotune_sweeps(self._h, int(apply), k, C.byref(rho), C.byref(ms)),
                    "biot_autotune_sweeps")
        return {"K_level": [int(v) for v in k if v > 0], "rho": rho.value, "ms_per_cycle": ms.value}

    def stats(self) -> dict:
        s = biot_stats()
        self._check(self._lib.biot_stats_get(self._h, C.byref(s)), "biot_stats_get")
        return {name: getattr(s, name) for name, _ in biot_stats._fields_}

    def sweep_timing(self, enable: bool):
        self._check(self._lib.biot_sweep_timing(self._h, int(enable)), "biot_sweep_timing")

    def sweep_timing_get(self):
        ms = C.c_double()
        n = C.c_long()
        self._check(self._lib.biot_sweep_timing_get(self._h, C.byref(ms), C.byref(n)),
                    "biot_sweep_timing_get")
        return ms.value, n.value


class Batch:
    """Many instances advanced together (biot_batch_*).  ``problems`` is a list of
    (params, sides) pairs; ``batch[i]`` is a Solver view of instance i (owned by
    the batch) for read-out."""

    def __init__(self, problems: Sequence):
        self._lib = load_library()
        n = len(problems)
        ps = (biot_params * n)()
        arr = (biot_side * (4 * n))()
        keep = []
        for i, (params, sides) in enumerate(problems):
            _fill_params(ps[i], params)
            keep += _fill_sides(arr, 4 * i, sides)
        h = C.c_void_p()
        code = self._lib.biot_batch_create(n, ps, arr, C.byref(h))
        if code != OK:
            raise BiotError(code, "biot_batch_create", self._lib.biot_last_error().decode(errors="replace"))
        self._h = h
        self._views = []
        for i, (params, _) in enumerate(problems):
            ih = C.c_void_p()
            self._lib.biot_batch_instance(self._h, i, C.byref(ih))
            self._views.append(Solver(params, None, _handle=ih, _owner=self))

    def __len__(self):
        return len(self._views)

    def __getitem__(self, i) -> Solver:
        return self._views[i]

    def step(self, n: int = 1) -> int:
        code = self._lib.biot_batch_step(self._h, int(n))
        if code not in (OK, ERR_NOT_CONVERGED):
            raise BiotError(code, "biot_batch_step", self._lib.biot_last_error().decode(errors="replace"))
        return code

    def step_async(self, n: int = 1):
        """biot_batch_step_async: queue n steps of every instance without waiting."""
        code = self._lib.biot_batch_step_async(self._h, int(n))
        if code != OK:
            raise BiotError(code, "biot_batch_step_async", self._lib.biot_last_error().decode(errors="replace"))

    def sync(self) -> int:
        """biot_batch_sync: wait for every instance's queued steps and reads."""
        code = self._lib.biot_batch_sync(self._h)
        if code not in (OK, ERR_NOT_CONVERGED):
            raise BiotError(code, "biot_batch_sync", self._lib.biot_last_error().decode(errors="replace"))
        self._inflight = []
        for v in self._views:
            v._inflight = []
        return code

    def read_async(self, eta=None, p=None, sigma=None):
        """biot_batch_read_async: per instance i, eta[i] / p[i] / sigma[i] are its
        host arrays (a list or an entry may be None); returns the instances'
        times.  The arrays are filled once read_wait returns."""
        n = len(self._views)
        lists = []
        for arrs, comps in ((eta, 2), (p, 1), (sigma, 3)):
            if arrs is None:
                lists.append(None)
                continue
            if len(arrs) != n:
                raise ValueError(f"need one entry per instance ({n})")
            for v, a in zip(self._views, arrs):
                shape = (v.ny, v.nx) if comps == 1 else (comps, v.ny, v.nx)
                if a is not None and (a.dtype != np.float64 or a.shape != shape or not a.flags.c_contiguous
                                      or not a.flags.writeable):
                    raise ValueError(f"read_async needs writeable C-contiguous float64 arrays of shape {shape}")
            lists.append((C.POINTER(C.c_double) * n)(*[_dptr(a) for a in arrs]))
        t = np.zeros(n)
        code = self._lib.biot_batch_read_async(self._h, *lists, _dptr(t))
        if code != OK:
            raise BiotError(code, "biot_batch_read_async", self._lib.biot_last_error().decode(errors="replace"))
        self._inflight = getattr(self, "_inflight", []) + [x for x in (eta, p, sigma) if x is not None]
        return t

    def read_wait(self):
        code = self._lib.biot_batch_read_wait(self._h)
        if code != OK:
            raise BiotError(code, "biot_batch_read_wait", self._lib.biot_last_error().decode(errors="replace"))
        self._inflight = []

    def stats(self) -> dict:
        a, b, c = C.c_long(), C.c_long(), C.c_long()
        self._lib.biot_batch_stats_get(self._h, C.byref(a), C.byref(b), C.byref(c))
        return dict(kernel_launches=a.value, launches_per_step=b.value, work_items_per_step=c.value)

    def close(self):
        if getattr(self, "_h", None):
            for v in self._views:
                v._h = None
            self._lib.biot_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def estimate_bytes(params: dict, sides: Sequence[dict]) -> int:
    lib = load_library()
    p = _fill_params(biot_params(), params)
    arr = (biot_side * 4)()
    keep = _fill_sides(arr, 0, sides)
    n = C.c_size_t()
    code = lib.biot_estimate_bytes(C.byref(p), arr, C.byref(n))
    del keep
    if code != OK:
        raise BiotError(code, "biot_estimate_bytes", lib.biot_last_error().decode(errors="replace"))
    return n.value


class Server:
    """Continuous-batching request loop (biot_server_*) on the current device."""

    def __init__(self, mem_budget_bytes: int, max_resident: int):
        self._lib = load_library()
        h = C.c_void_p()
        self._check(self._lib.biot_server_create(C.c_size_t(int(mem_budget_bytes)), int(max_resident), C.byref(h)),
                    "biot_server_create")
        self._h = h
        self._shape = {}

    def _check(self, code: int, where: str, allow=(OK,)):
        if code not in allow:
            raise BiotError(code, where, self._lib.biot_last_error().decode(errors="replace"))
        return code

    def submit(self, params: dict, sides: Sequence[dict], T: float) -> int:
        p = _fill_params(biot_params(), params)
        arr = (biot_side * 4)()
        keep = _fill_sides(arr, 0, sides)
        rid = C.c_uint64()
        self._check(self._lib.biot_server_submit(self._h, C.byref(p), arr, float(T), C.byref(rid)),
                    "biot_server_submit")
        del keep
        self._shape[rid.value] = (int(params["ny"]), int(params["nx"]))
        return rid.value

    def poll(self, rid: int) -> dict:
        info = biot_request_info()
        self._check(self._lib.biot_server_poll(self._h, C.c_uint64(rid), C.byref(info)), "biot_server_poll")
        return {name: getattr(info, name) for name, _ in biot_request_info._fields_}

    def wait(self, rid: int, timeout: float = 600.0) -> int:
        return self._check(self._lib.biot_server_wait(self._h, C.c_uint64(rid), float(timeout)), "biot_server_wait")

    def fetch(self, rid: int):
        ny, nx = self._shape[rid]
        eta = np.empty((2, ny, nx))
        p = np.empty((ny, nx))
        t = C.c_double()
        self._check(self._lib.biot_server_fetch(self._h, C.c_uint64(rid), _dptr(eta), _dptr(p), C.byref(t)),
                    "biot_server_fetch")
        return eta, p, t.value

    def release(self, rid: int):
        self._check(self._lib.biot_server_release(self._h, C.c_uint64(rid)), "biot_server_release")
        self._shape.pop(rid, None)

    def stats(self) -> dict:
        st = biot_server_stats()
        self._check(self._lib.biot_server_stats_get(self._h, C.byref(st)), "biot_server_stats_get")
        return {name: getattr(st, name) for name, _ in biot_server_stats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.biot_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
