"""ctypes wrapper of the FP64 CPU oracle (``biot_oracle.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It never touches the
CUDA library and the CUDA library never touches it.

The oracle is a plain restatement of the paper's Alg. 5 / 4 / 2 / 3 in FP64,
compiled with ``-O2 -ffp-contract=off`` so that no fused multiply-add changes
its rounding on any host.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "biot_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libbiot_oracle.so")
_lock = threading.Lock()
_lib = None
# Build flavours of the same source: "standard" (the oracle), and
# "reassociated", which lets the compiler reorder FP64 sums (no other change).
# The second one exists for one test only: how far the order of FP64 roundings
# alone moves the oracle's results at a given grid size.
_FLAVOURS = {"standard": ("libbiot_oracle.so", []),
             "reassociated": ("libbiot_oracle_reassoc.so",
                              ["-fassociative-math", "-fno-signed-zeros", "-fno-trapping-math"])}
_libs = {}

PERIODIC, SYMMETRY, DIRICHLET, NEUMANN = 0, 1, 2, 3
BOTTOM, RIGHT, TOP, LEFT = 0, 1, 2, 3


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("lam", C.c_double), ("mu", C.c_double), ("alpha", C.c_double),
                ("c0", C.c_double), ("kappa", C.c_double), ("dt", C.c_double),
                ("r", C.c_double), ("levels", C.c_int), ("K", C.c_int),
                ("gamma", C.c_double), ("tol", C.c_double), ("ne_max", C.c_int),
                ("ne_fixed", C.c_int), ("cycle", C.c_int), ("fmg", C.c_int), ("pgrad", C.c_int),
                ("K_level", C.c_int * 16)]


class _Side(C.Structure):
    _fields_ = [("eta_type", C.c_int), ("p_type", C.c_int),
                ("eta_profile", C.POINTER(C.c_double)), ("p_profile", C.POINTER(C.c_double))]


class _Stats(C.Structure):
    _fields_ = [("last_ne", C.c_int), ("last_res", C.c_double), ("total_cycles", C.c_long),
                ("notconv_steps", C.c_int), ("diverged", C.c_int), ("nstep", C.c_long),
                ("t", C.c_double), ("omega", C.c_double), ("om_s", C.c_double),
                ("om_d", C.c_double), ("kap_lattice", C.c_double), ("last_res_l2", C.c_double)]


def build(force: bool = False, flavour: str = "standard") -> str:
    """Compile the oracle into a shared library next to it (gcc, FP64, no FMA contraction)."""
    name, extra = _FLAVOURS[flavour]
    lib_path = os.path.join(_HERE, "_build", name)
    with _lock:
        if (not force and os.path.exists(lib_path)
                and os.path.getmtime(lib_path) >= os.path.getmtime(_SRC)):
            return lib_path
        os.makedirs(os.path.dirname(lib_path), exist_ok=True)
        tmp = lib_path + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math"] + extra + [
            "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP for the per-cell loops (orc_set_threads); without it the
        # pragmas are ignored and the oracle runs on one thread
        if subprocess.run(cmd[:-1] + ["-fopenmp", "-lm"], capture_output=True).returncode != 0:
            subprocess.run(cmd, check=True)
        os.replace(tmp, lib_path)
        return lib_path


def _load(flavour: str = "standard"):
    global _lib
    if flavour != "standard":
        if flavour not in _libs:
            _libs[flavour] = _declare(C.CDLL(build(flavour=flavour)))
        return _libs[flavour]
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def _declare(lib):
    """Argument and result types of the oracle's C functions."""
    P = C.POINTER(C.c_double)
    lib.orc_create.restype = C.c_void_p
    lib.orc_create.argtypes = [C.POINTER(_Params), C.POINTER(_Side)]
    lib.orc_destroy.argtypes = [C.c_void_p]
    for name in ("orc_step",):
        getattr(lib, name).argtypes = [C.c_void_p, C.c_int]
    lib.orc_solve_to.argtypes = [C.c_void_p, C.c_double]
    lib.orc_set_sources.argtypes = [C.c_void_p, P, P]
    lib.orc_read_u.argtypes = [C.c_void_p, P, P]
    lib.orc_read_p.argtypes = [C.c_void_p, P, P]
    lib.orc_read_stress.argtypes = [C.c_void_p, P]
    lib.orc_stats_get.argtypes = [C.c_void_p, C.POINTER(_Stats)]
    lib.orc_collide_cell.argtypes = [C.c_double, C.c_double, P, P, P]
    lib.orc_inverse_table.argtypes = [P]
    lib.orc_prepare_elastic.argtypes = [C.c_void_p]
    lib.orc_fixed_point_map.argtypes = [C.c_void_p, P, P]
    lib.orc_vcycle.argtypes = [C.c_void_p, C.c_int]
    lib.orc_vcycle.restype = C.c_double
    lib.orc_plain_pseudo_step.argtypes = [C.c_void_p]
    for name in ("orc_get_g", "orc_set_g", "orc_get_f", "orc_set_f"):
        getattr(lib, name).argtypes = [C.c_void_p, P]
    lib.orc_set_threads.argtypes = [C.c_int]
    lib.orc_get_threads.restype = C.c_int
    lib.orc_openmp.restype = C.c_int
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def collide_cell(lam_hat: float, mu_hat: float, g, F) -> np.ndarray:
    """Post-collision populations of one cell (Alg. 2, collision part), lattice units."""
    lib = _load()
    g = np.ascontiguousarray(g, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    out = np.zeros(8)
    lib.orc_collide_cell(lam_hat, mu_hat, _ptr(g), _ptr(F), _ptr(out))
    return out


def set_threads(n: int) -> int:
    """Threads of the oracle's per-cell loops (1 = serial, the default; the
    results are bitwise the same for every count).  Returns the count in use;
    it stays 1 when the oracle was built without OpenMP."""
    lib = _load()
    lib.orc_set_threads(int(n))
    return int(lib.orc_get_threads()) if openmp_enabled() else 1


def openmp_enabled() -> bool:
    """Whether the oracle library was built with OpenMP."""
    return bool(_load().orc_openmp())


def inverse_table() -> np.ndarray:
    """The oracle's copy of Tab. moments:inverse (rows ij, columns 10,01,11,s,d,12,21,22)."""
    out = np.zeros(64)
    _load().orc_inverse_table(_ptr(out))
    return out.reshape(8, 8)


class Oracle:
    """One instance of the coupled problem.

    ``params``: dict with keys nx, ny, lx, ly, lam, mu, alpha, c0, kappa, dt, r,
    levels, K, gamma, tol, ne_max, ne_fixed.
    ``sides``: list of 4 dicts (bottom, right, top, left) with ``eta_type``,
    ``p_type`` and optional ``eta_profile`` (2 x (2n+1)) / ``p_profile`` (2n+1).
    """

    def __init__(self, params: dict, sides, flavour: str = "standard"):
        lib = _load(flavour)
        self._lib = lib
        p = _Params()
        for name, _ in _Params._fields_:
            if name == "K_level":  # per-level sweeps (level j below the finest); 0 = K
                ks = list(params.get("K_level", ())) + [0] * 16
                p.K_level = (C.c_int * 16)(*ks[:16])
                continue
            # cycle, fmg, pgrad default to the paper's V-cycle and eq. pressure:gradient
            setattr(p, name, params[name] if name in params or name not in ("cycle", "fmg", "pgrad") else 0)
        self.nx, self.ny = params["nx"], params["ny"]
        self._keep = []
        arr = (_Side * 4)()
        for i, s in enumerate(sides):
            arr[i].eta_type = s["eta_type"]
            arr[i].p_type = s["p_type"]
            for key in ("eta_profile", "p_profile"):
                v = s.get(key)
                if v is not None:
                    v = np.ascontiguousarray(v, dtype=np.float64).ravel()
                    self._keep.append(v)
                    setattr(arr[i], key, _ptr(v))
                else:
                    setattr(arr[i], key, C.POINTER(C.c_double)())
        self._h = lib.orc_create(C.byref(p), arr)
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self._keep = []

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_sources(self, fbody=None, src=None):
        fb = None if fbody is None else np.ascontiguousarray(fbody, dtype=np.float64)
        sr = None if src is None else np.ascontiguousarray(src, dtype=np.float64)
        null = C.POINTER(C.c_double)()
        self._lib.orc_set_sources(self._h, _ptr(fb) if fb is not None else null,
                                  _ptr(sr) if sr is not None else null)

    def step(self, n: int = 1) -> int:
        return self._lib.orc_step(self._h, n)

    def solve_to(self, T: float) -> int:
        return self._lib.orc_solve_to(self._h, T)

    def read_u(self):
        out = np.zeros((2, self.ny, self.nx))
        t = C.c_double()
        self._lib.orc_read_u(self._h, _ptr(out), C.byref(t))
        return out, t.value

    def read_p(self):
        out = np.zeros((self.ny, self.nx))
        t = C.c_double()
        self._lib.orc_read_p(self._h, _ptr(out), C.byref(t))
        return out, t.value

    def read_stress(self):
        out = np.zeros((3, self.ny, self.nx))
        self._lib.orc_read_stress(self._h, _ptr(out))
        return out

    def stats(self) -> dict:
        s = _Stats()
        self._lib.orc_stats_get(self._h, C.byref(s))
        return {name: getattr(s, name) for name, _ in _Stats._fields_}

    # ---- component access for the pins -------------------------------------------
    def prepare_elastic(self):
        self._lib.orc_prepare_elastic(self._h)

    def fixed_point_map(self, g: np.ndarray) -> np.ndarray:
        g = np.ascontiguousarray(g, dtype=np.float64)
        out = np.zeros_like(g)
        self._lib.orc_fixed_point_map(self._h, _ptr(g), _ptr(out))
        return out

    def vcycle(self, reset_history: bool = False) -> float:
        return self._lib.orc_vcycle(self._h, int(reset_history))

    def plain_pseudo_step(self):
        self._lib.orc_plain_pseudo_step(self._h)

    def get_g(self) -> np.ndarray:
        out = np.zeros((self.ny, self.nx, 8))
        self._lib.orc_get_g(self._h, _ptr(out))
        return out

    def set_g(self, g: np.ndarray):
        g = np.ascontiguousarray(g, dtype=np.float64)
        self._lib.orc_set_g(self._h, _ptr(g))

    def get_f(self) -> np.ndarray:
        out = np.zeros((self.ny, self.nx, 9))
        self._lib.orc_get_f(self._h, _ptr(out))
        return out

    def set_f(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        self._lib.orc_set_f(self._h, _ptr(f))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
