"""FP64 CPU oracle for the asynchrony-tolerant finite-difference method (arXiv:1702.00496).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline and
reference legs are the only callers.  The product package never imports this module and the oracle
never imports the product.  The arithmetic lives in ``oracle.c`` (plain C, compiled with
``-ffp-contract=off``); this file compiles it and marshals arguments through ctypes.

Every function follows the paper passage named in ``oracle.c``.  Parity status of each part:
  - Philox4x32-10 delay words: pinned (generic round function checked against numpy's Philox4x64).
  - stencil taps: pinned (Taylor moment conditions of Eq. "cond", k=0 reduction, truncation terms).
  - synchronous run: pinned (exact discrete Fourier solution; convergence to Eq. "ana_sol").
  - asynchronous run: pinned statistically (order gates of Sec. 5.2) and by truncation terms.
  - adjoint: pinned (central finite differences, exact for the quadratic misfit; Richardson differences in alpha;
    Adams-Bashforth and Burgers' equation too).
  - error statistics: pinned (closed forms: constant offsets, boundary-only offsets, |I_I| from the PE geometry).
  - Adams-Bashforth runs: pinned (exact Fourier recurrence of the synchronous run; slopes -4 / -6 of Cases 4, 5).
  - rows expanded in space: pinned (exact Eq. "cond" rows, printed leading terms, slope -2 of Cases 2, 3).
  - Burgers' equation: pinned (Cole-Hopf solutions; slope -4 of Case 6 against a finer run).
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

SYNC, ASYNC_STD, AT = 0, 1, 2


class OrcCfg(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("order", C.c_int32), ("L", C.c_int32), ("scheme", C.c_int32),
        ("n", C.c_int64 * 3), ("pe", C.c_int32 * 3), ("nmodes", C.c_int32),
        ("c", C.c_double * 3), ("alpha", C.c_double), ("dt", C.c_double), ("seed", C.c_uint64),
        ("thresholds", C.POINTER(C.c_uint64)), ("amp", C.POINTER(C.c_double)),
        ("phase", C.POINTER(C.c_double)), ("kappa", C.POINTER(C.c_int32)), ("tsteps", C.c_int32), ("burgers", C.c_int32),
    ]


class OrcTap(C.Structure):
    _fields_ = [("j", C.c_int32), ("l", C.c_int32), ("c", C.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (with OpenMP when the compiler has it)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_OUT_DIR, exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("oracle build needs gcc")
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:-1] + ["-fopenmp", "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_delay_raw.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int, C.POINTER(C.c_uint64)]
        L.orc_delay_effective.argtypes = [C.c_int, C.c_int64, C.c_int]
        L.orc_time_width.argtypes = [C.c_int, C.c_int]
        L.orc_taps.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_int,
                               C.c_double, C.POINTER(OrcTap)]
        L.orc_num_sides.argtypes = [C.POINTER(OrcCfg)]
        L.orc_num_sides.restype = C.c_int64
        L.orc_check.argtypes = [C.POINTER(OrcCfg)]
        L.orc_initial.argtypes = [C.POINTER(OrcCfg), C.c_void_p]
        L.orc_analytic.argtypes = [C.POINTER(OrcCfg), C.c_double, C.c_void_p]
        L.orc_step.argtypes = [C.POINTER(OrcCfg), C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p]
        L.orc_run.argtypes = [C.POINTER(OrcCfg), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_error_stats.argtypes = [C.POINTER(OrcCfg), C.c_void_p, C.c_int64, C.c_void_p]
        L.orc_adjoint.argtypes = [C.POINTER(OrcCfg), C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_delay_log.argtypes = [C.POINTER(OrcCfg), C.c_int64, C.c_void_p]
        L.orc_run_samples.argtypes = [C.POINTER(OrcCfg), C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]
        _lib = L
    return _lib


class Config:
    """Owns the ctypes struct and the numpy arrays its pointers refer to."""

    def __init__(self, spec: dict):
        dim = int(spec["dim"])
        n = list(spec["n"]) + [1] * (3 - len(spec["n"]))
        pe = list(spec["pe"]) + [1] * (3 - len(spec["pe"]))
        c = list(spec.get("c", [0.0])) + [0.0] * (3 - len(spec.get("c", [0.0])))
        self.amp = np.ascontiguousarray(spec["amp"], dtype=np.float64).reshape(-1)
        self.phase = np.ascontiguousarray(spec["phase"], dtype=np.float64).reshape(-1)
        self.kappa = np.ascontiguousarray(spec["kappa"], dtype=np.int32).reshape(-1)
        thr = spec.get("thresholds")
        self.thr = None if thr is None else np.ascontiguousarray(thr, dtype=np.uint64)
        s = OrcCfg()
        s.dim, s.order, s.L, s.scheme = dim, int(spec["order"]), int(spec["L"]), int(spec["scheme"])
        s.n[:] = [int(v) for v in n]
        s.pe[:] = [int(v) for v in pe]
        s.nmodes = int(spec["nmodes"])
        s.c[:] = [float(v) for v in c]
        s.alpha, s.dt, s.seed = float(spec["alpha"]), float(spec["dt"]), int(spec["seed"])
        s.thresholds = (self.thr.ctypes.data_as(C.POINTER(C.c_uint64)) if self.thr is not None
                        else C.POINTER(C.c_uint64)())
        s.amp = self.amp.ctypes.data_as(C.POINTER(C.c_double))
        s.phase = self.phase.ctypes.data_as(C.POINTER(C.c_double))
        s.kappa = self.kappa.ctypes.data_as(C.POINTER(C.c_int32))
        s.tsteps = int(spec.get("tsteps", 1))
        s.burgers = int(spec.get("burgers", 0))
        self.s = s
        self.shape = (int(n[2]), int(n[1]), int(n[0])) if dim == 3 else (int(n[0]),)
        self.ntot = int(n[0] * n[1] * n[2])
        if lib().orc_check(C.byref(s)) != 0:
            raise ValueError(f"invalid oracle config {spec}")

    @property
    def num_sides(self) -> int:
        return int(lib().orc_num_sides(C.byref(self.s)))


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def delay_raw(seed, step, side, L, thresholds=None):
    thr = None if thresholds is None else np.ascontiguousarray(thresholds, dtype=np.uint64)
    ptr = thr.ctypes.data_as(C.POINTER(C.c_uint64)) if thr is not None else C.POINTER(C.c_uint64)()
    return int(lib().orc_delay_raw(int(seed), int(step), int(side), int(L), ptr))


def delay_effective(k, n, T):
    return int(lib().orc_delay_effective(int(k), int(n), int(T)))


def time_width(order, scheme):
    return int(lib().orc_time_width(int(order), int(scheme)))


def taps(order, scheme, deriv, pos, S, use_pe, kL, kR, dx):
    """List of (j, l, c) taps of one derivative at one point (see orc_taps)."""
    buf = (OrcTap * 32)()
    nt = lib().orc_taps(int(order), int(scheme), int(deriv), int(pos), int(S), int(use_pe), int(kL), int(kR),
                        float(dx), buf)
    return [(buf[t].j, buf[t].l, buf[t].c) for t in range(nt)]


def initial(cfg: Config) -> np.ndarray:
    u = np.empty(cfg.ntot, dtype=np.float64)
    lib().orc_initial(C.byref(cfg.s), u.ctypes.data)
    return u.reshape(cfg.shape)


def analytic(cfg: Config, t: float) -> np.ndarray:
    u = np.empty(cfg.ntot, dtype=np.float64)
    lib().orc_analytic(C.byref(cfg.s), float(t), u.ctypes.data)
    return u.reshape(cfg.shape)


def step(cfg: Config, levels, keff) -> np.ndarray:
    """One step from explicit levels (levels[m] = U^{n-m}) and effective side delays."""
    levs = [np.ascontiguousarray(v, dtype=np.float64).reshape(-1) for v in levels]
    arr = (C.c_void_p * len(levs))(*[v.ctypes.data for v in levs])
    k = np.ascontiguousarray(keff, dtype=np.int32)
    out = np.empty(cfg.ntot, dtype=np.float64)
    if lib().orc_step(C.byref(cfg.s), arr, k.ctypes.data, out.ctypes.data) != 0:
        raise ValueError("orc_step failed")
    return out.reshape(cfg.shape)


def _opt(u0):
    if u0 is None:
        return None, None
    a = np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
    return a, a.ctypes.data


def run(cfg: Config, nsteps: int, want_log: bool = True, want_history: bool = False, threads: int = 1, u0=None):
    """Returns (U^{nsteps}, raw delay log [nsteps, sides] uint8 or None, history or None)."""
    keep, p0 = _opt(u0)
    lib().orc_set_threads(int(threads))
    u = np.empty(cfg.ntot, dtype=np.float64)
    log = np.zeros((nsteps, cfg.num_sides), dtype=np.uint8) if want_log else None
    hist = np.empty((nsteps + 1, cfg.ntot), dtype=np.float64) if want_history else None
    rc = lib().orc_run(C.byref(cfg.s), p0, int(nsteps), u.ctypes.data,
                       log.ctypes.data if log is not None else None,
                       hist.ctypes.data if hist is not None else None)
    lib().orc_set_threads(1)
    if rc != 0:
        raise RuntimeError(f"orc_run failed ({rc})")
    return (u.reshape(cfg.shape), log,
            None if hist is None else hist.reshape((nsteps + 1,) + cfg.shape))


def run_samples(cfg: Config, nsteps: int, positions) -> np.ndarray:
    """U^{nsteps} of a 1D run from Eq. "IC" (forward Euler or Adams-Bashforth) at the given cells, each stepped only
    inside its domain of dependence (the same values as run(), bit for bit, at full sizes where a whole run would
    take too long)."""
    pos = np.ascontiguousarray(positions, dtype=np.int64)
    out = np.empty(pos.size, dtype=np.float64)
    rc = lib().orc_run_samples(C.byref(cfg.s), int(nsteps), int(pos.size), pos.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"orc_run_samples failed ({rc})")
    return out


def delay_log(cfg: Config, nsteps: int) -> np.ndarray:
    """Raw delays [nsteps, sides] uint8 of the run, without the field computation."""
    log = np.zeros((nsteps, cfg.num_sides), dtype=np.uint8)
    if lib().orc_delay_log(C.byref(cfg.s), int(nsteps), log.ctypes.data) != 0:
        raise RuntimeError("orc_delay_log failed")
    return log


STAT_NAMES = ("rms", "max_abs", "mean_abs", "mean", "rms_I", "rms_B", "ua_rms", "n_I", "n_B")


def error_stats(cfg: Config, u: np.ndarray, step_index: int) -> dict:
    out = np.zeros(9, dtype=np.float64)
    uu = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    if lib().orc_error_stats(C.byref(cfg.s), uu.ctypes.data, int(step_index), out.ctypes.data) != 0:
        raise RuntimeError("orc_error_stats failed")
    return dict(zip(STAT_NAMES, out.tolist()))


def adjoint(cfg: Config, nsteps: int, u_target: np.ndarray, u0=None):
    """Returns (J, dJ/dU^0, dJ/dalpha) for J = 1/2 ||U^{nsteps} - u_target||^2."""
    keep, p0 = _opt(u0)
    tgt = np.ascontiguousarray(u_target, dtype=np.float64).reshape(-1)
    g = np.empty(cfg.ntot, dtype=np.float64)
    ga = C.c_double()
    jj = C.c_double()
    if lib().orc_adjoint(C.byref(cfg.s), p0, int(nsteps), tgt.ctypes.data, g.ctypes.data, C.byref(ga), C.byref(jj)):
        raise RuntimeError("orc_adjoint failed")
    return jj.value, g.reshape(cfg.shape), ga.value
