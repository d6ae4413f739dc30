"""ctypes binding of libatfd (include/at.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Status codes other than AT_OK raise
``ATError`` carrying the code and ``at_last_error()``.  Device buffers are passed as torch tensors
(only their data pointers cross the boundary); the library borrows them.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

AT_OK = 0
AT_ERR_ARG, AT_ERR_SINGULAR, AT_ERR_INCONSISTENT, AT_ERR_CUDA = -1, -2, -3, -4
AT_ERR_TIMEOUT, AT_ERR_NONFINITE, AT_ERR_BOUNDS, AT_ERR_STATE = -5, -6, -7, -8
AT_SYNC, AT_ASYNC_STD, AT_AT, AT_AT_SPACE2, AT_AT_SPACE1 = 0, 1, 2, 3, 4

# every entry point include/at.h declares (checked by the CPU test of the boundary)
EXPORTS = (
    "at_coeffs", "at_stencil_taps", "at_solve_stencil", "at_delay", "at_ring_slots", "at_num_sides",
    "at_init", "at_step", "at_reset", "at_set_launch", "at_set_fusion", "at_sync", "at_state", "at_error_stats", "at_destroy", "at_last_error",
    "at_error_stats_noalloc",
    "at_adjoint_workspace", "at_adjoint_forward", "at_adjoint_backward",
    "at_ensemble_sizes", "at_ensemble_create", "at_ensemble_run", "at_ensemble_stats", "at_ensemble_destroy",
    "at_error_stats_ref",
)


class ATError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


class at_coeffs_t(C.Structure):
    _fields_ = [("deriv", C.c_int32), ("order", C.c_int32), ("L", C.c_int32), ("h", C.c_int32), ("T", C.c_int32),
                ("cd", C.c_double * 9), ("cd_num", C.c_int64 * 9), ("cd_den", C.c_int64),
                ("phi", C.c_double * 5), ("w", (C.c_double * 4) * 8), ("w_num", (C.c_int64 * 4) * 8),
                ("w_den", C.c_int64 * 8)]


class at_config_t(C.Structure):
    _fields_ = [("dim", C.c_int32), ("order", C.c_int32), ("L", C.c_int32), ("scheme", C.c_int32),
                ("n", C.c_int64 * 3), ("pe", C.c_int32 * 3), ("nmodes", C.c_int32),
                ("c", C.c_double * 3), ("alpha", C.c_double), ("dt", C.c_double), ("seed", C.c_uint64),
                ("thresholds", C.POINTER(C.c_uint64)), ("amp", C.POINTER(C.c_double)),
                ("phase", C.POINTER(C.c_double)), ("kappa", C.POINTER(C.c_int32)), ("tsteps", C.c_int32),
                ("burgers", C.c_int32)]


class at_member_t(C.Structure):
    _fields_ = [("nsteps", C.c_int64), ("group", C.c_int32), ("twin", C.c_int32)]


class at_group_stats_t(C.Structure):
    _fields_ = [("key", C.c_int64), ("count", C.c_int32), ("ntwin", C.c_int32), ("rms_mean", C.c_double),
                ("rms_var", C.c_double), ("abs_mean", C.c_double), ("diff_mean", C.c_double),
                ("diff_var", C.c_double), ("dabs_mean", C.c_double), ("dabs_var", C.c_double)]


class at_stats_t(C.Structure):
    _fields_ = [("rms", C.c_double), ("max_abs", C.c_double), ("mean_abs", C.c_double), ("mean", C.c_double),
                ("rms_I", C.c_double), ("rms_B", C.c_double), ("ua_rms", C.c_double),
                ("n_I", C.c_int64), ("n_B", C.c_int64), ("step", C.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libatfd.so.  There is no fallback: a missing or stale library is built, or this raises."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libatfd.so not found at {path}; run __graft_entry__.build()")
    L = C.CDLL(path)
    i32, i64, u64, vp, dp = C.c_int32, C.c_int64, C.c_uint64, C.c_void_p, C.POINTER(C.c_double)
    L.at_coeffs.argtypes = [i32, i32, i32, C.POINTER(at_coeffs_t)]
    L.at_stencil_taps.argtypes = [i32, i32, i32, i32, i32, i32, i32, C.POINTER(i32), C.POINTER(i32), dp,
                                  C.POINTER(i32)]
    L.at_solve_stencil.argtypes = [i32, i32, i32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64),
                                   C.POINTER(i64), dp, C.POINTER(i32)]
    L.at_delay.argtypes = [u64, i64, i64, i32, C.POINTER(u64)]
    L.at_ring_slots.argtypes = [C.POINTER(at_config_t), C.POINTER(i32)]
    L.at_num_sides.argtypes = [C.POINTER(at_config_t), C.POINTER(i64)]
    L.at_init.argtypes = [C.POINTER(at_config_t), vp, i64, vp, i64, vp, C.POINTER(vp)]
    L.at_step.argtypes = [vp, i64]
    L.at_sync.argtypes = [vp]
    L.at_reset.argtypes = [vp, vp]
    L.at_set_launch.argtypes = [vp, i32, i32]
    L.at_set_fusion.argtypes = [vp, i32, C.POINTER(i32)]
    L.at_state.argtypes = [vp, C.POINTER(i64), C.POINTER(vp)]
    L.at_error_stats.argtypes = [vp, C.POINTER(at_stats_t)]
    L.at_error_stats_ref.argtypes = [vp, vp, i32, C.POINTER(at_stats_t)]
    L.at_destroy.argtypes = [vp]
    L.at_last_error.restype = C.c_char_p
    L.at_error_stats_noalloc.argtypes = [C.POINTER(at_config_t), vp, i64, vp, C.POINTER(at_stats_t)]
    L.at_adjoint_workspace.argtypes = [vp, i64, i64, C.POINTER(i64)]
    L.at_adjoint_forward.argtypes = [vp, i64, i64, vp, i64]
    L.at_adjoint_backward.argtypes = [vp, vp, vp, C.POINTER(C.c_double)]
    L.at_ensemble_sizes.argtypes = [C.POINTER(at_config_t), C.POINTER(at_member_t), i32, C.POINTER(i64),
                                    C.POINTER(i64)]
    L.at_ensemble_create.argtypes = [C.POINTER(at_config_t), C.POINTER(at_member_t), i32, vp, i64, vp, i64, i32,
                                     i32, vp, C.POINTER(vp)]
    L.at_ensemble_run.argtypes = [vp]
    L.at_ensemble_stats.argtypes = [vp, C.POINTER(at_stats_t), dp, i32, C.POINTER(at_group_stats_t), i32,
                                    C.POINTER(i32)]
    L.at_ensemble_destroy.argtypes = [vp]
    _lib = L
    return L


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise ATError(rc, where, load().at_last_error().decode())
    return rc


def at_last_error() -> str:
    return load().at_last_error().decode()


def at_coeffs(deriv: int, order: int, L: int) -> at_coeffs_t:
    out = at_coeffs_t()
    _check(load().at_coeffs(deriv, order, L, C.byref(out)), "at_coeffs")
    return out


def at_stencil_taps(deriv, order, scheme, k, pos, side, cap=32):
    j = (C.c_int32 * cap)()
    l = (C.c_int32 * cap)()
    c = (C.c_double * cap)()
    nt = C.c_int32()
    _check(load().at_stencil_taps(deriv, order, scheme, k, pos, side, cap, j, l, c, C.byref(nt)), "at_stencil_taps")
    return [(j[t], l[t], c[t]) for t in range(nt.value)]


def at_solve_stencil(deriv, order, r, js, ls):
    """Returns (status, [(num, den)], [c], rank); status is AT_OK, AT_ERR_SINGULAR or AT_ERR_INCONSISTENT."""
    n = len(js)
    J = (C.c_int32 * n)(*js)
    Lv = (C.c_int32 * n)(*ls)
    num = (C.c_int64 * n)()
    den = (C.c_int64 * n)()
    cc = (C.c_double * n)()
    rank = C.c_int32()
    rc = load().at_solve_stencil(deriv, order, r, n, J, Lv, num, den, cc, C.byref(rank))
    if rc not in (AT_OK, AT_ERR_SINGULAR, AT_ERR_INCONSISTENT):
        _check(rc, "at_solve_stencil")
    return rc, [(num[i], den[i]) for i in range(n)], [cc[i] for i in range(n)], rank.value


def at_delay(seed, step, side, L, thresholds=None) -> int:
    thr = None if thresholds is None else np.ascontiguousarray(thresholds, dtype=np.uint64)
    ptr = thr.ctypes.data_as(C.POINTER(C.c_uint64)) if thr is not None else C.POINTER(C.c_uint64)()
    return _check(load().at_delay(int(seed), int(step), int(side), int(L), ptr), "at_delay")


class Config:
    """An at_config_t and the host arrays its pointers refer to, built from a workload spec dict."""

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
        s = at_config_t()
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
        self.tsteps = max(1, s.tsteps)
        self.dim = dim
        self.shape = (int(n[2]), int(n[1]), int(n[0])) if dim == 3 else (int(n[0]),)
        self.ntot = int(n[0] * n[1] * n[2])


def at_ring_slots(cfg: Config) -> int:
    R = C.c_int32()
    _check(load().at_ring_slots(C.byref(cfg.s), C.byref(R)), "at_ring_slots")
    return R.value


def at_num_sides(cfg: Config) -> int:
    nb = C.c_int64()
    _check(load().at_num_sides(C.byref(cfg.s), C.byref(nb)), "at_num_sides")
    return nb.value


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


def at_init(cfg: Config, ring, log=None, log_steps: int = 0, stream=None):
    """ring, log: CUDA torch tensors (float64 [R*ntot], uint8 [log_steps*sides]).  Returns the handle."""
    h = C.c_void_p()
    _check(load().at_init(C.byref(cfg.s), C.c_void_p(ring.data_ptr()), ring.numel(),
                          C.c_void_p(log.data_ptr()) if log is not None else None, int(log_steps),
                          _stream_ptr(stream), C.byref(h)), "at_init")
    return h


def at_step(h, nsteps: int) -> None:
    _check(load().at_step(h, int(nsteps)), "at_step")


def at_reset(h, u0=None) -> None:
    """u0: CUDA float64 tensor with the initial field, or None for Eq. "IC"."""
    _check(load().at_reset(h, C.c_void_p(u0.data_ptr()) if u0 is not None else None), "at_reset")


def at_set_launch(h, threads: int, blocks_per_sm: int) -> None:
    _check(load().at_set_launch(h, int(threads), int(blocks_per_sm)), "at_set_launch")


def at_set_fusion(h, k: int) -> int:
    """Block length of at_step: the largest admissible K <= k (1 = single steps); returns the K in use."""
    used = C.c_int32()
    _check(load().at_set_fusion(h, int(k), C.byref(used)), "at_set_fusion")
    return used.value


def at_sync(h) -> None:
    _check(load().at_sync(h), "at_sync")


def at_state(h):
    step = C.c_int64()
    ptr = C.c_void_p()
    _check(load().at_state(h, C.byref(step), C.byref(ptr)), "at_state")
    return step.value, ptr.value


def at_error_stats(h) -> dict:
    st = at_stats_t()
    _check(load().at_error_stats(h, C.byref(st)), "at_error_stats")
    return st.as_dict()


def at_error_stats_ref(h, ref, refine: int) -> dict:
    """Statistics of U^n - V for a reference field V (CUDA float64 tensor) `refine` times finer on every axis."""
    st = at_stats_t()
    _check(load().at_error_stats_ref(h, C.c_void_p(ref.data_ptr()), int(refine), C.byref(st)), "at_error_stats_ref")
    return st.as_dict()


def at_destroy(h) -> None:
    _check(load().at_destroy(h), "at_destroy")


def _config_array(cfgs):
    arr = (at_config_t * len(cfgs))()
    for i, c in enumerate(cfgs):
        arr[i] = c.s
    return arr


def _runs_array(count: int, nsteps, groups=None, twins=None):
    """at_member_t[count] from a step count (int: every member, or one per member), optional group labels and
    optional twin indices (-1: none)."""
    steps = [int(nsteps)] * count if not hasattr(nsteps, "__len__") else [int(v) for v in nsteps]
    if len(steps) != count:
        raise ValueError("one step count per member")
    arr = (at_member_t * count)()
    for r in range(count):
        arr[r].nsteps = steps[r]
        arr[r].group = -1 if groups is None else int(groups[r])
        arr[r].twin = -1 if twins is None else int(twins[r])
    return arr


def at_ensemble_sizes(cfgs, nsteps, groups=None, twins=None):
    """(ring doubles, log bytes) the members need."""
    arr = _config_array(cfgs)
    runs = _runs_array(len(cfgs), nsteps, groups, twins)
    ring, log = C.c_int64(), C.c_int64()
    _check(load().at_ensemble_sizes(arr, runs, len(cfgs), C.byref(ring), C.byref(log)), "at_ensemble_sizes")
    return ring.value, log.value


def at_ensemble_create(cfgs, nsteps, ring, log=None, threads=0, ctas_per_sm=0, stream=None, groups=None,
                       twins=None):
    arr = _config_array(cfgs)
    runs = _runs_array(len(cfgs), nsteps, groups, twins)
    h = C.c_void_p()
    _check(load().at_ensemble_create(arr, runs, len(cfgs), C.c_void_p(ring.data_ptr()), ring.numel(),
                                     C.c_void_p(log.data_ptr()) if log is not None else None,
                                     log.numel() if log is not None else 0, int(threads), int(ctas_per_sm),
                                     _stream_ptr(stream), C.byref(h)), "at_ensemble_create")
    return h


def at_ensemble_run(h) -> None:
    _check(load().at_ensemble_run(h), "at_ensemble_run")


def at_ensemble_stats(h, count: int):
    """Returns (per-member stats dicts with the twin differences under "diff" (RMS) and "dabs" (mean absolute),
    groups: list of dicts with key, count, mean, var (of the RMS errors), abs_mean (of the mean absolute errors),
    ntwin, diff_mean, diff_var, dabs_mean, dabs_var)."""
    per = (at_stats_t * count)()
    diff = (C.c_double * (2 * count))()
    cap = max(count, 64)
    grp = (at_group_stats_t * cap)()
    ng = C.c_int32()
    _check(load().at_ensemble_stats(h, per, diff, count, grp, cap, C.byref(ng)), "at_ensemble_stats")
    groups = [{"key": grp[g].key, "count": grp[g].count, "mean": grp[g].rms_mean, "var": grp[g].rms_var,
               "abs_mean": grp[g].abs_mean, "ntwin": grp[g].ntwin, "diff_mean": grp[g].diff_mean,
               "diff_var": grp[g].diff_var, "dabs_mean": grp[g].dabs_mean, "dabs_var": grp[g].dabs_var}
              for g in range(ng.value)]
    members = []
    for r in range(count):
        d = per[r].as_dict()
        d["diff"], d["dabs"] = diff[2 * r], diff[2 * r + 1]
        members.append(d)
    return members, groups


def at_ensemble_destroy(h) -> None:
    _check(load().at_ensemble_destroy(h), "at_ensemble_destroy")


def at_adjoint_workspace(h, nsteps: int, ckpt_every: int = 0) -> int:
    n = C.c_int64()
    _check(load().at_adjoint_workspace(h, int(nsteps), int(ckpt_every), C.byref(n)), "at_adjoint_workspace")
    return n.value


def at_adjoint_forward(h, nsteps: int, ckpt_every: int, work) -> None:
    _check(load().at_adjoint_forward(h, int(nsteps), int(ckpt_every), C.c_void_p(work.data_ptr()), work.numel()),
           "at_adjoint_forward")


def at_adjoint_backward(h, lam, grad_u0, want_alpha: bool = True):
    """lam = dJ/dU^nsteps, grad_u0 receives dJ/dU^0 (CUDA float64 tensors); returns dJ/dalpha (None when not
    requested: the sweep then skips the recompute of the forward levels)."""
    ga = C.c_double()
    _check(load().at_adjoint_backward(h, C.c_void_p(lam.data_ptr()), C.c_void_p(grad_u0.data_ptr()),
                                      C.byref(ga) if want_alpha else None), "at_adjoint_backward")
    return ga.value if want_alpha else None


def at_error_stats_noalloc(cfg: Config, u, step: int, stream=None) -> dict:
    """Statistics of a device field u (CUDA float64 tensor of the problem cfg at `step`) without any allocation
    inside the library (static device scratch).  The C entry point takes no length, so the tensor is checked here:
    a CUDA, float64, contiguous tensor of at least n0*n1*n2 elements; the call runs with u's device current."""
    import torch
    ntot = int(cfg.s.n[0]) * int(cfg.s.n[1]) * int(cfg.s.n[2])
    if not (isinstance(u, torch.Tensor) and u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()
            and u.numel() >= ntot):
        raise ATError(AT_ERR_ARG, "at_error_stats_noalloc (binding)",
                      f"u must be a contiguous CUDA float64 tensor of at least {ntot} elements")
    st = at_stats_t()
    with torch.cuda.device(u.device):
        _check(load().at_error_stats_noalloc(C.byref(cfg.s), C.c_void_p(u.data_ptr()), int(step),
                                             _stream_ptr(stream), C.byref(st)), "at_error_stats_noalloc")
    return st.as_dict()
