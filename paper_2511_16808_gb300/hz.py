"""Python binding of the libhz C ABI (include/hz.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Device arrays are
torch CUDA tensors (contiguous); host arrays are numpy arrays or CPU tensors.
Complex fields are complex128 (c128) or complex64 (c64) tensors.  No compute
happens here: a missing or unloadable libhz.so raises at import time.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("HZ_LIB", os.path.join(_PKG, "_build", "libhz.so"))
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "hz.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhz.so not found at {LIB_PATH}: build it with "
                      f"`python -m paper_2511_16808_gb300.build` (there is no CPU fallback)")
lib = C.CDLL(LIB_PATH)

MAX_LEVELS = 10
MAX_STENCIL = 343
NOALLOC_MAX_NODES = 262144

PATCH = {"jacobi": 0, "element": 1, "plus": 2, "rb": 3, "full": 4}
INTERGRID = {"linear": 0, "cubic": 1, "mixed": 2, "leveldep": 3}
PRECISION = {"fp64": 0, "mixed": 1}
STATUS = {0: "HZ_OK", 1: "HZ_ERR_INVALID_ARG", 2: "HZ_ERR_OOM", 3: "HZ_ERR_CUDA",
          4: "HZ_ERR_NOT_CONVERGED", 5: "HZ_ERR_BREAKDOWN", 6: "HZ_ERR_TIMEOUT",
          7: "HZ_ERR_BUSY", 8: "HZ_ERR_NO_DEVICE"}
HZ_OK, HZ_ERR_NOT_CONVERGED, HZ_ERR_TIMEOUT = 0, 4, 6


class hz_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double)]


class hz_opts(C.Structure):
    _fields_ = [("levels", C.c_int), ("patch", C.c_int * MAX_LEVELS),
                ("damping", C.c_double * MAX_LEVELS), ("nu1", C.c_int), ("nu2", C.c_int),
                ("intergrid", C.c_int), ("precision", C.c_int), ("restart_m", C.c_int),
                ("tol", C.c_double), ("max_iter", C.c_int), ("nrhs_max", C.c_int),
                ("cycle_visits", C.c_int), ("stencil", C.c_int)]


class hz_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("relres_est", C.c_double),
                ("relres_true", C.c_double)]


class hz_level_desc(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("nodes", C.c_int64), ("stencil_size", C.c_int),
                ("stencil_off", (C.c_int * 3) * MAX_STENCIL), ("smoother_size", C.c_int),
                ("smoother_off", (C.c_int * 3) * MAX_STENCIL), ("patch", C.c_int),
                ("damping", C.c_double), ("is_coarsest", C.c_int)]


class hz_server_opts(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_active", C.c_int), ("device", C.c_int),
                ("setup_threads", C.c_int), ("group_max", C.c_int)]


class hz_request(C.Structure):
    _fields_ = [("grid", hz_grid), ("kappa", C.c_void_p), ("gamma", C.c_void_p), ("gamma0", C.c_double),
                ("omega", C.c_double), ("shift_alpha", C.c_double), ("opts", hz_opts),
                ("q", C.c_void_p), ("p", C.c_void_p)]


REQ_STATE = {0: "queued", 1: "setup", 2: "solving", 3: "done", 4: "failed"}


class hz_ticket_info(C.Structure):
    _fields_ = [("state", C.c_int), ("status", C.c_int), ("info", hz_info), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("bytes", C.c_size_t), ("message", C.c_char * 128), ("group_size", C.c_int)]


class hz_server_counters(C.Structure):
    _fields_ = [("queued", C.c_int), ("setting_up", C.c_int), ("solving", C.c_int), ("done", C.c_int),
                ("failed", C.c_int), ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t),
                ("budget", C.c_size_t), ("max_active", C.c_int), ("elapsed_s", C.c_double),
                ("kernel_launches", C.c_int64), ("groups", C.c_int), ("grouped", C.c_int)]


class hz_tune_entry(C.Structure):
    _fields_ = [("kind", C.c_int), ("level", C.c_int), ("nrhs", C.c_int), ("candidate", C.c_int),
                ("us", C.c_double), ("chosen", C.c_int)]


class HzError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.hz_last_error().decode()
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")


_P = C.c_void_p
_SIGS = {
    "hz_abi_version": ([], C.c_int),
    "hz_status_string": ([C.c_int], C.c_char_p),
    "hz_last_error": ([], C.c_char_p),
    "hz_opts_default": ([C.c_int, C.POINTER(hz_opts)], C.c_int),
    "hz_default_damping": ([C.c_int, C.c_int, C.c_int], C.c_double),
    "hz_setup_bytes": ([C.POINTER(hz_grid), C.POINTER(hz_opts), C.POINTER(C.c_size_t)], C.c_int),
    "hz_setup": ([C.POINTER(hz_grid), _P, C.c_double, _P, C.c_double, C.c_double,
                  C.POINTER(hz_opts), _P, C.POINTER(_P)], C.c_int),
    "hz_destroy": ([_P], C.c_int),
    "hz_solve": ([_P, _P, _P, C.c_int, C.POINTER(hz_info), _P], C.c_int),
    "hz_precond_apply": ([_P, _P, _P, C.c_int, _P], C.c_int),
    "hz_apply_operator": ([_P, _P, _P, C.c_int, C.c_int, _P], C.c_int),
    "hz_kernel_launches": ([_P, C.POINTER(C.c_int64)], C.c_int),
    "hz_profile_select": ([_P, C.c_int], C.c_int),
    "hz_profile_read": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                         C.POINTER(C.c_double)], C.c_int),
    "hz_measure_peak": ([C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "hz_check_status": ([C.POINTER(C.c_int), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.c_int], C.c_int),
    "hz_check_wait_timeout": ([C.c_longlong, C.c_int, C.POINTER(C.c_int)], C.c_int),
    "hz_memory_stats": ([C.c_int, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], C.c_int),
    "hz_context_info": ([_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "hz_level_count": ([_P, C.POINTER(C.c_int)], C.c_int),
    "hz_level_describe": ([_P, C.c_int, C.POINTER(hz_level_desc)], C.c_int),
    "hz_level_export": ([_P, C.c_int, C.c_int, _P], C.c_int),
    "hz_level_residual": ([_P, C.c_int, _P, _P, _P, _P], C.c_int),
    "hz_level_smooth": ([_P, C.c_int, _P, _P, _P], C.c_int),
    "hz_level_smooth_noalloc": ([_P, C.c_int, _P, _P, _P], C.c_int),
    "hz_level_restrict": ([_P, C.c_int, _P, _P, _P], C.c_int),
    "hz_level_prolong_add": ([_P, C.c_int, _P, _P, _P], C.c_int),
    "hz_coarse_solve": ([_P, _P, _P, _P], C.c_int),
    "hz_autotune": ([_P, C.c_int, C.c_int, C.POINTER(hz_tune_entry), C.c_int, C.POINTER(C.c_int)], C.c_int),
    "hz_tune_set": ([_P, C.c_int, C.c_int, C.c_int, C.c_int], C.c_int),
    "hz_coarse_solve_batch": ([_P, _P, _P, C.c_int, C.c_int, _P], C.c_int),
    "hz_setup_seconds": ([_P, C.POINTER(C.c_double)], C.c_int),
    "hz_solve_history": ([_P, C.c_int, _P, _P, _P, C.POINTER(C.c_int)], C.c_int),
    "hz_cycle_factor": ([_P, _P, _P, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double),
                         C.POINTER(C.c_int), _P], C.c_int),
    "hz_lfa_factors": ([C.c_int, _P, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                        _P, _P], C.c_int),
    "hz_solve_begin": ([_P, _P, _P], C.c_int),
    "hz_solve_step": ([_P, C.c_int, C.POINTER(C.c_int)], C.c_int),
    "hz_solve_end": ([_P, _P, C.POINTER(hz_info), _P], C.c_int),
    "hz_server_create": ([C.POINTER(hz_server_opts), C.POINTER(_P)], C.c_int),
    "hz_server_submit": ([_P, C.POINTER(hz_request), C.POINTER(C.c_uint64)], C.c_int),
    "hz_server_poll": ([_P, C.c_uint64, C.POINTER(hz_ticket_info)], C.c_int),
    "hz_server_wait": ([_P, C.c_uint64, C.c_double, C.POINTER(hz_ticket_info)], C.c_int),
    "hz_server_stats": ([_P, C.POINTER(hz_server_counters)], C.c_int),
    "hz_server_destroy": ([_P], C.c_int),
    "hz_sched_create": ([C.c_size_t, C.c_int, C.POINTER(_P)], C.c_int),
    "hz_sched_offer": ([_P, C.c_uint64, C.c_size_t, C.POINTER(C.c_int)], C.c_int),
    "hz_sched_next": ([_P, C.POINTER(C.c_uint64), C.POINTER(C.c_int)], C.c_int),
    "hz_sched_release": ([_P, C.c_size_t], C.c_int),
    "hz_sched_state": ([_P, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), C.POINTER(C.c_int),
                        C.POINTER(C.c_int)], C.c_int),
    "hz_sched_destroy": ([_P], C.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def declared_symbols(header: str = HEADER_PATH):
    """Names of the functions declared in include/hz.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hz_[a-z0-9_]+)\s*\(", text)))


def _check(status: int, where: str, ok=(HZ_OK,)):
    if status not in ok:
        raise HzError(status, where)
    return status


def _ptr(a):
    """Raw address of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # noqa: BLE001
            pass
        return None
    return getattr(s, "cuda_stream", s)


# ------------------------------------------------------------------ library

def hz_abi_version() -> int:
    return lib.hz_abi_version()


def hz_check_wait_timeout(polls: int, arrive: bool):
    """(status, timed_out) of one bounded device wait (see hz.h)."""
    t = C.c_int()
    st = lib.hz_check_wait_timeout(int(polls), int(bool(arrive)), C.byref(t))
    _check(st, "hz_check_wait_timeout", ok=(HZ_OK, HZ_ERR_TIMEOUT))
    return st, bool(t.value)


def hz_check_status(clear: bool = False) -> dict:
    """Checked-index build: {'enabled', 'failures', 'line', 'index'} of the
    out-of-extent accesses since the last clear (line and index of the first)."""
    en, fails, first = C.c_int(), C.c_uint64(), C.c_uint64()
    _check(lib.hz_check_status(C.byref(en), C.byref(fails), C.byref(first), int(bool(clear))), "hz_check_status")
    return {"enabled": bool(en.value), "failures": fails.value, "line": first.value >> 40,
            "index": first.value & ((1 << 40) - 1)}


def hz_status_string(s: int) -> str:
    return lib.hz_status_string(s).decode()


def hz_last_error() -> str:
    return lib.hz_last_error().decode()


def hz_opts_default(dim: int) -> hz_opts:
    o = hz_opts()
    _check(lib.hz_opts_default(dim, C.byref(o)), "hz_opts_default")
    return o


def hz_default_damping(dim: int, patch, level: int) -> float:
    return lib.hz_default_damping(dim, PATCH.get(patch, patch), level)


def make_grid(dim: int, n, h: float) -> hz_grid:
    g = hz_grid()
    g.dim = dim
    n = list(n) + [1] * (3 - len(n))
    for a in range(3):
        g.n[a] = int(n[a])
    g.h = float(h)
    return g


def hz_setup_bytes(grid: hz_grid, opts: hz_opts) -> int:
    out = C.c_size_t()
    _check(lib.hz_setup_bytes(C.byref(grid), C.byref(opts), C.byref(out)), "hz_setup_bytes")
    return out.value


def hz_setup(grid: hz_grid, kappa, omega: float, gamma, gamma0: float, shift_alpha: float,
             opts: hz_opts, stream=None):
    """Returns an opaque context handle (int)."""
    ctx = C.c_void_p()
    _check(lib.hz_setup(C.byref(grid), _ptr(kappa), float(omega), _ptr(gamma), float(gamma0),
                        float(shift_alpha), C.byref(opts), _stream(stream), C.byref(ctx)), "hz_setup")
    return ctx.value


def hz_destroy(ctx) -> None:
    _check(lib.hz_destroy(ctx), "hz_destroy")


def hz_solve(ctx, q, p, nrhs: int = 1, stream=None):
    """Returns (converged: bool, [hz_info] * nrhs)."""
    infos = (hz_info * nrhs)()
    st = lib.hz_solve(ctx, _ptr(q), _ptr(p), nrhs, infos, _stream(stream))
    _check(st, "hz_solve", ok=(HZ_OK, HZ_ERR_NOT_CONVERGED))
    return st == HZ_OK, list(infos)


def hz_solve_begin(ctx, q, stream=None) -> None:
    _check(lib.hz_solve_begin(ctx, _ptr(q), _stream(stream)), "hz_solve_begin")


def hz_solve_step(ctx, block: bool = False) -> bool:
    """True once the asynchronous solve has finished."""
    done = C.c_int()
    _check(lib.hz_solve_step(ctx, int(bool(block)), C.byref(done)), "hz_solve_step")
    return bool(done.value)


def hz_solve_end(ctx, p, stream=None):
    """Returns (converged: bool, hz_info)."""
    info = hz_info()
    st = lib.hz_solve_end(ctx, _ptr(p), C.byref(info), _stream(stream))
    _check(st, "hz_solve_end", ok=(HZ_OK, HZ_ERR_NOT_CONVERGED))
    return st == HZ_OK, info


def hz_precond_apply(ctx, r, z, nrhs: int = 1, stream=None) -> None:
    _check(lib.hz_precond_apply(ctx, _ptr(r), _ptr(z), nrhs, _stream(stream)), "hz_precond_apply")


def hz_apply_operator(ctx, v, w, nrhs: int = 1, shifted: int = 0, stream=None) -> None:
    _check(lib.hz_apply_operator(ctx, _ptr(v), _ptr(w), nrhs, int(shifted), _stream(stream)),
           "hz_apply_operator")


def hz_kernel_launches(ctx) -> int:
    out = C.c_int64()
    _check(lib.hz_kernel_launches(ctx, C.byref(out)), "hz_kernel_launches")
    return out.value


def hz_measure_peak(kind: str = "fp64"):
    """(TFLOP/s, ms of the best launch) of the device's FP64 (kind 'fp64') or
    FP32 ('fp32') fused multiply-add pipe, measured by a chain kernel."""
    t, ms = C.c_double(), C.c_double()
    _check(lib.hz_measure_peak({"fp64": 0, "fp32": 1}.get(kind, kind), C.byref(t), C.byref(ms)), "hz_measure_peak")
    return t.value, ms.value


# 1: Gram-Schmidt update pass(es); 2: the pass with the FP64 operator and the
# inner products; 3: the whole V-cycle
PROFILE = {"none": 0, "gs_update": 1, "gs_apply": 2, "vcycle": 3}


def hz_profile_select(ctx, kernel_class) -> None:
    _check(lib.hz_profile_select(ctx, PROFILE.get(kernel_class, kernel_class)), "hz_profile_select")


def hz_profile_read(ctx) -> dict:
    ms, n, b, f = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
    _check(lib.hz_profile_read(ctx, C.byref(ms), C.byref(n), C.byref(b), C.byref(f)), "hz_profile_read")
    return {"ms": ms.value, "launches": n.value, "bytes": b.value, "flops": f.value}


# ------------------------------------------------------------------ components

def hz_level_count(ctx) -> int:
    out = C.c_int()
    _check(lib.hz_level_count(ctx, C.byref(out)), "hz_level_count")
    return out.value


def hz_level_describe(ctx, level: int) -> dict:
    d = hz_level_desc()
    _check(lib.hz_level_describe(ctx, level, C.byref(d)), "hz_level_describe")
    return {
        "n": tuple(d.n), "nodes": d.nodes,
        "stencil": [tuple(d.stencil_off[k]) for k in range(d.stencil_size)],
        "smoother": [tuple(d.smoother_off[k]) for k in range(d.smoother_size)],
        "patch": d.patch, "damping": d.damping, "is_coarsest": bool(d.is_coarsest),
    }


def hz_level_export(ctx, level: int, what: int) -> np.ndarray:
    """Stencil planes as a complex128 array [entries, nodes] (what 0: A_s, 1: Vanka sum)."""
    d = hz_level_describe(ctx, level)
    n = len(d["stencil"] if what == 0 else d["smoother"])
    out = np.zeros((n, d["nodes"]), dtype=np.complex128)
    _check(lib.hz_level_export(ctx, level, what, out.ctypes.data), "hz_level_export")
    return out


def hz_memory_stats(device: int = 0) -> dict:
    """{"pool_used_bytes", "device_allocations"}: bytes in use in the device's
    default stream-ordered pool and the library's device allocations so far."""
    used, n = C.c_uint64(), C.c_uint64()
    _check(lib.hz_memory_stats(device, C.byref(used), C.byref(n)), "hz_memory_stats")
    return {"pool_used_bytes": used.value, "device_allocations": n.value}


def hz_context_info(ctx) -> dict:
    """{"device", "precision" ('mixed' | 'fp64'), "nrhs_max"} of a context."""
    dev, prec, nr = C.c_int(), C.c_int(), C.c_int()
    _check(lib.hz_context_info(ctx, C.byref(dev), C.byref(prec), C.byref(nr)), "hz_context_info")
    return {"device": dev.value, "precision": {v: k for k, v in PRECISION.items()}[prec.value],
            "nrhs_max": nr.value}


def _level_fields(ctx, where, **fields):
    """Reject level fields the library would read or write out of bounds: each
    must be a contiguous CUDA tensor on the context's device, of the V-cycle
    element type (complex64 mixed / complex128 fp64) and exactly the node count
    of its level.  fields: name -> (tensor, level)."""
    info = hz_context_info(ctx)
    want = "torch.complex64" if info["precision"] == "mixed" else "torch.complex128"
    for name, (t, lv) in fields.items():
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise ValueError(f"{where}: {name} must be a CUDA tensor")
        if t.device.index != info["device"]:
            raise ValueError(f"{where}: {name} is on cuda:{t.device.index}, the context on cuda:{info['device']}")
        if str(t.dtype) != want:
            raise ValueError(f"{where}: {name} has dtype {t.dtype}, the context's V-cycle needs {want}")
        nodes = hz_level_describe(ctx, lv)["nodes"]
        if t.numel() != nodes:
            raise ValueError(f"{where}: {name} has {t.numel()} values, level {lv} has {nodes} nodes")
        if not t.is_contiguous():
            raise ValueError(f"{where}: {name} must be contiguous")


def hz_level_residual(ctx, level, u, f, r, stream=None):
    _level_fields(ctx, "hz_level_residual", u=(u, level), f=(f, level), r=(r, level))
    _check(lib.hz_level_residual(ctx, level, _ptr(u), _ptr(f), _ptr(r), _stream(stream)), "hz_level_residual")


def hz_level_smooth(ctx, level, u, f, stream=None):
    _level_fields(ctx, "hz_level_smooth", u=(u, level), f=(f, level))
    _check(lib.hz_level_smooth(ctx, level, _ptr(u), _ptr(f), _stream(stream)), "hz_level_smooth")


def hz_level_smooth_noalloc(ctx, level, u, f, stream=None):
    """hz_level_smooth without any device allocation (scratch in static device memory)."""
    _level_fields(ctx, "hz_level_smooth_noalloc", u=(u, level), f=(f, level))
    _check(lib.hz_level_smooth_noalloc(ctx, level, _ptr(u), _ptr(f), _stream(stream)),
           "hz_level_smooth_noalloc")


def hz_level_restrict(ctx, level, r, fc, stream=None):
    _level_fields(ctx, "hz_level_restrict", r=(r, level), fc=(fc, level + 1))
    _check(lib.hz_level_restrict(ctx, level, _ptr(r), _ptr(fc), _stream(stream)), "hz_level_restrict")


def hz_level_prolong_add(ctx, level, ec, u, stream=None):
    _level_fields(ctx, "hz_level_prolong_add", ec=(ec, level + 1), u=(u, level))
    _check(lib.hz_level_prolong_add(ctx, level, _ptr(ec), _ptr(u), _stream(stream)), "hz_level_prolong_add")


def hz_coarse_solve(ctx, f, u, stream=None):
    last = hz_level_count(ctx) - 1
    _level_fields(ctx, "hz_coarse_solve", f=(f, last), u=(u, last))
    _check(lib.hz_coarse_solve(ctx, _ptr(f), _ptr(u), _stream(stream)), "hz_coarse_solve")


def hz_coarse_solve_batch(ctx, f, u, nrhs, variant=-1, stream=None):
    """U = Ainv F on the coarsest level for nrhs right-hand sides (RHS
    innermost) with variant 0 (CUDA cores), s in 1..16 (tensor cores, K split s
    ways) or -1 (the context's choice)."""
    last = hz_level_count(ctx) - 1
    info = hz_context_info(ctx)
    want = "torch.complex64" if info["precision"] == "mixed" else "torch.complex128"
    nodes = hz_level_describe(ctx, last)["nodes"]
    for name, t in (("f", f), ("u", u)):
        if not (hasattr(t, "is_cuda") and t.is_cuda) or str(t.dtype) != want or t.numel() != nodes * nrhs:
            raise ValueError(f"hz_coarse_solve_batch: {name} must be a CUDA {want} tensor of {nodes * nrhs} values")
        if not t.is_contiguous():
            raise ValueError(f"hz_coarse_solve_batch: {name} must be contiguous")
    _check(lib.hz_coarse_solve_batch(ctx, _ptr(f), _ptr(u), nrhs, variant, _stream(stream)), "hz_coarse_solve_batch")


TUNE_KINDS = {0: "coarsest product", 1: "RHS pack", 2: "register budget", 3: "fused tile passes"}


def hz_autotune(ctx, nrhs: int = 1, reps: int = 10) -> list:
    """Times every candidate kernel choice for batch width nrhs and keeps the
    fastest on the context; returns one dict per candidate."""
    n = C.c_int()
    cap = 4 * MAX_LEVELS + 8                 # at most 3 knobs per level plus the coarsest's 5 candidates
    buf = (hz_tune_entry * (2 * cap))()
    _check(lib.hz_autotune(ctx, nrhs, reps, buf, 2 * cap, C.byref(n)), "hz_autotune")
    return [{"kind": e.kind, "knob": TUNE_KINDS.get(e.kind, e.kind), "level": e.level, "nrhs": e.nrhs,
             "candidate": e.candidate, "us": e.us, "chosen": bool(e.chosen)} for e in buf[: n.value]]


def hz_tune_set(ctx, kind: int, level: int, nrhs: int, candidate: int) -> None:
    _check(lib.hz_tune_set(ctx, kind, level, nrhs, candidate), "hz_tune_set")


def hz_setup_seconds(ctx) -> float:
    out = C.c_double()
    _check(lib.hz_setup_seconds(ctx, C.byref(out)), "hz_setup_seconds")
    return out.value


def hz_solve_history(ctx) -> dict:
    """{"iters", "relres_true", "relres_est"} lists of the last single-RHS solve."""
    n = C.c_int()
    _check(lib.hz_solve_history(ctx, 0, None, None, None, C.byref(n)), "hz_solve_history")
    k = n.value
    its = np.zeros(k, dtype=np.int32)
    rt = np.zeros(k)
    re = np.zeros(k)
    if k:
        _check(lib.hz_solve_history(ctx, k, its.ctypes.data, rt.ctypes.data, re.ctypes.data, C.byref(n)),
               "hz_solve_history")
    return {"iters": its.tolist(), "relres_true": rt.tolist(), "relres_est": re.tolist()}


def hz_cycle_factor(ctx, f, u, warmup: int = 5, target: float = 1e-9, max_iter: int = 300, stream=None):
    """(factor, iterations) of Eq. cf; u (device complex128) is updated in place."""
    fac, its = C.c_double(), C.c_int()
    _check(lib.hz_cycle_factor(ctx, _ptr(f), _ptr(u), int(warmup), float(target), int(max_iter),
                               C.byref(fac), C.byref(its), _stream(stream)), "hz_cycle_factor")
    return fac.value, its.value


def hz_lfa_factors(dim: int, stencil, patch: str, w, rk: str = "cubic", pk: str = "cubic", nu1: int = 1,
                   nu2: int = 1, samples: int = 128, want_mu: bool = True, want_rho: bool = True):
    """(mu_loc[w], rho_loc[w]) for a constant stencil given as 3^dim complex
    values in (dz, dy, dx) order (or a dict {offset: value})."""
    if isinstance(stencil, dict):
        arr = np.zeros((3,) * dim, dtype=np.complex128)
        for off, v in stencil.items():
            arr[tuple(o + 1 for o in reversed(off))] = v
        stencil = arr
    st = np.ascontiguousarray(np.asarray(stencil, dtype=np.complex128).reshape(-1))
    if st.size != 3 ** dim:
        raise ValueError("stencil needs 3^dim values")
    ws = np.ascontiguousarray(np.atleast_1d(np.asarray(w, dtype=np.float64)))
    mu = np.zeros(ws.size) if want_mu else None
    rho = np.zeros(ws.size) if want_rho else None
    _check(lib.hz_lfa_factors(dim, st.ctypes.data, PATCH[patch], ws.ctypes.data, ws.size, INTERGRID[rk],
                              INTERGRID[pk], nu1, nu2, samples, _ptr(mu), _ptr(rho)), "hz_lfa_factors")
    return mu, rho


# ------------------------------------------------------------------ serving

def hz_server_create(hbm_budget: int = 0, max_active: int = 0, device: int = -1, setup_threads: int = 0,
                     group_max: int = 0):
    o = hz_server_opts(int(hbm_budget), int(max_active), int(device), int(setup_threads), int(group_max))
    out = C.c_void_p()
    _check(lib.hz_server_create(C.byref(o), C.byref(out)), "hz_server_create")
    return out.value


def hz_server_submit(srv, req: hz_request) -> int:
    t = C.c_uint64()
    _check(lib.hz_server_submit(srv, C.byref(req), C.byref(t)), "hz_server_submit")
    return t.value


def hz_server_poll(srv, ticket: int) -> hz_ticket_info:
    out = hz_ticket_info()
    _check(lib.hz_server_poll(srv, ticket, C.byref(out)), "hz_server_poll")
    return out


def hz_server_wait(srv, ticket: int, timeout_s: float = -1.0) -> hz_ticket_info:
    out = hz_ticket_info()
    _check(lib.hz_server_wait(srv, ticket, float(timeout_s), C.byref(out)), "hz_server_wait")
    return out


def hz_server_stats(srv) -> dict:
    c = hz_server_counters()
    _check(lib.hz_server_stats(srv, C.byref(c)), "hz_server_stats")
    return {k: getattr(c, k) for k, _ in hz_server_counters._fields_}


def hz_server_destroy(srv) -> None:
    _check(lib.hz_server_destroy(srv), "hz_server_destroy")


def hz_sched_create(budget: int, max_active: int):
    out = C.c_void_p()
    _check(lib.hz_sched_create(int(budget), int(max_active), C.byref(out)), "hz_sched_create")
    return out.value


def hz_sched_offer(s, ticket: int, nbytes: int) -> bool:
    ok = C.c_int()
    _check(lib.hz_sched_offer(s, ticket, int(nbytes), C.byref(ok)), "hz_sched_offer")
    return bool(ok.value)


def hz_sched_next(s):
    """The admitted ticket, or None when the head of the queue does not fit."""
    t, ok = C.c_uint64(), C.c_int()
    _check(lib.hz_sched_next(s, C.byref(t), C.byref(ok)), "hz_sched_next")
    return t.value if ok.value else None


def hz_sched_release(s, nbytes: int) -> None:
    _check(lib.hz_sched_release(s, int(nbytes)), "hz_sched_release")


def hz_sched_state(s) -> dict:
    iu, pk, act, q = C.c_size_t(), C.c_size_t(), C.c_int(), C.c_int()
    _check(lib.hz_sched_state(s, C.byref(iu), C.byref(pk), C.byref(act), C.byref(q)), "hz_sched_state")
    return {"in_use": iu.value, "peak": pk.value, "active": act.value, "queued": q.value}


def hz_sched_destroy(s) -> None:
    _check(lib.hz_sched_destroy(s), "hz_sched_destroy")
