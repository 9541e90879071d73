"""ctypes binding of libfd.so: the names and arguments of include/fd.h, marshalling only.

Every computation happens in the CUDA library; this module only converts
Python values and torch tensors into the C ABI's plain pointers and sizes and
turns negative return codes into exceptions.  There is no fallback: if
libfd.so is missing or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfd.so")

FD_OK = 0
FD_ERR_INVALID_ARG = -1
FD_ERR_UNSTABLE = -2
FD_ERR_WORKSPACE = -3
FD_ERR_CUDA = -4
FD_ERR_NONFINITE = -5
FD_ERR_TIMEOUT = -6
FD_ERR_STATE = -7
FD_ERR_UNSUPPORTED = -8

FD_BC_DIRICHLET0, FD_BC_NOFLUX = 0, 1
FD_MEM_FULL, FD_MEM_SHORT, FD_MEM_ADAPTIVE = 0, 1, 2
FD_ADAPT_PAPER, FD_ADAPT_PARTITION = 0, 1
FD_F64, FD_F32, FD_BF16, FD_F16 = 0, 1, 2, 3
FD_FLAG_KAHAN = 1
FD_FLAG_ALLOW_UNSTABLE = 2
FD_FLAG_KEEP_TAPE = 4
FD_FLAG_INJECT_STALL = 8
FD_FLAG_PLAIN_STATE = 16
FD_FLAG_STEP_UPDATES = 32
FD_FLAG_FMA_FAR = 64
FD_FLAG_CLOSED_LOOP = 128

# every function include/fd.h declares
EXPORTS = (
    "fd_weights", "fd_schedule", "fd_workspace_bytes", "fd_init", "fd_set_state", "fd_step",
    "fd_run", "fd_get_state", "fd_current_step", "fd_adjoint", "fd_get_status", "fd_destroy",
    "fd_get_error_info",
    "fd_get_geometry", "fd_batch_workspace_bytes", "fd_batch_init", "fd_batch_set_state",
    "fd_batch_run", "fd_batch_get_state", "fd_batch_get_status", "fd_batch_get_geometry",
    "fd_batch_destroy",
    "fd_run_batch", "fd_strerror", "fd_run_static", "fd_save_bytes", "fd_save", "fd_load",
    "fd_memory_terms",
)


class FdError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class FdProblem(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("gamma", ctypes.c_double), ("alpha", ctypes.c_double),
        ("dt", ctypes.c_double), ("dx", ctypes.c_double),
        ("bc", ctypes.c_int), ("react", ctypes.c_double * 4),
        ("mem_mode", ctypes.c_int), ("mem_L", ctypes.c_int), ("mem_a", ctypes.c_int),
        ("adaptive_rule", ctypes.c_int),
        ("state_dtype", ctypes.c_int), ("hist_dtype", ctypes.c_int), ("accum_dtype", ctypes.c_int),
        ("flags", ctypes.c_uint), ("max_steps", ctypes.c_int), ("ckpt_every", ctypes.c_int),
        ("timeout_ms", ctypes.c_int),
        ("tile_threads", ctypes.c_int), ("chunk_terms", ctypes.c_int), ("stage_rows", ctypes.c_int),
        ("stages", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("head_lags", ctypes.c_int),
        ("nz", ctypes.c_int), ("time_block", ctypes.c_int), ("mem_tau", ctypes.c_double),
    ]


class FdGeometry(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("tile_threads", "tile_points", "tiles", "chunk_terms",
                                            "stage_rows", "stages", "ctas_per_sm", "grid",
                                            "head_lags")] + [
        ("units_total", ctypes.c_int64), ("hist_rows_total", ctypes.c_int64),
        ("terms_total", ctypes.c_int64), ("stream_rows_total", ctypes.c_int64),
        ("time_block", ctypes.c_int), ("block_updates", ctypes.c_int),
        ("far_tensor_cores", ctypes.c_int), ("head_rows_total", ctypes.c_int64),
        ("smem_bytes", ctypes.c_int64)]


_lib = None


def lib():
    """Load libfd.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfd.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        P = ctypes.POINTER(FdProblem)
        sz = ctypes.POINTER(ctypes.c_size_t)
        sig = {
            "fd_weights": [ctypes.c_double, i64, dp, dp],
            "fd_schedule": [P, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), i64, ctypes.POINTER(i64)],
            "fd_workspace_bytes": [P, sz],
            "fd_init": [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
            "fd_set_state": [vp, vp],
            "fd_step": [vp, ctypes.c_int],
            "fd_run": [vp, ctypes.c_int, vp],
            "fd_get_state": [vp, vp],
            "fd_current_step": [vp],
            "fd_adjoint": [vp, vp, vp, dp, dp, dp],
            "fd_get_status": [vp],
            "fd_get_error_info": [vp, ctypes.POINTER(ctypes.c_int64)],
            "fd_destroy": [vp],
            "fd_get_geometry": [vp, ctypes.POINTER(FdGeometry)],
            "fd_batch_workspace_bytes": [P, ctypes.c_int, sz],
            "fd_batch_init": [P, ctypes.c_int, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
            "fd_batch_set_state": [vp, ctypes.c_int, vp],
            "fd_batch_run": [vp],
            "fd_batch_get_state": [vp, ctypes.c_int, vp],
            "fd_batch_get_status": [vp],
            "fd_batch_get_geometry": [vp, ctypes.c_int, ctypes.POINTER(FdGeometry)],
            "fd_batch_destroy": [vp],
            "fd_run_batch": [P, ctypes.c_int, ctypes.POINTER(vp), vp, ctypes.c_size_t, vp],
            "fd_strerror": [ctypes.c_int],
            "fd_run_static": [P, vp, ctypes.c_int, vp, vp],
            "fd_save_bytes": [vp, sz],
            "fd_save": [vp, vp, ctypes.c_size_t],
            "fd_load": [vp, vp, ctypes.c_size_t],
            "fd_memory_terms": [vp, ctypes.POINTER(ctypes.c_int64)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.fd_current_step.restype = ctypes.c_int64
        L.fd_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().fd_strerror(code).decode()
    except Exception:  # library missing: still format the code
        return "error"


def check(code: int, where: str) -> int:
    if code < 0:
        raise FdError(code, where)
    return code


# ---- thin wrappers with the C names -------------------------------------------------------

def fd_weights(gamma: float, n: int, with_derivative: bool = False):
    import numpy as np
    psi = np.empty(n)
    dpsi = np.empty(n) if with_derivative else None
    dp = ctypes.POINTER(ctypes.c_double)
    check(lib().fd_weights(gamma, n, psi.ctypes.data_as(dp),
                           dpsi.ctypes.data_as(dp) if dpsi is not None else None), "fd_weights")
    return (psi, dpsi) if with_derivative else psi


def fd_schedule(p: FdProblem, k: int):
    import numpy as np
    lags = np.empty(k + 1, dtype=np.int64)
    mult = np.empty(k + 1, dtype=np.int64)
    n = ctypes.c_int64(0)
    ip = ctypes.POINTER(ctypes.c_int64)
    check(lib().fd_schedule(ctypes.byref(p), k, lags.ctypes.data_as(ip), mult.ctypes.data_as(ip),
                            k + 1, ctypes.byref(n)), "fd_schedule")
    return lags[:n.value].copy(), mult[:n.value].copy()


def fd_workspace_bytes(p: FdProblem) -> int:
    b = ctypes.c_size_t(0)
    check(lib().fd_workspace_bytes(ctypes.byref(p), ctypes.byref(b)), "fd_workspace_bytes")
    return b.value


def fd_init(p: FdProblem, ws_ptr: int, ws_bytes: int, stream: int) -> int:
    h = ctypes.c_void_p(0)
    check(lib().fd_init(ctypes.byref(p), ws_ptr, ws_bytes, stream, ctypes.byref(h)), "fd_init")
    return h.value


def fd_set_state(h: int, ptr: int):
    check(lib().fd_set_state(h, ptr), "fd_set_state")


def fd_step(h: int, n: int):
    check(lib().fd_step(h, n), "fd_step")


def fd_run(h: int, n: int, out_ptr: int | None):
    check(lib().fd_run(h, n, out_ptr), "fd_run")


def fd_get_state(h: int, out_ptr: int):
    check(lib().fd_get_state(h, out_ptr), "fd_get_state")


def fd_save_bytes(h: int) -> int:
    b = ctypes.c_size_t(0)
    check(lib().fd_save_bytes(h, ctypes.byref(b)), "fd_save_bytes")
    return b.value


def fd_save(h: int, buf_ptr: int, nbytes: int):
    check(lib().fd_save(h, buf_ptr, nbytes), "fd_save")


def fd_load(h: int, buf_ptr: int, nbytes: int):
    check(lib().fd_load(h, buf_ptr, nbytes), "fd_load")


def fd_current_step(h: int) -> int:
    return int(lib().fd_current_step(h))


def fd_get_status(h: int) -> int:
    return int(lib().fd_get_status(h))


def fd_memory_terms(h: int) -> int:
    """Memory terms used by the steps run so far, lag 0 included (closed loop: counted on the
    device)."""
    n = ctypes.c_int64(0)
    check(lib().fd_memory_terms(h, ctypes.byref(n)), "fd_memory_terms")
    return int(n.value)


ERROR_SITES = {0: "none", 1: "blocked far unit: history rows", 2: "blocked far unit: bulk copy",
               3: "blocked update: far count", 4: "blocked update: own rows",
               5: "blocked update: halo tile", 6: "chunk: history rows", 7: "chunk: bulk copy",
               8: "fixup: halo tile", 9: "injected stall", 10: "blocked far unit: running sum",
               11: "tensor-core far unit: copy, coefficients or MMAs",
               12: "blocked near unit: previous block's rows", 13: "blocked mid unit: the block's earlier rows",
               14: "closed-loop chunk: its step's decisions"}


def fd_get_error_info(h: int) -> dict:
    """Where a device wait gave up: site name and its eight raw words."""
    v = (ctypes.c_int64 * 8)()
    check(lib().fd_get_error_info(h, v), "fd_get_error_info")
    words = [int(x) for x in v]
    return {"site": ERROR_SITES.get(words[0], str(words[0])), "words": words}


def fd_adjoint(h: int, dj_duk_ptr: int, dj_du0_ptr: int | None):
    g, a = ctypes.c_double(0), ctypes.c_double(0)
    r = (ctypes.c_double * 4)()
    check(lib().fd_adjoint(h, dj_duk_ptr, dj_du0_ptr, ctypes.byref(g), ctypes.byref(a), r), "fd_adjoint")
    return g.value, a.value, [r[i] for i in range(4)]


def fd_get_geometry(h: int) -> dict:
    g = FdGeometry()
    check(lib().fd_get_geometry(h, ctypes.byref(g)), "fd_get_geometry")
    return {n: getattr(g, n) for n, _ in FdGeometry._fields_}


def fd_destroy(h: int):
    lib().fd_destroy(h)


def fd_batch_workspace_bytes(probs) -> int:
    arr = (FdProblem * len(probs))(*probs)
    b = ctypes.c_size_t(0)
    check(lib().fd_batch_workspace_bytes(arr, len(probs), ctypes.byref(b)), "fd_batch_workspace_bytes")
    return b.value


def fd_batch_init(probs, ws_ptr: int, ws_bytes: int, stream: int) -> int:
    arr = (FdProblem * len(probs))(*probs)
    h = ctypes.c_void_p(0)
    check(lib().fd_batch_init(arr, len(probs), ws_ptr, ws_bytes, stream, ctypes.byref(h)),
          "fd_batch_init")
    return h.value


def fd_batch_set_state(b: int, i: int, ptr: int):
    check(lib().fd_batch_set_state(b, i, ptr), "fd_batch_set_state")


def fd_batch_run(b: int):
    check(lib().fd_batch_run(b), "fd_batch_run")


def fd_batch_get_state(b: int, i: int, ptr: int):
    check(lib().fd_batch_get_state(b, i, ptr), "fd_batch_get_state")


def fd_batch_get_status(b: int) -> int:
    return int(lib().fd_batch_get_status(b))


def fd_batch_get_geometry(b: int, i: int) -> dict:
    g = FdGeometry()
    check(lib().fd_batch_get_geometry(b, i, ctypes.byref(g)), "fd_batch_get_geometry")
    return {n: getattr(g, n) for n, _ in FdGeometry._fields_}


def fd_batch_destroy(b: int):
    lib().fd_batch_destroy(b)


def fd_run_batch(probs, ptrs, ws_ptr: int, ws_bytes: int, stream: int):
    arr = (FdProblem * len(probs))(*probs)
    parr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    check(lib().fd_run_batch(arr, len(probs), parr, ws_ptr, ws_bytes, stream), "fd_run_batch")


def fd_strerror(code: int) -> str:
    return strerror(code)


def fd_run_static(p: FdProblem, u0_ptr: int, nsteps: int, out_ptr: int, stream: int):
    """Allocation-free forward run (scratch in the library's static device array)."""
    check(lib().fd_run_static(ctypes.byref(p), u0_ptr, nsteps, out_ptr, stream), "fd_run_static")
