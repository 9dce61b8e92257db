"""Python binding of libpdit (include/pdit.h): argument marshalling only.

Every step of the annealed p-dit sweep runs in the library's CUDA kernels.
PyTorch supplies device memory and streams for the device-buffer entry
point. If libpdit.so has not been built this module raises on import of the
library; there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import re

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpdit.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "pdit.h")

PDIT_OK = 0
PDIT_EINVAL = -1
PDIT_ERANGE = -2
PDIT_ENOMEM = -3
PDIT_ECUDA = -4
PDIT_EDEVICE = -5
PDIT_ENOTSUP = -6
PDIT_EIO = -7
PDIT_PLACE_AUTO = 0
PDIT_PLACE_SHARED = 1
PDIT_PLACE_GLOBAL = 2
PDIT_INFLUENCE_AUTO = 0
PDIT_INFLUENCE_TABLE = 1
PDIT_INFLUENCE_PRODUCTS = 2
PDIT_FORM_SYMMETRIC = 0
PDIT_FORM_GENERAL = 1
PDIT_FORM_FLOW_CLASSES = 2
PDIT_N_MAX = 256
PDIT_MODE_ANNEAL = 0
PDIT_MODE_PT = 1
PDIT_MODE_FIXED = 2
PDIT_MODE_CUPIM = 3
PDIT_FLAG_RESUME = 1
PDIT_STATUS_ENERGY_AUDIT = 1
PDIT_STATUS_SCHEDULE = 2
PDIT_BATCH_STOP_AT_TARGET = 1
PDIT_BATCH_GRAPH = 2

_lib = None


class PditError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = "%s failed: %s (%d)" % (what, strerror(code), code)
        if code == PDIT_ECUDA:
            msg += ": " + last_error()
        super().__init__(msg)
        self.code = code


class pdit_opts(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("replicas", ctypes.c_int),
        ("sweeps", ctypes.c_int),
        ("sweep_begin", ctypes.c_int),
        ("sweep_end", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("instance_id", ctypes.c_uint32),
        ("replica_base", ctypes.c_uint32),
        ("mode", ctypes.c_int),
        ("beta", ctypes.c_void_p),
        ("ladder_len", ctypes.c_int),
        ("exchange_period", ctypes.c_int),
        ("timeout_periods", ctypes.c_int),
        ("flags", ctypes.c_uint32),
        ("stream", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("best_perm", ctypes.c_void_p),
        ("best_cost", ctypes.c_void_p),
        ("replica_best_cost", ctypes.c_void_p),
        ("replica_best_perm", ctypes.c_void_p),
        ("replica_best_sweep", ctypes.c_void_p),
        ("replica_final_perm", ctypes.c_void_p),
        ("replica_final_cost", ctypes.c_void_p),
        ("replica_accepted", ctypes.c_void_p),
        ("replica_rung", ctypes.c_void_p),
        ("tables", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
        ("target", ctypes.c_void_p),
        ("reach_ns", ctypes.c_void_p),
        ("reach_sweep", ctypes.c_void_p),
        ("stop_at_target", ctypes.c_int),
    ]


class pdit_batch_item(ctypes.Structure):
    _fields_ = [
        ("qap", ctypes.c_void_p),
        ("replicas", ctypes.c_int),
        ("sweeps", ctypes.c_int),
        ("beta", ctypes.c_void_p),
        ("seed", ctypes.c_uint64),
        ("instance_id", ctypes.c_uint32),
        ("best_perm", ctypes.c_void_p),
        ("best_cost", ctypes.c_void_p),
        ("target", ctypes.c_void_p),
        ("reach_ns", ctypes.c_void_p),
        ("reach_sweep", ctypes.c_void_p),
    ]


def lib():
    """Load libpdit.so (built by paper_2605_24408_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libpdit.so is not built (run __graft_entry__.build()); "
                           "there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32p, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    L.qap_create.argtypes = [ctypes.c_int, vp, vp, ctypes.POINTER(vp)]
    L.qap_create.restype = ctypes.c_int
    L.qap_destroy.argtypes = [vp]
    L.qap_destroy.restype = None
    L.qap_n.argtypes = [vp]
    L.qap_n.restype = ctypes.c_int
    L.pdit_anneal.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_uint64, vp, vp]
    L.pdit_anneal.restype = ctypes.c_int
    L.pdit_opts_init.argtypes = [ctypes.POINTER(pdit_opts)]
    L.pdit_opts_init.restype = None
    L.pdit_workspace_bytes.argtypes = [vp, ctypes.POINTER(pdit_opts)]
    L.pdit_workspace_bytes.restype = ctypes.c_size_t
    L.pdit_anneal_ex.argtypes = [vp, ctypes.POINTER(pdit_opts)]
    L.pdit_anneal_ex.restype = ctypes.c_int
    L.pdit_beta_max.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.pdit_beta_max.restype = ctypes.c_int
    L.pdit_beta_schedule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, vp]
    L.pdit_beta_schedule.restype = ctypes.c_int
    L.pdit_set_warps_per_replica.argtypes = [vp, ctypes.c_int]
    L.pdit_set_warps_per_replica.restype = ctypes.c_int
    L.pdit_launch_shape.argtypes = [vp, ctypes.c_int, vp]
    L.pdit_launch_shape.restype = ctypes.c_int
    L.pdit_set_influence.argtypes = [vp, ctypes.c_int]
    L.pdit_set_influence.restype = ctypes.c_int
    L.pdit_set_pending_swaps.argtypes = [vp, ctypes.c_int]
    L.pdit_set_pending_swaps.restype = ctypes.c_int
    L.pdit_beta_range.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_uint64, vp, vp, vp]
    L.pdit_beta_range.restype = ctypes.c_int
    L.pdit_beta_ladder.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, vp]
    L.pdit_beta_ladder.restype = ctypes.c_int
    L.pdit_anneal_noalloc.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_uint64,
                                      vp, vp, vp, vp]
    L.pdit_anneal_noalloc.restype = ctypes.c_int
    L.pdit_autotune.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp]
    L.pdit_autotune.restype = ctypes.c_int
    L.pdit_probe_peaks.argtypes = [ctypes.c_int, vp]
    L.pdit_probe_peaks.restype = ctypes.c_int
    L.pdit_batch_create.argtypes = [ctypes.POINTER(pdit_batch_item), ctypes.c_int, ctypes.c_uint32,
                                    ctypes.POINTER(vp)]
    L.pdit_batch_create.restype = ctypes.c_int
    L.pdit_batch_run.argtypes = [vp, vp]
    L.pdit_batch_run.restype = ctypes.c_int
    L.pdit_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)]
    L.pdit_batch_info.restype = ctypes.c_int
    L.pdit_batch_destroy.argtypes = [vp]
    L.pdit_batch_destroy.restype = None
    L.pdit_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
    L.pdit_server_create.restype = ctypes.c_int
    L.pdit_server_submit.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                     ctypes.c_uint32, vp, ctypes.POINTER(ctypes.c_int64)]
    L.pdit_server_submit.restype = ctypes.c_int
    L.pdit_server_tick.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.pdit_server_tick.restype = ctypes.c_int
    L.pdit_server_result.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int), vp,
                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
    L.pdit_server_result.restype = ctypes.c_int
    L.pdit_server_destroy.argtypes = [vp]
    L.pdit_server_destroy.restype = None
    L.pdit_set_table_placement.argtypes = [vp, ctypes.c_int]
    L.pdit_set_table_placement.restype = ctypes.c_int
    L.pdit_set_replicas_per_cta.argtypes = [vp, ctypes.c_int]
    L.pdit_set_replicas_per_cta.restype = ctypes.c_int
    L.pdit_instance_form.argtypes = [vp]
    L.pdit_instance_form.restype = ctypes.c_int
    L.pdit_set_class_update.argtypes = [vp, ctypes.c_int]
    L.pdit_set_class_update.restype = ctypes.c_int
    L.pdit_read_qaplib.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), vp, vp, ctypes.c_size_t]
    L.pdit_read_qaplib.restype = ctypes.c_int
    L.pdit_read_qaplib_solution.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int64), vp, ctypes.c_int]
    L.pdit_read_qaplib_solution.restype = ctypes.c_int
    L.pdit_write_qaplib_solution.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_int64, vp]
    L.pdit_write_qaplib_solution.restype = ctypes.c_int
    L.pdit_strerror.argtypes = [ctypes.c_int]
    L.pdit_strerror.restype = ctypes.c_char_p
    L.pdit_last_error.argtypes = []
    L.pdit_last_error.restype = ctypes.c_char_p
    del i32p, i64p
    _lib = L
    return L


def header_functions(path: str = HEADER):
    """Names of the functions declared in include/pdit.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)) -
                  {"if", "sizeof", "for", "while", "return"})


def strerror(code: int) -> str:
    return lib().pdit_strerror(code).decode()


def last_error() -> str:
    return lib().pdit_last_error().decode()


def _check(rc: int, what: str):
    if rc != PDIT_OK:
        raise PditError(rc, what)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# --- handle ------------------------------------------------------------------

class Qap:
    """An uploaded instance (qap_create / qap_destroy)."""

    def __init__(self, D, F):
        D = np.ascontiguousarray(D, dtype=np.int32)
        F = np.ascontiguousarray(F, dtype=np.int32)
        if D.ndim != 2 or D.shape[0] != D.shape[1] or F.shape != D.shape:
            raise ValueError("D and F must be square and of the same shape")
        self.n = int(D.shape[0])
        h = ctypes.c_void_p()
        _check(lib().qap_create(self.n, _ptr(D), _ptr(F), ctypes.byref(h)), "qap_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().qap_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def qap_create_host_ptrs(n: int, D_ptr: int, F_ptr: int) -> Qap:
    """qap_create on raw host pointers (pinned buffers): n x n int32 each."""
    q = Qap.__new__(Qap)
    h = ctypes.c_void_p()
    _check(lib().qap_create(n, ctypes.c_void_p(D_ptr), ctypes.c_void_p(F_ptr), ctypes.byref(h)), "qap_create")
    q.handle = h
    q.n = n
    return q


def qap_create(D, F) -> Qap:
    return Qap(D, F)


def qap_destroy(q: Qap):
    q.close()


def pdit_anneal(q: Qap, replicas: int, beta_schedule, sweeps: int, seed: int):
    """Host-buffer entry point. Returns (best permutation int32[n], best cost)."""
    beta = np.ascontiguousarray(beta_schedule, dtype=np.float32)
    if beta.size < sweeps:
        raise ValueError("beta_schedule shorter than sweeps")
    perm = np.zeros(q.n, dtype=np.int32)
    cost = np.zeros(1, dtype=np.int64)
    _check(lib().pdit_anneal(q.handle, replicas, _ptr(beta) if sweeps else None, sweeps,
                             seed & 0xFFFFFFFFFFFFFFFF, _ptr(perm), _ptr(cost)), "pdit_anneal")
    return perm, int(cost[0])


def pdit_anneal_host_ptrs(q: Qap, replicas: int, beta_ptr: int, sweeps: int, seed: int,
                          perm_ptr: int, cost_ptr: int) -> int:
    """pdit_anneal on raw host pointers (for pinned buffers); returns the code."""
    return lib().pdit_anneal(q.handle, replicas, ctypes.c_void_p(beta_ptr), sweeps,
                             seed & 0xFFFFFFFFFFFFFFFF, ctypes.c_void_p(perm_ptr),
                             ctypes.c_void_p(cost_ptr))


def read_qaplib(path: str):
    """(D, F) int32 arrays of an instance in the QAPLIB text layout (A, B)."""
    n = ctypes.c_int(0)
    _check(lib().pdit_read_qaplib(os.fsencode(path), ctypes.byref(n), None, None, 0), "pdit_read_qaplib")
    D = np.zeros((n.value, n.value), np.int32)
    F = np.zeros_like(D)
    _check(lib().pdit_read_qaplib(os.fsencode(path), ctypes.byref(n), _ptr(D), _ptr(F), D.size),
           "pdit_read_qaplib")
    return D, F


def read_qaplib_solution(path: str):
    """(cost, 0-based permutation) of a solution file in the QAPLIB layout."""
    n = ctypes.c_int(0)
    cost = ctypes.c_int64(0)
    perm = np.zeros(PDIT_N_MAX, np.int32)
    _check(lib().pdit_read_qaplib_solution(os.fsencode(path), ctypes.byref(n), ctypes.byref(cost), _ptr(perm),
                                           PDIT_N_MAX), "pdit_read_qaplib_solution")
    return int(cost.value), perm[:n.value].copy()


def write_qaplib_solution(path: str, perm, cost: int):
    perm = np.ascontiguousarray(perm, np.int32)
    _check(lib().pdit_write_qaplib_solution(os.fsencode(path), perm.size, int(cost), _ptr(perm)),
           "pdit_write_qaplib_solution")


def pdit_instance_form(q: Qap) -> int:
    rc = lib().pdit_instance_form(q.handle)
    if rc < 0:
        raise PditError(rc, "pdit_instance_form")
    return rc


def pdit_set_class_update(q: Qap, enable: bool):
    _check(lib().pdit_set_class_update(q.handle, 1 if enable else 0), "pdit_set_class_update")


def pdit_set_warps_per_replica(q: Qap, wpr: int):
    _check(lib().pdit_set_warps_per_replica(q.handle, wpr), "pdit_set_warps_per_replica")


def pdit_set_table_placement(q: Qap, place: int):
    _check(lib().pdit_set_table_placement(q.handle, place), "pdit_set_table_placement")


def pdit_set_replicas_per_cta(q: Qap, g: int):
    _check(lib().pdit_set_replicas_per_cta(q.handle, g), "pdit_set_replicas_per_cta")


def pdit_set_influence(q: Qap, mode: int):
    _check(lib().pdit_set_influence(q.handle, mode), "pdit_set_influence")


def pdit_set_pending_swaps(q: Qap, k: int):
    _check(lib().pdit_set_pending_swaps(q.handle, k), "pdit_set_pending_swaps")


def pdit_autotune(q: Qap, replicas: int, beta, sweeps: int) -> tuple[int, int]:
    """Time the valid shapes on a short run (beta: CUDA float32 tensor of >= sweeps
    values) and keep the fastest on the handle. Returns (warps per replica, pending terms); the
    placement and replicas per CTA it chose are in pdit_launch_shape."""
    out = np.zeros(2, dtype=np.int32)
    _check(lib().pdit_autotune(q.handle, replicas, ctypes.c_void_p(beta.data_ptr()), sweeps, _ptr(out)),
           "pdit_autotune")
    return int(out[0]), int(out[1])


def pdit_launch_shape(q: Qap, replicas: int) -> dict:
    """The launch a call would use; 'influence' says whether it keeps the
    influence tables ('table') or forms the entries by dot products
    ('products', no table)."""
    out = np.zeros(7, dtype=np.int32)
    _check(lib().pdit_launch_shape(q.handle, replicas, _ptr(out)), "pdit_launch_shape")
    d = dict(zip(["warps_per_replica", "candidates_per_thread", "replicas_per_cta", "ctas",
                  "tables_in_smem", "smem_bytes", "pending_swaps"], (int(x) for x in out)))
    d["influence"] = "products" if d["tables_in_smem"] == 2 else "table"
    d["tables_in_smem"] = 1 if d["tables_in_smem"] == 1 else 0
    return d


def pdit_beta_max(q: Qap) -> float:
    out = ctypes.c_double()
    _check(lib().pdit_beta_max(q.handle, ctypes.byref(out)), "pdit_beta_max")
    return float(out.value)


def pdit_beta_range(q: Qap, points: int = 32, beta_min: float = 0.0, beta_max: float = 0.0,
                    replicas_per_point: int = 8, sweeps: int = 400, seed: int = 0):
    """Returns (beta_lo, beta_hi, mean ending energy per grid point)."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    curve = np.zeros(points, dtype=np.float64)
    _check(lib().pdit_beta_range(q.handle, points, beta_min, beta_max, replicas_per_point, sweeps,
                                 seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(lo), ctypes.byref(hi), _ptr(curve)),
           "pdit_beta_range")
    return float(lo.value), float(hi.value), curve


def pdit_beta_ladder(beta_lo: float, beta_hi: float, length: int = 10) -> np.ndarray:
    out = np.zeros(length, dtype=np.float32)
    _check(lib().pdit_beta_ladder(beta_lo, beta_hi, length, _ptr(out)), "pdit_beta_ladder")
    return out


def pdit_probe_peaks(iters: int = 2000) -> dict:
    """On-chip peaks of the current device (shared-memory load bandwidth,
    dp4a and 32-bit multiply-add rates), per second and per SM clock per SM."""
    out = np.zeros(10, dtype=np.float64)
    _check(lib().pdit_probe_peaks(iters, _ptr(out)), "pdit_probe_peaks")
    return {"smem_bytes_per_s": float(out[0]), "smem_bytes_per_clk_sm": float(out[1]),
            "dp4a_ops_per_s": float(out[2]), "dp4a_ops_per_clk_sm": float(out[3]),
            "imad_ops_per_s": float(out[4]), "imad_ops_per_clk_sm": float(out[5]),
            "mma_f16_macs_per_s": float(out[6]), "mma_f16_macs_per_clk_sm": float(out[7]),
            "mma_s8_macs_per_s": float(out[8]), "mma_s8_macs_per_clk_sm": float(out[9])}


def pdit_beta_schedule(kind: str, sweeps: int, beta_max: float) -> np.ndarray:
    out = np.zeros(max(sweeps, 1), dtype=np.float32)
    _check(lib().pdit_beta_schedule({"linear": 0, "geometric": 1}[kind], sweeps, beta_max, _ptr(out)),
           "pdit_beta_schedule")
    return out[:sweeps]


def pdit_anneal_noalloc(n: int, D_ptr: int, F_ptr: int, replicas: int, beta_ptr: int, sweeps: int,
                        seed: int, best_perm_ptr: int, best_cost_ptr: int, status_ptr: int = 0,
                        stream_ptr: int = 0) -> int:
    """The allocation-free entry point on raw device pointers (status_ptr 0:
    the audit bits are not reported); returns the code."""
    return lib().pdit_anneal_noalloc(n, ctypes.c_void_p(D_ptr), ctypes.c_void_p(F_ptr), replicas,
                                     ctypes.c_void_p(beta_ptr), sweeps, seed & 0xFFFFFFFFFFFFFFFF,
                                     ctypes.c_void_p(best_perm_ptr), ctypes.c_void_p(best_cost_ptr),
                                     ctypes.c_void_p(status_ptr), ctypes.c_void_p(stream_ptr))


def opts(**kw) -> pdit_opts:
    o = pdit_opts()
    lib().pdit_opts_init(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def pdit_workspace_bytes(q: Qap, o: pdit_opts) -> int:
    return int(lib().pdit_workspace_bytes(q.handle, ctypes.byref(o)))


def pdit_anneal_ex(q: Qap, o: pdit_opts):
    _check(lib().pdit_anneal_ex(q.handle, ctypes.byref(o)), "pdit_anneal_ex")


# --- torch convenience (device buffers, current stream) ----------------------

def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def anneal_device(q: Qap, replicas: int, beta, sweeps: int, seed: int, *, mode: int = PDIT_MODE_ANNEAL,
                  ladder_len: int = 0, exchange_period: int = 4, timeout_periods: int = 100,
                  instance_id: int = 0, replica_base: int = 0, sweep_begin: int = 0,
                  sweep_end: int = -1, resume: bool = False, workspace=None, per_replica: bool = False,
                  tables: bool = False, stream=None, target=None, stop_at_target: bool = False):
    """pdit_anneal_ex on torch device tensors. `beta` is a CUDA float32 tensor.
    Returns a dict of device tensors (asynchronous on the current stream)."""
    import torch

    dev = beta.device
    n, R = q.n, replicas
    out = {"best_perm": torch.empty(n, dtype=torch.int32, device=dev),
           "best_cost": torch.empty(1, dtype=torch.int64, device=dev),
           "status": torch.zeros(1, dtype=torch.int32, device=dev)}
    if per_replica:
        out.update(replica_best_cost=torch.empty(R, dtype=torch.int64, device=dev),
                   replica_best_perm=torch.empty(R, n, dtype=torch.int32, device=dev),
                   replica_best_sweep=torch.empty(R, dtype=torch.int32, device=dev),
                   replica_final_perm=torch.empty(R, n, dtype=torch.int32, device=dev),
                   replica_final_cost=torch.empty(R, dtype=torch.int64, device=dev),
                   replica_accepted=torch.empty(R, dtype=torch.int64, device=dev))
        if mode == PDIT_MODE_PT:
            out["replica_rung"] = torch.empty(R, dtype=torch.int32, device=dev)
    if tables:
        out["tables"] = torch.empty(R, n, n, dtype=torch.int32, device=dev)
    if target is not None:
        out["reach_ns"] = torch.empty(1, dtype=torch.int64, device=dev)
        out["reach_sweep"] = torch.empty(1, dtype=torch.int32, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    o = opts(replicas=R, sweeps=sweeps, seed=seed & 0xFFFFFFFFFFFFFFFF, instance_id=instance_id,
             replica_base=replica_base, mode=mode, beta=beta.data_ptr(), ladder_len=ladder_len,
             exchange_period=exchange_period, timeout_periods=timeout_periods,
             sweep_begin=sweep_begin, sweep_end=sweep_end,
             flags=PDIT_FLAG_RESUME if resume else 0, stream=st.cuda_stream)
    for k, t in out.items():
        setattr(o, k, t.data_ptr())
    if target is not None:
        o.target = target.data_ptr()
        o.stop_at_target = 1 if stop_at_target else 0
    if workspace is None:
        # sized for these exact options (the outputs asked for can change the plan)
        need = pdit_workspace_bytes(q, o)
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    o.workspace = workspace.data_ptr()
    o.workspace_bytes = workspace.numel()
    pdit_anneal_ex(q, o)
    out["workspace"] = workspace
    return out


# --- multi-instance batches ----------------------------------------------------

class Batch:
    """pdit_batch_create / pdit_batch_run / pdit_batch_destroy over torch device
    tensors. items: list of dicts with keys qap, replicas, sweeps, beta (CUDA
    float32 tensor), seed, instance_id, and optional target (CUDA int64 [1])."""

    def __init__(self, items, stop_at_target: bool = False, graph: bool = False):
        import torch

        self.items = items
        arr = (pdit_batch_item * len(items))()
        self.out = []
        for k, it in enumerate(items):
            q = it["qap"]
            dev = it["beta"].device
            o = {"best_perm": torch.empty(q.n, dtype=torch.int32, device=dev),
                 "best_cost": torch.empty(1, dtype=torch.int64, device=dev)}
            if it.get("target") is not None:
                o["reach_ns"] = torch.empty(1, dtype=torch.int64, device=dev)
                o["reach_sweep"] = torch.empty(1, dtype=torch.int32, device=dev)
            self.out.append(o)
            e = arr[k]
            e.qap = q.handle.value
            e.replicas = it["replicas"]
            e.sweeps = it["sweeps"]
            e.beta = it["beta"].data_ptr()
            e.seed = it.get("seed", 0) & 0xFFFFFFFFFFFFFFFF
            e.instance_id = it.get("instance_id", 0)
            e.best_perm = o["best_perm"].data_ptr()
            e.best_cost = o["best_cost"].data_ptr()
            if it.get("target") is not None:
                e.target = it["target"].data_ptr()
                e.reach_ns = o["reach_ns"].data_ptr()
                e.reach_sweep = o["reach_sweep"].data_ptr()
        flags = (PDIT_BATCH_STOP_AT_TARGET if stop_at_target else 0) | (PDIT_BATCH_GRAPH if graph else 0)
        h = ctypes.c_void_p()
        _check(lib().pdit_batch_create(arr, len(items), flags, ctypes.byref(h)), "pdit_batch_create")
        self.handle = h

    def run(self, stream=None):
        import torch

        st = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().pdit_batch_run(self.handle, ctypes.c_void_p(st.cuda_stream)), "pdit_batch_run")

    def info(self):
        c, w = ctypes.c_int(), ctypes.c_size_t()
        _check(lib().pdit_batch_info(self.handle, ctypes.byref(c), ctypes.byref(w)), "pdit_batch_info")
        return int(c.value), int(w.value)

    def close(self):
        if getattr(self, "handle", None):
            lib().pdit_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- serving ---------------------------------------------------------------------

class Server:
    """pdit_server_*: continuous-batching request loop (see include/pdit.h)."""

    def __init__(self, device_budget_bytes: int = 8 << 30, slice_sweeps: int = 100, max_active: int = 64):
        h = ctypes.c_void_p()
        _check(lib().pdit_server_create(device_budget_bytes, slice_sweeps, max_active, ctypes.byref(h)),
               "pdit_server_create")
        self.handle = h
        self.n = {}

    def submit(self, D, F, replicas: int, sweeps: int, seed: int, request_id: int, beta=None) -> int:
        D = np.ascontiguousarray(D, dtype=np.int32)
        F = np.ascontiguousarray(F, dtype=np.int32)
        b = None if beta is None else np.ascontiguousarray(beta, dtype=np.float32)
        t = ctypes.c_int64()
        _check(lib().pdit_server_submit(self.handle, D.shape[0], _ptr(D), _ptr(F), replicas, sweeps,
                                        seed & 0xFFFFFFFFFFFFFFFF, request_id,
                                        _ptr(b) if b is not None else None, ctypes.byref(t)),
               "pdit_server_submit")
        self.n[int(t.value)] = D.shape[0]
        return int(t.value)

    def tick(self):
        a, q = ctypes.c_int(), ctypes.c_int()
        _check(lib().pdit_server_tick(self.handle, ctypes.byref(a), ctypes.byref(q)), "pdit_server_tick")
        return int(a.value), int(q.value)

    def result(self, ticket: int):
        """(state, perm or None, cost or None, latency or None)."""
        st = ctypes.c_int()
        perm = np.zeros(self.n[ticket], dtype=np.int32)
        cost = ctypes.c_int64()
        lat = ctypes.c_double()
        _check(lib().pdit_server_result(self.handle, ticket, ctypes.byref(st), _ptr(perm), ctypes.byref(cost),
                                        ctypes.byref(lat)), "pdit_server_result")
        if st.value != 2:
            return int(st.value), None, None, None
        return 2, perm, int(cost.value), float(lat.value)

    def close(self):
        if getattr(self, "handle", None):
            lib().pdit_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
