"""CPU oracle for the annealed p-dit sweep (ctypes bindings to pdit_oracle.c).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline / reference arm may import this package. It
shares no code with the CUDA path. See pdit_oracle.c for the passages of the
paper each function follows.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdit_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_lib = None

I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
U32P = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
U64P = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
F32P = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, no contraction of float ops)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class _Replica(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int),
                ("D", ctypes.c_void_p), ("F", ctypes.c_void_p),
                ("p", ctypes.c_void_p), ("I", ctypes.c_void_p),
                ("E", ctypes.c_int64), ("general", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        c_int, c_u32, c_u64, c_i64, vp = ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
        L.oracle_philox4x32_10.argtypes = [U32P, U32P, U32P]
        L.oracle_philox4x32_10.restype = None
        L.oracle_update_draw.argtypes = [c_u64, c_u32, c_u32, c_u32, c_u32]
        L.oracle_update_draw.restype = c_u64
        L.oracle_init_perm.argtypes = [c_int, c_u64, c_u32, c_u32, I32P]
        L.oracle_init_perm.restype = None
        L.oracle_cost.argtypes = [c_int, I32P, I32P, I32P]
        L.oracle_cost.restype = c_i64
        L.oracle_influence.argtypes = [c_int, I32P, I32P, I32P, I64P]
        L.oracle_influence.restype = None
        L.oracle_influence_eq2.argtypes = [c_int, I32P, I32P, I32P, I64P]
        L.oracle_influence_eq2.restype = None
        L.oracle_delta_e.argtypes = [c_int, I32P, I32P, I32P, I64P, c_int, c_int]
        L.oracle_delta_e.restype = c_i64
        L.oracle_delta_e_eq3.argtypes = [c_int, I32P, I32P, I32P, I64P, c_int, c_int]
        L.oracle_delta_e_eq3.restype = c_i64
        L.oracle_is_symmetric.argtypes = [c_int, I32P]
        L.oracle_is_symmetric.restype = c_int
        L.oracle_expneg_f32.argtypes = [ctypes.c_float]
        L.oracle_expneg_f32.restype = ctypes.c_float
        L.oracle_weight.argtypes = [ctypes.c_float]
        L.oracle_weight.restype = c_u64
        L.oracle_choose.argtypes = [ctypes.POINTER(_Replica), c_int, ctypes.c_float, c_u64, vp, vp, vp]
        L.oracle_choose.restype = c_int
        L.oracle_pt_exchange.argtypes = [c_int, I64P, I32P, ctypes.POINTER(ctypes.c_int32), c_int]
        L.oracle_pt_exchange.restype = None
        L.oracle_anneal.argtypes = [c_int, I32P, I32P, c_int, c_int, c_int, c_int, c_int, c_int,
                                    F32P, c_int, c_u64, c_u32, c_int,
                                    I32P, I64P, I32P, I64P, I32P, I64P, vp, vp, vp,
                                    c_int, c_i64, vp, c_int]
        L.oracle_anneal.restype = c_int
        L.oracle_argmin_best.argtypes = [c_int, I64P]
        L.oracle_argmin_best.restype = c_int
        L.oracle_brute_force.argtypes = [c_int, I32P, I32P, I32P, ctypes.POINTER(ctypes.c_int64)]
        L.oracle_brute_force.restype = c_i64
        L.oracle_beta_max.argtypes = [c_int, I32P, I32P]
        L.oracle_beta_max.restype = ctypes.c_double
        L.oracle_beta_schedule.argtypes = [c_int, c_int, ctypes.c_double, F32P]
        L.oracle_beta_schedule.restype = None
        _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# --- Primitives --------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(np.ascontiguousarray(ctr, dtype=np.uint32),
                               np.ascontiguousarray(key, dtype=np.uint32), out)
    return out


def update_draw(seed: int, inst: int, rep: int, sweep: int, loc: int) -> int:
    return int(lib().oracle_update_draw(seed, inst, rep, sweep, loc))


def init_perm(n: int, seed: int, inst: int, rep: int) -> np.ndarray:
    p = np.zeros(n, dtype=np.int32)
    lib().oracle_init_perm(n, seed, inst, rep, p)
    return p


def cost(D, F, p) -> int:
    D, F = _i32(D), _i32(F)
    return int(lib().oracle_cost(D.shape[0], D, F, _i32(p)))


def influence(D, F, p) -> np.ndarray:
    D, F = _i32(D), _i32(F)
    n = D.shape[0]
    out = np.zeros((n, n), dtype=np.int64)
    lib().oracle_influence(n, D, F, _i32(p), out)
    return out


def influence_eq2(D, F, p) -> np.ndarray:
    D, F = _i32(D), _i32(F)
    n = D.shape[0]
    out = np.zeros((n, n), dtype=np.int64)
    lib().oracle_influence_eq2(n, D, F, _i32(p), out)
    return out


def delta_e(D, F, p, I, i: int, j: int) -> int:
    D, F = _i32(D), _i32(F)
    return int(lib().oracle_delta_e(D.shape[0], D, F, _i32(p),
                                    np.ascontiguousarray(I, dtype=np.int64), i, j))


def delta_e_eq3(D, F, p, Ip, i: int, j: int) -> int:
    """Eq. 3 as printed, with Eq. 2's table Ip (general D and F)."""
    D, F = _i32(D), _i32(F)
    return int(lib().oracle_delta_e_eq3(D.shape[0], D, F, _i32(p),
                                        np.ascontiguousarray(Ip, dtype=np.int64), i, j))


def is_symmetric(M) -> bool:
    M = _i32(M)
    return bool(lib().oracle_is_symmetric(M.shape[0], M))


def general_form(D, F) -> bool:
    """True when the oracle runs the general form for (D, F)."""
    return not (is_symmetric(D) and is_symmetric(F))


def expneg_f32(x: float) -> np.float32:
    return np.float32(lib().oracle_expneg_f32(float(np.float32(x))))


def weight(x: float) -> int:
    return int(lib().oracle_weight(float(np.float32(x))))


def choose(D, F, p, i: int, beta: float, r: int, general: bool | None = None):
    """One Eq. 5 update at location i from state p (table built from p).
    Returns (chosen j, dE[n] int64, weights[n] uint64, near-boundary flag)."""
    D, F, p = _i32(D), _i32(F), _i32(p).copy()
    n = D.shape[0]
    if general is None:
        general = general_form(D, F)
    I = influence_eq2(D, F, p) if general else influence(D, F, p)
    dE = np.zeros(n, dtype=np.int64)
    w = np.zeros(n, dtype=np.uint64)
    near = ctypes.c_int(0)
    rep = _Replica(n, D.ctypes.data, F.ctypes.data, p.ctypes.data, I.ctypes.data, cost(D, F, p),
                   1 if general else 0)
    j = lib().oracle_choose(ctypes.byref(rep), i, float(np.float32(beta)), r & 0xFFFFFFFFFFFFFFFF,
                            dE.ctypes.data, w.ctypes.data, ctypes.addressof(near))
    return j, dE, w, near.value


def pt_exchange(E, rung, since_top: int, timeout: int):
    """One exchange period for one set. Returns (new rung_of_slot, new counter)."""
    rung = np.ascontiguousarray(rung, dtype=np.int32).copy()
    c = ctypes.c_int32(since_top)
    lib().oracle_pt_exchange(len(rung), np.ascontiguousarray(E, dtype=np.int64), rung,
                             ctypes.byref(c), timeout)
    return rung, c.value


def brute_force(D, F):
    D, F = _i32(D), _i32(F)
    n = D.shape[0]
    p = np.zeros(n, dtype=np.int32)
    cnt = ctypes.c_int64(0)
    best = lib().oracle_brute_force(n, D, F, p, ctypes.byref(cnt))
    return int(best), p, int(cnt.value)


def beta_max(D, F) -> float:
    D, F = _i32(D), _i32(F)
    return float(lib().oracle_beta_max(D.shape[0], D, F))


def beta_schedule(kind: str, sweeps: int, bmax: float) -> np.ndarray:
    out = np.zeros(max(sweeps, 1), dtype=np.float32)
    lib().oracle_beta_schedule({"linear": 0, "geometric": 1}[kind], sweeps, bmax, out)
    return out[:sweeps]


# --- Full runs ---------------------------------------------------------------

def anneal(D, F, beta, sweeps: int, seed: int, rep_begin: int = 0, rep_end: int = 1,
           inst: int = 0, threads: int = 1, mode: str = "anneal", ladder_len: int = 0,
           period: int = 4, timeout: int = 100, near: bool = False, tables: bool = False,
           target=None, form: str = "auto") -> dict:
    """Runs replicas [rep_begin, rep_end). mode 'anneal': beta[s] per sweep;
    mode 'pt': beta is the ladder (rung 0 = smallest beta), sets of ladder_len
    consecutive replicas exchange every `period` sweeps; mode 'fixed':
    beta[k] for the k-th replica of the call, no exchange; mode 'cupim':
    concurrent updates, beta[s] per iteration. form 'auto': the symmetric
    form (table I) when D and F are symmetric, else the general form (Eq. 2's
    table Ip, Eq. 3 as printed); 'general': the general form always.
    out['tables'] holds the table of the form used; out['general'] says which."""
    D, F = _i32(D), _i32(F)
    n = D.shape[0]
    R = rep_end - rep_begin
    beta = np.ascontiguousarray(beta, dtype=np.float32)
    out = dict(final_perm=np.zeros((R, n), np.int32), final_cost=np.zeros(R, np.int64),
               best_perm=np.zeros((R, n), np.int32), best_cost=np.zeros(R, np.int64),
               best_sweep=np.zeros(R, np.int32), accepted=np.zeros(R, np.int64))
    nb = np.zeros(R, np.int64) if near else None
    tab = np.zeros((R, n, n), np.int64) if tables else None
    rung = np.zeros(R, np.int32) if mode == "pt" else None
    reach = np.zeros(R, np.int32) if target is not None else None
    rc = lib().oracle_anneal(
        n, D, F, rep_begin, rep_end, {"anneal": 0, "pt": 1, "fixed": 2, "cupim": 3}[mode], ladder_len, period, timeout,
        beta, sweeps, seed, inst, threads, out["final_perm"], out["final_cost"],
        out["best_perm"], out["best_cost"], out["best_sweep"], out["accepted"],
        nb.ctypes.data if nb is not None else None,
        tab.ctypes.data if tab is not None else None,
        rung.ctypes.data if rung is not None else None,
        1 if target is not None else 0, int(target) if target is not None else 0,
        reach.ctypes.data if reach is not None else None,
        {"auto": 0, "general": 1}[form])
    out["general"] = form == "general" or general_form(D, F)
    if rc != 0:
        raise ValueError("oracle_anneal rejected its arguments")
    if nb is not None:
        out["near_boundary"] = nb
    if tab is not None:
        out["tables"] = tab
    if rung is not None:
        out["rung"] = rung
    if reach is not None:
        out["reach_sweep"] = reach
    w = int(lib().oracle_argmin_best(R, out["best_cost"]))
    out["winner"] = w
    out["cost"] = int(out["best_cost"][w])
    out["perm"] = out["best_perm"][w].copy()
    return out


# --- beta-range selection (Implementation section, CPU-PIM Algorithm, Fig. 2b) ---

def beta_grid(points: int, bmin: float, bmax: float) -> np.ndarray:
    """Geometric grid of `points` betas from bmin to bmax (double, then binary32)."""
    return np.array([np.float32(bmin * (bmax / bmin) ** (k / (points - 1))) for k in range(points)],
                    dtype=np.float32)


def select_beta_range(mean_energy) -> tuple[int, int]:
    """Indices (lo, hi) from the mean ending energy per beta (ascending beta):
    lo = first point at or below min + 0.4 (max - min); hi = two points past
    the minimum, clamped to the grid."""
    e = np.asarray(mean_energy, dtype=np.float64)
    kmin = int(np.argmin(e))
    thr = e[kmin] + 0.4 * (e.max() - e[kmin])
    lo = int(np.flatnonzero(e <= thr)[0])
    hi = min(kmin + 2, len(e) - 1)
    return lo, hi


def beta_range(D, F, points: int = 32, bmin: float = 0.0, bmax: float = 0.0, rpp: int = 8,
               sweeps: int = 400, seed: int = 0, threads: int = 8):
    """Short fixed-beta trials without exchange; returns (beta_lo, beta_hi,
    mean ending energy per point, grid)."""
    if not (bmin > 0 and bmax > bmin):
        b = beta_max(D, F)
        bmin, bmax = b / 1000.0, b * 10.0
    grid = beta_grid(points, bmin, bmax)
    rbeta = np.repeat(grid, rpp).astype(np.float32)
    r = anneal(D, F, rbeta, sweeps, seed, 0, points * rpp, threads=threads, mode="fixed")
    mean = r["final_cost"].reshape(points, rpp).astype(np.float64).mean(axis=1)
    lo, hi = select_beta_range(mean)
    return float(grid[lo]), float(grid[hi]), mean, grid
