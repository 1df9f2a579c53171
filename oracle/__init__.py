"""NanoGS FP64 CPU oracle -- test infrastructure.

Python view of the plain C oracle in ``ngs_oracle.c``.  Only the tests, the
smoke check and the benchmark's CPU-baseline leg may import this package; the
library's product path must never reach it.

Every function takes numpy arrays (float32 or float64 splat arrays are cast
to float64) and returns numpy arrays.  Splats are a 5-tuple
``(xyz, log_scale, rot, logit, sh)`` or any object with those attributes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "ngs_oracle.c")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_ptr = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile ``ngs_oracle.c`` into ``liboracle.so`` next to it (gcc, -O2,
    no FP contraction so x86 and Arm hosts round alike, OpenMP on)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
               "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            L.orc_prefilter.restype = _i64
            L.orc_prefilter.argtypes = [_i64, _ptr, _dbl, _ptr]
            L.orc_knn_brute.restype = ctypes.c_int
            L.orc_knn_brute.argtypes = [_i64, _ptr, ctypes.c_int, _ptr]
            L.orc_knn_brute_queries.restype = ctypes.c_int
            L.orc_knn_brute_queries.argtypes = [_i64, _ptr, ctypes.c_int, _i64, _ptr, _ptr]
            L.orc_knn_grid.restype = ctypes.c_int
            L.orc_knn_grid.argtypes = [_i64, _ptr, ctypes.c_int, _ptr]
            L.orc_union_edges.restype = _i64
            L.orc_union_edges.argtypes = [_i64, ctypes.c_int, _ptr, _ptr, _ptr]
            L.orc_mc_draws.restype = None
            L.orc_mc_draws.argtypes = [_u64, _u32, ctypes.c_int, _ptr, _ptr]
            L.orc_edge_costs.restype = None
            L.orc_edge_costs.argtypes = [_i64, _ptr, _ptr, _ptr, _ptr, _ptr, ctypes.c_int,
                                         _i64, _ptr, _ptr, ctypes.c_int, _ptr, _ptr,
                                         ctypes.c_int, _dbl, _dbl, _ptr, _ptr, _ptr]
            L.orc_greedy.restype = _i64
            L.orc_greedy.argtypes = [_i64, _i64, _ptr, _ptr, _ptr, _i64, _ptr, _ptr]
            L.orc_merge_compact.restype = _i64
            L.orc_merge_compact.argtypes = [_i64, _ptr, _ptr, _ptr, _ptr, _ptr, ctypes.c_int,
                                            _i64, _ptr, _ptr, _dbl,
                                            _ptr, _ptr, _ptr, _ptr, _ptr]
            L.orc_simplify.restype = _i64
            L.orc_simplify.argtypes = [_i64, _ptr, _ptr, _ptr, _ptr, _ptr, ctypes.c_int, _i64,
                                       ctypes.c_int, _dbl, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _dbl, _dbl, _u64, _dbl, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, _ptr, _ptr, _ptr, _ptr, _ptr]
            L.orc_refresh_lists.restype = _i64
            L.orc_refresh_lists.argtypes = [_i64, ctypes.c_int, _ptr, _i64, _ptr, _ptr, _i64,
                                            _ptr, ctypes.c_int, _ptr, _ptr]
            L.orc_quat_to_R.restype = None
            L.orc_quat_to_R.argtypes = [_ptr, _ptr]
            L.orc_eig3.restype = ctypes.c_int
            L.orc_eig3.argtypes = [_ptr, _ptr, _ptr]
            L.orc_R_to_quat.restype = None
            L.orc_R_to_quat.argtypes = [_ptr, _ptr]
            L.orc_mpmm_moments.restype = None
            L.orc_mpmm_moments.argtypes = [_dbl, _ptr, _ptr, _ptr, _dbl, _ptr, _ptr, _ptr,
                                           ctypes.c_int, _ptr, _ptr, _ptr]
            L.orc_kl_gauss.restype = _dbl
            L.orc_kl_gauss.argtypes = [_ptr, _ptr, _ptr, _ptr]
            L.orc_idiv_gauss.restype = _dbl
            L.orc_idiv_gauss.argtypes = [_dbl, _ptr, _ptr, _dbl, _ptr, _ptr]
            L.orc_dgeo_pair.restype = _dbl
            L.orc_dgeo_pair.argtypes = [_ptr, _ptr, _ptr, _dbl, _ptr, _ptr, _ptr, _dbl,
                                        ctypes.c_int, _ptr, _ptr, ctypes.c_int]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _splat_arrays(s):
    if isinstance(s, (tuple, list)):
        xyz, ls, rot, logit, sh = s
    else:
        xyz, ls, rot, logit, sh = s.xyz, s.log_scale, s.rot, s.logit, s.sh
    sh = _d(sh)
    n = _d(xyz).reshape(-1, 3).shape[0]
    return (_d(xyz).reshape(n, 3), _d(ls).reshape(n, 3), _d(rot).reshape(n, 4),
            _d(logit).reshape(n), sh.reshape(n, -1) if n else sh.reshape(0, 48))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(t: int) -> int:
    """Threads of the oracle's parallel loops from now on (timing only; the
    results do not depend on it).  Returns the count in effect."""
    return int(lib().orc_set_num_threads(int(t)))


def k_effective(n: int, k: int) -> int:
    """k_eff = min(max(1, k), N - 1), Algorithm 1."""
    return min(max(1, k), n - 1)


def target_count(n0: int, ratio: float) -> int:
    """N_tgt = max(ceil(r N0), 1), Algorithm 1."""
    import math
    return max(int(math.ceil(ratio * n0)), 1)


def prefilter(logit, tau: float = 0.005):
    logit = _d(logit).reshape(-1)
    keep = np.zeros(logit.shape[0], dtype=np.uint8)
    cnt = lib().orc_prefilter(logit.shape[0], _p(logit), tau, _p(keep))
    return keep.astype(bool), int(cnt)


def knn(xyz, k: int = 16, method: str = "brute", queries=None):
    xyz = _d(xyz).reshape(-1, 3)
    n = xyz.shape[0]
    ke = k_effective(n, k)
    if ke <= 0:
        return np.zeros((0 if queries is None else len(queries), 0), dtype=np.int32)
    if queries is not None:
        q = np.ascontiguousarray(queries, dtype=np.int64)
        out = np.zeros((q.shape[0], ke), dtype=np.int32)
        lib().orc_knn_brute_queries(n, _p(xyz), k, q.shape[0], _p(q), _p(out))
        return out
    out = np.zeros((n, ke), dtype=np.int32)
    if method == "brute":
        lib().orc_knn_brute(n, _p(xyz), k, _p(out))
    else:
        lib().orc_knn_grid(n, _p(xyz), k, _p(out))
    return out


def union_edges(nbr):
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    n, ke = nbr.shape
    lo = np.zeros(max(1, n * ke), dtype=np.int32)
    hi = np.zeros(max(1, n * ke), dtype=np.int32)
    m = lib().orc_union_edges(n, ke, _p(nbr), _p(lo), _p(hi))
    return lo[:m].copy(), hi[:m].copy()


def mc_draws(seed: int, pass_index: int, S: int = 1):
    z = np.zeros((S, 3), dtype=np.float32)
    u = np.zeros(S, dtype=np.float32)
    lib().orc_mc_draws(seed, pass_index, S, _p(z), _p(u))
    return z, u


def edge_costs(splats, lo, hi, z, u, mode: int = 0, lambda_geo: float = 1.0,
               lambda_app: float = 1.0, parts: bool = False):
    xyz, ls, rot, logit, sh = _splat_arrays(splats)
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    z = np.ascontiguousarray(z, dtype=np.float32).reshape(-1, 3)
    u = np.ascontiguousarray(u, dtype=np.float32).reshape(-1)
    m = lo.shape[0]
    cost = np.zeros(m)
    dgeo = np.zeros(m)
    dapp = np.zeros(m)
    lib().orc_edge_costs(xyz.shape[0], _p(xyz), _p(ls), _p(rot), _p(logit), _p(sh), sh.shape[1],
                         m, _p(lo), _p(hi), z.shape[0], _p(z), _p(u), mode, lambda_geo,
                         lambda_app, _p(cost), _p(dgeo), _p(dapp))
    return (cost, dgeo, dapp) if parts else cost


def greedy(n: int, lo, hi, cost, P: int):
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    cost = _d(cost)
    m = lo.shape[0]
    cap = max(1, n // 2 + 1)
    plo = np.zeros(cap, dtype=np.int32)
    phi = np.zeros(cap, dtype=np.int32)
    cnt = lib().orc_greedy(n, m, _p(lo), _p(hi), _p(cost), P, _p(plo), _p(phi))
    return plo[:cnt].copy(), phi[:cnt].copy()


def merge_compact(splats, pair_lo, pair_hi, eig_floor: float = 1e-30):
    xyz, ls, rot, logit, sh = _splat_arrays(splats)
    n, F = sh.shape
    plo = np.ascontiguousarray(pair_lo, dtype=np.int32)
    phi = np.ascontiguousarray(pair_hi, dtype=np.int32)
    out = [np.zeros_like(a) for a in (xyz, ls, rot, logit, sh)]
    nn = lib().orc_merge_compact(n, _p(xyz), _p(ls), _p(rot), _p(logit), _p(sh), F,
                                 plo.shape[0], _p(plo), _p(phi), eig_floor,
                                 *[_p(a) for a in out])
    if nn < 0:
        raise ValueError("invalid pair list")
    return tuple(a[:nn].copy() for a in out)


def simplify(splats, target: int, k: int = 16, tau: float = 0.005, prefilter: bool = True,
             S: int = 1, mode: int = 0, lambda_geo: float = 1.0, lambda_app: float = 1.0,
             seed: int = 0, eig_floor: float = 1e-30, max_passes: int = 64,
             use_grid: bool = True, refresh_period: int = 1):
    arrs = [a.copy() for a in _splat_arrays(splats)]
    xyz, ls, rot, logit, sh = arrs
    n0, F = sh.shape
    passes = np.zeros(1, dtype=np.int32)
    pn = np.zeros(max_passes, dtype=np.int64)
    pe = np.zeros(max_passes, dtype=np.int64)
    pm = np.zeros(max_passes, dtype=np.int64)
    prq = np.zeros(max_passes, dtype=np.int64)
    nn = lib().orc_simplify(n0, _p(xyz), _p(ls), _p(rot), _p(logit), _p(sh), F, target, k,
                            tau, int(prefilter), S, mode, lambda_geo, lambda_app, seed,
                            eig_floor, max_passes, int(use_grid), int(refresh_period),
                            _p(passes), _p(pn), _p(pe), _p(pm), _p(prq))
    p = int(passes[0])
    stats = {"passes": p, "n": pn[:p].tolist(), "edges": pe[:p].tolist(),
             "pairs": pm[:p].tolist(), "requeried": prq[:p].tolist()}
    return tuple(a[:nn].copy() for a in arrs), stats


def refresh_lists(prev, pair_lo, pair_hi, xyz_new, k: int = 16):
    """Sec. 3.4 local refresh: (lists of the new splats, re-query flags)."""
    prev = np.ascontiguousarray(prev, dtype=np.int32)
    n_old, k_old = prev.shape
    plo = np.ascontiguousarray(pair_lo, dtype=np.int32)
    phi = np.ascontiguousarray(pair_hi, dtype=np.int32)
    xyz = _d(xyz_new).reshape(-1, 3)
    n_new = xyz.shape[0]
    ke = k_effective(n_new, k)
    out = np.full((n_new, max(ke, 0)), -1, dtype=np.int32)
    rq = np.zeros(n_new, dtype=np.uint8)
    lib().orc_refresh_lists(n_old, k_old, _p(prev), plo.shape[0], _p(plo), _p(phi), n_new,
                            _p(xyz), k, _p(out), _p(rq))
    return out, rq.astype(bool)


# ---- single-pair helpers (pins) ----

def quat_to_R(q):
    q = _d(q)
    R = np.zeros(9)
    lib().orc_quat_to_R(_p(q), _p(R))
    return R.reshape(3, 3)


def eig3(A):
    A = _d(A).reshape(9)
    lam = np.zeros(3)
    V = np.zeros(9)
    sweeps = lib().orc_eig3(_p(A), _p(lam), _p(V))
    return lam, V.reshape(3, 3), sweeps


def R_to_quat(R):
    R = _d(R).reshape(9)
    q = np.zeros(4)
    lib().orc_R_to_quat(_p(R), _p(q))
    return q


def mpmm_moments(wi, mui, Si, fi, wj, muj, Sj, fj):
    mui, Si, muj, Sj = _d(mui), _d(Si).reshape(9), _d(muj), _d(Sj).reshape(9)
    fi, fj = _d(fi).reshape(-1), _d(fj).reshape(-1)
    F = fi.shape[0]
    mum, Sm, fm = np.zeros(3), np.zeros(9), np.zeros(max(F, 1))
    lib().orc_mpmm_moments(wi, _p(mui), _p(Si), _p(fi), wj, _p(muj), _p(Sj), _p(fj), F,
                           _p(mum), _p(Sm), _p(fm))
    return mum, Sm.reshape(3, 3), fm[:F]


def kl_gauss(mui, Si, muj, Sj):
    return lib().orc_kl_gauss(_p(_d(mui)), _p(_d(Si).reshape(9)), _p(_d(muj)),
                              _p(_d(Sj).reshape(9)))


def idiv_gauss(mi, mui, Si, mj, muj, Sj):
    return lib().orc_idiv_gauss(mi, _p(_d(mui)), _p(_d(Si).reshape(9)), mj, _p(_d(muj)),
                                _p(_d(Sj).reshape(9)))


def dgeo_pair(si, sj, z, u=None, mode: int = 0):
    """si, sj: (xyz[3], log_scale[3], rot[4], logit) for one splat each."""
    z = np.ascontiguousarray(z, dtype=np.float32).reshape(-1, 3)
    S = z.shape[0]
    u = np.zeros(S, dtype=np.float32) if u is None else np.ascontiguousarray(u, np.float32)
    a = [_d(x) for x in si[:3]]
    b = [_d(x) for x in sj[:3]]
    return lib().orc_dgeo_pair(_p(a[0]), _p(a[1]), _p(a[2]), float(si[3]),
                               _p(b[0]), _p(b[1]), _p(b[2]), float(sj[3]),
                               S, _p(z), _p(u), mode)
