"""Thin Python binding of the C ABI in ``include/ngs.h``.

Argument marshalling only: every function of the same name forwards to
``libngs.so`` through ctypes, and every step of the simplification runs in
the library's CUDA kernels.  Torch tensors provide device memory and streams.
The library must be built (``paper_2603_16103_gb300.build.build()``); this
module raises if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

_LIB = None

NGS_OK = 0
NGS_ERR_INVALID_ARG = -1
NGS_ERR_OOM = -2
NGS_ERR_CUDA = -3
NGS_ERR_TIMEOUT = -4
NGS_ERR_BUDGET = -5
NGS_ERR_STATE = -6
NGS_STATS_MAX_PASSES = 64
NGS_MAX_K = 32
NGS_MAX_N = 1 << 26
NGS_MAX_S = 128
NGS_MAX_SCENES = 4096


class NgsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ngs error {code}: {msg}")
        self.code = code


class ngs_splats(ctypes.Structure):
    _fields_ = [("xyz", ctypes.c_void_p), ("log_scale", ctypes.c_void_p),
                ("rot", ctypes.c_void_p), ("opacity_logit", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("n", ctypes.c_int64), ("cap", ctypes.c_int64),
                ("sh_dim", ctypes.c_int32)]


class ngs_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("mc_samples", ctypes.c_int32),
                ("cost_mode", ctypes.c_int32), ("tau", ctypes.c_double),
                ("lambda_geo", ctypes.c_float), ("lambda_app", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("max_passes", ctypes.c_int32),
                ("fp64_policy", ctypes.c_int32), ("prefilter", ctypes.c_int32),
                ("eig_floor", ctypes.c_double), ("cost_tol", ctypes.c_double),
                ("refresh_period", ctypes.c_int32)]


class ngs_graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("k_eff", ctypes.c_int32), ("n_edges", ctypes.c_int64),
                ("nbr", ctypes.c_void_p), ("edge_lo", ctypes.c_void_p),
                ("edge_hi", ctypes.c_void_p)]


class ngs_stats(ctypes.Structure):
    _fields_ = [("n_input", ctypes.c_int64), ("n_filtered", ctypes.c_int64),
                ("n_output", ctypes.c_int64), ("passes", ctypes.c_int32),
                ("matching_rounds", ctypes.c_int32),
                ("pass_n", ctypes.c_int64 * NGS_STATS_MAX_PASSES),
                ("pass_edges", ctypes.c_int64 * NGS_STATS_MAX_PASSES),
                ("pass_pairs", ctypes.c_int64 * NGS_STATS_MAX_PASSES),
                ("fp64_cost_edges", ctypes.c_int64), ("eig_floor_hits", ctypes.c_int64),
                ("gpu_launches", ctypes.c_int64), ("near_tie_slots", ctypes.c_int64),
                ("requeried_rows", ctypes.c_int64), ("host_syncs", ctypes.c_int64)]

    def as_dict(self) -> dict:
        p = self.passes
        return {"n_input": self.n_input, "n_filtered": self.n_filtered,
                "n_output": self.n_output, "passes": p,
                "matching_rounds": self.matching_rounds,
                "pass_n": list(self.pass_n[:p]), "pass_edges": list(self.pass_edges[:p]),
                "pass_pairs": list(self.pass_pairs[:p]),
                "fp64_cost_edges": self.fp64_cost_edges,
                "eig_floor_hits": self.eig_floor_hits, "gpu_launches": self.gpu_launches,
                "near_tie_slots": self.near_tie_slots, "requeried_rows": self.requeried_rows,
                "host_syncs": self.host_syncs}


class ngs_tuning(ctypes.Structure):
    _fields_ = [("knn_block_min", ctypes.c_int32), ("cells_per_point", ctypes.c_int32),
                ("cost_blocks_per_sm", ctypes.c_int32), ("match_method", ctypes.c_int32),
                ("match_max_steps", ctypes.c_int32), ("scan_method", ctypes.c_int32),
                ("wait_budget_cycles", ctypes.c_int32),
                ("wait_test_tile", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class ngs_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("group_small", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("bytes_per_splat", ctypes.c_int64),
                ("small_rows", ctypes.c_int64), ("group_rows", ctypes.c_int64),
                ("dry_run_ns_per_splat", ctypes.c_double), ("priority_rows", ctypes.c_int64)]


class ngs_job_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("slot", ctypes.c_int32), ("group", ctypes.c_int64),
                ("group_size", ctypes.c_int32), ("n_in", ctypes.c_int64),
                ("target", ctypes.c_int64), ("n_out", ctypes.c_int64),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("finish_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class ngs_server_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in (
        "submitted", "finished", "failed", "queued", "running", "groups", "reserved_bytes",
        "peak_reserved_bytes", "workspace_bytes", "peak_workspace_bytes", "gpu_launches")]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


NGS_JOB_QUEUED = 1
NGS_JOB_RUNNING = 2
NGS_JOB_DONE = 0

_P = ctypes.c_void_p
_SIGS = {
    "ngs_default_params": (None, [ctypes.POINTER(ngs_params)]),
    "ngs_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ngs_params), _P]),
    "ngs_destroy": (ctypes.c_int, [_P]),
    "ngs_set_params": (ctypes.c_int, [_P, ctypes.POINTER(ngs_params)]),
    "ngs_last_error": (ctypes.c_char_p, []),
    "ngs_prefilter": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats)]),
    "ngs_build_graph": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats), ctypes.POINTER(ngs_graph)]),
    "ngs_build_graph_refresh": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats), _P, ctypes.c_int64,
                                               ctypes.c_int32, _P, ctypes.c_int64,
                                               ctypes.POINTER(ngs_graph),
                                               ctypes.POINTER(ctypes.c_int64)]),
    "ngs_edge_costs": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats), ctypes.POINTER(ngs_graph),
                                      ctypes.c_uint32, _P]),
    "ngs_select_pairs": (ctypes.c_int, [_P, ctypes.POINTER(ngs_graph), _P, ctypes.c_int64, _P,
                                        ctypes.POINTER(ctypes.c_int64)]),
    "ngs_merge_compact": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats), _P, ctypes.c_int64]),
    "ngs_selftest_ff": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int64, _P]),
    "ngs_simplify": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats), ctypes.c_int64,
                                    ctypes.POINTER(ngs_stats)]),
    "ngs_batch_simplify": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                          ctypes.POINTER(ngs_stats)]),
    "ngs_simplify_host": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats), ctypes.c_int64,
                                         ctypes.POINTER(ngs_stats)]),
    "ngs_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "ngs_profile_count": (ctypes.c_int, [_P]),
    "ngs_profile_get": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                       ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double)]),
    "ngs_profile_reset": (ctypes.c_int, [_P]),
    "ngs_launch_count": (ctypes.c_int64, [_P]),
    "ngs_knn_noalloc": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _P, _P]),
    "ngs_workspace_bytes": (ctypes.c_int64, [_P]),
    "ngs_release_workspace": (ctypes.c_int, [_P]),
    "ngs_pool_usage": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64)]),
    "ngs_set_stream": (ctypes.c_int, [_P, _P]),
    "ngs_default_tuning": (None, [ctypes.POINTER(ngs_tuning)]),
    "ngs_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(ngs_tuning)]),
    "ngs_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(ngs_tuning)]),
    "ngs_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats), ctypes.POINTER(ngs_tuning),
                                    ctypes.POINTER(ctypes.c_double)]),
    "ngs_server_default_config": (None, [ctypes.POINTER(ngs_server_config)]),
    "ngs_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ngs_params),
                                         ctypes.POINTER(ngs_server_config)]),
    "ngs_server_destroy": (ctypes.c_int, [_P]),
    "ngs_serve_submit": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats), ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "ngs_serve_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int64)]),
    "ngs_serve_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_int64)]),
    "ngs_serve_info": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ngs_job_info)]),
    "ngs_server_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(ngs_server_stats)]),
    "ngs_server_clock": (ctypes.c_double, [_P]),
    "ngs_serve_replay": (ctypes.c_int, [_P, ctypes.POINTER(ngs_splats),
                                        ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_uint64)]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libngs.so (building it first if asked); raise if unavailable."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run build() first")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(rc: int):
    if rc != NGS_OK:
        raise NgsError(rc, load().ngs_last_error().decode(errors="replace"))


# ---------------------------------------------------------------- same-name wrappers

def ngs_default_params() -> ngs_params:
    p = ngs_params()
    load().ngs_default_params(ctypes.byref(p))
    return p


def ngs_create(params: ngs_params | None = None, stream=None) -> int:
    ctx = _P()
    s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    _check(load().ngs_create(ctypes.byref(ctx), ctypes.byref(params) if params else None,
                             _P(s)))
    return ctx.value


def ngs_destroy(ctx: int):
    _check(load().ngs_destroy(_P(ctx)))


def ngs_set_params(ctx: int, params: ngs_params):
    _check(load().ngs_set_params(_P(ctx), ctypes.byref(params)))


def ngs_last_error() -> str:
    return load().ngs_last_error().decode(errors="replace")


def ngs_prefilter(ctx: int, s: ngs_splats) -> int:
    _check(load().ngs_prefilter(_P(ctx), ctypes.byref(s)))
    return s.n


def ngs_build_graph(ctx: int, s: ngs_splats) -> ngs_graph:
    g = ngs_graph()
    _check(load().ngs_build_graph(_P(ctx), ctypes.byref(s), ctypes.byref(g)))
    return g


def ngs_build_graph_refresh(ctx: int, s: ngs_splats, prev_ptr: int, n_old: int, k_old: int,
                            pairs_ptr: int, n_pairs: int):
    g = ngs_graph()
    nq = ctypes.c_int64(0)
    _check(load().ngs_build_graph_refresh(_P(ctx), ctypes.byref(s), _P(prev_ptr), n_old, k_old,
                                          _P(pairs_ptr), n_pairs, ctypes.byref(g),
                                          ctypes.byref(nq)))
    return g, nq.value


def ngs_edge_costs(ctx: int, s: ngs_splats, g: ngs_graph, pass_index: int, cost_ptr: int):
    _check(load().ngs_edge_costs(_P(ctx), ctypes.byref(s), ctypes.byref(g), pass_index,
                                 _P(cost_ptr)))


def ngs_select_pairs(ctx: int, g: ngs_graph, cost_ptr: int, max_pairs: int,
                     pairs_ptr: int) -> int:
    n = ctypes.c_int64(0)
    _check(load().ngs_select_pairs(_P(ctx), ctypes.byref(g), _P(cost_ptr), max_pairs,
                                   _P(pairs_ptr), ctypes.byref(n)))
    return n.value


def ngs_merge_compact(ctx: int, s: ngs_splats, pairs_ptr: int, n_pairs: int) -> int:
    _check(load().ngs_merge_compact(_P(ctx), ctypes.byref(s), _P(pairs_ptr), n_pairs))
    return s.n


def ngs_simplify(ctx: int, s: ngs_splats, target: int) -> dict:
    st = ngs_stats()
    _check(load().ngs_simplify(_P(ctx), ctypes.byref(s), target, ctypes.byref(st)))
    return st.as_dict()


def ngs_batch_simplify(ctx: int, scenes, targets) -> dict:
    """scenes: list of ngs_splats (updated in place), targets: list of ints."""
    n = len(scenes)
    arr = (ngs_splats * max(1, n))(*scenes)
    tg = (ctypes.c_int64 * max(1, n))(*[int(t) for t in targets])
    st = ngs_stats()
    _check(load().ngs_batch_simplify(_P(ctx), arr, tg, n, ctypes.byref(st)))
    for i in range(n):
        scenes[i].n = arr[i].n
    return st.as_dict()


def ngs_simplify_host(ctx: int, s: ngs_splats, target: int) -> dict:
    st = ngs_stats()
    _check(load().ngs_simplify_host(_P(ctx), ctypes.byref(s), target, ctypes.byref(st)))
    return st.as_dict()


def ngs_knn_noalloc(xyz_ptr: int, n: int, k: int, nbr_ptr: int, stream=None):
    """Directed kNN table into caller-owned memory without any allocation."""
    s = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
    _check(load().ngs_knn_noalloc(_P(xyz_ptr), n, k, _P(nbr_ptr), _P(s)))


def ngs_profile_enable(ctx: int, enable: bool):
    _check(load().ngs_profile_enable(_P(ctx), int(enable)))


def ngs_profile(ctx: int) -> list:
    """[(name, launches, ms)] accumulated since the last reset."""
    L = load()
    out = []
    for i in range(L.ngs_profile_count(_P(ctx))):
        name = ctypes.c_char_p()
        launches = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(L.ngs_profile_get(_P(ctx), i, ctypes.byref(name), ctypes.byref(launches),
                                 ctypes.byref(ms)))
        out.append((name.value.decode(), launches.value, ms.value))
    return out


def ngs_profile_reset(ctx: int):
    _check(load().ngs_profile_reset(_P(ctx)))


def ngs_launch_count(ctx: int) -> int:
    return int(load().ngs_launch_count(_P(ctx)))


# ---------------------------------------------------------------- tensor helpers

class DeviceSplats:
    """Splat arrays as contiguous FP32 tensors (device or pinned host)."""

    def __init__(self, xyz, log_scale, rot, logit, sh, n=None):
        self.xyz, self.log_scale, self.rot, self.logit, self.sh = xyz, log_scale, rot, logit, sh
        self.n = xyz.shape[0] if n is None else n

    @classmethod
    def from_numpy(cls, scene, device="cuda", pin=False):
        def t(a):
            x = torch.from_numpy(a).contiguous()
            if device == "cpu":
                return x.pin_memory() if pin else x
            return x.to(device)
        return cls(t(scene.xyz), t(scene.log_scale), t(scene.rot), t(scene.logit), t(scene.sh))

    def clone(self):
        return DeviceSplats(*(a.clone() for a in self.tensors()), n=self.n)

    def tensors(self):
        return (self.xyz, self.log_scale, self.rot, self.logit, self.sh)

    def struct(self) -> ngs_splats:
        s = ngs_splats()
        s.xyz, s.log_scale, s.rot = self.xyz.data_ptr(), self.log_scale.data_ptr(), self.rot.data_ptr()
        s.opacity_logit, s.sh = self.logit.data_ptr(), self.sh.data_ptr()
        s.n = self.n
        s.cap = self.xyz.shape[0]
        s.sh_dim = self.sh.shape[1]
        return s

    def numpy(self):
        return tuple(a[:self.n].detach().cpu().numpy() for a in self.tensors())


class Context:
    """Owns one ngs_ctx bound to a torch stream."""

    def __init__(self, params: ngs_params | None = None, stream=None, **kw):
        p = params or ngs_default_params()
        for k, v in kw.items():
            setattr(p, k, v)
        self.params = p
        self.handle = ngs_create(p, stream)

    def close(self):
        if self.handle:
            ngs_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # step by step -------------------------------------------------------
    def prefilter(self, ds: DeviceSplats) -> int:
        s = ds.struct()
        ds.n = ngs_prefilter(self.handle, s)
        return ds.n

    def build_graph(self, ds: DeviceSplats):
        """Returns (graph struct, nbr [n,k_eff], edge_lo, edge_hi) as int32 tensor copies."""
        s = ds.struct()
        g = ngs_build_graph(self.handle, s)
        dev = ds.xyz.device
        nbr = _wrap_i32(g.nbr, g.n * g.k_eff, dev).view(g.n, g.k_eff).clone() if g.k_eff > 0 \
            else torch.zeros((g.n, 0), dtype=torch.int32, device=dev)
        lo = _wrap_i32(g.edge_lo, g.n_edges, dev).clone()
        hi = _wrap_i32(g.edge_hi, g.n_edges, dev).clone()
        return g, nbr, lo, hi

    def build_graph_refresh(self, ds: DeviceSplats, prev_nbr, pairs):
        """Local refresh (Sec. 3.4) after merging `pairs` (int32 [m, 2], old
        rows) into splats whose lists were `prev_nbr` (int32 [n_old, k_old]).
        Returns (graph struct, nbr, edge_lo, edge_hi, rows queried anew)."""
        s = ds.struct()
        prev = prev_nbr.contiguous()
        pr = pairs.contiguous()
        g, nq = ngs_build_graph_refresh(self.handle, s, prev.data_ptr(), prev.shape[0],
                                        prev.shape[1] if prev.dim() == 2 else 0,
                                        pr.data_ptr(), pr.shape[0])
        dev = ds.xyz.device
        nbr = _wrap_i32(g.nbr, g.n * g.k_eff, dev).view(g.n, g.k_eff).clone() if g.k_eff > 0 \
            else torch.zeros((g.n, 0), dtype=torch.int32, device=dev)
        lo = _wrap_i32(g.edge_lo, g.n_edges, dev).clone()
        hi = _wrap_i32(g.edge_hi, g.n_edges, dev).clone()
        return g, nbr, lo, hi, nq

    def edge_costs(self, ds: DeviceSplats, g: ngs_graph, pass_index: int = 0):
        cost = torch.empty(max(1, g.n_edges), dtype=torch.float32, device=ds.xyz.device)
        ngs_edge_costs(self.handle, ds.struct(), g, pass_index, cost.data_ptr())
        return cost[:g.n_edges]

    def select_pairs(self, g: ngs_graph, cost, max_pairs: int):
        pairs = torch.empty((max(1, max_pairs), 2), dtype=torch.int32, device=cost.device)
        n = ngs_select_pairs(self.handle, g, cost.data_ptr(), max_pairs, pairs.data_ptr())
        return pairs[:n]

    def merge_compact(self, ds: DeviceSplats, pairs) -> int:
        pairs = pairs.contiguous()
        s = ds.struct()
        ds.n = ngs_merge_compact(self.handle, s, pairs.data_ptr(), pairs.shape[0])
        return ds.n

    def simplify(self, ds: DeviceSplats, target: int) -> dict:
        s = ds.struct()
        st = ngs_simplify(self.handle, s, target)
        ds.n = s.n
        return st

    def tuning(self) -> dict:
        t = ngs_tuning()
        _check(load().ngs_get_tuning(_P(self.handle), ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = ngs_tuning()
        _check(load().ngs_get_tuning(_P(self.handle), ctypes.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        _check(load().ngs_set_tuning(_P(self.handle), ctypes.byref(t)))

    def autotune(self, sample: DeviceSplats):
        """Measure the candidate tunings on `sample`; returns (tuning dict, ms)."""
        t, ms = ngs_tuning(), ctypes.c_double()
        s = sample.struct()
        _check(load().ngs_autotune(_P(self.handle), ctypes.byref(s), ctypes.byref(t),
                                   ctypes.byref(ms)))
        return t.as_dict(), ms.value

    def batch_simplify(self, scenes, targets) -> dict:
        """Simplify several DeviceSplats in one call (each in place)."""
        structs = [ds.struct() for ds in scenes]
        st = ngs_batch_simplify(self.handle, structs, targets)
        for ds, s in zip(scenes, structs):
            ds.n = s.n
        return st

    def selftest_ff(self, op: int, x, y=None):
        """Float-float arithmetic of the refined edge costs on host float64
        arrays (ngs_selftest_ff); returns the results widened to float64."""
        import numpy as np
        x = np.ascontiguousarray(x, dtype=np.float64)
        yy = None if y is None else np.ascontiguousarray(y, dtype=np.float64)
        out = np.empty_like(x)
        _check(load().ngs_selftest_ff(_P(self.handle), op, x.ctypes.data,
                                      None if yy is None else yy.ctypes.data, x.size,
                                      out.ctypes.data))
        return out

    def simplify_host(self, hs: DeviceSplats, target: int) -> dict:
        s = hs.struct()
        st = ngs_simplify_host(self.handle, s, target)
        hs.n = s.n
        return st


class _DevArray:
    """Minimal __cuda_array_interface__ view of a ctx-owned int32 device array."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<i4",
                                         "data": (ptr, False), "version": 3, "strides": None}


def _wrap_i32(ptr, count, device):
    """Copy `count` int32 values from a ctx-owned device pointer into a new tensor."""
    if count <= 0 or not ptr:
        return torch.zeros(0, dtype=torch.int32, device=device)
    return torch.as_tensor(_DevArray(ptr, count), device=device).clone()


# ---------------------------------------------------------------- serving form
def ngs_default_tuning() -> ngs_tuning:
    t = ngs_tuning()
    load().ngs_default_tuning(ctypes.byref(t))
    return t


def ngs_server_default_config() -> ngs_server_config:
    c = ngs_server_config()
    load().ngs_server_default_config(ctypes.byref(c))
    return c


class Server:
    """Request loop of the serving form (see ngs_server_create)."""

    def __init__(self, params: ngs_params | None = None, **cfg):
        c = ngs_server_default_config()
        for k, v in cfg.items():
            setattr(c, k, v)
        self.config = c
        p = params or ngs_default_params()
        h = _P()
        _check(load().ngs_server_create(ctypes.byref(h), ctypes.byref(p), ctypes.byref(c)))
        self.handle = h.value

    def close(self):
        if self.handle:
            load().ngs_server_destroy(_P(self.handle))
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, s: ngs_splats, target: int) -> int:
        jid = ctypes.c_uint64()
        _check(load().ngs_serve_submit(_P(self.handle), ctypes.byref(s), target,
                                       ctypes.byref(jid)))
        return jid.value

    def poll(self, jid: int):
        done, n = ctypes.c_int(), ctypes.c_int64()
        _check(load().ngs_serve_poll(_P(self.handle), jid, ctypes.byref(done), ctypes.byref(n)))
        return bool(done.value), n.value

    def wait(self, jid: int, timeout_s: float = 600.0) -> int:
        n = ctypes.c_int64()
        _check(load().ngs_serve_wait(_P(self.handle), jid, timeout_s, ctypes.byref(n)))
        return n.value

    def info(self, jid: int) -> dict:
        i = ngs_job_info()
        _check(load().ngs_serve_info(_P(self.handle), jid, ctypes.byref(i)))
        return i.as_dict()

    def stats(self) -> dict:
        st = ngs_server_stats()
        _check(load().ngs_server_get_stats(_P(self.handle), ctypes.byref(st)))
        return st.as_dict()

    def clock(self) -> float:
        return load().ngs_server_clock(_P(self.handle))

    def replay(self, jobs, targets, arrivals):
        """jobs: list of ngs_splats; returns the job ids (raises on a submit error)."""
        n = len(jobs)
        arr = (ngs_splats * max(1, n))(*jobs)
        tg = (ctypes.c_int64 * max(1, n))(*[int(t) for t in targets])
        at = (ctypes.c_double * max(1, n))(*[float(a) for a in arrivals])
        ids = (ctypes.c_uint64 * max(1, n))()
        _check(load().ngs_serve_replay(_P(self.handle), arr, tg, at, n, ids))
        return list(ids[:n])
