"""GB300 PSCTL solver: k-clique densest subgraph search by Frank-Wolfe over
the succinct clique tree (arxiv 2403.05775).

This package is a thin ctypes binding of ``libkdss.so`` (``include/kdss.h``):
the Python functions carry the C entry points' names and only marshal
arguments.  Every step of the path -- CSR build, peeling, SCT build, PBUpdate
iterations, extraction -- runs in the library's CUDA kernels.  PyTorch, when
present, supplies the CUDA stream and the device memory (its caching
allocator); without it the library allocates stream-ordered memory itself.
There is no CPU fallback: without the built library every call raises.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build_ext

KDSS_OK = 0
KDSS_ERR_INVALID_ARG = -1
KDSS_ERR_BAD_GRAPH = -2
KDSS_ERR_OOM = -3
KDSS_ERR_OVERFLOW = -4
KDSS_ERR_TIMEOUT = -5
KDSS_ERR_CUDA = -6
KDSS_ERR_CANCELLED = -7
KDSS_ERR_UNSUPPORTED = -8

KDSS_INT64 = 0
KDSS_FP64 = 1
KDSS_FP32K = 2
KDSS_RULE_DEFAULT = 0
KDSS_RULE_INTEGER = 1
KDSS_RULE_CONTINUOUS = 2
KDSS_ORDER_PEEL = 0
KDSS_ORDER_CORE = 1
KDSS_FLAG_PROFILE = 1
KDSS_FLAG_KEEP_GRAPH = 2
KDSS_FLAG_ASYNC = 4
KDSS_FLAG_TEST_BARRIER_TIMEOUT = 8
KDSS_FLAG_ROOTED = 16
KDSS_FLAG_PER_ITERATION = 32

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class kdss_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("order", C.c_int32), ("flags", C.c_uint32),
                ("check_every", C.c_int32), ("eps_stop", C.c_double), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
                ("chunk", C.c_int32), ("threads_per_path", C.c_int32), ("rule", C.c_int32)]


class kdss_batch_tuning(C.Structure):
    _fields_ = [("chunk", C.c_int32), ("threads_per_path", C.c_int32), ("autotuned", C.c_int32),
                ("ntried", C.c_int32), ("tried_chunk", C.c_int32 * 8),
                ("tried_threads_per_path", C.c_int32 * 8), ("tried_ms", C.c_float * 8)]


class kdss_graph_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("src", C.c_void_p), ("dst", C.c_void_p),
                ("on_device", C.c_int32)]


class kdss_sct_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("eta_k", C.c_int64), ("L_k", C.c_int64),
                ("c_k_lo", C.c_uint64), ("c_k_hi", C.c_uint64), ("k", C.c_int32),
                ("degeneracy", C.c_int32), ("max_out_degree", C.c_int32),
                ("max_pair_len", C.c_int32), ("device_bytes", C.c_int64),
                ("pairs_per_class", C.c_int64 * 8)]


class kdss_sct_count_stats(C.Structure):
    _fields_ = [("eta_k", C.c_int64), ("L_k", C.c_int64), ("c_k_lo", C.c_uint64),
                ("c_k_hi", C.c_uint64), ("pairs_per_class", C.c_int64 * 8),
                ("roots_total", C.c_int64), ("roots_done", C.c_int64), ("roots_cut", C.c_int64),
                ("cut_pairs", C.c_int64), ("cut_nodes", C.c_int64), ("m", C.c_int64),
                ("complete", C.c_int32), ("max_pair_len", C.c_int32), ("degeneracy", C.c_int32),
                ("max_out_degree", C.c_int32), ("count_bits", C.c_int32), ("reserved", C.c_int32),
                ("seconds", C.c_double)]


class kdss_result(C.Structure):
    _fields_ = [("istar", C.c_int64), ("ids", C.POINTER(C.c_int32)), ("count_lo", C.c_uint64),
                ("count_hi", C.c_uint64), ("density", C.c_double), ("upper_bound", C.c_double),
                ("rho_prime", C.c_double), ("gap", C.c_double), ("T", C.c_int32),
                ("t_used", C.c_int32), ("status", C.c_int32), ("reserved", C.c_int32)]


class kdss_server_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("order", C.c_int32), ("check_every", C.c_int32),
                ("max_active", C.c_int32), ("eps_stop", C.c_double), ("hbm_budget", C.c_int64),
                ("flags", C.c_uint32), ("reserved", C.c_int32)]


class kdss_query_timing(C.Structure):
    _fields_ = [("queue_ms", C.c_double), ("build_ms", C.c_double), ("wait_ms", C.c_double),
                ("iterate_ms", C.c_double), ("latency_ms", C.c_double), ("iterations", C.c_int32),
                ("peak_batch", C.c_int32), ("resident_bytes", C.c_int64)]


class kdss_server_stats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("submitted", "completed", "failed", "pending", "active",
                                        "resident_bytes", "peak_resident_bytes", "hbm_budget",
                                        "replays", "captures")] + \
               [("peak_active", C.c_int32), ("reserved", C.c_int32)]


class kdss_cpsample_stats(C.Structure):
    _fields_ = [("paths_total", C.c_uint64), ("samples", C.c_int64), ("samples_clique", C.c_int64),
                ("cliques", C.c_int64), ("colors", C.c_int32), ("reserved", C.c_int32)]


class kdss_timing(C.Structure):
    _fields_ = [("fw_kernel_ms", C.c_double), ("step_kernel_ms", C.c_double),
                ("fw_launches", C.c_int64), ("step_launches", C.c_int64)]


class kdss_query(C.Structure):
    _fields_ = [("graph", kdss_graph_desc), ("k", C.c_int32), ("T", C.c_int32)]


class KdssError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"kdss error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return build_ext.LIB


def load(build_if_missing: bool = False):
    """Load libkdss.so.  Raises when the library is not built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build_ext.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(
                    "libkdss.so is not built; run __graft_entry__.build() "
                    "(the solver has no CPU fallback)")
            build_ext.build()
        L = C.CDLL(path)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        P = C.POINTER
        sig = {
            "kdss_build_sct": (i32, [P(kdss_graph_desc), i32, P(kdss_opts), P(vp)]),
            "kdss_sct_from_pairs": (i32, [i64, i32, i64, vp, vp, vp, i32, P(kdss_opts), P(vp)]),
            "kdss_solve_streamed": (i32, [P(kdss_graph_desc), i32, i32, i32, P(kdss_opts),
                                          P(kdss_result)]),
            "kdss_sct_count": (i32, [P(kdss_graph_desc), i32, C.c_double, P(kdss_opts),
                                     P(kdss_sct_count_stats)]),
            "kdss_sct_info": (i32, [vp, P(kdss_sct_stats)]),
            "kdss_sct_copy_pairs": (i32, [vp, vp, vp, vp]),
            "kdss_sct_copy_graph": (i32, [vp, vp, vp, vp, vp, vp]),
            "kdss_fw_iterate": (i32, [vp, P(vp), i32, P(kdss_opts)]),
            "kdss_fw_iterate_at": (i32, [vp, i32, P(vp), i32, P(kdss_opts)]),
            "kdss_state_copy_r": (i32, [vp, vp, P(i32)]),
            "kdss_state_timing": (i32, [vp, P(kdss_timing)]),
            "kdss_extract": (i32, [vp, vp, P(kdss_opts), P(kdss_result)]),
            "kdss_solve": (i32, [P(kdss_graph_desc), i32, i32, P(kdss_opts), P(kdss_result)]),
            "kdss_solve_batch": (i32, [P(kdss_query), i32, P(kdss_result), P(kdss_opts)]),
            "kdss_sct_free": (None, [vp]),
            "kdss_state_free": (None, [vp]),
            "kdss_result_free": (None, [P(kdss_result)]),
            "kdss_last_error": (C.c_char_p, []),
            "kdss_version": (C.c_char_p, []),
            "kdss_kernel_launches": (i64, []),
            "kdss_batch_last_tuning": (i32, [P(kdss_batch_tuning)]),
            "kdss_fw_iterate_noalloc": (i32, [vp, vp, i32, i32, vp]),
            "kdss_fw_cliques": (i32, [vp, P(vp), i32, P(kdss_opts)]),
            "kdss_build_sct_multi": (i32, [P(kdss_graph_desc), i32, P(kdss_opts), P(vp)]),
            "kdss_sct_restrict": (i32, [vp, i32, P(kdss_opts), P(vp)]),
            "kdss_sct_share_prefixes": (i32, [vp, i64, P(kdss_opts), P(vp)]),
            "kdss_sct_shared_words": (i32, [vp, P(i64), P(i64)]),
            "kdss_cpsample": (i32, [P(kdss_graph_desc), i32, i64, i32, C.c_uint64, P(kdss_opts),
                                    P(kdss_result), P(kdss_cpsample_stats)]),
            "kdss_sct_copy_cliques": (i32, [vp, vp, i64, P(i64)]),
            "kdss_server_create": (i32, [P(kdss_server_opts), P(vp)]),
            "kdss_server_submit": (i32, [vp, P(kdss_query), P(i64)]),
            "kdss_server_wait": (i32, [vp, i64, i32, P(kdss_result), P(kdss_query_timing)]),
            "kdss_server_get_stats": (i32, [vp, P(kdss_server_stats)]),
            "kdss_server_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(rc):
    if rc != KDSS_OK:
        msg = load().kdss_last_error()
        raise KdssError(rc, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# torch plumbing: stream and caching allocator
# ---------------------------------------------------------------------------

def _torch():
    try:
        import torch
        return torch if torch.cuda.is_available() else None
    except Exception:  # pragma: no cover - torch is optional
        return None


_torch_api = {}


def _torch_alloc(size, stream, ctx):
    try:
        return _torch_api["alloc"](int(size), stream=int(stream or 0))
    except Exception:  # reported to the library as a failed allocation
        return None


def _torch_free(ptr, size, stream, ctx):
    try:
        _torch_api["free"](int(ptr))
    except Exception:  # interpreter shutdown: the process releases the memory
        pass


_ALLOC_CB = ALLOC_FN(_torch_alloc)
_FREE_CB = FREE_FN(_torch_free)


def make_opts(precision=KDSS_INT64, order=KDSS_ORDER_PEEL, flags=0, stream=None,
              allocator="torch", check_every=0, eps_stop=0.0, chunk=0,
              threads_per_path=0, rule=KDSS_RULE_DEFAULT) -> kdss_opts:
    """Build a kdss_opts.  stream: a torch.cuda.Stream, a raw cudaStream_t
    (int) or None (torch's current stream when torch is present).
    allocator: 'torch' (caching allocator) or 'library' (cudaMallocAsync).
    rule: KDSS_RULE_DEFAULT (the precision's rule), KDSS_RULE_INTEGER or
    KDSS_RULE_CONTINUOUS (checked against the precision by the library)."""
    o = kdss_opts()
    o.precision, o.order, o.flags, o.rule = precision, order, flags, int(rule)
    o.check_every, o.eps_stop = check_every, eps_stop
    o.chunk, o.threads_per_path = int(chunk), int(threads_per_path)
    t = _torch()
    if stream is None and t is not None:
        stream = t.cuda.current_stream()
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    o.stream = stream or None
    if allocator == "torch" and t is not None:
        _torch_api.setdefault("alloc", t.cuda.caching_allocator_alloc)
        _torch_api.setdefault("free", t.cuda.caching_allocator_delete)
        o.alloc, o.free = _ALLOC_CB, _FREE_CB
    elif allocator not in ("torch", "library"):
        raise ValueError(allocator)
    return o


def _is_cuda_tensor(a):
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _graph_desc(n, src, dst):
    """Host arrays (numpy, lists or CPU tensors; copied by the library), or
    CUDA int32 tensors on the current device (read in place, on_device)."""
    g = kdss_graph_desc()
    g.n = int(n)
    keep = []
    if _is_cuda_tensor(src) or _is_cuda_tensor(dst):
        for a in (src, dst):
            if not _is_cuda_tensor(a) or str(a.dtype) != "torch.int32" or not a.is_contiguous():
                raise ValueError("device edge arrays: src and dst must both be contiguous "
                                 "CUDA int32 tensors")
        if src.numel() != dst.numel():
            raise ValueError("src and dst differ in length")
        import torch
        if src.device != dst.device or src.device.index != torch.cuda.current_device():
            raise ValueError("src and dst must be on the current CUDA device")
        g.m = src.numel()
        g.src, g.dst, g.on_device = src.data_ptr(), dst.data_ptr(), 1
        keep = [src, dst]
    else:
        # CPU tensors take the host path
        src = src.numpy() if hasattr(src, "data_ptr") else src
        dst = dst.numpy() if hasattr(dst, "data_ptr") else dst
        s = np.ascontiguousarray(src, np.int32)
        d = np.ascontiguousarray(dst, np.int32)
        if s.shape != d.shape:
            raise ValueError("src and dst differ in length")
        g.m = s.size
        g.src, g.dst, g.on_device = s.ctypes.data, d.ctypes.data, 0
        keep = [s, d]
    return g, keep


class Sct:
    """Owning wrapper of a kdss_sct* handle."""

    def __init__(self, ptr):
        self.ptr = C.c_void_p(ptr)

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value and _lib is not None:
            _lib.kdss_sct_free(self.ptr)
            self.ptr = C.c_void_p(None)

    free = __del__


class State:
    """Owning wrapper of a kdss_state* handle."""

    def __init__(self, ptr):
        self.ptr = C.c_void_p(ptr)

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value and _lib is not None:
            _lib.kdss_state_free(self.ptr)
            self.ptr = C.c_void_p(None)

    free = __del__


def _result_dict(r: kdss_result):
    ids = np.ctypeslib.as_array(r.ids, shape=(r.istar,)).copy() if r.istar > 0 and r.ids else \
        np.zeros(0, np.int32)
    return dict(istar=int(r.istar), ids=ids, count=int(r.count_lo) | (int(r.count_hi) << 64),
                density=r.density, upper_bound=r.upper_bound, rho_prime=r.rho_prime,
                gap=r.gap, T=int(r.T), t_used=int(r.t_used), status=int(r.status))


# ---------------------------------------------------------------------------
# entry points (names of include/kdss.h)
# ---------------------------------------------------------------------------

def kdss_build_sct(n, src, dst, k, opts: kdss_opts | None = None) -> Sct:
    L = load()
    g, keep = _graph_desc(n, src, dst)
    out = C.c_void_p()
    _check(L.kdss_build_sct(C.byref(g), int(k), C.byref(opts or make_opts()), C.byref(out)))
    del keep
    return Sct(out.value)


def kdss_build_sct_multi(n, src, dst, k_max, opts: kdss_opts | None = None) -> Sct:
    """A k-agnostic SCT (every pair with |V_h| <= k_max), to be restricted."""
    L = load()
    g, keep = _graph_desc(n, src, dst)
    out = C.c_void_p()
    _check(L.kdss_build_sct_multi(C.byref(g), int(k_max), C.byref(opts or make_opts()), C.byref(out)))
    del keep
    return Sct(out.value)


def kdss_sct_restrict(multi: Sct, k, opts: kdss_opts | None = None) -> Sct:
    """P_k of a k-agnostic SCT as an ordinary SCT handle."""
    out = C.c_void_p()
    _check(load().kdss_sct_restrict(multi.ptr, int(k), C.byref(opts or make_opts()), C.byref(out)))
    return Sct(out.value)


def kdss_sct_share_prefixes(s: Sct, chunk_pairs: int = 0, opts: kdss_opts | None = None) -> Sct:
    """The prefix-shared form of an SCT's pairs as a new handle."""
    out = C.c_void_p()
    _check(load().kdss_sct_share_prefixes(s.ptr, int(chunk_pairs), C.byref(opts or make_opts()),
                                          C.byref(out)))
    return Sct(out.value)


def kdss_sct_shared_words(s: Sct) -> dict:
    """Node words kept by a prefix-shared SCT and the chunks an iteration decodes."""
    w, ch = C.c_int64(0), C.c_int64(0)
    _check(load().kdss_sct_shared_words(s.ptr, C.byref(w), C.byref(ch)))
    return {"words": w.value, "chunks": ch.value}


def kdss_sct_count(n, src, dst, k, budget_s=0.0, opts: kdss_opts | None = None) -> dict:
    """Sizes of P_k from the count-only pass (nothing stored); see
    include/kdss.h for the sampling order when the budget cuts it short."""
    L = load()
    g, keep = _graph_desc(n, src, dst)
    st = kdss_sct_count_stats()
    _check(L.kdss_sct_count(C.byref(g), int(k), float(budget_s), C.byref(opts or make_opts()),
                            C.byref(st)))
    del keep
    d = {f: getattr(st, f) for f, _ in kdss_sct_count_stats._fields_ if f != "pairs_per_class"}
    d["pairs_per_class"] = list(st.pairs_per_class)[:6]
    d["c_k"] = int(st.c_k_lo) | (int(st.c_k_hi) << 64)
    return d


def kdss_sct_from_pairs(n, k, pair_off, nodes, h, opts: kdss_opts | None = None) -> Sct:
    po = np.ascontiguousarray(pair_off, np.int64)
    nd = np.ascontiguousarray(nodes, np.int32)
    hh = np.ascontiguousarray(h, np.int32)
    if po.size != hh.size + 1 or po[0] != 0 or int(po[-1]) != nd.size:
        raise ValueError("pair_off must hold len(h) + 1 offsets from 0 to len(nodes)")
    L = load()
    out = C.c_void_p()
    _check(L.kdss_sct_from_pairs(int(n), int(k), hh.size, po.ctypes.data, nd.ctypes.data,
                                 hh.ctypes.data, 0, C.byref(opts or make_opts()), C.byref(out)))
    return Sct(out.value)


def kdss_sct_info(s: Sct) -> dict:
    st = kdss_sct_stats()
    _check(load().kdss_sct_info(s.ptr, C.byref(st)))
    d = {f: getattr(st, f) for f, _ in kdss_sct_stats._fields_ if f != "pairs_per_class"}
    d["pairs_per_class"] = list(st.pairs_per_class)[:5]
    d["c_k"] = int(st.c_k_lo) | (int(st.c_k_hi) << 64)
    return d


def kdss_sct_copy_pairs(s: Sct) -> dict:
    info = kdss_sct_info(s)
    po = np.zeros(info["eta_k"] + 1, np.int64)
    nodes = np.zeros(info["L_k"], np.int32)
    h = np.zeros(info["eta_k"], np.int32)
    _check(load().kdss_sct_copy_pairs(s.ptr, po.ctypes.data, nodes.ctypes.data, h.ctypes.data))
    return dict(pair_off=po, nodes=nodes, h=h)


def kdss_sct_copy_graph(s: Sct) -> dict:
    info = kdss_sct_info(s)
    n, m = info["n"], info["m"]
    out = dict(off=np.zeros(n + 1, np.int64), adj=np.zeros(2 * m, np.int32),
               core=np.zeros(n, np.int32), round=np.zeros(n, np.int32),
               rank=np.zeros(n, np.int32))
    _check(load().kdss_sct_copy_graph(s.ptr, out["off"].ctypes.data, out["adj"].ctypes.data,
                                      out["core"].ctypes.data, out["round"].ctypes.data,
                                      out["rank"].ctypes.data))
    return out


def kdss_fw_iterate_at(s: Sct, k: int, state: State | None, T: int,
                       opts: kdss_opts | None = None) -> State:
    """kdss_fw_iterate over P_k of a k-agnostic SCT (pairs outside P_k
    skipped by the kernels)."""
    L = load()
    p = C.c_void_p(state.ptr.value if state is not None else None)
    _check(L.kdss_fw_iterate_at(s.ptr, int(k), C.byref(p), int(T), C.byref(opts or make_opts())))
    if state is None:
        return State(p.value)
    return state


def kdss_fw_iterate(s: Sct, state: State | None, T: int, opts: kdss_opts | None = None) -> State:
    L = load()
    p = C.c_void_p(state.ptr.value if state is not None else None)
    _check(L.kdss_fw_iterate(s.ptr, C.byref(p), int(T), C.byref(opts or make_opts())))
    if state is None:
        return State(p.value)
    return state


def kdss_fw_cliques(s: Sct, state: State | None, T: int, opts: kdss_opts | None = None) -> State:
    """Alg. 1 over the explicit k-clique list (expanded from the SCT)."""
    L = load()
    p = C.c_void_p(state.ptr.value if state is not None else None)
    _check(L.kdss_fw_cliques(s.ptr, C.byref(p), int(T), C.byref(opts or make_opts())))
    if state is None:
        return State(p.value)
    return state


def kdss_cpsample(n, src, dst, k, t, T, seed, opts: kdss_opts | None = None) -> dict:
    """CPSample (Alg. 4): sampled k-color paths, Alg. 1 over the sampled
    cliques, sampled-density prefix.  Returns the result dict with 'stats'."""
    L = load()
    g, keep = _graph_desc(n, src, dst)
    r = kdss_result()
    st = kdss_cpsample_stats()
    rc = L.kdss_cpsample(C.byref(g), int(k), int(t), int(T), int(seed) & 0xFFFFFFFFFFFFFFFF,
                         C.byref(opts or make_opts()), C.byref(r), C.byref(st))
    try:
        _check(rc)
        out = _result_dict(r)
        out["stats"] = {f: getattr(st, f) for f, _ in kdss_cpsample_stats._fields_ if f != "reserved"}
        return out
    finally:
        L.kdss_result_free(C.byref(r))
        del keep


def kdss_sct_copy_cliques(s: Sct) -> np.ndarray:
    """The explicit k-clique list as a (c_k, k) int32 array."""
    L = load()
    cnt = C.c_int64()
    _check(L.kdss_sct_copy_cliques(s.ptr, None, 0, C.byref(cnt)))
    k = kdss_sct_info(s)["k"]
    out = np.zeros((cnt.value, k), np.int32)
    if cnt.value:
        _check(L.kdss_sct_copy_cliques(s.ptr, out.ctypes.data, cnt.value, C.byref(cnt)))
    return out


def kdss_state_copy_r(st: State, n: int, precision: int):
    dt = np.float32 if precision == KDSS_FP32K else (np.float64 if precision == KDSS_FP64 else np.uint64)
    r = np.zeros(n, dt)
    t = C.c_int32()
    _check(load().kdss_state_copy_r(st.ptr, r.ctypes.data, C.byref(t)))
    return r, int(t.value)


def kdss_state_timing(st: State) -> dict:
    tm = kdss_timing()
    _check(load().kdss_state_timing(st.ptr, C.byref(tm)))
    return {f: getattr(tm, f) for f, _ in kdss_timing._fields_}


def kdss_extract(s: Sct, st: State, opts: kdss_opts | None = None) -> dict:
    L = load()
    r = kdss_result()
    _check(L.kdss_extract(s.ptr, st.ptr, C.byref(opts or make_opts()), C.byref(r)))
    try:
        return _result_dict(r)
    finally:
        L.kdss_result_free(C.byref(r))


def kdss_solve_streamed(n, src, dst, k, T, nchunks, opts: kdss_opts | None = None) -> dict:
    """kdss_solve with the SCT rebuilt root range by root range inside every
    iteration (for SCTs that do not fit the device)."""
    L = load()
    g, keep = _graph_desc(n, src, dst)
    r = kdss_result()
    rc = L.kdss_solve_streamed(C.byref(g), int(k), int(T), int(nchunks),
                               C.byref(opts or make_opts()), C.byref(r))
    try:
        _check(rc)
        return _result_dict(r)
    finally:
        L.kdss_result_free(C.byref(r))
        del keep


def kdss_solve(n, src, dst, k, T, opts: kdss_opts | None = None) -> dict:
    L = load()
    g, keep = _graph_desc(n, src, dst)
    r = kdss_result()
    rc = L.kdss_solve(C.byref(g), int(k), int(T), C.byref(opts or make_opts()), C.byref(r))
    try:
        _check(rc)
        return _result_dict(r)
    finally:
        L.kdss_result_free(C.byref(r))
        del keep


def kdss_solve_batch(queries, opts: kdss_opts | None = None) -> list:
    """queries: list of (n, src, dst, k, T).  Returns one dict per query
    (with its status; failed queries carry no result)."""
    L = load()
    nq = len(queries)
    arr = (kdss_query * max(nq, 1))()
    keep = []
    for i, (n, src, dst, k, T) in enumerate(queries):
        g, kp = _graph_desc(n, src, dst)
        keep.append(kp)
        arr[i].graph, arr[i].k, arr[i].T = g, int(k), int(T)
    res = (kdss_result * max(nq, 1))()
    rc = L.kdss_solve_batch(arr, nq, res, C.byref(opts or make_opts()))
    out = []
    try:
        for i in range(nq):
            out.append(_result_dict(res[i]))
    finally:
        for i in range(nq):
            L.kdss_result_free(C.byref(res[i]))
    if rc != KDSS_OK and all(o["status"] != KDSS_OK for o in out):
        _check(rc)
    return out


def kdss_batch_last_tuning() -> dict:
    """The work-queue configuration of this thread's last kdss_solve_batch and
    the candidates its autotuner timed."""
    t = kdss_batch_tuning()
    _check(load().kdss_batch_last_tuning(C.byref(t)))
    n = t.ntried
    return {"chunk": t.chunk, "threads_per_path": t.threads_per_path,
            "autotuned": bool(t.autotuned),
            "tried": [{"chunk": t.tried_chunk[i], "threads_per_path": t.tried_threads_per_path[i],
                       "ms": float(t.tried_ms[i])} for i in range(n)]}


def kdss_version() -> str:
    return load().kdss_version().decode()


def kdss_kernel_launches() -> int:
    return int(load().kdss_kernel_launches())


def kdss_fw_iterate_noalloc(s: Sct, r_dev, t_done: int, T: int, stream=None) -> None:
    """Rule-I FW iterations on a caller-owned device vector r (n uint64
    values, given as a CUDA tensor of 8-byte elements or a raw device
    pointer), using only the library's fixed scratch area -- for callers that
    cannot allocate device memory while they iterate."""
    if hasattr(r_dev, "data_ptr"):
        n = kdss_sct_info(s)["n"]
        if not getattr(r_dev, "is_cuda", False):
            raise KdssError(KDSS_ERR_INVALID_ARG, "r must be a CUDA tensor")
        if r_dev.element_size() != 8 or not r_dev.is_contiguous():
            raise KdssError(KDSS_ERR_INVALID_ARG, "r must be contiguous with 8-byte elements")
        if r_dev.numel() < n:
            raise KdssError(KDSS_ERR_INVALID_ARG, f"r holds {r_dev.numel()} values, the SCT has n = {n}")
        ptr = r_dev.data_ptr()
    else:
        ptr = int(r_dev)   # a raw device pointer: the library checks where it points
    if stream is None:
        t = _torch()
        stream = t.cuda.current_stream() if t is not None else None
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(load().kdss_fw_iterate_noalloc(s.ptr, C.c_void_p(ptr), int(t_done), int(T),
                                          C.c_void_p(stream or None)))


# ---------------------------------------------------------------------------
# query server (include/kdss_server.h)
# ---------------------------------------------------------------------------

class Server:
    """Continuous-batching server: submit() queues a query and returns its
    ticket, wait() returns the result dict with a ``timing`` entry."""

    def __init__(self, precision=KDSS_INT64, order=KDSS_ORDER_PEEL, check_every=5,
                 eps_stop=0.0, max_active=0, hbm_budget=0, flags=0):
        L = load()
        o = kdss_server_opts(precision=precision, order=order, check_every=check_every,
                             max_active=max_active, eps_stop=eps_stop, hbm_budget=int(hbm_budget),
                             flags=int(flags))
        p = C.c_void_p()
        _check(L.kdss_server_create(C.byref(o), C.byref(p)))
        self.ptr = p

    def submit(self, n, src, dst, k, T) -> int:
        g, keep = _graph_desc(n, src, dst)
        q = kdss_query()
        q.graph, q.k, q.T = g, int(k), int(T)
        t = C.c_int64()
        _check(load().kdss_server_submit(self.ptr, C.byref(q), C.byref(t)))
        del keep          # the server copied the edge list
        return int(t.value)

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        L = load()
        r = kdss_result()
        tm = kdss_query_timing()
        rc = L.kdss_server_wait(self.ptr, int(ticket), int(timeout_ms), C.byref(r), C.byref(tm))
        if rc == KDSS_ERR_TIMEOUT or rc == KDSS_ERR_INVALID_ARG:
            _check(rc)
        try:
            out = _result_dict(r)
        finally:
            L.kdss_result_free(C.byref(r))
        out["status"] = int(rc)
        out["message"] = (L.kdss_last_error() or b"").decode()
        out["timing"] = {f: getattr(tm, f) for f, _ in kdss_query_timing._fields_}
        return out

    def stats(self) -> dict:
        st = kdss_server_stats()
        _check(load().kdss_server_get_stats(self.ptr, C.byref(st)))
        return {f: getattr(st, f) for f, _ in kdss_server_stats._fields_ if f != "reserved"}

    def close(self):
        if self.ptr:
            load().kdss_server_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
