"""CPU oracle for PSCTL (arxiv 2403.05775) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded C implementation (``kdss_oracle.c``) of what
the GPU solver computes, loaded through ctypes.  Only the test suite, the smoke
check of ``__graft_entry__`` and the benchmark's CPU-baseline leg may import
this package.  It shares no code with the CUDA solver: the two meet only in
the seeded input generators of ``synth``.

Each wrapper names the passage of the paper its C function restates; the
readings taken where the paper is silent are listed at the top of the C file.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "kdss_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libkdss_oracle.so")

_lock = threading.Lock()
_lib = None

i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build``."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC)):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"]
    try:   # host threads for orc_fw_sync_par; without OpenMP it runs serially
        subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            L.orc_free.argtypes = [C.c_void_p]
            L.orc_binom.restype = C.c_uint64
            L.orc_binom.argtypes = [C.c_int64, C.c_int64, C.POINTER(C.c_int)]
            L.orc_csr.restype = C.c_int
            L.orc_csr.argtypes = [C.c_int64, C.c_int64, i32p, i32p,
                                  C.POINTER(C.POINTER(C.c_int64)),
                                  C.POINTER(C.POINTER(C.c_int32)), C.POINTER(C.c_int64)]
            L.orc_peel.restype = C.c_int64
            L.orc_peel.argtypes = [C.c_int64, i64p, i32p, i32p, i32p]
            L.orc_order.argtypes = [C.c_int64, i32p, i32p, C.c_int, i32p, i32p]
            L.orc_list_cliques.restype = C.c_int64
            L.orc_list_cliques.argtypes = [C.c_int64, i64p, i32p, C.c_int, C.c_int64,
                                           C.POINTER(C.POINTER(C.c_int32))]
            L.orc_sct.restype = C.c_int64
            L.orc_sct.argtypes = [C.c_int64, i64p, i32p, i32p, i32p, C.c_int, C.c_int,
                                  C.POINTER(C.POINTER(C.c_int64)),
                                  C.POINTER(C.POINTER(C.c_int32)),
                                  C.POINTER(C.POINTER(C.c_int32)), C.POINTER(C.c_int64)]
            for nm in ("orc_pbupdate_alg3", "orc_pbupdate_greedy", "orc_pbupdate_level"):
                f = getattr(L, nm)
                f.restype = C.c_int
                f.argtypes = [C.c_int, i32p, u64p, C.c_int, C.c_int, u64p]
            L.orc_pbupdate_cont.restype = C.c_int
            L.orc_pbupdate_cont.argtypes = [C.c_int, i32p, f64p, C.c_int, C.c_int, f64p]
            for nm in ("orc_fw_sync", "orc_fw_seq"):
                f = getattr(L, nm)
                f.restype = C.c_int
                f.argtypes = [C.c_int64, C.c_int64, i64p, i32p, i32p, C.c_int, C.c_int, u64p]
            L.orc_fw_sync_par.restype = C.c_int
            L.orc_fw_sync_par.argtypes = [C.c_int64, C.c_int64, i64p, i32p, i32p, C.c_int,
                                          C.c_int, u64p, C.c_int]
            L.orc_fw_cont.restype = C.c_int
            L.orc_fw_cont.argtypes = [C.c_int64, C.c_int64, i64p, i32p, i32p, C.c_int,
                                      C.c_int, f64p]
            L.orc_binom128.restype = C.c_int
            L.orc_binom128.argtypes = [C.c_int64, C.c_int64, C.POINTER(C.c_uint64),
                                       C.POINTER(C.c_uint64)]
            L.orc_fw_cont_par.restype = C.c_int
            L.orc_fw_cont_par.argtypes = [C.c_int64, C.c_int64, i64p, i32p, i32p, C.c_int,
                                          C.c_int, f64p, C.c_int]
            L.orc_fw_cliques.argtypes = [C.c_int64, i32p, C.c_int, C.c_int, u64p]
            L.orc_fw_cliques_sync.restype = None
            L.orc_fw_cliques_sync.argtypes = [C.c_int64, C.c_int64, i32p, C.c_int, C.c_int, u64p]
            u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
            L.orc_color_greedy.restype = C.c_int
            L.orc_color_greedy.argtypes = [C.c_int64, i64p, i32p, i32p, i32p]
            L.orc_ccpath_dp.restype = C.c_int
            L.orc_ccpath_dp.argtypes = [C.c_int64, i64p, i32p, i32p, C.c_int, u64p]
            L.orc_ccpath_sample.restype = C.c_int
            L.orc_ccpath_sample.argtypes = [C.c_int64, i64p, i32p, i32p, C.c_int, u64p, C.c_int64,
                                            C.c_uint64, i32p, u8p, C.POINTER(C.c_uint64)]
            L.orc_sort_desc_u64.argtypes = [C.c_int64, u64p, i32p]
            L.orc_sort_desc_f64.argtypes = [C.c_int64, f64p, i32p]
            L.orc_prefix_counts_cliques.argtypes = [C.c_int64, i32p, C.c_int64, i32p,
                                                    C.c_int, u64p, u64p]
            L.orc_prefix_counts_pairs.restype = C.c_int
            L.orc_prefix_counts_pairs.argtypes = [C.c_int64, i32p, C.c_int64, i64p, i32p,
                                                  i32p, C.c_int, u64p, u64p, u64p, u64p]
            L.orc_argmax_density.restype = C.c_int64
            L.orc_argmax_density.argtypes = [C.c_int64, u64p, u64p]
            L.orc_brute_best.restype = C.c_int
            L.orc_brute_best.argtypes = [C.c_int, C.c_int64, u32p, u64p,
                                         C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                                         C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]
            _lib = L
    return _lib


def _take(ptr, count, dtype):
    if count == 0 or not ptr:
        if ptr:
            lib().orc_free(C.cast(ptr, C.c_void_p))
        return np.zeros(0, dtype=dtype)
    arr = np.ctypeslib.as_array(ptr, shape=(count,)).astype(dtype, copy=True)
    lib().orc_free(C.cast(ptr, C.c_void_p))
    return arr


def binom(a: int, b: int) -> int:
    """C(a, b) (Lemma 2.6 counts); raises when it needs more than 64 bits."""
    ovf = C.c_int(0)
    v = lib().orc_binom(a, b, C.byref(ovf))
    if ovf.value:
        raise OverflowError(f"C({a},{b}) exceeds 64 bits")
    return int(v)


def binom128(a: int, b: int) -> int:
    """C(a, b) exact in 128 bits; raises when it needs more."""
    lo, hi = C.c_uint64(0), C.c_uint64(0)
    if lib().orc_binom128(a, b, C.byref(lo), C.byref(hi)):
        raise OverflowError(f"C({a},{b}) exceeds 128 bits")
    return int(lo.value) | (int(hi.value) << 64)


# --------------------------------------------------------------------------
# A1-A2: graph, peeling, vertex order
# --------------------------------------------------------------------------

def csr(n: int, src, dst):
    """Simple undirected graph of Sec. 2 as CSR (off int64[n+1], adj int32)."""
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    po, pa, na = C.POINTER(C.c_int64)(), C.POINTER(C.c_int32)(), C.c_int64(0)
    rc = lib().orc_csr(n, src.size, src, dst, C.byref(po), C.byref(pa), C.byref(na))
    if rc != 0:
        raise ValueError(f"bad graph (code {rc})")
    return _take(po, n + 1, np.int64), _take(pa, na.value, np.int32)


def peel(n: int, off, adj):
    """Core numbers and peel rounds; returns (core, round, degeneracy)."""
    core = np.zeros(n, np.int32)
    rnd = np.zeros(n, np.int32)
    d = lib().orc_peel(n, off, adj, core, rnd)
    return core, rnd, int(d)


ORDER_PEEL = 0   # key (peel round, id): a degeneracy order
ORDER_CORE = 1   # key (core number, id)


def order(n: int, core, rnd, kind: int = ORDER_PEEL):
    rank = np.zeros(n, np.int32)
    vert = np.zeros(n, np.int32)
    lib().orc_order(n, core, rnd, kind, rank, vert)
    return rank, vert


# --------------------------------------------------------------------------
# O1: explicit k-cliques
# --------------------------------------------------------------------------

def list_cliques(n: int, off, adj, k: int, limit: int = -1):
    """All k-cliques as a (c, k) int32 array, ids ascending in each row."""
    p = C.POINTER(C.c_int32)()
    c = lib().orc_list_cliques(n, off, adj, k, limit, C.byref(p))
    if c < 0:
        if p:
            lib().orc_free(C.cast(p, C.c_void_p))
        raise OverflowError("clique limit exceeded")
    return _take(p, c * k, np.int32).reshape(c, k)


def count_cliques(n: int, off, adj, k: int, limit: int = -1) -> int:
    c = lib().orc_list_cliques(n, off, adj, k, limit, None)
    if c < 0:
        raise OverflowError("clique limit exceeded")
    return int(c)


# --------------------------------------------------------------------------
# O2: SCT restricted to P_k
# --------------------------------------------------------------------------

def sct(n: int, off, adj, rank, vert, k: int):
    """Pairs of P_k in root order then depth-first order.
    Returns dict(pair_off int64[np+1], nodes int32, h int32[np])."""
    po, pn, ph, nn = (C.POINTER(C.c_int64)(), C.POINTER(C.c_int32)(),
                      C.POINTER(C.c_int32)(), C.c_int64(0))
    npairs = lib().orc_sct(n, off, adj, rank, vert, k, 0, C.byref(po), C.byref(pn),
                           C.byref(ph), C.byref(nn))
    pair_off = _take(po, npairs + 1, np.int64) if npairs > 0 else np.zeros(1, np.int64)
    if npairs == 0 and po:
        pass
    return dict(pair_off=pair_off, nodes=_take(pn, nn.value, np.int32),
                h=_take(ph, npairs, np.int32))


def canonical_pairs(s):
    """Canonical form of an SCT: every pair as (sorted V_h, sorted V_p),
    pairs sorted lexicographically."""
    out = []
    po, nodes, h = s["pair_off"], s["nodes"], s["h"]
    for q in range(len(h)):
        seg = nodes[po[q]:po[q + 1]]
        out.append((tuple(sorted(seg[:h[q]].tolist())), tuple(sorted(seg[h[q]:].tolist()))))
    out.sort()
    return out


# --------------------------------------------------------------------------
# PBUpdate (Alg. 3) and its two independent restatements
# --------------------------------------------------------------------------

def _pb(fn, ids, r, h, k):
    ids = np.ascontiguousarray(ids, np.int32)
    r = np.ascontiguousarray(r, np.uint64)
    out = np.zeros(ids.size, np.uint64)
    rc = fn(ids.size, ids, r, h, k, out)
    if rc != 0:
        raise OverflowError(f"pbupdate failed ({rc})")
    return out


def pbupdate_alg3(ids, r, h, k):
    return _pb(lib().orc_pbupdate_alg3, ids, r, h, k)


def pbupdate_greedy(ids, r, h, k):
    return _pb(lib().orc_pbupdate_greedy, ids, r, h, k)


def pbupdate_level(ids, r, h, k):
    return _pb(lib().orc_pbupdate_level, ids, r, h, k)


def pbupdate_cont(ids, r, h, k):
    ids = np.ascontiguousarray(ids, np.int32)
    r = np.ascontiguousarray(r, np.float64)
    out = np.zeros(ids.size, np.float64)
    rc = lib().orc_pbupdate_cont(ids.size, ids, r, h, k, out)
    if rc != 0:
        raise OverflowError(f"pbupdate_cont failed ({rc})")
    return out


# --------------------------------------------------------------------------
# O3 / O4: Frank-Wolfe iterations
# --------------------------------------------------------------------------

def fw_sync(n, s, k, T, r0=None):
    """Alg. 2, synchronous reading: r_T (uint64, cumulative, r_0 = 0)."""
    r = np.zeros(n, np.uint64) if r0 is None else np.array(r0, np.uint64)
    rc = lib().orc_fw_sync(n, len(s["h"]), s["pair_off"], s["nodes"], s["h"], k, T, r)
    if rc != 0:
        raise OverflowError(f"fw_sync failed ({rc})")
    return r


def fw_sync_par(n, s, k, T, threads=None, r0=None):
    """fw_sync with the pairs of each iteration split over host threads
    (same r_T; a timing baseline)."""
    threads = threads or os.cpu_count() or 1
    r = np.zeros(n, np.uint64) if r0 is None else np.array(r0, np.uint64)
    rc = lib().orc_fw_sync_par(n, len(s["h"]), s["pair_off"], s["nodes"], s["h"], k, T, r,
                               int(threads))
    if rc != 0:
        raise OverflowError(f"fw_sync_par failed ({rc})")
    return r


def fw_seq(n, s, k, T, r0=None):
    """Alg. 2 as printed: pairs update r in place, in array order."""
    r = np.zeros(n, np.uint64) if r0 is None else np.array(r0, np.uint64)
    rc = lib().orc_fw_seq(n, len(s["h"]), s["pair_off"], s["nodes"], s["h"], k, T, r)
    if rc != 0:
        raise OverflowError(f"fw_seq failed ({rc})")
    return r


def fw_cont(n, s, k, T, r0=None):
    """Synchronous iterations of the continuous rule, FP64, cumulative r."""
    r = np.zeros(n, np.float64) if r0 is None else np.array(r0, np.float64)
    rc = lib().orc_fw_cont(n, len(s["h"]), s["pair_off"], s["nodes"], s["h"], k, T, r)
    if rc != 0:
        raise OverflowError(f"fw_cont failed ({rc})")
    return r


def fw_cont_par(n, s, k, T, threads=None, r0=None):
    """fw_cont with the pairs' water levels computed on host threads; the
    additions happen in pair order, so r equals fw_cont's bit for bit."""
    threads = threads or os.cpu_count() or 1
    r = np.zeros(n, np.float64) if r0 is None else np.array(r0, np.float64)
    rc = lib().orc_fw_cont_par(n, len(s["h"]), s["pair_off"], s["nodes"], s["h"], k, T, r,
                               int(threads))
    if rc != 0:
        raise OverflowError(f"fw_cont_par failed ({rc})")
    return r


def fw_cliques(n, cliques, k, T, r0=None):
    """Alg. 1 over the explicit list (each clique +1 to its argmin (r, id))."""
    cl = np.ascontiguousarray(cliques, np.int32).reshape(-1)
    r = np.zeros(n, np.uint64) if r0 is None else np.array(r0, np.uint64)
    lib().orc_fw_cliques(cl.size // k if k else 0, cl, k, T, r)
    return r


def fw_cliques_sync(n, cliques, k, T, r0=None):
    """Alg. 1 over the explicit list, synchronous reading (every clique of an
    iteration reads r_{t-1}; units summed after the iteration)."""
    cl = np.ascontiguousarray(cliques, np.int32).reshape(-1)
    r = np.zeros(n, np.uint64) if r0 is None else np.array(r0, np.uint64)
    lib().orc_fw_cliques_sync(n, cl.size // k if k else 0, cl, k, T, r)
    return r


# --------------------------------------------------------------------------
# O5: extraction
# --------------------------------------------------------------------------

def sort_desc(r):
    """Node order by (r desc, id asc) (the final sort of Alg. 2, reading R4)."""
    n = len(r)
    out = np.zeros(n, np.int32)
    if np.asarray(r).dtype == np.float64:
        lib().orc_sort_desc_f64(n, np.ascontiguousarray(r, np.float64), out)
    else:
        lib().orc_sort_desc_u64(n, np.ascontiguousarray(r, np.uint64), out)
    return out


def _to_int(lo, hi):
    return [int(a) | (int(b) << 64) for a, b in zip(lo, hi)]


def prefix_counts_cliques(n, order_, cliques, k):
    """C_k(V_i), i = 0..n, from the explicit list (Python ints)."""
    cl = np.ascontiguousarray(cliques, np.int32).reshape(-1)
    lo = np.zeros(n + 1, np.uint64)
    hi = np.zeros(n + 1, np.uint64)
    lib().orc_prefix_counts_cliques(n, np.ascontiguousarray(order_, np.int32),
                                    cl.size // k, cl, k, lo, hi)
    return lo, hi


def prefix_counts_pairs(n, order_, s, k):
    """(C_k(V_i) lo, hi, F_i lo, hi) from the SCT pairs, i = 0..n."""
    lo, hi, flo, fhi = (np.zeros(n + 1, np.uint64) for _ in range(4))
    lib().orc_prefix_counts_pairs(n, np.ascontiguousarray(order_, np.int32), len(s["h"]),
                                  s["pair_off"], s["nodes"], s["h"], k, lo, hi, flo, fhi)
    return lo, hi, flo, fhi


def argmax_density(lo, hi):
    """Largest i maximising counts[i] / i (exact)."""
    n = len(lo) - 1
    return int(lib().orc_argmax_density(n, np.ascontiguousarray(lo, np.uint64),
                                        np.ascontiguousarray(hi, np.uint64)))


def brute_best(n, masks, weights):
    """Max over subsets S of (sum of weights of items inside S) / |S|.
    Returns (best_mask, num, den, union_of_all_maximisers)."""
    masks = np.ascontiguousarray(masks, np.uint32)
    weights = np.ascontiguousarray(weights, np.uint64)
    bm, bn, bd, un = C.c_uint32(), C.c_uint64(), C.c_uint64(), C.c_uint32()
    rc = lib().orc_brute_best(n, masks.size, masks, weights, C.byref(bm), C.byref(bn),
                              C.byref(bd), C.byref(un))
    if rc != 0:
        raise ValueError("brute force needs n <= 24")
    return int(bm.value), int(bn.value), int(bd.value), int(un.value)


# --------------------------------------------------------------------------
# The whole path (A1-A6) in one call
# --------------------------------------------------------------------------

def solve(n, src, dst, k, T, order_kind=ORDER_PEEL, mode="sync", with_cliques=False,
          threads=1):
    """Run the oracle's path: graph, order, SCT, T iterations, extraction.

    mode: 'sync' (rule I, synchronous), 'seq' (rule I, in place), 'cont'
    (continuous rule, FP64).  threads > 1 runs the synchronous iterations on
    that many host threads (same result).  Returns a dict with the SCT, r_T,
    the order, the extracted prefix (i*, ids, exact count) and the bounds."""
    off, adj = csr(n, src, dst)
    core, rnd, degen = peel(n, off, adj)
    rank, vert = order(n, core, rnd, order_kind)
    s = sct(n, off, adj, rank, vert, k)
    if mode == "sync":
        r = fw_sync(n, s, k, T) if threads <= 1 else fw_sync_par(n, s, k, T, threads)
    elif mode == "seq":
        r = fw_seq(n, s, k, T)
    elif mode == "cont":
        r = fw_cont(n, s, k, T)
    else:
        raise ValueError(mode)
    ordr = sort_desc(r)
    lo, hi, flo, fhi = prefix_counts_pairs(n, ordr, s, k)
    istar = argmax_density(lo, hi) if n > 0 else 0
    count = int(lo[istar]) | (int(hi[istar]) << 64) if n > 0 else 0
    ck = int(lo[n]) | (int(hi[n]) << 64) if n > 0 else 0
    F = _to_int(flo, fhi)
    rho_prime_max = max((F[i] / i for i in range(1, n + 1)), default=0.0)
    rmax = float(np.max(r)) / T if n > 0 and T > 0 else 0.0
    out = dict(off=off, adj=adj, core=core, round=rnd, degeneracy=degen, rank=rank,
               vert=vert, sct=s, r=r, order=ordr, istar=istar,
               ids=np.sort(ordr[:istar]), count=count, c_k=ck,
               density=count / istar if istar else 0.0,
               upper_bound=rmax, rho_prime_max=rho_prime_max)
    if with_cliques:
        out["cliques"] = list_cliques(n, off, adj, k)
    return out


# --------------------------------------------------------------------------
# CPSample (Sec. 5, Alg. 4); readings S1-S4 in kdss_oracle.c
# --------------------------------------------------------------------------

def color_greedy(n, off, adj, rank):
    """S1: greedy colouring by decreasing rank; returns (colour, #colours)."""
    color = np.zeros(max(n, 1), np.int32)
    nc = lib().orc_color_greedy(n, off, adj, np.ascontiguousarray(rank, np.int32), color)
    return color[:n], int(nc)


def ccpath_dp(n, off, adj, color, k):
    """S2: dp[v, i-1] = increasing-colour paths of i vertices from v."""
    dp = np.zeros(max(n, 1) * k, np.uint64)
    if lib().orc_ccpath_dp(n, off, adj, np.ascontiguousarray(color, np.int32), k, dp) != 0:
        raise OverflowError("more than 2^64 color paths")
    return dp[:n * k].reshape(n, k)


def ccpath_sample(n, off, adj, color, k, dp, t, seed):
    """S3: t uniform k-color paths; returns (paths (t, k), is_clique, #paths)."""
    paths = np.zeros(max(t, 1) * k, np.int32)
    flags = np.zeros(max(t, 1), np.uint8)
    tot = C.c_uint64(0)
    rc = lib().orc_ccpath_sample(n, off, adj, np.ascontiguousarray(color, np.int32), k,
                                 np.ascontiguousarray(dp, np.uint64).reshape(-1), int(t),
                                 int(seed) & 0xFFFFFFFFFFFFFFFF, paths, flags, C.byref(tot))
    if rc != 0:
        raise OverflowError("more than 2^64 color paths")
    return paths[:t * k].reshape(t, k), flags[:t].astype(bool), int(tot.value)


def cpsample(n, src, dst, k, t, T, seed, order_kind=ORDER_PEEL):
    """Alg. 4: t sampled k-color paths, the set of cliques among them (S4),
    T synchronous iterations of Alg. 1 over that set (reading R1), and the
    prefix of largest |C_k(V_i) & sample| / i (ties to the larger i)."""
    off, adj = csr(n, src, dst)
    core, rnd, _ = peel(n, off, adj)
    rank, _ = order(n, core, rnd, order_kind)
    color, ncol = color_greedy(n, off, adj, rank)
    dp = ccpath_dp(n, off, adj, color, k)
    paths, flags, total = ccpath_sample(n, off, adj, color, k, dp, t, seed)
    cl = np.sort(paths[flags], axis=1)
    cl = np.unique(cl, axis=0) if len(cl) else cl.reshape(0, k)
    r = fw_cliques_sync(n, cl, k, T)
    ordr = sort_desc(r)
    lo, hi = prefix_counts_cliques(n, ordr, cl, k)
    i = argmax_density(lo, hi) if n > 0 else 0
    return dict(color=color, ncolors=ncol, paths_total=total, samples_clique=int(flags.sum()),
                cliques=cl, r=r, istar=i, ids=np.sort(ordr[:i]), count=int(lo[i]) if n else 0,
                density=(int(lo[i]) / i) if i else 0.0,
                upper_bound=float(r.max()) / T if n and T else 0.0)
