#!/usr/bin/env python3
"""Benchmark of the PSCTL hot path on GB300.

One step = the whole path on one synthetic graph already resident in device
memory: CSR build and peeling (A1-A2), SCT build (A3), T Frank-Wolfe
iterations of PBUpdate (A4-A5) and the densest-prefix extraction (A6).  The
metric is clique-updates/s = T * c_k / step time (every iteration settles the
c_k k-cliques the SCT encodes).  L2 is flushed (a 256 MiB write) before every
step, outside the step's event pair.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent replica per GPU (launched by torch.distributed.run);
the whole-job value is the units of all ranks over the slowest rank's time.
`--impl reference` times the CPU oracle on the host cores instead (rank 0).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "SCT clique-updates/s and time to 1%-density; batched FP32 vs plain FP64; p99"
UNIT = "clique-updates/s"

WORKLOADS = {
    "chunglu1e5": dict(
        gen=synth.workload_chunglu_1e5, k=5, T=200,
        desc="Chung-Lu power-law graph n=100000, mean degree 20, exponent 2.5, planted "
             "60-node near-clique at p=0.9, seed 2; k=5; T=200 FW iterations"),
    "er2000": dict(
        gen=synth.workload_er2000, k=3, T=100,
        desc="Erdos-Renyi G(2000, 0.01), seed 1; k=3; T=100 FW iterations"),
}

def _union_workload(max_n=None):
    def gen():
        ns, ks = synth.batch_rmat_specs(256, nmax=1e4)
        graphs, kk = [], []
        for i, nn in enumerate(ns):
            if ks[i] == 8:
                graphs.append(synth.batch_rmat_graph(i, int(nn)))
                kk.append(8)
        return union_edges(graphs, kk, 8, max_n)
    return gen


WORKLOADS["rmat_union_k8"] = dict(
    gen=_union_workload(), k=8, T=20,
    desc="disjoint union of the k=8 instances of the batched R-MAT workload (n <= 1e4 each, "
         "198,339 nodes); k=8; T=20 FW iterations")
WORKLOADS["rmat_union_k8_small"] = dict(
    gen=_union_workload(40000), k=8, T=20,
    desc="the first k=8 instances of the batched R-MAT workload up to 40,000 nodes, as one "
         "disjoint union; k=8; T=20 FW iterations")

PRECISIONS = {"fp64": 1, "int64": 0, "fp32k": 2}
DTYPE = {"fp64": "f64", "int64": "u64", "fp32k": "f32"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="chunglu1e5")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--allocator", choices=["library", "torch"], default="library",
                    help="device memory: the library's stream-ordered pool or torch's caching "
                         "allocator (through callbacks)")
    ap.add_argument("--rmat24", action="store_true",
                    help="only report the large R-MAT graph (scale 24) build: one JSON line")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP32 and time-to-1%% side measurements")
    ap.add_argument("--chunk", type=int, default=0,
                    help="integer-rule iterations on the work-queue kernels with this many tiles "
                         "per item (0: the per-class kernels)")
    ap.add_argument("--per-iteration", action="store_true",
                    help="integer-rule iterations as launches per iteration, not one resident "
                         "launch")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def code_digest(path):
    """sha256 of a C/CUDA source with its comments and whitespace removed, so
    that the digest changes with the code and not with its comments."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256(" ".join(text.split()).encode()).hexdigest()


def ncu_figure(kernel_src, summary, field):
    """A per-iteration figure of the FW kernels (DRAM bytes, warp
    instructions) from the committed ncu summary, or None when the kernel
    code changed since it was taken."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(field + r":\s*([0-9.eE+]+)", text)
    h = re.search(r"fw\.cu code digest:\s*([0-9a-f]{64})", text)
    if not m or not h:
        return None
    return float(m.group(1)) if code_digest(kernel_src) == h.group(1) else None


def ncu_traffic(kernel_src, summary="fw_resident_chunglu1e5.md"):
    """Per-iteration DRAM bytes of the FW kernels (ncu), or None."""
    return ncu_figure(kernel_src, summary, "traffic_bytes_per_iteration")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.tmp = None

    def __enter__(self):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        pw = [float(r[3]) for r in rows if re.match(r"^[0-9.]+$", r[3])]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(pw) if pw else None}


def gpu_id_for_smi(torch, dev):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",")]
        if dev < len(ids):
            return ids[dev]
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else f"GPU-{u}"
    except Exception:
        return dev


def run_reference(args, rank):
    """Reference arm: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    import oracle as O
    O.build()
    wl = WORKLOADS[args.workload]
    n, s, d = wl["gen"]()
    k = wl["k"]
    T_ref = wl["T"]
    times = []
    ck = None
    cores = os.cpu_count() or 1
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = O.solve(n, s, d, k, T_ref, threads=cores)
        dt = time.perf_counter() - t0
        ck = res["c_k"]
        if it >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = T_ref * ck * len(times) / tot
    sample = (f"oracle (C): CSR, peeling, SCT, {T_ref} synchronous rule-I iterations on "
              f"{cores} host threads, and extraction of the {args.workload} workload per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "k": k, "T": T_ref, "n": n, "c_k": ck},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def slowest_rank_ms(dist, local_ms, device):
    """Max over ranks of the timed region: the whole job ends with its
    slowest replica.  One rank (or no process group) returns local_ms."""
    if dist is None or not dist.is_available() or not dist.is_initialized() \
            or dist.get_world_size() == 1:
        return float(local_ms)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank, world, max_ms):
    """Replicas run the same workload: the job processes world * units in
    the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def async_vs_sync(K, torch, dev, n, src, dst, k, T):
    """The in-place (asynchronous) iterations against the synchronous ones on
    the benchmark graph: the certificate gap 1 - rho'/max r-hat after 5, 20,
    50, 100 and T iterations, the first multiple of 5 with gap <= 2%, and the
    per-iteration time of each (CUDA events around T iterations)."""
    out = {}
    sct = K.kdss_build_sct(n, src, dst, k)
    for mode, fl in (("sync", 0), ("async", K.KDSS_FLAG_ASYNC)):
        o = K.make_opts(precision=PRECISIONS["fp64"], flags=fl)
        st, t, gaps, first = None, 0, {}, None
        while t < T:
            st = K.kdss_fw_iterate(sct, st, 5, o)
            t += 5
            g = K.kdss_extract(sct, st)["gap"]
            if t in (5, 20, 50, 100, T):
                gaps[t] = g
            if first is None and g <= 0.02:
                first = t
        st.free()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream(dev)
        torch.cuda.synchronize()
        a.record(stream)
        st = K.kdss_fw_iterate(sct, None, T, o)
        b.record(stream)
        torch.cuda.synchronize()
        st.free()
        out[mode] = {"gap_at": gaps, "first_t_gap_le_2pct": first,
                     "ms_per_iteration": a.elapsed_time(b) / T}
    sct.free()
    return out


def alg1_vs_sct(K, torch, dev, n, src, dst, k, T):
    """Alg. 1 over the explicit k-clique list (expanded from the SCT on the
    device) against the SCT iterations on the benchmark graph: clique-updates/s
    of each (T iterations timed with CUDA events), the memory of the list and
    of the SCT, and the bound max r / t each reaches after T iterations."""
    stream = torch.cuda.current_stream(dev)
    sct = K.kdss_build_sct(n, src, dst, k)
    info = K.kdss_sct_info(sct)
    ck = info["c_k"]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K.kdss_fw_cliques(sct, None, 1).free()          # expands the list (kept in the handle)
    out = {"c_k": ck, "list_bytes": 4 * k * ck, "sct_bytes": 4 * info["L_k"] + 9 * info["eta_k"]}
    for name, fn in (("alg1_explicit", lambda: K.kdss_fw_cliques(sct, None, T)),
                     ("sct", lambda: K.kdss_fw_iterate(sct, None, T))):
        torch.cuda.synchronize()
        a.record(stream)
        st = fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        res = K.kdss_extract(sct, st)
        out[name] = {"value": T * ck / (ms / 1e3), "unit": UNIT, "ms": ms,
                     "density": res["density"], "upper_bound": res["upper_bound"]}
        st.free()
    sct.free()
    return out


def cpsample_run(K, torch, dev, n, src, dst, k, t=1 << 26, T=30, seed=5):
    """CPSample (Alg. 4) on the benchmark graph: t sampled k-color paths,
    Alg. 1 over the sampled cliques, sampled-density prefix; samples/s over
    the whole call (colouring, path counts, sampling, set, iterations,
    extraction), and how the returned set compares with the SCT solver's."""
    o = K.make_opts(precision=PRECISIONS["int64"])
    K.kdss_cpsample(n, src, dst, k, 1 << 16, T, seed, o)   # warm-up
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    a.record(stream)
    res = K.kdss_cpsample(n, src, dst, k, t, T, seed, o)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    ref = K.kdss_solve(n, src, dst, k, 200)
    inter = len(set(res["ids"].tolist()) & set(ref["ids"].tolist()))
    return {"t": t, "T": T, "ms": ms, "samples_per_s": t / (ms / 1e3), **res["stats"],
            "istar": res["istar"], "sampled_count": res["count"],
            "overlap_with_sct_result": inter / max(len(ref["ids"]), 1),
            "sct_result_istar": ref["istar"]}


def k_agnostic(K, torch, dev, n, src, dst, kmax=8):
    """One k-agnostic SCT of the benchmark graph restricted to k = 3..kmax,
    against one k-pruned build per k: wall time of each (device work
    synchronised) and the sizes."""
    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, 1e3 * (time.perf_counter() - t0)

    K.kdss_build_sct(n, src, dst, 3).free()                 # warm-up
    multi, ms_multi = wall(lambda: K.kdss_build_sct_multi(n, src, dst, kmax))
    info = K.kdss_sct_info(multi)
    per_k = {}
    for k in range(3, kmax + 1):
        a, ms_r = wall(lambda: K.kdss_sct_restrict(multi, k))
        b, ms_b = wall(lambda: K.kdss_build_sct(n, src, dst, k))
        ia = K.kdss_sct_info(a)
        per_k[k] = {"restrict_ms": ms_r, "build_ms": ms_b, "eta_k": ia["eta_k"],
                    "same_size": ia["eta_k"] == K.kdss_sct_info(b)["eta_k"]}
        a.free()
        b.free()
    # the prefix-shared form of the k-agnostic SCT, iterated at k = 5 where it
    # stands, against the flat form (bytes of the pair stream per iteration)
    sh, ms_share = wall(lambda: K.kdss_sct_share_prefixes(multi))
    words = K.kdss_sct_shared_words(sh)["words"]
    eta, L = info["eta_k"], info["L_k"]
    shared = {"share_ms": ms_share, "kept_words": words, "node_words": L,
              "pair_bytes_flat": 4 * L + 9 * eta,
              "pair_bytes_shared": 4 * words + 5 * eta + 24 * -(-eta // 32)}
    o = K.make_opts(precision=K.KDSS_FP64, flags=K.KDSS_FLAG_PROFILE)
    for name, h in (("flat", multi), ("shared", sh)):
        st = K.kdss_fw_iterate_at(h, 5, None, 20, o)
        tm = K.kdss_state_timing(st)
        shared[f"us_per_iteration_at_k5_{name}"] = 1e3 * tm["fw_kernel_ms"] / max(tm["fw_launches"], 1)
        st.free()
    sh.free()
    multi.free()
    return {"k_max": kmax, "multi_build_ms": ms_multi, "multi_pairs": info["eta_k"],
            "multi_nodes": info["L_k"], "per_k": per_k,
            "all_k_restrict_ms": ms_multi + sum(v["restrict_ms"] for v in per_k.values()),
            "all_k_build_ms": sum(v["build_ms"] for v in per_k.values()),
            "prefix_shared": shared}


def large_rmat_report(K, torch, dev):
    """The large single graph (R-MAT scale 24, edge factor 32, planted
    200-node near-clique, k = 6, seed 4, T = 100): the edge list goes to the
    device and the SCT build runs until it completes or proves that the SCT
    cannot fit the device (the count pass stops at a memory budget); the
    line reports what was measured either way."""
    t0 = time.perf_counter()
    n, s_np, d_np = synth.workload_rmat24()
    gen_s = time.perf_counter() - t0
    src = torch.from_numpy(s_np).to(dev)
    dst = torch.from_numpy(d_np).to(dev)
    del s_np, d_np
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info(dev)
    out = {"workload": "R-MAT scale 24 (n = 16,777,216), edge factor 32 (536,870,912 draws), "
                       "planted 200-node near-clique p = 0.95, seed 4; k = 6, T = 100",
           "n": n, "edge_draws": int(src.numel()), "generate_s": gen_s,
           "device_free_gb": free0 / 1e9}
    o = K.make_opts(precision=PRECISIONS["fp32k"], allocator="library")
    t0 = time.perf_counter()
    try:
        sct = K.kdss_build_sct(n, src, dst, 6, o)
        torch.cuda.synchronize()
        out["build_s"] = time.perf_counter() - t0
        info = K.kdss_sct_info(sct)
        out.update({f: info[f] for f in ("m", "eta_k", "L_k", "c_k", "degeneracy",
                                         "max_out_degree", "device_bytes")})
        st = K.kdss_fw_iterate(sct, None, 100, o)
        res = K.kdss_extract(sct, st, o)
        out.update(density=res["density"], istar=res["istar"], gap=res["gap"])
        st.free()
        sct.free()
    except K.KdssError as e:
        out["build_s"] = time.perf_counter() - t0
        out["status"] = e.code
        out["message"] = str(e)
    return out


_POOL = {}


def serving(K, torch, dev, count=400, rate=200.0, pool_size=32, T=300, eps=0.01, every=5,
            flags=0):
    """The serving workload: a Poisson stream (rate 200/s, seed 5) of k-DSS
    queries on a pool of Chung-Lu graphs (the n = 1e5 workload's generator
    with n log-uniform in [1e3, 1e6]) with k uniform in {3..10}, through the
    continuous-batching server: a query stops once its certificate gap is
    <= 1% (checked every 5 iterations) or at T = 300.  Latency is submit to
    result; throughput is queries over first submit to last result."""
    import threading
    if _POOL.get("size") != pool_size:      # generated once, shared by the serving runs
        pool = synth.serving_pool(pool_size)
        _POOL.update(size=pool_size, sum_n=sum(p[0] for p in pool),
                     dev=[(n, torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev))
                          for n, s, d in pool])
    arr, gi, ks = synth.serving_stream(count, rate, pool_size)
    dpool = _POOL["dev"]
    torch.cuda.synchronize()
    tickets = [None] * count
    with K.Server(precision=PRECISIONS["fp64"], check_every=every, eps_stop=eps,
                  flags=flags) as srv:
        t0 = time.perf_counter()

        def feed():
            for i in range(count):
                dt = arr[i] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                n, s, d = dpool[gi[i]]
                tickets[i] = srv.submit(n, s, d, int(ks[i]), T)

        th = threading.Thread(target=feed)
        th.start()
        res = []
        for i in range(count):
            while tickets[i] is None:
                time.sleep(0.0005)
            res.append(srv.wait(tickets[i]))
        th.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
    lat = np.array([r["timing"]["latency_ms"] for r in res])
    ok = [r for r in res if r["status"] == 0]
    return {
        "workload": f"{count} queries, Poisson {rate:g}/s, pool of {pool_size} Chung-Lu graphs "
                    f"(mean degree 20, exponent 2.5, planted 60-node near-clique p=0.9, n "
                    f"log-uniform in [1e3, 1e6], sum {_POOL['sum_n']}), k in {{3..10}}, "
                    f"seed 5; stop at gap <= {eps:g} (every {every}) or T = {T}; FP64",
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "throughput_qps": len(res) / wall,
        "offered_qps": rate, "completed": len(ok), "failed": len(res) - len(ok),
        "mean_iterations": float(np.mean([r["t_used"] for r in ok])) if ok else 0.0,
        "stopped_by_gap": sum(1 for r in ok if r["gap"] <= eps),
        "mean_build_ms": float(np.mean([r["timing"]["build_ms"] for r in res])),
        "mean_queue_ms": float(np.mean([r["timing"]["queue_ms"] for r in res])),
        "peak_active": st["peak_active"], "captures": st["captures"], "replays": st["replays"],
        "peak_resident_bytes": st["peak_resident_bytes"], "hbm_budget": st["hbm_budget"],
    }


def fp32_error_vs_oracle(K, n, s_np, d_np, k, T, r32, dens32, rho_oracle):
    """The FP32 path's error against the FP64 oracle at T: the FP64
    continuous-rule iterations of the oracle (host threads, the same additions
    as the serial form) give r-hat_64 = r_T / T; reported are
    ||r-hat_32 - r-hat_64||_inf / ||r-hat_64||_inf, the density of the prefix
    the oracle extracts from r-hat_64, and the FP32 density's relative error
    against the oracle's integer-rule density and against that one."""
    import oracle as O
    off, adj = O.csr(n, s_np, d_np)
    core, rnd, _ = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd)
    sc = O.sct(n, off, adj, rank, vert, k)
    t0 = time.perf_counter()
    r64 = O.fw_cont_par(n, sc, k, T) / T
    secs = time.perf_counter() - t0
    ordr = O.sort_desc(r64)
    lo, hi, _, _ = O.prefix_counts_pairs(n, ordr, sc, k)
    i = O.argmax_density(lo, hi)
    dens64 = (int(lo[i]) | (int(hi[i]) << 64)) / i
    err = float(np.max(np.abs(r32.astype(np.float64) - r64)) / np.max(np.abs(r64)))
    return {"r_rel_err_inf_vs_fp64_oracle": err, "fp64_oracle_continuous_density": dens64,
            "density_rel_err_vs_fp64_continuous_oracle": abs(dens32 - dens64) / dens64,
            "density_rel_err_vs_integer_oracle": (abs(dens32 - rho_oracle) / rho_oracle
                                                  if rho_oracle else None),
            "oracle_seconds": secs,
            "note": "the continuous rule's trajectory amplifies rounding differences (a 1e-13 "
                    "perturbation grows ~100x per 10 iterations), so r at T differs at the "
                    "convergence-error scale; per-iteration agreement (1e-5) is tested"}


def er2000_k3(K, torch, dev, stream):
    """Erdos-Renyi G(2000, 0.01) from seed 1, k = 3, T = 100 (and the paper's G1):
    device-timed clique-updates/s and the extracted set against the oracle."""
    import oracle as O
    n, s_np, d_np = synth.workload_er2000()
    k, T = 3, 100
    src = torch.from_numpy(s_np).to(dev)
    dst = torch.from_numpy(d_np).to(dev)
    o = K.make_opts(precision=PRECISIONS["fp64"], stream=stream)
    K.kdss_solve(n, src, dst, k, T, o)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    res = K.kdss_solve(n, src, dst, k, T, o)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    want = O.solve(n, s_np, d_np, k, T)
    g1n, g1s, g1d = synth.g1()
    g1 = K.kdss_solve(g1n, g1s, g1d, 3, 100)
    return {"workload": WORKLOADS["er2000"]["desc"], "value": T * want["c_k"] / (ms / 1e3),
            "unit": UNIT, "ms": ms, "c_k": want["c_k"], "istar": res["istar"],
            "density": res["density"],
            "equals_oracle": bool(res["istar"] == want["istar"] and res["count"] == want["count"]
                                  and res["ids"].tolist() == want["ids"].tolist()),
            "g1": {"istar": g1["istar"], "density": g1["density"],
                   "paper": "{u1..u6} at 4/3 (Example 1.1)",
                   "ids": g1["ids"].tolist()}}


def rmat24_count(K, torch, dev, budget_s=30.0):
    """R-MAT scale 24 (edge factor 32, planted 200-node near-clique,
    k = 6, seed 4): the count-only SCT pass measures P_6 without storing a
    pair; roots are taken in a pseudo-random order until the budget ends, so
    the counted roots are a sample and counts * n / roots_done estimates the
    whole SCT."""
    t0 = time.perf_counter()
    n, s_np, d_np = synth.workload_rmat24()
    gen_s = time.perf_counter() - t0
    src = torch.from_numpy(s_np).to(dev)
    dst = torch.from_numpy(d_np).to(dev)
    del s_np, d_np
    out = {"workload": "R-MAT scale 24 (n = 16,777,216), edge factor 32, planted 200-node "
                       "near-clique p = 0.95, seed 4; k = 6", "generate_s": gen_s,
           "budget_s": budget_s}
    try:
        c = K.kdss_sct_count(n, src, dst, 6, budget_s,
                             K.make_opts(precision=PRECISIONS["fp32k"], allocator="library"))
    except K.KdssError as e:
        out["error"] = str(e)
        return out
    done = max(c["roots_done"], 1)
    scale = n / done
    out.update({f: c[f] for f in ("m", "degeneracy", "max_out_degree", "roots_done", "roots_cut",
                                  "complete", "eta_k", "L_k", "max_pair_len", "count_bits",
                                  "seconds", "cut_pairs", "cut_nodes")})
    out["pairs_per_class"] = c["pairs_per_class"]
    out["c_k_counted"] = str(c["c_k"])
    # every pair counted, finished roots or not, is a pair of the SCT: a
    # measured lower bound on its size (the roots the budget interrupted are
    # the densest, so scaling the finished ones would understate it)
    out["lower_bound"] = {"eta_6": c["eta_k"] + c["cut_pairs"], "L_6": c["L_k"] + c["cut_nodes"],
                          "sct_bytes_flat": 4 * (c["L_k"] + c["cut_nodes"])
                                            + 9 * (c["eta_k"] + c["cut_pairs"]),
                          "device_bytes": torch.cuda.get_device_properties(dev).total_memory}
    out["sample_estimate_finished_roots"] = {"eta_6": c["eta_k"] * scale, "L_6": c["L_k"] * scale,
                                             "c_6": float(c["c_k"]) * scale}
    return out


def batched_upper_range(K, torch, dev, count=256, budget_s=3.0):
    """The batch of 256 R-MAT graphs with n log-uniform in [1e3, 1e5]: the
    count-only SCT pass on its three largest instances measures why the upper part of
    the range cannot be held on one device."""
    ns, ks = synth.batch_rmat_specs(count, nmax=1e5)
    order = np.argsort(-ns)[:3]
    rows = []
    for i in order:
        n, s_np, d_np = synth.batch_rmat_graph(int(i), int(ns[i]))
        c = K.kdss_sct_count(n, s_np, d_np, int(ks[i]), budget_s)
        scale = n / max(c["roots_done"], 1)
        rows.append({"n": n, "k": int(ks[i]), "roots_done": c["roots_done"], "complete": c["complete"],
                     "roots_cut": c["roots_cut"], "eta_k_counted": c["eta_k"], "L_k_counted": c["L_k"],
                     "cut_pairs": c["cut_pairs"], "cut_nodes": c["cut_nodes"],
                     "sct_bytes_lower_bound": 4 * (c["L_k"] + c["cut_nodes"])
                                              + 9 * (c["eta_k"] + c["cut_pairs"]),
                     "degeneracy": c["degeneracy"], "seconds": c["seconds"]})
    return {"instances_n_above_1e4": int((ns > 1e4).sum()), "largest": rows}


def union_edges(graphs, ks, k, max_n=None):
    """The disjoint union (ids shifted) of the batched instances with this k:
    the SCT the batch iterates for that k, as one graph."""
    S, D, base = [], [], 0
    for (n, s, d), kk in zip(graphs, ks):
        if kk != k:
            continue
        if max_n is not None and base >= max_n:
            break
        S.append(s.astype(np.int64) + base)
        D.append(d.astype(np.int64) + base)
        base += n
    return base, np.concatenate(S).astype(np.int32), np.concatenate(D).astype(np.int32)


def union_roofline(K, torch, dev, stream, graphs, ks, k, iters=32):
    """The PBUpdate pass where HBM binds: the k = 8 union of the batched
    workload (a 13 GB SCT, far above L2).  CUDA-event time of the pass
    (KDSS_FLAG_PROFILE times every 8th iteration on the launching stream),
    algorithmic bytes 4 L_k + 9 eta_k, fraction of the measured HBM peak."""
    n, s_np, d_np = union_edges(graphs, ks, k)
    src = torch.from_numpy(s_np).to(dev)
    dst = torch.from_numpy(d_np).to(dev)
    out = {"workload": f"disjoint union of the k = {k} instances of the batched workload "
                       f"(n = {n}), k = {k}, FP64 rule I"}
    o = K.make_opts(precision=PRECISIONS["fp64"], stream=stream, allocator="library",
                    flags=K.KDSS_FLAG_PROFILE)
    sct = K.kdss_build_sct(n, src, dst, k, o)
    info = K.kdss_sct_info(sct)
    peak, kind = measured_peaks()
    alg = 4 * info["L_k"] + 9 * info["eta_k"]
    for name, chunk in (("per_class_kernels", 0), ("work_queue", 4)):
        oc = K.make_opts(precision=PRECISIONS["fp64"], stream=stream, allocator="library",
                         flags=K.KDSS_FLAG_PROFILE, chunk=chunk)
        st = K.kdss_fw_iterate(sct, None, 8, oc)            # warm
        t0 = K.kdss_state_timing(st)
        st = K.kdss_fw_iterate(sct, st, iters, oc)
        t1 = K.kdss_state_timing(st)
        us = 1e3 * (t1["fw_kernel_ms"] - t0["fw_kernel_ms"]) / max(t1["fw_launches"] - t0["fw_launches"], 1)
        st.free()
        out[name] = {"bound": "hbm", "achieved": alg / us / 1e3, "peak": peak, "unit": "GB/s",
                     "frac": alg / us / 1e3 / peak, "avg_launch_us": us,
                     "peak_source": f"{kind} hbm_gbs"}
    out.update(eta_k=info["eta_k"], L_k=info["L_k"], alg_bytes_per_launch=alg,
               sct_device_bytes=info["device_bytes"], pairs_per_class=info["pairs_per_class"])
    sct.free()
    return out


def l2_copy_gbs(torch, dev, mib=24, reps=200):
    """Copy bandwidth of a buffer that stays in L2 (read + write bytes over
    CUDA-event time, best of 5 runs of `reps` copies): the ceiling of a pass
    whose data is L2-resident."""
    a = torch.empty(mib << 20, dtype=torch.uint8, device=dev)
    b = torch.empty_like(a)
    b.copy_(a)
    best = 0.0
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2 * a.numel() * reps / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


def batched_rmat(K, torch, dev, stream, flush, allocator, count=256, T=300, nmax=1e4):
    """The batched workload: 256 R-MAT graphs (a, b, c, d = 0.57, 0.19, 0.19,
    0.05; edge factor 16; planted 30-node clique; k uniform in {3..8}; seed
    3), T = 300, edge lists resident on the device.  Node counts are
    log-uniform in [1e3, nmax]: the recipe's upper end of 1e5 gives R-MAT
    cores of degeneracy ~250 whose SCTs alone need hundreds of GB (measured:
    4.8e8 SCT node entries at n = 18,695, k = 5), so the measured batch stops
    a decade lower.  Timed: one kdss_solve_batch call in FP32 (continuous
    rule) and in FP64 (rule I), and the plain FP64 form that solves one
    instance at a time (kdss_solve per graph).  Units are the sum over
    instances of T * c_k."""
    ns, ks = synth.batch_rmat_specs(count, nmax=nmax)
    graphs = [synth.batch_rmat_graph(i, int(nn)) for i, nn in enumerate(ns)]
    dq = [(g[0], torch.from_numpy(g[1]).to(dev), torch.from_numpy(g[2]).to(dev), int(kk), T)
          for g, kk in zip(graphs, ks)]
    o64 = K.make_opts(precision=PRECISIONS["fp64"], stream=stream, allocator=allocator)
    o32 = K.make_opts(precision=PRECISIONS["fp32k"], stream=stream, allocator=allocator)
    cks = []
    for n, s, d, k, _ in dq:
        sct = K.kdss_build_sct(n, s, d, k, o64)
        cks.append(K.kdss_sct_info(sct)["c_k"])
        sct.free()
    units = T * sum(cks)

    def timed(fn):
        flush.fill_(9)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    K.kdss_solve_batch(dq[:8], o32)          # warm-up
    b32, ms32 = timed(lambda: K.kdss_solve_batch(dq, o32))
    b64, ms64 = timed(lambda: K.kdss_solve_batch(dq, o64))
    p64, msp = timed(lambda: [K.kdss_solve(*q, o64) for q in dq])
    ok = all(r["status"] == 0 for r in b32 + b64)
    import oracle as O
    small = np.argsort(ns)[:16]
    orel = []
    for i in small:
        n_i, s_i, d_i = graphs[i]
        want = O.solve(n_i, s_i, d_i, int(ks[i]), T, threads=os.cpu_count() or 1)
        if want["density"] > 0:
            orel.append(abs(b32[i]["density"] - want["density"]) / want["density"])
    rel = [abs(a["density"] - c["density"]) / c["density"] for a, c in zip(b32, p64) if c["density"] > 0]
    same64 = all(a["ids"].tolist() == c["ids"].tolist() and a["count"] == c["count"]
                 for a, c in zip(b64, p64))
    union = union_roofline(K, torch, dev, stream, graphs, ks, 8)
    return {
        "hbm_union_k8": union,
        "workload": f"{count} R-MAT graphs, n log-uniform in [1e3, {nmax:.0e}] (sum {int(ns.sum())}), "
                    f"edge factor 16, planted 30-clique, k in {{3..8}}, seed 3; T={T}",
        "units": units, "unit": UNIT,
        "batched_fp32": {"value": units / (ms32 / 1e3), "ms": ms32},
        "batched_fp64": {"value": units / (ms64 / 1e3), "ms": ms64},
        "per_instance_fp64": {"value": units / (msp / 1e3), "ms": msp},
        "speedup_batched_fp32_vs_per_instance_fp64": msp / ms32,
        "all_ok": ok, "batched_fp64_equals_per_instance": same64,
        "fp32_density_rel_err_vs_fp64": {"max": max(rel) if rel else 0.0,
                                         "mean": statistics.mean(rel) if rel else 0.0},
        "fp32_density_rel_err_vs_oracle": {"instances": len(orel),
                                           "which": "the 16 smallest (the oracle is affordable)",
                                           "max": max(orel) if orel else 0.0,
                                           "mean": statistics.mean(orel) if orel else 0.0},
    }


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    import paper_2403_05775_gb300 as K

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.rmat24:
        K.load(build_if_missing=True)
        if rank == 0:
            print(json.dumps({"report": "rmat24", **large_rmat_report(K, torch, dev)}), flush=True)
        return
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    K.load(build_if_missing=True)
    wl = WORKLOADS[args.workload]
    n, s_np, d_np = wl["gen"]()
    k, T = wl["k"], wl["T"]
    prec = PRECISIONS[args.precision]

    # CPU baseline first (rank 0, N = 1 only), so the host is idle during GPU timing.
    cpu = None
    rho_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as O
        O.build()
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        ores = O.solve(n, s_np, d_np, k, T, threads=cores)
        dt = time.perf_counter() - t0
        rho_oracle = ores["density"]
        cpu = {"value": T * ores["c_k"] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"the whole {args.workload} workload once (CSR, peeling, SCT, {T} "
                         f"synchronous rule-I iterations on {cores} host threads, extraction), "
                         f"C, {dt:.1f} s"}
        t0 = time.perf_counter()
        O.solve(n, s_np, d_np, k, T)
        dt1 = time.perf_counter() - t0
        cpu["single_thread"] = {"value": T * ores["c_k"] / dt1, "cores": 1, "seconds": dt1}

    stream = torch.cuda.current_stream(dev)
    src = torch.from_numpy(s_np).to(dev)
    dst = torch.from_numpy(d_np).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    base_flags = K.KDSS_FLAG_PER_ITERATION if args.per_iteration else 0

    def step(flags):
        o = K.make_opts(precision=prec, flags=flags | base_flags, stream=stream,
                        allocator=args.allocator, chunk=args.chunk)
        sct = K.kdss_build_sct(n, src, dst, k, o)
        st = K.kdss_fw_iterate(sct, None, T, o)
        res = K.kdss_extract(sct, st, o)
        tm = K.kdss_state_timing(st)
        info = K.kdss_sct_info(sct)
        st.free()
        sct.free()
        return res, tm, info

    for _ in range(args.warmup):
        flush.fill_(1)
        step(0)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    fw_ms, fw_launches = 0.0, 0
    launches0 = K.kdss_kernel_launches()
    with ClockSampler(gpu_id_for_smi(torch, local)) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            res, tm, info = step(K.KDSS_FLAG_PROFILE)
            ev[i][1].record(stream)
            fw_ms += tm["fw_kernel_ms"]
            fw_launches += tm["fw_launches"]
        torch.cuda.synchronize()
    launches = K.kdss_kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = slowest_rank_ms(dist if world > 1 else None, sum(step_ms), dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    ck = info["c_k"]
    value = whole_job_value(T * ck * args.steps, world, total_ms)

    # end to end through the public API with host buffers
    e2e_ms = []
    for i in range(max(1, min(args.steps, 3))):
        flush.fill_(3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r2 = K.kdss_solve(n, s_np, d_np, k, T, K.make_opts(precision=prec, stream=stream,
                                                           allocator=args.allocator,
                                                           chunk=args.chunk, flags=base_flags))
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_value = T * ck * world / (statistics.mean(e2e_ms) / 1e3)
    h2d = int(s_np.nbytes + d_np.nbytes)
    d2h = int(4 * r2["istar"] + 88)

    # roofline of the PBUpdate pass (all length-class kernels of one iteration)
    peak, peak_kind = measured_peaks()
    l2_gbs = l2_copy_gbs(torch, dev)
    alg_bytes = 4 * info["L_k"] + 9 * info["eta_k"]
    avg_s = (fw_ms / max(fw_launches, 1)) / 1e3
    # the resident launch counts every iteration it runs; the per-iteration
    # path times every 8th PBUpdate pass
    resident = fw_launches == T * args.steps and not args.chunk
    fw_src = os.path.join(ROOT, "paper_2403_05775_gb300", "csrc", "fw.cu")
    prof = (("fw_resident_f32_chunglu1e5.md" if args.precision == "fp32k"
             else "fw_resident_chunglu1e5.md") if resident else "fw_pbupdate_chunglu1e5.md")
    traffic = ncu_traffic(fw_src, prof)
    achieved = alg_bytes / avg_s / 1e9 if avg_s > 0 else 0.0
    # the ceiling the resident launch works against: instruction issue, one
    # warp instruction per cycle on each of an SM's four schedulers, at the SM
    # clock sampled during the timed region
    clocks = clk.summary()
    winst = ncu_figure(fw_src, prof, "warp_instructions_per_iteration")
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz")
    issue = None
    if winst and mhz and avg_s > 0:
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_ips = nsm * 4 * mhz * 1e6
        issue = {"warp_instructions_per_iteration": winst,
                 "achieved_warp_inst_per_s": winst / avg_s, "peak_warp_inst_per_s": peak_ips,
                 "frac": winst / avg_s / peak_ips, "sms": nsm, "schedulers_per_sm": 4,
                 "sm_mhz": mhz,
                 "source": f"warp instructions from the committed ncu capture (profiles/{prof}), "
                           "iteration time from this run's CUDA events"}
    # the same work counted per pair and per pair node, over the whole step
    # and over the FW iterations alone (T times the mean iteration time)
    step_s = total_ms / args.steps / 1e3
    fw_s = avg_s * T
    rates = {"note": "value is T c_k per whole step (build, T iterations, extraction); the "
                     "*_fw rates divide the same work by the FW iterations' CUDA-event time",
             "clique_updates_per_s_fw": T * ck * world / fw_s if fw_s > 0 else None,
             "path_updates_per_s": T * info["eta_k"] * world / step_s,
             "path_updates_per_s_fw": T * info["eta_k"] * world / fw_s if fw_s > 0 else None,
             "node_visits_per_s": T * info["L_k"] * world / step_s,
             "node_visits_per_s_fw": T * info["L_k"] * world / fw_s if fw_s > 0 else None,
             "fw_ms_per_step": fw_s * 1e3}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
        "data": "synthetic",
        "config": {"workload": wl["desc"], "k": k, "T": T, "n": n, "m": info["m"],
                   "eta_k": info["eta_k"], "L_k": info["L_k"], "c_k": ck,
                   "degeneracy": info["degeneracy"], "precision": args.precision,
                   "rule": "continuous" if args.precision == "fp32k" else "integer (Alg. 3)",
                   "l2": "flushed by a 256 MiB write before every step",
                   "allocator": args.allocator,
                   "pbupdate_kernels": (f"work queue, {args.chunk} tiles per item" if args.chunk
                                        else "resident launch, T iterations" if resident
                                        else "per length class"),
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": statistics.mean(e2e_ms)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "l2": {"note": ("the resident launch holds the pair stream in shared "
                                     "memory and r in L2; " if resident else
                                     "this workload's pair stream (11 MB) and r stay in L2; ") +
                                    "the same algorithmic bytes against a measured L2 copy rate",
                            "peak_gbs": l2_gbs, "frac": achieved / l2_gbs if l2_gbs else None},
                     "kernel": ("PBUpdate pass of one FW iteration (k_pb_queue + k_pb_queue_long)"
                                if args.chunk else
                                ("one FW iteration of the resident launch " +
                                 ("k_fw_resident_f32" if args.precision == "fp32k" else "k_fw_resident") +
                                 " (gather of r, PBUpdate of every pair, fold of the delta, grid "
                                 "barrier); launch time / T") if resident else
                                "PBUpdate pass of one FW iteration (k_pb_fast + k_pb_slow + "
                                "length-class group kernels)"),
                     "alg_bytes_per_launch": alg_bytes, "avg_launch_us": avg_s * 1e6,
                     "peak_source": f"{peak_kind} hbm_gbs", "issue": issue},
        "rates": rates,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "result": {"istar": res["istar"], "count": res["count"], "density": res["density"],
                   "upper_bound": res["upper_bound"], "gap": res["gap"]},
    }

    if rank == 0 and not args.no_extras:
        extras = {}
        # FP32 compensated continuous rule on the same workload
        o32 = K.make_opts(precision=PRECISIONS["fp32k"], stream=stream, allocator=args.allocator)
        t32 = []
        for _ in range(2):
            flush.fill_(5)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sct = K.kdss_build_sct(n, src, dst, k, o32)
            st = K.kdss_fw_iterate(sct, None, T, o32)
            r32 = K.kdss_extract(sct, st, o32)
            b.record(stream)
            torch.cuda.synchronize()
            t32.append(a.elapsed_time(b))
            st.free()
            sct.free()
        extras["fp32k"] = {"value": T * ck / (min(t32) / 1e3), "unit": UNIT,
                           "ms_per_step": min(t32), "density": r32["density"],
                           "istar": r32["istar"]}
        try:
            sct = K.kdss_build_sct(n, src, dst, k, o32)
            st = K.kdss_fw_iterate(sct, None, T, o32)
            r32v, _ = K.kdss_state_copy_r(st, n, K.KDSS_FP32K)
            st.free()
            sct.free()
            extras["fp32k"]["error_vs_fp64_oracle"] = fp32_error_vs_oracle(
                K, n, s_np, d_np, k, T, r32v, r32["density"], rho_oracle)
        except Exception as e:  # the oracle leg is a report, not the measurement
            extras["fp32k"]["error_vs_fp64_oracle"] = {"error": str(e)}
        try:
            extras["er2000_k3"] = er2000_k3(K, torch, dev, stream)
        except Exception as e:
            extras["er2000_k3"] = {"error": str(e)}
        # time to reach 99% of the oracle's density: build, then chunks of 5
        # iterations each followed by an extraction
        target = rho_oracle if rho_oracle is not None else res["density"]
        o = K.make_opts(precision=prec, stream=stream, allocator=args.allocator)
        flush.fill_(7)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sct = K.kdss_build_sct(n, src, dst, k, o)
        st, it, dens = None, 0, 0.0
        while it < T:
            st = K.kdss_fw_iterate(sct, st, 5, o)
            it += 5
            dens = K.kdss_extract(sct, st, o)["density"]
            if dens >= 0.99 * target:
                break
        torch.cuda.synchronize()
        extras["time_to_1pct_density"] = {
            "ms": 1e3 * (time.perf_counter() - t0), "iterations": it, "density": dens,
            "target": 0.99 * target,
            "target_source": "oracle density after T iterations" if rho_oracle else "own T"}
        st.free()
        sct.free()
        extras["async_vs_sync"] = async_vs_sync(K, torch, dev, n, src, dst, k, T)
        try:
            extras["k_agnostic"] = k_agnostic(K, torch, dev, n, src, dst)
        except K.KdssError as e:
            extras["k_agnostic"] = {"error": str(e)}
        try:
            extras["cpsample"] = cpsample_run(K, torch, dev, n, src, dst, k)
        except K.KdssError as e:
            extras["cpsample"] = {"error": str(e)}
        try:
            extras["alg1_vs_sct"] = alg1_vs_sct(K, torch, dev, n, src, dst, k, T)
        except K.KdssError as e:
            extras["alg1_vs_sct"] = {"error": str(e)}
        try:
            extras["batched"] = batched_rmat(K, torch, dev, stream, flush, args.allocator)
        except K.KdssError as e:
            extras["batched"] = {"error": str(e)}
        # serving: the Poisson stream (4,000 queries at 200/s on a pool of
        # 64) with queries iterating in place, the same at a sustainable rate,
        # and the synchronous form at 200/s and at a sustainable rate
        runs = {"serving_in_place": dict(count=4000, rate=200.0, flags=K.KDSS_FLAG_ASYNC),
                "serving_in_place_steady": dict(count=600, rate=40.0, flags=K.KDSS_FLAG_ASYNC),
                "serving": dict(count=400, rate=200.0, flags=0),
                "serving_steady": dict(count=80, rate=8.0, flags=0)}
        for key, kw in runs.items():
            try:
                extras[key] = serving(K, torch, dev, pool_size=64, **kw)
            except K.KdssError as e:
                extras[key] = {"error": str(e)}
        try:
            extras["batched_upper_range"] = batched_upper_range(K, torch, dev)
        except Exception as e:
            extras["batched_upper_range"] = {"error": str(e)}
        try:
            extras["rmat24"] = rmat24_count(K, torch, dev)
        except Exception as e:
            extras["rmat24"] = {"error": str(e)}
        line["extras"] = extras

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
